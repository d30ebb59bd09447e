// mixed.cu -- mixed-precision evaluation: the embedding-net and fitting-net
// GEMMs run on the 5th-generation tensor cores (tcgen05.mma, BF16 operands in
// shared memory, FP32 accumulators in tensor memory); tanh runs in FP32; the
// environment matrix, the descriptor contraction T = R~^T G / N_m and
// D = T_<^T T, the contractions of the backward pass with gT, the pair
// gradients, forces, virial and energy sum stay in FP64.
//
// Kernel shapes.  One CTA = 4 warps = the 128 lanes of a tcgen05 accumulator,
// one thread per row.  Embedding kernels: rows are the real neighbours of one
// atom for one neighbour type (up to 128 per tile); layer 0 (1 -> e1) runs on
// the CUDA cores, layers 1 and 2 are MMAs of 128 x N x K with the net's
// transposed weights as the B operand.  Fitting kernel: rows are 128 atoms of
// one type; layer 1 streams the descriptor (converted to BF16) and the weight
// K-chunks through double-buffered shared memory.
//
// Split operands (DP_PREC_MIXED_SPLIT, template flag SPLIT of the embedding
// kernels): every FP32 row operand and weight is stored as a BF16 high part
// and the BF16 value of its remainder, and each K-slice issues hi*hi + hi*lo +
// lo*hi into the same FP32 accumulator (~16 bits per operand instead of 8).
// The operand buffers double; layer 1's operands and weights share one region
// with the layer-2 row operands (EmbPlan) and batches hold fewer atoms, so two
// CTAs still fit per SM.  That mode runs its fitting net on fit_oz.cu's exact
// digit kernels, not on k_fit_mx.
//
// G store (plain BF16 operands): k_embed_tan_mx evaluates the net with its
// s-tangent once and keeps G and dG/ds (FP32) of every real row in HBM, with T
// and D as k_embed_fwd_mx forms them; k_embed_bwd_stmx streams them through the
// double-float contractions with dE/dT.  Without the store k_embed_bwd_mx
// recomputes them.
//
// Supported shapes: embedding widths (e1, 2 e1, 4 e1) with e1 in {16, 25, 32}
// (the paper's doubling nets), fitting layers of equal width <= 256 after the
// first one.  Every wait on the tensor core is bounded; on a timeout the
// kernel flags DPF_MMA_TIMEOUT, stops issuing work, waits once more, frees its
// tensor memory and returns.
#include <cuda_bf16.h>

#include "dp_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int MXT = 128;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&p);
}

// 8 consecutive K-values of one row into the canonical K-major layout
__device__ __forceinline__ void st8(unsigned char *base, int row, int k0, int K, const float (&v)[8])
{
    uint4 u;
    u.x = pack_bf16x2(v[0], v[1]);
    u.y = pack_bf16x2(v[2], v[3]);
    u.z = pack_bf16x2(v[4], v[5]);
    u.w = pack_bf16x2(v[6], v[7]);
    *reinterpret_cast<uint4 *>(base + tc::kmajor_offset(row, k0, K)) = u;
}

// 8 consecutive K-values of one row as BF16 high parts (hi) and the BF16 values
// of the remainders v - hi (lo): hi + lo carries ~16 significant bits
__device__ __forceinline__ void st8_split(unsigned char *hi, unsigned char *lo, int row, int k0, int K,
                                          const float (&v)[8])
{
    float r[8];
    uint4 u;
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(v[q], v[q + 1]);
        r[q] = v[q] - __low2float(p);
        r[q + 1] = v[q + 1] - __high2float(p);
        (&u.x)[q / 2] = *reinterpret_cast<const uint32_t *>(&p);
    }
    const uint32_t ofs = tc::kmajor_offset(row, k0, K);
    *reinterpret_cast<uint4 *>(hi + ofs) = u;
    u.x = pack_bf16x2(r[0], r[1]);
    u.y = pack_bf16x2(r[2], r[3]);
    u.z = pack_bf16x2(r[4], r[5]);
    u.w = pack_bf16x2(r[6], r[7]);
    *reinterpret_cast<uint4 *>(lo + ofs) = u;
}

// A row operand: plain BF16, or high and low parts
template <bool SPLIT>
__device__ __forceinline__ void st8_op(unsigned char *base, int bytes, int row, int k0, int K, const float (&v)[8])
{
    if constexpr (SPLIT) st8_split(base, base + bytes, row, k0, K, v);
    else st8(base, row, k0, K, v);
}

// D (+)= A B^T for one K-slice: one MMA, or three on the split operands
// (hi hi + hi lo + lo hi; the lo lo term is below FP32 rounding)
template <bool SPLIT>
__device__ __forceinline__ void mma_op(uint32_t d, uint32_t a, uint32_t abytes, uint32_t b, uint32_t bbytes, int K,
                                       uint32_t idesc, bool acc)
{
    const uint32_t sbo = (uint32_t)K * 16;
    tc::mma_bf16(d, tc::make_desc(a, 128, sbo), tc::make_desc(b, 128, sbo), idesc, acc);
    if constexpr (SPLIT) {
        tc::mma_bf16(d, tc::make_desc(a, 128, sbo), tc::make_desc(b + bbytes, 128, sbo), idesc, true);
        tc::mma_bf16(d, tc::make_desc(a + abytes, 128, sbo), tc::make_desc(b, 128, sbo), idesc, true);
    }
}

// Double-float arithmetic for the FP64 contractions (T = R~^T G and the
// backward products with gT): a sum S = sh + sl of two FP32 numbers gathers
// a (bh + bl), a an FP32 value (G, dG/ds) and bh + bl an FP64 value split into
// two FP32 parts.  a bh is formed exactly as p + e (e by FMA), p joins sh by
// an error-free two-sum, and the sum's rounding error, e and a bl go to sl;
// the result is within about 2^-46 of the sum of the products, relative to
// the sum of their magnitudes.  Every step is an _rn intrinsic, so no
// multiply-add contraction can change the error-free transformations.
__device__ __forceinline__ void df_fma(float &sh, float &sl, float a, float bh, float bl)
{
    const float p = __fmul_rn(a, bh);
    const float e = __fmaf_rn(a, bh, -p);
    const float s = __fadd_rn(sh, p);
    const float z = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(p, z));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, __fmaf_rn(a, bl, e)));
}

// v = h + l to about 2^-48 relative (h = v rounded to FP32, l = the rest rounded)
__device__ __forceinline__ void df_split(double v, float &h, float &l)
{
    h = __double2float_rn(v);
    l = __double2float_rn(v - (double)h);
}

__device__ __forceinline__ double df_value(float h, float l) { return (double)h + (double)l; }

__device__ __forceinline__ void copy16(unsigned char *dst, const unsigned char *__restrict__ src, int bytes)
{
    for (int q = threadIdx.x * 16; q < bytes; q += blockDim.x * 16)
        *reinterpret_cast<uint4 *>(dst + q) = *reinterpret_cast<const uint4 *>(src + q);
}

// CTA-wide barrier that also orders tensor-core operations and makes the
// threads' shared-memory writes visible to the tensor core.
__device__ __forceinline__ void tc_sync()
{
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Bounded wait on the MMA barrier; returns false for the whole CTA if any
// thread gave up.
__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t &phase, int32_t *status)
{
    const bool ok = tc::mbar_wait(mbar, phase);
    phase ^= 1u;
    const bool bad = __syncthreads_or(!ok);
    if (bad && threadIdx.x == 0) atomicOr(status, DPF_MMA_TIMEOUT);
    tc::fence_after_sync();
    return !bad;
}

constexpr int pad16(int v) { return (v + 15) / 16 * 16; }
constexpr int tcols_for(int n) { return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : (n <= 256 ? 256 : 512))); }

struct RowGeo {
    double s, ds, R[4], d[3], r;
};

__device__ __forceinline__ void geometry(const DevModel &m, const double *__restrict__ x, const double xi[3], int j,
                                         const Box3 &box, RowGeo &g)
{
    const double xj[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
    g.r = dp_pinned_dist(xi, xj, box, g.d);
    dp_switch(g.r, m.rcut_smth, m.rcut, g.s, g.ds);
    const double inv = 1.0 / g.r;
    g.R[0] = g.s;
    g.R[1] = g.s * g.d[0] * inv;
    g.R[2] = g.s * g.d[1] * inv;
    g.R[3] = g.s * g.d[2] * inv;
}

// ------------------------------------------------------------ embedding --
//
// Packing: a CTA owns a balanced contiguous share of the type-sorted atoms
// and walks it in batches of up to AB atoms of one centre type.  For each
// neighbour type b the batch's real rows are cut into 32-row groups, each
// group belonging to one atom; a tile of the MMA is 4 groups (one per warp),
// so tiles are full even when an atom has only ~30 neighbours of a type.
// Per-warp partial sums are merged into per-atom accumulators in warp order
// after each tile, which keeps every result reproducible bit for bit.

constexpr int AB_MAX = 8;                        // atoms per batch (at most)
constexpr int MAXG = AB_MAX * (DP_MAX_NM / 32);  // 32-row groups per batch and type (upper bound)

template <int E1>
struct EmbShape {
    static constexpr int E2 = 2 * E1, E3 = 4 * E1;
    static constexpr int K1p = pad16(E1), N1p = pad16(E2), K2p = N1p, N2p = pad16(E3);
    static constexpr int A0B = MXT * K1p * 2, A1B = MXT * K2p * 2;      // bytes
    static constexpr int B1B = N1p * K1p * 2, B2B = N2p * K2p * 2;
};

constexpr size_t zmax(size_t a, size_t b) { return a > b ? a : b; }

// Shared-memory plan of the embedding kernels (byte offsets from the dynamic
// buffer).  Plain BF16: every operand has its own buffer and batches hold 8
// atoms.  Split operands (two copies of everything): layer 1's operands and
// weights (A0, dA0, B1) and the layer-2 row operands (A1, dA1) share one region
// R -- layer 1's MMAs are complete before the layer-2 operands are written, and
// B1 is copied again for every tile -- and batches hold 4 atoms (2 for e1 = 32),
// so that two CTAs fit per SM.
template <int E1, bool SPLIT>
struct EmbPlan {
    using S = EmbShape<E1>;
    static constexpr int X = SPLIT ? 2 : 1;
    static constexpr int AB = SPLIT ? (E1 >= 32 ? 2 : 4) : AB_MAX;
    static constexpr size_t a0 = (size_t)X * S::A0B, a1 = (size_t)X * S::A1B;
    static constexpr size_t b1 = (size_t)X * S::B1B, b2 = (size_t)X * S::B2B;
    // forward.  Plain: A0, A1, B1, B2.  Split: region R = [A0, B1 | A1], then B2.
    static constexpr size_t FA0 = 0, FA1 = SPLIT ? 0 : a0, FB1 = SPLIT ? a0 : a0 + a1;
    static constexpr size_t FB2 = SPLIT ? zmax(a0 + b1, a1) : a0 + a1 + b1;
    static constexpr size_t FEND = FB2 + b2;
    // backward.  Plain: A0, dA0, A1, dA1, B1, B2.  Split: R = [A0, dA0, B1 | A1, dA1], then B2.
    static constexpr size_t BA0 = 0, BdA0 = a0;
    static constexpr size_t BA1 = SPLIT ? 0 : 2 * a0, BdA1 = BA1 + a1;
    static constexpr size_t BB1 = SPLIT ? 2 * a0 : 2 * a0 + 2 * a1;
    static constexpr size_t BB2 = SPLIT ? zmax(2 * a0 + b1, 2 * a1) : 2 * a0 + 2 * a1 + b1;
    static constexpr size_t BEND = BB2 + b2;
    // bytes from the start that are free between tiles (dE/dD of one atom is staged
    // there): the region R when split, the row operands otherwise (B1 stays resident)
    static constexpr size_t BFREE = SPLIT ? BB2 : 2 * a0 + 2 * a1;
};

struct BatchInfo {
    int ids[AB_MAX];         // atom indices of the batch
    int grp_atom[MAXG];      // batch index of each 32-row group
    int grp_r0[MAXG];        // first row of each group
    int ngroups;
};

// Next batch [first, first + k) of one type inside [first, hi), k <= ab.
__device__ __forceinline__ int batch_size(int first, int hi, const int *tstart, int T, int ab, int &a)
{
    a = 0;
    while (a + 1 < T && first >= tstart[a + 1]) ++a;
    return min(ab, min(hi, tstart[a + 1]) - first);
}

// Group list of neighbour type b for the batch (one thread builds it).
__device__ __forceinline__ void build_groups(BatchInfo &bi, int k, const int32_t *__restrict__ nreal, int T, int b)
{
    int g = 0;
    for (int j = 0; j < k; ++j) {
        const int nb = nreal[(size_t)bi.ids[j] * T + b];
        for (int r0 = 0; r0 < nb; r0 += 32) {
            bi.grp_atom[g] = j;
            bi.grp_r0[g] = r0;
            ++g;
        }
    }
    bi.ngroups = g;
}

template <int E1, bool SPLIT>
__global__ void __launch_bounds__(MXT, 1) k_embed_fwd_mx(
    DevModel m, MixedModel mx, const double *__restrict__ x, const int32_t *__restrict__ types, Box3 box, int N,
    const int32_t *__restrict__ type_perm, const int32_t *__restrict__ type_start, const int32_t *__restrict__ nlist,
    const int32_t *__restrict__ nreal, double *__restrict__ Tout, double *__restrict__ Dout, int32_t *status)
{
    using S = EmbShape<E1>;
    using P = EmbPlan<E1, SPLIT>;
    constexpr int E2 = S::E2, E3 = S::E3, K1p = S::K1p, N1p = S::N1p, K2p = S::K2p, N2p = S::N2p;
    constexpr int TCOLS = tcols_for(N2p);
    constexpr int X = P::X;  // operand copies: high (and low) parts
    constexpr int AB = P::AB;
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *A0 = smraw + P::FA0;
    unsigned char *A1 = smraw + P::FA1;
    unsigned char *B1 = smraw + P::FB1;
    unsigned char *B2 = smraw + P::FB2;
    double *Tw = reinterpret_cast<double *>(smraw + P::FEND);  // [4][4][E3] per-warp partial of one tile
    double *Tacc = Tw + 4 * 4 * E3;                         // [AB][4][E3] per-atom sums
    float *Gt = reinterpret_cast<float *>(Tacc + AB * 4 * E3);  // [4][32][17]
    float *Rth = Gt + 4 * 32 * 17;                          // [4][32][4]: R~ = Rth + Rtl
    float *Rtl = Rth + 4 * 32 * 4;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ BatchInfo bi;
    __shared__ int tstart[DP_MAX_TYPES + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = m.ntypes, nm = m.nm;
    if (tid <= T) tstart[tid] = type_start[tid];
    if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc_sync();
    const uint32_t tbase = tslot;
    const uint32_t tlane = tbase + ((uint32_t)(32 * warp) << 16);
    const uint32_t idesc1 = tc::make_idesc_bf16(MXT, N1p), idesc2 = tc::make_idesc_bf16(MXT, N2p);
    uint32_t phase = 0;
    bool alive = true;
    int staged = -1;
    float *Gw = Gt + warp * 32 * 17;
    float *Rwh = Rth + warp * 32 * 4, *Rwl = Rtl + warp * 32 * 4;
    double *Tww = Tw + warp * 4 * E3;
    const int lo = (int)(((long long)blockIdx.x * N) / gridDim.x);
    const int hi = (int)(((long long)(blockIdx.x + 1) * N) / gridDim.x);

    for (int first = lo; first < hi && alive;) {
        int a;
        const int k = batch_size(first, hi, tstart, T, AB, a);
        __syncthreads();
        if (tid < AB) bi.ids[tid] = tid < k ? type_perm[first + tid] : 0;
        for (int q = tid; q < AB * 4 * E3; q += MXT) Tacc[q] = 0.0;
        __syncthreads();
        const bool a_ok = (unsigned)a < (unsigned)T;
        for (int b = 0; b < T && alive && a_ok; ++b) {
            if (tid == 0) build_groups(bi, k, nreal, T, b);
            __syncthreads();
            const int G = bi.ngroups;
            if (G == 0) continue;
            const int net = a * T + b;
            if (net != staged) {
                if constexpr (!SPLIT) copy16(B1, mx.emb_ops + mx.emb_off[net][0], X * S::B1B);
                copy16(B2, mx.emb_ops + mx.emb_off[net][1], X * S::B2B);
                staged = net;
            }
            const float *P32 = mx.p32 + m.emb_base[net];
            const float *W0 = P32, *b0 = P32 + E1, *b1 = P32 + 2 * E1 + E1 * E2, *b2 = b1 + E2 + E2 * E3;
            for (int t0 = 0; t0 < G && alive; t0 += 4) {
                // split operands: B1 shares its region with the layer-2 operands of the last tile
                if constexpr (SPLIT) copy16(B1, mx.emb_ops + mx.emb_off[net][0], X * S::B1B);
                const int g = t0 + warp;
                const bool warp_live = g < G;
                const int j = warp_live ? bi.grp_atom[g] : 0;
                const int i = bi.ids[j];
                const int r = warp_live ? bi.grp_r0[g] + lane : 0;
                const bool valid = warp_live && r < nreal[(size_t)i * T + b];
                RowGeo gg;
                gg.s = 0.0;
                gg.R[0] = gg.R[1] = gg.R[2] = gg.R[3] = 0.0;
                if (valid) {
                    const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
                    geometry(m, x, xi, nlist[(size_t)i * nm + m.sel_off[b] + r], box, gg);
                }
                float h0[E1];
                const float s32 = (float)gg.s;
#pragma unroll
                for (int o = 0; o < E1; ++o) h0[o] = tanhf(fmaf(s32, W0[o], b0[o]));
#pragma unroll
                for (int k8 = 0; k8 < K1p; k8 += 8) {
                    float v[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = (k8 + q < E1) ? h0[k8 + q] : 0.f;
                    st8_op<SPLIT>(A0, S::A0B, tid, k8, K1p, v);
                }
                tc_sync();
                if (tid == 0) {
#pragma unroll
                    for (int kk = 0; kk < K1p / 16; ++kk)
                        mma_op<SPLIT>(tbase, tc::smem_u32(A0) + kk * 256, S::A0B, tc::smem_u32(B1) + kk * 256, S::B1B,
                                      K1p, idesc1, kk > 0);
                    tc::mma_commit(&mbar);
                }
                alive = tc_wait(&mbar, phase, status);
                float h1[E2];
#pragma unroll
                for (int o = 0; o < E2; ++o) h1[o] = 0.f;
                if (alive && warp_live) {
#pragma unroll
                    for (int cc = 0; cc < N1p; cc += 16) {
                        float v[16];
                        tc::tmem_ld16(tlane + cc, v);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int o = cc + q;
                            if (o < E2) h1[o] = h0[o < E1 ? o : o - E1] + tanhf(v[q] + b1[o]);
                        }
                    }
                }
#pragma unroll
                for (int k8 = 0; k8 < K2p; k8 += 8) {
                    float v[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = (k8 + q < E2) ? h1[k8 + q] : 0.f;
                    st8_op<SPLIT>(A1, S::A1B, tid, k8, K2p, v);
                }
                tc_sync();
                if (!alive) break;
                if (tid == 0) {
#pragma unroll
                    for (int kk = 0; kk < K2p / 16; ++kk)
                        mma_op<SPLIT>(tbase, tc::smem_u32(A1) + kk * 256, S::A1B, tc::smem_u32(B2) + kk * 256, S::B2B,
                                      K2p, idesc2, kk > 0);
                    tc::mma_commit(&mbar);
                }
                alive = tc_wait(&mbar, phase, status);
                // epilogue 2: G = (h1, h1) + tanh(z2 + b2); the warp's partial of T = R~^T G in
                // double-float arithmetic (exact products of G with R~'s FP32 parts)
                if (alive && warp_live) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) df_split(valid ? gg.R[c] : 0.0, Rwh[lane * 4 + c], Rwl[lane * 4 + c]);
#pragma unroll
                    for (int cc = 0; cc < N2p; cc += 16) {
                        float v[16];
                        tc::tmem_ld16(tlane + cc, v);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int o = cc + q;
                            float G2 = 0.f;
                            if (o < E3 && valid) G2 = h1[o < E2 ? o : o - E2] + tanhf(v[q] + b2[o]);
                            Gw[lane * 17 + q] = G2;
                        }
                        __syncwarp();
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int p = lane + 32 * u, c = p >> 4, q = p & 15, o = cc + q;
                            if (o < E3) {
                                float sh = 0.f, sl = 0.f;
#pragma unroll 8
                                for (int rr = 0; rr < 32; ++rr)
                                    df_fma(sh, sl, Gw[rr * 17 + q], Rwh[rr * 4 + c], Rwl[rr * 4 + c]);
                                Tww[c * E3 + o] = df_value(sh, sl);
                            }
                        }
                        __syncwarp();
                    }
                }
                tc_sync();
                // merge the tile's warp partials into the atoms' sums, warps in order
                if (alive) {
                    for (int p = tid; p < 4 * E3; p += MXT) {
#pragma unroll
                        for (int w = 0; w < 4; ++w)
                            if (t0 + w < G) Tacc[bi.grp_atom[t0 + w] * 4 * E3 + p] += Tw[w * 4 * E3 + p];
                    }
                }
                __syncthreads();
            }
        }
        if (!alive) break;
        // T = scale * sum; D = T_<^T T, per atom of the batch
        const int nd = m.m2 * E3;
        for (int j = 0; j < k; ++j) {
            const int i = bi.ids[j];
            double *Tj = Tacc + j * 4 * E3;
            for (int p = tid; p < 4 * E3; p += MXT) {
                const double v = Tj[p] * m.desc_scale;
                Tj[p] = v;
                Tout[(size_t)i * 4 * E3 + p] = v;
            }
            __syncthreads();
            for (int q = tid; q < nd; q += MXT) {
                const int a2 = q / E3, b2i = q - a2 * E3;
                double acc = Tj[a2] * Tj[b2i];
                acc = fma(Tj[E3 + a2], Tj[E3 + b2i], acc);
                acc = fma(Tj[2 * E3 + a2], Tj[2 * E3 + b2i], acc);
                acc = fma(Tj[3 * E3 + a2], Tj[3 * E3 + b2i], acc);
                Dout[(size_t)i * nd + q] = acc;
            }
        }
        first += k;
    }
    if (!alive) tc::mbar_wait(&mbar, phase ^ 1u);  // once more for an MMA still in flight
    tc_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, TCOLS);
}

// Atoms per batch of the tangent forward (its T sums take [AB][4][M] doubles of
// shared memory; two CTAs per SM for every width).
constexpr int tan_ab(int e1) { return e1 >= 32 ? 4 : AB_MAX; }

// TAN = false: the backward (k_embed_bwd_mx).  TAN = true (plain BF16
// operands only): the forward with the s-tangent (k_embed_tan_mx): the same
// value and tangent products, but the last epilogue stores G and dG/ds of each
// row in HBM (Gsto: [N nm][2 M] floats, slot i nm + sel_off[b] + r) and
// accumulates T = R~^T G in double-float arithmetic as k_embed_fwd_mx does;
// the batch's T and D = T_<^T T leave as in k_embed_fwd_mx.
template <int E1, bool SPLIT, bool TAN>
__device__ __forceinline__ void embed_mx_tangent_body(
    const DevModel &m, const MixedModel &mx, const double *__restrict__ x, const int32_t *__restrict__ types,
    Box3 box, int N, const int32_t *__restrict__ type_perm, const int32_t *__restrict__ type_start,
    const int32_t *__restrict__ nlist, const int32_t *__restrict__ nreal, double *__restrict__ Tio,
    const double *__restrict__ gD, double *__restrict__ pair_g, double *__restrict__ f_own,
    double *__restrict__ vir_part, double *__restrict__ Dout, float *__restrict__ Gsto, int32_t *status)
{
    static_assert(!(TAN && SPLIT), "the tangent forward takes plain BF16 operands");
    using S = EmbShape<E1>;
    constexpr int E2 = S::E2, E3 = S::E3, K1p = S::K1p, N1p = S::N1p, K2p = S::K2p, N2p = S::N2p;
    constexpr int TOFF = N2p;                 // tangent accumulator column offset
    constexpr int TCOLS = tcols_for(2 * N2p);
    using P = EmbPlan<E1, SPLIT>;
    constexpr int X = P::X;                   // operand copies: high (and low) parts
    constexpr int AB = TAN ? tan_ab(E1) : P::AB;
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *A0 = smraw + P::BA0;
    unsigned char *dA0 = smraw + P::BdA0;
    unsigned char *A1 = smraw + P::BA1;
    unsigned char *dA1 = smraw + P::BdA1;
    unsigned char *B1 = smraw + P::BB1;
    unsigned char *B2 = smraw + P::BB2;
    double *Ts = reinterpret_cast<double *>(smraw + P::BEND);  // [4][E3]
    double *red = Ts + 4 * E3;                               // [4][12]
    double *facc = red + 4 * 12;                             // [AB][12]
    float *gTh = reinterpret_cast<float *>(facc + AB * 12);  // [AB][4][E3], scaled: gT = gTh + gTl
    float *gTl = gTh + AB * 4 * E3;
    // TAN, in the same place: per-warp T partials of one tile, the batch's T sums, R~ parts
    double *Tw = reinterpret_cast<double *>(smraw + P::BEND);  // [4][4][E3]
    double *Tacc = Tw + 4 * 4 * E3;                           // [AB][4][E3]
    float *Rth = reinterpret_cast<float *>(Tacc + AB * 4 * E3);  // [4][32][4]: R~ = Rth + Rtl
    float *Rtl = Rth + 4 * 32 * 4;
    // and G of 16 features x 32 rows per warp ([4][32][17]) in the layer-2 row operands A1, dA1
    // (contiguous with plain operands), idle once their MMAs are done
    float *Gt = reinterpret_cast<float *>(A1);
    static_assert(!TAN || (P::BdA1 == P::BA1 + S::A1B && 4 * 32 * 17 * sizeof(float) <= 2 * (size_t)S::A1B),
                  "the G staging fits in A1, dA1");
    // dE/dD of one atom [M2][E3] in the operand buffers, when it fits there
    double *gds = reinterpret_cast<double *>(smraw);
    const bool gd_fits = (size_t)m.m2 * E3 * sizeof(double) <= P::BFREE;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ BatchInfo bi;
    __shared__ int tstart[DP_MAX_TYPES + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = m.ntypes, nm = m.nm, m2 = m.m2;
    if (tid <= T) tstart[tid] = type_start[tid];
    if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc_sync();
    const uint32_t tbase = tslot;
    const uint32_t tlane = tbase + ((uint32_t)(32 * warp) << 16);
    const uint32_t idesc1 = tc::make_idesc_bf16(MXT, N1p), idesc2 = tc::make_idesc_bf16(MXT, N2p);
    uint32_t phase = 0;
    bool alive = true;
    int staged = -1;
    const int lo = (int)(((long long)blockIdx.x * N) / gridDim.x);
    const int hi = (int)(((long long)(blockIdx.x + 1) * N) / gridDim.x);

    for (int first = lo; first < hi && alive;) {
        int a;
        const int k = batch_size(first, hi, tstart, T, AB, a);
        __syncthreads();
        if (tid < AB) bi.ids[tid] = tid < k ? type_perm[first + tid] : 0;
        if constexpr (TAN)
            for (int q = tid; q < AB * 4 * E3; q += MXT) Tacc[q] = 0.0;
        else
            for (int q = tid; q < AB * 12; q += MXT) facc[q] = 0.0;
        __syncthreads();
        // gT[c][x] = [x < M2] sum_b gD[x][b] T[c][b] + sum_{a<M2} gD[a][x] T[c][a], times the scale
        // (dE/dD of the atom staged in the operand buffers, idle between tiles, when it fits)
        for (int j = 0; j < (TAN ? 0 : k); ++j) {
            const int i = bi.ids[j];
            for (int p = tid; p < 4 * E3; p += MXT) Ts[p] = Tio[(size_t)i * 4 * E3 + p];
            const double *gd = gD + (size_t)i * m2 * E3;
            if (gd_fits) {
                const double2 *src = reinterpret_cast<const double2 *>(gd);
                double2 *dst = reinterpret_cast<double2 *>(gds);
                for (int p = tid; p < m2 * E3 / 2; p += MXT) dst[p] = src[p];
                gd = gds;
            }
            __syncthreads();
            for (int p = tid; p < 4 * E3; p += MXT) {
                const int cc = p / E3, xx = p - cc * E3;
                double acc = 0.0, acc2 = 0.0;
                if (xx < m2)
                    for (int b2i = 0; b2i < E3; b2i += 2) {  // two chains (E3 = 4 e1 is even)
                        acc = fma(gd[xx * E3 + b2i], Ts[cc * E3 + b2i], acc);
                        acc2 = fma(gd[xx * E3 + b2i + 1], Ts[cc * E3 + b2i + 1], acc2);
                    }
                for (int a2 = 0; a2 < m2; ++a2) acc = fma(gd[a2 * E3 + xx], Ts[cc * E3 + a2], acc);
                df_split((acc + acc2) * m.desc_scale, gTh[j * 4 * E3 + p], gTl[j * 4 * E3 + p]);
            }
            __syncthreads();
        }
        const bool a_ok = (unsigned)a < (unsigned)T;
        for (int b = 0; b < T && alive && a_ok; ++b) {
            if (tid == 0) build_groups(bi, k, nreal, T, b);
            __syncthreads();
            const int G = bi.ngroups;
            if (G == 0) continue;
            const int net = a * T + b;
            if (net != staged) {
                if constexpr (!SPLIT) copy16(B1, mx.emb_ops + mx.emb_off[net][0], X * S::B1B);
                copy16(B2, mx.emb_ops + mx.emb_off[net][1], X * S::B2B);
                staged = net;
            }
            const float *P32 = mx.p32 + m.emb_base[net];
            const float *W0 = P32, *b0 = P32 + E1, *b1 = P32 + 2 * E1 + E1 * E2, *b2 = b1 + E2 + E2 * E3;
            for (int t0 = 0; t0 < G && alive; t0 += 4) {
                // split operands: B1 shares its region with the layer-2 operands of the last tile
                if constexpr (SPLIT) copy16(B1, mx.emb_ops + mx.emb_off[net][0], X * S::B1B);
                const int g = t0 + warp;
                const bool warp_live = g < G;
                const int j = warp_live ? bi.grp_atom[g] : 0;
                const int i = bi.ids[j];
                const int r = warp_live ? bi.grp_r0[g] + lane : 0;
                const bool valid = warp_live && r < nreal[(size_t)i * T + b];
                const int slot = m.sel_off[b] + r;
                RowGeo gg;
                gg.s = gg.ds = 0.0;
                gg.R[0] = gg.R[1] = gg.R[2] = gg.R[3] = 0.0;
                gg.d[0] = gg.d[1] = gg.d[2] = 0.0;
                gg.r = 1.0;
                if (valid) {
                    const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
                    geometry(m, x, xi, nlist[(size_t)i * nm + slot], box, gg);
                }
                float h0[E1], dh0[E1];
                const float s32 = (float)gg.s;
#pragma unroll
                for (int o = 0; o < E1; ++o) {
                    const float t = tanhf(fmaf(s32, W0[o], b0[o]));
                    h0[o] = t;
                    dh0[o] = fmaf(-t, t, 1.f) * W0[o];
                }
#pragma unroll
                for (int k8 = 0; k8 < K1p; k8 += 8) {
                    float v[8], dv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        v[q] = (k8 + q < E1) ? h0[k8 + q] : 0.f;
                        dv[q] = (k8 + q < E1) ? dh0[k8 + q] : 0.f;
                    }
                    st8_op<SPLIT>(A0, S::A0B, tid, k8, K1p, v);
                    st8_op<SPLIT>(dA0, S::A0B, tid, k8, K1p, dv);
                }
                tc_sync();
                if (tid == 0) {
#pragma unroll
                    for (int kk = 0; kk < K1p / 16; ++kk) {
                        const uint32_t bb = tc::smem_u32(B1) + kk * 256;
                        mma_op<SPLIT>(tbase, tc::smem_u32(A0) + kk * 256, S::A0B, bb, S::B1B, K1p, idesc1, kk > 0);
                        mma_op<SPLIT>(tbase + TOFF, tc::smem_u32(dA0) + kk * 256, S::A0B, bb, S::B1B, K1p, idesc1,
                                      kk > 0);
                    }
                    tc::mma_commit(&mbar);
                }
                alive = tc_wait(&mbar, phase, status);
                float h1[E2], dh1[E2];
#pragma unroll
                for (int o = 0; o < E2; ++o) h1[o] = dh1[o] = 0.f;
                if (alive && warp_live) {
#pragma unroll
                    for (int cc = 0; cc < N1p; cc += 16) {
                        float v[16], dv[16];
                        tc::tmem_ld16(tlane + cc, v);
                        tc::tmem_ld16(tlane + TOFF + cc, dv);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int o = cc + q;
                            if (o < E2) {
                                const int os = o < E1 ? o : o - E1;
                                const float t = tanhf(v[q] + b1[o]);
                                h1[o] = h0[os] + t;
                                dh1[o] = fmaf(fmaf(-t, t, 1.f), dv[q], dh0[os]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int k8 = 0; k8 < K2p; k8 += 8) {
                    float v[8], dv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        v[q] = (k8 + q < E2) ? h1[k8 + q] : 0.f;
                        dv[q] = (k8 + q < E2) ? dh1[k8 + q] : 0.f;
                    }
                    st8_op<SPLIT>(A1, S::A1B, tid, k8, K2p, v);
                    st8_op<SPLIT>(dA1, S::A1B, tid, k8, K2p, dv);
                }
                tc_sync();
                if (!alive) break;
                if (tid == 0) {
#pragma unroll
                    for (int kk = 0; kk < K2p / 16; ++kk) {
                        const uint32_t bb = tc::smem_u32(B2) + kk * 256;
                        mma_op<SPLIT>(tbase, tc::smem_u32(A1) + kk * 256, S::A1B, bb, S::B2B, K2p, idesc2, kk > 0);
                        mma_op<SPLIT>(tbase + TOFF, tc::smem_u32(dA1) + kk * 256, S::A1B, bb, S::B2B, K2p, idesc2,
                                      kk > 0);
                    }
                    tc::mma_commit(&mbar);
                }
                alive = tc_wait(&mbar, phase, status);
                if constexpr (TAN) {
                // epilogue 2: G and dG/ds of the row to HBM (16-byte stores, 16 features at a time);
                // the warp's partial of T = R~^T G in double-float arithmetic, as k_embed_fwd_mx
                if (alive && warp_live) {
                    float *Gw = Gt + warp * 32 * 17;
                    float *Rwh = Rth + warp * 32 * 4, *Rwl = Rtl + warp * 32 * 4;
                    double *Tww = Tw + warp * 4 * E3;
                    float *gro = Gsto + ((size_t)i * nm + slot) * (2 * E3);
#pragma unroll
                    for (int c = 0; c < 4; ++c) df_split(valid ? gg.R[c] : 0.0, Rwh[lane * 4 + c], Rwl[lane * 4 + c]);
#pragma unroll
                    for (int cc = 0; cc < N2p; cc += 16) {
                        float v[16], dv[16], Gv[16], dGv[16];
                        tc::tmem_ld16(tlane + cc, v);
                        tc::tmem_ld16(tlane + TOFF + cc, dv);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int o = cc + q;
                            Gv[q] = 0.f;
                            dGv[q] = 0.f;
                            if (o < E3 && valid) {
                                const int os = o < E2 ? o : o - E2;
                                const float t = tanhf(v[q] + b2[o]);
                                Gv[q] = h1[os] + t;
                                dGv[q] = fmaf(fmaf(-t, t, 1.f), dv[q], dh1[os]);
                            }
                            Gw[lane * 17 + q] = Gv[q];
                        }
                        if (valid) {
                            // E3 = 4 e1: a group of 4 features is wholly inside or wholly outside
#pragma unroll
                            for (int q = 0; q < 16; q += 4)
                                if (cc + q < E3) {
                                    *reinterpret_cast<float4 *>(gro + cc + q) =
                                        make_float4(Gv[q], Gv[q + 1], Gv[q + 2], Gv[q + 3]);
                                    *reinterpret_cast<float4 *>(gro + E3 + cc + q) =
                                        make_float4(dGv[q], dGv[q + 1], dGv[q + 2], dGv[q + 3]);
                                }
                        }
                        __syncwarp();
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int p = lane + 32 * u, c = p >> 4, q = p & 15, o = cc + q;
                            if (o < E3) {
                                float sh = 0.f, sl = 0.f;
#pragma unroll 8
                                for (int rr = 0; rr < 32; ++rr)
                                    df_fma(sh, sl, Gw[rr * 17 + q], Rwh[rr * 4 + c], Rwl[rr * 4 + c]);
                                Tww[c * E3 + o] = df_value(sh, sl);
                            }
                        }
                        __syncwarp();
                    }
                }
                tc_sync();
                // merge the tile's warp partials into the atoms' sums, warps in order
                if (alive) {
                    for (int p = tid; p < 4 * E3; p += MXT) {
#pragma unroll
                        for (int w = 0; w < 4; ++w)
                            if (t0 + w < G) Tacc[bi.grp_atom[t0 + w] * 4 * E3 + p] += Tw[w * 4 * E3 + p];
                    }
                }
                __syncthreads();
                } else {
                // epilogue 2: G, dG/ds and the contractions with gT of the row's atom in
                // double-float arithmetic (exact products with gT's FP32 parts)
                double fo[3] = {0.0, 0.0, 0.0}, vir[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) vir[q] = 0.0;
                if (alive && warp_live) {
                    const float *gh = gTh + j * 4 * E3, *gl = gTl + j * 4 * E3;
                    float rah[4] = {0.f, 0.f, 0.f, 0.f}, ral[4] = {0.f, 0.f, 0.f, 0.f};
                    float rbh[4] = {0.f, 0.f, 0.f, 0.f}, rbl[4] = {0.f, 0.f, 0.f, 0.f};
                    // G and dG/ds of 16 features go through this thread's column of the layer-2
                    // operand buffer (idle once its MMA is done), so that the contraction is one
                    // compact loop rather than unrolled code for every feature
                    static_assert(2 * 16 * MXT * sizeof(float) <= 2 * S::A1B, "G, dG/ds staging fits in A1, dA1");
                    float *Gst = reinterpret_cast<float *>(A1) + tid, *dGst = Gst + 16 * MXT;
#pragma unroll
                    for (int cc = 0; cc < N2p; cc += 16) {
                        float v[16], dv[16];
                        tc::tmem_ld16(tlane + cc, v);
                        tc::tmem_ld16(tlane + TOFF + cc, dv);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int o = cc + q;
                            if (o < E3) {
                                const int os = o < E2 ? o : o - E2;
                                const float t = tanhf(v[q] + b2[o]);
                                Gst[q * MXT] = h1[os] + t;
                                dGst[q * MXT] = fmaf(fmaf(-t, t, 1.f), dv[q], dh1[os]);
                            }
                        }
                        const int nq = E3 - cc < 16 ? E3 - cc : 16;
#pragma unroll 1
                        for (int q = 0; q < nq; ++q) {
                            const float G2 = Gst[q * MXT], dG = dGst[q * MXT];
                            const int o = cc + q;
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const float bh = gh[c * E3 + o], bl = gl[c * E3 + o];
                                df_fma(rah[c], ral[c], G2, bh, bl);
                                df_fma(rbh[c], rbl[c], dG, bh, bl);
                            }
                        }
                    }
                    double ra[4], rb[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        ra[c] = df_value(rah[c], ral[c]);
                        rb[c] = df_value(rbh[c], rbl[c]);
                    }
                    if (valid) {
                        double gR0 = ra[0];
#pragma unroll
                        for (int c = 0; c < 4; ++c) gR0 = fma(gg.R[c], rb[c], gR0);
                        const double inv = 1.0 / gg.r;
                        const double u[3] = {gg.d[0] * inv, gg.d[1] * inv, gg.d[2] * inv};
                        const double dot = ra[1] * u[0] + ra[2] * u[1] + ra[3] * u[2];
                        const double sr = gg.s * inv;
                        const double coef = gR0 * gg.ds + gg.ds * dot - sr * dot;
                        double gv[3];
#pragma unroll
                        for (int bb = 0; bb < 3; ++bb) gv[bb] = fma(u[bb], coef, sr * ra[1 + bb]);
                        double *pg = pair_g + ((size_t)i * nm + slot) * 3;
                        pg[0] = gv[0];
                        pg[1] = gv[1];
                        pg[2] = gv[2];
#pragma unroll
                        for (int aa = 0; aa < 3; ++aa) {
                            fo[aa] = gv[aa];
#pragma unroll
                            for (int bb = 0; bb < 3; ++bb) vir[aa * 3 + bb] = -gg.d[aa] * gv[bb];
                        }
                    }
                    // the group's own-force and virial part: fixed shuffle tree
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) fo[q] += __shfl_xor_sync(0xffffffffu, fo[q], off);
#pragma unroll
                        for (int q = 0; q < 9; ++q) vir[q] += __shfl_xor_sync(0xffffffffu, vir[q], off);
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) red[warp * 12 + q] = fo[q];
#pragma unroll
                        for (int q = 0; q < 9; ++q) red[warp * 12 + 3 + q] = vir[q];
                    }
                }
                tc_sync();
                if (alive && tid < 12) {
#pragma unroll
                    for (int w = 0; w < 4; ++w)
                        if (t0 + w < G) facc[bi.grp_atom[t0 + w] * 12 + tid] += red[w * 12 + tid];
                }
                __syncthreads();
                }
            }
        }
        if (!alive) break;
        if constexpr (TAN) {
            // T = scale * sum; D = T_<^T T, per atom of the batch (as k_embed_fwd_mx)
            const int nd = m2 * E3;
            for (int j = 0; j < k; ++j) {
                const int i = bi.ids[j];
                double *Tj = Tacc + j * 4 * E3;
                for (int p = tid; p < 4 * E3; p += MXT) {
                    const double v = Tj[p] * m.desc_scale;
                    Tj[p] = v;
                    Tio[(size_t)i * 4 * E3 + p] = v;
                }
                __syncthreads();
                for (int q = tid; q < nd; q += MXT) {
                    const int a2 = q / E3, b2i = q - a2 * E3;
                    double acc = Tj[a2] * Tj[b2i];
                    acc = fma(Tj[E3 + a2], Tj[E3 + b2i], acc);
                    acc = fma(Tj[2 * E3 + a2], Tj[2 * E3 + b2i], acc);
                    acc = fma(Tj[3 * E3 + a2], Tj[3 * E3 + b2i], acc);
                    Dout[(size_t)i * nd + q] = acc;
                }
            }
        } else {
            for (int q = tid; q < k * 12; q += MXT) {
                const int j = q / 12, c = q - j * 12;
                const int i = bi.ids[j];
                if (c < 3) f_own[(size_t)i * 3 + c] = facc[q];
                else vir_part[(size_t)i * 9 + c - 3] = facc[q];
            }
        }
        first += k;
    }
    if (!alive) tc::mbar_wait(&mbar, phase ^ 1u);
    tc_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, TCOLS);
}

template <int E1, bool SPLIT>
__global__ void __launch_bounds__(MXT, 1) k_embed_bwd_mx(
    DevModel m, MixedModel mx, const double *__restrict__ x, const int32_t *__restrict__ types, Box3 box, int N,
    const int32_t *__restrict__ type_perm, const int32_t *__restrict__ type_start, const int32_t *__restrict__ nlist,
    const int32_t *__restrict__ nreal, double *__restrict__ Tin, const double *__restrict__ gD,
    double *__restrict__ pair_g, double *__restrict__ f_own, double *__restrict__ vir_part, int32_t *status)
{
    embed_mx_tangent_body<E1, SPLIT, false>(m, mx, x, types, box, N, type_perm, type_start, nlist, nreal, Tin, gD,
                                            pair_g, f_own, vir_part, nullptr, nullptr, status);
}

template <int E1>
__global__ void __launch_bounds__(MXT, 1) k_embed_tan_mx(
    DevModel m, MixedModel mx, const double *__restrict__ x, const int32_t *__restrict__ types, Box3 box, int N,
    const int32_t *__restrict__ type_perm, const int32_t *__restrict__ type_start, const int32_t *__restrict__ nlist,
    const int32_t *__restrict__ nreal, double *__restrict__ Tout, double *__restrict__ Dout,
    float *__restrict__ Gsto, int32_t *status)
{
    embed_mx_tangent_body<E1, false, true>(m, mx, x, types, box, N, type_perm, type_start, nlist, nreal, Tout,
                                           nullptr, nullptr, nullptr, nullptr, Dout, Gsto, status);
}

// Error-free sum of two double-float numbers: (h, l) += (h2, l2).
__device__ __forceinline__ void df_add(float &h, float &l, float h2, float l2)
{
    const float s = __fadd_rn(h, h2);
    const float z = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, z)), __fsub_rn(h2, z));
    h = s;
    l = __fadd_rn(l, __fadd_rn(l2, err));
}

// ------------------------------------------------------ streaming backward --
//
// k_embed_bwd_stmx: the mixed backward once k_embed_tan_mx has stored G and
// dG/ds (FP32) of every real row.  One warp per atom: dE/dT in FP64 (as
// k_embed_bwd_mx), split into two FP32 parts; the atom's real rows 32 at a
// time, lane q on the geometry of row q; in 8 steps of 4 rows, 8 lanes per
// row form sum_f G[f] gT[c][f] and sum_f dG[f] gT[c][f] in double-float
// arithmetic over the features u, u + 8, ... (exact products with gT's parts),
// a transposing shuffle tree of error-free double-float sums leaves component
// u on lane u, and the row's lane applies the chain rule through R~(r_ij) in
// FP64.  Fixed summation order: bit-reproducible.
constexpr int SMW = 4;  // warps (atoms in flight) per CTA

template <int E1>
__global__ void __launch_bounds__(SMW * 32, 4) k_embed_bwd_stmx(
    DevModel m, const double *__restrict__ x, const int32_t *__restrict__ types, Box3 box, int N,
    const int32_t *__restrict__ nlist, const int32_t *__restrict__ nreal, const double *__restrict__ Tin,
    const double *__restrict__ gD, const float *__restrict__ Gsto, double *__restrict__ pair_g,
    double *__restrict__ f_own, double *__restrict__ vir_part)
{
    constexpr int E3 = 4 * E1, KF = (E3 + 7) / 8;
    static_assert(4 * E3 >= 32 * 8, "the row sums [32][8] fit in the T buffer");
    // per warp: R1 holds T of the atom, then dE/dT as FP32 parts (gth, gtl); R2 holds dE/dT in
    // FP64 while it is formed, then the row sums [32][8]
    __shared__ double R1sh[SMW][4 * E3];
    __shared__ double R2sh[SMW][4 * E3];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int sub = lane & 7, gq = lane >> 3;
    const int T = m.ntypes, nm = m.nm, m2 = m.m2;
    double *Ts = R1sh[w], *gTd = R2sh[w], *sa_s = R2sh[w];
    float *gth = reinterpret_cast<float *>(R1sh[w]), *gtl = gth + 4 * E3;

    for (int i = blockIdx.x * SMW + w; i < N; i += gridDim.x * SMW) {
        const int a = types[i];
        const bool a_ok = (unsigned)a < (unsigned)T;
        for (int p = lane; p < 4 * E3; p += 32) Ts[p] = Tin[(size_t)i * 4 * E3 + p];
        __syncwarp();
        {
            // the 4 M2 long sums first, two per lane with every lane busy (two chains each), then
            // every entry's M2 short terms on top of them; then the FP32 parts over T
            const double *gd = gD + (size_t)i * m2 * E3;
            for (int p = lane; p < 4 * m2; p += 32) {
                const int cc = p / m2, xx = p - cc * m2;
                double acc = 0.0, acc2 = 0.0;
                for (int b2i = 0; b2i < E3; b2i += 2) {  // E3 = 4 e1 is even
                    acc = fma(gd[xx * E3 + b2i], Ts[cc * E3 + b2i], acc);
                    acc2 = fma(gd[xx * E3 + b2i + 1], Ts[cc * E3 + b2i + 1], acc2);
                }
                gTd[cc * E3 + xx] = acc + acc2;
            }
            __syncwarp();
            for (int p = lane; p < 4 * E3; p += 32) {
                const int cc = p / E3, xx = p - cc * E3;
                double acc = xx < m2 ? gTd[p] : 0.0;
                for (int a2 = 0; a2 < m2; ++a2) acc = fma(gd[a2 * E3 + xx], Ts[cc * E3 + a2], acc);
                gTd[p] = acc * m.desc_scale;
            }
            __syncwarp();
            for (int p = lane; p < 4 * E3; p += 32) df_split(gTd[p], gth[p], gtl[p]);
        }
        __syncwarp();
        int nr = 0;
        if (a_ok)
            for (int b = 0; b < T; ++b) nr += nreal[(size_t)i * T + b];
        const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        double fo[3] = {0.0, 0.0, 0.0}, vir[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) vir[q] = 0.0;
        for (int q0 = 0; q0 < nr; q0 += 32) {
            // row q0 + lane: its slot (type block and rank) and geometry
            int slot = -1;
            if (q0 + lane < nr) {
                int rem = q0 + lane;
                for (int b = 0; b < T; ++b) {
                    const int nb = nreal[(size_t)i * T + b];
                    if (slot < 0 && rem < nb) slot = m.sel_off[b] + rem;
                    rem -= nb;
                }
            }
            RowGeo gg;
            gg.s = gg.ds = 0.0;
            gg.R[0] = gg.R[1] = gg.R[2] = gg.R[3] = 0.0;
            gg.d[0] = gg.d[1] = gg.d[2] = 0.0;
            gg.r = 1.0;
            if (slot >= 0) geometry(m, x, xi, nlist[(size_t)i * nm + slot], box, gg);
            // the 8 sums of rows q0 + 4 it + gq, 8 lanes per row
            for (int it = 0; it < 8 && q0 + 4 * it < nr; ++it) {
                const int sl = __shfl_sync(0xffffffffu, slot, 4 * it + gq);
                float ph[8], pl[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) ph[c] = pl[c] = 0.f;
                if (sl >= 0) {
                    const float *gr = Gsto + ((size_t)i * nm + sl) * (2 * E3);
#pragma unroll
                    for (int k = 0; k < KF; ++k) {
                        const int ff = sub + 8 * k;
                        if (8 * k + 8 <= E3 || ff < E3) {
                            const float G = gr[ff], dG = gr[E3 + ff];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const float bh = gth[c * E3 + ff], bl = gtl[c * E3 + ff];
                                df_fma(ph[c], pl[c], G, bh, bl);
                                df_fma(ph[4 + c], pl[4 + c], dG, bh, bl);
                            }
                        }
                    }
                }
                // transposing tree over the row's 8 lanes: lane u ends with component u
#pragma unroll
                for (int o = 4, n = 4; o >= 1; o >>= 1, n >>= 1) {
                    const bool up = (sub & o) != 0;
#pragma unroll
                    for (int k = 0; k < n; ++k) {
                        const float sh = up ? ph[k] : ph[n + k], sl2 = up ? pl[k] : pl[n + k];
                        float kh = up ? ph[n + k] : ph[k], kl = up ? pl[n + k] : pl[k];
                        const float rh = __shfl_xor_sync(0xffffffffu, sh, o);
                        const float rl = __shfl_xor_sync(0xffffffffu, sl2, o);
                        df_add(kh, kl, rh, rl);
                        ph[k] = kh;
                        pl[k] = kl;
                    }
                }
                sa_s[(4 * it + gq) * 8 + sub] = df_value(ph[0], pl[0]);
            }
            __syncwarp();
            // chain rule through R~(r_ij) in FP64, lane q on row q0 + q
            if (slot >= 0) {
                double ra[4], rb[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    ra[c] = sa_s[lane * 8 + c];
                    rb[c] = sa_s[lane * 8 + 4 + c];
                }
                double gR0 = ra[0];
#pragma unroll
                for (int c = 0; c < 4; ++c) gR0 = fma(gg.R[c], rb[c], gR0);
                const double inv = 1.0 / gg.r;
                const double u[3] = {gg.d[0] * inv, gg.d[1] * inv, gg.d[2] * inv};
                const double dot = ra[1] * u[0] + ra[2] * u[1] + ra[3] * u[2];
                const double sr = gg.s * inv;
                const double coef = gR0 * gg.ds + gg.ds * dot - sr * dot;
                double gv[3];
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) gv[bb] = fma(u[bb], coef, sr * ra[1 + bb]);
                double *pg = pair_g + ((size_t)i * nm + slot) * 3;
                pg[0] = gv[0];
                pg[1] = gv[1];
                pg[2] = gv[2];
#pragma unroll
                for (int aa = 0; aa < 3; ++aa) {
                    fo[aa] += gv[aa];
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) vir[aa * 3 + bb] -= gg.d[aa] * gv[bb];
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
            for (int q = 0; q < 3; ++q) fo[q] += __shfl_xor_sync(0xffffffffu, fo[q], off);
#pragma unroll
            for (int q = 0; q < 9; ++q) vir[q] += __shfl_xor_sync(0xffffffffu, vir[q], off);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 3; ++q) f_own[(size_t)i * 3 + q] = fo[q];
#pragma unroll
            for (int q = 0; q < 9; ++q) vir_part[(size_t)i * 9 + q] = vir[q];
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------------- fitting --

constexpr int FIT_KC = 64;  // K per streamed chunk
constexpr int FIT_NS = 3;   // pipeline stages

__device__ __forceinline__ void bulk_g2s_mx(void *dst, const void *src, uint32_t bytes, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            tc::smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx_mx(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tc::smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

// The descriptor D (FP64, [N][K1]) as BF16 tiles of the fitting kernel's A
// operand: tile = 128 atoms of one type in type order, [K1p / 64] chunks of
// 128 x 64 in the canonical K-major layout.  One warp per row of a tile.
__global__ void __launch_bounds__(256) k_d2bf(const double *__restrict__ D, int K1, int nK,
                                              const int32_t *__restrict__ type_perm,
                                              const int32_t *__restrict__ type_start, int ntypes,
                                              unsigned char *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    int tl = gw / MXT;
    const int r = gw % MXT;
    int first = 0, cnt = -1;
    for (int t = 0; t < ntypes; ++t) {
        const int n_t = type_start[t + 1] - type_start[t];
        const int tiles = (n_t + MXT - 1) / MXT;
        if (tl < tiles) {
            first = type_start[t] + tl * MXT;
            cnt = min(MXT, n_t - tl * MXT);
            break;
        }
        tl -= tiles;
    }
    if (cnt < 0) return;
    const int i = r < cnt ? type_perm[first + r] : -1;
    unsigned char *o = out + (size_t)(gw / MXT) * nK * (MXT * FIT_KC * 2);
    for (int g8 = lane; g8 < nK * (FIT_KC / 8); g8 += 32) {
        const int k0 = g8 * 8, kc = k0 / FIT_KC;
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = (i >= 0 && k0 + q < K1) ? (float)D[(size_t)i * K1 + k0 + q] : 0.f;
        st8(o + (size_t)kc * (MXT * FIT_KC * 2), r, k0 % FIT_KC, FIT_KC, v);
    }
}

// One CTA = one tile of up to 128 atoms of one type.
__global__ void __launch_bounds__(MXT, 1) k_fit_mx(DevModel m, MixedModel mx, int N,
                                                   const int32_t *__restrict__ type_perm,
                                                   const int32_t *__restrict__ type_start,
                                                   const double *__restrict__ D, double *__restrict__ Ei,
                                                   double *__restrict__ gD, float *__restrict__ tbuf,
                                                   float *__restrict__ hbuf, int32_t *status)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *Ab = smraw;                               // [FIT_NS][128][64] bf16 (layer-1 input chunks)
    unsigned char *Bb = Ab + FIT_NS * MXT * FIT_KC * 2;      // [FIT_NS][256][64] bf16 (weight chunks)
    unsigned char *Hb = Bb + FIT_NS * 256 * FIT_KC * 2;      // [128][256] bf16 (activation / gradient)
    static_assert(MXT * 17 * sizeof(double) <= FIT_NS * MXT * FIT_KC * 2, "the dE/dD staging fits in the A ring");
    __shared__ __align__(8) uint64_t full[FIT_NS], empty[FIT_NS], dbar;
    __shared__ uint32_t tslot;
    __shared__ int pfail;
    __shared__ int rows_atom[MXT];
    constexpr int HK = 256;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    (void)lane;
    const int M = m.M, K1 = m.m2 * M, nf = m.n_fit;

    int bid = blockIdx.x, a = -1, first = 0, cnt = 0;
    const int tile_id = blockIdx.x;
    for (int t = 0; t < m.ntypes; ++t) {
        const int n_t = type_start[t + 1] - type_start[t];
        const int tiles = (n_t + MXT - 1) / MXT;
        if (bid < tiles) {
            a = t;
            first = type_start[t] + bid * MXT;
            cnt = min(MXT, n_t - bid * MXT);
            break;
        }
        bid -= tiles;
    }
    if (a < 0) return;
    if (warp == 0) tc::tmem_alloc(&tslot, 256);
    if (tid == 0) {
        for (int q = 0; q < FIT_NS; ++q) {
            tc::mbar_init(&full[q], 1);
            tc::mbar_init(&empty[q], 1);
        }
        tc::mbar_init(&dbar, 1);
        pfail = 0;
    }
    int ctr = 0;         // chunks issued so far (thread 0)
    uint32_t dph = 0;    // parity of the next completion of dbar
    rows_atom[tid] = tid < cnt ? type_perm[first + tid] : -1;
    tc_sync();
    const uint32_t tbase = tslot;
    const uint32_t tlane = tbase + ((uint32_t)(32 * warp) << 16);
    const int my = rows_atom[tid];
    const bool warp_live = 32 * warp < cnt;
    bool alive = true;
    const float *P32 = mx.p32 + m.fit_base[a];
    // per-tile activation buffers, column-major over the tile's 128 rows so that a warp's
    // accesses are contiguous: t of layer l, feature n at tb[(l HK + n) MXT]; h at hb[n MXT]
    float *tb = tbuf + (size_t)tile_id * nf * HK * MXT + tid;
    float *hb = hbuf + (size_t)tile_id * HK * MXT + tid;

    // Streamed GEMM into TMEM columns [0, Np): K-chunks of FIT_KC.  B (weights,
    // K-chunked, chunk kc at Bsrc + kc * chunk_bytes + row_off_bytes) always comes
    // by bulk copy; A is the layer-1 input (the descriptor's BF16 tile, bulk
    // copy) or the resident activation Hb.  One thread runs a FIT_NS-stage ring:
    // wait for the chunk, issue its MMAs, release the stage by commit, refill the
    // stage of the previous chunk.  Chunks are numbered across calls (ctr) so the
    // barrier parities stay consistent; every call ends with all MMAs complete.
    const unsigned char *dtile = mx.dtile + (size_t)tile_id * (mx.fit_kp[0] / FIT_KC) * (MXT * FIT_KC * 2);
    auto gemm = [&](bool from_D, int nK, const unsigned char *Bsrc, int64_t chunk_bytes, int64_t row_off_bytes,
                    int Np) -> bool {
        const uint32_t idesc = tc::make_idesc_bf16(MXT, Np);
        const uint32_t bbytes = (uint32_t)Np * FIT_KC * 2;
        const uint32_t abytes = from_D ? (uint32_t)MXT * FIT_KC * 2 : 0u;
        if (tid == 0) {
            const int c0 = ctr;
            int issued = 0, consumed = 0;
            auto load = [&](int c) {
                const int s = c % FIT_NS, kc = c - c0;
                mbar_expect_tx_mx(&full[s], abytes + bbytes);
                bulk_g2s_mx(Bb + (size_t)s * 256 * FIT_KC * 2, Bsrc + kc * chunk_bytes + row_off_bytes, bbytes,
                            &full[s]);
                if (from_D)
                    bulk_g2s_mx(Ab + (size_t)s * MXT * FIT_KC * 2, dtile + (size_t)kc * MXT * FIT_KC * 2, abytes,
                                &full[s]);
                ++issued;
            };
            for (int c = c0; c < c0 + FIT_NS && c < c0 + nK; ++c) load(c);
            bool ok = true;
            for (int c = c0; c < c0 + nK; ++c) {
                const int s = c % FIT_NS, kc = c - c0;
                if (!tc::mbar_wait(&full[s], (c / FIT_NS) & 1)) {
                    ok = false;
                    break;
                }
                ++consumed;
#pragma unroll
                for (int kk = 0; kk < FIT_KC / 16; ++kk) {
                    const uint64_t ad =
                        from_D ? tc::make_desc(tc::smem_u32(Ab + (size_t)s * MXT * FIT_KC * 2) + kk * 256, 128, FIT_KC * 16)
                               : tc::make_desc(tc::smem_u32(Hb) + (kc * (FIT_KC / 16) + kk) * 256, 128, HK * 16);
                    const uint64_t bd =
                        tc::make_desc(tc::smem_u32(Bb + (size_t)s * 256 * FIT_KC * 2) + kk * 256, 128, FIT_KC * 16);
                    tc::mma_bf16(tbase, ad, bd, idesc, kc > 0 || kk > 0);
                }
                tc::mma_commit(&empty[s]);
                if (c - 1 >= c0 && c - 1 + FIT_NS < c0 + nK) {
                    const int ps = (c - 1) % FIT_NS;
                    if (!tc::mbar_wait(&empty[ps], ((c - 1) / FIT_NS) & 1)) {
                        ok = false;
                        break;
                    }
                    load(c - 1 + FIT_NS);
                }
            }
            tc::mma_commit(&dbar);
            if (!ok) {
                atomicOr(status, DPF_MMA_TIMEOUT);
                for (int c = c0 + consumed; c < c0 + issued; ++c) tc::mbar_wait(&full[c % FIT_NS], (c / FIT_NS) & 1);
                pfail = 1;
            }
            ctr = c0 + nK;
        }
        const bool waited = tc::mbar_wait(&dbar, dph);
        dph ^= 1u;
        const bool bad = __syncthreads_or(!waited) || pfail;
        tc::fence_after_sync();
        if (bad && tid == 0) atomicOr(status, DPF_MMA_TIMEOUT);
        return !bad;
    };

    // ---------------- forward
    int Kin = K1;
    for (int l = 0; l < nf && alive; ++l) {
        const int F = m.fit[l];
        const int Np = mx.fit_np[l];
        const int nK = mx.fit_kp[l] / FIT_KC;
        const unsigned char *Bsrc = mx.fit_fwd + mx.fit_fwd_off[a][l];
        alive = gemm(l == 0, nK, Bsrc, (int64_t)Np * 128, 0, Np);
        if (!alive) break;
        // bias offset in the FP64 parameter layout
        int64_t boff = 0;
        {
            int kin = K1;
            for (int q = 0; q <= l; ++q) {
                boff += (int64_t)kin * m.fit[q];
                if (q < l) boff += m.fit[q];
                kin = m.fit[q];
            }
        }
        const float *bias = P32 + boff;
        if (warp_live) {
            for (int cc = 0; cc < Np; cc += 16) {
                float v[16];
                tc::tmem_ld16(tlane + cc, v);
                if (my >= 0) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int n = cc + q;
                        if (n < F) {
                            const float t = tanhf(v[q] + bias[n]);
                            tb[(l * HK + n) * MXT] = t;
                            hb[n * MXT] = (l > 0 ? hb[n * MXT] : 0.f) + t;  // equal-width skip after the first layer
                        }
                    }
                }
            }
        }
        __syncthreads();
        // next layer's A operand (bf16, zero-padded to 256)
        for (int k8 = 0; k8 < HK; k8 += 8) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = (my >= 0 && k8 + q < F) ? hb[(k8 + q) * MXT] : 0.f;
            st8(Hb, tid, k8, HK, v);
        }
        tc_sync();
        Kin = F;
    }
    // output layer (FP64 accumulation of the dot product)
    const float *wo = nullptr;
    {
        int64_t off = 0;
        int kin = K1;
        for (int q = 0; q < nf; ++q) {
            off += (int64_t)kin * m.fit[q] + m.fit[q];
            kin = m.fit[q];
        }
        wo = P32 + off;
    }
    if (alive && my >= 0) {
        double e = (double)wo[Kin];
        for (int n = 0; n < Kin; ++n) e = fma((double)hb[n * MXT], (double)wo[n], e);
        Ei[my] = e;
    }

    // ---------------- backward: gh = w_out; gz_l = gh * (1 - t_l^2)
    if (my >= 0)
        for (int n = 0; n < Kin; ++n) hb[n * MXT] = wo[n];
    for (int l = nf - 1; l >= 0 && alive; --l) {
        const int F = m.fit[l];
        const int Kl = (l == 0) ? K1 : m.fit[l - 1];
        for (int k8 = 0; k8 < HK; k8 += 8) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int n = k8 + q;
                float gz = 0.f;
                if (my >= 0 && n < F) {
                    const float t = tb[(l * HK + n) * MXT];
                    gz = hb[n * MXT] * fmaf(-t, t, 1.f);
                }
                v[q] = gz;
            }
            st8(Hb, tid, k8, HK, v);
        }
        tc_sync();
        const int nK = mx.fit_fp[l] / FIT_KC;
        const int Kinp = mx.fit_kinp[l];
        const unsigned char *Bsrc = mx.fit_bwd + mx.fit_bwd_off[a][l];
        // output columns in chunks of up to 256 (128 for the wide first layer)
        const int NB = Kinp <= 256 ? Kinp : 128;
        for (int n0 = 0; n0 < Kinp && alive; n0 += NB) {
            const int nb = min(NB, Kinp - n0);
            alive = gemm(false, nK, Bsrc, (int64_t)Kinp * 128, (int64_t)(n0 / 8) * 1024, nb);
            if (!alive) break;
            if (l == 0) {
                // dE/dD through shared memory (the A ring is idle in the backward), 16 columns at
                // a time, so that each half-warp stores 128 contiguous bytes of one atom's row
                double *stage = reinterpret_cast<double *>(Ab);  // [MXT][17]
                for (int cc = 0; cc < nb; cc += 16) {
                    if (warp_live) {
                        float v[16];
                        tc::tmem_ld16(tlane + cc, v);
#pragma unroll
                        for (int q = 0; q < 16; ++q) stage[tid * 17 + q] = (double)v[q];
                    }
                    __syncthreads();
                    for (int p = tid; p < MXT * 16; p += MXT) {
                        const int row = p >> 4, q = p & 15, n = n0 + cc + q;
                        const int at = rows_atom[row];
                        if (at >= 0 && n < Kl) gD[(size_t)at * K1 + n] = stage[row * 17 + q];
                    }
                    __syncthreads();
                }
            } else if (warp_live) {
                for (int cc = 0; cc < nb; cc += 16) {
                    float v[16];
                    tc::tmem_ld16(tlane + cc, v);
                    if (my >= 0) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int n = n0 + cc + q;
                            if (n < Kl) hb[n * MXT] = v[q] + hb[n * MXT];  // equal widths: the skip passes gh through
                        }
                    }
                }
            }
            tc_sync();
        }
    }
    tc_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

template <int E1, bool SPLIT>
size_t fwd_smem()
{
    using S = EmbShape<E1>;
    using P = EmbPlan<E1, SPLIT>;
    return P::FEND + sizeof(double) * (4 * 4 * S::E3 + P::AB * 4 * S::E3) + sizeof(float) * (4 * 32 * 17 + 2 * 4 * 32 * 4);
}
template <int E1, bool SPLIT>
size_t bwd_smem()
{
    using S = EmbShape<E1>;
    using P = EmbPlan<E1, SPLIT>;
    return P::BEND + sizeof(double) * (4 * S::E3 + 48 + P::AB * 12) + sizeof(float) * 2 * P::AB * 4 * S::E3;
}

template <int E1>
size_t tan_smem()
{
    using S = EmbShape<E1>;
    using P = EmbPlan<E1, false>;
    return P::BEND + sizeof(double) * (4 * 4 * S::E3 + tan_ab(E1) * 4 * S::E3) + sizeof(float) * 2 * 4 * 32 * 4;
}

// CTAs per SM that fit next to each other (shared memory; a 1 KB reserve per CTA)
inline int ctas_per_sm(size_t smem) { return 2 * (smem + 2048) <= 232448 ? 2 : 1; }

template <int E1, bool SPLIT>
cudaError_t launch_fwd(cudaStream_t st, const DevModel &m, const MixedModel &mx, const double *x,
                       const int32_t *types, Box3 box, int N, const FormatBuffers &fb, const NlistBuffers &nb,
                       EvalBuffers eb, int num_sms, int32_t *status)
{
    const size_t smem = fwd_smem<E1, SPLIT>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e =
            cudaFuncSetAttribute(k_embed_fwd_mx<E1, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    // one or two CTAs per SM (tensor memory: 128 columns each), each a balanced share of the atoms
    int grid = ctas_per_sm(smem) * num_sms;
    if (grid > (N + 7) / 8) grid = (N + 7) / 8;
    k_embed_fwd_mx<E1, SPLIT><<<grid, MXT, smem, st>>>(m, mx, x, types, box, N, nb.type_perm, nb.type_start,
                                                       fb.nlist, fb.nreal, eb.T, eb.D, status);
    return cudaGetLastError();
}

template <int E1, bool SPLIT>
cudaError_t launch_bwd(cudaStream_t st, const DevModel &m, const MixedModel &mx, const double *x,
                       const int32_t *types, Box3 box, int N, const FormatBuffers &fb, const NlistBuffers &nb,
                       EvalBuffers eb, int num_sms, int32_t *status)
{
    const size_t smem = bwd_smem<E1, SPLIT>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e =
            cudaFuncSetAttribute(k_embed_bwd_mx<E1, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    // one or two CTAs per SM (tensor memory: <= 256 columns each), each a balanced share of the atoms
    int grid = ctas_per_sm(smem) * num_sms;
    if (grid > (N + 7) / 8) grid = (N + 7) / 8;
    k_embed_bwd_mx<E1, SPLIT><<<grid, MXT, smem, st>>>(m, mx, x, types, box, N, nb.type_perm, nb.type_start,
                                                       fb.nlist, fb.nreal, eb.T, eb.gD, eb.pair_g, eb.f_own,
                                                       eb.vir_part, status);
    return cudaGetLastError();
}

template <int E1>
cudaError_t launch_tan(cudaStream_t st, const DevModel &m, const MixedModel &mx, const double *x,
                       const int32_t *types, Box3 box, int N, const FormatBuffers &fb, const NlistBuffers &nb,
                       EvalBuffers eb, int num_sms, int32_t *status)
{
    const size_t smem = tan_smem<E1>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_embed_tan_mx<E1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    int grid = ctas_per_sm(smem) * num_sms;
    if (grid > (N + 7) / 8) grid = (N + 7) / 8;
    k_embed_tan_mx<E1><<<grid, MXT, smem, st>>>(m, mx, x, types, box, N, nb.type_perm, nb.type_start, fb.nlist,
                                                fb.nreal, eb.T, eb.D, eb.Gmx, status);
    return cudaGetLastError();
}

template <int E1>
cudaError_t launch_bwd_stmx(cudaStream_t st, const DevModel &m, const double *x, const int32_t *types, Box3 box,
                            int N, const FormatBuffers &fb, EvalBuffers eb, int num_sms)
{
    int grid = (N + SMW - 1) / SMW;
    if (grid > 4 * num_sms) grid = 4 * num_sms;
    if (grid < 1) grid = 1;
    k_embed_bwd_stmx<E1><<<grid, SMW * 32, 0, st>>>(m, x, types, box, N, fb.nlist, fb.nreal, eb.T, eb.gD, eb.Gmx,
                                                    eb.pair_g, eb.f_own, eb.vir_part);
    return cudaGetLastError();
}

}  // namespace

size_t dp_mx_store_bytes(const DevModel &m, int64_t natoms)
{
    return (size_t)natoms * (size_t)m.nm * 2 * (size_t)m.M * sizeof(float);
}

cudaError_t dp_launch_embed_tan_mx(cudaStream_t st, const DevModel &m, const MixedModel &mx, const double *x,
                                   const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                   const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                   int64_t *launches)
{
    *launches += 1;
    if (mx.split) return cudaErrorInvalidValue;
    switch (m.emb[0]) {
    case 16: return launch_tan<16>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 25: return launch_tan<25>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 32: return launch_tan<32>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t dp_launch_embed_bwd_stmx(cudaStream_t st, const DevModel &m, const double *x, const int32_t *types,
                                     Box3 box, int N, const FormatBuffers &fb, EvalBuffers eb, int num_sms,
                                     int64_t *launches)
{
    *launches += 1;
    switch (m.emb[0]) {
    case 16: return launch_bwd_stmx<16>(st, m, x, types, box, N, fb, eb, num_sms);
    case 25: return launch_bwd_stmx<25>(st, m, x, types, box, N, fb, eb, num_sms);
    case 32: return launch_bwd_stmx<32>(st, m, x, types, box, N, fb, eb, num_sms);
    default: return cudaErrorInvalidValue;
    }
}

bool dp_mixed_supported(const DevModel &m)
{
    if (m.n_emb != 3) return false;
    const int e1 = m.emb[0];
    if (!(e1 == 16 || e1 == 25 || e1 == 32)) return false;
    if (m.emb[1] != 2 * e1 || m.emb[2] != 4 * e1) return false;
    for (int l = 0; l < m.n_fit; ++l) {
        if (m.fit[l] % 16 != 0 || m.fit[l] > 256) return false;
        if (l > 0 && m.fit[l] != m.fit[l - 1]) return false;
    }
    return true;
}

cudaError_t dp_launch_embed_fwd_mx(cudaStream_t st, const DevModel &m, const MixedModel &mx, const double *x,
                                   const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                   const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                   int64_t *launches)
{
    *launches += 1;
    const bool sp = mx.split != 0;
    switch (m.emb[0]) {
    case 16: return sp ? launch_fwd<16, true>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status)
                       : launch_fwd<16, false>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 25: return sp ? launch_fwd<25, true>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status)
                       : launch_fwd<25, false>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 32: return sp ? launch_fwd<32, true>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status)
                       : launch_fwd<32, false>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t dp_launch_embed_bwd_mx(cudaStream_t st, const DevModel &m, const MixedModel &mx, const double *x,
                                   const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                   const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                   int64_t *launches)
{
    *launches += 1;
    const bool sp = mx.split != 0;
    switch (m.emb[0]) {
    case 16: return sp ? launch_bwd<16, true>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status)
                       : launch_bwd<16, false>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 25: return sp ? launch_bwd<25, true>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status)
                       : launch_bwd<25, false>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 32: return sp ? launch_bwd<32, true>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status)
                       : launch_bwd<32, false>(st, m, mx, x, types, box, N, fb, nb, eb, num_sms, status);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t dp_launch_fit_mx(cudaStream_t st, const DevModel &m, const MixedModel &mx, int N,
                             const NlistBuffers &nb, EvalBuffers eb, int32_t *status, int64_t *launches)
{
    const size_t smem = FIT_NS * MXT * FIT_KC * 2 + FIT_NS * 256 * FIT_KC * 2 + MXT * 256 * 2;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_fit_mx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int grid = (N + MXT - 1) / MXT + m.ntypes;
    const int K1 = m.m2 * m.M;
    k_d2bf<<<(grid * MXT * 32 + 255) / 256, 256, 0, st>>>(eb.D, K1, mx.fit_kp[0] / FIT_KC, nb.type_perm,
                                                          nb.type_start, m.ntypes, mx.dtile);
    *launches += 1;
    k_fit_mx<<<grid, MXT, smem, st>>>(m, mx, N, nb.type_perm, nb.type_start, eb.D, eb.Ei, eb.gD, eb.fit_t,
                                      eb.fit_h, status);
    *launches += 1;
    return cudaGetLastError();
}
