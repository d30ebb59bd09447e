// embed_x.cu -- FP64 environment matrix, embedding net and descriptor
// (Algorithm 2; Eqs. embedding, embedding-first, embedding-rest, descrpt)
// with the embedding net's dense layers on the tensor cores at FP64 accuracy.
//
// The doubling embedding net (widths e1, 2e1, 4e1) costs 2 e1 (2 e1) + 2 (2 e1)(4 e1)
// FLOP per neighbour row.  Layer 0 (1 -> e1) runs on the FP64 units (one row
// per lane, the warps splitting the columns); layer 1 and the last layer are
// exact products of digit expansions (as the fitting net's GEMMs, csrc/fit_oz.cu):
//   h (|h| < 2)   -> S = 7 digits in base 2^8 of round(h 2^55),
//   W column f    -> 7 digits of round(W[., f] 2^(56 - f_f)),  2^f_f > max |W[., f]|,
//   z[f][row] = 2^(1 + f_f) sum_{g=2}^{8} 2^(-8 g) C_g,  C_g = sum_{s+t=g} A_s B_t,
// with K <= 64, so K 4^7 (S + 2) < 2^24: every partial sum of every C_g is an
// integer the FP32 accumulators hold exactly.  The MMAs are transposed: M = the
// output features (the rows of W^T; 128 for the last layer, 64 for layer 1),
// N = 32 neighbour rows.  In the last layer's epilogue thread f owns feature f
// of the 32 rows: it adds the bias, applies the FP64 tanh and the (h1, h1) skip,
// and accumulates its column of T = R~^T G in registers; layer 1's epilogue
// (an M = 64 accumulator: 16 lanes of each warp's quarter) writes h1 back as
// FP64 rows.  One CTA (16 warps) per SM, persistent over the type-sorted
// atoms; the current net's weight digits and column exponents arrive by one
// bulk copy.  Bounded waits; on a timeout the kernel sets DPF_MMA_TIMEOUT,
// frees its tensor memory and returns.
//
// Kernels: k_embed_fwd_x (G, T, D) and k_embed_bwd_x (G and dG/ds recomputed,
// contracted with dE/dT) when G is not kept; k_embed_tan_x (G and dG/ds once,
// stored in HBM, with T and D) and the streaming k_embed_bwd_st when it is.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dp_internal.cuh"
#include "oz.cuh"
#include "tc.cuh"

namespace {

constexpr int XS = 7;        // digits
constexpr int XBETA = 8;     // digit width (bits)
constexpr int XNR = 32;      // neighbour rows per MMA (N)
constexpr int XM = 128;      // output features per MMA (M), 4 e1 <= 128
constexpr int XGR = 512;     // rows of one neighbour block whose geometry is staged at once

constexpr int XM1 = 64;      // output features of the layer-1 MMA (M), 2 e1 <= 64

constexpr int k2p_of(int e1) { return (2 * e1 + 15) / 16 * 16; }
constexpr int k1p_of(int e1) { return (e1 + 15) / 16 * 16; }
// layer 1 (e1 -> 2 e1) on the tensor cores as well, where its weight digits fit
// in shared memory next to each kernel's buffers (both kernels, every supported width)
constexpr bool l1fwd_of(int e1) { return e1 <= 32; }
constexpr bool l1bwd_of(int e1) { return e1 <= 32; }
// bytes of the last layer's weights: digits [XS][128 x K2p] bf16, then 128 int32 exponents
constexpr size_t w2_bytes(int e1) { return (size_t)XS * XM * k2p_of(e1) * 2 + XM * 4; }
// bytes of layer 1's weights: digits [XS][64 x K1p] bf16, then 64 int32 exponents
constexpr size_t w1_bytes(int e1) { return l1fwd_of(e1) ? (size_t)XS * XM1 * k1p_of(e1) * 2 + XM1 * 4 : 0; }
// bytes of one net's weight block: the last layer's part, then layer 1's
constexpr size_t net_bytes(int e1) { return w2_bytes(e1) + w1_bytes(e1); }

__device__ __forceinline__ void bulk_g2s_x(void *dst, const void *src, uint32_t bytes, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            tc::smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx_x(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tc::smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

// Both embedding kernels run 16 warps (four per SM sub-partition, to hide the
// latency of their dependent FP64 chains).  In the epilogues warps w, w + 4,
// w + 8 and w + 12 share TMEM lanes 32 (w % 4) .. + 31: each thread owns 8
// rows of the last layer's accumulator (32x32b layout) and 4 rows of each
// lane-half of layer 1's M = 64 accumulator.
constexpr int XTB = 512;                   // threads of the embedding kernels
constexpr int XRB = XNR * 4 / (XTB / 32);  // rows per thread in the last layer's epilogue (8)
constexpr int XQB = XRB / 2;               // rows per thread per lane-half in layer 1's epilogue (4)

// y[q] = 2^p_q sum_{g=2}^{8} C_g[q] 2^(8 (8 - g)) for the 8 columns at taddr
// (group g at column offset (g - 2) * XNR), with p_q = p0 + (rowexp ? rowexp[q] :
// 0): the group sums are integers below 2^24, so they are combined exactly in
// two int64 Horner chains (g = 2..4 and g = 5..8, below 2^41 and 2^49) and
// converted once, y = (hi 2^32 + lo) 2^p_q with one rounding -- on the integer
// pipe (oz_i64x2_scaled), bit for bit fma((double)hi, 2^32, (double)lo) 2^p_q.
__device__ __forceinline__ void combine_groups_8(uint32_t taddr, double (&y)[8], int p0, const int *rowexp)
{
    static_assert(XS == 7 && XBETA == 8, "combine_groups_8 assumes 7 digits of 8 bits");
    long long hi[8], lo[8];
#pragma unroll
    for (int g = 2; g <= XS + 1; ++g) {
        float v[8];
        tc::tmem_ld8(taddr + (uint32_t)(g - 2) * XNR, v);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long long iv = (long long)__float2int_rn(v[q]);
            if (g == 2) hi[q] = iv;
            else if (g <= 4) hi[q] = (hi[q] << XBETA) + iv;
            else if (g == 5) lo[q] = iv;
            else lo[q] = (lo[q] << XBETA) + iv;
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = oz_i64x2_scaled(hi[q], lo[q], p0 + (rowexp ? rowexp[q] : 0));
}

// combine_groups_8 for an M = 64 accumulator: the 4 columns that
// tc::tmem_ld16x2_4 (second half 16 columns on) gives this thread, scaled by
// 2^(p0 + rowexp[j]).
__device__ __forceinline__ void combine_groups4(uint32_t taddr, double (&y)[4], int p0, const int *rowexp)
{
    long long hi[4], lo[4];
#pragma unroll
    for (int g = 2; g <= XS + 1; ++g) {
        float v[4];
        tc::tmem_ld16x2_4<16>(taddr + (uint32_t)(g - 2) * XNR, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long iv = (long long)__float2int_rn(v[q]);
            if (g == 2) hi[q] = iv;
            else if (g <= 4) hi[q] = (hi[q] << XBETA) + iv;
            else if (g == 5) lo[q] = iv;
            else lo[q] = (lo[q] << XBETA) + iv;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) y[q] = oz_i64x2_scaled(hi[q], lo[q], p0 + (rowexp ? rowexp[q] : 0));
}

template <int E1>
struct XShape {
    static constexpr int E2 = 2 * E1, E3 = 4 * E1, K2p = k2p_of(E1), K1p = k1p_of(E1);
    static constexpr bool L1 = l1fwd_of(E1);  // layer 1 on the tensor cores
    // odd row strides (in doubles): one row per lane reads without bank conflicts
    static constexpr int LD0 = (E1 % 2) ? E1 + 2 : E1 + 1, LD1 = (E2 % 2) ? E2 + 2 : E2 + 1;
    static constexpr size_t WD = net_bytes(E1);              // weight digits + exponents (both layers)
    static constexpr size_t NB = net_bytes(E1);              // stride of the nets' weight blocks
    static constexpr size_t BD = (size_t)XS * XNR * K2p * 2;  // row digits
    // FP64 region: W1 (E1 x E2, SIMT layer 1 only), w0, b0 (E1), b1 (E2), b2 (XM), H0, H1,
    // Rt (XGR x 4), srow (XGR); after an atom's last chunk the geometry rows hold Tsm
    // ([XTB / XM] x 4 x XM: one T partial per row group)
    static constexpr size_t F64 =
        (L1 ? 0 : (size_t)E1 * E2) + 2 * E1 + E2 + XM + XNR * LD0 + XNR * LD1 + XGR * 4 + XGR;
    static_assert((XTB / XM) * 4 * XM <= XGR * 5, "the T partials fit in the geometry rows");
    static constexpr size_t SMEM = WD + BD + F64 * 8;
    static_assert(!L1 || (XS * XNR * K1p * 2 <= BD && E2 <= XM1), "layer 1's digits use the row-digit buffer");
    static_assert(SMEM + 1024 <= 232448, "dynamic plus static shared memory above the 227 KB opt-in limit");
};

template <int E1>
__global__ void __launch_bounds__(XTB, 1) k_embed_fwd_x(DevModel m, const unsigned char *__restrict__ wx,
                                                       const double *__restrict__ x,
                                                       const int32_t *__restrict__ types, Box3 box, int N,
                                                       const int32_t *__restrict__ type_perm,
                                                       const int32_t *__restrict__ nlist,
                                                       const int32_t *__restrict__ nreal, double *__restrict__ Tout,
                                                       double *__restrict__ Dout, int32_t *status)
{
    using X = XShape<E1>;
    constexpr int E2 = X::E2, E3 = X::E3, K2p = X::K2p, K1p = X::K1p, LD0 = X::LD0, LD1 = X::LD1;
    constexpr bool L1 = X::L1;
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *Wd = smraw;                                   // weight digits, then exponents
    const int *fexp = reinterpret_cast<const int *>(Wd + (size_t)XS * XM * K2p * 2);
    unsigned char *Wd1 = Wd + w2_bytes(E1);                      // layer 1's weight digits (L1)
    const int *fexp1 = reinterpret_cast<const int *>(Wd1 + (size_t)XS * XM1 * K1p * 2);
    unsigned char *Bd = Wd + X::WD;                              // row digits
    double *W1s = reinterpret_cast<double *>(Bd + X::BD);       // SIMT layer 1 only
    double *w0s = W1s + (L1 ? 0 : E1 * E2);
    double *b0s = w0s + E1;
    double *b1s = b0s + E1;
    double *b2s = b1s + E2;
    double *H0 = b2s + XM;
    double *H1 = H0 + XNR * LD0;
    double *Rga = H1 + XNR * LD1;   // environment rows of the block [XGR][4]
    double *sga = Rga + XGR * 4;    // s of the block [XGR]
    double *Tsm = Rga;              // [XTB / XM][4][XM], once the atom's chunks are done
    __shared__ __align__(8) uint64_t mbar_w, mbar_m;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = m.ntypes, nm = m.nm;

    if (warp == 0) tc::tmem_alloc(&tslot, 256);
    if (tid == 0) {
        tc::mbar_init(&mbar_w, 1);
        tc::mbar_init(&mbar_m, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tslot;
    const uint32_t tlane = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t idesc = tc::make_idesc_bf16(XM, XNR);
    uint32_t ph_w = 0, ph_m = 0;
    bool alive = true;
    bool pend_w = false, pend_m = false;  // a copy or MMAs still in flight after a timeout
    int staged = -1;
    const int f = tid & (XM - 1);  // epilogue: this thread's output feature
    const int grp = tid >> 7;      // ... and rows XRB grp .. XRB grp + XRB - 1 of the chunk

    for (int ii = blockIdx.x; ii < N && alive; ii += gridDim.x) {
        const int i = type_perm[ii];
        const int a = types[i];
        const bool a_ok = (unsigned)a < (unsigned)T;
        const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        double tacc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = 0; b < T && alive; ++b) {
            const int nb = a_ok ? nreal[(size_t)i * T + b] : 0;
            if (nb == 0) continue;
            const int net = a * T + b;
            if (net != staged) {
                __syncthreads();
                if (tid == 0) {
                    mbar_expect_tx_x(&mbar_w, (uint32_t)X::WD);
                    bulk_g2s_x(Wd, wx + (size_t)net * X::NB, (uint32_t)X::WD, &mbar_w);
                }
                const double *src = m.params + m.emb_base[net];
                for (int q = tid; q < E1; q += XTB) {
                    w0s[q] = src[q];
                    b0s[q] = src[E1 + q];
                }
                if constexpr (!L1)
                    for (int q = tid; q < E1 * E2; q += XTB) W1s[q] = src[2 * E1 + q];
                for (int q = tid; q < E2; q += XTB) b1s[q] = src[2 * E1 + E1 * E2 + q];
                for (int q = tid; q < XM; q += XTB)
                    b2s[q] = q < E3 ? src[2 * E1 + E1 * E2 + E2 + E2 * E3 + q] : 0.0;
                const bool ok = tc::mbar_wait(&mbar_w, ph_w);
                ph_w ^= 1u;
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) atomicOr(status, DPF_MMA_TIMEOUT);
                    alive = false;
                    pend_w = true;
                    break;
                }
                staged = net;
            }
            const int cexp = 1 + (f < E3 ? fexp[f] : 0) - XBETA * (XS + 1);  // scale of the group sums
            for (int c0 = 0; c0 < nb && alive; c0 += XNR) {
                const int nv = min(XNR, nb - c0);  // valid rows of the chunk
                // geometry of the next XGR rows of the block, one row per thread
                if (c0 % XGR == 0) {
                    __syncthreads();
                    for (int q = tid; q < XGR; q += XTB) {
                        const int r = c0 + q;
                        double s = 0.0, R[4] = {0.0, 0.0, 0.0, 0.0};
                        if (r < nb) {
                            const int j = nlist[(size_t)i * nm + m.sel_off[b] + r];
                            const double xj[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
                            double d[3], ds;
                            const double rr = dp_pinned_dist(xi, xj, box, d);
                            dp_switch(rr, m.rcut_smth, m.rcut, s, ds);
                            const double inv = 1.0 / rr;
                            R[0] = s;
                            R[1] = s * d[0] * inv;
                            R[2] = s * d[1] * inv;
                            R[3] = s * d[2] * inv;
                        }
                        sga[q] = s;
#pragma unroll
                        for (int c = 0; c < 4; ++c) Rga[q * 4 + c] = R[c];
                    }
                }
                const double *srow = sga + (c0 % XGR);
                const double *Rt = Rga + (c0 % XGR) * 4;
                __syncthreads();
                // layer 0: h0 = tanh(s w0 + b0), one row per lane, warps split the columns
                {
                    const double sv = srow[lane];
                    for (int o = warp; o < E1; o += XTB / 32) H0[lane * LD0 + o] = dp_tanh64(fma(sv, w0s[o], b0s[o]), m.tanh_tab);
                }
                __syncthreads();
                // layer 1: h1 = (h0, h0) + tanh(h0 W1 + b1)
                if constexpr (L1) {
                    // digits of h0 (fixed scale: |h0| <= 1), then z1^T (64 features x 32 rows)
                    for (int p = tid; p < XNR * (K1p / 8); p += XTB) {
                        const int row = p % XNR, k0 = (p / XNR) * 8;
                        long long I[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const double v = (k0 + q < E1) ? H0[row * LD0 + k0 + q] : 0.0;
                            I[q] = oz_rint_pow2(v, 55);  // round(v 2^55)
                        }
                        const uint32_t ofs = tc::kmajor_offset(row, k0, K1p);
                        for (int sd = XS - 1; sd >= 0; --sd) {
                            int dg[8];
#pragma unroll
                            for (int q = 0; q < 8; ++q) dg[q] = sd > 0 ? oz_digit_step(I[q], XBETA) : (int)I[q];
                            uint4 u;
                            u.x = (uint32_t)oz_bf16_int(dg[0]) | ((uint32_t)oz_bf16_int(dg[1]) << 16);
                            u.y = (uint32_t)oz_bf16_int(dg[2]) | ((uint32_t)oz_bf16_int(dg[3]) << 16);
                            u.z = (uint32_t)oz_bf16_int(dg[4]) | ((uint32_t)oz_bf16_int(dg[5]) << 16);
                            u.w = (uint32_t)oz_bf16_int(dg[6]) | ((uint32_t)oz_bf16_int(dg[7]) << 16);
                            *reinterpret_cast<uint4 *>(Bd + (size_t)sd * XNR * K1p * 2 + ofs) = u;
                        }
                    }
                    tc::fence_proxy_async();
                    tc::fence_before_sync();
                    __syncthreads();
                    tc::fence_after_sync();
                    if (tid == 0) {
                        const uint32_t wa = tc::smem_u32(Wd1), ba = tc::smem_u32(Bd);
                        const uint32_t idesc1 = tc::make_idesc_bf16(XM1, XNR);
#pragma unroll
                        for (int s = 1; s <= XS; ++s)
#pragma unroll
                            for (int t = 1; t + s <= XS + 1; ++t)
#pragma unroll
                                for (int kk = 0; kk < K1p / 16; ++kk)
                                    tc::mma_bf16(
                                        tbase + (uint32_t)(s + t - 2) * XNR,
                                        tc::make_desc(wa + (uint32_t)(s - 1) * XM1 * K1p * 2 + kk * 256, 128, K1p * 16),
                                        tc::make_desc(ba + (uint32_t)(t - 1) * XNR * K1p * 2 + kk * 256, 128, K1p * 16),
                                        idesc1, s > 1 || kk > 0);
                        tc::mma_commit(&mbar_m);
                    }
                    {
                        const bool ok = tc::mbar_wait(&mbar_m, ph_m);
                        ph_m ^= 1u;
                        const bool bad = __syncthreads_or(!ok);
                        tc::fence_after_sync();
                        if (bad) {
                            if (tid == 0) atomicOr(status, DPF_MMA_TIMEOUT);
                            alive = false;
                            pend_m = true;
                            break;
                        }
                    }
                    // epilogue: the warp's TMEM quarter holds features 16 (warp % 4) .. + 15 in
                    // its first 16 lanes; lanes < 16 take rows 0..15, the others rows 16..31,
                    // and warps w, w + 4, w + 8, w + 12 take 4 of them each
                    const int f1 = 16 * (warp & 3) + (lane & 15);
                    const int r0 = 16 * (lane >> 4) + XQB * (warp >> 2);
                    double y1[XQB];
                    combine_groups4(tlane + XQB * (uint32_t)(warp >> 2), y1,
                                    1 + (f1 < E2 ? fexp1[f1] : 0) - XBETA * (XS + 1), nullptr);
                    const int n1 = E2 - 16 * (warp & 3);  // real features of this warp's quarter
                    static_assert(XQB == 4, "the sparse-quarter path maps 4 features x 8 rows to the lanes");
                    if (n1 > 0 && n1 <= 4) {
                        // at most 4 real features: one (feature, row) item per lane -- feature L / 8 of
                        // the quarter, row (L / 4) % 2 lane-half, row L % 4 of the warp's block
                        const int fi = lane >> 3, hf = (lane >> 2) & 1, j = lane & 3;
                        double ys = 0.0;
#pragma unroll
                        for (int k = 0; k < XQB; ++k) {
                            const double a = __shfl_sync(0xffffffffu, y1[k], fi + 16 * hf);
                            if (k == j) ys = a;
                        }
                        if (fi < n1) {
                            const int fq = 16 * (warp & 3) + fi, row = 16 * hf + XQB * (warp >> 2) + j;
                            const int os = fq < E1 ? fq : fq - E1;
                            H1[row * LD1 + fq] = H0[row * LD0 + os] + dp_tanh64(ys + b1s[fq], m.tanh_tab);
                        }
                    } else if (f1 < E2) {
                        const double bb = b1s[f1];
                        const int os = f1 < E1 ? f1 : f1 - E1;
#pragma unroll
                        for (int j = 0; j < XQB; ++j) {
                            const int row = r0 + j;
                            H1[row * LD1 + f1] = H0[row * LD0 + os] + dp_tanh64(y1[j] + bb, m.tanh_tab);
                        }
                    }
                    tc::fence_before_sync();
                } else {
                    const double *hr = H0 + lane * LD0;
                    for (int o = warp; o < E2; o += XTB / 32) {
                        double z = b1s[o];
#pragma unroll 5
                        for (int q = 0; q < E1; ++q) z = fma(hr[q], W1s[q * E2 + o], z);
                        H1[lane * LD1 + o] = hr[o < E1 ? o : o - E1] + dp_tanh64(z, m.tanh_tab);
                    }
                }
                __syncthreads();
                // digits of h1 (fixed scale: |h1| < 2), 8 columns per thread-iteration
                for (int p = tid; p < XNR * (K2p / 8); p += XTB) {
                    const int row = p % XNR, k0 = (p / XNR) * 8;  // lanes on consecutive rows
                    long long I[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const double v = (k0 + q < E2) ? H1[row * LD1 + k0 + q] : 0.0;
                        I[q] = oz_rint_pow2(v, 55);  // round(v 2^55)
                    }
                    const uint32_t ofs = tc::kmajor_offset(row, k0, K2p);
                    for (int sd = XS - 1; sd >= 0; --sd) {
                        int dg[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) dg[q] = sd > 0 ? oz_digit_step(I[q], XBETA) : (int)I[q];
                        uint4 u;
                        u.x = (uint32_t)oz_bf16_int(dg[0]) | ((uint32_t)oz_bf16_int(dg[1]) << 16);
                        u.y = (uint32_t)oz_bf16_int(dg[2]) | ((uint32_t)oz_bf16_int(dg[3]) << 16);
                        u.z = (uint32_t)oz_bf16_int(dg[4]) | ((uint32_t)oz_bf16_int(dg[5]) << 16);
                        u.w = (uint32_t)oz_bf16_int(dg[6]) | ((uint32_t)oz_bf16_int(dg[7]) << 16);
                        *reinterpret_cast<uint4 *>(Bd + (size_t)sd * XNR * K2p * 2 + ofs) = u;
                    }
                }
                tc::fence_proxy_async();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
                // z2^T (128 features x 32 rows) = W2^T digits x h1 digits, group g at columns (g - 2) * 32
                if (tid == 0) {
                    const uint32_t wa = tc::smem_u32(Wd), ba = tc::smem_u32(Bd);
#pragma unroll
                    for (int s = 1; s <= XS; ++s) {
#pragma unroll
                        for (int t = 1; t + s <= XS + 1; ++t) {
#pragma unroll
                            for (int kk = 0; kk < K2p / 16; ++kk) {
                                const uint64_t ad = tc::make_desc(wa + (uint32_t)(s - 1) * XM * K2p * 2 + kk * 256, 128,
                                                                  K2p * 16);
                                const uint64_t bd = tc::make_desc(ba + (uint32_t)(t - 1) * XNR * K2p * 2 + kk * 256, 128,
                                                                  K2p * 16);
                                tc::mma_bf16(tbase + (uint32_t)(s + t - 2) * XNR, ad, bd, idesc, s > 1 || kk > 0);
                            }
                        }
                    }
                    tc::mma_commit(&mbar_m);
                }
                {
                    const bool ok = tc::mbar_wait(&mbar_m, ph_m);
                    ph_m ^= 1u;
                    const bool bad = __syncthreads_or(!ok);
                    tc::fence_after_sync();
                    if (bad) {
                        if (tid == 0) atomicOr(status, DPF_MMA_TIMEOUT);
                        alive = false;
                        pend_m = true;
                        break;
                    }
                }
                // epilogue: feature f of rows XRB grp .. XRB grp + XRB - 1 of the chunk
                double y[XRB];
                combine_groups_8(tlane + XRB * grp, y, cexp, nullptr);
                const int nq = E3 - 32 * (warp & 3);  // real features of this warp's TMEM quarter
                static_assert(XRB == 8, "the sparse-quarter path maps 4 features x 8 rows to the lanes");
                if (nq > 0 && nq <= 32 / XRB) {
                    // a quarter with at most 4 real features: one (feature, row) item per lane (feature
                    // L / 8 of the quarter, row L % 8), so the FP64 work runs once, not once per row
                    const int fi = lane >> 3, r = lane & 7;
                    double ys = 0.0;
#pragma unroll
                    for (int k = 0; k < XRB; ++k) {
                        const double a = __shfl_sync(0xffffffffu, y[k], fi);
                        if (k == r) ys = a;
                    }
                    const int fq = 32 * (warp & 3) + fi, q = XRB * grp + r;
                    double pc[4] = {0.0, 0.0, 0.0, 0.0};
                    if (fi < nq && q < nv) {
                        const int fsq = fq < E2 ? fq : fq - E2;
                        const double G = H1[q * LD1 + fsq] + dp_tanh64(ys + b2s[fq], m.tanh_tab);
#pragma unroll
                        for (int c = 0; c < 4; ++c) pc[c] = Rt[q * 4 + c] * G;
                    }
                    // sum over the 8 rows (lanes 8 fi .. 8 fi + 7), then lane fi, which holds the
                    // T column of feature fq, adds it
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                        for (int c = 0; c < 4; ++c) pc[c] += __shfl_xor_sync(0xffffffffu, pc[c], o);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const double v = __shfl_sync(0xffffffffu, pc[c], 8 * (lane & 3));
                        if (lane < nq) tacc[c] += v;
                    }
                } else if (f < E3) {
                    const double bf = b2s[f];
                    const int fs = f < E2 ? f : f - E2;
#pragma unroll
                    for (int qq = 0; qq < XRB; ++qq) {
                        const int q = XRB * grp + qq;
                        if (q < nv) {
                            const double z = y[qq] + bf;
                            const double G = H1[q * LD1 + fs] + dp_tanh64(z, m.tanh_tab);
#pragma unroll
                            for (int c = 0; c < 4; ++c) tacc[c] = fma(Rt[q * 4 + c], G, tacc[c]);
                        }
                    }
                }
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
            }
        }
        if (!alive) break;
        // T (the four row groups' partials summed in group order, scaled) and D = T_<^T T
        if (grp > 0 && f < E3) {
#pragma unroll
            for (int c = 0; c < 4; ++c) Tsm[4 * XM * grp + c * E3 + f] = tacc[c];
        }
        __syncthreads();
        if (grp == 0 && f < E3) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                double v = tacc[c];
#pragma unroll
                for (int g = 1; g < XTB / XM; ++g) v += Tsm[4 * XM * g + c * E3 + f];
                v *= m.desc_scale;
                Tsm[c * E3 + f] = v;
                Tout[(size_t)i * 4 * E3 + c * E3 + f] = v;
            }
        }
        __syncthreads();
        const int nd = m.m2 * E3;
        for (int q = tid; q < nd; q += XTB) {
            const int a2 = q / E3, b2 = q - a2 * E3;
            double acc = Tsm[a2] * Tsm[b2];
            acc = fma(Tsm[E3 + a2], Tsm[E3 + b2], acc);
            acc = fma(Tsm[2 * E3 + a2], Tsm[2 * E3 + b2], acc);
            acc = fma(Tsm[3 * E3 + a2], Tsm[3 * E3 + b2], acc);
            Dout[(size_t)i * nd + q] = acc;
        }
        __syncthreads();
    }
    // after a timeout: once more (bounded) for the copy or the MMAs still in flight
    if (pend_w) tc::mbar_wait(&mbar_w, ph_w ^ 1u);
    if (pend_m) tc::mbar_wait(&mbar_m, ph_m ^ 1u);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

template <int E1>
cudaError_t launch_fwd_x(cudaStream_t st, const DevModel &m, const unsigned char *wx, const double *x,
                         const int32_t *types, Box3 box, int N, const FormatBuffers &fb, const NlistBuffers &nb,
                         EvalBuffers eb, int num_sms, int32_t *status)
{
    using X = XShape<E1>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e =
            cudaFuncSetAttribute(k_embed_fwd_x<E1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X::SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    int grid = num_sms;
    if (grid > N) grid = N;
    if (grid < 1) grid = 1;
    k_embed_fwd_x<E1><<<grid, XTB, X::SMEM, st>>>(m, wx, x, types, box, N, nb.type_perm, fb.nlist, fb.nreal, eb.T,
                                                 eb.D, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- backward --
//
// k_embed_bwd_x recomputes G and its s-tangent dG/ds (G is never stored) with
// the same split: layer 0 and its tangent on the FP64 units; layer 1's
// products z1 = h0 W1 and dz1 = dh0 W1 and the last layer's z2 = h1 W2 and
// dz2 = dh1 W2 on the tensor cores (values with the fixed scale 2^1, tangents
// with a per-row power-of-two scale; a value and its tangent land in separate
// tensor-memory columns).  In the last
// layer's epilogue thread f forms G[f] and dG[f] of its rows and the partials
// G gT[c][f], dG gT[c][f]; a warp shuffle tree sums them over its 32 features,
// the four warps' sums are added in fixed order, and warp 0 (one lane per row)
// applies the chain rule through R~(r_ij) as k_embed_bwd does: pair gradients,
// the atom's own force and virial parts.

template <int E1>
struct XBShape {
    static constexpr int E2 = 2 * E1, E3 = 4 * E1, K2p = k2p_of(E1), K1p = k1p_of(E1);
    static constexpr bool L1 = l1bwd_of(E1);  // layer 1 on the tensor cores
    // odd row strides (in doubles): one row per lane reads without bank conflicts
    static constexpr int LD0 = (E1 % 2) ? E1 + 2 : E1 + 1, LD1 = (E2 % 2) ? E2 + 2 : E2 + 1;
    static constexpr int GR = 64;  // rows whose geometry is staged at once
    static constexpr int GS = 11;  // doubles per staged row
    // weight digits + exponents copied: the last layer's, and layer 1's (L1)
    static constexpr size_t WD = w2_bytes(E1) + (L1 ? w1_bytes(E1) : 0);
    static constexpr size_t NB = net_bytes(E1);
    static constexpr size_t BD = (size_t)XS * XNR * K2p * 2;
    // FP64: W1 (SIMT layer 1 only), w0, b0, b1, b2, H0, dH0 (aliased by the reduction
    // buffer), H1, dH1 (aliased by gT [4][XM] in each atom's prologue), geometry [GR][GS]
    // (10 values, odd stride)
    static constexpr size_t H0SZ = (size_t)2 * XNR * LD0;
    static constexpr size_t RED = (size_t)(XTB / 32) * XRB * 8;
    static constexpr size_t F64 = (L1 ? 0 : (size_t)E1 * E2) + 2 * E1 + E2 + XM + (H0SZ > RED ? H0SZ : RED) +
                                  2 * XNR * LD1 + GR * GS;
    static_assert(4 * XM <= XNR * LD1 && 4 * E3 <= XNR * LD1, "T and gT fit in the h1 and dh1 rows");
    // + two [XNR] int32 row exponents (layer 2's and layer 1's tangent rows)
    static constexpr size_t SMEM = WD + BD + F64 * 8 + 2 * XNR * 4;
    static_assert(GR % XNR == 0 && GR <= XTB, "geometry is staged one row per thread, whole chunks at a time");
    static_assert(!L1 || (2 * XS * XNR * K1p * 2 <= BD && E2 <= XM1),
                  "layer 1's value and tangent digits share the row-digit buffer");
    static_assert(SMEM + 1024 <= 232448, "dynamic plus static shared memory above the 227 KB opt-in limit");
};

// TAN = false: the backward (k_embed_bwd_x).  TAN = true: the forward with the
// s-tangent (k_embed_tan_x): the same value and tangent products, but instead of
// contracting G and dG/ds with dE/dT (not known yet) the epilogue stores both
// rows in HBM (Gst: [N nm][2 M], slot i nm + sel_off[b] + r, G then dG/ds) and
// accumulates T = R~^T G; the atom's T and D = T_<^T T leave as in k_embed_fwd_x.
template <int E1, bool TAN>
__device__ __forceinline__ void embed_tangent_body(const DevModel &m, const unsigned char *__restrict__ wx,
                                                   const double *__restrict__ x,
                                                   const int32_t *__restrict__ types, Box3 box, int N,
                                                   const int32_t *__restrict__ type_perm,
                                                   const int32_t *__restrict__ nlist,
                                                   const int32_t *__restrict__ nreal, double *__restrict__ Tio,
                                                   const double *__restrict__ gD, double *__restrict__ pair_g,
                                                   double *__restrict__ f_own, double *__restrict__ vir_part,
                                                   double *__restrict__ Dout, double *__restrict__ Gst,
                                                   int32_t *status)
{
    using X = XBShape<E1>;
    constexpr int E2 = X::E2, E3 = X::E3, K2p = X::K2p, K1p = X::K1p, LD0 = X::LD0, LD1 = X::LD1, GR = X::GR,
                  GS = X::GS;
    constexpr bool L1 = X::L1;
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *Wd = smraw;
    const int *fexp = reinterpret_cast<const int *>(Wd + (size_t)XS * XM * K2p * 2);
    unsigned char *Wd1 = Wd + w2_bytes(E1);  // layer 1's weight digits (L1)
    const int *fexp1 = reinterpret_cast<const int *>(Wd1 + (size_t)XS * XM1 * K1p * 2);
    unsigned char *Bd = Wd + X::WD;
    double *W1s = reinterpret_cast<double *>(Bd + X::BD);  // SIMT layer 1 only
    double *w0s = W1s + (L1 ? 0 : E1 * E2);
    double *b0s = w0s + E1;
    double *b1s = b0s + E1;
    double *b2s = b1s + E2;
    double *H0 = b2s + XM;
    double *dH0 = H0 + XNR * LD0;
    double *red = H0;  // [16 warps][8 rows][8], used after layer 1 (aliases H0, dH0)
    double *H1 = H0 + (X::H0SZ > X::RED ? X::H0SZ : X::RED);
    double *dH1 = H1 + XNR * LD1;
    double *geo = dH1 + XNR * LD1;  // [GR][GS]: s, ds, R[4], d[3], r
    // gT [4][XM] of the atom: written and read into registers in the atom's prologue,
    // before the first chunk writes dh1
    double *gTs = dH1;
    int *erow = reinterpret_cast<int *>(geo + GR * GS);  // [XNR] tangent row exponents
    int *erow0 = erow + XNR;                            // [XNR] the same for layer 1's input (L1)
    __shared__ __align__(8) uint64_t mbar_w, mbar_m;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = m.ntypes, nm = m.nm, m2 = m.m2;

    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    if (tid == 0) {
        tc::mbar_init(&mbar_w, 1);
        tc::mbar_init(&mbar_m, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tslot;
    const uint32_t tlane = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t idesc = tc::make_idesc_bf16(XM, XNR);
    uint32_t ph_w = 0, ph_m = 0;
    bool alive = true, pend_w = false, pend_m = false;
    int staged = -1;
    const int f = tid & (XM - 1);
    const int grp = tid >> 7;  // last layer: rows XRB grp .. XRB grp + XRB - 1

    // z^T = W2^T digits x (row digits in Bd) into 7 groups at column base col0
    auto mma_rows = [&](uint32_t col0) -> bool {
        if (tid == 0) {
            const uint32_t wa = tc::smem_u32(Wd), ba = tc::smem_u32(Bd);
#pragma unroll
            for (int s = 1; s <= XS; ++s)
#pragma unroll
                for (int t = 1; t + s <= XS + 1; ++t)
#pragma unroll
                    for (int kk = 0; kk < K2p / 16; ++kk)
                        tc::mma_bf16(tbase + col0 + (uint32_t)(s + t - 2) * XNR,
                                     tc::make_desc(wa + (uint32_t)(s - 1) * XM * K2p * 2 + kk * 256, 128, K2p * 16),
                                     tc::make_desc(ba + (uint32_t)(t - 1) * XNR * K2p * 2 + kk * 256, 128, K2p * 16),
                                     idesc, s > 1 || kk > 0);
            tc::mma_commit(&mbar_m);
        }
        const bool ok = tc::mbar_wait(&mbar_m, ph_m);
        ph_m ^= 1u;
        const bool bad = __syncthreads_or(!ok);
        tc::fence_after_sync();
        if (bad) {
            if (tid == 0) atomicOr(status, DPF_MMA_TIMEOUT);
            pend_m = true;
        }
        return !bad;
    };
    // digits of the 32 x E2 rows of src (row scale 2^(56 - e_r), e_r from erow or fixed)
    auto make_digits = [&](const double *src, bool fixed) {
        for (int p = tid; p < XNR * (K2p / 8); p += XTB) {
            const int row = p % XNR, k0 = (p / XNR) * 8;  // lanes on consecutive rows
            const int sk = XBETA * XS - (fixed ? 1 : erow[row]);  // round(v 2^sk)
            long long I[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) I[q] = (k0 + q < E2) ? oz_rint_pow2(src[row * LD1 + k0 + q], sk) : 0ll;
            const uint32_t ofs = tc::kmajor_offset(row, k0, K2p);
            for (int sd = XS - 1; sd >= 0; --sd) {
                int dg[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) dg[q] = sd > 0 ? oz_digit_step(I[q], XBETA) : (int)I[q];
                uint4 u;
                u.x = (uint32_t)oz_bf16_int(dg[0]) | ((uint32_t)oz_bf16_int(dg[1]) << 16);
                u.y = (uint32_t)oz_bf16_int(dg[2]) | ((uint32_t)oz_bf16_int(dg[3]) << 16);
                u.z = (uint32_t)oz_bf16_int(dg[4]) | ((uint32_t)oz_bf16_int(dg[5]) << 16);
                u.w = (uint32_t)oz_bf16_int(dg[6]) | ((uint32_t)oz_bf16_int(dg[7]) << 16);
                *reinterpret_cast<uint4 *>(Bd + (size_t)sd * XNR * K2p * 2 + ofs) = u;
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    };
    // layer 1: digits of the 32 x E1 rows of H0 (fixed scale 2^55) at Bd and of dH0
    // (row scale 2^(56 - erow0)) after them
    auto make_digits1 = [&]() {
        constexpr int NP = XNR * (K1p / 8);
        for (int p = tid; p < 2 * NP; p += XTB) {
            const int which = p / NP, pp = p - which * NP;
            const int row = pp % XNR, k0 = (pp / XNR) * 8;
            const double *src = which ? dH0 : H0;
            const int sk = XBETA * XS - (which ? erow0[row] : 1);  // round(v 2^sk)
            long long I[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) I[q] = (k0 + q < E1) ? oz_rint_pow2(src[row * LD0 + k0 + q], sk) : 0ll;
            const uint32_t ofs = tc::kmajor_offset(row, k0, K1p);
            unsigned char *dst = Bd + (size_t)which * XS * XNR * K1p * 2;
            for (int sd = XS - 1; sd >= 0; --sd) {
                int dg[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) dg[q] = sd > 0 ? oz_digit_step(I[q], XBETA) : (int)I[q];
                uint4 u;
                u.x = (uint32_t)oz_bf16_int(dg[0]) | ((uint32_t)oz_bf16_int(dg[1]) << 16);
                u.y = (uint32_t)oz_bf16_int(dg[2]) | ((uint32_t)oz_bf16_int(dg[3]) << 16);
                u.z = (uint32_t)oz_bf16_int(dg[4]) | ((uint32_t)oz_bf16_int(dg[5]) << 16);
                u.w = (uint32_t)oz_bf16_int(dg[6]) | ((uint32_t)oz_bf16_int(dg[7]) << 16);
                *reinterpret_cast<uint4 *>(dst + (size_t)sd * XNR * K1p * 2 + ofs) = u;
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    };
    // z1^T = W1^T digits x row digits (M = 64): value into 7 groups at column 0,
    // tangent at column 256
    auto mma_l1 = [&]() -> bool {
        if (tid == 0) {
            const uint32_t wa = tc::smem_u32(Wd1), ba = tc::smem_u32(Bd);
            const uint32_t idesc1 = tc::make_idesc_bf16(XM1, XNR);
#pragma unroll
            for (int v = 0; v < 2; ++v)
#pragma unroll
                for (int s = 1; s <= XS; ++s)
#pragma unroll
                    for (int t = 1; t + s <= XS + 1; ++t)
#pragma unroll
                        for (int kk = 0; kk < K1p / 16; ++kk)
                            tc::mma_bf16(
                                tbase + (uint32_t)v * 256 + (uint32_t)(s + t - 2) * XNR,
                                tc::make_desc(wa + (uint32_t)(s - 1) * XM1 * K1p * 2 + kk * 256, 128, K1p * 16),
                                tc::make_desc(ba + (uint32_t)(v * XS + t - 1) * XNR * K1p * 2 + kk * 256, 128,
                                              K1p * 16),
                                idesc1, s > 1 || kk > 0);
            tc::mma_commit(&mbar_m);
        }
        const bool ok = tc::mbar_wait(&mbar_m, ph_m);
        ph_m ^= 1u;
        const bool bad = __syncthreads_or(!ok);
        tc::fence_after_sync();
        if (bad) {
            if (tid == 0) atomicOr(status, DPF_MMA_TIMEOUT);
            pend_m = true;
        }
        return !bad;
    };

    for (int ii = blockIdx.x; ii < N && alive; ii += gridDim.x) {
        const int i = type_perm[ii];
        const int a = types[i];
        const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        // gT[c][x] = scale ([x < M2] sum_b gD[x][b] T[c][b] + sum_{a<M2} gD[a][x] T[c][a])
        if constexpr (!TAN) {
            double *Ts = H1;  // T of this atom, [4][E3]
            for (int p = tid; p < 4 * E3; p += XTB) Ts[p] = Tio[(size_t)i * 4 * E3 + p];
            __syncthreads();
            const double *g = gD + (size_t)i * m2 * E3;
            for (int p = tid; p < 4 * E3; p += XTB) {
                const int cc = p / E3, xx = p - cc * E3;
                double acc = 0.0;
                if (xx < m2)
                    for (int b2 = 0; b2 < E3; ++b2) acc = fma(g[xx * E3 + b2], Ts[cc * E3 + b2], acc);
                for (int a2 = 0; a2 < m2; ++a2) acc = fma(g[a2 * E3 + xx], Ts[cc * E3 + a2], acc);
                gTs[cc * XM + xx] = acc * m.desc_scale;
            }
            __syncthreads();
        }
        double gt[4] = {0.0, 0.0, 0.0, 0.0}, gtp[4] = {0.0, 0.0, 0.0, 0.0};  // dE/dT of this thread's
                                                                            // feature, and of lane ^ 16's
        if constexpr (!TAN) {
#pragma unroll
            for (int c = 0; c < 4; ++c) gt[c] = f < E3 ? gTs[c * XM + f] : 0.0;
#pragma unroll
            for (int c = 0; c < 4; ++c) gtp[c] = __shfl_xor_sync(0xffffffffu, gt[c], 16);
        }
        double tacc[4] = {0.0, 0.0, 0.0, 0.0};  // TAN: this thread's column of T over its rows
        double fo[3] = {0.0, 0.0, 0.0}, vir[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) vir[q] = 0.0;

        const bool a_ok = (unsigned)a < (unsigned)T;
        for (int b = 0; b < T && alive; ++b) {
            const int nb = a_ok ? nreal[(size_t)i * T + b] : 0;
            if (nb == 0) continue;
            const int net = a * T + b;
            if (net != staged) {
                __syncthreads();
                if (tid == 0) {
                    mbar_expect_tx_x(&mbar_w, (uint32_t)X::WD);
                    bulk_g2s_x(Wd, wx + (size_t)net * X::NB, (uint32_t)X::WD, &mbar_w);
                }
                const double *src = m.params + m.emb_base[net];
                for (int q = tid; q < E1; q += XTB) {
                    w0s[q] = src[q];
                    b0s[q] = src[E1 + q];
                }
                if constexpr (!L1)
                    for (int q = tid; q < E1 * E2; q += XTB) W1s[q] = src[2 * E1 + q];
                for (int q = tid; q < E2; q += XTB) b1s[q] = src[2 * E1 + E1 * E2 + q];
                for (int q = tid; q < XM; q += XTB)
                    b2s[q] = q < E3 ? src[2 * E1 + E1 * E2 + E2 + E2 * E3 + q] : 0.0;
                const bool ok = tc::mbar_wait(&mbar_w, ph_w);
                ph_w ^= 1u;
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) atomicOr(status, DPF_MMA_TIMEOUT);
                    alive = false;
                    pend_w = true;
                    break;
                }
                staged = net;
            }
            const int fx = f < E3 ? fexp[f] : 0;
            for (int c0 = 0; c0 < nb && alive; c0 += XNR) {
                const int nv = min(XNR, nb - c0);
                if (c0 % GR == 0) {
                    __syncthreads();
                    for (int q = tid; q < GR; q += XTB) {
                        const int r = c0 + q;
                        double *gq = geo + q * GS;
                        double s = 0.0, ds = 0.0, d[3] = {0.0, 0.0, 0.0}, rr = 1.0;
                        if (r < nb) {
                            const int j = nlist[(size_t)i * nm + m.sel_off[b] + r];
                            const double xj[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
                            rr = dp_pinned_dist(xi, xj, box, d);
                            dp_switch(rr, m.rcut_smth, m.rcut, s, ds);
                        }
                        const double inv = 1.0 / rr;
                        gq[0] = s;
                        gq[1] = ds;
                        gq[2] = s;
                        gq[3] = s * d[0] * inv;
                        gq[4] = s * d[1] * inv;
                        gq[5] = s * d[2] * inv;
                        gq[6] = d[0];
                        gq[7] = d[1];
                        gq[8] = d[2];
                        gq[9] = rr;
                    }
                }
                const double *gc = geo + (c0 % GR) * GS;  // this chunk's rows
                __syncthreads();
                // layer 0 and its tangent
                {
                    const double sv = gc[lane * GS];
                    for (int o = warp; o < E1; o += XTB / 32) {
                        const double w0 = w0s[o];
                        const double t = dp_tanh64(fma(sv, w0, b0s[o]), m.tanh_tab);
                        H0[lane * LD0 + o] = t;
                        dH0[lane * LD0 + o] = fma(-t, t, 1.0) * w0;
                    }
                }
                __syncthreads();
                // layer 1 and its tangent
                if constexpr (L1) {
                    // tangent row exponents of layer 1's input: 2^e > max_k |dh0[row][k]|
                    {
                        const int row = tid >> 3, part = tid & 7;
                        double mx = 0.0;
                        if (row < XNR)
                            for (int k = part; k < E1; k += 8) mx = fmax(mx, fabs(dH0[row * LD0 + k]));
#pragma unroll
                        for (int o = 4; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                        if (row < XNR && part == 0) {
                            int e = 0;
                            if (mx > 0.0) {
                                frexp(mx, &e);
                                e = max(e, -900);
                            }
                            erow0[row] = e;
                        }
                    }
                    __syncthreads();
                    make_digits1();
                    if (!mma_l1()) {
                        alive = false;
                        break;
                    }
                    // epilogue: the warp's TMEM quarter holds features 16 (warp % 4) .. + 15 in
                    // its first 16 lanes; lanes < 16 take rows 0..15, the others rows 16..31,
                    // and warps w, w + 4, w + 8, w + 12 take 4 of them each
                    const int f1 = 16 * (warp & 3) + (lane & 15);
                    const int r0 = 16 * (lane >> 4) + XQB * (warp >> 2);
                    const uint32_t ta = tlane + XQB * (uint32_t)(warp >> 2);
                    const int fx1 = f1 < E2 ? fexp1[f1] : 0;
                    double y1[XQB], dy1[XQB];
                    combine_groups4(ta, y1, 1 + fx1 - XBETA * (XS + 1), nullptr);
                    combine_groups4(ta + 256, dy1, fx1 - XBETA * (XS + 1), erow0 + r0);
                    const int n1 = E2 - 16 * (warp & 3);  // real features of this warp's quarter
                    static_assert(XQB == 4, "the sparse-quarter path maps 4 features x 8 rows to the lanes");
                    if (n1 > 0 && n1 <= 4) {
                        // at most 4 real features: one (feature, row) item per lane (as in the forward)
                        const int fi = lane >> 3, hf = (lane >> 2) & 1, j = lane & 3;
                        double ys = 0.0, dzs = 0.0;
#pragma unroll
                        for (int k = 0; k < XQB; ++k) {
                            const double a = __shfl_sync(0xffffffffu, y1[k], fi + 16 * hf);
                            const double b = __shfl_sync(0xffffffffu, dy1[k], fi + 16 * hf);
                            if (k == j) {
                                ys = a;
                                dzs = b;
                            }
                        }
                        if (fi < n1) {
                            const int fq = 16 * (warp & 3) + fi, row = 16 * hf + XQB * (warp >> 2) + j;
                            const int os = fq < E1 ? fq : fq - E1;
                            const double t = dp_tanh64(ys + b1s[fq], m.tanh_tab);
                            H1[row * LD1 + fq] = H0[row * LD0 + os] + t;
                            dH1[row * LD1 + fq] = fma(fma(-t, t, 1.0), dzs, dH0[row * LD0 + os]);
                        }
                    } else if (f1 < E2) {
                        const double bb = b1s[f1];
                        const int os = f1 < E1 ? f1 : f1 - E1;
#pragma unroll
                        for (int j = 0; j < XQB; ++j) {
                            const int row = r0 + j;
                            const double t = dp_tanh64(y1[j] + bb, m.tanh_tab);
                            const double dz = dy1[j];
                            H1[row * LD1 + f1] = H0[row * LD0 + os] + t;
                            dH1[row * LD1 + f1] = fma(fma(-t, t, 1.0), dz, dH0[row * LD0 + os]);
                        }
                    }
                    tc::fence_before_sync();
                } else {
                    const double *hr = H0 + lane * LD0, *dhr = dH0 + lane * LD0;
                    for (int o = warp; o < E2; o += XTB / 32) {
                        double z = b1s[o], dz = 0.0;
#pragma unroll 5
                        for (int q = 0; q < E1; ++q) {
                            const double w = W1s[q * E2 + o];
                            z = fma(hr[q], w, z);
                            dz = fma(dhr[q], w, dz);
                        }
                        const double t = dp_tanh64(z, m.tanh_tab);
                        const int os = o < E1 ? o : o - E1;
                        H1[lane * LD1 + o] = hr[os] + t;
                        dH1[lane * LD1 + o] = fma(fma(-t, t, 1.0), dz, dhr[os]);
                    }
                }
                __syncthreads();
                // tangent row exponents: 2^e > max_k |dh1[row][k]| (one warp per 8 rows, 4 lanes per row)
                {
                    const int row = tid >> 3, part = tid & 7;
                    double mx = 0.0;
                    if (row < XNR)
                        for (int k = part; k < E2; k += 8) mx = fmax(mx, fabs(dH1[row * LD1 + k]));
#pragma unroll
                    for (int o = 4; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                    if (row < XNR && part == 0) {
                        // 2^e > max |dh1| (e >= -900 keeps every scale below a normal number; a zero row takes 0)
                        int e = 0;
                        if (mx > 0.0) {
                            frexp(mx, &e);
                            e = max(e, -900);
                        }
                        erow[row] = e;
                    }
                }
                // value then tangent products, digits through the same buffer
                make_digits(H1, true);
                if (!mma_rows(0)) {
                    alive = false;
                    break;
                }
                make_digits(dH1, false);
                if (!mma_rows(256)) {
                    alive = false;
                    break;
                }
                // epilogue: feature f of rows XRB grp .. XRB grp + XRB - 1
                double yv[XRB], yt[XRB];
                combine_groups_8(tlane + XRB * grp, yv, 1 + fx - XBETA * (XS + 1), nullptr);
                combine_groups_8(tlane + 256 + XRB * grp, yt, fx - XBETA * (XS + 1), erow + XRB * grp);
                const double bf = f < E3 ? b2s[f] : 0.0;
                const int fs = f < E2 ? f : (f < E3 ? f - E2 : 0);
                if constexpr (TAN) {
                // G and dG/ds of the chunk's rows to HBM, this thread's column of T over its rows
                double *gro = Gst + ((size_t)i * nm + m.sel_off[b] + c0) * (2 * E3);
                const int nq = E3 - 32 * (warp & 3);  // real features of this warp's TMEM quarter
                static_assert(XRB == 8, "the sparse-quarter path maps 4 features x 8 rows to the lanes");
                if (nq > 0 && nq <= 32 / XRB) {
                    // at most 4 real features: one (feature, row) item per lane (feature L / 8 of the
                    // quarter, row L % 8), as in the backward
                    const int fi = lane >> 3, r = lane & 7;
                    double ys = 0.0, ts = 0.0;
#pragma unroll
                    for (int k = 0; k < XRB; ++k) {
                        const double a = __shfl_sync(0xffffffffu, yv[k], fi);
                        const double b = __shfl_sync(0xffffffffu, yt[k], fi);
                        if (k == r) {
                            ys = a;
                            ts = b;
                        }
                    }
                    const int fq = 32 * (warp & 3) + fi, q = XRB * grp + r;
                    double pc[4] = {0.0, 0.0, 0.0, 0.0};
                    if (fi < nq && q < nv) {
                        const int fsq = fq < E2 ? fq : fq - E2;
                        const double t = dp_tanh64(ys + b2s[fq], m.tanh_tab);
                        const double G = H1[q * LD1 + fsq] + t;
                        const double dG = fma(fma(-t, t, 1.0), ts, dH1[q * LD1 + fsq]);
                        gro[(size_t)q * (2 * E3) + fq] = G;
                        gro[(size_t)q * (2 * E3) + E3 + fq] = dG;
#pragma unroll
                        for (int c = 0; c < 4; ++c) pc[c] = gc[q * GS + 2 + c] * G;
                    }
                    // sum over the 8 rows (lanes 8 fi .. 8 fi + 7); lane fi, which owns feature fq's
                    // column of T, adds it
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                        for (int c = 0; c < 4; ++c) pc[c] += __shfl_xor_sync(0xffffffffu, pc[c], o);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const double v = __shfl_sync(0xffffffffu, pc[c], 8 * (lane & 3));
                        if (lane < nq) tacc[c] += v;
                    }
                } else if (nq > 0 && f < E3) {
#pragma unroll
                    for (int qq = 0; qq < XRB; ++qq) {
                        const int q = XRB * grp + qq;
                        if (q < nv) {
                            const double t = dp_tanh64(yv[qq] + bf, m.tanh_tab);
                            const double G = H1[q * LD1 + fs] + t;
                            const double dG = fma(fma(-t, t, 1.0), yt[qq], dH1[q * LD1 + fs]);
                            gro[(size_t)q * (2 * E3) + f] = G;
                            gro[(size_t)q * (2 * E3) + E3 + f] = dG;
#pragma unroll
                            for (int c = 0; c < 4; ++c) tacc[c] = fma(gc[q * GS + 2 + c], G, tacc[c]);
                        }
                    }
                }
                } else {
                double *rw = red + (warp * XRB) * 8;  // this warp's [XRB rows][8]
                const int nq = E3 - 32 * (warp & 3);  // real features of this warp's TMEM quarter
                static_assert(XRB == 8, "the sparse-quarter path maps 4 features x 8 rows to the lanes");
                if (nq <= 0) {
                    // padding only: zero partials
                    rw[lane] = 0.0;
                    rw[32 + lane] = 0.0;
                } else if (nq <= 32 / XRB) {
                    // a quarter with at most 4 real features (e.g. 96..99 of 100): its 4 x 8 (feature,
                    // row) items go one per lane, so the FP64 work runs once instead of once per row on
                    // mostly idle lanes; lane L takes feature L / 8 of the quarter and row L % 8
                    const int fi = lane >> 3, r = lane & 7;
                    double ys = 0.0, ts = 0.0;
#pragma unroll
                    for (int k = 0; k < XRB; ++k) {
                        const double a = __shfl_sync(0xffffffffu, yv[k], fi);
                        const double b = __shfl_sync(0xffffffffu, yt[k], fi);
                        if (k == r) {
                            ys = a;
                            ts = b;
                        }
                    }
                    double g4[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) g4[c] = __shfl_sync(0xffffffffu, gt[c], fi);
                    const int fq = 32 * (warp & 3) + fi, q = XRB * grp + r;
                    double p[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) p[c] = 0.0;
                    if (fi < nq && q < nv) {
                        const int fsq = fq < E2 ? fq : fq - E2;
                        const double t = dp_tanh64(ys + b2s[fq], m.tanh_tab);
                        const double G = H1[q * LD1 + fsq] + t;
                        const double dG = fma(fma(-t, t, 1.0), ts, dH1[q * LD1 + fsq]);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            p[c] = G * g4[c];
                            p[4 + c] = dG * g4[c];
                        }
                    }
                    // sum over the quarter's features (lanes r, r + 8, r + 16, r + 24)
#pragma unroll
                    for (int o = 8; o < 32; o <<= 1)
#pragma unroll
                        for (int c = 0; c < 8; ++c) p[c] += __shfl_xor_sync(0xffffffffu, p[c], o);
                    // lane L writes components 2 (L / 8) and 2 (L / 8) + 1 of row L % 8
                    double w0 = p[0], w1 = p[1];
                    if (fi == 1) {
                        w0 = p[2];
                        w1 = p[3];
                    } else if (fi == 2) {
                        w0 = p[4];
                        w1 = p[5];
                    } else if (fi == 3) {
                        w0 = p[6];
                        w1 = p[7];
                    }
                    rw[r * 8 + 2 * fi] = w0;
                    rw[r * 8 + 2 * fi + 1] = w1;
                } else {
                // partials p[r][c] = G gT[c] (c < 4), dG gT[c - 4] for 4 rows at a time, summed over
                // the warp's 32 features by a transposing shuffle tree (31 adds per lane): lane L ends
                // with the sum of row L / 8, component L % 8
#pragma unroll 1
                for (int q4 = 0; q4 < XRB; q4 += 4) {
                    double G[4], dG[4];
#pragma unroll
                    for (int r4 = 0; r4 < 4; ++r4) {
                        const int qq = q4 + r4, q = XRB * grp + qq;
                        G[r4] = 0.0;
                        dG[r4] = 0.0;
                        if (q < nv && f < E3) {
                            const double t = dp_tanh64(yv[qq] + bf, m.tanh_tab);
                            G[r4] = H1[q * LD1 + fs] + t;
                            const double dz2 = yt[qq];
                            dG[r4] = fma(fma(-t, t, 1.0), dz2, dH1[q * LD1 + fs]);
                        }
                    }
                    // first level of the tree on the factors: lanes below 16 keep rows 0, 1 of the four,
                    // the others rows 2, 3; each receives its partner's G and dG of its kept rows and
                    // forms both features' products itself (with the partner's dE/dT, gtp)
                    const bool hi16 = (lane & 16) != 0;
                    double p[16];
                    {
                        double kG[2], kD[2], rG[2], rD[2];
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            kG[r] = hi16 ? G[2 + r] : G[r];
                            kD[r] = hi16 ? dG[2 + r] : dG[r];
                            rG[r] = __shfl_xor_sync(0xffffffffu, hi16 ? G[r] : G[2 + r], 16);
                            rD[r] = __shfl_xor_sync(0xffffffffu, hi16 ? dG[r] : dG[2 + r], 16);
                        }
#pragma unroll
                        for (int r = 0; r < 2; ++r)
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                p[r * 8 + c] = fma(rG[r], gtp[c], kG[r] * gt[c]);
                                p[r * 8 + 4 + c] = fma(rD[r], gtp[c], kD[r] * gt[c]);
                            }
                    }
#pragma unroll
                    for (int w = 8, n = 8; w >= 1; w >>= 1, n >>= 1) {
                        const bool up = (lane & w) != 0;
#pragma unroll
                        for (int k = 0; k < n; ++k) {
                            const double send = up ? p[k] : p[n + k];
                            const double keep = up ? p[n + k] : p[k];
                            p[k] = keep + __shfl_xor_sync(0xffffffffu, send, w);
                        }
                    }
                    rw[(q4 + (lane >> 3)) * 8 + (lane & 7)] = p[0];
                }
                }
                __syncthreads();
                // chain rule through R~(r_ij), one lane per row (warp 0)
                if (warp == 0 && lane < nv) {
                    const int q = lane, hq = q / XRB, qq = q % XRB;
                    double sa[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) sa[c] = 0.0;
                    for (int w = 4 * hq; w < 4 * hq + 4; ++w)
#pragma unroll
                        for (int c = 0; c < 8; ++c) sa[c] += red[(w * XRB + qq) * 8 + c];
                    const double *gq = gc + q * GS;
                    const double gs = gq[0], gds = gq[1], gd[3] = {gq[6], gq[7], gq[8]}, gr = gq[9];
                    double gR0 = sa[0];
#pragma unroll
                    for (int c = 0; c < 4; ++c) gR0 = fma(gq[2 + c], sa[4 + c], gR0);
                    const double inv = 1.0 / gr;
                    const double u[3] = {gd[0] * inv, gd[1] * inv, gd[2] * inv};
                    const double dot = sa[1] * u[0] + sa[2] * u[1] + sa[3] * u[2];
                    const double sr = gs * inv;
                    const double coef = gR0 * gds + gds * dot - sr * dot;
                    double gv[3];
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) gv[bb] = fma(u[bb], coef, sr * sa[1 + bb]);
                    double *pg = pair_g + ((size_t)i * nm + m.sel_off[b] + c0 + q) * 3;
                    pg[0] = gv[0];
                    pg[1] = gv[1];
                    pg[2] = gv[2];
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa) {
                        fo[aa] += gv[aa];
#pragma unroll
                        for (int bb = 0; bb < 3; ++bb) vir[aa * 3 + bb] -= gd[aa] * gv[bb];
                    }
                }
                }
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
            }
        }
        if (!alive) break;
        if constexpr (TAN) {
            // T (the four row groups' partials summed in group order, scaled) and D = T_<^T T,
            // as k_embed_fwd_x; the partials go through the h1 / dh1 rows
            double *Tsm = H1;
            if (grp > 0 && f < E3) {
#pragma unroll
                for (int c = 0; c < 4; ++c) Tsm[4 * XM * grp + c * E3 + f] = tacc[c];
            }
            __syncthreads();
            if (grp == 0 && f < E3) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    double v = tacc[c];
#pragma unroll
                    for (int g = 1; g < XTB / XM; ++g) v += Tsm[4 * XM * g + c * E3 + f];
                    v *= m.desc_scale;
                    Tsm[c * E3 + f] = v;
                    Tio[(size_t)i * 4 * E3 + c * E3 + f] = v;
                }
            }
            __syncthreads();
            const int nd = m2 * E3;
            for (int q = tid; q < nd; q += XTB) {
                const int a2 = q / E3, b2 = q - a2 * E3;
                double acc = Tsm[a2] * Tsm[b2];
                acc = fma(Tsm[E3 + a2], Tsm[E3 + b2], acc);
                acc = fma(Tsm[2 * E3 + a2], Tsm[2 * E3 + b2], acc);
                acc = fma(Tsm[3 * E3 + a2], Tsm[3 * E3 + b2], acc);
                Dout[(size_t)i * nd + q] = acc;
            }
        } else if (warp == 0) {
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
        }
        __syncthreads();
    }
    if (pend_w) tc::mbar_wait(&mbar_w, ph_w ^ 1u);
    if (pend_m) tc::mbar_wait(&mbar_m, ph_m ^ 1u);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

template <int E1>
__global__ void __launch_bounds__(XTB, 1) k_embed_bwd_x(DevModel m, const unsigned char *__restrict__ wx,
                                                       const double *__restrict__ x,
                                                       const int32_t *__restrict__ types, Box3 box, int N,
                                                       const int32_t *__restrict__ type_perm,
                                                       const int32_t *__restrict__ nlist,
                                                       const int32_t *__restrict__ nreal, double *__restrict__ Tin,
                                                       const double *__restrict__ gD, double *__restrict__ pair_g,
                                                       double *__restrict__ f_own, double *__restrict__ vir_part,
                                                       int32_t *status)
{
    embed_tangent_body<E1, false>(m, wx, x, types, box, N, type_perm, nlist, nreal, Tin, gD, pair_g, f_own,
                                  vir_part, nullptr, nullptr, status);
}

template <int E1>
__global__ void __launch_bounds__(XTB, 1) k_embed_tan_x(DevModel m, const unsigned char *__restrict__ wx,
                                                       const double *__restrict__ x,
                                                       const int32_t *__restrict__ types, Box3 box, int N,
                                                       const int32_t *__restrict__ type_perm,
                                                       const int32_t *__restrict__ nlist,
                                                       const int32_t *__restrict__ nreal, double *__restrict__ Tout,
                                                       double *__restrict__ Dout, double *__restrict__ Gst,
                                                       int32_t *status)
{
    embed_tangent_body<E1, true>(m, wx, x, types, box, N, type_perm, nlist, nreal, Tout, nullptr, nullptr, nullptr,
                                 nullptr, Dout, Gst, status);
}

template <int E1, bool TAN>
cudaError_t launch_tangent_x(cudaStream_t st, const DevModel &m, const unsigned char *wx, const double *x,
                             const int32_t *types, Box3 box, int N, const FormatBuffers &fb, const NlistBuffers &nb,
                             EvalBuffers eb, int num_sms, int32_t *status)
{
    using X = XBShape<E1>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e;
        if constexpr (TAN)
            e = cudaFuncSetAttribute(k_embed_tan_x<E1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X::SMEM);
        else
            e = cudaFuncSetAttribute(k_embed_bwd_x<E1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X::SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    int grid = num_sms;
    if (grid > N) grid = N;
    if (grid < 1) grid = 1;
    if constexpr (TAN)
        k_embed_tan_x<E1><<<grid, XTB, X::SMEM, st>>>(m, wx, x, types, box, N, nb.type_perm, fb.nlist, fb.nreal,
                                                     eb.T, eb.D, eb.Gst, status);
    else
        k_embed_bwd_x<E1><<<grid, XTB, X::SMEM, st>>>(m, wx, x, types, box, N, nb.type_perm, fb.nlist, fb.nreal,
                                                     eb.T, eb.gD, eb.pair_g, eb.f_own, eb.vir_part, status);
    return cudaGetLastError();
}

// ------------------------------------------------------ streaming backward --
//
// k_embed_bwd_st: the backward once k_embed_tan_x has stored G and dG/ds of
// every real row, so nothing of the embedding net is recomputed.  One warp per
// atom: dE/dT of the atom (as k_embed_bwd_x computes it) into shared memory,
// then the atom's real rows (its type blocks one after the other) 32 at a
// time: lane q takes the geometry of row q; in 8 steps of 4 rows, 8 lanes per
// row form sa[c] = sum_f G[f] gT[c][f] and sa[4 + c] = sum_f dG[f] gT[c][f]
// (lane u of the 8 over the features u, u + 8, ...), summed over the 8 lanes by
// a transposing shuffle tree (7 adds; lane u ends with component u); lane q
// then applies the chain rule through R~(r_ij) to its row: pair gradient, and
// the atom's own force and virial parts.  Every sum runs in a fixed order: the
// results are bit-reproducible.
constexpr int STW = 4;  // warps (atoms in flight) per CTA

template <int E1>
__global__ void __launch_bounds__(STW * 32, 4) k_embed_bwd_st(DevModel m, const double *__restrict__ x,
                                                             const int32_t *__restrict__ types, Box3 box, int N,
                                                             const int32_t *__restrict__ nlist,
                                                             const int32_t *__restrict__ nreal,
                                                             const double *__restrict__ Tin,
                                                             const double *__restrict__ gD,
                                                             const double *__restrict__ Gst,
                                                             double *__restrict__ pair_g, double *__restrict__ f_own,
                                                             double *__restrict__ vir_part)
{
    constexpr int E3 = 4 * E1, KF = (E3 + 7) / 8;
    static_assert(4 * E3 >= 32 * 8, "the row sums [32][8] fit in the T buffer");
    __shared__ double Tsh[STW][4 * E3];  // T of the warp's atom, then the row sums [32][8]
    __shared__ double gTsh[STW][4 * E3];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int sub = lane & 7, gq = lane >> 3;
    const int T = m.ntypes, nm = m.nm, m2 = m.m2;
    double *Ts = Tsh[w], *sa_s = Tsh[w];
    double *gTw = gTsh[w];

    for (int i = blockIdx.x * STW + w; i < N; i += gridDim.x * STW) {
        const int a = types[i];
        const bool a_ok = (unsigned)a < (unsigned)T;
        // gT[c][x] = scale ([x < M2] sum_b gD[x][b] T[c][b] + sum_{a<M2} gD[a][x] T[c][a])
        for (int p = lane; p < 4 * E3; p += 32) Ts[p] = Tin[(size_t)i * 4 * E3 + p];
        __syncwarp();
        {
            // the 4 M2 long sums first, two per lane with every lane busy (two chains each), then
            // every entry's M2 short terms on top of them
            const double *g = gD + (size_t)i * m2 * E3;
            for (int p = lane; p < 4 * m2; p += 32) {
                const int cc = p / m2, xx = p - cc * m2;
                double acc = 0.0, acc2 = 0.0;
                for (int b2 = 0; b2 < E3; b2 += 2) {  // E3 = 4 e1 is even
                    acc = fma(g[xx * E3 + b2], Ts[cc * E3 + b2], acc);
                    acc2 = fma(g[xx * E3 + b2 + 1], Ts[cc * E3 + b2 + 1], acc2);
                }
                gTw[cc * E3 + xx] = acc + acc2;
            }
            __syncwarp();
            for (int p = lane; p < 4 * E3; p += 32) {
                const int cc = p / E3, xx = p - cc * E3;
                double acc = xx < m2 ? gTw[p] : 0.0;
                for (int a2 = 0; a2 < m2; ++a2) acc = fma(g[a2 * E3 + xx], Ts[cc * E3 + a2], acc);
                gTw[p] = acc * m.desc_scale;
            }
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
            double s = 0.0, ds = 0.0, d[3] = {0.0, 0.0, 0.0}, rr = 1.0;
            if (slot >= 0) {
                const int j = nlist[(size_t)i * nm + slot];
                const double xj[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
                rr = dp_pinned_dist(xi, xj, box, d);
                dp_switch(rr, m.rcut_smth, m.rcut, s, ds);
            }
            // the 8 sums of rows q0 + 4 it + gq, 8 lanes per row
            for (int it = 0; it < 8 && q0 + 4 * it < nr; ++it) {
                const int sl = __shfl_sync(0xffffffffu, slot, 4 * it + gq);
                double p[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) p[c] = 0.0;
                if (sl >= 0) {
                    const double *gr = Gst + ((size_t)i * nm + sl) * (2 * E3);
#pragma unroll
                    for (int k = 0; k < KF; ++k) {
                        const int ff = sub + 8 * k;
                        if (8 * k + 8 <= E3 || ff < E3) {
                            const double G = gr[ff], dG = gr[E3 + ff];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const double gt = gTw[c * E3 + ff];
                                p[c] = fma(G, gt, p[c]);
                                p[4 + c] = fma(dG, gt, p[4 + c]);
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
                        const double send = up ? p[k] : p[n + k];
                        const double keep = up ? p[n + k] : p[k];
                        p[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                    }
                }
                sa_s[(4 * it + gq) * 8 + sub] = p[0];
            }
            __syncwarp();
            // chain rule through R~(r_ij), lane q on row q0 + q
            if (slot >= 0) {
                double sa[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) sa[c] = sa_s[lane * 8 + c];
                const double inv = 1.0 / rr;
                const double R[4] = {s, s * d[0] * inv, s * d[1] * inv, s * d[2] * inv};
                double gR0 = sa[0];
#pragma unroll
                for (int c = 0; c < 4; ++c) gR0 = fma(R[c], sa[4 + c], gR0);
                const double u[3] = {d[0] * inv, d[1] * inv, d[2] * inv};
                const double dot = sa[1] * u[0] + sa[2] * u[1] + sa[3] * u[2];
                const double sr = s * inv;
                const double coef = gR0 * ds + ds * dot - sr * dot;
                double gv[3];
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) gv[bb] = fma(u[bb], coef, sr * sa[1 + bb]);
                double *pg = pair_g + ((size_t)i * nm + slot) * 3;
                pg[0] = gv[0];
                pg[1] = gv[1];
                pg[2] = gv[2];
#pragma unroll
                for (int aa = 0; aa < 3; ++aa) {
                    fo[aa] += gv[aa];
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) vir[aa * 3 + bb] -= d[aa] * gv[bb];
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

template <int E1>
cudaError_t launch_bwd_st(cudaStream_t st, const DevModel &m, const double *x, const int32_t *types, Box3 box,
                          int N, const FormatBuffers &fb, EvalBuffers eb, int num_sms)
{
    int grid = (N + STW - 1) / STW;
    if (grid > 4 * num_sms) grid = 4 * num_sms;
    if (grid < 1) grid = 1;
    k_embed_bwd_st<E1><<<grid, STW * 32, 0, st>>>(m, x, types, box, N, fb.nlist, fb.nreal, eb.T, eb.gD, eb.Gst,
                                                  eb.pair_g, eb.f_own, eb.vir_part);
    return cudaGetLastError();
}

}  // namespace

bool dp_ex_supported(const DevModel &m)
{
    if (m.n_emb != 3) return false;
    const int e1 = m.emb[0];
    if (e1 != 16 && e1 != 25 && e1 != 32) return false;
    if (m.emb[1] != 2 * e1 || m.emb[2] != 4 * e1) return false;
    return m.M == 4 * e1;
}

size_t dp_ex_bytes(const DevModel &m) { return (size_t)m.ntypes * m.ntypes * net_bytes(m.emb[0]); }

// Digits of the columns of W [K][F] (row-major) as the rows of an Mrows x Kp
// K-major operand: row f holds column f of W scaled by 2^(56 - e_f), 2^e_f > max |W[., f]|
// (e_f = 0 and zero digits for an all-zero or too small column).
static void split_columns(const double *W, int K, int F, int Mrows, int Kp, uint16_t *dig, int32_t *ex)
{
    for (int f = 0; f < Mrows; ++f) {
        double mx = 0.0;
        if (f < F)
            for (int k = 0; k < K; ++k) mx = std::max(mx, std::fabs(W[(size_t)k * F + f]));
        int ef = 0;
        bool zero = !(mx > 0.0);
        if (!zero) {
            std::frexp(mx, &ef);
            if (ef < XBETA * XS - 1020) zero = true;
        }
        if (zero) ef = 0;
        ex[f] = ef;
        const double scale = zero ? 0.0 : std::ldexp(1.0, XBETA * XS - ef);
        for (int k = 0; k < Kp; ++k) {
            long long I = (f < F && k < K) ? std::llrint(W[(size_t)k * F + f] * scale) : 0;
            const uint32_t ofs = tc::kmajor_offset(f, k, Kp) / 2;
            for (int sd = XS - 1; sd >= 0; --sd) {
                const int d = sd > 0 ? oz_digit_step(I, XBETA) : (int)I;
                dig[(size_t)sd * Mrows * Kp + ofs] = oz_bf16_int(d);
            }
        }
    }
}

void dp_ex_split_weights(const DevModel &m, const double *h_params, unsigned char *out)
{
    const int e1 = m.emb[0], e2 = 2 * e1, e3 = 4 * e1, K2p = k2p_of(e1), K1p = k1p_of(e1);
    const size_t nb = net_bytes(e1);
    for (int net = 0; net < m.ntypes * m.ntypes; ++net) {
        unsigned char *blk = out + (size_t)net * nb;
        std::memset(blk, 0, nb);
        const double *W1 = h_params + m.emb_base[net] + 2 * e1;  // [e1][e2]
        const double *W2 = W1 + e1 * e2 + e2;                    // [e2][e3]
        split_columns(W2, e2, e3, XM, K2p, reinterpret_cast<uint16_t *>(blk),
                      reinterpret_cast<int32_t *>(blk + (size_t)XS * XM * K2p * 2));
        if (w1_bytes(e1) > 0) {
            unsigned char *b1 = blk + w2_bytes(e1);
            split_columns(W1, e1, e2, XM1, K1p, reinterpret_cast<uint16_t *>(b1),
                          reinterpret_cast<int32_t *>(b1 + (size_t)XS * XM1 * K1p * 2));
        }
    }
}

cudaError_t dp_launch_embed_bwd_x(cudaStream_t st, const DevModel &m, const unsigned char *wx, const double *x,
                                  const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                  const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                  int64_t *launches)
{
    *launches += 1;
    switch (m.emb[0]) {
    case 16: return launch_tangent_x<16, false>(st, m, wx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 25: return launch_tangent_x<25, false>(st, m, wx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 32: return launch_tangent_x<32, false>(st, m, wx, x, types, box, N, fb, nb, eb, num_sms, status);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t dp_launch_embed_fwd_x(cudaStream_t st, const DevModel &m, const unsigned char *wx, const double *x,
                                  const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                  const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                  int64_t *launches)
{
    *launches += 1;
    switch (m.emb[0]) {
    case 16: return launch_fwd_x<16>(st, m, wx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 25: return launch_fwd_x<25>(st, m, wx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 32: return launch_fwd_x<32>(st, m, wx, x, types, box, N, fb, nb, eb, num_sms, status);
    default: return cudaErrorInvalidValue;
    }
}

size_t dp_ex_store_bytes(const DevModel &m, int64_t natoms)
{
    return (size_t)natoms * (size_t)m.nm * 2 * (size_t)m.M * sizeof(double);
}

cudaError_t dp_launch_embed_tan_x(cudaStream_t st, const DevModel &m, const unsigned char *wx, const double *x,
                                  const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                  const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                  int64_t *launches)
{
    *launches += 1;
    switch (m.emb[0]) {
    case 16: return launch_tangent_x<16, true>(st, m, wx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 25: return launch_tangent_x<25, true>(st, m, wx, x, types, box, N, fb, nb, eb, num_sms, status);
    case 32: return launch_tangent_x<32, true>(st, m, wx, x, types, box, N, fb, nb, eb, num_sms, status);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t dp_launch_embed_bwd_st(cudaStream_t st, const DevModel &m, const double *x, const int32_t *types,
                                   Box3 box, int N, const FormatBuffers &fb, EvalBuffers eb, int num_sms,
                                   int64_t *launches)
{
    *launches += 1;
    switch (m.emb[0]) {
    case 16: return launch_bwd_st<16>(st, m, x, types, box, N, fb, eb, num_sms);
    case 25: return launch_bwd_st<25>(st, m, x, types, box, N, fb, eb, num_sms);
    case 32: return launch_bwd_st<32>(st, m, x, types, box, N, fb, eb, num_sms);
    default: return cudaErrorInvalidValue;
    }
}
