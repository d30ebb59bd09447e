// fit_oz.cu -- the fitting net N_a (Eqs. fitting, fitting-detail; one net per
// centre type, Remark 1), forward and backward to the descriptor, with FP64
// accuracy and every GEMM on the 5th-generation tensor cores.
//
// Exact splitting (Ozaki's scheme).  A GEMM Y = X W with FP64 operands is
// written with a power-of-two scale per row of X (2^e_r >= max_k |X_rk|) and
// per column of W (2^f_n), and the scaled values as S signed digits in base
// 2^beta:
//   X_rk = 2^e_r sum_s a_s,rk 2^(-beta s),   W_kn = 2^f_n sum_t b_t,kn 2^(-beta t),
// with |a_1|, |b_1| <= 2^beta and |a_s|, |b_t| <= 2^(beta-1) for s, t >= 2
// (balanced digits of the integers round(X_rk 2^(beta S - e_r))).  Then
//   Y_rn = 2^(e_r + f_n) sum_g 2^(-beta g) C_g,   C_g = sum_{s+t=g} A_s B_t,
// summed over g = 2 .. S+1 (the terms beyond are below the expansions' own
// precision: FP64 rounding for the 55-bit plans of the FP64 mode, 2^-28
// relative for the 28-bit plans of the split mixed mode).  A digit
// is an integer of at most 8 bits, exact in BF16; every product is exact in
// FP32, and beta is chosen per GEMM from its contraction length K so that
//   K 4^(beta-1) (S + 2) < 2^24,
// which bounds every partial sum of every C_g: the FP32 tensor-core
// accumulators hold C_g exactly, in any summation order.  The result is the
// exact product of the digit expansions, rounded once per group into FP64,
// and is reproducible bit for bit.
//
// Kernels.  k_oz_split: one warp per row of a 128-atom tile of one type;
// row maximum, exponent, digits written as S BF16 matrices in the canonical
// K-major layout of the MMA A operand (16-column chunks).  The weights'
// digits are made once on the host.  k_oz_gemm: one CTA per (tile, 32-column
// chunk of Y); one thread streams the digit chunks of A and W with bulk copies
// (cp.async.bulk, a 2- to 4-stage ring on mbarriers) and issues S(S+1)/2 MMAs
// of 128 x 32 x 16 per chunk into S group accumulators in tensor memory; the
// epilogue (4 warps, one row per thread) combines the groups exactly in int64,
// converts once (one rounding) and applies the layer's bias, tanh and skip
// (forward) or the skip gradient (backward).  Every wait is bounded; on a timeout the kernel sets
// DPF_MMA_TIMEOUT, waits for its copies and MMAs, frees tensor memory and
// returns.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dp_internal.cuh"
#include "tc.cuh"
#include "oz.cuh"

namespace {

constexpr int OZ_STMAX = 4;                 // pipeline stages (at most)
constexpr int OZ_A_BLK = DP_OZ_TILE * DP_OZ_KC;  // elements of one A digit chunk (128 x 16)
constexpr int OZ_B_BLK = DP_OZ_NC * DP_OZ_KC;    // elements of one W digit chunk (32 x 16)

struct TileRef {
    int a, first, cnt;
};

// Tile index -> (type, first position in type_perm, atoms); a = -1 past the end.
__device__ __forceinline__ TileRef oz_tile(int tl, const int32_t *__restrict__ type_start, int ntypes)
{
    TileRef t{-1, 0, 0};
    for (int a = 0; a < ntypes; ++a) {
        const int n_a = type_start[a + 1] - type_start[a];
        const int tiles = (n_a + DP_OZ_TILE - 1) / DP_OZ_TILE;
        if (tl < tiles) {
            t.a = a;
            t.first = type_start[a] + tl * DP_OZ_TILE;
            t.cnt = min(DP_OZ_TILE, n_a - tl * DP_OZ_TILE);
            return t;
        }
        tl -= tiles;
    }
    return t;
}

// ------------------------------------------------------------------ split --

struct OzSplitArgs {
    int mode;  // 0: x = src; 1: x = src (1 - t^2); 2: x = w_out (1 - t^2) and E_i = src . w_out + b_out
    const double *src;
    int lds;
    const double *tv;
    int ldt;
    const double *wout[DP_MAX_TYPES];
    const double *bout[DP_MAX_TYPES];
    double *Ei;
    int K, nK, beta, S;
    const int32_t *type_perm, *type_start;
    int ntypes;
    uint16_t *a;
    int32_t *aexp;
    int64_t a_stride;
};

// One warp per group of 8 rows of a tile (a row group of the canonical
// layout), so that every digit plane of a 16-column chunk is written as one
// contiguous 256-byte block: lane = row (0..7) + 8 * (column half) + 16 *
// (chunk parity).
__global__ void __launch_bounds__(256) k_oz_split(OzSplitArgs p)
{
    const int lane = threadIdx.x & 31;
    const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int tl = gw / (DP_OZ_TILE / 8), r0 = (gw % (DP_OZ_TILE / 8)) * 8;
    const TileRef T = oz_tile(tl, p.type_start, p.ntypes);
    if (T.a < 0) return;
    const int Kp = p.nK * DP_OZ_KC;
    const double *wo = p.mode == 2 ? p.wout[T.a] : nullptr;
    const int bS = p.beta * p.S;

    // value of column k of row r of the tile (0 past the row's end or the tile's atoms)
    auto value = [&](int i, int k) -> double {
        if (i < 0 || k >= p.K) return 0.0;
        double v = p.mode == 2 ? wo[k] : p.src[(size_t)i * p.lds + k];
        if (p.mode != 0) {
            const double t = p.tv[(size_t)i * p.ldt + k];
            v *= fma(-t, t, 1.0);
        }
        return v;
    };

    // per row: output-layer energy (mode 2) and exponent, lanes striding over k
    int e_row = 0;  // lane j < 8 keeps the exponent of row r0 + j
    double sc_row = 0.0;
    for (int j = 0; j < 8; ++j) {
        const int r = r0 + j;
        const int i = r < T.cnt ? p.type_perm[T.first + r] : -1;
        if (p.mode == 2) {
            double e = 0.0;
            if (i >= 0)
                for (int k = lane; k < p.K; k += 32) e = fma(p.src[(size_t)i * p.lds + k], wo[k], e);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
            if (i >= 0 && lane == 0) p.Ei[i] = *p.bout[T.a] + e;
        }
        double mx = 0.0;
        for (int k = lane; k < p.K; k += 32) mx = fmax(mx, fabs(value(i, k)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int e = 0;
        bool zero = !(mx > 0.0);
        if (!zero) {
            frexp(mx, &e);
            if (e < bS - 1020) zero = true;  // below 2^-960: a zero row
        }
        if (zero) e = 0;
        if (lane == j) {
            e_row = e;
            sc_row = zero ? 0.0 : oz_pow2(bS - e);
        }
    }
    if (lane < 8) p.aexp[(size_t)tl * DP_OZ_TILE + r0 + lane] = e_row;

    // digits: lane handles row r0 + (lane & 7), columns kh*8 .. kh*8+7 of chunk kc
    const int jr = lane & 7, kh = (lane >> 3) & 1, cpar = lane >> 4;
    const int r = r0 + jr;
    const int i = r < T.cnt ? p.type_perm[T.first + r] : -1;
    const double scale = __shfl_sync(0xffffffffu, sc_row, jr);
    uint16_t *out = p.a + (size_t)tl * p.a_stride;
    const int ofs = oz_kofs(r, kh * 8);
    for (int kc = cpar; kc < p.nK; kc += 2) {
        const int k8 = kc * DP_OZ_KC + kh * 8;
        long long I[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) I[q] = __double2ll_rn(value(i, k8 + q) * scale);
        for (int sd = p.S - 1; sd >= 0; --sd) {
            int d[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) d[q] = sd > 0 ? oz_digit_step(I[q], p.beta) : (int)I[q];
            uint4 u;
            u.x = (uint32_t)oz_bf16_int(d[0]) | ((uint32_t)oz_bf16_int(d[1]) << 16);
            u.y = (uint32_t)oz_bf16_int(d[2]) | ((uint32_t)oz_bf16_int(d[3]) << 16);
            u.z = (uint32_t)oz_bf16_int(d[4]) | ((uint32_t)oz_bf16_int(d[5]) << 16);
            u.w = (uint32_t)oz_bf16_int(d[6]) | ((uint32_t)oz_bf16_int(d[7]) << 16);
            *reinterpret_cast<uint4 *>(out + ((size_t)kc * p.S + sd) * OZ_A_BLK + ofs) = u;
        }
    }
    (void)Kp;
}

// ------------------------------------------------------------------- gemm --

struct OzGemmArgs {
    const uint16_t *a;
    const int32_t *aexp;
    int64_t a_stride;
    const uint16_t *w;
    const int32_t *wexp;
    OzGemm g;
    const int32_t *type_perm, *type_start;
    int ntypes;
    int epi;      // 0: forward (bias, tanh, skip); 1: backward (skip gradient)
    int skip;     // skip kind of the layer
    int skip_in;  // input width of the layer
    const double *bias[DP_MAX_TYPES];
    const double *hin;  // forward: layer input (skip); backward: dL/dh_l per atom
    int ldh;
    const double *gbc[DP_MAX_TYPES];  // backward: dL/dh_l broadcast per type (last layer), else null
    double *tout;
    double *hout;
    int ldo;
    const double *tanh_tab;
    int32_t *status;
    int nst;        // pipeline stages
    uint32_t tcols; // tensor-memory columns allocated (S * 32 rounded up to 256 or 512)
};

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            tc::smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tc::smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

// y 2^e: one multiplication while 2^e is a normal number (exact, or rounded
// once when the product is subnormal, as ldexp rounds it), ldexp otherwise
__device__ __forceinline__ double scale2(double y, int e)
{
    return (e >= -1022 && e <= 1023) ? y * oz_pow2(e) : ldexp(y, e);
}

template <int S>
__global__ void __launch_bounds__(DP_OZ_TILE, 1) k_oz_gemm(OzGemmArgs p)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t full[OZ_STMAX], empty[OZ_STMAX], done;
    __shared__ int fe_s[DP_OZ_NC];
    __shared__ double bias_s[DP_OZ_NC];
    __shared__ uint32_t tslot;
    __shared__ int fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const OzGemm &g = p.g;
    const int nchunk = blockIdx.x % g.nN;
    const TileRef T = oz_tile(blockIdx.x / g.nN, p.type_start, p.ntypes);
    if (T.a < 0) return;
    const int tl = blockIdx.x / g.nN;
    const int nK = g.nK;
    const uint32_t a_bytes = (uint32_t)S * OZ_A_BLK * 2, b_bytes = (uint32_t)S * OZ_B_BLK * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    const int NST = p.nst;

    if (warp == 0) tc::tmem_alloc(&tslot, p.tcols);
    if (tid < DP_OZ_NC) {
        const int col = nchunk * DP_OZ_NC + tid;
        fe_s[tid] = p.wexp[g.e_off[T.a] + col];
        bias_s[tid] = (p.epi == 0 && col < g.N) ? p.bias[T.a][col] : 0.0;
    }
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&done, 1);
        fail = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tslot;

    if (tid == 0) {
        const uint16_t *asrc = p.a + (size_t)tl * p.a_stride;
        const uint16_t *bsrc = p.w + g.w_off[T.a] + (size_t)nchunk * nK * S * OZ_B_BLK;
        int issued = 0;  // chunks whose copies were issued
        auto load = [&](int kc) {
            unsigned char *st = smraw + (size_t)(kc % NST) * stage_bytes;
            mbar_expect_tx(&full[kc % NST], stage_bytes);
            bulk_g2s(st, asrc + (size_t)kc * S * OZ_A_BLK, a_bytes, &full[kc % NST]);
            bulk_g2s(st + a_bytes, bsrc + (size_t)kc * S * OZ_B_BLK, b_bytes, &full[kc % NST]);
            ++issued;
        };
        for (int kc = 0; kc < NST && kc < nK; ++kc) load(kc);
        const uint32_t idesc = tc::make_idesc_bf16(DP_OZ_TILE, DP_OZ_NC);
        int consumed = 0;
        bool ok = true;
        for (int kc = 0; kc < nK; ++kc) {
            const int st = kc % NST;
            if (!tc::mbar_wait(&full[st], (kc / NST) & 1)) {
                ok = false;
                break;
            }
            ++consumed;
            const uint32_t abase = tc::smem_u32(smraw + (size_t)st * stage_bytes);
            // descriptors of digit plane 1; plane s is (s - 1) blocks further (the
            // address field holds bytes / 16 and stays below 2^14 inside shared memory)
            const uint64_t ad0 = tc::make_desc(abase, 128, 256);
            const uint64_t bd0 = tc::make_desc(abase + a_bytes, 128, 256);
#pragma unroll
            for (int s = 1; s <= S; ++s) {
#pragma unroll
                for (int t = 1; t + s <= S + 1; ++t)
                    tc::mma_bf16(tbase + (uint32_t)(s + t - 2) * DP_OZ_NC, ad0 + (uint64_t)((s - 1) * OZ_A_BLK * 2 / 16),
                                 bd0 + (uint64_t)((t - 1) * OZ_B_BLK * 2 / 16), idesc, kc > 0 || s > 1);
            }
            tc::mma_commit(&empty[st]);
            // refill the stage of the previous chunk once its MMAs are done
            if (kc >= 1 && kc - 1 + NST < nK) {
                const int ps = (kc - 1) % NST;
                if (!tc::mbar_wait(&empty[ps], ((kc - 1) / NST) & 1)) {
                    ok = false;
                    break;
                }
                load(kc - 1 + NST);
            }
        }
        tc::mma_commit(&done);
        if (!ok) {
            fail = 1;
            atomicOr(p.status, DPF_MMA_TIMEOUT);
            // copies still in flight must land before the CTA leaves
            for (int kc = consumed; kc < issued; ++kc) tc::mbar_wait(&full[kc % NST], (kc / NST) & 1);
        }
    }
    const bool waited = tc::mbar_wait(&done, 0);
    const bool bad = __syncthreads_or(!waited) || fail;
    tc::fence_after_sync();
    if (bad) {
        if (tid == 0) atomicOr(p.status, DPF_MMA_TIMEOUT);
    } else {
        const int r = tid;
        const int i = r < T.cnt ? p.type_perm[T.first + r] : -1;
        const uint32_t tl_lane = tbase + ((uint32_t)(32 * warp) << 16);
        // y = sum_{g=2}^{S+1} C_g 2^(beta (S + 1 - g)): the group sums are integers
        // below 2^24, combined exactly in two int64 Horner chains (the H groups of
        // largest scale, then the rest; each chain below 2^(25 + beta (H - 1)) <= 2^53
        // for every (beta, S) of oz_beta) and converted once: y = hi 2^(beta (S - H)) + lo.
        // Then y 2^escale = sum_g C_g 2^(-beta g).  Sixteen columns at a time.
        constexpr int H = (S + 1) / 2;
        const long long sh = 1ll << g.beta;
        const double chi = oz_pow2(g.beta * (S - H));
        const int escale = -g.beta * (S + 1);
        const int er = i >= 0 ? p.aexp[(size_t)tl * DP_OZ_TILE + r] : 0;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            long long hi[16], lo[16];
            __syncwarp();  // the loads below are warp-wide; the previous half's stores diverge
#pragma unroll
            for (int gg = 2; gg <= S + 1; ++gg) {
                float v[16];
                tc::tmem_ld16(tl_lane + (uint32_t)(gg - 2) * DP_OZ_NC + 16 * h, v);
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                    const long long iv = (long long)__float2int_rn(v[n]);
                    if (gg == 2) hi[n] = iv;
                    else if (gg <= H + 1) hi[n] = hi[n] * sh + iv;
                    else if (gg == H + 2) lo[n] = iv;
                    else lo[n] = lo[n] * sh + iv;
                }
            }
            if (i < 0) continue;
            const int c0 = 16 * h;                       // first column of this half in the chunk
            const int n0 = nchunk * DP_OZ_NC + c0;       // ... and in Y
            const int *fe = fe_s + c0;
            const double *bs = bias_s + c0;
            double *ho = p.hout + (size_t)i * p.ldo;
            if (p.epi == 0) {
                const double *hin = p.hin + (size_t)i * p.ldh;
                double *to = p.tout + (size_t)i * p.ldo;
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                    const int col = n0 + n;
                    if (col < g.N) {
                        const double z =
                            scale2(fma((double)hi[n], chi, (double)lo[n]), er + fe[n] + escale) + bs[n];
                        const double t = dp_tanh64(z, p.tanh_tab);
                        const double sk =
                            p.skip == 2 ? hin[col % p.skip_in] : (p.skip == 1 ? hin[col] : 0.0);
                        to[col] = t;
                        ho[col] = sk + t;
                    }
                }
            } else {
                const double *gh = p.gbc[T.a] != nullptr ? p.gbc[T.a] : p.hin + (size_t)i * p.ldh;
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                    const int q = n0 + n;
                    if (q < g.N) {
                        double v = scale2(fma((double)hi[n], chi, (double)lo[n]), er + fe[n] + escale);
                        if (p.skip == 1) v += gh[q];
                        else if (p.skip == 2) v += gh[q] + gh[q + p.skip_in];
                        ho[q] = v;
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, p.tcols);
}

// digit width and count for a contraction of length K and `bits` bits per operand
void oz_beta(int K, int bits, int &beta, int &S)
{
    for (beta = 7; beta >= 4; --beta) {
        S = (bits + beta - 1) / beta;
        const double bound = (double)K * std::pow(4.0, beta - 1) * (S + 2);
        if (bound < 16777216.0) return;
    }
    beta = 0;
    S = 0;
}

// Up to 8 digits: 2 stages and 256 tensor-memory columns, so two CTAs share an
// SM (one's epilogue overlaps the other's MMAs); more digits: 4 stages, one CTA.
int gemm_stages(int S)
{
    if (S <= 8) return 2;
    const int fit = (int)((225 * 1024) / ((size_t)S * (OZ_A_BLK + OZ_B_BLK) * 2));
    return fit < OZ_STMAX ? fit : OZ_STMAX;
}
uint32_t gemm_tcols(int S) { return S * DP_OZ_NC <= 256 ? 256u : 512u; }
size_t gemm_smem(int S) { return (size_t)gemm_stages(S) * S * (OZ_A_BLK + OZ_B_BLK) * 2; }

}  // namespace

bool dp_oz_plan(const DevModel &m, OzModel &oz, int64_t &w_elems, int64_t &e_elems, int bits)
{
    std::memset(&oz, 0, sizeof(oz));
    const int nf = m.n_fit;
    if (nf < 1 || nf > DP_MAX_LAYERS) return false;
    int kin = m.m2 * m.M;
    int fmax = 0, in_w = 0;
    w_elems = 0;
    e_elems = 0;
    for (int l = 0; l < nf; ++l) {
        const int F = m.fit[l];
        if (F > DP_MAX_FIT_W) return false;
        fmax = std::max(fmax, F);
        OzGemm *gs[2] = {&oz.fwd[l], &oz.bwd[l]};
        const int Ks[2] = {kin, F}, Ns[2] = {F, kin};
        for (int d = 0; d < 2; ++d) {
            OzGemm &g = *gs[d];
            g.K = Ks[d];
            g.N = Ns[d];
            g.nK = (g.K + DP_OZ_KC - 1) / DP_OZ_KC;
            g.nN = (g.N + DP_OZ_NC - 1) / DP_OZ_NC;
            oz_beta(g.K, bits, g.beta, g.S);
            if (g.beta == 0 || g.S * DP_OZ_NC > 512 || gemm_smem(g.S) > 225 * 1024) return false;
            if (!(g.S == 4 || g.S == 5 || g.S == 8 || g.S == 10 || g.S == 11 || g.S == 14)) return false;
            in_w = std::max(in_w, g.nK * g.S * OZ_A_BLK);
            for (int a = 0; a < m.ntypes; ++a) {
                g.w_off[a] = w_elems;
                w_elems += (int64_t)g.nN * g.nK * g.S * OZ_B_BLK;
                g.e_off[a] = e_elems;
                e_elems += (int64_t)g.nN * DP_OZ_NC;
            }
        }
        kin = F;
    }
    oz.in_w = in_w;
    oz.fmax = fmax;
    oz.ok = 1;
    return true;
}

void dp_oz_split_weights(const DevModel &m, const double *h_params, const OzModel &oz, uint16_t *w, int32_t *e)
{
    const int nf = m.n_fit;
    for (int a = 0; a < m.ntypes; ++a) {
        const double *W = h_params + m.fit_base[a];
        int kin = m.m2 * m.M;
        for (int l = 0; l < nf; ++l) {
            const int F = m.fit[l];
            // element (k, n) of W_l is W[k * F + n]; the forward GEMM's B operand is
            // B[n][k] = W[k][n] (columns n), the backward's is B[q][n] = W[q][n] (rows q)
            for (int d = 0; d < 2; ++d) {
                const OzGemm &g = d == 0 ? oz.fwd[l] : oz.bwd[l];
                auto elem = [&](int row, int k) -> double {  // B[row][k]
                    if (d == 0) return (k < kin && row < F) ? W[(size_t)k * F + row] : 0.0;
                    return (k < F && row < kin) ? W[(size_t)row * F + k] : 0.0;
                };
                const int Np = g.nN * DP_OZ_NC, Kp = g.nK * DP_OZ_KC;
                for (int row = 0; row < Np; ++row) {
                    double mx = 0.0;
                    for (int k = 0; k < Kp; ++k) mx = std::max(mx, std::fabs(elem(row, k)));
                    int ex = 0;
                    bool zero = !(mx > 0.0);
                    if (!zero) {
                        std::frexp(mx, &ex);
                        if (ex < g.beta * g.S - 1020) zero = true;
                    }
                    if (zero) ex = 0;
                    e[g.e_off[a] + row] = ex;
                    const double scale = zero ? 0.0 : std::ldexp(1.0, g.beta * g.S - ex);
                    const int nc = row / DP_OZ_NC, rl = row % DP_OZ_NC;
                    for (int k = 0; k < Kp; ++k) {
                        long long I = std::llrint(elem(row, k) * scale);
                        const int kc = k / DP_OZ_KC;
                        uint16_t *blk = w + g.w_off[a] + ((size_t)nc * g.nK + kc) * g.S * OZ_B_BLK;
                        for (int s = g.S - 1; s >= 0; --s) {
                            const int dg = s > 0 ? oz_digit_step(I, g.beta) : (int)I;
                            blk[(size_t)s * OZ_B_BLK + oz_kofs(rl, k % DP_OZ_KC)] = oz_bf16_int(dg);
                        }
                    }
                }
            }
            W += (size_t)kin * F + F;
            kin = F;
        }
    }
}

cudaError_t dp_launch_fit_oz(cudaStream_t st, const DevModel &m, const OzModel &oz, const OzBuffers &ob, int N,
                             const NlistBuffers &nb, EvalBuffers eb, int32_t *status, int64_t *launches)
{
    const int nf = m.n_fit, T = m.ntypes;
    const int tiles = (N + DP_OZ_TILE - 1) / DP_OZ_TILE + T;
    if (tiles > ob.tiles) return cudaErrorInvalidValue;
    static size_t configured = 0;
    {
        size_t need = 0;
        for (int l = 0; l < nf; ++l) need = std::max(need, std::max(gemm_smem(oz.fwd[l].S), gemm_smem(oz.bwd[l].S)));
        if (need > configured) {
            cudaError_t e = cudaFuncSetAttribute(k_oz_gemm<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_oz_gemm<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_oz_gemm<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_oz_gemm<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_oz_gemm<11>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_oz_gemm<14>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
            if (e != cudaSuccess) return e;
            configured = need;
        }
    }
    const int K1 = m.m2 * m.M;
    const size_t plane = (size_t)ob.nmax * oz.fmax;
    double *H[2] = {ob.h, ob.h + plane};
    double *G[2] = {ob.g, ob.g + plane};
    // parameter offsets of layer l (W_l, b_l) and of the output layer inside a type's block
    int64_t boff[DP_MAX_LAYERS], wo_off = 0;
    {
        int64_t off = 0;
        int kin = K1;
        for (int l = 0; l < nf; ++l) {
            off += (int64_t)kin * m.fit[l];
            boff[l] = off;
            off += m.fit[l];
            kin = m.fit[l];
        }
        wo_off = off;
    }
    const int split_blocks = (tiles * (DP_OZ_TILE / 8) * 32 + 255) / 256;

    auto split = [&](int mode, const double *src, int lds, const double *tv, const OzGemm &g) -> cudaError_t {
        OzSplitArgs a;
        std::memset(&a, 0, sizeof(a));
        a.mode = mode;
        a.src = src;
        a.lds = lds;
        a.tv = tv;
        a.ldt = oz.fmax;
        for (int t = 0; t < T; ++t) {
            a.wout[t] = m.params + m.fit_base[t] + wo_off;
            a.bout[t] = m.params + m.fit_base[t] + wo_off + m.fit[nf - 1];
        }
        a.Ei = eb.Ei;
        a.K = g.K;
        a.nK = g.nK;
        a.beta = g.beta;
        a.S = g.S;
        a.type_perm = nb.type_perm;
        a.type_start = nb.type_start;
        a.ntypes = T;
        a.a = ob.a;
        a.aexp = ob.aexp;
        a.a_stride = ob.a_stride;
        k_oz_split<<<split_blocks, 256, 0, st>>>(a);
        *launches += 1;
        return cudaGetLastError();
    };
    auto gemm = [&](const OzGemm &g, int epi, int skip, int skip_in, int l, const double *hin, int ldh,
                    bool bcast_wout, double *tout, double *hout, int ldo) -> cudaError_t {
        OzGemmArgs a;
        std::memset(&a, 0, sizeof(a));
        a.a = ob.a;
        a.aexp = ob.aexp;
        a.a_stride = ob.a_stride;
        a.w = oz.w;
        a.wexp = oz.wexp;
        a.g = g;
        a.type_perm = nb.type_perm;
        a.type_start = nb.type_start;
        a.ntypes = T;
        a.epi = epi;
        a.skip = skip;
        a.skip_in = skip_in;
        for (int t = 0; t < T; ++t) {
            a.bias[t] = m.params + m.fit_base[t] + boff[l];
            a.gbc[t] = bcast_wout ? m.params + m.fit_base[t] + wo_off : nullptr;
        }
        a.hin = hin;
        a.ldh = ldh;
        a.tout = tout;
        a.hout = hout;
        a.ldo = ldo;
        a.tanh_tab = m.tanh_tab;
        a.status = status;
        a.nst = gemm_stages(g.S);
        a.tcols = gemm_tcols(g.S);
        const size_t smem = gemm_smem(g.S);
        switch (g.S) {
        case 4: k_oz_gemm<4><<<tiles * g.nN, DP_OZ_TILE, smem, st>>>(a); break;
        case 5: k_oz_gemm<5><<<tiles * g.nN, DP_OZ_TILE, smem, st>>>(a); break;
        case 8: k_oz_gemm<8><<<tiles * g.nN, DP_OZ_TILE, smem, st>>>(a); break;
        case 10: k_oz_gemm<10><<<tiles * g.nN, DP_OZ_TILE, smem, st>>>(a); break;
        case 11: k_oz_gemm<11><<<tiles * g.nN, DP_OZ_TILE, smem, st>>>(a); break;
        default: k_oz_gemm<14><<<tiles * g.nN, DP_OZ_TILE, smem, st>>>(a); break;
        }
        *launches += 1;
        return cudaGetLastError();
    };

    cudaError_t e;
    // forward: h_l = skip(h_{l-1}) + tanh(h_{l-1} W_l + b_l), h_{-1} = D
    int kin = K1;
    for (int l = 0; l < nf; ++l) {
        const double *x = l == 0 ? eb.D : H[(l - 1) & 1];
        const int ldx = l == 0 ? K1 : oz.fmax;
        if ((e = split(0, x, ldx, nullptr, oz.fwd[l])) != cudaSuccess) return e;
        if ((e = gemm(oz.fwd[l], 0, dp_skip_kind(kin, m.fit[l]), kin, l, x, ldx, false,
                      ob.t + (size_t)l * plane, H[l & 1], oz.fmax)) != cudaSuccess)
            return e;
        kin = m.fit[l];
    }
    // output layer (E_i) and dL/dz of the last layer (dL/dh = w_out)
    if ((e = split(2, H[(nf - 1) & 1], oz.fmax, ob.t + (size_t)(nf - 1) * plane, oz.bwd[nf - 1])) != cudaSuccess)
        return e;
    // backward: dL/dh_{l-1} = (dL/dz_l) W_l^T + skip'(dL/dh_l)
    for (int l = nf - 1; l >= 0; --l) {
        const int kin_l = l == 0 ? K1 : m.fit[l - 1];
        const bool last = l == nf - 1;
        double *out = l == 0 ? eb.gD : G[(l - 1) & 1];
        const int ldo = l == 0 ? K1 : oz.fmax;
        if ((e = gemm(oz.bwd[l], 1, dp_skip_kind(kin_l, m.fit[l]), kin_l, l, last ? nullptr : G[l & 1], oz.fmax,
                      last, nullptr, out, ldo)) != cudaSuccess)
            return e;
        if (l > 0)
            if ((e = split(1, G[(l - 1) & 1], oz.fmax, ob.t + (size_t)(l - 1) * plane, oz.bwd[l - 1])) != cudaSuccess)
                return e;
    }
    return cudaSuccess;
}
