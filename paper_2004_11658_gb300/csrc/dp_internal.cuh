// dp_internal.cuh -- types and helpers shared by the CUDA translation units
// of the GB300 Deep Potential library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dp.h"

#define DP_MAX_EMB_W 128     // widest embedding layer
#define DP_MAX_FIT_W 256     // widest fitting layer
#define DP_MAX_NM 1024       // N_m limit

// Device-side status bits (accumulated with atomicOr, read by the host).
enum : int32_t {
    DPF_SEL_OVERFLOW = 1,
    DPF_CAND_OVERFLOW = 2,
    DPF_STALE = 4,
    DPF_NONFINITE = 8,
    DPF_BAD_TYPE = 16,
    DPF_MMA_TIMEOUT = 32,   // a tensor-core completion wait gave up
};

// Model description passed by value to kernels.
struct DevModel {
    int ntypes, nm;
    int sel[DP_MAX_TYPES], sel_off[DP_MAX_TYPES];
    int n_emb, emb[DP_MAX_LAYERS];
    int M, m2;
    int n_fit, fit[DP_MAX_LAYERS];
    int emb_net_size;                       // doubles per embedding net
    double rcut, rcut_smth, desc_scale;
    const double *params;                   // device
    const double *tanh_tab;                 // device, see dp_tanh64
    int64_t emb_base[DP_MAX_TYPES * DP_MAX_TYPES];
    int64_t fit_base[DP_MAX_TYPES];
};

struct Box3 {
    double L[3];
};

// ---------------------------------------------------------------------------
// Pinned distance arithmetic.  Candidate sets and sort keys must be identical
// to the CPU reference bit for bit, so the minimum image and |r| are computed
// with explicitly rounded operations (no FMA contraction):
//   d = xj - xi; d -= L * rint(d / L); r = sqrt((dx*dx + dy*dy) + dz*dz).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dp_min_image_1(double xj, double xi, double L)
{
    double v = __dsub_rn(xj, xi);
    double n = rint(__ddiv_rn(v, L));
    return __dsub_rn(v, __dmul_rn(L, n));
}

__device__ __forceinline__ double dp_pinned_dist(const double *xi, const double *xj, const Box3 &b,
                                                 double d[3])
{
    d[0] = dp_min_image_1(xj[0], xi[0], b.L[0]);
    d[1] = dp_min_image_1(xj[1], xi[1], b.L[1]);
    d[2] = dp_min_image_1(xj[2], xi[2], b.L[2]);
    double r2 = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    r2 = __dadd_rn(r2, __dmul_rn(d[2], d[2]));
    return __dsqrt_rn(r2);
}

// Packed sort key of Algorithm 1: (type, floor(|r| * 1e8), j) as
// type << 60 | q << 26 | j  (4 + 34 + 26 bits; |r| < 171 A, j < 2^26).
__device__ __forceinline__ uint64_t dp_pack_key(int type, double r, int j)
{
    uint64_t q = (uint64_t)floor(__dmul_rn(r, 1e8));
    return ((uint64_t)type << 60) | (q << 26) | (uint64_t)j;
}
#define DP_KEY_NONE 0xFFFFFFFFFFFFFFFFull

// Switching function s(r) = w(r)/r and ds/dr (w: quintic smooth step between
// rcut_smth and rcut; the paper fixes only that w falls smoothly to 0 at rcut).
__device__ __forceinline__ void dp_switch(double r, double rs, double rc, double &s, double &ds)
{
    if (r < rs) {
        double inv = 1.0 / r;
        s = inv;
        ds = -inv * inv;
    } else if (r < rc) {
        double u = (r - rs) / (rc - rs);
        double u2 = u * u;
        double w = u2 * u * (-6.0 * u2 + 15.0 * u - 10.0) + 1.0;
        double um1 = u - 1.0;
        double dw = -30.0 * u2 * um1 * um1 / (rc - rs);
        double inv = 1.0 / r;
        s = w * inv;
        ds = (dw - w * inv) * inv;
    } else {
        s = 0.0;
        ds = 0.0;
    }
}

// FP64 tanh by piecewise Taylor polynomials (tanh64.cu): interval k is
// centred at k/40, k = 0..DP_TANH_NINT-1, and stores [centre, a_0 .. a_7].
#define DP_TANH_INV_H 40
#define DP_TANH_NINT 766
#define DP_TANH_NCOEF 8
#define DP_TANH_STRIDE (DP_TANH_NCOEF + 1)
// Fills the table on the current device (once) and returns its device address.
cudaError_t dp_tanh_setup(const double **table);

__device__ __forceinline__ double dp_tanh64(double x, const double *__restrict__ tab)
{
    const double ax = fabs(x);
    // |x| >= 19.125: +-1 is tanh correctly rounded (1 - tanh(19.125) < 2^-54)
    const long long bits = __double_as_longlong(ax);
    if (bits >= 0x4033200000000000ll) return bits > 0x7ff0000000000000ll ? x : copysign(1.0, x);  // NaN stays NaN
    // k = round-half-even(40 |x|) from the bits of |x| = m 2^(e - 1075) on the
    // integer pipe (the value fma(|x|, 40, 1.5 2^52) would give in its low bits)
    int k = 0;
    {
        const int e = (int)(bits >> 52);
        const int sh = 1075 - e;  // >= 48 below the cutoff
        if (e != 0 && sh < 62) {
            const long long mk = ((bits & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll) * DP_TANH_INV_H;  // < 2^59
            long long r = mk >> sh;
            const long long rem = mk & ((1ll << sh) - 1), half = 1ll << (sh - 1);
            if (rem > half || (rem == half && (r & 1))) r += 1;
            k = (int)r;
        }
    }
    const double *c = tab + k * DP_TANH_STRIDE;
    const double t = ax - c[0];
    double p = c[DP_TANH_NCOEF];
#pragma unroll
    for (int n = DP_TANH_NCOEF - 1; n >= 1; --n) p = fma(p, t, c[n]);
    return copysign(p, x);
}

// Skip kind of an (in -> out) layer: 2 = (x, x), 1 = x, 0 = none.
__host__ __device__ __forceinline__ int dp_skip_kind(int in, int out)
{
    return out == 2 * in ? 2 : (out == in ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Kernel launchers (each returns cudaGetLastError()).
// ---------------------------------------------------------------------------
struct NlistBuffers {
    int32_t *cand;        // [N][cap]
    int32_t *ncand;       // [N]
    double *xref;         // [N][3]
    int32_t *cell_count;  // [ncell]
    int32_t *cell_start;  // [ncell + 1]
    int32_t *cell_cursor; // [ncell]
    int32_t *cell_atoms;  // [N]
    int32_t *cell_sorted; // [N]
    int32_t *atom_cell;   // [N]
    int32_t *type_perm;   // [N]
    int32_t *type_start;  // [ntypes + 1]
};

struct FormatBuffers {
    int32_t *nlist;   // [N][nm]
    uint64_t *keys;   // [N][nm]
    int32_t *nreal;   // [N][ntypes]
};

// gate == nullptr: unconditional build; otherwise every kernel returns at
// once unless *gate != 0, and the last one clears *gate.
cudaError_t dp_launch_build(cudaStream_t st, const DevModel &m, const double *x, const int32_t *types,
                            Box3 box, int N, double rlist, int cap, int nc[3], NlistBuffers nb,
                            int32_t *status, int32_t *gate, int64_t *launches);
// Type partition of the centres 0..n-1 alone (sub-region evaluation: atoms
// n..N-1 are ghosts); the build computes it for all N atoms.
cudaError_t dp_launch_type_perm(cudaStream_t st, const DevModel &m, const int32_t *types, int n,
                                NlistBuffers nb, int32_t *status, int64_t *launches);
// Sets *gate if an atom moved more than sqrt(stale2) from its reference position.
cudaError_t dp_launch_check_stale(cudaStream_t st, const double *x, const double *xref, int N, Box3 box,
                                  double stale2, int32_t *gate, int64_t *launches);
// Algorithm 1 on the candidates within rcut.  sort_small (a power of two,
// 64..1024) is the width of the first pass's sorting network; atoms with more
// neighbours go to a second pass as wide as cap.  retry: device int32
// [1 + N] (count, then atom list), cleared here.
cudaError_t dp_launch_format(cudaStream_t st, const DevModel &m, const double *x,
                             const int32_t *types, Box3 box, int N, int cap, int sort_small, double skin,
                             NlistBuffers nb, FormatBuffers fb, int32_t *status, int32_t *retry,
                             int64_t *launches);

struct EvalBuffers {
    double *T;         // [N][4][M]
    double *D;         // [N][m2*M]
    double *gD;        // [N][m2*M]
    double *Ei;        // [N]
    double *pair_g;    // [N][nm][3]
    double *f_own;     // [N][3]
    double *vir_part;  // [N][9]
    float *fit_t;      // mixed mode: tanh values of the fitting layers [tile][n_fit][256][128]
    float *fit_h;      // mixed mode: fitting activation / gradient [tile][256][128]
    double *Gst;       // FP64 mode, when it fits: G and dG/ds of every neighbour slot [N nm][2 M]
    float *Gmx;        // mixed mode (plain BF16), when it fits: the same in FP32
};

// Mixed-precision operands: BF16 copies of the weight matrices in the
// tensor-core layout (see tc.cuh), FP32 copies of biases and small vectors.
struct MixedModel {
    const unsigned char *emb_ops;                            // bf16 operands, bytes
    int64_t emb_off[DP_MAX_TYPES * DP_MAX_TYPES][2];         // W1^T, W2^T per net (byte offsets); each
                                                             // is followed by its low part (split mode)
    int split;                                               // 1: embedding GEMMs on hi + lo operands
    const float *p32;                                        // all parameters in fp32, FP64 layout
    const unsigned char *fit_fwd, *fit_bwd;                  // bf16 operands, bytes
    int64_t fit_fwd_off[DP_MAX_TYPES][DP_MAX_LAYERS];        // W_l^T, K-chunks of 64
    int64_t fit_bwd_off[DP_MAX_TYPES][DP_MAX_LAYERS];        // W_l,   K-chunks of 64
    int fit_np[DP_MAX_LAYERS];     // F_l padded to 16 (MMA N, forward)
    int fit_kp[DP_MAX_LAYERS];     // K_in,l padded to 64 (forward K)
    int fit_kinp[DP_MAX_LAYERS];   // K_in,l padded to 16 (MMA N, backward)
    int fit_fp[DP_MAX_LAYERS];     // F_l padded to 64 (backward K)
    unsigned char *dtile;          // scratch: the descriptor in BF16, [tile][K1p/64][128 x 64] canonical
};

cudaError_t dp_launch_embed_fwd(cudaStream_t st, const DevModel &m, const double *x,
                                const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                const NlistBuffers &nb, EvalBuffers eb, int num_sms,
                                int64_t *launches);
cudaError_t dp_launch_fit(cudaStream_t st, const DevModel &m, int N, const NlistBuffers &nb,
                          EvalBuffers eb, int64_t *launches);
cudaError_t dp_launch_embed_bwd(cudaStream_t st, const DevModel &m, const double *x,
                                const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                const NlistBuffers &nb, EvalBuffers eb, int num_sms,
                                int64_t *launches);
// Forces on all N atoms from the centres 0..nloc-1 (nloc == N: every atom
// is a centre; nloc < N: atoms nloc..N-1 are ghosts and receive only the
// increments of the centres).
cudaError_t dp_launch_force(cudaStream_t st, const DevModel &m, const double *x,
                            const int32_t *types, Box3 box, int N, int nloc, int cap,
                            const NlistBuffers &nb, const FormatBuffers &fb, EvalBuffers eb,
                            double *force, int64_t *launches);
cudaError_t dp_launch_reduce(cudaStream_t st, int N, EvalBuffers eb, double *energy,
                             double *virial, double *atom_energy, int32_t *status,
                             int64_t *launches);

// FP64 fitting net with its GEMMs on the tensor cores by exact splitting
// (csrc/fit_oz.cu).  Every GEMM Y = X W (X: 128-atom tiles, W: weights) is
//   Y = 2^(e_r + f_n) sum_{s+t <= S+1} 2^(-beta (s+t)) (A_s B_t),
// A_s, B_t the integer digits (|.| <= 2^beta) of X and W in base 2^beta
// relative to per-row / per-column power-of-two scales, stored as BF16; the
// products and their sums over K are integers below 2^24, so the FP32 tensor
// core accumulators hold them exactly and Y is an FP64-accurate product.
constexpr int DP_OZ_TILE = 128;  // atoms per tile (MMA M)
constexpr int DP_OZ_NC = 32;     // output columns per CTA (MMA N)
constexpr int DP_OZ_KC = 16;     // K per chunk (MMA K)
struct OzGemm {
    int K, N;          // contraction and output widths (unpadded)
    int nK, nN;        // chunks of DP_OZ_KC and DP_OZ_NC
    int beta, S;       // digit width (bits) and digit count
    int64_t w_off[DP_MAX_TYPES];  // element offset of the type's weight digits
    int64_t e_off[DP_MAX_TYPES];  // offset of the type's column exponents
};
struct OzModel {
    int ok;                                   // the model's fitting net is supported
    OzGemm fwd[DP_MAX_LAYERS];                // h_l = act(h_{l-1} W_l + b_l)
    OzGemm bwd[DP_MAX_LAYERS];                // g_{l-1} = gz_l W_l^T (+ skip)
    int in_w;                                 // widest GEMM input (K), padded
    int fmax;                                 // widest hidden layer
    const uint16_t *w;                        // device: weight digits
    const int32_t *wexp;                      // device: column exponents
};
struct OzBuffers {
    uint16_t *a;            // A digits, [tiles][a_stride]
    int32_t *aexp;          // row exponents, [tiles][128]
    int64_t a_stride;       // elements per tile
    int tiles;              // tile capacity
    double *t;              // tanh values [n_fit][Nmax][fmax]
    double *h;              // activations, 2 x [Nmax][fmax]
    double *g;              // gradients, 2 x [Nmax][fmax]
    int64_t nmax;
};
// Host: shapes of the split GEMMs (returns false if the fitting net is not
// supported: hidden widths must be <= DP_MAX_FIT_W), then the weight digits.
// bits: the digit expansions carry at least this many bits of every operand
// (55: FP64 accuracy; fewer give a cheaper product of lower accuracy)
bool dp_oz_plan(const DevModel &m, OzModel &oz, int64_t &w_elems, int64_t &e_elems, int bits = 55);
void dp_oz_split_weights(const DevModel &m, const double *h_params, const OzModel &oz, uint16_t *w, int32_t *e);
cudaError_t dp_launch_fit_oz(cudaStream_t st, const DevModel &m, const OzModel &oz, const OzBuffers &ob, int N,
                             const NlistBuffers &nb, EvalBuffers eb, int32_t *status, int64_t *launches);

// FP64 embedding forward with its last layer on the tensor cores by exact
// splitting (csrc/embed_x.cu): 3-layer doubling nets with e1 in {16, 25, 32}.
bool dp_ex_supported(const DevModel &m);
size_t dp_ex_bytes(const DevModel &m);
void dp_ex_split_weights(const DevModel &m, const double *h_params, unsigned char *out);
cudaError_t dp_launch_embed_fwd_x(cudaStream_t st, const DevModel &m, const unsigned char *wx, const double *x,
                                  const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                  const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                  int64_t *launches);
cudaError_t dp_launch_embed_bwd_x(cudaStream_t st, const DevModel &m, const unsigned char *wx, const double *x,
                                  const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                  const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                  int64_t *launches);
// The same forward with the s-tangent, G and dG/ds stored in eb.Gst (bytes for
// natoms atoms: dp_ex_store_bytes), and the streaming backward that reads them.
size_t dp_ex_store_bytes(const DevModel &m, int64_t natoms);
cudaError_t dp_launch_embed_tan_x(cudaStream_t st, const DevModel &m, const unsigned char *wx, const double *x,
                                  const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                  const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                  int64_t *launches);
cudaError_t dp_launch_embed_bwd_st(cudaStream_t st, const DevModel &m, const double *x, const int32_t *types,
                                   Box3 box, int N, const FormatBuffers &fb, EvalBuffers eb, int num_sms,
                                   int64_t *launches);

// Mixed precision (BF16 tensor-core GEMMs, FP64 environment / contractions).
// The tangent forward storing G and dG/ds (FP32) in eb.Gmx (bytes for natoms
// atoms: dp_mx_store_bytes) and the streaming backward that reads them.
size_t dp_mx_store_bytes(const DevModel &m, int64_t natoms);
cudaError_t dp_launch_embed_tan_mx(cudaStream_t st, const DevModel &m, const MixedModel &mx, const double *x,
                                   const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                   const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                   int64_t *launches);
cudaError_t dp_launch_embed_bwd_stmx(cudaStream_t st, const DevModel &m, const double *x, const int32_t *types,
                                     Box3 box, int N, const FormatBuffers &fb, EvalBuffers eb, int num_sms,
                                     int64_t *launches);
cudaError_t dp_launch_embed_fwd_mx(cudaStream_t st, const DevModel &m, const MixedModel &mx, const double *x,
                                   const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                   const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                   int64_t *launches);
cudaError_t dp_launch_fit_mx(cudaStream_t st, const DevModel &m, const MixedModel &mx, int N,
                             const NlistBuffers &nb, EvalBuffers eb, int32_t *status, int64_t *launches);
cudaError_t dp_launch_embed_bwd_mx(cudaStream_t st, const DevModel &m, const MixedModel &mx, const double *x,
                                   const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                   const NlistBuffers &nb, EvalBuffers eb, int num_sms, int32_t *status,
                                   int64_t *launches);
// true if the mixed-precision kernels support this model shape
bool dp_mixed_supported(const DevModel &m);

// Parameter gradient of cE E + sum lambda . F (pgrad.cu).
struct PGradBuffers {
    double *dT;       // [N][4][M] tangent of T
    double *dD;       // [N][m2*M]
    double *Db, *dDb; // [N][m2*M] adjoints of D and dD
    double *fit_scr;  // dp_pgrad_fit_scratch(N) doubles
    double *rowscr;   // dp_pgrad_row_scratch(num_sms) doubles
    double *slices;   // [num_sms][nparams] per-CTA gradient partials
};
size_t dp_pgrad_fit_scratch(int N);
size_t dp_pgrad_row_scratch(int num_sms);
cudaError_t dp_launch_pgrad(cudaStream_t st, const DevModel &m, int64_t nparams, const double *x, const int32_t *types,
                            Box3 box, int N, const double *lam, double cE, const FormatBuffers &fb,
                            const NlistBuffers &nb, EvalBuffers eb, PGradBuffers pb, int num_sms, double *grad,
                            int64_t *launches);

// MD integrator kernels.
cudaError_t dp_launch_kick_drift(cudaStream_t st, int N, double *x, double *v, const double *f,
                                 const int32_t *types, const double *inv_mass_conv, double dt,
                                 Box3 box, int64_t *launches);
cudaError_t dp_launch_kick_thermo(cudaStream_t st, int N, double *v, const double *f,
                                  const int32_t *types, const double *inv_mass_conv,
                                  const double *mass, double dt, double *ke_part,
                                  int64_t *launches);
cudaError_t dp_launch_thermo(cudaStream_t st, int N, const double *ke_part, const double *energy,
                             const double *virial, double volume, double *thermo_row,
                             int64_t *launches);
