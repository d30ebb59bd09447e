/*
 * dp.h -- C ABI of the GB300 Deep Potential hot path.
 *
 * Method: Lu et al., "86 PFLOPS Deep Potential Molecular Dynamics simulation
 * of 100 million atoms with ab initio accuracy" (arXiv 2004.11658).  One call
 * of dp_eval computes the energy E = sum_i E_i (Sec. 2, Eq. ei), the forces
 * F_i = -grad_{r_i} E (Remark 2, Eq. dp-force) and the virial of a
 * smooth-edition Deep Potential model on one GPU; dp_md_step advances
 * velocity-Verlet molecular dynamics (Sec. 4).
 *
 * Conventions (all entry points):
 *   - Units: Angstrom, eV, fs, amu, K.
 *   - Arrays named "device" are caller-owned CUDA device pointers, contiguous,
 *     row-major; the library never frees them.  Arrays named "host" are
 *     caller-owned host memory, read during the call only.
 *   - Coordinates are [N][3] float64, types [N] int32 in [0, ntypes).
 *   - box is host double[9], a row-major 3x3 cell; only orthorhombic
 *     (diagonal) cells are supported, others give DP_ERR_BOX.
 *   - Work is enqueued on the stream given to dp_ctx_create.  With sync mode
 *     on (the default) each call ends by reading a 4-byte device status word,
 *     which synchronises that stream; with sync mode off the call returns
 *     after enqueueing and device-side conditions are read by dp_ctx_status.
 *   - No C++ exception crosses this boundary.  On error a message is kept in
 *     thread-local storage (dp_last_error).
 *   - A context is not thread safe: use one context per host thread.
 */
#ifndef DP_GB300_H
#define DP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t dp_status;

#define DP_OK                 0
#define DP_ERR_ARG           -1   /* bad pointer, size or descriptor           */
#define DP_ERR_BOX           -2   /* non-orthorhombic or too small cell        */
#define DP_ERR_SEL_OVERFLOW  -3   /* a neighbour within rcut did not fit sel;
                                     results are written for the truncated list */
#define DP_ERR_NLIST_STALE   -4   /* an atom moved more than skin/2 since the
                                     last candidate build; results are written  */
#define DP_ERR_NONFINITE     -5   /* NaN/Inf in the energy or virial           */
#define DP_ERR_FILE          -6   /* model file missing, truncated or corrupt  */
#define DP_ERR_CUDA          -7   /* a CUDA call failed                        */
#define DP_ERR_UNSUPPORTED   -8   /* widths or type counts beyond the limits   */
#define DP_ERR_CAPACITY      -9   /* an atom had more candidates than cand_cap */
#define DP_ERR_NOMEM        -10   /* device allocation failed                  */
#define DP_ERR_TYPE         -11   /* a type id outside [0, ntypes)             */

#define DP_MAX_TYPES   8
#define DP_MAX_LAYERS  4

/* Model hyper-parameters (Sec. 2; the paper's models are described in Sec. 4).
 *   sel[a]      : neighbour slots for type a; N_m = sum(sel) (Sec. 2, Sec. 3.2.2)
 *   emb[0..n_emb): embedding widths s_1..s_m, s_m = M (Eqs. embedding-first/-rest)
 *   m2          : M^<, the columns of G kept in G^< (Eq. descrpt)
 *   fit[0..n_fit): hidden widths of the fitting net (Eqs. fitting, fitting-detail)
 *   desc_scale_nm: 1 -> the descriptor uses T = R~^T G / N_m; 0 -> unscaled
 *   rcut, rcut_smth: the gate w(r) is 1 below rcut_smth, 0 from rcut on.
 * Limits: ntypes <= 8, 1 <= n_emb <= 4 with widths <= 128, n_fit <= 4 with
 * widths <= 256, m2 <= M, N_m <= 1024. */
typedef struct {
    int32_t ntypes;
    int32_t sel[DP_MAX_TYPES];
    int32_t n_emb;
    int32_t emb[DP_MAX_LAYERS];
    int32_t m2;
    int32_t n_fit;
    int32_t fit[DP_MAX_LAYERS];
    int32_t desc_scale_nm;
    int32_t reserved;
    double rcut;
    double rcut_smth;
} dp_model_desc;

typedef struct dp_model dp_model;
typedef struct dp_ctx dp_ctx;

/* Precision modes of a context. */
#define DP_PREC_FP64  0   /* every step with float64 accuracy; the dense products
                             (the fitting-net GEMMs and, for 3-layer doubling
                             embedding nets with s_1 in {16, 25, 32}, the last
                             embedding layer and layer 1 with their s-tangents)
                             run on the tensor cores as exact products of BF16
                             digit expansions of
                             the FP64 operands (every partial sum an integer
                             below 2^24, held exactly by the FP32 accumulators),
                             the rest on the FP64 units; other shapes run as
                             FP64_SIMT */
#define DP_PREC_FP64_SIMT 2  /* every step in float64 on the FP64 units */
#define DP_PREC_MIXED 1   /* embedding- and fitting-net GEMMs on the tensor cores
                             (BF16 operands, FP32 accumulation, FP32 tanh); the
                             environment matrix, the descriptor contraction
                             T = R~^T G / N_m and D, the backward contractions,
                             forces, virial, energy sum and the integrator in
                             FP64.  Needs a 3-layer doubling embedding net with
                             s_1 in {16, 25, 32} and equal fitting widths
                             (multiples of 16, <= 256) after the first layer;
                             other shapes give DP_ERR_UNSUPPORTED. */
#define DP_PREC_MIXED_SPLIT 3  /* DP_PREC_MIXED with the embedding-net GEMMs on split
                             operands -- every FP32 activation and weight is the sum
                             of a BF16 high part and the BF16 value of its
                             remainder, and each product is hi*hi + hi*lo + lo*hi
                             (three MMAs into the FP32 accumulator), ~16 bits
                             per operand instead of 8 -- and the fitting net as
                             exact products of 28-bit digit expansions of its
                             operands (the FP64 mode's kernels with 4-5 digits
                             instead of 8-11: FP32-level accuracy).
                             For systems whose forces are small sums of many large
                             pair terms (a nearly symmetric crystal), where the
                             rounding of each atom's dE/dD and of each neighbour's
                             G does not cancel.  Same shapes as DP_PREC_MIXED. */

/* Thread-local text of the last error (never NULL). */
const char *dp_last_error(void);
/* Static text for a status code. */
const char *dp_status_string(dp_status s);

/* Number of float64 parameters of a model with this descriptor, or -1 if the
 * descriptor is invalid.  Flat layout: for every ordered type pair (a, b),
 * a-major, the embedding net G^{a,b} (Remark 1): W0[s1], b0[s1], then per
 * layer l W[s_l][s_{l+1}] (input index first), b[s_{l+1}]; then for every
 * type a the fitting net N_a: W1[m2*M][f1], b1[f1], W_l[f_{l-1}][f_l], b_l[f_l],
 * w_out[f_last], b_out. */
int64_t dp_model_nparams(const dp_model_desc *desc);

/* Create a model from a host descriptor and host parameters (copied to the
 * current CUDA device).  *out is owned by the caller; free with dp_model_free. */
dp_status dp_model_create(const dp_model_desc *desc, const double *params, int64_t nparams,
                          dp_model **out);
/* Seeded model (the paper's models are trained, Sec. 2 and Sec. 4, and no
 * trained model is available, so weights are drawn from a seed).  Element k
 * of the flat parameter vector (layout of dp_model_nparams) is
 *     scale * n_k,
 * with n_k the k-th standard normal of one stream: splitmix64 outputs
 * z_i = mix(seed + i * 0x9E3779B97F4A7C15), i = 1, 2, ... (Steele, Lea and
 * Flood, 2014), uniforms u1 = ((z_{2p+1} >> 11) + 1) * 2^-53 in (0, 1] and
 * u2 = (z_{2p+2} >> 11) * 2^-53 in [0, 1), and Box-Muller:
 * n_{2p} = sqrt(-2 ln u1) cos(2 pi u2), n_{2p+1} = sqrt(-2 ln u1) sin(2 pi u2).
 * Scales: every weight matrix n / sqrt(fan_in + fan_out) (embedding layer 0:
 * fan_in 1), the first fitting layer's weights then times fit_in_gain; every
 * hidden bias n; output weights (out_scale * n) / sqrt(f_last + 1); b_out 0.
 * dp_model_params_from_seed writes the nparams host doubles of params (nparams
 * must equal dp_model_nparams(desc)); dp_model_from_seed creates the model
 * directly (as dp_model_create).  The values are reproducible on every
 * machine whose libm gives the same log, sin and cos. */
dp_status dp_model_params_from_seed(const dp_model_desc *desc, uint64_t seed, double fit_in_gain,
                                    double out_scale, double *params, int64_t nparams);
dp_status dp_model_from_seed(const dp_model_desc *desc, uint64_t seed, double fit_in_gain,
                             double out_scale, dp_model **out);

/* Load / save the binary model file: "DPGB300M" magic, uint32 version 1,
 * the descriptor fields as little-endian int32/float64 in declaration order,
 * int64 nparams, nparams float64.  DP_ERR_FILE on a short or corrupt file. */
dp_status dp_model_load(const char *path, dp_model **out);
dp_status dp_model_save(const dp_model *model, const char *path);
void dp_model_free(dp_model *model);

/* Create a context for up to natoms_max atoms.  cand_cap is the capacity of
 * one atom's candidate list (neighbours within rcut + skin); 0 picks a
 * default from the density at the first dp_build_nlist.  stream is a
 * cudaStream_t (NULL = legacy default stream).  The context owns all scratch
 * memory of the path (O(natoms_max * N_m) words); it does not own the model,
 * which must outlive it. */
dp_status dp_ctx_create(const dp_model *model, int64_t natoms_max, int32_t cand_cap,
                        int32_t precision, void *stream, dp_ctx **out);
void dp_ctx_free(dp_ctx *ctx);

/* FP64 contexts of the tensor-core embedding kernels and mixed-precision
 * contexts with plain BF16 operands (DP_PREC_MIXED), 3-layer doubling nets with
 * s_1 in {16, 25, 32}: the back-propagation of Sec. 2 (Eq. embedding through
 * the chain rule of the environment matrix, Sec. 3.2) needs, for every real
 * neighbour row, G and its derivative dG/ds with respect to the row's s(r).
 * With the store on, the forward computes both once and keeps them in device
 * memory (natoms_max * N_m * 2 * M values, FP64 or FP32 as the context
 * computes them: 86.8 / 43.4 GB for 393,216 water atoms with N_m = 138,
 * M = 100), and the backward reads them instead of evaluating the embedding
 * net a second time; off, the backward recomputes them.  Both give the same
 * atomic energies, and forces and virial equal up to the order of the sums
 * over the M features.  dp_ctx_create turns the store on when it takes at most
 * half of the device memory free at that moment.  on = 1 allocates it
 * (DP_ERR_NOMEM if that fails, the context unchanged), on = 0 frees it;
 * DP_ERR_UNSUPPORTED for other contexts when on = 1.  Synchronises the
 * context's stream.  dp_ctx_embed_store returns 1 when the store is on, 0
 * when off, -1 for NULL. */
dp_status dp_ctx_set_embed_store(dp_ctx *ctx, int32_t on);
int32_t dp_ctx_embed_store(const dp_ctx *ctx);
/* sync = 1 (default): every call reads the device status word at its end.
 * sync = 0: calls only enqueue; dp_ctx_status reads the accumulated word. */
dp_status dp_ctx_set_sync(dp_ctx *ctx, int32_t sync);
dp_status dp_ctx_status(dp_ctx *ctx);
/* Kernels launched through this context since creation. */
int64_t dp_ctx_launches(const dp_ctx *ctx);

/* Per-kernel-group device time, measured with CUDA events recorded on the
 * context's stream around every launch while timing is on.  Groups:
 * 0 build (cell list + candidates + type order), 1 format (Algorithm 1),
 * 2 embed_fwd, 3 fit, 4 embed_bwd, 5 force (ProdForce gather), 6 reduce
 * (energy/virial sums), 7 md (integrator and thermo kernels). */
#define DP_KERNEL_GROUPS 8
/* on = 1 starts timing and clears the accumulators; on = 0 stops it. */
dp_status dp_ctx_set_timing(dp_ctx *ctx, int32_t on);
/* Accumulated milliseconds ms[8] and launch counts launches[8] (either may
 * be NULL); synchronises the context's stream. */
dp_status dp_ctx_kernel_times(dp_ctx *ctx, double *ms, int64_t *launches);
/* Static name of a kernel group ("build", "format", ...), or "?". */
const char *dp_kernel_group_name(int32_t group);

/* Cell-list neighbour candidates (the neighbour list with a buffer of width
 * skin, Sec. 3.2.2 and Sec. 4): for every atom, all j != i with minimum-image
 * |r_ij| <= rcut + skin.  coords, types: device.  Also records the reference
 * positions for the staleness check and the type-sorted atom order.
 * Requires box edges >= 2 (rcut + skin).  Enqueued; see sync mode. */
dp_status dp_build_nlist(dp_ctx *ctx, const double *coords, const int32_t *types,
                         const double box[9], int64_t N, double skin);

/* Algorithm 1 (formatted neighbour list) from the current coordinates and the
 * candidates of the last dp_build_nlist: the neighbours within rcut -- L(i)
 * of Sec. 2 -- in type blocks of sel[a] slots in type order, each block sorted
 * by (floor(|r_ij| * 1e8), j), truncated to sel[a] and padded with -1.  Writes
 * nlist[N][N_m] (int32 atom indices) and nreal[N][ntypes] (entries kept in
 * each block).  Either output may be NULL.  Device pointers.  The result does
 * not depend on the skin of the candidates.  DP_ERR_SEL_OVERFLOW if a
 * neighbour within rcut was cut. */
dp_status dp_format_nlist(dp_ctx *ctx, const double *coords, const int32_t *types,
                          const double box[9], int64_t N, int32_t *nlist, int32_t *nreal);

/* The FP64 tanh used by the FP64 kernels (piecewise degree-8 Taylor
 * polynomials of tanh on intervals of width 1/20: truncation below 1e-16,
 * |error| with FP64 rounding below 4e-16 absolute),
 * exposed so that its accuracy can be checked: y[i] = tanh(x[i]) for n device
 * doubles, on stream (NULL = legacy default); returns after the stream has
 * finished.  The paper's nets use tanh as their activation (Eqs.
 * embedding-first, embedding-rest, fitting-detail). */
dp_status dp_tanh_f64(const double *x, double *y, int64_t n, void *stream);

/* No-allocation variant of dp_format_nlist.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory at
 * the time they need the list -- a host MD engine that owns a fixed device
 * budget and forbids allocations after start-up, or code running where
 * cudaMalloc is not allowed.  It needs no context and no model object: it
 * reads the descriptor (ntypes, sel, rcut) from the host struct, builds the
 * candidates (all j != i with minimum-image |r_ij| <= rcut + skin) by brute
 * force and runs Algorithm 1, writing the same nlist[N][N_m] and
 * nreal[N][ntypes] (device, caller-owned, both required) as dp_format_nlist
 * for the same candidate radius.  coords, types: device; box: host double[9];
 * stream: cudaStream_t (NULL = legacy default stream); the call returns after
 * the stream has finished the work.
 * Every cell edge must be at least 2 (rcut + skin), as for dp_build_nlist
 * (DP_ERR_BOX otherwise).
 * Scratch: one file-scope device array of fixed size (about 21 MB) that every
 * GPU loading the library holds until the process exits; it bounds
 * N <= DP_NOALLOC_MAX_ATOMS and the candidates of an atom to
 * DP_NOALLOC_CAND_CAP.  Larger N gives DP_ERR_CAPACITY before any work, more
 * candidates give DP_ERR_CAPACITY after it.  The call makes no cudaMalloc,
 * cudaFree or other allocating call.  Its first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current, so make that first call before any stream capture.  With lazy
 * module loading (the CUDA default) that first call is also when the driver
 * loads the array's module and commits its ~21 MB on the device: a caller
 * with a fixed device budget should make one call at start-up.  All calls
 * share the array, which keeps the last call's contents: calls that overlap
 * on the GPU (other streams, other host threads) race and must not be made. */
#define DP_NOALLOC_MAX_ATOMS 2048
#define DP_NOALLOC_CAND_CAP 512
dp_status dp_format_nlist_noalloc(const dp_model_desc *desc, const double *coords,
                                  const int32_t *types, const double box[9], int64_t N,
                                  double skin, int32_t *nlist, int32_t *nreal, void *stream);

/* Energy, forces and virial (Sec. 2; Algorithms 1 and 2; Eqs. embedding,
 * descrpt, fitting; Remark 2).  energy: device double[1]; force: device
 * [N][3]; virial: device double[9], Xi[a][b] = -sum_{i,j} r_ij[a] dE_i/dr_ij[b]
 * (= sum_i r_i[a] F_i[b] for an isolated cluster); atom_energy: device [N] or
 * NULL.  Uses the candidates of the last dp_build_nlist for the same N (built
 * with skin 0 when there is none). */
dp_status dp_eval(dp_ctx *ctx, const double *coords, const int32_t *types, const double box[9],
                  int64_t N, double *energy, double *force, double *virial,
                  double *atom_energy);

/* Sub-region evaluation for spatial domain decomposition (Sec. 3.1 and
 * Remark 4).  Atoms [0, nloc) are the centres (the atoms a process owns);
 * atoms [nloc, N) are ghost atoms, copies of other processes' atoms within
 * the ghost width of the sub-region, that enter only as neighbours.
 * energy: sum of E_i over the centres; virial: -sum over the centres i of
 * r_ij[a] dE_i/dr_ij[b]; force: device [N][3], for the centres the sum of
 * all increments of the centres, for a ghost the increments -dE_i/dr_j of
 * the centres i (which its owner adds to the atom's force: the reverse halo
 * exchange); atom_energy: device [nloc] or NULL.  Summed over the
 * sub-regions of a partition these equal dp_eval of the whole system.  The
 * cell is periodic as given: a non-periodic edge of a sub-region is padded by
 * the caller (edge >= sub-region + 2 ghost widths + rcut + skin).  nloc == N
 * is dp_eval; nloc == 0 gives zero energy and forces.  DP_ERR_ARG unless
 * 0 <= nloc <= N. */
dp_status dp_eval_local(dp_ctx *ctx, const double *coords, const int32_t *types, const double box[9],
                        int64_t N, int64_t nloc, double *energy, double *force, double *virial,
                        double *atom_energy);

/* nsteps of velocity-Verlet NVE (Sec. 4): v += F/m dt/2; x += v dt; wrap
 * into the cell; rebuild the candidates when the context's MD step counter
 * is a multiple of rebuild_every (and at the first step of a context), and
 * also, with skin > 0, at any step where an atom has moved more than skin/2
 * since the last build (checked on the device every step, no host sync);
 * Algorithm 1 + evaluation; v += F/m dt/2.  coords, vel: device [N][3],
 * updated in place.  mass_per_type: host [ntypes] (amu).  thermo: device
 * [nsteps][4] = (E_pot, E_kin, T, P) per step (eV, eV, K, eV/A^3,
 * P = (2 E_kin + tr Xi)/(3V), T with 3N-3 degrees of freedom) or NULL.
 * The force of the current coordinates is kept in the context between calls
 * (computed first when absent).  With skin = 0 the list must be rebuilt
 * every step (rebuild_every = 1) to stay exact. */
dp_status dp_md_step(dp_ctx *ctx, double *coords, double *vel, const int32_t *types,
                     const double box[9], const double *mass_per_type, int64_t N,
                     double dt_fs, int32_t nsteps, int32_t rebuild_every, double skin,
                     double *thermo);
/* The two halves of one velocity-Verlet step (Sec. 4) as separate calls, for
 * drivers that evaluate the forces themselves between them (the slab
 * decomposition of Sec. 3.1, whose forces come from dp_eval_local and the
 * halo exchanges):
 *   dp_md_kick_drift: v += F/m dt/2; x += v dt; x wrapped into [0, L) of box
 *                     (box NULL: no wrapping, for drivers that keep positions
 *                     continuous between their own wraps);
 *   dp_md_kick:       v += F/m dt/2.
 * coords, vel: device [N][3], updated in place; force: device [N][3] (eV/A);
 * types: device [N]; mass_per_type: host [ntypes] (amu, > 0).  The same
 * arithmetic as dp_md_step.  N <= the context's natoms_max. */
dp_status dp_md_kick_drift(dp_ctx *ctx, double *coords, double *vel, const double *force,
                           const int32_t *types, const double box[9], const double *mass_per_type,
                           int64_t N, double dt_fs);
dp_status dp_md_kick(dp_ctx *ctx, double *vel, const double *force, const int32_t *types,
                     const double *mass_per_type, int64_t N, double dt_fs);
/* Parameter gradient for training (the paper trains the model by
 * back-propagation; forces are -grad E, Remark 2):
 *     grad = d/dW [ cE * E(W) + sum_i lambda_i . F_i(W) ],
 * i.e. the gradient of any loss L(E, F) with cE = dL/dE and lambda = dL/dF,
 * at the current coordinates.  The force term is a mixed second derivative,
 * evaluated as forward tangents of the environment matrix, embedding,
 * descriptor and fitting nets along the neighbour displacements
 * lambda_j - lambda_i followed by reverse mode; G is recomputed, never
 * stored.  lambda: device [N][3]; grad: device [nparams] (flat layout of
 * dp_model_nparams), overwritten.  FP64 contexts only (DP_ERR_UNSUPPORTED
 * otherwise).  Reproducible bit for bit.  Scratch of about
 * num_SMs * nparams doubles plus ~30 KB per atom is allocated on the first
 * call. */
dp_status dp_param_grad(dp_ctx *ctx, const double *coords, const int32_t *types, const double box[9],
                        int64_t N, double cE, const double *lambda, double *grad);
/* Replace the parameters of a model (host array, nparams doubles).  Contexts
 * made from the model see the new values on their next call; mixed-precision
 * contexts keep the BF16 copies made at their creation and must be recreated.
 * Values equal bit for bit to the current ones change nothing (no upload, the
 * FP64 contexts keep their weight digits). */
dp_status dp_model_set_params(dp_model *model, const double *params, int64_t nparams);

/* Copy the context's MD force ([N][3]) to a device buffer. */
dp_status dp_md_get_force(dp_ctx *ctx, double *force, int64_t N);
/* Forget the MD force and step counter (next dp_md_step recomputes both). */
dp_status dp_md_reset(dp_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* DP_GB300_H */
