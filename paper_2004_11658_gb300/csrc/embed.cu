// embed.cu -- environment matrix (Algorithm 2), embedding net (Eqs. embedding,
// embedding-first, embedding-rest) and descriptor (Eq. descrpt) in FP64, and
// the backward pass through them to the pair gradients dE_i/dr_ij.
//
// Design (GB300, FP64 mode).  The embedding tensor G (atoms x N_m x M) never
// touches HBM.  One CTA of 8 warps handles one atom at a time (persistent
// loop over the type-sorted atoms).  The atom's real neighbours (slots before
// nreal in each type block; padded slots and slots beyond rcut have a zero
// environment row and are skipped, which is exact) are processed in chunks of
// 32 rows, one row per lane; the 8 warps split the output columns of every
// layer.  Activations stay in shared memory, the current net's weights are
// staged in shared memory and read as warp-uniform broadcasts.
//
//   k_embed_fwd: R~ rows, G = L_m o ... o L_0(s), T = scale * R~^T G (4 x M),
//                D = T_<^T T (M2 x M).  T and D go to global memory (small).
//   k_embed_bwd: recomputes G together with its derivative dG/ds (forward-mode
//                tangent, one extra GEMM per layer instead of storing G), then
//                gR~[k][c] = sum_m G[k][m] gT[c][m] and
//                dE/ds[k]  = sum_c R~[k][c] sum_m dG/ds[k][m] gT[c][m],
//                and the chain rule through R~(r_ij) gives g_ij = dE_i/dr_ij.
//                Writes g_ij per slot, sum_j g_ij (the atom's own force part)
//                and -sum_j r_ij (x) g_ij (the atom's virial part).
#include "dp_internal.cuh"

namespace {

constexpr int ROWS = 32;          // rows per chunk (one per lane)
constexpr int NTHREADS = 256;     // 8 warps
constexpr int NWARPS = NTHREADS / 32;

struct RowGeom {
    double s, ds, R[4], d[3], r;
};

__device__ __forceinline__ void row_geometry(const DevModel &m, const double *__restrict__ x,
                                             const double xi[3], int j, const Box3 &box, RowGeom &g)
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

__device__ __forceinline__ void stage_net(const DevModel &m, int net, double *Wsm)
{
    const double *src = m.params + m.emb_base[net];
    for (int q = threadIdx.x; q < m.emb_net_size; q += blockDim.x) Wsm[q] = src[q];
}

__global__ void __launch_bounds__(NTHREADS) k_embed_fwd(
    DevModel m, const double *__restrict__ x, const int32_t *__restrict__ types, Box3 box, int N,
    const int32_t *__restrict__ type_perm, const int32_t *__restrict__ nlist,
    const int32_t *__restrict__ nreal, double *__restrict__ Tout, double *__restrict__ Dout, int LD,
    int wsz)
{
    extern __shared__ double sm[];
    double *Wsm = sm;
    double *bufA = Wsm + wsz;
    double *bufB = bufA + ROWS * LD;
    double *Rt = bufB + ROWS * LD;   // [32][4]
    double *srow = Rt + ROWS * 4;    // [32]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int M = m.M, ne = m.n_emb, e1 = m.emb[0], T = m.ntypes, nm = m.nm;
    const int npairs = 4 * M;  // <= 512 = 2 * NTHREADS
    int staged = -1;

    for (int ii = blockIdx.x; ii < N; ii += gridDim.x) {
        const int i = type_perm[ii];
        const int a = types[i];
        const bool a_ok = (unsigned)a < (unsigned)T;  // invalid types are flagged by format
        const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        double tacc[2] = {0.0, 0.0};
        for (int b = 0; b < T; ++b) {
            const int nb = a_ok ? nreal[(size_t)i * T + b] : 0;
            if (nb == 0) continue;
            const int net = a * T + b;
            if (net != staged) {
                __syncthreads();
                stage_net(m, net, Wsm);
                staged = net;
                __syncthreads();
            }
            for (int c0 = 0; c0 < nb; c0 += ROWS) {
                if (warp == 0) {
                    RowGeom g;
                    g.s = 0.0;
                    g.R[0] = g.R[1] = g.R[2] = g.R[3] = 0.0;
                    if (c0 + lane < nb) {
                        const int j = nlist[(size_t)i * nm + m.sel_off[b] + c0 + lane];
                        row_geometry(m, x, xi, j, box, g);
                    }
                    srow[lane] = g.s;
                    Rt[lane * 4 + 0] = g.R[0];
                    Rt[lane * 4 + 1] = g.R[1];
                    Rt[lane * 4 + 2] = g.R[2];
                    Rt[lane * 4 + 3] = g.R[3];
                }
                __syncthreads();
                // layer 0: tanh(s W0 + b0)
                {
                    const double sv = srow[lane];
                    for (int o = warp; o < e1; o += NWARPS)
                        bufA[lane * LD + o] = dp_tanh64(fma(sv, Wsm[o], Wsm[e1 + o]), m.tanh_tab);
                }
                __syncthreads();
                double *in = bufA, *out = bufB;
                int woff = 2 * e1, win = e1;
                for (int l = 1; l < ne; ++l) {
                    const int wout = m.emb[l];
                    const double *W = Wsm + woff;
                    const double *bb = W + win * wout;
                    const int sk = dp_skip_kind(win, wout);
                    const double *hr = in + lane * LD;
                    for (int o = warp; o < wout; o += NWARPS) {
                        double z = bb[o];
                        for (int q = 0; q < win; ++q) z = fma(hr[q], W[q * wout + o], z);
                        const double t = dp_tanh64(z, m.tanh_tab);
                        const double skip = sk == 2 ? hr[o < win ? o : o - win] : (sk == 1 ? hr[o] : 0.0);
                        out[lane * LD + o] = skip + t;
                    }
                    __syncthreads();
                    woff += win * wout + wout;
                    win = wout;
                    double *tmp = in;
                    in = out;
                    out = tmp;
                }
                // T += R~^T G over the chunk's rows
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int p = tid + u * NTHREADS;
                    if (p < npairs) {
                        const int cc = p / M, mm = p - cc * M;
                        double acc = tacc[u];
#pragma unroll 8
                        for (int r = 0; r < ROWS; ++r) acc = fma(Rt[r * 4 + cc], in[r * LD + mm], acc);
                        tacc[u] = acc;
                    }
                }
                __syncthreads();
            }
        }
        // T (scaled) and D = T_<^T T
        double *Tsm = bufA;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int p = tid + u * NTHREADS;
            if (p < npairs) {
                const double v = tacc[u] * m.desc_scale;
                Tsm[p] = v;
                Tout[(size_t)i * npairs + p] = v;
            }
        }
        __syncthreads();
        const int nd = m.m2 * M;
        for (int q = tid; q < nd; q += NTHREADS) {
            const int a2 = q / M, b2 = q - a2 * M;
            double acc = Tsm[a2] * Tsm[b2];
            acc = fma(Tsm[M + a2], Tsm[M + b2], acc);
            acc = fma(Tsm[2 * M + a2], Tsm[2 * M + b2], acc);
            acc = fma(Tsm[3 * M + a2], Tsm[3 * M + b2], acc);
            Dout[(size_t)i * nd + q] = acc;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(NTHREADS) k_embed_bwd(
    DevModel m, const double *__restrict__ x, const int32_t *__restrict__ types, Box3 box, int N,
    const int32_t *__restrict__ type_perm, const int32_t *__restrict__ nlist,
    const int32_t *__restrict__ nreal, const double *__restrict__ Tin, const double *__restrict__ gD,
    double *__restrict__ pair_g, double *__restrict__ f_own, double *__restrict__ vir_part, int LD,
    int wsz)
{
    extern __shared__ double sm[];
    double *Wsm = sm;
    double *A = Wsm + wsz;                 // value  [32][LD]
    double *dA = A + ROWS * LD;            // tangent
    double *B = dA + ROWS * LD;
    double *dB = B + ROWS * LD;
    double *gTs = dB + ROWS * LD;          // [4][M], scaled by desc_scale
    double *red = gTs + 4 * DP_MAX_EMB_W;  // [NWARPS][32][8]
    double *srow = red + NWARPS * ROWS * 8;  // [32]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int M = m.M, m2 = m.m2, ne = m.n_emb, e1 = m.emb[0], T = m.ntypes, nm = m.nm;
    const int npairs = 4 * M;
    int staged = -1;

    for (int ii = blockIdx.x; ii < N; ii += gridDim.x) {
        const int i = type_perm[ii];
        const int a = types[i];
        const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};

        // gT[c][x] = [x < M2] sum_b gD[x][b] T[c][b] + sum_{a<M2} gD[a][x] T[c][a]
        {
            double *Ts = A;  // T of this atom, [4][M]
            for (int p = tid; p < npairs; p += NTHREADS) Ts[p] = Tin[(size_t)i * npairs + p];
            __syncthreads();
            const double *g = gD + (size_t)i * m2 * M;
            for (int p = tid; p < npairs; p += NTHREADS) {
                const int cc = p / M, xx = p - cc * M;
                double acc = 0.0;
                if (xx < m2)
                    for (int b2 = 0; b2 < M; ++b2) acc = fma(g[xx * M + b2], Ts[cc * M + b2], acc);
                for (int a2 = 0; a2 < m2; ++a2) acc = fma(g[a2 * M + xx], Ts[cc * M + a2], acc);
                gTs[p] = acc * m.desc_scale;
            }
            __syncthreads();
        }

        double fo[3] = {0.0, 0.0, 0.0};
        double vir[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) vir[q] = 0.0;

        const bool a_ok = (unsigned)a < (unsigned)T;  // invalid types are flagged by format
        for (int b = 0; b < T; ++b) {
            const int nb = a_ok ? nreal[(size_t)i * T + b] : 0;
            if (nb == 0) continue;
            const int net = a * T + b;
            if (net != staged) {
                __syncthreads();
                stage_net(m, net, Wsm);
                staged = net;
                __syncthreads();
            }
            for (int c0 = 0; c0 < nb; c0 += ROWS) {
                RowGeom g;  // meaningful in warp 0 only
                const bool valid = c0 + lane < nb;
                int slot = m.sel_off[b] + c0 + lane;
                if (warp == 0) {
                    g.s = g.ds = 0.0;
                    g.R[0] = g.R[1] = g.R[2] = g.R[3] = 0.0;
                    g.d[0] = g.d[1] = g.d[2] = 0.0;
                    g.r = 1.0;
                    if (valid) {
                        const int j = nlist[(size_t)i * nm + slot];
                        row_geometry(m, x, xi, j, box, g);
                    }
                    srow[lane] = g.s;
                }
                __syncthreads();
                // layer 0 with tangent: t = tanh(s W0 + b0), dt/ds = (1 - t^2) W0
                {
                    const double sv = srow[lane];
                    for (int o = warp; o < e1; o += NWARPS) {
                        const double w0 = Wsm[o];
                        const double t = dp_tanh64(fma(sv, w0, Wsm[e1 + o]), m.tanh_tab);
                        A[lane * LD + o] = t;
                        dA[lane * LD + o] = fma(-t, t, 1.0) * w0;
                    }
                }
                __syncthreads();
                double *in = A, *din = dA, *out = B, *dout = dB;
                int woff = 2 * e1, win = e1;
                double ra[4] = {0.0, 0.0, 0.0, 0.0}, rb[4] = {0.0, 0.0, 0.0, 0.0};
                for (int l = 1; l < ne; ++l) {
                    const int wout = m.emb[l];
                    const double *W = Wsm + woff;
                    const double *bb = W + win * wout;
                    const int sk = dp_skip_kind(win, wout);
                    const double *hr = in + lane * LD, *dhr = din + lane * LD;
                    const bool last = (l == ne - 1);
                    for (int o = warp; o < wout; o += NWARPS) {
                        double z = bb[o], dz = 0.0;
                        for (int q = 0; q < win; ++q) {
                            const double w = W[q * wout + o];
                            z = fma(hr[q], w, z);
                            dz = fma(dhr[q], w, dz);
                        }
                        const double t = dp_tanh64(z, m.tanh_tab);
                        const int os = o < win ? o : o - win;
                        const double skip = sk == 2 ? hr[os] : (sk == 1 ? hr[o] : 0.0);
                        const double dskip = sk == 2 ? dhr[os] : (sk == 1 ? dhr[o] : 0.0);
                        const double h = skip + t;
                        const double dh = fma(fma(-t, t, 1.0), dz, dskip);
                        if (last) {
#pragma unroll
                            for (int cc = 0; cc < 4; ++cc) {
                                const double gt = gTs[cc * M + o];
                                ra[cc] = fma(h, gt, ra[cc]);
                                rb[cc] = fma(dh, gt, rb[cc]);
                            }
                        } else {
                            out[lane * LD + o] = h;
                            dout[lane * LD + o] = dh;
                        }
                    }
                    if (!last) {
                        __syncthreads();
                        double *t1 = in, *t2 = din;
                        in = out;
                        din = dout;
                        out = t1;
                        dout = t2;
                    }
                    woff += win * wout + wout;
                    win = wout;
                }
                if (ne == 1) {
                    // G = L_0(s): the layer-0 outputs are the embedding
                    for (int o = warp; o < e1; o += NWARPS) {
                        const double h = A[lane * LD + o], dh = dA[lane * LD + o];
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            const double gt = gTs[cc * M + o];
                            ra[cc] = fma(h, gt, ra[cc]);
                            rb[cc] = fma(dh, gt, rb[cc]);
                        }
                    }
                }
                double *rw = red + (warp * ROWS + lane) * 8;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    rw[cc] = ra[cc];
                    rw[4 + cc] = rb[cc];
                }
                __syncthreads();
                if (warp == 0 && valid) {
                    double sa[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) sa[q] = 0.0;
                    for (int w = 0; w < NWARPS; ++w) {
                        const double *src = red + (w * ROWS + lane) * 8;
#pragma unroll
                        for (int q = 0; q < 8; ++q) sa[q] += src[q];
                    }
                    // dE/dR~ row: gR[c] = sa[c]; the s-dependence of G adds to column 0
                    double gR0 = sa[0];
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) gR0 = fma(g.R[cc], sa[4 + cc], gR0);
                    const double inv = 1.0 / g.r;
                    const double u[3] = {g.d[0] * inv, g.d[1] * inv, g.d[2] * inv};
                    const double dot = sa[1] * u[0] + sa[2] * u[1] + sa[3] * u[2];
                    const double sr = g.s * inv;
                    const double coef = gR0 * g.ds + g.ds * dot - sr * dot;
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
                        for (int bb = 0; bb < 3; ++bb) vir[aa * 3 + bb] -= g.d[aa] * gv[bb];
                    }
                }
                __syncthreads();
            }
        }
        if (warp == 0) {
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
    }
}

int emb_max_width(const DevModel &m)
{
    int w = 0;
    for (int l = 0; l < m.n_emb; ++l) w = m.emb[l] > w ? m.emb[l] : w;
    return w;
}

// Widest layer whose output the backward kernel keeps in shared memory (all
// but the last one, whose columns are contracted with gT as they are made).
int emb_stored_width(const DevModel &m)
{
    if (m.n_emb == 1) return m.emb[0];
    int w = 0;
    for (int l = 0; l + 1 < m.n_emb; ++l) w = m.emb[l] > w ? m.emb[l] : w;
    return w;
}

}  // namespace

cudaError_t dp_launch_embed_fwd(cudaStream_t st, const DevModel &m, const double *x,
                                const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                const NlistBuffers &nb, EvalBuffers eb, int num_sms,
                                int64_t *launches)
{
    const int LD = emb_max_width(m) + 1;
    const int wsz = (m.emb_net_size + 1) & ~1;
    const size_t smem = sizeof(double) * ((size_t)wsz + 2 * ROWS * LD + ROWS * 4 + ROWS);
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_embed_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_embed_fwd, NTHREADS, smem);
    if (per_sm < 1) per_sm = 1;
    int grid = num_sms * per_sm;
    if (grid > N) grid = N;
    if (grid < 1) grid = 1;
    k_embed_fwd<<<grid, NTHREADS, smem, st>>>(m, x, types, box, N, nb.type_perm, fb.nlist, fb.nreal,
                                              eb.T, eb.D, LD, wsz);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t dp_launch_embed_bwd(cudaStream_t st, const DevModel &m, const double *x,
                                const int32_t *types, Box3 box, int N, const FormatBuffers &fb,
                                const NlistBuffers &nb, EvalBuffers eb, int num_sms,
                                int64_t *launches)
{
    // A holds the atom's T (4 x M) in the prologue, so ROWS * LD >= 4M.
    int LD = emb_stored_width(m) + 1;
    if (ROWS * LD < 4 * m.M) LD = (4 * m.M + ROWS - 1) / ROWS;
    const int wsz = (m.emb_net_size + 1) & ~1;
    const size_t smem = sizeof(double) *
                        ((size_t)wsz + 4 * ROWS * LD + 4 * DP_MAX_EMB_W + NWARPS * ROWS * 8 + ROWS);
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_embed_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_embed_bwd, NTHREADS, smem);
    if (per_sm < 1) per_sm = 1;
    int grid = num_sms * per_sm;
    if (grid > N) grid = N;
    if (grid < 1) grid = 1;
    k_embed_bwd<<<grid, NTHREADS, smem, st>>>(m, x, types, box, N, nb.type_perm, fb.nlist, fb.nreal,
                                              eb.T, eb.gD, eb.pair_g, eb.f_own, eb.vir_part, LD, wsz);
    *launches += 1;
    return cudaGetLastError();
}
