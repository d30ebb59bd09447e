// pgrad.cu -- parameter gradient of   Phi(W) = cE E(W) + sum_i lambda_i . F_i(W)
// in FP64: the gradient of any loss on the energy and the forces, with
// cE = dLoss/dE and lambda = dLoss/dF (Remark 2: F = -grad E, so the force
// term is a mixed second derivative).  For atom i,
//   sum_j lambda_j . dE_i/dr_j = sum_k delta r_ik . dE_i/dr_ik,  delta r_ik = lambda_k - lambda_i,
// the directional derivative of E_i along its neighbour displacements, so
// Phi = sum_i (cE E_i - dE_i) with dE_i the forward tangent of E_i.
//
//   k_pg_tan   per atom: rows R~ and their tangents dR~ = (dR~/dr_ij) delta r_ij,
//              G and dG/ds (embedding net with its s-tangent), T, dT, D, dD.
//   k_pg_fit   per tile of atoms: fitting net primal and tangent forward, then
//              reverse mode of cE E - dE; writes dPhi/dD, dPhi/d(dD) and
//              accumulates the fitting weights' gradient in the CTA's slice.
//   k_pg_emb   per atom: dPhi/dT, dPhi/d(dT), then per row dPhi/dG,
//              dPhi/d(dG) and reverse mode through the recomputed embedding
//              net; weight gradients accumulate in shared memory and are added
//              to the CTA's slice when the net changes.
//   k_pg_reduce sums the slices in a fixed order (reproducible bit for bit).
// G is recomputed in k_pg_emb, never stored.
#include "dp_internal.cuh"

namespace {

constexpr int ROWS = 32;
constexpr int NT = 256;
constexpr int NW = NT / 32;

__device__ __forceinline__ void stage(const double *__restrict__ src, double *dst, int n)
{
    for (int q = threadIdx.x; q < n; q += blockDim.x) dst[q] = src[q];
}

struct PGRow {
    double s, ds, R[4], dR[4];
};

// Row geometry: s, R~ and the tangent dR~ = J (lambda_j - lambda_i), J = dR~/dr_ij.
__device__ __forceinline__ void pg_row(const DevModel &m, const double *__restrict__ x, const double *__restrict__ lam,
                                       const double xi[3], const double li[3], int j, const Box3 &box, PGRow &g)
{
    const double xj[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
    double d[3];
    const double r = dp_pinned_dist(xi, xj, box, d);
    double s, ds;
    dp_switch(r, m.rcut_smth, m.rcut, s, ds);
    const double inv = 1.0 / r;
    const double u[3] = {d[0] * inv, d[1] * inv, d[2] * inv};
    const double dr[3] = {lam[3 * j] - li[0], lam[3 * j + 1] - li[1], lam[3 * j + 2] - li[2]};
    g.s = s;
    g.R[0] = s;
    g.R[1] = s * u[0];
    g.R[2] = s * u[1];
    g.R[3] = s * u[2];
    const double udr = u[0] * dr[0] + u[1] * dr[1] + u[2] * dr[2];
    g.dR[0] = ds * udr;
    for (int a = 0; a < 3; ++a) g.dR[1 + a] = ds * u[a] * udr + s * inv * (dr[a] - u[a] * udr);
    g.ds = g.dR[0];
}

// Embedding layers l >= 1 of the current chunk, value and s-tangent:
// z = h W + b, t = tanh(z), h' = skip(h) + t, dz = dh W, dh' = skip(dh) + (1 - t^2) dz.
// Layer outputs go to per-layer buffers (offsets lo[l]) of H, DH, TT, DZ.
template <bool STORE_ALL>
__device__ __forceinline__ void emb_forward(const DevModel &m, const double *Wsm, double *H, double *DH, double *TT,
                                            double *DZ, int LD, const int *lo, int lane, int warp)
{
    int woff = 2 * m.emb[0], win = m.emb[0];
    for (int l = 1; l < m.n_emb; ++l) {
        const int wout = m.emb[l];
        const double *W = Wsm + woff, *bb = W + win * wout;
        const int sk = dp_skip_kind(win, wout);
        const double *hr = H + lane * LD + lo[l - 1], *dhr = DH + lane * LD + lo[l - 1];
        for (int o = warp; o < wout; o += NW) {
            double z = bb[o], dz = 0.0;
            for (int q = 0; q < win; ++q) {
                const double wq = W[q * wout + o];
                z = fma(hr[q], wq, z);
                dz = fma(dhr[q], wq, dz);
            }
            const double t = dp_tanh64(z, m.tanh_tab);
            const int os = o < win ? o : o - win;
            const double skip = sk == 2 ? hr[os] : (sk == 1 ? hr[o] : 0.0);
            const double dskip = sk == 2 ? dhr[os] : (sk == 1 ? dhr[o] : 0.0);
            H[lane * LD + lo[l] + o] = skip + t;
            DH[lane * LD + lo[l] + o] = fma(fma(-t, t, 1.0), dz, dskip);
            if (STORE_ALL) {
                TT[lane * LD + lo[l] + o] = t;
                DZ[lane * LD + lo[l] + o] = dz;
            }
        }
        __syncthreads();
        woff += win * wout + wout;
        win = wout;
    }
}

__global__ void __launch_bounds__(NT) k_pg_tan(DevModel m, const double *__restrict__ x, const int32_t *__restrict__ types,
                                               Box3 box, int N, const double *__restrict__ lam,
                                               const int32_t *__restrict__ nlist, const int32_t *__restrict__ nreal,
                                               double *__restrict__ Tout, double *__restrict__ dTout,
                                               double *__restrict__ Dout, double *__restrict__ dDout, int LD, int wsz)
{
    extern __shared__ double sm[];
    double *Wsm = sm;
    double *H = Wsm + wsz;            // [32][LD] all layer outputs (value)
    double *DH = H + ROWS * LD;       // [32][LD] tangent wrt s (unit)
    double *Rt = DH + ROWS * LD;      // [32][4]
    double *dRt = Rt + ROWS * 4;      // [32][4]
    double *sv = dRt + ROWS * 4;      // [32] s, then ds
    double *dsv = sv + ROWS;
    double *Ts = dsv + ROWS;          // [4][M]
    double *dTs = Ts + 4 * DP_MAX_EMB_W;
    __shared__ int lo[DP_MAX_LAYERS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int M = m.M, T = m.ntypes, nm = m.nm, e1 = m.emb[0];
    if (tid == 0) {
        int o = 0;
        for (int l = 0; l < m.n_emb; ++l) { lo[l] = o; o += m.emb[l]; }
    }
    const int gl = [&] { int o = 0; for (int l = 0; l + 1 < m.n_emb; ++l) o += m.emb[l]; return o; }();
    int staged = -1;
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
        const int a = types[i];
        const bool a_ok = (unsigned)a < (unsigned)T;
        const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        const double li[3] = {lam[3 * i], lam[3 * i + 1], lam[3 * i + 2]};
        double tacc[2] = {0.0, 0.0}, dtacc[2] = {0.0, 0.0};
        for (int b = 0; b < T; ++b) {
            const int nb = a_ok ? nreal[(size_t)i * T + b] : 0;
            if (nb == 0) continue;
            const int net = a * T + b;
            if (net != staged) {
                __syncthreads();
                stage(m.params + m.emb_base[net], Wsm, m.emb_net_size);
                staged = net;
            }
            __syncthreads();
            for (int c0 = 0; c0 < nb; c0 += ROWS) {
                if (warp == 0) {
                    PGRow g;
                    g.s = g.ds = 0.0;
                    for (int c = 0; c < 4; ++c) g.R[c] = g.dR[c] = 0.0;
                    if (c0 + lane < nb)
                        pg_row(m, x, lam, xi, li, nlist[(size_t)i * nm + m.sel_off[b] + c0 + lane], box, g);
                    for (int c = 0; c < 4; ++c) {
                        Rt[lane * 4 + c] = g.R[c];
                        dRt[lane * 4 + c] = g.dR[c];
                    }
                    sv[lane] = g.s;
                    dsv[lane] = g.ds;
                }
                __syncthreads();
                for (int o = warp; o < e1; o += NW) {
                    const double w0 = Wsm[o];
                    const double t = dp_tanh64(fma(sv[lane], w0, Wsm[e1 + o]), m.tanh_tab);
                    H[lane * LD + o] = t;
                    DH[lane * LD + o] = fma(-t, t, 1.0) * w0;
                }
                __syncthreads();
                emb_forward<false>(m, Wsm, H, DH, nullptr, nullptr, LD, lo, lane, warp);
                // T += R^T G,  dT += dR^T G + R^T (ds dG/ds)
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int p = tid + u * NT;
                    if (p < 4 * M) {
                        const int cc = p / M, mm = p - cc * M;
                        double acc = tacc[u], dacc = dtacc[u];
                        for (int r = 0; r < ROWS; ++r) {
                            const double G = H[r * LD + gl + mm];
                            acc = fma(Rt[r * 4 + cc], G, acc);
                            dacc = fma(dRt[r * 4 + cc], G, dacc);
                            dacc = fma(Rt[r * 4 + cc] * dsv[r], DH[r * LD + gl + mm], dacc);
                        }
                        tacc[u] = acc;
                        dtacc[u] = dacc;
                    }
                }
                __syncthreads();
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int p = tid + u * NT;
            if (p < 4 * M) {
                const double v = tacc[u] * m.desc_scale, dv = dtacc[u] * m.desc_scale;
                Ts[p] = v;
                dTs[p] = dv;
                Tout[(size_t)i * 4 * M + p] = v;
                dTout[(size_t)i * 4 * M + p] = dv;
            }
        }
        __syncthreads();
        const int nd = m.m2 * M;
        for (int q = tid; q < nd; q += NT) {
            const int a2 = q / M, b2 = q - a2 * M;
            double acc = 0.0, dacc = 0.0;
            for (int cc = 0; cc < 4; ++cc) {
                acc = fma(Ts[cc * M + a2], Ts[cc * M + b2], acc);
                dacc = fma(dTs[cc * M + a2], Ts[cc * M + b2], dacc);
                dacc = fma(Ts[cc * M + a2], dTs[cc * M + b2], dacc);
            }
            Dout[(size_t)i * nd + q] = acc;
            dDout[(size_t)i * nd + q] = dacc;
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------- fitting --

constexpr int FRT = 16;                    // atoms per tile
constexpr int FJ = DP_MAX_FIT_W / 16;      // output columns per thread

// Per atom scratch of the fitting pass, FP64, each [n_fit][FW]: tanh values,
// tangent pre-activations, layer outputs and their tangents.
constexpr int FW = DP_MAX_FIT_W;

__global__ void __launch_bounds__(NT, 1) k_pg_fit(DevModel m, int N, const int32_t *__restrict__ type_perm,
                                                  const int32_t *__restrict__ type_start, double cE,
                                                  const double *__restrict__ D, const double *__restrict__ dD,
                                                  double *__restrict__ scr, double *__restrict__ Db,
                                                  double *__restrict__ dDb, double *__restrict__ slices,
                                                  int64_t nparams)
{
    extern __shared__ double sm[];
    double *Hs = sm;                   // [FRT][FW + 1] layer input (value)
    double *dHs = Hs + FRT * (FW + 1); // tangent
    double *Zb = dHs + FRT * (FW + 1); // [FRT][FW + 1] adjoint of z
    double *dZb = Zb + FRT * (FW + 1); // adjoint of dz
    __shared__ int rows_atom[FRT];
    __shared__ int tstart[DP_MAX_TYPES + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int M = m.M, K1 = m.m2 * M, nf = m.n_fit, T = m.ntypes;
    const int LDS = FW + 1;
    double *slice = slices + (size_t)blockIdx.x * nparams;
    if (tid <= T) tstart[tid] = type_start[tid];
    __syncthreads();
    const int lo = (int)(((long long)blockIdx.x * N) / gridDim.x);
    const int hi = (int)(((long long)(blockIdx.x + 1) * N) / gridDim.x);
    for (int first = lo; first < hi;) {
        int a = 0;
        while (a + 1 < T && first >= tstart[a + 1]) ++a;
        const int cnt = min(FRT, min(hi, tstart[a + 1]) - first);
        __syncthreads();
        if (tid < FRT) rows_atom[tid] = tid < cnt ? type_perm[first + tid] : -1;
        __syncthreads();
        const int my = rows_atom[ty];
        const int64_t pbase = m.fit_base[a];
        const double *P = m.params + pbase;
        // layer offsets in the parameter vector
        int64_t Woff[DP_MAX_LAYERS], boff[DP_MAX_LAYERS];
        {
            int64_t o = 0;
            int kin = K1;
            for (int l = 0; l < nf; ++l) {
                Woff[l] = o;
                o += (int64_t)kin * m.fit[l];
                boff[l] = o;
                o += m.fit[l];
                kin = m.fit[l];
            }
        }
        const int64_t wo_off = boff[nf - 1] + m.fit[nf - 1];
        double *sc = scr + (size_t)(my < 0 ? 0 : my) * 4 * DP_MAX_LAYERS * FW;  // t, dz, h, dh per layer
        // ---------------- forward, value and tangent
        int Kin = K1;
        for (int l = 0; l < nf; ++l) {
            const int F = m.fit[l];
            const double *W = P + Woff[l], *bl = P + boff[l];
            double acc[FJ], dacc[FJ];
#pragma unroll
            for (int jj = 0; jj < FJ; ++jj) acc[jj] = dacc[jj] = 0.0;
            for (int k = 0; k < Kin; ++k) {
                double xv = 0.0, dxv = 0.0;
                if (my >= 0) {
                    if (l == 0) {
                        xv = D[(size_t)my * K1 + k];
                        dxv = dD[(size_t)my * K1 + k];
                    } else {
                        xv = Hs[ty * LDS + k];
                        dxv = dHs[ty * LDS + k];
                    }
                }
                const double *wr = W + (size_t)k * F;
#pragma unroll
                for (int jj = 0; jj < FJ; ++jj) {
                    const int n = tx + 16 * jj;
                    if (n < F) {
                        const double wv = __ldg(wr + n);
                        acc[jj] = fma(xv, wv, acc[jj]);
                        dacc[jj] = fma(dxv, wv, dacc[jj]);
                    }
                }
            }
            const int sk = (l == 0) ? 0 : dp_skip_kind(Kin, F);
            double hn[FJ], dhn[FJ];
#pragma unroll
            for (int jj = 0; jj < FJ; ++jj) {
                const int n = tx + 16 * jj;
                hn[jj] = dhn[jj] = 0.0;
                if (n < F && my >= 0) {
                    const double t = dp_tanh64(acc[jj] + bl[n], m.tanh_tab);
                    const double skip = sk == 1 ? Hs[ty * LDS + n] : 0.0;
                    const double dskip = sk == 1 ? dHs[ty * LDS + n] : 0.0;
                    hn[jj] = skip + t;
                    dhn[jj] = fma(fma(-t, t, 1.0), dacc[jj], dskip);
                    sc[(0 * DP_MAX_LAYERS + l) * FW + n] = t;
                    sc[(1 * DP_MAX_LAYERS + l) * FW + n] = dacc[jj];
                    sc[(2 * DP_MAX_LAYERS + l) * FW + n] = hn[jj];
                    sc[(3 * DP_MAX_LAYERS + l) * FW + n] = dhn[jj];
                }
            }
            __syncthreads();
#pragma unroll
            for (int jj = 0; jj < FJ; ++jj) {
                const int n = tx + 16 * jj;
                if (n < F) {
                    Hs[ty * LDS + n] = hn[jj];
                    dHs[ty * LDS + n] = dhn[jj];
                }
            }
            __syncthreads();
            Kin = F;
        }
        // ---------------- reverse of cE E - dE, E = h.wo + bo, dE = dh.wo
        const double *wo = P + wo_off;
        // output weights: d/dwo = sum_rows (cE h - dh); d/dbo = cE * rows
        for (int n = tid; n <= Kin; n += NT) {
            double acc = 0.0;
            for (int r = 0; r < cnt; ++r)
                acc += n < Kin ? (cE * Hs[r * LDS + n] - dHs[r * LDS + n]) : cE;
            slice[pbase + wo_off + n] += acc;
        }
        __syncthreads();
        // adjoints of the last layer's output: hb = cE wo, dhb = -wo (kept in Hs / dHs)
        for (int n = tx; n < Kin; n += 16) {
            Hs[ty * LDS + n] = my >= 0 ? cE * wo[n] : 0.0;
            dHs[ty * LDS + n] = my >= 0 ? -wo[n] : 0.0;
        }
        __syncthreads();
        for (int l = nf - 1; l >= 0; --l) {
            const int F = m.fit[l];
            const int Kl = (l == 0) ? K1 : m.fit[l - 1];
            const double *W = P + Woff[l];
            const int sk = (l == 0) ? 0 : dp_skip_kind(Kl, F);
            // z-adjoints of this layer
            for (int n = tx; n < F; n += 16) {
                double zb = 0.0, dzb = 0.0;
                if (my >= 0) {
                    const double t = sc[(0 * DP_MAX_LAYERS + l) * FW + n];
                    const double dz = sc[(1 * DP_MAX_LAYERS + l) * FW + n];
                    const double one = fma(-t, t, 1.0);
                    const double dtb = dHs[ty * LDS + n];
                    double tb = Hs[ty * LDS + n];
                    dzb = one * dtb;
                    tb = fma(-2.0 * t * dz, dtb, tb);
                    zb = one * tb;
                }
                Zb[ty * LDS + n] = zb;
                dZb[ty * LDS + n] = dzb;
            }
            __syncthreads();
            // weight and bias gradients: W[q][n] += x[q] zb[n] + dx[q] dzb[n] over the tile's rows
            for (int64_t e = tid; e < (int64_t)Kl * F; e += NT) {
                const int q = (int)(e / F), n = (int)(e - (int64_t)q * F);
                double acc = 0.0;
                for (int r = 0; r < cnt; ++r) {
                    const int at = rows_atom[r];
                    double xv, dxv;
                    if (l == 0) {
                        xv = D[(size_t)at * K1 + q];
                        dxv = dD[(size_t)at * K1 + q];
                    } else {
                        const double *sr = scr + (size_t)at * 4 * DP_MAX_LAYERS * FW;
                        xv = sr[(2 * DP_MAX_LAYERS + l - 1) * FW + q];
                        dxv = sr[(3 * DP_MAX_LAYERS + l - 1) * FW + q];
                    }
                    acc = fma(xv, Zb[r * LDS + n], acc);
                    acc = fma(dxv, dZb[r * LDS + n], acc);
                }
                slice[pbase + Woff[l] + e] += acc;
            }
            for (int n = tid; n < F; n += NT) {
                double acc = 0.0;
                for (int r = 0; r < cnt; ++r) acc += Zb[r * LDS + n];
                slice[pbase + boff[l] + n] += acc;
            }
            // input adjoints: xb[q] = sum_n zb[n] W[q][n] + skip,  dxb likewise
            if (l > 0) {
                double nb_[FJ], dnb_[FJ];
#pragma unroll
                for (int jj = 0; jj < FJ; ++jj) {
                    const int q = tx + 16 * jj;
                    double acc = 0.0, dacc = 0.0;
                    if (q < Kl) {
                        const double *wr = W + (size_t)q * F;
                        for (int n = 0; n < F; ++n) {
                            const double wv = __ldg(wr + n);
                            acc = fma(Zb[ty * LDS + n], wv, acc);
                            dacc = fma(dZb[ty * LDS + n], wv, dacc);
                        }
                        if (sk == 1) {
                            acc += Hs[ty * LDS + q];
                            dacc += dHs[ty * LDS + q];
                        }
                    }
                    nb_[jj] = acc;
                    dnb_[jj] = dacc;
                }
                __syncthreads();
#pragma unroll
                for (int jj = 0; jj < FJ; ++jj) {
                    const int q = tx + 16 * jj;
                    if (q < Kl) {
                        Hs[ty * LDS + q] = nb_[jj];
                        dHs[ty * LDS + q] = dnb_[jj];
                    }
                }
            } else {
                // dPhi/dD and dPhi/d(dD)
                for (int k = tx; k < K1; k += 16) {
                    double acc = 0.0, dacc = 0.0;
                    const double *wr = W + (size_t)k * F;
                    for (int n = 0; n < F; ++n) {
                        const double wv = __ldg(wr + n);
                        acc = fma(Zb[ty * LDS + n], wv, acc);
                        dacc = fma(dZb[ty * LDS + n], wv, dacc);
                    }
                    if (my >= 0) {
                        Db[(size_t)my * K1 + k] = acc;
                        dDb[(size_t)my * K1 + k] = dacc;
                    }
                }
            }
            __syncthreads();
        }
        first += cnt;
    }
}

// -------------------------------------------------------------- embedding --

__global__ void __launch_bounds__(NT, 1) k_pg_emb(DevModel m, const double *__restrict__ x,
                                                  const int32_t *__restrict__ types, Box3 box, int N,
                                                  const double *__restrict__ lam, const int32_t *__restrict__ nlist,
                                                  const int32_t *__restrict__ nreal, const double *__restrict__ Tin,
                                                  const double *__restrict__ dTin, const double *__restrict__ Db,
                                                  const double *__restrict__ dDb, double *__restrict__ slices,
                                                  int64_t nparams, double *__restrict__ rowscr, int LD, int wsz)
{
    extern __shared__ double sm[];
    double *Wsm = sm;                  // net weights
    double *ZB = Wsm + wsz;            // [32][maxw] z adjoints of one layer
    double *DZB = ZB + ROWS * DP_MAX_EMB_W;
    double *Rt = DZB + ROWS * DP_MAX_EMB_W;   // [32][4]
    double *dRt = Rt + ROWS * 4;
    double *sv = dRt + ROWS * 4;       // [32]
    double *dsv = sv + ROWS;
    double *Ts = dsv + ROWS;           // [4][M] T, dT, Tb, dTb
    double *dTs = Ts + 4 * DP_MAX_EMB_W;
    double *Tb = dTs + 4 * DP_MAX_EMB_W;
    double *dTb = Tb + 4 * DP_MAX_EMB_W;
    // per-CTA global rows [32][LD]: layer outputs, tangents, tanh values,
    // tangent pre-activations, value and tangent adjoints
    double *H = rowscr + (size_t)blockIdx.x * 6 * ROWS * LD;
    double *DH = H + ROWS * LD;
    double *TT = DH + ROWS * LD;
    double *DZ = TT + ROWS * LD;
    double *AB = DZ + ROWS * LD;
    double *DAB = AB + ROWS * LD;
    __shared__ int lo[DP_MAX_LAYERS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int M = m.M, m2 = m.m2, T = m.ntypes, nm = m.nm, e1 = m.emb[0], ne = m.n_emb;
    if (tid == 0) {
        int o = 0;
        for (int l = 0; l < ne; ++l) { lo[l] = o; o += m.emb[l]; }
    }
    double *slice = slices + (size_t)blockIdx.x * nparams;
    int staged = -1;
    double *Gsm = nullptr;  // gradient of the staged net: the CTA's slice
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
        const int a = types[i];
        const bool a_ok = (unsigned)a < (unsigned)T;
        const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        const double li[3] = {lam[3 * i], lam[3 * i + 1], lam[3 * i + 2]};
        // Tb, dTb from dPhi/dD, dPhi/d(dD) with D = T_<^T T, dD = dT_<^T T + T_<^T dT
        __syncthreads();
        for (int p = tid; p < 4 * M; p += NT) {
            Ts[p] = Tin[(size_t)i * 4 * M + p];
            dTs[p] = dTin[(size_t)i * 4 * M + p];
        }
        __syncthreads();
        {
            const double *db = Db + (size_t)i * m2 * M, *ddb = dDb + (size_t)i * m2 * M;
            for (int p = tid; p < 4 * M; p += NT) {
                const int cc = p / M, xx = p - cc * M;
                double tb = 0.0, dtb = 0.0;
                if (xx < m2)
                    for (int b2 = 0; b2 < M; ++b2) {
                        tb = fma(db[xx * M + b2], Ts[cc * M + b2], tb);
                        tb = fma(ddb[xx * M + b2], dTs[cc * M + b2], tb);
                        dtb = fma(ddb[xx * M + b2], Ts[cc * M + b2], dtb);
                    }
                for (int a2 = 0; a2 < m2; ++a2) {
                    tb = fma(db[a2 * M + xx], Ts[cc * M + a2], tb);
                    tb = fma(ddb[a2 * M + xx], dTs[cc * M + a2], tb);
                    dtb = fma(ddb[a2 * M + xx], Ts[cc * M + a2], dtb);
                }
                Tb[p] = tb * m.desc_scale;    // folds the scale of T = scale R^T G
                dTb[p] = dtb * m.desc_scale;
            }
        }
        __syncthreads();
        for (int b = 0; b < T; ++b) {
            const int nb = a_ok ? nreal[(size_t)i * T + b] : 0;
            if (nb == 0) continue;
            const int net = a * T + b;
            if (net != staged) {
                __syncthreads();
                stage(m.params + m.emb_base[net], Wsm, m.emb_net_size);
                staged = net;
                Gsm = slice + m.emb_base[net];
                __syncthreads();
            }
            for (int c0 = 0; c0 < nb; c0 += ROWS) {
                if (warp == 0) {
                    PGRow g;
                    g.s = g.ds = 0.0;
                    for (int c = 0; c < 4; ++c) g.R[c] = g.dR[c] = 0.0;
                    if (c0 + lane < nb)
                        pg_row(m, x, lam, xi, li, nlist[(size_t)i * nm + m.sel_off[b] + c0 + lane], box, g);
                    for (int c = 0; c < 4; ++c) {
                        Rt[lane * 4 + c] = g.R[c];
                        dRt[lane * 4 + c] = g.dR[c];
                    }
                    sv[lane] = g.s;
                    dsv[lane] = g.ds;
                }
                __syncthreads();
                // forward: value and tangent (now scaled by ds), all layers kept
                for (int o = warp; o < e1; o += NW) {
                    const double w0 = Wsm[o];
                    const double dz = dsv[lane] * w0;
                    const double t = dp_tanh64(fma(sv[lane], w0, Wsm[e1 + o]), m.tanh_tab);
                    H[lane * LD + o] = t;
                    TT[lane * LD + o] = t;
                    DZ[lane * LD + o] = dz;
                    DH[lane * LD + o] = fma(-t, t, 1.0) * dz;
                }
                __syncthreads();
                emb_forward<true>(m, Wsm, H, DH, TT, DZ, LD, lo, lane, warp);
                // adjoints of G and dG:  Gb = R Tb + dR dTb,  dGb = R dTb  (rows past nb have R = dR = 0)
                const int gl = lo[ne - 1];
                for (int o = warp; o < M; o += NW) {
                    double gb = 0.0, dgb = 0.0;
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        gb = fma(Rt[lane * 4 + cc], Tb[cc * M + o], gb);
                        gb = fma(dRt[lane * 4 + cc], dTb[cc * M + o], gb);
                        dgb = fma(Rt[lane * 4 + cc], dTb[cc * M + o], dgb);
                    }
                    AB[lane * LD + gl + o] = gb;
                    DAB[lane * LD + gl + o] = dgb;
                }
                __syncthreads();
                // reverse through layers ne-1 .. 1
                int woff_end = m.emb_net_size;
                for (int l = ne - 1; l >= 1; --l) {
                    const int out = m.emb[l], in = m.emb[l - 1];
                    const int woff = woff_end - out - in * out;  // W_l start
                    const double *W = Wsm + woff;
                    double *gW = Gsm + woff, *gb = gW + in * out;
                    const int sk = dp_skip_kind(in, out);
                    // z adjoints
                    for (int o = warp; o < out; o += NW) {
                        const double t = TT[lane * LD + lo[l] + o], dz = DZ[lane * LD + lo[l] + o];
                        const double one = fma(-t, t, 1.0);
                        const double dtb = DAB[lane * LD + lo[l] + o];
                        double tb = AB[lane * LD + lo[l] + o];
                        const double dzb = one * dtb;
                        tb = fma(-2.0 * t * dz, dtb, tb);
                        ZB[lane * DP_MAX_EMB_W + o] = one * tb;
                        DZB[lane * DP_MAX_EMB_W + o] = dzb;
                    }
                    __syncthreads();
                    // weight gradients (rows in order): gW[q][o] += sum_r h[r][q] zb[r][o] + dh[r][q] dzb[r][o]
                    for (int e = tid; e < in * out; e += NT) {
                        const int q = e / out, o = e - q * out;
                        double acc = gW[e];
                        for (int r = 0; r < ROWS; ++r) {
                            acc = fma(H[r * LD + lo[l - 1] + q], ZB[r * DP_MAX_EMB_W + o], acc);
                            acc = fma(DH[r * LD + lo[l - 1] + q], DZB[r * DP_MAX_EMB_W + o], acc);
                        }
                        gW[e] = acc;
                    }
                    for (int o = tid; o < out; o += NT) {
                        double acc = gb[o];
                        for (int r = 0; r < ROWS; ++r) acc += ZB[r * DP_MAX_EMB_W + o];
                        gb[o] = acc;
                    }
                    // input adjoints
                    for (int q = warp; q < in; q += NW) {
                        double acc = 0.0, dacc = 0.0;
                        for (int o = 0; o < out; ++o) {
                            const double wv = W[q * out + o];
                            acc = fma(ZB[lane * DP_MAX_EMB_W + o], wv, acc);
                            dacc = fma(DZB[lane * DP_MAX_EMB_W + o], wv, dacc);
                        }
                        if (sk == 2) {
                            acc += AB[lane * LD + lo[l] + q] + AB[lane * LD + lo[l] + q + in];
                            dacc += DAB[lane * LD + lo[l] + q] + DAB[lane * LD + lo[l] + q + in];
                        } else if (sk == 1) {
                            acc += AB[lane * LD + lo[l] + q];
                            dacc += DAB[lane * LD + lo[l] + q];
                        }
                        AB[lane * LD + lo[l - 1] + q] = acc;
                        DAB[lane * LD + lo[l - 1] + q] = dacc;
                    }
                    __syncthreads();
                    woff_end = woff;
                }
                // layer 0: z0 = s W0 + b0, dz0 = ds W0
                for (int o = warp; o < e1; o += NW) {
                    const double t = TT[lane * LD + o], dz = DZ[lane * LD + o];
                    const double one = fma(-t, t, 1.0);
                    const double dtb = DAB[lane * LD + o];
                    double tb = AB[lane * LD + o];
                    const double dzb = one * dtb;
                    tb = fma(-2.0 * t * dz, dtb, tb);
                    ZB[lane * DP_MAX_EMB_W + o] = one * tb;
                    DZB[lane * DP_MAX_EMB_W + o] = dzb;
                }
                __syncthreads();
                for (int o = tid; o < e1; o += NT) {
                    double gw = Gsm[o], gb = Gsm[e1 + o];
                    for (int r = 0; r < ROWS; ++r) {
                        gw = fma(sv[r], ZB[r * DP_MAX_EMB_W + o], gw);
                        gw = fma(dsv[r], DZB[r * DP_MAX_EMB_W + o], gw);
                        gb += ZB[r * DP_MAX_EMB_W + o];
                    }
                    Gsm[o] = gw;
                    Gsm[e1 + o] = gb;
                }
                __syncthreads();
            }
        }
    }
}

__global__ void k_pg_reduce(const double *__restrict__ slices, int nslices, int64_t nparams, double *__restrict__ grad)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nparams; p += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < nslices; ++c) acc += slices[(size_t)c * nparams + p];
        grad[p] = acc;
    }
}

}  // namespace

size_t dp_pgrad_fit_scratch(int N) { return (size_t)N * 4 * DP_MAX_LAYERS * FW; }

size_t dp_pgrad_row_scratch(int num_sms) { return (size_t)num_sms * 6 * ROWS * (4 * DP_MAX_EMB_W + 1); }

cudaError_t dp_launch_pgrad(cudaStream_t st, const DevModel &m, int64_t nparams, const double *x, const int32_t *types,
                            Box3 box, int N, const double *lam, double cE, const FormatBuffers &fb,
                            const NlistBuffers &nb, EvalBuffers eb, PGradBuffers pb, int num_sms, double *grad,
                            int64_t *launches)
{
    int maxw = 0, se = 0;
    for (int l = 0; l < m.n_emb; ++l) {
        maxw = m.emb[l] > maxw ? m.emb[l] : maxw;
        se += m.emb[l];
    }
    const int LD = se + 1;
    const int wsz = (m.emb_net_size + 1) & ~1;
    const int grid_emb = num_sms < N ? num_sms : (N > 0 ? N : 1);
    cudaError_t e;
    // slices: one per CTA of k_pg_fit / k_pg_emb (both use num_sms CTAs)
    e = cudaMemsetAsync(pb.slices, 0, sizeof(double) * (size_t)num_sms * nparams, st);
    if (e != cudaSuccess) return e;
    {
        const size_t smem = sizeof(double) * ((size_t)wsz + 2 * ROWS * LD + 2 * ROWS * 4 + 2 * ROWS + 8 * DP_MAX_EMB_W);
        e = cudaFuncSetAttribute(k_pg_tan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_pg_tan<<<grid_emb, NT, smem, st>>>(m, x, types, box, N, lam, fb.nlist, fb.nreal, eb.T, pb.dT, eb.D, pb.dD,
                                             LD, wsz);
    }
    {
        const size_t smem = sizeof(double) * 4 * FRT * (FW + 1);
        e = cudaFuncSetAttribute(k_pg_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int grid = num_sms;
        k_pg_fit<<<grid, NT, smem, st>>>(m, N, nb.type_perm, nb.type_start, cE, eb.D, pb.dD, pb.fit_scr, pb.Db, pb.dDb,
                                         pb.slices, nparams);
    }
    {
        const size_t smem = sizeof(double) * ((size_t)wsz + 2 * ROWS * DP_MAX_EMB_W + 2 * ROWS * 4 + 2 * ROWS +
                                              16 * DP_MAX_EMB_W);
        e = cudaFuncSetAttribute(k_pg_emb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_pg_emb<<<num_sms, NT, smem, st>>>(m, x, types, box, N, lam, fb.nlist, fb.nreal, eb.T, pb.dT, pb.Db, pb.dDb,
                                            pb.slices, nparams, pb.rowscr, LD, wsz);
    }
    k_pg_reduce<<<(int)((nparams + 255) / 256 < 4096 ? (nparams + 255) / 256 : 4096), 256, 0, st>>>(
        pb.slices, num_sms, nparams, grad);
    *launches += 4;
    (void)maxw;
    (void)grid_emb;
    return cudaGetLastError();
}
