// fit.cu -- fitting net N_a (Eqs. fitting, fitting-detail; one net per centre
// type, Remark 1) forward and backward in FP64: E_i = N_a(D_i) and
// gD_i = dE_i/dD_i.
//
// One CTA takes a tile of RT atoms of the same type from the type-sorted atom
// order, so every layer is a small dense GEMM (RT x K) . (K x F).  Weights are
// streamed through shared memory in chunks of KC rows; activations and the
// tanh values of every layer stay in shared memory for the backward pass,
// which applies d tanh = 1 - tanh^2 (Sec. 3.2.3) and the transposed weights.
// Reading of Eq. fitting-detail: the first layer (input width m2*M != f1) is
// plain tanh(x W + b), equal-width layers are x + tanh(x W + b), the output
// layer is linear.
#include "dp_internal.cuh"

namespace {

constexpr int RT = 16;       // atoms per tile (one per thread row)
constexpr int KC = 16;       // weight rows per streamed chunk
constexpr int NTH = 256;     // 16 x 16 threads
constexpr int NJ = DP_MAX_FIT_W / 16;  // output columns per thread

__global__ void __launch_bounds__(NTH, 1) k_fit(
    DevModel m, int N, const int32_t *__restrict__ type_perm, const int32_t *__restrict__ type_start,
    const double *__restrict__ D, double *__restrict__ Ei, double *__restrict__ gD, int LDH, int LDW)
{
    extern __shared__ double sm[];
    double *Xs = sm;                       // [RT][KC + 1]
    double *Ws = Xs + RT * (KC + 1);       // weight chunk, LDW doubles
    double *Hs = Ws + LDW;                 // [RT][LDH] current activation / gradient
    double *Gs = Hs + RT * LDH;            // [RT][LDH] gz of the current layer
    double *Ts = Gs + RT * LDH;            // [n_fit][RT][LDH] tanh values
    __shared__ int rows_atom[RT];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int M = m.M, K1 = m.m2 * M, nf = m.n_fit;

    // tile -> (type, first row)
    int bid = blockIdx.x, a = -1, first = 0, cnt = 0;
    for (int t = 0; t < m.ntypes; ++t) {
        const int n_t = type_start[t + 1] - type_start[t];
        const int tiles = (n_t + RT - 1) / RT;
        if (bid < tiles) {
            a = t;
            first = type_start[t] + bid * RT;
            cnt = min(RT, n_t - bid * RT);
            break;
        }
        bid -= tiles;
    }
    if (a < 0) return;
    if (tid < RT) rows_atom[tid] = tid < cnt ? type_perm[first + tid] : -1;
    __syncthreads();
    const int my_atom = rows_atom[ty];
    const double *P = m.params + m.fit_base[a];

    // ---------------- forward
    double acc[NJ];
    int Kin = K1;
    const double *Wl = P;
    for (int l = 0; l < nf; ++l) {
        const int F = m.fit[l];
        const double *bl = Wl + (size_t)Kin * F;
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) acc[jj] = 0.0;
        for (int k0 = 0; k0 < Kin; k0 += KC) {
            if (l == 0) {
                const int r = tid / KC, kk = tid % KC;  // RT*KC == NTH
                const int at = rows_atom[r];
                Xs[r * (KC + 1) + kk] = (at >= 0 && k0 + kk < Kin) ? D[(size_t)at * K1 + k0 + kk] : 0.0;
            }
            for (int q = tid; q < KC * F; q += NTH) {
                const int kk = q / F, n = q - kk * F;
                Ws[kk * (F + 1) + n] = (k0 + kk < Kin) ? Wl[(size_t)(k0 + kk) * F + n] : 0.0;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < KC; ++kk) {
                const double xv = (l == 0) ? Xs[ty * (KC + 1) + kk]
                                           : (k0 + kk < Kin ? Hs[ty * LDH + k0 + kk] : 0.0);
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) {
                    const int n = tx + 16 * jj;
                    if (n < F) acc[jj] = fma(xv, Ws[kk * (F + 1) + n], acc[jj]);
                }
            }
            __syncthreads();
        }
        const int sk = (l == 0) ? 0 : dp_skip_kind(Kin, F);
        double hnew[NJ];
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
            const int n = tx + 16 * jj;
            hnew[jj] = 0.0;
            if (n < F) {
                const double t = tanh(acc[jj] + bl[n]);
                Ts[(l * RT + ty) * LDH + n] = t;
                const double skip = sk == 2 ? Hs[ty * LDH + (n < Kin ? n : n - Kin)]
                                            : (sk == 1 ? Hs[ty * LDH + n] : 0.0);
                hnew[jj] = skip + t;
            }
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
            const int n = tx + 16 * jj;
            if (n < F) Hs[ty * LDH + n] = hnew[jj];
        }
        __syncthreads();
        Wl = bl + F;
        Kin = F;
    }
    // output layer: E = h . w_out + b_out
    const double *wo = Wl;
    const double bo = wo[Kin];
    {
        double part = 0.0;
        for (int n = tx; n < Kin; n += 16) part = fma(Hs[ty * LDH + n], wo[n], part);
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if (tx == 0 && my_atom >= 0) Ei[my_atom] = part + bo;
    }
    __syncthreads();

    // ---------------- backward: gh = dE/dh of the last hidden layer = w_out
    for (int n = tx; n < Kin; n += 16) Hs[ty * LDH + n] = wo[n];
    __syncthreads();
    // layer offsets (walk forward once)
    const double *Wls[DP_MAX_LAYERS];
    {
        const double *w = P;
        int kin = K1;
        for (int l = 0; l < nf; ++l) {
            Wls[l] = w;
            w += (size_t)kin * m.fit[l] + m.fit[l];
            kin = m.fit[l];
        }
    }
    for (int l = nf - 1; l >= 0; --l) {
        const int F = m.fit[l];
        const int Kl = (l == 0) ? K1 : m.fit[l - 1];
        const double *W = Wls[l];
        // gz = gh * (1 - t^2)
        for (int n = tx; n < F; n += 16) {
            const double t = Ts[(l * RT + ty) * LDH + n];
            Gs[ty * LDH + n] = Hs[ty * LDH + n] * fma(-t, t, 1.0);
        }
        __syncthreads();
        if (l > 0) {
            // gx[q] = sum_n gz[n] W[q][n] + skip(gh)
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) acc[jj] = 0.0;
            for (int n0 = 0; n0 < F; n0 += KC) {
                for (int q = tid; q < Kl * KC; q += NTH) {
                    const int qq = q / KC, nn = q - qq * KC;
                    Ws[qq * (KC + 1) + nn] = (n0 + nn < F) ? W[(size_t)qq * F + n0 + nn] : 0.0;
                }
                __syncthreads();
#pragma unroll 4
                for (int nn = 0; nn < KC; ++nn) {
                    const double gz = (n0 + nn < F) ? Gs[ty * LDH + n0 + nn] : 0.0;
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) {
                        const int q = tx + 16 * jj;
                        if (q < Kl) acc[jj] = fma(gz, Ws[q * (KC + 1) + nn], acc[jj]);
                    }
                }
                __syncthreads();
            }
            const int sk = dp_skip_kind(Kl, F);
            double gnew[NJ];
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) {
                const int q = tx + 16 * jj;
                gnew[jj] = acc[jj];
                if (q < Kl) {
                    if (sk == 1) gnew[jj] += Hs[ty * LDH + q];
                    else if (sk == 2) gnew[jj] += Hs[ty * LDH + q] + Hs[ty * LDH + q + Kl];
                }
            }
            __syncthreads();
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) {
                const int q = tx + 16 * jj;
                if (q < Kl) Hs[ty * LDH + q] = gnew[jj];
            }
            __syncthreads();
        } else {
            // gD[k] = sum_n gz[n] W1[k][n], k < m2*M, in chunks of KC rows of W1
            for (int k0 = 0; k0 < K1; k0 += KC) {
                for (int q = tid; q < KC * F; q += NTH) {
                    const int kk = q / F, n = q - kk * F;
                    Ws[kk * (F + 1) + n] = (k0 + kk < K1) ? W[(size_t)(k0 + kk) * F + n] : 0.0;
                }
                __syncthreads();
                {
                    const int k = k0 + tx;
                    double s = 0.0;
                    for (int n = 0; n < F; ++n) s = fma(Gs[ty * LDH + n], Ws[tx * (F + 1) + n], s);
                    if (my_atom >= 0 && k < K1) gD[(size_t)my_atom * K1 + k] = s;
                }
                __syncthreads();
            }
        }
    }
}

}  // namespace

cudaError_t dp_launch_fit(cudaStream_t st, const DevModel &m, int N, const NlistBuffers &nb,
                          EvalBuffers eb, int64_t *launches)
{
    int maxf = 0;
    for (int l = 0; l < m.n_fit; ++l) maxf = m.fit[l] > maxf ? m.fit[l] : maxf;
    const int LDH = maxf + 1;
    // weight chunk: KC x (F+1) forward, Kl x (KC+1) backward
    const int LDW = (KC * (maxf + 1) > maxf * (KC + 1) ? KC * (maxf + 1) : maxf * (KC + 1));
    const size_t smem = sizeof(double) *
                        ((size_t)RT * (KC + 1) + LDW + 2 * RT * LDH + (size_t)m.n_fit * RT * LDH);
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    const int grid = (N + RT - 1) / RT + m.ntypes;  // upper bound on the per-type tiles
    k_fit<<<grid, NTH, smem, st>>>(m, N, nb.type_perm, nb.type_start, eb.D, eb.Ei, eb.gD, LDH, LDW);
    *launches += 1;
    return cudaGetLastError();
}
