// fit.cu -- fitting net N_a (Eqs. fitting, fitting-detail; one net per centre
// type, Remark 1) forward and backward in FP64: E_i = N_a(D_i) and
// gD_i = dE_i/dD_i.
//
// Persistent kernel, one CTA per SM: CTA c owns an equal contiguous share of
// the type-sorted atom order and walks it in tiles of up to RT atoms of one
// type, so every layer is a small dense GEMM (RT x K) . (K x F) and all SMs
// finish together.  Weights stream through shared memory in chunks of KC
// rows with cp.async double buffering (the load of chunk c+1 overlaps the
// FMAs on chunk c); activations and each layer's tanh values stay in shared
// memory for the backward pass, which applies d tanh = 1 - tanh^2
// (Sec. 3.2.3) and the transposed weights.  A warp whose two rows are both
// past the end of a ragged tile skips the FMA loops.
// Reading of Eq. fitting-detail: the first layer (input width m2*M != f1) is
// plain tanh(x W + b), equal-width layers are x + tanh(x W + b), the output
// layer is linear.
#include "dp_internal.cuh"

namespace {

constexpr int RT = 16;       // atoms per tile (one per thread row)
constexpr int KC = 16;       // weight rows per streamed chunk
constexpr int NTH = 256;     // 16 x 16 threads
constexpr int NJ = DP_MAX_FIT_W / 16;  // output columns per thread

__device__ __forceinline__ void cp_async8(double *dst, const double *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Forward-layer chunk: rows k0..k0+KC of W[K][F] into buf[KC][F+1] (zeros past K).
__device__ __forceinline__ void load_fwd_chunk(double *buf, const double *__restrict__ W, int K, int F, int k0)
{
    for (int q = threadIdx.x; q < KC * F; q += NTH) {
        const int kk = q / F, n = q - kk * F;
        if (k0 + kk < K) cp_async8(buf + kk * (F + 1) + n, W + (size_t)(k0 + kk) * F + n);
        else buf[kk * (F + 1) + n] = 0.0;
    }
}

// Layer-1 input chunk: D[atom][k0..k0+KC] of the tile's rows into xs[RT][KC+1].
__device__ __forceinline__ void load_x_chunk(double *xs, const double *__restrict__ D, const int *rows_atom,
                                             int K, int k0)
{
    const int r = threadIdx.x / KC, kk = threadIdx.x % KC;  // RT*KC == NTH
    const int at = rows_atom[r];
    if (at >= 0 && k0 + kk < K) cp_async8(xs + r * (KC + 1) + kk, D + (size_t)at * K + k0 + kk);
    else xs[r * (KC + 1) + kk] = 0.0;
}

// Backward-layer chunk: columns n0..n0+KC of W[Kl][F] into buf[Kl][KC+1].
__device__ __forceinline__ void load_bwd_chunk(double *buf, const double *__restrict__ W, int Kl, int F, int n0)
{
    for (int q = threadIdx.x; q < Kl * KC; q += NTH) {
        const int qq = q / KC, nn = q - qq * KC;
        if (n0 + nn < F) cp_async8(buf + qq * (KC + 1) + nn, W + (size_t)qq * F + n0 + nn);
        else buf[qq * (KC + 1) + nn] = 0.0;
    }
}

__global__ void __launch_bounds__(NTH, 1) k_fit(
    DevModel m, int N, const int32_t *__restrict__ type_perm, const int32_t *__restrict__ type_start,
    const double *__restrict__ D, double *__restrict__ Ei, double *__restrict__ gD, int LDH, int LDW)
{
    extern __shared__ double sm[];
    double *Xs = sm;                       // [2][RT][KC + 1]
    double *Ws = Xs + 2 * RT * (KC + 1);   // [2][LDW] weight chunks
    double *Hs = Ws + 2 * LDW;             // [RT][LDH] current activation / gradient
    double *Gs = Hs + RT * LDH;            // [RT][LDH] gz of the current layer
    double *Ts = Gs + RT * LDH;            // [n_fit][RT][LDH] tanh values
    __shared__ int rows_atom[RT];
    __shared__ int tstart[DP_MAX_TYPES + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int M = m.M, K1 = m.m2 * M, nf = m.n_fit, T = m.ntypes;
    if (tid <= T) tstart[tid] = type_start[tid];
    __syncthreads();

    // this CTA's share of the type-sorted order
    const int lo = (int)(((long long)blockIdx.x * N) / gridDim.x);
    const int hi = (int)(((long long)(blockIdx.x + 1) * N) / gridDim.x);

    for (int first = lo; first < hi;) {
        int a = 0;
        while (a + 1 < T && first >= tstart[a + 1]) ++a;
        const int cnt = min(RT, min(hi, tstart[a + 1]) - first);
        __syncthreads();  // previous tile done with rows_atom / smem
        if (tid < RT) rows_atom[tid] = tid < cnt ? type_perm[first + tid] : -1;
        __syncthreads();
        const int my_atom = rows_atom[ty];
        const bool warp_live = (ty & ~1) < cnt;  // rows ty and ty^1 of this warp
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
            const int nch = (Kin + KC - 1) / KC;
            if (l == 0) load_x_chunk(Xs, D, rows_atom, Kin, 0);
            load_fwd_chunk(Ws, Wl, Kin, F, 0);
            cp_async_commit();
            for (int c = 0; c < nch; ++c) {
                const int k0 = c * KC;
                if (c + 1 < nch) {
                    if (l == 0) load_x_chunk(Xs + ((c + 1) & 1) * RT * (KC + 1), D, rows_atom, Kin, k0 + KC);
                    load_fwd_chunk(Ws + ((c + 1) & 1) * LDW, Wl, Kin, F, k0 + KC);
                    cp_async_commit();
                    cp_async_wait_1();
                } else {
                    cp_async_wait_0();
                }
                __syncthreads();
                const double *wb = Ws + (c & 1) * LDW;
                const double *xb = Xs + (c & 1) * RT * (KC + 1);
                if (warp_live) {
#pragma unroll 4
                    for (int kk = 0; kk < KC; ++kk) {
                        const double xv = (l == 0) ? xb[ty * (KC + 1) + kk]
                                                   : (k0 + kk < Kin ? Hs[ty * LDH + k0 + kk] : 0.0);
#pragma unroll
                        for (int jj = 0; jj < NJ; ++jj) {
                            const int n = tx + 16 * jj;
                            if (n < F) acc[jj] = fma(xv, wb[kk * (F + 1) + n], acc[jj]);
                        }
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
                    const double t = dp_tanh64(acc[jj] + bl[n], m.tanh_tab);
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
                const int nch = (F + KC - 1) / KC;
                load_bwd_chunk(Ws, W, Kl, F, 0);
                cp_async_commit();
                for (int c = 0; c < nch; ++c) {
                    const int n0 = c * KC;
                    if (c + 1 < nch) {
                        load_bwd_chunk(Ws + ((c + 1) & 1) * LDW, W, Kl, F, n0 + KC);
                        cp_async_commit();
                        cp_async_wait_1();
                    } else {
                        cp_async_wait_0();
                    }
                    __syncthreads();
                    const double *wb = Ws + (c & 1) * LDW;
                    if (warp_live) {
#pragma unroll 4
                        for (int nn = 0; nn < KC; ++nn) {
                            const double gz = (n0 + nn < F) ? Gs[ty * LDH + n0 + nn] : 0.0;
#pragma unroll
                            for (int jj = 0; jj < NJ; ++jj) {
                                const int q = tx + 16 * jj;
                                if (q < Kl) acc[jj] = fma(gz, wb[q * (KC + 1) + nn], acc[jj]);
                            }
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
                const int nch = (K1 + KC - 1) / KC;
                load_fwd_chunk(Ws, W, K1, F, 0);
                cp_async_commit();
                for (int c = 0; c < nch; ++c) {
                    const int k0 = c * KC;
                    if (c + 1 < nch) {
                        load_fwd_chunk(Ws + ((c + 1) & 1) * LDW, W, K1, F, k0 + KC);
                        cp_async_commit();
                        cp_async_wait_1();
                    } else {
                        cp_async_wait_0();
                    }
                    __syncthreads();
                    const double *wb = Ws + (c & 1) * LDW;
                    if (warp_live) {
                        const int k = k0 + tx;
                        double s = 0.0;
                        for (int n = 0; n < F; ++n) s = fma(Gs[ty * LDH + n], wb[tx * (F + 1) + n], s);
                        if (my_atom >= 0 && k < K1) gD[(size_t)my_atom * K1 + k] = s;
                    }
                    __syncthreads();
                }
            }
        }
        first += cnt;
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
    const size_t smem = sizeof(double) * ((size_t)2 * RT * (KC + 1) + 2 * (size_t)LDW + 2 * RT * LDH +
                                          (size_t)m.n_fit * RT * LDH);
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = sms;
    if (grid > (N + 1) / 2) grid = (N + 1) / 2;  // keep >= 2 atoms per CTA on small systems
    if (grid < 1) grid = 1;
    k_fit<<<grid, NTH, smem, st>>>(m, N, nb.type_perm, nb.type_start, eb.D, eb.Ei, eb.gD, LDH, LDW);
    *launches += 1;
    return cudaGetLastError();
}
