// tanh64.cu -- FP64 tanh for the FP64 kernels: piecewise Taylor polynomials.
//
// tanh(|x|) on [0, 19.125) is split into intervals of width 1/40; on interval
// k (centre c_k = k/40, k = round(40 |x|)) it is the degree-7 Taylor polynomial
//   sum_n a_{k,n} t^n,  t = |x| - c_k,  |t| <= 1/80,
// and tanh(|x|) = 1 beyond (1 - tanh(19.125) < 2^-54, below half the spacing
// of the doubles under 1, so 1 is tanh correctly rounded).  The coefficients come
// from the derivatives of tanh, which are polynomials in T = tanh:
//   d/dx P(T) = P'(T) (1 - T^2),   a_{k,n} = P_n(tanh(c_k)) / n!,
// so each interval needs only tanh(c_k).  The Taylor remainder is bounded by
// (1/80)^8 max|tanh^(8)| / 8! = 1.8e-17 (tanh's nearest singularities are at
// +-i pi/2); on the interval at 0, where tanh is odd, the first neglected term
// is of degree 9, so the relative error there stays near one unit in the last
// place.  Evaluation: one interval index (integer pipe), one subtraction and
// 7 FMAs in FP64 -- about a quarter of the FP64 pipe slots of the library
// tanh.  The table (766 intervals x 9 doubles, 55 KB) is read through L1.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "dp_internal.cuh"

namespace {

__device__ double dp_tanh_table[DP_TANH_NINT * DP_TANH_STRIDE];

std::mutex g_mu;
const double *g_addr[64] = {nullptr};

// a[n] = P_n(T) / n! for n = 0..DP_TANH_NCOEF-1, P_0(T) = T.
void taylor_coeffs(double c, double *a)
{
    const double T = std::tanh(c);
    // polynomial coefficients of P_n in T (degree n + 1)
    std::vector<double> P = {0.0, 1.0};  // P_0 = T
    double fact = 1.0;
    for (int n = 0; n < DP_TANH_NCOEF; ++n) {
        if (n > 0) fact *= n;
        double v = 0.0;
        for (int d = (int)P.size() - 1; d >= 0; --d) v = v * T + P[d];
        a[n] = v / fact;
        // P_{n+1}(T) = P_n'(T) (1 - T^2)
        std::vector<double> dP(P.size() > 1 ? P.size() - 1 : 1, 0.0);
        for (size_t d = 1; d < P.size(); ++d) dP[d - 1] = d * P[d];
        std::vector<double> Q(dP.size() + 2, 0.0);
        for (size_t d = 0; d < dP.size(); ++d) {
            Q[d] += dP[d];
            Q[d + 2] -= dP[d];
        }
        P.swap(Q);
    }
}

}  // namespace

cudaError_t dp_tanh_setup(const double **table)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_addr[dev]) {
        *table = g_addr[dev];
        return cudaSuccess;
    }
    std::vector<double> tab((size_t)DP_TANH_NINT * DP_TANH_STRIDE);
    for (int k = 0; k < DP_TANH_NINT; ++k) {
        const double c = (double)k / DP_TANH_INV_H;
        tab[(size_t)k * DP_TANH_STRIDE] = c;
        taylor_coeffs(c, tab.data() + (size_t)k * DP_TANH_STRIDE + 1);
    }
    e = cudaMemcpyToSymbol(dp_tanh_table, tab.data(), sizeof(double) * tab.size());
    if (e != cudaSuccess) return e;
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, dp_tanh_table);
    if (e != cudaSuccess) return e;
    g_addr[dev] = (const double *)p;
    *table = g_addr[dev];
    return cudaSuccess;
}

namespace {

__global__ void k_tanh64(const double *__restrict__ x, double *__restrict__ y, int64_t n,
                         const double *__restrict__ tab)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = dp_tanh64(x[i], tab);
}

}  // namespace

extern "C" dp_status dp_tanh_f64(const double *x, double *y, int64_t n, void *stream)
{
    if (!x || !y || n < 0) return DP_ERR_ARG;
    const double *tab = nullptr;
    if (dp_tanh_setup(&tab) != cudaSuccess) return DP_ERR_CUDA;
    if (n == 0) return DP_OK;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_tanh64<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, y, n, tab);
    if (cudaGetLastError() != cudaSuccess) return DP_ERR_CUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return DP_ERR_CUDA;
    return DP_OK;
}
