// force.cu -- ProdForce / ProdVirial / energy sum (Sec. 3.2.2, Remark 2,
// Remark 4) and the velocity-Verlet kernels (Sec. 4).
//
// Force on atom j:  F_j = sum_k g_jk  -  sum_{i : j in nlist(i)} g_ij,
// with g_ij = dE_i/dr_ij.  The first sum is produced by the embedding backward
// kernel; the second ("j-side" terms, which Remark 4 says cannot be obtained
// from the i-side by Newton's third law) is gathered here without atomics: one
// warp per atom j walks j's candidate list (the candidate relation is
// symmetric), recomputes the sort key that j has in i's formatted list with
// the same pinned arithmetic, and finds it by binary search in i's sorted
// type block.  Every sum runs in a fixed order, so results are reproducible
// run to run.  In a sub-region evaluation (Sec. 3.1) only atoms below nloc
// are centres; the ghost atoms above it collect the j-side increments that
// are sent back to the processes owning them.
#include "dp_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

__global__ void __launch_bounds__(128) k_force_gather(
    DevModel m, const double *__restrict__ x, const int32_t *__restrict__ types, Box3 box, int N,
    int nloc, int cap, const int32_t *__restrict__ cand, const int32_t *__restrict__ ncand,
    const uint64_t *__restrict__ keys, const int32_t *__restrict__ nreal,
    const double *__restrict__ pair_g, const double *__restrict__ f_own, double *__restrict__ force)
{
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= N) return;
    const int nm = m.nm, T = m.ntypes;
    const int tj = types[j];
    const bool centre = j < nloc;
    if ((unsigned)tj >= (unsigned)T) {  // flagged by format; only the own part
        if (lane == 0)
            for (int q = 0; q < 3; ++q) force[3 * j + q] = centre ? f_own[3 * j + q] : 0.0;
        return;
    }
    int off = 0;
#pragma unroll
    for (int a = 0; a < DP_MAX_TYPES; ++a)
        if (a == tj) off = m.sel_off[a];
    const double xj[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
    double f[3] = {0.0, 0.0, 0.0};
    const int n = ncand[j];
    const int32_t *row = cand + (size_t)j * cap;
    for (int p = lane; p < n; p += 32) {
        const int i = row[p];
        if (i >= nloc) continue;  // a ghost is no centre
        const int nb = nreal[(size_t)i * T + tj];
        if (nb == 0) continue;
        const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        double d[3];
        const double r = dp_pinned_dist(xi, xj, box, d);  // r_ij = x_j - x_i, as in i's list
        if (!(r < m.rcut)) continue;
        const uint64_t key = dp_pack_key(tj, r, j);
        const uint64_t *kb = keys + (size_t)i * nm + off;
        int lo = 0, hi = nb;  // search [lo, hi)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (kb[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        if (lo < nb && kb[lo] == key) {
            const double *g = pair_g + ((size_t)i * nm + off + lo) * 3;
            f[0] -= g[0];
            f[1] -= g[1];
            f[2] -= g[2];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        f[0] += __shfl_xor_sync(FULL, f[0], o);
        f[1] += __shfl_xor_sync(FULL, f[1], o);
        f[2] += __shfl_xor_sync(FULL, f[2], o);
    }
    if (lane == 0) {
        force[3 * j + 0] = (centre ? f_own[3 * j + 0] : 0.0) + f[0];
        force[3 * j + 1] = (centre ? f_own[3 * j + 1] : 0.0) + f[1];
        force[3 * j + 2] = (centre ? f_own[3 * j + 2] : 0.0) + f[2];
    }
}

// E = sum E_i and Xi = sum_i vir_i by one CTA in a fixed order (deterministic):
// strided per-thread sums, a fixed shuffle tree per warp, then warp 0 over the
// 32 warp results.
__global__ void __launch_bounds__(1024) k_reduce(int N, const double *__restrict__ Ei,
                                                 const double *__restrict__ vir_part,
                                                 double *__restrict__ energy, double *__restrict__ virial,
                                                 double *__restrict__ atom_energy, int32_t *status)
{
    __shared__ double s[10][32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    double acc[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) acc[q] = 0.0;
    for (int i = t; i < N; i += 1024) {
        const double e = Ei[i];
        acc[0] += e;
        if (atom_energy) atom_energy[i] = e;
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[1 + q] += vir_part[(size_t)i * 9 + q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] += __shfl_xor_sync(FULL, acc[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 10; ++q) s[q][warp] = acc[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < 10; ++q) acc[q] = s[q][lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 10; ++q) acc[q] += __shfl_xor_sync(FULL, acc[q], o);
        if (lane == 0) {
            energy[0] = acc[0];
            bool bad = !isfinite(acc[0]);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                virial[q] = acc[1 + q];
                bad |= !isfinite(acc[1 + q]);
            }
            if (bad) atomicOr(status, DPF_NONFINITE);
        }
    }
}

// v += dt/2 * F/m ; x += dt * v ; wrap x into [0, L) (no wrapping where L = 0)
__global__ void k_kick_drift(int N, double *__restrict__ x, double *__restrict__ v,
                             const double *__restrict__ f, const int32_t *__restrict__ types,
                             const double *__restrict__ inv_mass_conv, double dt, Box3 box)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double c = 0.5 * dt * inv_mass_conv[min(max(types[i], 0), DP_MAX_TYPES - 1)];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double vv = v[3 * i + a] + c * f[3 * i + a];
        v[3 * i + a] = vv;
        double xx = x[3 * i + a] + dt * vv;
        const double L = box.L[a];
        if (L > 0.0) {
            double n = floor(__ddiv_rn(xx, L));
            xx = __dsub_rn(xx, __dmul_rn(L, n));
        }
        x[3 * i + a] = xx;
    }
}

// v += dt/2 * F/m ; per-atom kinetic energy m v^2 / 2 (amu A^2/fs^2)
__global__ void k_kick_thermo(int N, double *__restrict__ v, const double *__restrict__ f,
                              const int32_t *__restrict__ types, const double *__restrict__ inv_mass_conv,
                              const double *__restrict__ mass, double dt, double *__restrict__ ke_part)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int t = min(max(types[i], 0), DP_MAX_TYPES - 1);
    const double c = 0.5 * dt * inv_mass_conv[t];
    double ke = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double vv = v[3 * i + a] + c * f[3 * i + a];
        v[3 * i + a] = vv;
        ke += vv * vv;
    }
    ke_part[i] = 0.5 * mass[t] * ke;
}

#define DP_ACC_CONV 9.648533212e-3   // (eV/A/amu) -> A/fs^2
#define DP_KB 8.617333262e-5         // eV/K

__global__ void __launch_bounds__(1024) k_thermo(int N, const double *__restrict__ ke_part,
                                                 const double *__restrict__ energy,
                                                 const double *__restrict__ virial, double volume,
                                                 double *__restrict__ thermo_row)
{
    __shared__ double s[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    double acc = 0.0;
    for (int i = t; i < N; i += 1024) acc += ke_part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) s[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = s[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (lane == 0) {
            const double ke = acc / DP_ACC_CONV;
            const double dof = 3.0 * (double)N - 3.0;
            thermo_row[0] = energy[0];
            thermo_row[1] = ke;
            thermo_row[2] = 2.0 * ke / (dof * DP_KB);
            thermo_row[3] = (2.0 * ke + virial[0] + virial[4] + virial[8]) / (3.0 * volume);
        }
    }
}

}  // namespace

cudaError_t dp_launch_force(cudaStream_t st, const DevModel &m, const double *x,
                            const int32_t *types, Box3 box, int N, int nloc, int cap,
                            const NlistBuffers &nb, const FormatBuffers &fb, EvalBuffers eb,
                            double *force, int64_t *launches)
{
    k_force_gather<<<(N + 3) / 4, 128, 0, st>>>(m, x, types, box, N, nloc, cap, nb.cand, nb.ncand, fb.keys,
                                                fb.nreal, eb.pair_g, eb.f_own, force);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t dp_launch_reduce(cudaStream_t st, int N, EvalBuffers eb, double *energy,
                             double *virial, double *atom_energy, int32_t *status,
                             int64_t *launches)
{
    k_reduce<<<1, 1024, 0, st>>>(N, eb.Ei, eb.vir_part, energy, virial, atom_energy, status);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t dp_launch_kick_drift(cudaStream_t st, int N, double *x, double *v, const double *f,
                                 const int32_t *types, const double *inv_mass_conv, double dt,
                                 Box3 box, int64_t *launches)
{
    k_kick_drift<<<(N + 255) / 256, 256, 0, st>>>(N, x, v, f, types, inv_mass_conv, dt, box);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t dp_launch_kick_thermo(cudaStream_t st, int N, double *v, const double *f,
                                  const int32_t *types, const double *inv_mass_conv,
                                  const double *mass, double dt, double *ke_part,
                                  int64_t *launches)
{
    k_kick_thermo<<<(N + 255) / 256, 256, 0, st>>>(N, v, f, types, inv_mass_conv, mass, dt, ke_part);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t dp_launch_thermo(cudaStream_t st, int N, const double *ke_part, const double *energy,
                             const double *virial, double volume, double *thermo_row,
                             int64_t *launches)
{
    k_thermo<<<1, 1024, 0, st>>>(N, ke_part, energy, virial, volume, thermo_row);
    *launches += 1;
    return cudaGetLastError();
}
