// nlist.cu -- neighbour candidates (cell list with skin) and Algorithm 1
// (formatted neighbour list) on sm_103a.
//
// Candidates: the paper keeps the neighbour list on the CPU (Sec. 3.2.2) and
// updates it every 10-50 steps with a 2 A buffer (Sec. 4).  Here it is built
// on the GPU from a cell list whose cell edge is >= rcut + skin, so the 27
// surrounding cells hold every candidate.  Each atom's candidates are listed
// in a fixed order (cells in stencil order, atoms of a cell by index), so the
// build is deterministic.
//
// Formatting (Algorithm 1 + Sec. 3.2.2): one warp per atom packs every
// candidate into a 64-bit key (type, floor(|r_ij| * 1e8), j) -- the compressed
// element of Sec. 3.2.2 with binary fields instead of decimal ones -- sorts the
// keys with a register bitonic network across the warp, keeps the first sel_a
// keys of each type block and pads the rest with -1.
#include <algorithm>

#include "dp_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double wrap1(double v, double L)
{
    double n = floor(__ddiv_rn(v, L));
    return __dsub_rn(v, __dmul_rn(L, n));
}

// Every build kernel takes a gate: with gate == nullptr it always runs; with a
// device flag it returns at once unless the flag is set (device-side
// conditional rebuild, no host round trip).
#define DP_GATED(gate) \
    if ((gate) != nullptr && *(gate) == 0) return

__global__ void k_zero_cells(int32_t *__restrict__ cell_count, int ncell, const int32_t *gate)
{
    DP_GATED(gate);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) cell_count[c] = 0;
}

// Sets *gate when an atom has moved more than skin/2 (squared: stale2) from
// its position at the last build.
__global__ void k_check_stale(const double *__restrict__ x, const double *__restrict__ xref, int N, Box3 box,
                              double stale2, int32_t *gate)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double d[3];
    const double xr[3] = {xref[3 * i], xref[3 * i + 1], xref[3 * i + 2]};
    const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    const double r = dp_pinned_dist(xr, xi, box, d);
    if (__dmul_rn(r, r) > stale2) *gate = 1;
}

__global__ void k_cell_assign(const double *__restrict__ x, const int32_t *__restrict__ types, int N,
                              int ntypes, Box3 box, int nx, int ny, int nz,
                              int32_t *__restrict__ cell_count, int32_t *__restrict__ atom_cell,
                              int32_t *status, const int32_t *gate)
{
    DP_GATED(gate);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int t = types[i];
    if (t < 0 || t >= ntypes) atomicOr(status, DPF_BAD_TYPE);
    int n[3] = {nx, ny, nz}, c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double w = wrap1(x[3 * i + a], box.L[a]);
        int q = (int)(w / box.L[a] * n[a]);
        c[a] = q < 0 ? 0 : (q >= n[a] ? n[a] - 1 : q);
    }
    int cell = (c[2] * ny + c[1]) * nx + c[0];
    atom_cell[i] = cell;
    atomicAdd(&cell_count[cell], 1);
}

// Exclusive scan of the cell counts by one CTA (ncell is at most a few 10^4).
__global__ void k_cell_scan(const int32_t *__restrict__ cell_count, int ncell,
                            int32_t *__restrict__ cell_start, int32_t *__restrict__ cell_cursor,
                            const int32_t *gate)
{
    DP_GATED(gate);
    __shared__ int32_t part[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int chunk = (ncell + nt - 1) / nt;
    const int b = t * chunk, e = min(ncell, b + chunk);
    int s = 0;
    for (int c = b; c < e; ++c) s += cell_count[c];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int q = 0; q < nt; ++q) {
            int v = part[q];
            part[q] = run;
            run += v;
        }
        cell_start[ncell] = run;
    }
    __syncthreads();
    int run = part[t];
    for (int c = b; c < e; ++c) {
        cell_start[c] = run;
        cell_cursor[c] = 0;
        run += cell_count[c];
    }
}

__global__ void k_cell_fill(const int32_t *__restrict__ atom_cell, int N,
                            const int32_t *__restrict__ cell_start, int32_t *__restrict__ cell_cursor,
                            int32_t *__restrict__ cell_atoms, const int32_t *gate)
{
    DP_GATED(gate);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int c = atom_cell[i];
    int p = atomicAdd(&cell_cursor[c], 1);
    cell_atoms[cell_start[c] + p] = i;
}

// Order each cell's atoms by index (rank sort; cells hold ~10^2 atoms), so the
// candidate order does not depend on the atomics of k_cell_fill.
__global__ void k_cell_sort(const int32_t *__restrict__ cell_start, int ncell,
                            const int32_t *__restrict__ cell_atoms, int32_t *__restrict__ cell_sorted,
                            const int32_t *gate)
{
    DP_GATED(gate);
    int c = blockIdx.x;
    if (c >= ncell) return;
    int b = cell_start[c], e = cell_start[c + 1], n = e - b;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        int v = cell_atoms[b + p], rank = 0;
        for (int q = 0; q < n; ++q) rank += cell_atoms[b + q] < v;
        cell_sorted[b + rank] = v;
    }
}

__device__ __forceinline__ void append_candidate(bool take, int j, int lane, int &n, int cap,
                                                 int32_t *__restrict__ row)
{
    unsigned bal = __ballot_sync(FULL, take);
    int pos = n + __popc(bal & ((1u << lane) - 1u));
    if (take && pos < cap) row[pos] = j;
    n += __popc(bal);
}

// One warp per atom: scan the 27 cells around the atom's cell.
__global__ void __launch_bounds__(128) k_cand_cells(
    const double *__restrict__ x, int N, Box3 box, int nx, int ny, int nz,
    const int32_t *__restrict__ atom_cell, const int32_t *__restrict__ cell_start,
    const int32_t *__restrict__ cell_sorted, double rlist, int cap, int32_t *__restrict__ cand,
    int32_t *__restrict__ ncand, double *__restrict__ xref, int32_t *status, const int32_t *gate)
{
    DP_GATED(gate);
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;
    const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    const int ci = atom_cell[i];
    const int cx = ci % nx, cy = (ci / nx) % ny, cz = ci / (nx * ny);
    int32_t *row = cand + (size_t)i * cap;
    int n = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int qx = (cx + dx + nx) % nx, qy = (cy + dy + ny) % ny, qz = (cz + dz + nz) % nz;
                int c = (qz * ny + qy) * nx + qx;
                int b = cell_start[c], e = cell_start[c + 1];
                for (int p0 = b; p0 < e; p0 += 32) {
                    int p = p0 + lane;
                    bool take = false;
                    int j = -1;
                    if (p < e) {
                        j = cell_sorted[p];
                        if (j != i) {
                            double d[3];
                            const double xj[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
                            double r = dp_pinned_dist(xi, xj, box, d);
                            take = r <= rlist;
                        }
                    }
                    append_candidate(take, j, lane, n, cap, row);
                }
            }
    if (lane == 0) {
        if (n > cap) atomicOr(status, DPF_CAND_OVERFLOW);
        ncand[i] = min(n, cap);
        xref[3 * i] = xi[0];
        xref[3 * i + 1] = xi[1];
        xref[3 * i + 2] = xi[2];
    }
}

// Small boxes (< 3 cells along an axis): every j, in index order.
__global__ void __launch_bounds__(128) k_cand_brute(const double *__restrict__ x, int N, Box3 box,
                                                    double rlist, int cap,
                                                    int32_t *__restrict__ cand,
                                                    int32_t *__restrict__ ncand,
                                                    double *__restrict__ xref, int32_t *status,
                                                    const int32_t *gate)
{
    DP_GATED(gate);
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;
    const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    int32_t *row = cand + (size_t)i * cap;
    int n = 0;
    for (int j0 = 0; j0 < N; j0 += 32) {
        int j = j0 + lane;
        bool take = false;
        if (j < N && j != i) {
            double d[3];
            const double xj[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
            take = dp_pinned_dist(xi, xj, box, d) <= rlist;
        }
        append_candidate(take, j, lane, n, cap, row);
    }
    if (lane == 0) {
        if (n > cap) atomicOr(status, DPF_CAND_OVERFLOW);
        ncand[i] = min(n, cap);
        xref[3 * i] = xi[0];
        xref[3 * i + 1] = xi[1];
        xref[3 * i + 2] = xi[2];
    }
}

// Stable partition of the atoms by type (one CTA): type_perm lists type-0
// atoms in index order, then type-1 atoms, ...; type_start[a] is the offset.
__global__ void k_type_perm(const int32_t *__restrict__ types, int N, int ntypes,
                            int32_t *__restrict__ type_perm, int32_t *__restrict__ type_start,
                            int32_t *status, int32_t *gate)
{
    DP_GATED(gate);
    __shared__ int32_t cnt[DP_MAX_TYPES][1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int chunk = (N + nt - 1) / nt;
    const int b = t * chunk, e = min(N, b + chunk);
    int local[DP_MAX_TYPES];
#pragma unroll
    for (int a = 0; a < DP_MAX_TYPES; ++a) local[a] = 0;
    bool bad = false;
    for (int i = b; i < e; ++i) {
        const int raw = types[i];
        bad |= raw < 0 || raw >= ntypes;
        int ty = min(max(raw, 0), ntypes - 1);
#pragma unroll
        for (int a = 0; a < DP_MAX_TYPES; ++a) local[a] += (a == ty);
    }
    if (bad) atomicOr(status, DPF_BAD_TYPE);
#pragma unroll
    for (int a = 0; a < DP_MAX_TYPES; ++a) cnt[a][t] = local[a];
    __syncthreads();
    if (t < DP_MAX_TYPES) {
        int run = 0;
        for (int q = 0; q < nt; ++q) {
            int v = cnt[t][q];
            cnt[t][q] = run;
            run += v;
        }
        local[0] = run;  // total of type t
    }
    __shared__ int32_t tot[DP_MAX_TYPES];
    if (t < DP_MAX_TYPES) tot[t] = local[0];
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int a = 0; a < ntypes; ++a) {
            type_start[a] = run;
            run += tot[a];
        }
        type_start[ntypes] = run;
    }
    __syncthreads();
    int pos[DP_MAX_TYPES];
    int base = 0;
#pragma unroll
    for (int a = 0; a < DP_MAX_TYPES; ++a) {
        pos[a] = base + cnt[a][t];
        base += (a < ntypes) ? tot[a] : 0;
    }
    for (int i = b; i < e; ++i) {
        int ty = min(max(types[i], 0), ntypes - 1);
#pragma unroll
        for (int a = 0; a < DP_MAX_TYPES; ++a)
            if (a == ty) type_perm[pos[a]++] = i;
    }
    // last kernel of a gated build: every thread has read the gate (the
    // barriers above), so it can be cleared for the next step
    if (gate != nullptr && t == 0) *gate = 0;
}

// ---------------------------------------------------------------- format --

// Bitonic sort of KPL*32 keys held KPL per lane in blocked order
// (element p = lane*KPL + e), ascending.
template <int KPL>
__device__ __forceinline__ void warp_bitonic_sort(uint64_t (&v)[KPL], int lane)
{
    constexpr int NTOT = KPL * 32;
#pragma unroll
    for (int k = 2; k <= NTOT; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= KPL) {
                const int lm = j / KPL;
#pragma unroll
                for (int e = 0; e < KPL; ++e) {
                    const int p = lane * KPL + e;
                    uint64_t o = __shfl_xor_sync(FULL, v[e], lm);
                    const bool up = (p & k) == 0;
                    const bool lower = (p & j) == 0;
                    const bool keep_min = (lower == up);
                    v[e] = keep_min ? (v[e] < o ? v[e] : o) : (v[e] > o ? v[e] : o);
                }
            } else {
#pragma unroll
                for (int e = 0; e < KPL; ++e) {
                    const int pe = e ^ j;
                    if (pe > e) {
                        const int p = lane * KPL + e;
                        const bool up = (p & k) == 0;
                        uint64_t a = v[e], b = v[pe];
                        const bool sw = up ? (a > b) : (a < b);
                        v[e] = sw ? b : a;
                        v[pe] = sw ? a : b;
                    }
                }
            }
        }
    }
}

// One warp per atom.  The candidates within rcut -- L(i) of Sec. 2 -- are
// keyed and compacted into a per-warp shared buffer with ballots, then sorted
// by a KPL*32-wide bitonic network in registers.  In the first pass (retry
// list null) an atom with more than KPL*32 keys is appended to the retry list
// and left to a second launch with a network as wide as the candidate cap.
template <int KPL>
__global__ void __launch_bounds__(128) k_format(
    DevModel m, const double *__restrict__ x, const int32_t *__restrict__ types, Box3 box, int N,
    int cap, double stale2, const int32_t *__restrict__ cand, const int32_t *__restrict__ ncand,
    const double *__restrict__ xref, int32_t *__restrict__ nlist, uint64_t *__restrict__ keys,
    int32_t *__restrict__ nreal, int32_t *status, int32_t *retry_count, int32_t *retry_list, int retry_pass)
{
    constexpr int S = 32 * KPL;
    __shared__ uint64_t kbuf[4][S];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int i;
    if (retry_pass) {
        if (w >= *retry_count) return;
        i = retry_list[w];
    } else {
        if (w >= N) return;
        i = w;
    }
    const int nm = m.nm, T = m.ntypes;
    const double xi[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    const int ncnd = ncand[i];
    if (!retry_pass && lane == 0 && stale2 > 0.0) {
        double d[3];
        const double xr[3] = {xref[3 * i], xref[3 * i + 1], xref[3 * i + 2]};
        double r = dp_pinned_dist(xr, xi, box, d);
        if (r * r > stale2) atomicOr(status, DPF_STALE);
    }
    const int32_t *row = cand + (size_t)i * cap;
    uint64_t *kb = kbuf[wl];
    int n = 0;
    for (int c0 = 0; c0 < ncnd; c0 += 32) {
        const int idx = c0 + lane;
        bool take = false;
        uint64_t key = 0;
        if (idx < ncnd) {
            const int j = row[idx];
            const int tj = types[j];
            if ((unsigned)tj < (unsigned)T) {
                double d[3];
                const double xj[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
                const double r = dp_pinned_dist(xi, xj, box, d);
                if (r <= m.rcut) {
                    take = true;
                    key = dp_pack_key(tj, r, j);
                }
            } else {
                atomicOr(status, DPF_BAD_TYPE);
            }
        }
        const unsigned bal = __ballot_sync(FULL, take);
        const int pos = n + __popc(bal & ((1u << lane) - 1u));
        if (take && pos < S) kb[pos] = key;
        n += __popc(bal);
    }
    if (n > S) {  // cannot happen in the retry pass (S >= cap >= ncand)
        if (lane == 0) {
            const int slot = atomicAdd(retry_count, 1);
            retry_list[slot] = i;
        }
        return;
    }
    __syncwarp();
    uint64_t v[KPL];
#pragma unroll
    for (int e = 0; e < KPL; ++e) {
        const int p = lane * KPL + e;
        v[e] = p < n ? kb[p] : DP_KEY_NONE;
    }
    warp_bitonic_sort<KPL>(v, lane);

    int32_t *nrow = nlist + (size_t)i * nm;
    uint64_t *krow = keys + (size_t)i * nm;
    for (int s = lane; s < nm; s += 32) {
        nrow[s] = -1;
        krow[s] = DP_KEY_NONE;
    }
    __syncwarp();
    // start of each type block in the sorted sequence (start[T] = n)
    int start[DP_MAX_TYPES + 1];
#pragma unroll
    for (int a = 0; a <= DP_MAX_TYPES; ++a) {
        int c = n;
        if (a < T) {
            c = 0;
#pragma unroll
            for (int e = 0; e < KPL; ++e) c += (v[e] != DP_KEY_NONE) && ((int)(v[e] >> 60) < a);
            c = __reduce_add_sync(FULL, c);
        }
        start[a] = c;
    }
    int ovf = 0;
#pragma unroll
    for (int e = 0; e < KPL; ++e) {
        if (v[e] == DP_KEY_NONE) continue;
        const int ta = (int)(v[e] >> 60);
        const int j = (int)(v[e] & 0x3FFFFFFull);
        int st = 0, sel = 0, off = 0;
#pragma unroll
        for (int a = 0; a < DP_MAX_TYPES; ++a)
            if (a == ta) {
                st = start[a];
                sel = m.sel[a];
                off = m.sel_off[a];
            }
        const int rank = lane * KPL + e - st;
        if (rank < sel) {
            nrow[off + rank] = j;
            krow[off + rank] = v[e];
        } else {
            ++ovf;
        }
    }
    if (lane < T) {
        int st = 0, en = 0, sel = 0;
#pragma unroll
        for (int a = 0; a < DP_MAX_TYPES; ++a)
            if (a == lane) {
                st = start[a];
                en = start[a + 1];
                sel = m.sel[a];
            }
        nreal[(size_t)i * T + lane] = min(en - st, sel);
    }
    ovf = __reduce_add_sync(FULL, ovf);
    if (lane == 0 && ovf) atomicOr(status, DPF_SEL_OVERFLOW);
}

}  // namespace

cudaError_t dp_launch_build(cudaStream_t st, const DevModel &m, const double *x, const int32_t *types,
                            Box3 box, int N, double rlist, int cap, int nc[3], NlistBuffers nb,
                            int32_t *status, int32_t *gate, int64_t *launches)
{
    const int TB = 256;
    const bool cells = nc[0] >= 3 && nc[1] >= 3 && nc[2] >= 3;
    const int wblocks = (N + 3) / 4;  // 4 warps (atoms) per 128-thread CTA
    if (cells) {
        const int ncell = nc[0] * nc[1] * nc[2];
        k_zero_cells<<<(ncell + TB - 1) / TB, TB, 0, st>>>(nb.cell_count, ncell, gate);
        k_cell_assign<<<(N + TB - 1) / TB, TB, 0, st>>>(x, types, N, m.ntypes, box, nc[0], nc[1], nc[2],
                                                        nb.cell_count, nb.atom_cell, status, gate);
        k_cell_scan<<<1, 1024, 0, st>>>(nb.cell_count, ncell, nb.cell_start, nb.cell_cursor, gate);
        k_cell_fill<<<(N + TB - 1) / TB, TB, 0, st>>>(nb.atom_cell, N, nb.cell_start, nb.cell_cursor,
                                                      nb.cell_atoms, gate);
        k_cell_sort<<<ncell, 128, 0, st>>>(nb.cell_start, ncell, nb.cell_atoms, nb.cell_sorted, gate);
        k_cand_cells<<<wblocks, 128, 0, st>>>(x, N, box, nc[0], nc[1], nc[2], nb.atom_cell,
                                              nb.cell_start, nb.cell_sorted, rlist, cap, nb.cand,
                                              nb.ncand, nb.xref, status, gate);
        *launches += 6;
    } else {
        k_cand_brute<<<wblocks, 128, 0, st>>>(x, N, box, rlist, cap, nb.cand, nb.ncand, nb.xref,
                                              status, gate);
        *launches += 1;
    }
    k_type_perm<<<1, 1024, 0, st>>>(types, N, m.ntypes, nb.type_perm, nb.type_start, status, gate);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t dp_launch_type_perm(cudaStream_t st, const DevModel &m, const int32_t *types, int n,
                                NlistBuffers nb, int32_t *status, int64_t *launches)
{
    k_type_perm<<<1, 1024, 0, st>>>(types, n, m.ntypes, nb.type_perm, nb.type_start, status, nullptr);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t dp_launch_check_stale(cudaStream_t st, const double *x, const double *xref, int N, Box3 box,
                                  double stale2, int32_t *gate, int64_t *launches)
{
    k_check_stale<<<(N + 255) / 256, 256, 0, st>>>(x, xref, N, box, stale2, gate);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t dp_launch_format(cudaStream_t st, const DevModel &m, const double *x,
                             const int32_t *types, Box3 box, int N, int cap, int sort_small, double skin,
                             NlistBuffers nb, FormatBuffers fb, int32_t *status, int32_t *retry,
                             int64_t *launches)
{
    const int blocks = (N + 3) / 4;
    const double stale2 = skin > 0.0 ? 0.25 * skin * skin : 0.0;
    cudaMemsetAsync(retry, 0, sizeof(int32_t), st);
#define DP_FMT(K, RP)                                                                                  \
    k_format<K><<<blocks, 128, 0, st>>>(m, x, types, box, N, cap, stale2, nb.cand, nb.ncand, nb.xref,  \
                                        fb.nlist, fb.keys, fb.nreal, status, retry, retry + 1, RP)
    // first pass: network of sort_small keys
    switch (sort_small) {
    case 64: DP_FMT(2, 0); break;
    case 128: DP_FMT(4, 0); break;
    case 256: DP_FMT(8, 0); break;
    case 512: DP_FMT(16, 0); break;
    default: DP_FMT(32, 0); break;
    }
    // second pass for the atoms the first one could not hold (returns at once when none)
    if (sort_small < cap) {
        if (cap <= 128) DP_FMT(4, 1);
        else if (cap <= 256) DP_FMT(8, 1);
        else if (cap <= 512) DP_FMT(16, 1);
        else DP_FMT(32, 1);
        *launches += 1;
    }
#undef DP_FMT
    *launches += 1;
    return cudaGetLastError();
}
