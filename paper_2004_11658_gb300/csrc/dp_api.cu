// dp_api.cu -- host runtime behind the C ABI of include/dp.h: model and
// context objects, scratch memory, argument checks, the launch sequence of one
// evaluation and of velocity-Verlet MD, and the device status word.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dp_internal.cuh"

namespace {

thread_local std::string g_last_error = "";

bool is_mixed(int32_t precision) { return precision == DP_PREC_MIXED || precision == DP_PREC_MIXED_SPLIT; }

dp_status fail(dp_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

dp_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(DP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define DP_CUDA(call, where)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);   \
    } while (0)

const double kAccConv = 9.648533212e-3;  // (eV/A/amu) -> A/fs^2

int64_t desc_nparams(const dp_model_desc &d)
{
    const int T = d.ntypes;
    int64_t emb = 0;
    int prev = 1;
    for (int l = 0; l < d.n_emb; ++l) {
        emb += (int64_t)prev * d.emb[l] + d.emb[l];
        prev = d.emb[l];
    }
    const int M = d.emb[d.n_emb - 1];
    int64_t fit = 0;
    prev = d.m2 * M;
    for (int l = 0; l < d.n_fit; ++l) {
        fit += (int64_t)prev * d.fit[l] + d.fit[l];
        prev = d.fit[l];
    }
    fit += prev + 1;
    return (int64_t)T * T * emb + (int64_t)T * fit;
}

dp_status check_desc(const dp_model_desc *d)
{
    if (!d) return fail(DP_ERR_ARG, "descriptor is NULL");
    if (d->ntypes < 1 || d->ntypes > DP_MAX_TYPES) return fail(DP_ERR_UNSUPPORTED, "ntypes must be in [1, 8]");
    int nm = 0;
    for (int a = 0; a < d->ntypes; ++a) {
        if (d->sel[a] < 0) return fail(DP_ERR_ARG, "sel must be >= 0");
        nm += d->sel[a];
    }
    if (nm < 1 || nm > DP_MAX_NM) return fail(DP_ERR_UNSUPPORTED, "sum(sel) must be in [1, 1024]");
    if (d->n_emb < 1 || d->n_emb > DP_MAX_LAYERS) return fail(DP_ERR_UNSUPPORTED, "n_emb must be in [1, 4]");
    for (int l = 0; l < d->n_emb; ++l)
        if (d->emb[l] < 1 || d->emb[l] > DP_MAX_EMB_W)
            return fail(DP_ERR_UNSUPPORTED, "embedding widths must be in [1, 128]");
    const int M = d->emb[d->n_emb - 1];
    if (d->m2 < 1 || d->m2 > M) return fail(DP_ERR_ARG, "m2 must be in [1, M]");
    if (d->n_fit < 1 || d->n_fit > DP_MAX_LAYERS) return fail(DP_ERR_UNSUPPORTED, "n_fit must be in [1, 4]");
    for (int l = 0; l < d->n_fit; ++l)
        if (d->fit[l] < 1 || d->fit[l] > DP_MAX_FIT_W)
            return fail(DP_ERR_UNSUPPORTED, "fitting widths must be in [1, 256]");
    if (d->fit[0] == d->m2 * M || d->fit[0] == 2 * d->m2 * M)
        return fail(DP_ERR_UNSUPPORTED, "a skip connection on the first fitting layer is not supported");
    if (d->desc_scale_nm != 0 && d->desc_scale_nm != 1) return fail(DP_ERR_ARG, "desc_scale_nm must be 0 or 1");
    {
        // shared memory of the fitting kernel: chunks, activations and one
        // tanh buffer per layer (16 atoms x (max width + 1) doubles each)
        int maxf = 0;
        for (int l = 0; l < d->n_fit; ++l) maxf = d->fit[l] > maxf ? d->fit[l] : maxf;
        const long ldw = 16L * (maxf + 1) > 17L * maxf ? 16L * (maxf + 1) : 17L * maxf;
        const long bytes = 8L * (2 * 16 * 17 + 2 * ldw + (2L + d->n_fit) * 16 * (maxf + 1));
        if (bytes > 227L * 1024)
            return fail(DP_ERR_UNSUPPORTED, "fitting net too wide/deep for the fitting kernel's shared memory");
    }
    if (!(d->rcut > 0.0) || !(d->rcut_smth >= 0.0) || !(d->rcut_smth < d->rcut))
        return fail(DP_ERR_ARG, "need 0 <= rcut_smth < rcut");
    return DP_OK;
}

}  // namespace

struct dp_model {
    dp_model_desc desc;
    int64_t nparams;
    double *d_params;
    double *h_params;
    int64_t version;  // incremented by dp_model_set_params
    DevModel dev;
};

struct dp_ctx {
    const dp_model *model;
    DevModel m;
    int64_t natoms_max;
    int32_t cap_fixed, cap;
    int32_t precision;
    cudaStream_t stream;
    int num_sms;
    int sync;
    int64_t launches;
    // device status word + pinned host mirror
    int32_t *d_status;
    int32_t *d_gate;   // conditional-rebuild flag (0 between steps)
    int32_t *d_retry;  // Algorithm 1 second-pass list: count, then atoms
    int sort_small;    // width of the first-pass sorting network
    int32_t *h_status;
    // neighbour candidates
    NlistBuffers nb;
    int64_t ncell_cap;
    int nc[3];
    bool nlist_valid;
    int64_t nlist_N;
    int64_t perm_n;    // centres covered by nb.type_perm (-1: unknown)
    double skin;
    FormatBuffers fb;
    EvalBuffers eb;
    double *d_energy, *d_virial;
    // MD state
    double *md_force, *ke_part, *d_inv_mass_conv, *d_mass, *h_mass_stage;
    double last_mass[DP_MAX_TYPES];
    // parameter gradient scratch (allocated on first use)
    PGradBuffers pb;
    // FP64 fitting net on the tensor cores (exact splitting): weight digits
    // (made from the model's parameters of version oz_version) and scratch
    bool use_oz;
    OzModel oz;
    OzBuffers ob;
    uint16_t *d_oz_w;
    int32_t *d_oz_e;
    int64_t oz_w_elems, oz_e_elems, oz_version;
    // FP64 embedding kernels with layers 1 and 2 on the tensor cores: weight digits per net
    bool use_ex;
    unsigned char *d_ex_w;
    int64_t ex_version;
    // mixed precision: BF16 / FP32 copies of the parameters
    MixedModel mx;
    float *d_p32;
    unsigned char *d_emb_ops, *d_fit_fwd, *d_fit_bwd, *d_dtile;
    bool md_force_valid;
    int64_t md_N;
    int64_t md_step;
    // kernel-group timing
    bool timing;
    std::vector<cudaEvent_t> events;
    size_t events_used;
    struct Span {
        size_t a, b;
        int group;
    };
    std::vector<Span> spans;
    double group_ms[DP_KERNEL_GROUPS];
    int64_t group_launches[DP_KERNEL_GROUPS];
};

namespace {

template <class T>
dp_status dev_alloc(T **p, size_t count, const char *what)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(DP_ERR_NOMEM, std::string("cudaMalloc failed for ") + what);
    }
    return DP_OK;
}

void dev_free(void *p)
{
    if (p) cudaFree(p);
}

DevModel make_devmodel(const dp_model_desc &d, const double *dparams)
{
    DevModel m;
    std::memset(&m, 0, sizeof(m));
    m.ntypes = d.ntypes;
    m.nm = 0;
    for (int a = 0; a < d.ntypes; ++a) {
        m.sel[a] = d.sel[a];
        m.sel_off[a] = m.nm;
        m.nm += d.sel[a];
    }
    m.n_emb = d.n_emb;
    for (int l = 0; l < d.n_emb; ++l) m.emb[l] = d.emb[l];
    m.M = d.emb[d.n_emb - 1];
    m.m2 = d.m2;
    m.n_fit = d.n_fit;
    for (int l = 0; l < d.n_fit; ++l) m.fit[l] = d.fit[l];
    m.rcut = d.rcut;
    m.rcut_smth = d.rcut_smth;
    m.desc_scale = d.desc_scale_nm ? 1.0 / (double)m.nm : 1.0;
    m.params = dparams;
    int64_t net = 2 * d.emb[0];
    for (int l = 1; l < d.n_emb; ++l) net += (int64_t)d.emb[l - 1] * d.emb[l] + d.emb[l];
    m.emb_net_size = (int)net;
    int64_t off = 0;
    for (int a = 0; a < d.ntypes; ++a)
        for (int b = 0; b < d.ntypes; ++b) {
            m.emb_base[a * d.ntypes + b] = off;
            off += net;
        }
    for (int a = 0; a < d.ntypes; ++a) {
        m.fit_base[a] = off;
        int prev = d.m2 * m.M;
        for (int l = 0; l < d.n_fit; ++l) {
            off += (int64_t)prev * d.fit[l] + d.fit[l];
            prev = d.fit[l];
        }
        off += prev + 1;
    }
    return m;
}

dp_status read_box(const double *box, Box3 &b)
{
    if (!box) return fail(DP_ERR_ARG, "box is NULL");
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            if (r != c && box[3 * r + c] != 0.0)
                return fail(DP_ERR_BOX, "only orthorhombic (diagonal) cells are supported");
    for (int a = 0; a < 3; ++a) {
        b.L[a] = box[4 * a];
        if (!(b.L[a] > 0.0) || !std::isfinite(b.L[a])) return fail(DP_ERR_BOX, "cell edges must be positive");
    }
    return DP_OK;
}

dp_status finish(dp_ctx *c)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (!c->sync) return DP_OK;
    return dp_ctx_status(c);
}

enum { G_BUILD = 0, G_FORMAT, G_EMBED_FWD, G_FIT, G_EMBED_BWD, G_FORCE, G_REDUCE, G_MD };

// float -> bfloat16 bits, round to nearest even (NaN kept quiet)
uint16_t to_bf16(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// element offset of (row, k) in the tensor-core K-major layout with K columns
size_t kofs(int row, int k, int K)
{
    return (size_t)(row >> 3) * K * 8 + (size_t)(k >> 3) * 64 + (size_t)(row & 7) * 8 + (size_t)(k & 7);
}

int pad_to(int v, int q) { return (v + q - 1) / q * q; }

// BF16 operands of the tensor-core kernels and an FP32 copy of every
// parameter, built once per context from the model's host parameters.
dp_status build_mixed(dp_ctx *c)
{
    const dp_model *md = c->model;
    const DevModel &m = c->m;
    const double *P = md->h_params;
    const int T = m.ntypes, e1 = m.emb[0], e2 = m.emb[1], e3 = m.emb[2];
    const int K1p = pad_to(e1, 16), N1p = pad_to(e2, 16), K2p = N1p, N2p = pad_to(e3, 16);
    MixedModel &mx = c->mx;
    std::memset(&mx, 0, sizeof(mx));
    // embedding: per net W1^T [N1p][K1p] and its low part, W2^T [N2p][K2p] and its
    // low part (hi = the BF16 value, lo = the BF16 value of the remainder w - hi)
    const size_t b1 = (size_t)N1p * K1p, b2 = (size_t)N2p * K2p;
    const size_t net_elems = pad_to((int)(2 * b1 + 2 * b2), 128);
    std::vector<uint16_t> emb((size_t)T * T * net_elems, 0);
    auto split_store = [](uint16_t *hi, uint16_t *lo, size_t at, double w) {
        const uint16_t h = to_bf16((float)w);
        const uint32_t u = (uint32_t)h << 16;
        float hf;
        std::memcpy(&hf, &u, 4);
        hi[at] = h;
        lo[at] = to_bf16((float)(w - (double)hf));
    };
    for (int net = 0; net < T * T; ++net) {
        const double *W1 = P + m.emb_base[net] + 2 * e1;
        const double *W2 = W1 + (size_t)e1 * e2 + e2;
        uint16_t *o1 = emb.data() + net * net_elems, *o1l = o1 + b1, *o2 = o1l + b1, *o2l = o2 + b2;
        for (int n = 0; n < e2; ++n)
            for (int k = 0; k < e1; ++k) split_store(o1, o1l, kofs(n, k, K1p), W1[(size_t)k * e2 + n]);
        for (int n = 0; n < e3; ++n)
            for (int k = 0; k < e2; ++k) split_store(o2, o2l, kofs(n, k, K2p), W2[(size_t)k * e3 + n]);
        mx.emb_off[net][0] = (int64_t)(net * net_elems) * 2;
        mx.emb_off[net][1] = (int64_t)(net * net_elems + 2 * b1) * 2;
    }
    mx.split = c->precision == DP_PREC_MIXED_SPLIT ? 1 : 0;
    // fitting: per type and layer, W^T (forward) and W (backward), K-chunks of 64
    const int K1 = m.m2 * m.M;
    std::vector<uint16_t> fwd, bwd;
    for (int a = 0; a < T; ++a) {
        const double *W = P + m.fit_base[a];
        int kin = K1;
        for (int l = 0; l < m.n_fit; ++l) {
            const int F = m.fit[l];
            const int Np = pad_to(F, 16), Kp = pad_to(kin, 64), Kinp = pad_to(kin, 16), Fp = pad_to(F, 64);
            mx.fit_np[l] = Np;
            mx.fit_kp[l] = Kp;
            mx.fit_kinp[l] = Kinp;
            mx.fit_fp[l] = Fp;
            size_t f0 = fwd.size(), g0 = bwd.size();
            fwd.resize(f0 + (size_t)Kp * Np, 0);
            bwd.resize(g0 + (size_t)Fp * Kinp, 0);
            mx.fit_fwd_off[a][l] = (int64_t)f0 * 2;
            mx.fit_bwd_off[a][l] = (int64_t)g0 * 2;
            for (int k = 0; k < kin; ++k)
                for (int n = 0; n < F; ++n) {
                    const uint16_t v = to_bf16((float)W[(size_t)k * F + n]);
                    fwd[f0 + (size_t)(k / 64) * Np * 64 + kofs(n, k % 64, 64)] = v;   // element (n, k) of W^T
                    bwd[g0 + (size_t)(n / 64) * Kinp * 64 + kofs(k, n % 64, 64)] = v;  // element (k, n) of W
                }
            W += (size_t)kin * F + F;
            kin = F;
        }
    }
    std::vector<float> p32((size_t)md->nparams);
    for (int64_t q = 0; q < md->nparams; ++q) p32[q] = (float)P[q];
    dp_status s = DP_OK;
    if ((s = dev_alloc(&c->d_p32, p32.size(), "fp32 params"))) return s;
    if ((s = dev_alloc(&c->d_emb_ops, emb.size() * 2, "bf16 embedding operands"))) return s;
    if ((s = dev_alloc(&c->d_fit_fwd, fwd.size() * 2, "bf16 fitting operands"))) return s;
    if ((s = dev_alloc(&c->d_fit_bwd, bwd.size() * 2, "bf16 fitting operands"))) return s;
    DP_CUDA(cudaMemcpy(c->d_p32, p32.data(), p32.size() * 4, cudaMemcpyHostToDevice), "mixed operands");
    DP_CUDA(cudaMemcpy(c->d_emb_ops, emb.data(), emb.size() * 2, cudaMemcpyHostToDevice), "mixed operands");
    DP_CUDA(cudaMemcpy(c->d_fit_fwd, fwd.data(), fwd.size() * 2, cudaMemcpyHostToDevice), "mixed operands");
    DP_CUDA(cudaMemcpy(c->d_fit_bwd, bwd.data(), bwd.size() * 2, cudaMemcpyHostToDevice), "mixed operands");
    mx.p32 = c->d_p32;
    mx.emb_ops = c->d_emb_ops;
    mx.fit_fwd = c->d_fit_fwd;
    mx.fit_bwd = c->d_fit_bwd;
    (void)K2p;
    return DP_OK;
}

dp_status flush_spans(dp_ctx *c)
{
    if (c->spans.empty()) return DP_OK;
    DP_CUDA(cudaStreamSynchronize(c->stream), "timing");
    for (const auto &sp : c->spans) {
        float ms = 0.f;
        DP_CUDA(cudaEventElapsedTime(&ms, c->events[sp.a], c->events[sp.b]), "timing");
        c->group_ms[sp.group] += ms;
    }
    c->spans.clear();
    c->events_used = 0;
    return DP_OK;
}

// Records an event before a launch group and another after it (timing on only).
struct GroupTimer {
    dp_ctx *c;
    int group;
    size_t a;
    int64_t before;
    GroupTimer(dp_ctx *c_, int g) : c(c_), group(g), a(0), before(c_->launches)
    {
        if (c->timing) a = next_event();
    }
    size_t next_event()
    {
        if (c->events_used + 2 > 65536) flush_spans(c);
        if (c->events_used >= c->events.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            c->events.push_back(e);
        }
        size_t k = c->events_used++;
        cudaEventRecord(c->events[k], c->stream);
        return k;
    }
    ~GroupTimer()
    {
        c->group_launches[group] += c->launches - before;
        if (c->timing) c->spans.push_back({a, next_event(), group});
    }
};

int default_cap(const dp_ctx *c, const Box3 &b, int64_t N, double rlist)
{
    const double vol = b.L[0] * b.L[1] * b.L[2];
    const double rho = (double)N / vol;
    const double expect = rho * 4.0 / 3.0 * M_PI * rlist * rlist * rlist;
    int cap = (int)std::ceil((1.5 * expect + 64.0) / 32.0) * 32;
    if (cap > (int)N) cap = (int)((N + 31) / 32 * 32);
    if (cap < 32) cap = 32;
    if (cap > 1024) cap = 1024;
    (void)c;
    return cap;
}

dp_status check_common(dp_ctx *c, const double *coords, const int32_t *types, int64_t N)
{
    if (!c) return fail(DP_ERR_ARG, "context is NULL");
    if (!coords || !types) return fail(DP_ERR_ARG, "coords/types is NULL");
    if (N < 1 || N > c->natoms_max) return fail(DP_ERR_ARG, "N must be in [1, natoms_max]");
    return DP_OK;
}

dp_status do_build(dp_ctx *c, const double *coords, const int32_t *types, const Box3 &b, int64_t N,
                   double skin, bool gated = false)
{
    if (!(skin >= 0.0)) return fail(DP_ERR_ARG, "skin must be >= 0");
    const double rlist = c->m.rcut + skin;
    for (int a = 0; a < 3; ++a)
        if (b.L[a] < 2.0 * rlist)
            return fail(DP_ERR_BOX, "every cell edge must be >= 2 (rcut + skin)");
    // candidate capacity
    int cap = c->cap_fixed > 0 ? c->cap_fixed : default_cap(c, b, N, rlist);
    if (cap > c->cap || c->nb.cand == nullptr) {
        dev_free(c->nb.cand);
        c->nb.cand = nullptr;
        dp_status s = dev_alloc(&c->nb.cand, (size_t)c->natoms_max * cap, "candidates");
        if (s) return s;
        c->cap = cap;
    }
    // cells
    int nc[3];
    int64_t ncell = 1;
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)std::floor(b.L[a] / rlist);
        if (nc[a] < 1) nc[a] = 1;
        if (nc[a] > 1024) nc[a] = 1024;
        ncell *= nc[a];
    }
    if (nc[0] >= 3 && nc[1] >= 3 && nc[2] >= 3 && ncell > c->ncell_cap) {
        dev_free(c->nb.cell_count);
        dev_free(c->nb.cell_start);
        dev_free(c->nb.cell_cursor);
        c->nb.cell_count = c->nb.cell_start = c->nb.cell_cursor = nullptr;
        dp_status s;
        if ((s = dev_alloc(&c->nb.cell_count, (size_t)ncell, "cells"))) return s;
        if ((s = dev_alloc(&c->nb.cell_start, (size_t)ncell + 1, "cells"))) return s;
        if ((s = dev_alloc(&c->nb.cell_cursor, (size_t)ncell, "cells"))) return s;
        c->ncell_cap = ncell;
    }
    for (int a = 0; a < 3; ++a) c->nc[a] = nc[a];
    {
        // first-pass sort width: 1.15 x the mean number of neighbours within
        // rcut, rounded up to a power of two (denser atoms take the second pass)
        const double vol = b.L[0] * b.L[1] * b.L[2];
        const double expect = (double)N / vol * 4.0 / 3.0 * M_PI * c->m.rcut * c->m.rcut * c->m.rcut;
        int sw = 64;
        while (sw < 1.15 * expect + 8.0 && sw < 1024) sw *= 2;
        c->sort_small = sw;
    }
    GroupTimer tm(c, G_BUILD);
    cudaError_t e = cudaSuccess;
    if (gated) e = dp_launch_check_stale(c->stream, coords, c->nb.xref, (int)N, b, 0.25 * skin * skin, c->d_gate,
                                         &c->launches);
    if (e == cudaSuccess)
        e = dp_launch_build(c->stream, c->m, coords, types, b, (int)N, rlist, c->cap, nc, c->nb, c->d_status,
                            gated ? c->d_gate : nullptr, &c->launches);
    if (e != cudaSuccess) return cuda_fail(e, "dp_build_nlist");
    c->nlist_valid = true;
    c->nlist_N = N;
    // a gated build may or may not have rebuilt the type partition (over N)
    if (!gated || c->perm_n != N) c->perm_n = gated ? -1 : N;
    c->skin = skin;
    return DP_OK;
}

// The type partition of the centres 0..n-1 (all atoms, or the owned atoms of
// a sub-region).
dp_status ensure_perm(dp_ctx *c, const int32_t *types, int64_t n)
{
    if (c->perm_n == n) return DP_OK;
    GroupTimer tm(c, G_BUILD);
    cudaError_t e = dp_launch_type_perm(c->stream, c->m, types, (int)n, c->nb, c->d_status, &c->launches);
    if (e != cudaSuccess) return cuda_fail(e, "type partition");
    c->perm_n = n;
    return DP_OK;
}

dp_status enqueue_format(dp_ctx *c, const double *coords, const int32_t *types, const Box3 &b, int64_t N)
{
    GroupTimer tm(c, G_FORMAT);
    cudaError_t e = dp_launch_format(c->stream, c->m, coords, types, b, (int)N, c->cap, c->sort_small, c->skin,
                                     c->nb, c->fb, c->d_status, c->d_retry, &c->launches);
    if (e != cudaSuccess) return cuda_fail(e, "format");
    return DP_OK;
}

// Weight digits of the tensor-core FP64 fitting net (again whenever the
// model's parameters changed) and its scratch (first use).
dp_status ensure_oz(dp_ctx *c)
{
    dp_status s = DP_OK;
    if (!c->ob.a) {
        const int64_t N = c->natoms_max;
        const int T = c->m.ntypes, nf = c->m.n_fit;
        OzBuffers &ob = c->ob;
        ob.tiles = (int)((N + DP_OZ_TILE - 1) / DP_OZ_TILE) + T;
        ob.a_stride = c->oz.in_w;
        ob.nmax = N;
        const size_t plane = (size_t)N * c->oz.fmax;
        if ((s = dev_alloc(&ob.a, (size_t)ob.tiles * ob.a_stride, "fitting digits"))) return s;
        if ((s = dev_alloc(&ob.aexp, (size_t)ob.tiles * DP_OZ_TILE, "fitting digits"))) return s;
        if ((s = dev_alloc(&ob.t, (size_t)nf * plane, "fitting activations"))) return s;
        if ((s = dev_alloc(&ob.h, 2 * plane, "fitting activations"))) return s;
        if ((s = dev_alloc(&ob.g, 2 * plane, "fitting activations"))) return s;
    }
    if (c->oz_version != c->model->version) {
        std::vector<uint16_t> w((size_t)c->oz_w_elems, 0);
        std::vector<int32_t> e((size_t)c->oz_e_elems, 0);
        dp_oz_split_weights(c->m, c->model->h_params, c->oz, w.data(), e.data());
        DP_CUDA(cudaStreamSynchronize(c->stream), "fitting digits");
        DP_CUDA(cudaMemcpy(c->d_oz_w, w.data(), w.size() * 2, cudaMemcpyHostToDevice), "fitting digits");
        DP_CUDA(cudaMemcpy(c->d_oz_e, e.data(), e.size() * 4, cudaMemcpyHostToDevice), "fitting digits");
        c->oz_version = c->model->version;
    }
    return DP_OK;
}

dp_status ensure_ex(dp_ctx *c)
{
    if (c->ex_version == c->model->version) return DP_OK;
    std::vector<unsigned char> w(dp_ex_bytes(c->m), 0);
    dp_ex_split_weights(c->m, c->model->h_params, w.data());
    DP_CUDA(cudaStreamSynchronize(c->stream), "embedding digits");
    DP_CUDA(cudaMemcpy(c->d_ex_w, w.data(), w.size(), cudaMemcpyHostToDevice), "embedding digits");
    c->ex_version = c->model->version;
    return DP_OK;
}

dp_status enqueue_eval(dp_ctx *c, const double *coords, const int32_t *types, const Box3 &b, int64_t N,
                       int64_t nloc, double *energy, double *force, double *virial, double *atom_energy)
{
    dp_status s = ensure_perm(c, types, nloc);
    if (s) return s;
    cudaError_t e;
    const bool mixed = is_mixed(c->precision);
    const int n = (int)nloc;  // the centres
    if (n > 0) {
        if ((s = enqueue_format(c, coords, types, b, nloc))) return s;
        if (!mixed && c->use_ex && (s = ensure_ex(c))) return s;
        {
            GroupTimer tm(c, G_EMBED_FWD);
            e = mixed && c->eb.Gmx
                    ? dp_launch_embed_tan_mx(c->stream, c->m, c->mx, coords, types, b, n, c->fb, c->nb, c->eb,
                                             c->num_sms, c->d_status, &c->launches)
                : mixed     ? dp_launch_embed_fwd_mx(c->stream, c->m, c->mx, coords, types, b, n, c->fb, c->nb,
                                                     c->eb, c->num_sms, c->d_status, &c->launches)
                : c->use_ex && c->eb.Gst
                    ? dp_launch_embed_tan_x(c->stream, c->m, c->d_ex_w, coords, types, b, n, c->fb, c->nb, c->eb,
                                            c->num_sms, c->d_status, &c->launches)
                : c->use_ex ? dp_launch_embed_fwd_x(c->stream, c->m, c->d_ex_w, coords, types, b, n, c->fb, c->nb,
                                                    c->eb, c->num_sms, c->d_status, &c->launches)
                            : dp_launch_embed_fwd(c->stream, c->m, coords, types, b, n, c->fb, c->nb, c->eb,
                                                  c->num_sms, &c->launches);
            if (e != cudaSuccess) return cuda_fail(e, "embed_fwd");
        }
        if (c->use_oz && (s = ensure_oz(c))) return s;
        {
            GroupTimer tm(c, G_FIT);
            e = mixed && !c->use_oz
                    ? dp_launch_fit_mx(c->stream, c->m, c->mx, n, c->nb, c->eb, c->d_status, &c->launches)
                : c->use_oz ? dp_launch_fit_oz(c->stream, c->m, c->oz, c->ob, n, c->nb, c->eb, c->d_status,
                                               &c->launches)
                            : dp_launch_fit(c->stream, c->m, n, c->nb, c->eb, &c->launches);
            if (e != cudaSuccess) return cuda_fail(e, "fit");
        }
        {
            GroupTimer tm(c, G_EMBED_BWD);
            e = mixed && c->eb.Gmx
                    ? dp_launch_embed_bwd_stmx(c->stream, c->m, coords, types, b, n, c->fb, c->eb, c->num_sms,
                                               &c->launches)
                : mixed     ? dp_launch_embed_bwd_mx(c->stream, c->m, c->mx, coords, types, b, n, c->fb, c->nb,
                                                     c->eb, c->num_sms, c->d_status, &c->launches)
                : c->use_ex && c->eb.Gst
                    ? dp_launch_embed_bwd_st(c->stream, c->m, coords, types, b, n, c->fb, c->eb, c->num_sms,
                                             &c->launches)
                : c->use_ex ? dp_launch_embed_bwd_x(c->stream, c->m, c->d_ex_w, coords, types, b, n, c->fb, c->nb,
                                                    c->eb, c->num_sms, c->d_status, &c->launches)
                            : dp_launch_embed_bwd(c->stream, c->m, coords, types, b, n, c->fb, c->nb, c->eb,
                                                  c->num_sms, &c->launches);
            if (e != cudaSuccess) return cuda_fail(e, "embed_bwd");
        }
    }
    {
        GroupTimer tm(c, G_FORCE);
        if ((e = dp_launch_force(c->stream, c->m, coords, types, b, (int)N, n, c->cap, c->nb, c->fb, c->eb, force,
                                 &c->launches)) != cudaSuccess)
            return cuda_fail(e, "force");
    }
    {
        GroupTimer tm(c, G_REDUCE);
        if ((e = dp_launch_reduce(c->stream, n, c->eb, energy, virial, atom_energy, c->d_status,
                                  &c->launches)) != cudaSuccess)
            return cuda_fail(e, "reduce");
    }
    return DP_OK;
}

// Device copies of conv/m and m per type (uploaded when the masses change).
dp_status upload_masses(dp_ctx *c, const double *mass_per_type)
{
    const int T = c->m.ntypes;
    bool same = true;
    for (int a = 0; a < T; ++a) {
        if (!(mass_per_type[a] > 0.0)) return fail(DP_ERR_ARG, "masses must be positive");
        same = same && c->last_mass[a] == mass_per_type[a];
    }
    if (same) return DP_OK;
    // the pinned staging buffer may still feed an earlier asynchronous copy
    DP_CUDA(cudaStreamSynchronize(c->stream), "masses");
    for (int a = 0; a < T; ++a) {
        c->h_mass_stage[a] = kAccConv / mass_per_type[a];
        c->h_mass_stage[DP_MAX_TYPES + a] = mass_per_type[a];
        c->last_mass[a] = mass_per_type[a];
    }
    DP_CUDA(cudaMemcpyAsync(c->d_inv_mass_conv, c->h_mass_stage, sizeof(double) * T, cudaMemcpyHostToDevice,
                            c->stream),
            "masses");
    DP_CUDA(cudaMemcpyAsync(c->d_mass, c->h_mass_stage + DP_MAX_TYPES, sizeof(double) * T, cudaMemcpyHostToDevice,
                            c->stream),
            "masses");
    return DP_OK;
}

// ------------------------------------------------------------ seeded weights
// The paper's models are trained (Sec. 2) and none is shipped, so models are
// drawn from a seed.  Element k of the flat parameter vector takes the k-th
// standard normal of one stream: splitmix64 (Steele, Lea and Flood, 2014; its
// i-th output mixes seed + i * 0x9E3779B97F4A7C15, i = 1, 2, ...) gives 53-bit
// uniforms, and the Box-Muller transform turns outputs (2p+1, 2p+2) into the
// normals 2p (cosine branch) and 2p+1 (sine branch).
uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double seeded_normal(uint64_t seed, int64_t k)
{
    const uint64_t p = (uint64_t)k >> 1;
    const double u1 = (double)((splitmix64_at(seed, 2 * p + 1) >> 11) + 1) * 0x1p-53;   // (0, 1]
    const double u2 = (double)(splitmix64_at(seed, 2 * p + 2) >> 11) * 0x1p-53;         // [0, 1)
    const double r = std::sqrt(-2.0 * std::log(u1));
    const double th = 6.283185307179586 * u2;
    return (k & 1) ? r * std::sin(th) : r * std::cos(th);
}

// Walks the flat layout of dp_model_nparams and writes every element.
void fill_seeded(const dp_model_desc &d, uint64_t seed, double fit_in_gain, double out_scale, double *P)
{
    int64_t k = 0;
    auto weights = [&](int64_t n, int fan_in, int fan_out, double gain) {
        const double den = std::sqrt((double)(fan_in + fan_out));
        for (int64_t q = 0; q < n; ++q, ++k) {
            double w = seeded_normal(seed, k) / den;
            if (gain != 1.0) w = w * gain;
            P[k] = w;
        }
    };
    auto biases = [&](int64_t n) {
        for (int64_t q = 0; q < n; ++q, ++k) P[k] = seeded_normal(seed, k);
    };
    const int T = d.ntypes, M = d.emb[d.n_emb - 1];
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            int prev = 1;
            for (int l = 0; l < d.n_emb; ++l) {
                weights((int64_t)prev * d.emb[l], prev, d.emb[l], 1.0);
                biases(d.emb[l]);
                prev = d.emb[l];
            }
        }
    for (int a = 0; a < T; ++a) {
        int prev = d.m2 * M;
        for (int l = 0; l < d.n_fit; ++l) {
            weights((int64_t)prev * d.fit[l], prev, d.fit[l], l == 0 ? fit_in_gain : 1.0);
            biases(d.fit[l]);
            prev = d.fit[l];
        }
        const double den = std::sqrt((double)(prev + 1));
        for (int q = 0; q < prev; ++q, ++k) P[k] = (out_scale * seeded_normal(seed, k)) / den;
        P[k++] = 0.0;   // b_out
    }
}

}  // namespace

// Lets other translation units (the no-allocation entry point) report errors
// through dp_last_error().
void dp_set_last_error(const char *msg) { g_last_error = msg; }

extern "C" {

const char *dp_last_error(void) { return g_last_error.c_str(); }

const char *dp_status_string(dp_status s)
{
    switch (s) {
    case DP_OK: return "ok";
    case DP_ERR_ARG: return "invalid argument";
    case DP_ERR_BOX: return "unsupported or too small cell";
    case DP_ERR_SEL_OVERFLOW: return "a neighbour within rcut did not fit sel";
    case DP_ERR_NLIST_STALE: return "neighbour candidates are stale (moved > skin/2)";
    case DP_ERR_NONFINITE: return "non-finite energy or virial";
    case DP_ERR_FILE: return "model file error";
    case DP_ERR_CUDA: return "CUDA error";
    case DP_ERR_UNSUPPORTED: return "unsupported model shape";
    case DP_ERR_CAPACITY: return "candidate capacity exceeded";
    case DP_ERR_NOMEM: return "device allocation failed";
    case DP_ERR_TYPE: return "atom type out of range";
    default: return "unknown status";
    }
}

int64_t dp_model_nparams(const dp_model_desc *desc)
{
    if (check_desc(desc) != DP_OK) return -1;
    return desc_nparams(*desc);
}

dp_status dp_model_create(const dp_model_desc *desc, const double *params, int64_t nparams, dp_model **out)
{
    if (!out) return fail(DP_ERR_ARG, "out is NULL");
    *out = nullptr;
    dp_status s = check_desc(desc);
    if (s) return s;
    if (!params) return fail(DP_ERR_ARG, "params is NULL");
    const int64_t need = desc_nparams(*desc);
    if (nparams != need) return fail(DP_ERR_ARG, "nparams does not match the descriptor (" + std::to_string(need) + ")");
    dp_model *m = new (std::nothrow) dp_model();
    if (!m) return fail(DP_ERR_NOMEM, "host allocation failed");
    m->desc = *desc;
    m->nparams = need;
    m->h_params = (double *)std::malloc(sizeof(double) * need);
    if (!m->h_params) {
        delete m;
        return fail(DP_ERR_NOMEM, "host allocation failed");
    }
    std::memcpy(m->h_params, params, sizeof(double) * need);
    for (int64_t q = 0; q < need; ++q)
        if (!std::isfinite(params[q])) {
            std::free(m->h_params);
            delete m;
            return fail(DP_ERR_ARG, "non-finite parameter");
        }
    if ((s = dev_alloc(&m->d_params, (size_t)need, "params"))) {
        std::free(m->h_params);
        delete m;
        return s;
    }
    cudaError_t e = cudaMemcpy(m->d_params, params, sizeof(double) * need, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->d_params);
        std::free(m->h_params);
        delete m;
        return cuda_fail(e, "dp_model_create");
    }
    m->dev = make_devmodel(*desc, m->d_params);
    *out = m;
    return DP_OK;
}

void dp_model_free(dp_model *m)
{
    if (!m) return;
    dev_free(m->d_params);
    std::free(m->h_params);
    delete m;
}

static const char kMagic[8] = {'D', 'P', 'G', 'B', '3', '0', '0', 'M'};

dp_status dp_model_save(const dp_model *m, const char *path)
{
    if (!m || !path) return fail(DP_ERR_ARG, "model/path is NULL");
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(DP_ERR_FILE, std::string("cannot open ") + path);
    const dp_model_desc &d = m->desc;
    uint32_t ver = 1;
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&ver, 4, 1, f) == 1;
    int32_t ints[1 + DP_MAX_TYPES + 1 + DP_MAX_LAYERS + 1 + 1 + DP_MAX_LAYERS + 2];
    int p = 0;
    ints[p++] = d.ntypes;
    for (int a = 0; a < DP_MAX_TYPES; ++a) ints[p++] = d.sel[a];
    ints[p++] = d.n_emb;
    for (int l = 0; l < DP_MAX_LAYERS; ++l) ints[p++] = d.emb[l];
    ints[p++] = d.m2;
    ints[p++] = d.n_fit;
    for (int l = 0; l < DP_MAX_LAYERS; ++l) ints[p++] = d.fit[l];
    ints[p++] = d.desc_scale_nm;
    ints[p++] = d.reserved;
    ok = ok && std::fwrite(ints, 4, p, f) == (size_t)p;
    ok = ok && std::fwrite(&d.rcut, 8, 1, f) == 1 && std::fwrite(&d.rcut_smth, 8, 1, f) == 1;
    ok = ok && std::fwrite(&m->nparams, 8, 1, f) == 1;
    ok = ok && std::fwrite(m->h_params, 8, m->nparams, f) == (size_t)m->nparams;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? DP_OK : fail(DP_ERR_FILE, std::string("short write to ") + path);
}

dp_status dp_model_load(const char *path, dp_model **out)
{
    if (!path || !out) return fail(DP_ERR_ARG, "path/out is NULL");
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(DP_ERR_FILE, std::string("cannot open ") + path);
    char magic[8];
    uint32_t ver = 0;
    dp_model_desc d;
    std::memset(&d, 0, sizeof(d));
    int32_t ints[1 + DP_MAX_TYPES + 1 + DP_MAX_LAYERS + 1 + 1 + DP_MAX_LAYERS + 2];
    const int nint = (int)(sizeof(ints) / sizeof(ints[0]));
    int64_t np = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(&ver, 4, 1, f) == 1 && ver == 1 && std::fread(ints, 4, nint, f) == (size_t)nint &&
              std::fread(&d.rcut, 8, 1, f) == 1 && std::fread(&d.rcut_smth, 8, 1, f) == 1 &&
              std::fread(&np, 8, 1, f) == 1;
    if (!ok) {
        std::fclose(f);
        return fail(DP_ERR_FILE, std::string("bad header in ") + path);
    }
    int p = 0;
    d.ntypes = ints[p++];
    for (int a = 0; a < DP_MAX_TYPES; ++a) d.sel[a] = ints[p++];
    d.n_emb = ints[p++];
    for (int l = 0; l < DP_MAX_LAYERS; ++l) d.emb[l] = ints[p++];
    d.m2 = ints[p++];
    d.n_fit = ints[p++];
    for (int l = 0; l < DP_MAX_LAYERS; ++l) d.fit[l] = ints[p++];
    d.desc_scale_nm = ints[p++];
    d.reserved = ints[p++];
    if (check_desc(&d) != DP_OK || np != desc_nparams(d)) {
        std::fclose(f);
        return fail(DP_ERR_FILE, std::string("inconsistent descriptor in ") + path);
    }
    double *buf = (double *)std::malloc(sizeof(double) * np);
    if (!buf) {
        std::fclose(f);
        return fail(DP_ERR_NOMEM, "host allocation failed");
    }
    ok = std::fread(buf, 8, np, f) == (size_t)np;
    std::fclose(f);
    if (!ok) {
        std::free(buf);
        return fail(DP_ERR_FILE, std::string("truncated parameters in ") + path);
    }
    dp_status s = dp_model_create(&d, buf, np, out);
    std::free(buf);
    if (s == DP_ERR_ARG) return fail(DP_ERR_FILE, std::string("corrupt parameters in ") + path);
    return s;
}

dp_status dp_model_params_from_seed(const dp_model_desc *desc, uint64_t seed, double fit_in_gain,
                                    double out_scale, double *params, int64_t nparams)
{
    dp_status s = check_desc(desc);
    if (s) return s;
    if (!params) return fail(DP_ERR_ARG, "params is NULL");
    const int64_t need = desc_nparams(*desc);
    if (nparams != need) return fail(DP_ERR_ARG, "nparams does not match the descriptor (" + std::to_string(need) + ")");
    if (!std::isfinite(fit_in_gain) || !std::isfinite(out_scale))
        return fail(DP_ERR_ARG, "fit_in_gain and out_scale must be finite");
    fill_seeded(*desc, seed, fit_in_gain, out_scale, params);
    return DP_OK;
}

dp_status dp_model_from_seed(const dp_model_desc *desc, uint64_t seed, double fit_in_gain, double out_scale,
                             dp_model **out)
{
    if (!out) return fail(DP_ERR_ARG, "out is NULL");
    *out = nullptr;
    dp_status s = check_desc(desc);
    if (s) return s;
    const int64_t n = desc_nparams(*desc);
    std::vector<double> P;
    try {
        P.resize((size_t)n);
    } catch (...) {
        return fail(DP_ERR_NOMEM, "host allocation failed");
    }
    if ((s = dp_model_params_from_seed(desc, seed, fit_in_gain, out_scale, P.data(), n))) return s;
    return dp_model_create(desc, P.data(), n, out);
}

void dp_ctx_free(dp_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    dev_free(c->d_status);
    dev_free(c->d_gate);
    dev_free(c->d_retry);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_mass_stage) cudaFreeHost(c->h_mass_stage);
    void *bufs[] = {c->nb.cand, c->nb.ncand, c->nb.xref, c->nb.cell_count, c->nb.cell_start,
                    c->nb.cell_cursor, c->nb.cell_atoms, c->nb.cell_sorted, c->nb.atom_cell,
                    c->nb.type_perm, c->nb.type_start, c->fb.nlist, c->fb.keys, c->fb.nreal,
                    c->eb.T, c->eb.D, c->eb.gD, c->eb.Ei, c->eb.pair_g, c->eb.f_own, c->eb.vir_part,
                    c->d_energy, c->d_virial, c->md_force, c->ke_part, c->d_inv_mass_conv, c->d_mass,
                    c->eb.fit_t, c->eb.fit_h, c->d_p32, c->d_emb_ops, c->d_fit_fwd, c->d_fit_bwd,
                    c->pb.dT, c->pb.dD, c->pb.Db, c->pb.dDb, c->pb.fit_scr, c->pb.rowscr, c->pb.slices,
                    c->d_oz_w, c->d_oz_e, c->ob.a, c->ob.aexp, c->ob.t, c->ob.h, c->ob.g, c->d_dtile, c->d_ex_w,
                    c->eb.Gst, c->eb.Gmx};
    for (void *p : bufs) dev_free(p);
    delete c;
}

dp_status dp_ctx_create(const dp_model *model, int64_t natoms_max, int32_t cand_cap, int32_t precision,
                        void *stream, dp_ctx **out)
{
    if (!out) return fail(DP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!model) return fail(DP_ERR_ARG, "model is NULL");
    if (natoms_max < 1 || natoms_max >= (1 << 26)) return fail(DP_ERR_ARG, "natoms_max must be in [1, 2^26)");
    if (cand_cap < 0 || cand_cap > 1024) return fail(DP_ERR_ARG, "cand_cap must be in [0, 1024]");
    if (precision != DP_PREC_FP64 && !is_mixed(precision) && precision != DP_PREC_FP64_SIMT)
        return fail(DP_ERR_UNSUPPORTED, "unknown precision mode");
    if (is_mixed(precision) && !dp_mixed_supported(model->dev))
        return fail(DP_ERR_UNSUPPORTED, "mixed precision needs a 3-layer doubling embedding net (s_1 in {16, 25, 32}) "
                                        "and equal fitting widths (multiples of 16, <= 256) after the first layer");
    dp_ctx *c = new (std::nothrow) dp_ctx();
    if (!c) return fail(DP_ERR_NOMEM, "host allocation failed");
    c->model = model;
    c->m = model->dev;
    c->natoms_max = natoms_max;
    c->cap_fixed = cand_cap;
    c->cap = 0;
    c->perm_n = -1;
    c->precision = precision;
    c->stream = (cudaStream_t)stream;
    c->sync = 1;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (c->num_sms < 1) c->num_sms = 1;
    const size_t N = (size_t)natoms_max, nm = (size_t)c->m.nm, T = (size_t)c->m.ntypes, M = (size_t)c->m.M;
    const size_t nd = (size_t)c->m.m2 * M;
    dp_status s = DP_OK;
#define ALLOC(ptr, n) \
    if (!s) s = dev_alloc(&(ptr), (n), #ptr)
    ALLOC(c->d_status, 1);
    ALLOC(c->d_gate, 1);
    ALLOC(c->d_retry, N + 1);
    ALLOC(c->nb.ncand, N);
    ALLOC(c->nb.xref, 3 * N);
    ALLOC(c->nb.cell_atoms, N);
    ALLOC(c->nb.cell_sorted, N);
    ALLOC(c->nb.atom_cell, N);
    ALLOC(c->nb.type_perm, N);
    ALLOC(c->nb.type_start, T + 1);
    ALLOC(c->fb.nlist, N * nm);
    ALLOC(c->fb.keys, N * nm);
    ALLOC(c->fb.nreal, N * T);
    ALLOC(c->eb.T, N * 4 * M);
    ALLOC(c->eb.D, N * nd);
    ALLOC(c->eb.gD, N * nd);
    ALLOC(c->eb.Ei, N);
    ALLOC(c->eb.pair_g, N * nm * 3);
    ALLOC(c->eb.f_own, 3 * N);
    ALLOC(c->eb.vir_part, 9 * N);
    ALLOC(c->d_energy, 1);
    ALLOC(c->d_virial, 9);
    ALLOC(c->md_force, 3 * N);
    ALLOC(c->ke_part, N);
    ALLOC(c->d_inv_mass_conv, DP_MAX_TYPES);
    ALLOC(c->d_mass, DP_MAX_TYPES);
    if (is_mixed(precision)) {
        // one [rows][128] block per 128-atom tile of one type (N / 128 + ntypes tiles at most)
        const size_t fit_rows = (size_t)N + 128 * (size_t)c->m.ntypes;
        ALLOC(c->eb.fit_t, fit_rows * c->m.n_fit * 256);
        ALLOC(c->eb.fit_h, fit_rows * 256);
    }
    c->use_oz = false;
    c->oz_version = -1;
    c->use_ex = false;
    c->ex_version = -1;
    if (precision == DP_PREC_FP64 && dp_ex_supported(c->m)) {
        ALLOC(c->d_ex_w, dp_ex_bytes(c->m));
        c->use_ex = true;
        // G and dG/ds stored by the forward, when that takes at most half of the free memory
        size_t fr = 0, tot = 0;
        const size_t gb = dp_ex_store_bytes(c->m, (int64_t)N);
        if (!s && cudaMemGetInfo(&fr, &tot) == cudaSuccess && gb <= fr / 2) {
            if (cudaMalloc((void **)&c->eb.Gst, gb) != cudaSuccess) {
                c->eb.Gst = nullptr;
                cudaGetLastError();
            }
        }
        cudaGetLastError();
    }
    // G and dG/ds (FP32) stored by the mixed forward (plain BF16 operands), on the same rule
    if (!s && precision == DP_PREC_MIXED) {
        size_t fr = 0, tot = 0;
        const size_t gb = dp_mx_store_bytes(c->m, (int64_t)N);
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && gb <= fr / 2) {
            if (cudaMalloc((void **)&c->eb.Gmx, gb) != cudaSuccess) {
                c->eb.Gmx = nullptr;
                cudaGetLastError();
            }
        }
        cudaGetLastError();
    }
    // the split mixed mode runs its fitting net as exact products of 28-bit digit
    // expansions (FP32-level accuracy, a quarter of the FP64 plans' MMAs)
    if ((precision == DP_PREC_FP64 || precision == DP_PREC_MIXED_SPLIT) &&
        dp_oz_plan(c->m, c->oz, c->oz_w_elems, c->oz_e_elems, precision == DP_PREC_MIXED_SPLIT ? 28 : 55)) {
        ALLOC(c->d_oz_w, (size_t)c->oz_w_elems);
        ALLOC(c->d_oz_e, (size_t)c->oz_e_elems);
        c->oz.w = c->d_oz_w;
        c->oz.wexp = c->d_oz_e;
        c->use_oz = true;
    }
#undef ALLOC
    if (!s && is_mixed(precision)) s = build_mixed(c);
    if (!s && is_mixed(precision)) {
        // BF16 descriptor tiles of the fitting kernel: [tiles][K1p / 64][128 x 64]
        const size_t tiles = (N + 127) / 128 + T;
        s = dev_alloc(&c->d_dtile, tiles * (size_t)c->mx.fit_kp[0] * 128 * 2, "bf16 descriptor tiles");
        c->mx.dtile = c->d_dtile;
    }
    if (!s) {
        const double *tab = nullptr;
        cudaError_t e = dp_tanh_setup(&tab);
        if (e != cudaSuccess) s = cuda_fail(e, "tanh table");
        c->m.tanh_tab = tab;
    }
    if (!s && cudaMallocHost((void **)&c->h_status, sizeof(int32_t)) != cudaSuccess) {
        c->h_status = nullptr;
        s = fail(DP_ERR_NOMEM, "pinned allocation failed");
    }
    if (!s && cudaMallocHost((void **)&c->h_mass_stage, sizeof(double) * 2 * DP_MAX_TYPES) != cudaSuccess) {
        c->h_mass_stage = nullptr;
        s = fail(DP_ERR_NOMEM, "pinned allocation failed");
    }
    if (!s) {
        cudaError_t e = cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_gate, 0, sizeof(int32_t), c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) s = cuda_fail(e, "dp_ctx_create");
    }
    if (s) {
        dp_ctx_free(c);
        return s;
    }
    *out = c;
    return DP_OK;
}

dp_status dp_ctx_set_embed_store(dp_ctx *c, int32_t on)
{
    if (!c) return fail(DP_ERR_ARG, "context is NULL");
    const bool mx = c->precision == DP_PREC_MIXED;
    if (on && !c->use_ex && !mx)
        return fail(DP_ERR_UNSUPPORTED, "the store needs an FP64 context of the tensor-core embedding kernels "
                                        "or a mixed-precision context with plain BF16 operands");
    const bool have = c->eb.Gst != nullptr || c->eb.Gmx != nullptr;
    if ((on != 0) == have) return DP_OK;
    DP_CUDA(cudaStreamSynchronize(c->stream), "dp_ctx_set_embed_store");
    if (!on) {
        dev_free(c->eb.Gst);
        dev_free(c->eb.Gmx);
        c->eb.Gst = nullptr;
        c->eb.Gmx = nullptr;
        return DP_OK;
    }
    if (mx) return dev_alloc(&c->eb.Gmx, dp_mx_store_bytes(c->m, c->natoms_max) / sizeof(float), "G and dG/ds rows");
    return dev_alloc(&c->eb.Gst, dp_ex_store_bytes(c->m, c->natoms_max) / sizeof(double), "G and dG/ds rows");
}

int32_t dp_ctx_embed_store(const dp_ctx *c)
{
    return c ? ((c->eb.Gst != nullptr || c->eb.Gmx != nullptr) ? 1 : 0) : -1;
}

dp_status dp_ctx_set_sync(dp_ctx *c, int32_t sync)
{
    if (!c) return fail(DP_ERR_ARG, "context is NULL");
    c->sync = sync ? 1 : 0;
    return DP_OK;
}

int64_t dp_ctx_launches(const dp_ctx *c) { return c ? c->launches : -1; }

dp_status dp_ctx_set_timing(dp_ctx *c, int32_t on)
{
    if (!c) return fail(DP_ERR_ARG, "context is NULL");
    if (on) {
        dp_status s = flush_spans(c);
        if (s) return s;
        for (int g = 0; g < DP_KERNEL_GROUPS; ++g) {
            c->group_ms[g] = 0.0;
            c->group_launches[g] = 0;
        }
    }
    c->timing = on != 0;
    return DP_OK;
}

dp_status dp_ctx_kernel_times(dp_ctx *c, double *ms, int64_t *launches)
{
    if (!c) return fail(DP_ERR_ARG, "context is NULL");
    dp_status s = flush_spans(c);
    if (s) return s;
    for (int g = 0; g < DP_KERNEL_GROUPS; ++g) {
        if (ms) ms[g] = c->group_ms[g];
        if (launches) launches[g] = c->group_launches[g];
    }
    return DP_OK;
}

const char *dp_kernel_group_name(int32_t g)
{
    static const char *names[DP_KERNEL_GROUPS] = {"build", "format", "embed_fwd", "fit",
                                                  "embed_bwd", "force", "reduce", "md"};
    return (g >= 0 && g < DP_KERNEL_GROUPS) ? names[g] : "?";
}

dp_status dp_ctx_status(dp_ctx *c)
{
    if (!c) return fail(DP_ERR_ARG, "context is NULL");
    DP_CUDA(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream),
            "status read");
    DP_CUDA(cudaStreamSynchronize(c->stream), "status read");
    const int32_t f = *c->h_status;
    DP_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), c->stream), "status reset");
    if (f & DPF_MMA_TIMEOUT) return fail(DP_ERR_CUDA, "a tensor-core completion wait timed out");
    if (f & DPF_BAD_TYPE) return fail(DP_ERR_TYPE, "an atom type is outside [0, ntypes)");
    if (f & DPF_CAND_OVERFLOW) return fail(DP_ERR_CAPACITY, "an atom has more candidates than cand_cap");
    if (f & DPF_NONFINITE) return fail(DP_ERR_NONFINITE, "non-finite energy or virial");
    if (f & DPF_SEL_OVERFLOW) return fail(DP_ERR_SEL_OVERFLOW, "a neighbour within rcut did not fit sel");
    if (f & DPF_STALE) return fail(DP_ERR_NLIST_STALE, "an atom moved more than skin/2 since the last build");
    return DP_OK;
}

dp_status dp_build_nlist(dp_ctx *c, const double *coords, const int32_t *types, const double box[9], int64_t N,
                         double skin)
{
    dp_status s = check_common(c, coords, types, N);
    if (s) return s;
    Box3 b;
    if ((s = read_box(box, b))) return s;
    if ((s = do_build(c, coords, types, b, N, skin))) return s;
    return finish(c);
}

dp_status dp_format_nlist(dp_ctx *c, const double *coords, const int32_t *types, const double box[9], int64_t N,
                          int32_t *nlist, int32_t *nreal)
{
    dp_status s = check_common(c, coords, types, N);
    if (s) return s;
    Box3 b;
    if ((s = read_box(box, b))) return s;
    if (!c->nlist_valid || c->nlist_N != N)
        if ((s = do_build(c, coords, types, b, N, 0.0))) return s;
    if ((s = enqueue_format(c, coords, types, b, N))) return s;
    if (nlist)
        DP_CUDA(cudaMemcpyAsync(nlist, c->fb.nlist, sizeof(int32_t) * N * c->m.nm, cudaMemcpyDeviceToDevice,
                                c->stream),
                "dp_format_nlist");
    if (nreal)
        DP_CUDA(cudaMemcpyAsync(nreal, c->fb.nreal, sizeof(int32_t) * N * c->m.ntypes, cudaMemcpyDeviceToDevice,
                                c->stream),
                "dp_format_nlist");
    return finish(c);
}

dp_status dp_eval(dp_ctx *c, const double *coords, const int32_t *types, const double box[9], int64_t N,
                  double *energy, double *force, double *virial, double *atom_energy)
{
    dp_status s = check_common(c, coords, types, N);
    if (s) return s;
    if (!energy || !force || !virial) return fail(DP_ERR_ARG, "energy/force/virial is NULL");
    Box3 b;
    if ((s = read_box(box, b))) return s;
    if (!c->nlist_valid || c->nlist_N != N)
        if ((s = do_build(c, coords, types, b, N, 0.0))) return s;
    if ((s = enqueue_eval(c, coords, types, b, N, N, energy, force, virial, atom_energy))) return s;
    return finish(c);
}

dp_status dp_eval_local(dp_ctx *c, const double *coords, const int32_t *types, const double box[9], int64_t N,
                        int64_t nloc, double *energy, double *force, double *virial, double *atom_energy)
{
    dp_status s = check_common(c, coords, types, N);
    if (s) return s;
    if (!energy || !force || !virial) return fail(DP_ERR_ARG, "energy/force/virial is NULL");
    if (nloc < 0 || nloc > N) return fail(DP_ERR_ARG, "nloc must be in [0, N]");
    Box3 b;
    if ((s = read_box(box, b))) return s;
    if (!c->nlist_valid || c->nlist_N != N)
        if ((s = do_build(c, coords, types, b, N, 0.0))) return s;
    if ((s = enqueue_eval(c, coords, types, b, N, nloc, energy, force, virial, atom_energy))) return s;
    return finish(c);
}

dp_status dp_md_step(dp_ctx *c, double *coords, double *vel, const int32_t *types, const double box[9],
                     const double *mass_per_type, int64_t N, double dt_fs, int32_t nsteps, int32_t rebuild_every,
                     double skin, double *thermo)
{
    dp_status s = check_common(c, coords, types, N);
    if (s) return s;
    if (!vel || !mass_per_type) return fail(DP_ERR_ARG, "vel/mass_per_type is NULL");
    if (nsteps < 0 || rebuild_every < 0 || !(dt_fs > 0.0)) return fail(DP_ERR_ARG, "bad nsteps/rebuild_every/dt");
    Box3 b;
    if ((s = read_box(box, b))) return s;
    if ((s = upload_masses(c, mass_per_type))) return s;
    const double vol = b.L[0] * b.L[1] * b.L[2];
    if (!c->md_force_valid || c->md_N != N) {
        if ((s = do_build(c, coords, types, b, N, skin))) return s;
        if ((s = enqueue_eval(c, coords, types, b, N, N, c->d_energy, c->md_force, c->d_virial, nullptr)))
            return s;
        c->md_force_valid = true;
        c->md_N = N;
        c->md_step = 0;
    }
    for (int st = 1; st <= nsteps; ++st) {
        cudaError_t e;
        {
            GroupTimer tm(c, G_MD);
            e = dp_launch_kick_drift(c->stream, (int)N, coords, vel, c->md_force, types, c->d_inv_mass_conv, dt_fs,
                                     b, &c->launches);
        }
        if (e != cudaSuccess) return cuda_fail(e, "kick_drift");
        c->md_step += 1;
        if (rebuild_every > 0 && c->md_step % rebuild_every == 0) {
            if ((s = do_build(c, coords, types, b, N, skin))) return s;
        } else if (skin > 0.0) {
            // rebuild on the device as soon as an atom has moved more than skin/2
            if ((s = do_build(c, coords, types, b, N, skin, true))) return s;
        }
        if ((s = enqueue_eval(c, coords, types, b, N, N, c->d_energy, c->md_force, c->d_virial, nullptr)))
            return s;
        {
            GroupTimer tm(c, G_MD);
            e = dp_launch_kick_thermo(c->stream, (int)N, vel, c->md_force, types, c->d_inv_mass_conv, c->d_mass,
                                      dt_fs, c->ke_part, &c->launches);
            if (e == cudaSuccess && thermo)
                e = dp_launch_thermo(c->stream, (int)N, c->ke_part, c->d_energy, c->d_virial, vol,
                                     thermo + (size_t)(st - 1) * 4, &c->launches);
        }
        if (e != cudaSuccess) return cuda_fail(e, "kick_thermo");
    }
    return finish(c);
}

dp_status dp_md_kick_drift(dp_ctx *c, double *coords, double *vel, const double *force, const int32_t *types,
                           const double box[9], const double *mass_per_type, int64_t N, double dt_fs)
{
    dp_status s = check_common(c, coords, types, N);
    if (s) return s;
    if (!vel || !force || !mass_per_type) return fail(DP_ERR_ARG, "vel/force/mass_per_type is NULL");
    if (!(dt_fs > 0.0)) return fail(DP_ERR_ARG, "dt must be positive");
    Box3 b;
    if (box) {
        if ((s = read_box(box, b))) return s;
    } else {
        b.L[0] = b.L[1] = b.L[2] = 0.0;   // no wrapping
    }
    if ((s = upload_masses(c, mass_per_type))) return s;
    if (N > 0) {
        GroupTimer tm(c, G_MD);
        cudaError_t e = dp_launch_kick_drift(c->stream, (int)N, coords, vel, force, types, c->d_inv_mass_conv, dt_fs,
                                             b, &c->launches);
        if (e != cudaSuccess) return cuda_fail(e, "kick_drift");
    }
    return finish(c);
}

dp_status dp_md_kick(dp_ctx *c, double *vel, const double *force, const int32_t *types,
                     const double *mass_per_type, int64_t N, double dt_fs)
{
    if (!c) return fail(DP_ERR_ARG, "context is NULL");
    if (N < 0 || N > c->natoms_max) return fail(DP_ERR_ARG, "N out of range");
    if (N > 0 && (!vel || !force || !types)) return fail(DP_ERR_ARG, "vel/force/types is NULL");
    if (!mass_per_type) return fail(DP_ERR_ARG, "mass_per_type is NULL");
    if (!(dt_fs > 0.0)) return fail(DP_ERR_ARG, "dt must be positive");
    dp_status s;
    if ((s = upload_masses(c, mass_per_type))) return s;
    if (N > 0) {
        GroupTimer tm(c, G_MD);
        cudaError_t e = dp_launch_kick_thermo(c->stream, (int)N, vel, force, types, c->d_inv_mass_conv, c->d_mass,
                                              dt_fs, c->ke_part, &c->launches);
        if (e != cudaSuccess) return cuda_fail(e, "kick");
    }
    return finish(c);
}

dp_status dp_model_set_params(dp_model *md, const double *params, int64_t nparams)
{
    if (!md || !params) return fail(DP_ERR_ARG, "model/params is NULL");
    if (nparams != md->nparams) return fail(DP_ERR_ARG, "nparams does not match the model");
    // the same values again (a training loop evaluating several frames with
    // one set of parameters): nothing to upload, the contexts' derived copies
    // (weight digits, BF16 weights) stay valid
    if (std::memcmp(md->h_params, params, sizeof(double) * nparams) == 0) return DP_OK;
    for (int64_t q = 0; q < nparams; ++q)
        if (!std::isfinite(params[q])) return fail(DP_ERR_ARG, "non-finite parameter");
    std::memcpy(md->h_params, params, sizeof(double) * nparams);
    DP_CUDA(cudaMemcpy(md->d_params, params, sizeof(double) * nparams, cudaMemcpyHostToDevice), "dp_model_set_params");
    md->version += 1;
    return DP_OK;
}

dp_status dp_param_grad(dp_ctx *c, const double *coords, const int32_t *types, const double box[9], int64_t N,
                        double cE, const double *lambda, double *grad)
{
    dp_status s = check_common(c, coords, types, N);
    if (s) return s;
    if (!lambda || !grad) return fail(DP_ERR_ARG, "lambda/grad is NULL");
    if (is_mixed(c->precision)) return fail(DP_ERR_UNSUPPORTED, "parameter gradients need an FP64 context");
    for (int l = 1; l < c->m.n_fit; ++l)
        if (dp_skip_kind(c->m.fit[l - 1], c->m.fit[l]) == 2)
            return fail(DP_ERR_UNSUPPORTED, "parameter gradients support equal-width fitting skips only");
    Box3 b;
    if ((s = read_box(box, b))) return s;
    if (!c->nlist_valid || c->nlist_N != N)
        if ((s = do_build(c, coords, types, b, N, 0.0))) return s;
    const int64_t np = c->model->nparams;
    const size_t Nmax = (size_t)c->natoms_max, M = (size_t)c->m.M, nd = (size_t)c->m.m2 * M;
    if (!c->pb.slices) {
#define ALLOCP(ptr, n) \
    if (!s) s = dev_alloc(&(ptr), (n), #ptr)
        ALLOCP(c->pb.dT, Nmax * 4 * M);
        ALLOCP(c->pb.dD, Nmax * nd);
        ALLOCP(c->pb.Db, Nmax * nd);
        ALLOCP(c->pb.dDb, Nmax * nd);
        ALLOCP(c->pb.fit_scr, dp_pgrad_fit_scratch((int)Nmax));
        ALLOCP(c->pb.rowscr, dp_pgrad_row_scratch(c->num_sms));
        ALLOCP(c->pb.slices, (size_t)c->num_sms * np);
#undef ALLOCP
        if (s) return s;
    }
    if ((s = ensure_perm(c, types, N))) return s;
    if ((s = enqueue_format(c, coords, types, b, N))) return s;
    cudaError_t e = dp_launch_pgrad(c->stream, c->m, np, coords, types, b, (int)N, lambda, cE, c->fb, c->nb, c->eb,
                                    c->pb, c->num_sms, grad, &c->launches);
    if (e != cudaSuccess) return cuda_fail(e, "dp_param_grad");
    return finish(c);
}

dp_status dp_md_get_force(dp_ctx *c, double *force, int64_t N)
{
    if (!c || !force) return fail(DP_ERR_ARG, "context/force is NULL");
    if (!c->md_force_valid || c->md_N != N) return fail(DP_ERR_ARG, "no MD force for this N");
    DP_CUDA(cudaMemcpyAsync(force, c->md_force, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, c->stream),
            "dp_md_get_force");
    return finish(c);
}

dp_status dp_md_reset(dp_ctx *c)
{
    if (!c) return fail(DP_ERR_ARG, "context is NULL");
    c->md_force_valid = false;
    c->md_step = 0;
    return DP_OK;
}

}  // extern "C"
