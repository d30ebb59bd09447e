/*
 * dp_oracle.c -- plain, slow, FP64 CPU oracle of the Deep Potential
 * energy/force/virial evaluation and velocity-Verlet MD.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg call this file.  It shares no code, header or
 * table with the CUDA library.
 *
 * Paper: Lu et al., "86 PFLOPS Deep Potential Molecular Dynamics simulation of
 * 100 million atoms with ab initio accuracy" (arXiv 2004.11658).
 *
 *   orc_switch      s(r) = w(r)/r                          Sec. 2 (env. matrix)
 *   orc_candidates  brute-force neighbour candidates with skin   Sec. 3.2.2, Sec. 4
 *   orc_candidates_cells  the same candidates from a cell list  Sec. 3.2.2, Sec. 4
 *   orc_format      formatted neighbour list                Algorithm 1 + Sec. 3.2.2 text
 *   orc_eval        env. matrix (Alg. 2), embedding net (Eqs. embedding,
 *                   embedding-first, embedding-rest), descriptor (Eq. descrpt),
 *                   fitting net (Eqs. fitting, fitting-detail), E = sum E_i,
 *                   force F = -grad E by back-propagation (Remark 2), virial
 *   orc_md          velocity Verlet (Sec. 4)
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - w(r): quintic smooth step between rcut_smth and rcut (C2 at both ends);
 *   - descriptor scale: T = R^T G / N_m when desc_scale_nm = 1, N_m = sum(sel);
 *   - fitting net: the first layer (input width != output width) has no skip,
 *     equal-width layers use x + tanh(xW + b), the output layer is linear;
 *   - embedding layers with s_k = 2 s_{k-1} use (x,x) + tanh, equal widths use
 *     x + tanh, other widths plain tanh; layer 0 is plain tanh (Eq. embedding-first);
 *   - sort key (type, floor(|r| * 1e8), index), ties by smaller index;
 *   - virial Xi = -sum_{i,k} r_ij (x) dE_i/dr_ij  (= sum_i r_i (x) F_i for a cluster).
 *
 * Distances use the pinned arithmetic: minimum image d - L*rint(d/L), then
 * r^2 = (dx*dx + dy*dy) + dz*dz, r = sqrt(r^2), compiled without FMA
 * contraction (-ffp-contract=off), so that candidate sets and sort keys are
 * reproducible bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXT 8
#define ORC_MAXL 4

typedef struct {
    int ntypes;
    int sel[ORC_MAXT];
    int n_emb;
    int emb[ORC_MAXL];
    int m2;
    int n_fit;
    int fit[ORC_MAXL];
    int desc_scale_nm;
    double rcut, rcut_smth;
    int nm;                         /* N_m = sum sel */
    int sel_off[ORC_MAXT];          /* first slot of each type block */
    /* parameter offsets */
    long emb_W[ORC_MAXT][ORC_MAXT][ORC_MAXL];
    long emb_b[ORC_MAXT][ORC_MAXT][ORC_MAXL];
    long fit_W[ORC_MAXT][ORC_MAXL];
    long fit_b[ORC_MAXT][ORC_MAXL];
    long fit_wo[ORC_MAXT];
    long fit_bo[ORC_MAXT];
    long nparams;
} orc_model;

/* idesc = [ntypes, sel[8], n_emb, emb[4], m2, n_fit, fit[4], desc_scale_nm]
 * ddesc = [rcut, rcut_smth]                                                */
static int orc_parse(const int32_t *idesc, const double *ddesc, orc_model *m)
{
    memset(m, 0, sizeof(*m));
    int p = 0;
    m->ntypes = idesc[p++];
    for (int a = 0; a < ORC_MAXT; ++a) m->sel[a] = idesc[p++];
    m->n_emb = idesc[p++];
    for (int l = 0; l < ORC_MAXL; ++l) m->emb[l] = idesc[p++];
    m->m2 = idesc[p++];
    m->n_fit = idesc[p++];
    for (int l = 0; l < ORC_MAXL; ++l) m->fit[l] = idesc[p++];
    m->desc_scale_nm = idesc[p++];
    m->rcut = ddesc[0];
    m->rcut_smth = ddesc[1];
    if (m->ntypes < 1 || m->ntypes > ORC_MAXT || m->n_emb < 1 || m->n_emb > ORC_MAXL ||
        m->n_fit < 1 || m->n_fit > ORC_MAXL)
        return -1;
    m->nm = 0;
    for (int a = 0; a < m->ntypes; ++a) { m->sel_off[a] = m->nm; m->nm += m->sel[a]; }
    long off = 0;
    for (int a = 0; a < m->ntypes; ++a)
        for (int b = 0; b < m->ntypes; ++b) {
            int prev = 1;
            for (int l = 0; l < m->n_emb; ++l) {
                m->emb_W[a][b][l] = off; off += (long)prev * m->emb[l];
                m->emb_b[a][b][l] = off; off += m->emb[l];
                prev = m->emb[l];
            }
        }
    int M = m->emb[m->n_emb - 1];
    for (int a = 0; a < m->ntypes; ++a) {
        int prev = m->m2 * M;
        for (int l = 0; l < m->n_fit; ++l) {
            m->fit_W[a][l] = off; off += (long)prev * m->fit[l];
            m->fit_b[a][l] = off; off += m->fit[l];
            prev = m->fit[l];
        }
        m->fit_wo[a] = off; off += prev;
        m->fit_bo[a] = off; off += 1;
    }
    m->nparams = off;
    return 0;
}

long orc_nparams(const int32_t *idesc, const double *ddesc)
{
    orc_model m;
    if (orc_parse(idesc, ddesc, &m)) return -1;
    return m.nparams;
}

/* ---------------------------------------------------------------- geometry */

static void orc_min_image(const double *box, const double *xi, const double *xj, double d[3])
{
    for (int a = 0; a < 3; ++a) {
        double v = xj[a] - xi[a];
        double n = rint(v / box[a]);
        double shift = box[a] * n;
        d[a] = v - shift;
    }
}

static double orc_norm(const double d[3])
{
    double r2 = d[0] * d[0] + d[1] * d[1];
    r2 = r2 + d[2] * d[2];
    return sqrt(r2);
}

/* s(r) = w(r)/r with w a smooth gate: 1 below rs, 0 from rc on, and in
 * between w = u^3(-6u^2 + 15u - 10) + 1, u = (r - rs)/(rc - rs).  Sec. 2
 * asks only for a gate that goes smoothly from 1 to 0 at rc; this quintic is
 * the reading taken here.  Also returns ds/dr. */
int orc_switch(double r, double rs, double rc, double *s, double *ds)
{
    if (r < rs) {
        *s = 1.0 / r;
        *ds = -1.0 / (r * r);
    } else if (r < rc) {
        double u = (r - rs) / (rc - rs);
        double w = u * u * u * (-6.0 * u * u + 15.0 * u - 10.0) + 1.0;
        double dwdu = -30.0 * u * u * (u - 1.0) * (u - 1.0);
        double dw = dwdu / (rc - rs);
        *s = w / r;
        *ds = dw / r - w / (r * r);
    } else {
        *s = 0.0;
        *ds = 0.0;
    }
    return 0;
}

/* Brute-force O(N^2) neighbour candidates: every j != i with minimum-image
 * |r_ij| <= rlist (rlist = rcut + skin; the paper's L(i) plus the MD buffer of
 * Sec. 4), in increasing j.  Returns the number of atoms whose list was cut at
 * cap (0 when none). */
int64_t orc_candidates(int64_t N, const double *x, const double *box, double rlist,
                       int32_t cap, int32_t *ncand, int32_t *cand)
{
    int64_t over = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : over)
    for (int64_t i = 0; i < N; ++i) {
        int32_t n = 0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double d[3];
            orc_min_image(box, x + 3 * i, x + 3 * j, d);
            double r = orc_norm(d);
            if (r <= rlist) {
                if (n < cap) cand[i * cap + n] = (int32_t)j;
                ++n;
            }
        }
        if (n > cap) { over += 1; n = cap; }
        ncand[i] = n;
    }
    return over;
}

/* Cell-list neighbour candidates (Sec. 3.2.2 builds the list from cells;
 * Sec. 4 adds the skin): the same set as orc_candidates, in the same
 * increasing-j order, for the centres 0..ncentre-1.  The box is cut into
 * n_a = floor(L_a / rlist) cells per axis (slightly fewer when L_a / rlist is
 * an integer, so that every cell edge exceeds rlist by a margin larger than the
 * rounding of the cell index); a neighbour within rlist then lies in one of
 * the 27 cells around the centre's cell, each visited once since n_a >= 3.
 * Distances use the same minimum-image arithmetic as the brute-force build, so
 * the two sets agree bit for bit.  Returns -1 (nothing written) when an axis
 * has fewer than 3 cells; otherwise the number of centres whose list was cut
 * at cap. */
static int orc_cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_candidates_cells(int64_t N, int64_t ncentre, const double *x, const double *box, double rlist,
                             int32_t cap, int32_t *ncand, int32_t *cand)
{
    int nc[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)floor(box[a] / rlist * (1.0 - 1e-9));
        if (nc[a] < 3) return -1;
    }
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *cell_of = malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t *start = calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)ncell);
    int32_t *members = malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    /* cell of every atom, from its position wrapped into [0, L) */
    for (int64_t i = 0; i < N; ++i) {
        int64_t c = 0;
        for (int a = 0; a < 3; ++a) {
            double v = x[3 * i + a] - box[a] * floor(x[3 * i + a] / box[a]);
            int k = (int)floor(v / box[a] * nc[a]);
            if (k < 0) k = 0;
            if (k >= nc[a]) k = nc[a] - 1;
            c = c * nc[a] + k;
        }
        cell_of[i] = c;
        start[c + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    for (int64_t c = 0; c < ncell; ++c) fill[c] = start[c];
    for (int64_t i = 0; i < N; ++i) members[fill[cell_of[i]]++] = (int32_t)i;   /* increasing i per cell */
    int64_t over = 0;
#pragma omp parallel reduction(+ : over)
    {
        int64_t bufcap = 1024;
        int32_t *buf = malloc(sizeof(int32_t) * (size_t)bufcap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < ncentre; ++i) {
            int64_t c = cell_of[i];
            int ci[3];
            ci[2] = (int)(c % nc[2]);
            ci[1] = (int)((c / nc[2]) % nc[1]);
            ci[0] = (int)(c / ((int64_t)nc[1] * nc[2]));
            int64_t n = 0;
            for (int d0 = -1; d0 <= 1; ++d0)
                for (int d1 = -1; d1 <= 1; ++d1)
                    for (int d2 = -1; d2 <= 1; ++d2) {
                        int k0 = (ci[0] + d0 + nc[0]) % nc[0];
                        int k1 = (ci[1] + d1 + nc[1]) % nc[1];
                        int k2 = (ci[2] + d2 + nc[2]) % nc[2];
                        int64_t cc = ((int64_t)k0 * nc[1] + k1) * nc[2] + k2;
                        for (int64_t q = start[cc]; q < start[cc + 1]; ++q) {
                            int32_t j = members[q];
                            if (j == i) continue;
                            double d[3];
                            orc_min_image(box, x + 3 * i, x + 3 * (int64_t)j, d);
                            if (orc_norm(d) <= rlist) {
                                if (n == bufcap) {
                                    bufcap *= 2;
                                    buf = realloc(buf, sizeof(int32_t) * (size_t)bufcap);
                                }
                                buf[n++] = j;
                            }
                        }
                    }
            qsort(buf, (size_t)n, sizeof(int32_t), orc_cmp_i32);
            int64_t keep = n < cap ? n : cap;
            for (int64_t k = 0; k < keep; ++k) cand[i * cap + k] = buf[k];
            if (n > cap) over += 1;
            ncand[i] = (int32_t)keep;
        }
        free(buf);
    }
    free(cell_of); free(start); free(fill); free(members);
    return over;
}

/* Candidates of every atom: the cell list when each axis has at least 3
 * cells, brute force otherwise (both give the same list). */
static int64_t orc_candidates_any(int64_t N, const double *x, const double *box, double rlist, int32_t cap,
                                  int32_t *ncand, int32_t *cand)
{
    int64_t r = orc_candidates_cells(N, N, x, box, rlist, cap, ncand, cand);
    if (r >= 0) return r;
    return orc_candidates(N, x, box, rlist, cap, ncand, cand);
}

/* Number of OpenMP threads the oracle uses from now on (n >= 1). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------- Algorithm 1 */

typedef struct {
    int alpha;        /* type of neighbour j */
    uint64_t q;       /* floor(|r_ij| * 1e8) */
    int j;
    double r;
} orc_S;

static int orc_S_cmp(const void *pa, const void *pb)
{
    const orc_S *a = (const orc_S *)pa, *b = (const orc_S *)pb;
    if (a->alpha != b->alpha) return a->alpha < b->alpha ? -1 : 1;
    if (a->q != b->q) return a->q < b->q ? -1 : 1;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    return 0;
}

/* Algorithm 1 (Formatting the neighbour list) on L(i) = {j : |r_ij| <= rcut}
 * (Sec. 2): the candidates of atom i (built with a buffer, Sec. 4) are
 * restricted to L(i); S(i,k) = (alpha(j), |r_ij|, j) is sorted by type, then
 * distance, then smaller index on ties (Sec. 3.2.2 text; the distance is the
 * 1e-8 A quantum of the compressed key), the first sel_alpha entries of each
 * type are kept and the rest of the type block is padded with -1.
 * Outputs: nlist[N][N_m]; nreal[N][T] = entries kept in block T;
 * overflow[N] = neighbours within rcut that did not fit sel. */
int orc_format(int64_t N, const double *x, const int32_t *types, const double *box,
               const int32_t *ncand, const int32_t *cand, int32_t cap, int32_t ntypes,
               const int32_t *sel, double rcut, int32_t *nlist, int32_t *nreal,
               int64_t *overflow)
{
    int nm = 0, off[ORC_MAXT];
    for (int a = 0; a < ntypes; ++a) { off[a] = nm; nm += sel[a]; }
#pragma omp parallel
    {
        orc_S *S = (orc_S *)malloc(sizeof(orc_S) * (size_t)(cap > 0 ? cap : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < N; ++i) {
            int n = 0;
            for (int k = 0; k < ncand[i]; ++k) {
                int j = cand[i * cap + k];
                double d[3];
                orc_min_image(box, x + 3 * i, x + 3 * j, d);
                double r = orc_norm(d);
                if (r > rcut) continue;
                S[n].alpha = types[j];
                S[n].q = (uint64_t)floor(r * 1e8);
                S[n].j = j;
                S[n].r = r;
                ++n;
            }
            qsort(S, (size_t)n, sizeof(orc_S), orc_S_cmp);
            int cnt[ORC_MAXT] = {0};
            int64_t over = 0;
            for (int k = 0; k < nm; ++k) nlist[i * nm + k] = -1;
            for (int k = 0; k < n; ++k) {
                int a = S[k].alpha;
                if (cnt[a] < sel[a]) {
                    nlist[i * nm + off[a] + cnt[a]] = S[k].j;
                    cnt[a]++;
                } else {
                    over++;
                }
            }
            for (int a = 0; a < ntypes; ++a) nreal[i * ntypes + a] = cnt[a];
            overflow[i] = over;
        }
        free(S);
    }
    return 0;
}

/* ------------------------------------------------------------- evaluation */

typedef struct {
    double *R;       /* [nm][4] environment matrix rows */
    double *rij;     /* [nm][3] */
    double *rr;      /* [nm] |r_ij| */
    int *real;       /* [nm] row non-zero */
    double *h;       /* [nm][sum emb] layer outputs */
    double *t;       /* [nm][sum emb] tanh values */
    double *T;       /* [4][M] */
    double *gT;      /* [4][M] */
    double *D;       /* [M2*M] */
    double *gD;      /* [M2*M] */
    double *fh;      /* [n_fit][maxf] fitting layer outputs */
    double *ft;      /* [n_fit][maxf] fitting tanh values */
    double *gbuf0, *gbuf1; /* [max width] */
    double *gG;      /* [max emb] */
} orc_ws;

static int orc_max_width(const orc_model *m)
{
    int w = m->m2 * m->emb[m->n_emb - 1];
    for (int l = 0; l < m->n_emb; ++l) if (m->emb[l] > w) w = m->emb[l];
    for (int l = 0; l < m->n_fit; ++l) if (m->fit[l] > w) w = m->fit[l];
    return w;
}

static void orc_ws_alloc(const orc_model *m, orc_ws *w)
{
    int nm = m->nm, M = m->emb[m->n_emb - 1], se = 0, mf = 0;
    for (int l = 0; l < m->n_emb; ++l) se += m->emb[l];
    for (int l = 0; l < m->n_fit; ++l) if (m->fit[l] > mf) mf = m->fit[l];
    int mw = orc_max_width(m);
    w->R = calloc((size_t)nm * 4, sizeof(double));
    w->rij = calloc((size_t)nm * 3, sizeof(double));
    w->rr = calloc((size_t)nm, sizeof(double));
    w->real = calloc((size_t)nm, sizeof(int));
    w->h = calloc((size_t)nm * se, sizeof(double));
    w->t = calloc((size_t)nm * se, sizeof(double));
    w->T = calloc((size_t)4 * M, sizeof(double));
    w->gT = calloc((size_t)4 * M, sizeof(double));
    w->D = calloc((size_t)m->m2 * M, sizeof(double));
    w->gD = calloc((size_t)m->m2 * M, sizeof(double));
    w->fh = calloc((size_t)m->n_fit * mf, sizeof(double));
    w->ft = calloc((size_t)m->n_fit * mf, sizeof(double));
    w->gbuf0 = calloc((size_t)mw, sizeof(double));
    w->gbuf1 = calloc((size_t)mw, sizeof(double));
    w->gG = calloc((size_t)M, sizeof(double));
}

static void orc_ws_free(orc_ws *w)
{
    free(w->R); free(w->rij); free(w->rr); free(w->real); free(w->h); free(w->t);
    free(w->T); free(w->gT); free(w->D); free(w->gD); free(w->fh); free(w->ft);
    free(w->gbuf0); free(w->gbuf1); free(w->gG);
}

/* Skip term of a layer with input width `in` and output width `out`:
 * (x, x) when out == 2 in, x when out == in, none otherwise. */
static int orc_skip_kind(int in, int out)
{
    if (out == 2 * in) return 2;
    if (out == in) return 1;
    return 0;
}

/* One atom: E_i and the pair gradients g[k] = dE_i/dr_ij (k = slot). */
static double orc_atom(const orc_model *m, const double *P, int64_t i, const double *x,
                       const int32_t *types, const double *box, const int32_t *nlist,
                       orc_ws *w, double *g /* [nm][3] */, double *desc_out)
{
    const int nm = m->nm, ne = m->n_emb, M = m->emb[ne - 1], M2 = m->m2;
    int se = 0;
    for (int l = 0; l < ne; ++l) se += m->emb[l];
    const int ai = types[i];
    const double c = m->desc_scale_nm ? 1.0 / nm : 1.0;

    /* Algorithm 2: environment matrix rows; padded slots give zero rows. */
    for (int k = 0; k < nm; ++k) {
        int j = nlist[i * nm + k];
        w->real[k] = 0;
        w->R[4 * k + 0] = w->R[4 * k + 1] = w->R[4 * k + 2] = w->R[4 * k + 3] = 0.0;
        if (j < 0) continue;
        double d[3];
        orc_min_image(box, x + 3 * i, x + 3 * j, d);
        double r = orc_norm(d);
        double s, ds;
        orc_switch(r, m->rcut_smth, m->rcut, &s, &ds);
        w->rij[3 * k + 0] = d[0]; w->rij[3 * k + 1] = d[1]; w->rij[3 * k + 2] = d[2];
        w->rr[k] = r;
        if (s == 0.0) continue;          /* r >= rcut: zero row */
        w->real[k] = 1;
        w->R[4 * k + 0] = s;
        w->R[4 * k + 1] = s * d[0] / r;
        w->R[4 * k + 2] = s * d[1] / r;
        w->R[4 * k + 3] = s * d[2] / r;
    }

    /* Embedding net per non-zero row (a zero row multiplies G by 0). */
    for (int k = 0; k < nm; ++k) {
        if (!w->real[k]) continue;
        int aj = types[nlist[i * nm + k]];
        double *h = w->h + (size_t)k * se, *t = w->t + (size_t)k * se;
        /* L_0(x) = tanh(x W_0 + b_0) */
        const double *W = P + m->emb_W[ai][aj][0], *b = P + m->emb_b[ai][aj][0];
        for (int o = 0; o < m->emb[0]; ++o) {
            t[o] = tanh(w->R[4 * k] * W[o] + b[o]);
            h[o] = t[o];
        }
        int in_off = 0;
        for (int l = 1; l < ne; ++l) {
            int in = m->emb[l - 1], out = m->emb[l], out_off = in_off + in;
            const double *Wl = P + m->emb_W[ai][aj][l], *bl = P + m->emb_b[ai][aj][l];
            int sk = orc_skip_kind(in, out);
            for (int o = 0; o < out; ++o) {
                double z = bl[o];
                for (int q = 0; q < in; ++q) z += h[in_off + q] * Wl[q * out + o];
                t[out_off + o] = tanh(z);
                double skip = sk == 2 ? h[in_off + (o % in)] : (sk == 1 ? h[in_off + o] : 0.0);
                h[out_off + o] = skip + t[out_off + o];
            }
            in_off = out_off;
        }
    }
    const int g_off = se - M;   /* offset of G = last layer output */

    /* Eq. descrpt: T = c R^T G (4 x M), D = T_<^T T (M2 x M). */
    for (int cc = 0; cc < 4; ++cc)
        for (int mm = 0; mm < M; ++mm) {
            double acc = 0.0;
            for (int k = 0; k < nm; ++k)
                if (w->real[k]) acc += w->R[4 * k + cc] * w->h[(size_t)k * se + g_off + mm];
            w->T[cc * M + mm] = c * acc;
        }
    for (int a = 0; a < M2; ++a)
        for (int b2 = 0; b2 < M; ++b2) {
            double acc = 0.0;
            for (int cc = 0; cc < 4; ++cc) acc += w->T[cc * M + a] * w->T[cc * M + b2];
            w->D[a * M + b2] = acc;
        }
    if (desc_out) memcpy(desc_out + (size_t)i * M2 * M, w->D, sizeof(double) * M2 * M);

    /* Eqs. fitting / fitting-detail, per centre type (Remark 1). */
    const int nf = m->n_fit;
    int mf = 0;
    for (int l = 0; l < nf; ++l) if (m->fit[l] > mf) mf = m->fit[l];
    const double *xin = w->D;
    int in = M2 * M;
    for (int l = 0; l < nf; ++l) {
        int out = m->fit[l];
        const double *W = P + m->fit_W[ai][l], *b = P + m->fit_b[ai][l];
        int sk = orc_skip_kind(in, out);
        double *th = w->ft + (size_t)l * mf, *hh = w->fh + (size_t)l * mf;
        for (int o = 0; o < out; ++o) {
            double z = b[o];
            for (int q = 0; q < in; ++q) z += xin[q] * W[(size_t)q * out + o];
            th[o] = tanh(z);
            double skip = sk == 2 ? xin[o % in] : (sk == 1 ? xin[o] : 0.0);
            hh[o] = skip + th[o];
        }
        xin = hh;
        in = out;
    }
    double Ei = P[m->fit_bo[ai]];
    {
        const double *wo = P + m->fit_wo[ai];
        for (int q = 0; q < in; ++q) Ei += xin[q] * wo[q];
    }

    /* ---- back-propagation (Remark 2): dE_i/dD, then dE_i/dT, dE_i/dR~, dE_i/dr_ij */
    double *gh = w->gbuf0, *gx = w->gbuf1;
    for (int q = 0; q < in; ++q) gh[q] = P[m->fit_wo[ai] + q];
    for (int l = nf - 1; l >= 0; --l) {
        int out = m->fit[l];
        int lin = l == 0 ? M2 * M : m->fit[l - 1];
        const double *W = P + m->fit_W[ai][l];
        const double *th = w->ft + (size_t)l * mf;
        int sk = orc_skip_kind(lin, out);
        for (int q = 0; q < lin; ++q) gx[q] = 0.0;
        for (int o = 0; o < out; ++o) {
            double gz = gh[o] * (1.0 - th[o] * th[o]);
            for (int q = 0; q < lin; ++q) gx[q] += gz * W[(size_t)q * out + o];
            if (sk == 2) gx[o % lin] += gh[o];
            else if (sk == 1) gx[o] += gh[o];
        }
        double *tmp = gh; gh = gx; gx = tmp;
    }
    memcpy(w->gD, gh, sizeof(double) * M2 * M);

    /* D[a][b] = sum_c T[c][a] T[c][b]  =>  gT[c][x] = [x<M2] sum_b gD[x][b] T[c][b] + sum_a gD[a][x] T[c][a] */
    for (int cc = 0; cc < 4; ++cc)
        for (int xx = 0; xx < M; ++xx) {
            double acc = 0.0;
            if (xx < M2)
                for (int b2 = 0; b2 < M; ++b2) acc += w->gD[xx * M + b2] * w->T[cc * M + b2];
            for (int a = 0; a < M2; ++a) acc += w->gD[a * M + xx] * w->T[cc * M + a];
            w->gT[cc * M + xx] = acc;
        }

    for (int k = 0; k < nm; ++k) {
        g[3 * k + 0] = g[3 * k + 1] = g[3 * k + 2] = 0.0;
        if (!w->real[k]) continue;
        int aj = types[nlist[i * nm + k]];
        const double *h = w->h + (size_t)k * se, *t = w->t + (size_t)k * se;
        /* T = c sum_k R[k]^T G[k]: gG[k][m] = c sum_c R[k][c] gT[c][m],
         *                          gR[k][c] = c sum_m G[k][m] gT[c][m] */
        double gR[4];
        for (int cc = 0; cc < 4; ++cc) {
            double acc = 0.0;
            for (int mm = 0; mm < M; ++mm) acc += h[g_off + mm] * w->gT[cc * M + mm];
            gR[cc] = c * acc;
        }
        for (int mm = 0; mm < M; ++mm) {
            double acc = 0.0;
            for (int cc = 0; cc < 4; ++cc) acc += w->R[4 * k + cc] * w->gT[cc * M + mm];
            w->gG[mm] = c * acc;
        }
        /* back through the embedding layers */
        double *ga = w->gbuf0, *gb = w->gbuf1;
        for (int mm = 0; mm < M; ++mm) ga[mm] = w->gG[mm];
        int out_off = se - M;
        for (int l = ne - 1; l >= 1; --l) {
            int out = m->emb[l], lin = m->emb[l - 1], in_off = out_off - lin;
            const double *Wl = P + m->emb_W[ai][aj][l];
            int sk = orc_skip_kind(lin, out);
            for (int q = 0; q < lin; ++q) gb[q] = 0.0;
            for (int o = 0; o < out; ++o) {
                double tt = t[out_off + o];
                double gz = ga[o] * (1.0 - tt * tt);
                for (int q = 0; q < lin; ++q) gb[q] += gz * Wl[q * out + o];
                if (sk == 2) gb[o % lin] += ga[o];
                else if (sk == 1) gb[o] += ga[o];
            }
            double *tmp = ga; ga = gb; gb = tmp;
            out_off = in_off;
        }
        double gs = 0.0;
        {
            const double *W0 = P + m->emb_W[ai][aj][0];
            for (int o = 0; o < m->emb[0]; ++o) gs += ga[o] * (1.0 - t[o] * t[o]) * W0[o];
        }
        (void)h;
        gR[0] += gs;
        /* R~ row = s(r) (1, x/r, y/r, z/r):  dR0/dr_b = s' u_b,
         * d(s u_a)/dr_b = s' u_a u_b + s (delta_ab - u_a u_b) / r */
        double r = w->rr[k], s, ds;
        orc_switch(r, m->rcut_smth, m->rcut, &s, &ds);
        double u[3] = {w->rij[3 * k] / r, w->rij[3 * k + 1] / r, w->rij[3 * k + 2] / r};
        for (int bb = 0; bb < 3; ++bb) {
            double acc = gR[0] * ds * u[bb];
            for (int a = 0; a < 3; ++a) {
                double dRa = ds * u[a] * u[bb] + s * ((a == bb ? 1.0 : 0.0) - u[a] * u[bb]) / r;
                acc += gR[1 + a] * dRa;
            }
            g[3 * k + bb] = acc;
        }
    }
    return Ei;
}

/* Energy, forces and virial of the centres 0..nloc-1 for a formatted
 * neighbour list (nlist[nloc][N_m]); atoms nloc..N-1 are only neighbours (the
 * ghost atoms of a sub-region, Sec. 3.1).
 * F_i += dE_i/dr_ij, F_j -= dE_i/dr_ij (Remark 2 and Remark 4: the j-side
 * terms are kept, there is no Newton-3 shortcut), so ghost atoms receive the
 * force increments that Sec. 3.1 sends back to their owners; virial
 * Xi[a][b] = -sum r_ij[a] dE_i/dr_ij[b] over the centres, row-major 3x3;
 * E and atom_energy over the centres.  force is [N][3].  Any output pointer
 * may be NULL except energy. */
int orc_eval_local(const int32_t *idesc, const double *ddesc, const double *params, int64_t N, int64_t nloc,
                   const double *x, const int32_t *types, const double *box, const int32_t *nlist,
                   double *energy, double *force, double *virial, double *atom_energy,
                   double *descriptor)
{
    orc_model m;
    if (orc_parse(idesc, ddesc, &m)) return -1;
    if (nloc < 0 || nloc > N) return -1;
    const int nm = m.nm;
    double *Ei = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *g = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * nm * 3);
    if (!Ei || !g) { free(Ei); free(g); return -2; }
#pragma omp parallel
    {
        orc_ws w;
        orc_ws_alloc(&m, &w);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < nloc; ++i)
            Ei[i] = orc_atom(&m, params, i, x, types, box, nlist, &w, g + (size_t)i * nm * 3,
                             descriptor);
        orc_ws_free(&w);
    }
    double E = 0.0;
    for (int64_t i = 0; i < nloc; ++i) E += Ei[i];
    *energy = E;
    if (atom_energy) memcpy(atom_energy, Ei, sizeof(double) * (size_t)nloc);
    if (force) for (int64_t q = 0; q < 3 * N; ++q) force[q] = 0.0;
    double V[9] = {0};
    for (int64_t i = 0; i < nloc; ++i)
        for (int k = 0; k < nm; ++k) {
            int j = nlist[i * nm + k];
            if (j < 0) continue;
            const double *gk = g + ((size_t)i * nm + k) * 3;
            if (gk[0] == 0.0 && gk[1] == 0.0 && gk[2] == 0.0) continue;
            double d[3];
            orc_min_image(box, x + 3 * i, x + 3 * j, d);
            for (int a = 0; a < 3; ++a) {
                if (force) {
                    force[3 * i + a] += gk[a];
                    force[3 * (int64_t)j + a] -= gk[a];
                }
                for (int b = 0; b < 3; ++b) V[3 * a + b] -= d[a] * gk[b];
            }
        }
    if (virial) memcpy(virial, V, sizeof(V));
    free(Ei);
    free(g);
    return 0;
}

/* All N atoms are centres (a whole periodic system). */
int orc_eval(const int32_t *idesc, const double *ddesc, const double *params, int64_t N,
             const double *x, const int32_t *types, const double *box, const int32_t *nlist,
             double *energy, double *force, double *virial, double *atom_energy,
             double *descriptor)
{
    return orc_eval_local(idesc, ddesc, params, N, N, x, types, box, nlist, energy, force, virial, atom_energy,
                          descriptor);
}

/* ---------------------------------------------------------------------- MD */

static void orc_wrap(double *x, int64_t N, const double *box)
{
    for (int64_t i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = x[3 * i + a];
            double n = floor(v / box[a]);
            double shift = box[a] * n;
            x[3 * i + a] = v - shift;
        }
}

#define ORC_ACC_CONV 9.648533212e-3   /* (eV/A/amu) -> A/fs^2 */
#define ORC_KB 8.617333262e-5         /* eV/K */

/* Velocity-Verlet NVE (Sec. 4): half kick, drift, wrap, candidate rebuild every
 * `rebuild_every` steps (cell list, or brute force in small boxes; rcut + skin), Algorithm 1 every step,
 * force evaluation, half kick.  thermo[s] = (E_pot, E_kin, T, P) after step s
 * (eV, eV, K, eV/A^3), P = (2 E_kin + tr Xi) / (3V).  force (N x 3, in/out)
 * holds F(x) of the input coordinates when *have_force != 0, and is computed
 * first otherwise.  Returns 0, or the number of formatting overflows seen
 * (positive), or <0 on a candidate-capacity failure. */
int64_t orc_md(const int32_t *idesc, const double *ddesc, const double *params, int64_t N,
               double *x, double *v, const int32_t *types, const double *box,
               const double *mass_per_type, double dt, int32_t nsteps, int32_t rebuild_every,
               double skin, int32_t cap, double *force, int32_t *have_force, double *thermo)
{
    orc_model m;
    if (orc_parse(idesc, ddesc, &m)) return -1;
    const int nm = m.nm, T = m.ntypes;
    int32_t *ncand = malloc(sizeof(int32_t) * (size_t)N);
    int32_t *cand = malloc(sizeof(int32_t) * (size_t)N * cap);
    int32_t *nlist = malloc(sizeof(int32_t) * (size_t)N * nm);
    int32_t *nreal = malloc(sizeof(int32_t) * (size_t)N * T);
    int64_t *ovf = malloc(sizeof(int64_t) * (size_t)N);
    double *xref = malloc(sizeof(double) * 3 * (size_t)N);
    int64_t status = 0;
    double E = 0.0, V[9];
    const double vol = box[0] * box[1] * box[2];
    if (orc_candidates_any(N, x, box, m.rcut + skin, cap, ncand, cand)) { status = -3; goto done; }
    memcpy(xref, x, sizeof(double) * 3 * (size_t)N);
    if (!*have_force) {
        orc_format(N, x, types, box, ncand, cand, cap, T, m.sel, m.rcut, nlist, nreal, ovf);
        for (int64_t i = 0; i < N; ++i) status += ovf[i];
        orc_eval(idesc, ddesc, params, N, x, types, box, nlist, &E, force, V, NULL, NULL);
        *have_force = 1;
    }
    for (int s = 1; s <= nsteps; ++s) {
        for (int64_t i = 0; i < N; ++i) {
            double f = 0.5 * dt * ORC_ACC_CONV / mass_per_type[types[i]];
            for (int a = 0; a < 3; ++a) v[3 * i + a] += f * force[3 * i + a];
        }
        for (int64_t q = 0; q < 3 * N; ++q) x[q] += dt * v[q];
        orc_wrap(x, N, box);
        int rebuild = rebuild_every > 0 && s % rebuild_every == 0;
        if (!rebuild && skin > 0.0) {
            /* rebuild early once an atom has moved more than skin/2 */
            for (int64_t i = 0; i < N && !rebuild; ++i) {
                double d[3];
                orc_min_image(box, xref + 3 * i, x + 3 * i, d);
                double r = orc_norm(d);
                if (r * r > 0.25 * skin * skin) rebuild = 1;
            }
        }
        if (rebuild) {
            if (orc_candidates_any(N, x, box, m.rcut + skin, cap, ncand, cand)) { status = -3; goto done; }
            memcpy(xref, x, sizeof(double) * 3 * (size_t)N);
        }
        orc_format(N, x, types, box, ncand, cand, cap, T, m.sel, m.rcut, nlist, nreal, ovf);
        for (int64_t i = 0; i < N; ++i) status += ovf[i];
        orc_eval(idesc, ddesc, params, N, x, types, box, nlist, &E, force, V, NULL, NULL);
        double ke = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double mi = mass_per_type[types[i]];
            double f = 0.5 * dt * ORC_ACC_CONV / mi;
            for (int a = 0; a < 3; ++a) {
                v[3 * i + a] += f * force[3 * i + a];
                ke += 0.5 * mi * v[3 * i + a] * v[3 * i + a];
            }
        }
        ke /= ORC_ACC_CONV;
        if (thermo) {
            double dof = 3.0 * (double)N - 3.0;
            thermo[4 * (s - 1) + 0] = E;
            thermo[4 * (s - 1) + 1] = ke;
            thermo[4 * (s - 1) + 2] = 2.0 * ke / (dof * ORC_KB);
            thermo[4 * (s - 1) + 3] = (2.0 * ke + V[0] + V[4] + V[8]) / (3.0 * vol);
        }
    }
done:
    free(ncand); free(cand); free(nlist); free(nreal); free(ovf); free(xref);
    return status;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------ parameter gradient */

/* Gradient with respect to every model parameter of
 *     Phi(W) = cE * E(W) + sum_i lambda_i . F_i(W)
 *            = cE * E(W) - sum_i lambda_i . dE/dr_i,
 * i.e. the parameter gradient of any loss on the energy and forces, with
 * cE = dLoss/dE and lambda_i = dLoss/dF_i (Remark 2: F = -grad E).  Per atom
 * i, the second term is the directional derivative of E_i along the
 * neighbour displacements delta r_ij = lambda_j - lambda_i; it is evaluated
 * by forward tangents through the environment matrix (Algorithm 2), the
 * embedding net, the descriptor and the fitting net, then differentiated by
 * plain reverse mode.  grad[nparams] is overwritten. */
typedef struct {
    double *R, *dR, *J;      /* [nm][4], [nm][4], [nm][4][3] */
    double *s, *ds;          /* [nm] */
    int *real;
    double *h, *t, *dh;      /* embedding [nm][se] */
    double *T, *dT, *Tb, *dTb;   /* [4][M] */
    double *D, *dD, *Db, *dDb;   /* [M2*M] */
    double *fh, *ft, *fdh;   /* fitting [nf][mf] */
    double *a0, *a1, *b0, *b1;   /* adjoint buffers [max width] */
    double *g;               /* per-thread gradient [nparams] */
} orc_gws;

static void orc_gws_alloc(const orc_model *m, orc_gws *w)
{
    int nm = m->nm, M = m->emb[m->n_emb - 1], se = 0, mf = 0;
    for (int l = 0; l < m->n_emb; ++l) se += m->emb[l];
    for (int l = 0; l < m->n_fit; ++l) if (m->fit[l] > mf) mf = m->fit[l];
    int mw = orc_max_width(m);
    w->R = calloc((size_t)nm * 4, 8); w->dR = calloc((size_t)nm * 4, 8); w->J = calloc((size_t)nm * 12, 8);
    w->s = calloc(nm, 8); w->ds = calloc(nm, 8); w->real = calloc(nm, sizeof(int));
    w->h = calloc((size_t)nm * se, 8); w->t = calloc((size_t)nm * se, 8); w->dh = calloc((size_t)nm * se, 8);
    w->T = calloc(4 * M, 8); w->dT = calloc(4 * M, 8); w->Tb = calloc(4 * M, 8); w->dTb = calloc(4 * M, 8);
    w->D = calloc(m->m2 * M, 8); w->dD = calloc(m->m2 * M, 8); w->Db = calloc(m->m2 * M, 8); w->dDb = calloc(m->m2 * M, 8);
    w->fh = calloc((size_t)m->n_fit * mf, 8); w->ft = calloc((size_t)m->n_fit * mf, 8); w->fdh = calloc((size_t)m->n_fit * mf, 8);
    w->a0 = calloc(mw, 8); w->a1 = calloc(mw, 8); w->b0 = calloc(mw, 8); w->b1 = calloc(mw, 8);
    w->g = calloc((size_t)m->nparams, 8);
}

static void orc_gws_free(orc_gws *w)
{
    free(w->R); free(w->dR); free(w->J); free(w->s); free(w->ds); free(w->real);
    free(w->h); free(w->t); free(w->dh); free(w->T); free(w->dT); free(w->Tb); free(w->dTb);
    free(w->D); free(w->dD); free(w->Db); free(w->dDb); free(w->fh); free(w->ft); free(w->fdh);
    free(w->a0); free(w->a1); free(w->b0); free(w->b1); free(w->g);
}

/* reverse through one layer  h = skip(x) + tanh(x W + b),  dh = skip(dx) + (1-t^2)(dx W)
 * given the primal/tangent adjoints hb, dhb of the output; accumulates the
 * adjoints of the input into xb, dxb and the weight gradient into gW, gb. */
static void orc_layer_rev(const double *x, const double *dx, const double *t, const double *W, int in, int out,
                          int sk, const double *hb, const double *dhb, double *xb, double *dxb, double *gW,
                          double *gb)
{
    for (int q = 0; q < in; ++q) { xb[q] = 0.0; dxb[q] = 0.0; }
    for (int o = 0; o < out; ++o) {
        /* recompute dz = dx . W[:, o] */
        double dz = 0.0;
        for (int q = 0; q < in; ++q) dz += dx[q] * W[(size_t)q * out + o];
        const double tt = t[o], one = 1.0 - tt * tt;
        double tb = hb[o];
        const double dtb = dhb[o];
        const double dzb = one * dtb;
        tb += -2.0 * tt * dz * dtb;
        const double zb = one * tb;
        for (int q = 0; q < in; ++q) {
            gW[(size_t)q * out + o] += x[q] * zb + dx[q] * dzb;
            xb[q] += zb * W[(size_t)q * out + o];
            dxb[q] += dzb * W[(size_t)q * out + o];
        }
        gb[o] += zb;
        if (sk == 2) { xb[o % in] += hb[o]; dxb[o % in] += dhb[o]; }
        else if (sk == 1) { xb[o] += hb[o]; dxb[o] += dhb[o]; }
    }
}

static void orc_atom_grad(const orc_model *m, const double *P, int64_t i, const double *x, const int32_t *types,
                          const double *box, const int32_t *nlist, double cE, const double *lam, orc_gws *w)
{
    const int nm = m->nm, ne = m->n_emb, M = m->emb[ne - 1], M2 = m->m2, nf = m->n_fit;
    int se = 0, mf = 0;
    for (int l = 0; l < ne; ++l) se += m->emb[l];
    for (int l = 0; l < nf; ++l) if (m->fit[l] > mf) mf = m->fit[l];
    const int ai = types[i];
    const double c = m->desc_scale_nm ? 1.0 / nm : 1.0;
    double *g = w->g;

    /* rows of the environment matrix, their Jacobians and tangents (Algorithm 2) */
    for (int k = 0; k < nm; ++k) {
        w->real[k] = 0;
        int j = nlist[i * nm + k];
        if (j < 0) continue;
        double d[3];
        orc_min_image(box, x + 3 * i, x + 3 * j, d);
        double r = orc_norm(d), s, ds;
        orc_switch(r, m->rcut_smth, m->rcut, &s, &ds);
        if (s == 0.0) continue;
        w->real[k] = 1;
        double u[3] = {d[0] / r, d[1] / r, d[2] / r};
        double *R = w->R + 4 * k, *J = w->J + 12 * k;
        R[0] = s; R[1] = s * u[0]; R[2] = s * u[1]; R[3] = s * u[2];
        for (int b = 0; b < 3; ++b) {
            J[b] = ds * u[b];
            for (int a = 0; a < 3; ++a)
                J[3 * (1 + a) + b] = ds * u[a] * u[b] + s * ((a == b ? 1.0 : 0.0) - u[a] * u[b]) / r;
        }
        double dr[3];
        for (int b = 0; b < 3; ++b) dr[b] = lam[3 * (int64_t)j + b] - lam[3 * i + b];
        for (int cc = 0; cc < 4; ++cc) {
            double acc = 0.0;
            for (int b = 0; b < 3; ++b) acc += J[3 * cc + b] * dr[b];
            w->dR[4 * k + cc] = acc;
        }
        w->s[k] = s;
        w->ds[k] = w->dR[4 * k];
    }
    /* embedding: primal and tangent */
    for (int k = 0; k < nm; ++k) {
        if (!w->real[k]) continue;
        int aj = types[nlist[i * nm + k]];
        double *h = w->h + (size_t)k * se, *t = w->t + (size_t)k * se, *dh = w->dh + (size_t)k * se;
        const double *W0 = P + m->emb_W[ai][aj][0], *b0 = P + m->emb_b[ai][aj][0];
        for (int o = 0; o < m->emb[0]; ++o) {
            t[o] = tanh(w->s[k] * W0[o] + b0[o]);
            h[o] = t[o];
            dh[o] = (1.0 - t[o] * t[o]) * (w->ds[k] * W0[o]);
        }
        int in_off = 0;
        for (int l = 1; l < ne; ++l) {
            int in = m->emb[l - 1], out = m->emb[l], out_off = in_off + in;
            const double *Wl = P + m->emb_W[ai][aj][l], *bl = P + m->emb_b[ai][aj][l];
            int sk = orc_skip_kind(in, out);
            for (int o = 0; o < out; ++o) {
                double z = bl[o], dz = 0.0;
                for (int q = 0; q < in; ++q) {
                    z += h[in_off + q] * Wl[q * out + o];
                    dz += dh[in_off + q] * Wl[q * out + o];
                }
                t[out_off + o] = tanh(z);
                double skip = sk == 2 ? h[in_off + (o % in)] : (sk == 1 ? h[in_off + o] : 0.0);
                double dskip = sk == 2 ? dh[in_off + (o % in)] : (sk == 1 ? dh[in_off + o] : 0.0);
                h[out_off + o] = skip + t[out_off + o];
                dh[out_off + o] = dskip + (1.0 - t[out_off + o] * t[out_off + o]) * dz;
            }
            in_off = out_off;
        }
    }
    const int g_off = se - M;
    /* descriptor and its tangent (Eq. descrpt) */
    for (int cc = 0; cc < 4; ++cc)
        for (int mm = 0; mm < M; ++mm) {
            double acc = 0.0, dacc = 0.0;
            for (int k = 0; k < nm; ++k) {
                if (!w->real[k]) continue;
                const double G = w->h[(size_t)k * se + g_off + mm], dG = w->dh[(size_t)k * se + g_off + mm];
                acc += w->R[4 * k + cc] * G;
                dacc += w->dR[4 * k + cc] * G + w->R[4 * k + cc] * dG;
            }
            w->T[cc * M + mm] = c * acc;
            w->dT[cc * M + mm] = c * dacc;
        }
    for (int a = 0; a < M2; ++a)
        for (int b = 0; b < M; ++b) {
            double acc = 0.0, dacc = 0.0;
            for (int cc = 0; cc < 4; ++cc) {
                acc += w->T[cc * M + a] * w->T[cc * M + b];
                dacc += w->dT[cc * M + a] * w->T[cc * M + b] + w->T[cc * M + a] * w->dT[cc * M + b];
            }
            w->D[a * M + b] = acc;
            w->dD[a * M + b] = dacc;
        }
    /* fitting net: primal and tangent */
    const double *xin = w->D, *dxin = w->dD;
    int in = M2 * M;
    for (int l = 0; l < nf; ++l) {
        int out = m->fit[l];
        const double *W = P + m->fit_W[ai][l], *b = P + m->fit_b[ai][l];
        int sk = orc_skip_kind(in, out);
        double *th = w->ft + (size_t)l * mf, *hh = w->fh + (size_t)l * mf, *dhh = w->fdh + (size_t)l * mf;
        for (int o = 0; o < out; ++o) {
            double z = b[o], dz = 0.0;
            for (int q = 0; q < in; ++q) {
                z += xin[q] * W[(size_t)q * out + o];
                dz += dxin[q] * W[(size_t)q * out + o];
            }
            th[o] = tanh(z);
            double skip = sk == 2 ? xin[o % in] : (sk == 1 ? xin[o] : 0.0);
            double dskip = sk == 2 ? dxin[o % in] : (sk == 1 ? dxin[o] : 0.0);
            hh[o] = skip + th[o];
            dhh[o] = dskip + (1.0 - th[o] * th[o]) * dz;
        }
        xin = hh;
        dxin = dhh;
        in = out;
    }
    /* reverse: Phi_i = cE E_i - dE_i,  E_i = h_L . wo + bo,  dE_i = dh_L . wo */
    {
        const double *wo = P + m->fit_wo[ai];
        double *gwo = g + m->fit_wo[ai];
        for (int q = 0; q < in; ++q) {
            gwo[q] += cE * xin[q] - dxin[q];
            w->a0[q] = cE * wo[q];
            w->b0[q] = -wo[q];
        }
        g[m->fit_bo[ai]] += cE;
    }
    double *hb = w->a0, *dhb = w->b0, *xb = w->a1, *dxb = w->b1;
    for (int l = nf - 1; l >= 0; --l) {
        int out = m->fit[l], lin = l == 0 ? M2 * M : m->fit[l - 1];
        const double *xl = l == 0 ? w->D : w->fh + (size_t)(l - 1) * mf;
        const double *dxl = l == 0 ? w->dD : w->fdh + (size_t)(l - 1) * mf;
        orc_layer_rev(xl, dxl, w->ft + (size_t)l * mf, P + m->fit_W[ai][l], lin, out, orc_skip_kind(lin, out),
                      hb, dhb, xb, dxb, g + m->fit_W[ai][l], g + m->fit_b[ai][l]);
        double *t1 = hb; hb = xb; xb = t1;
        double *t2 = dhb; dhb = dxb; dxb = t2;
    }
    memcpy(w->Db, hb, sizeof(double) * M2 * M);
    memcpy(w->dDb, dhb, sizeof(double) * M2 * M);
    /* descriptor reverse: D = T_<^T T, dD = dT_<^T T + T_<^T dT */
    for (int cc = 0; cc < 4; ++cc)
        for (int xx = 0; xx < M; ++xx) {
            double tb = 0.0, dtb = 0.0;
            if (xx < M2)
                for (int b = 0; b < M; ++b) {
                    tb += w->Db[xx * M + b] * w->T[cc * M + b] + w->dDb[xx * M + b] * w->dT[cc * M + b];
                    dtb += w->dDb[xx * M + b] * w->T[cc * M + b];
                }
            for (int a = 0; a < M2; ++a) {
                tb += w->Db[a * M + xx] * w->T[cc * M + a] + w->dDb[a * M + xx] * w->dT[cc * M + a];
                dtb += w->dDb[a * M + xx] * w->T[cc * M + a];
            }
            w->Tb[cc * M + xx] = tb;
            w->dTb[cc * M + xx] = dtb;
        }
    /* per row: Gb = c (R Tb + dR dTb), dGb = c R dTb, then back through the embedding */
    for (int k = 0; k < nm; ++k) {
        if (!w->real[k]) continue;
        int aj = types[nlist[i * nm + k]];
        const double *h = w->h + (size_t)k * se, *t = w->t + (size_t)k * se, *dh = w->dh + (size_t)k * se;
        double *Gb = w->a0, *dGb = w->b0;
        for (int mm = 0; mm < M; ++mm) {
            double acc = 0.0, dacc = 0.0;
            for (int cc = 0; cc < 4; ++cc) {
                acc += w->R[4 * k + cc] * w->Tb[cc * M + mm] + w->dR[4 * k + cc] * w->dTb[cc * M + mm];
                dacc += w->R[4 * k + cc] * w->dTb[cc * M + mm];
            }
            Gb[mm] = c * acc;
            dGb[mm] = c * dacc;
        }
        double *ob = w->a0, *dob = w->b0, *ib = w->a1, *dib = w->b1;
        int out_off = se - M;
        for (int l = ne - 1; l >= 1; --l) {
            int out = m->emb[l], lin = m->emb[l - 1], in_off = out_off - lin;
            orc_layer_rev(h + in_off, dh + in_off, t + out_off, P + m->emb_W[ai][aj][l], lin, out,
                          orc_skip_kind(lin, out), ob, dob, ib, dib, g + m->emb_W[ai][aj][l],
                          g + m->emb_b[ai][aj][l]);
            double *t1 = ob; ob = ib; ib = t1;
            double *t2 = dob; dob = dib; dib = t2;
            out_off = in_off;
        }
        /* layer 0: h0 = tanh(s W0 + b0), dh0 = (1 - t0^2) ds W0 */
        const double *W0 = P + m->emb_W[ai][aj][0];
        double *gW0 = g + m->emb_W[ai][aj][0], *gb0 = g + m->emb_b[ai][aj][0];
        for (int o = 0; o < m->emb[0]; ++o) {
            const double tt = t[o], one = 1.0 - tt * tt, dz = w->ds[k] * W0[o];
            double tb = ob[o];
            const double dzb = one * dob[o];
            tb += -2.0 * tt * dz * dob[o];
            const double zb = one * tb;
            gW0[o] += w->s[k] * zb + w->ds[k] * dzb;
            gb0[o] += zb;
        }
    }
}

int orc_param_grad(const int32_t *idesc, const double *ddesc, const double *params, int64_t N, const double *x,
                   const int32_t *types, const double *box, const int32_t *nlist, double cE, const double *lam,
                   double *grad)
{
    orc_model m;
    if (orc_parse(idesc, ddesc, &m)) return -1;
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    double *parts = calloc((size_t)nth * m.nparams, sizeof(double));
    if (!parts) return -2;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        orc_gws w;
        orc_gws_alloc(&m, &w);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i) orc_atom_grad(&m, params, i, x, types, box, nlist, cE, lam, &w);
        memcpy(parts + (size_t)tid * m.nparams, w.g, sizeof(double) * m.nparams);
        orc_gws_free(&w);
    }
    for (long q = 0; q < m.nparams; ++q) {
        double acc = 0.0;
        for (int th = 0; th < nth; ++th) acc += parts[(size_t)th * m.nparams + q];
        grad[q] = acc;
    }
    free(parts);
    return 0;
}
