/*
 * CPU oracle for the CCD hot path of "Time of Impact Dataset for Continuous
 * Collision Detection and a Scalable Conservative Algorithm" (Belgrod et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.  It shares no code,
 * header, table or constant generator with the CUDA library; it is written
 * plainly so that each step can be checked against the paper by eye.
 *
 * Contents
 *   1. Box construction, Section "Construction of the Boxes": FP64 extents
 *      over t=0 and t=1, then single precision by round-to-nearest followed by
 *      one nextafterf step when the nearest value is not conservative.
 *   2. Broad phase, Section "Broad-Phase" / Algorithm 2: the candidate set
 *      it reaches is, by the "Guarantees" section, exactly the set of
 *      vertex-face and edge-edge pairs whose boxes overlap.  Two independent
 *      implementations: O(n^2) brute force and a serial sweep on one axis.
 *   3. Narrow phase, Section "Narrow-Phase" / Algorithm 3 (ProcessInterval),
 *      with the readings of the paper's silent points stated at each step:
 *      a serial depth-first interval bisection in FP64.
 *
 * Compiled with -ffp-contract=off: every fused multiply-add below is an
 * explicit call to fma(), and no other expression may be contracted.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* 1. Boxes                                                            */
/* ------------------------------------------------------------------ */

/* Section "Construction of the Boxes": round to the nearest float, and if that
 * value is not below (reading: not <=) the double, step down once. */
static float f32_down(double x)
{
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}

static float f32_up(double x)
{
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

/* Vertex ids of box b (global numbering: vertices, then edges, then faces).
 * Returns the number of vertices (1, 2 or 3). */
static int box_vertices(int64_t b, int64_t nV, int64_t nE, const int32_t *E,
                        const int32_t *F, int64_t ids[3])
{
    if (b < nV) { ids[0] = b; return 1; }
    if (b < nV + nE) {
        int64_t e = b - nV;
        ids[0] = E[2 * e]; ids[1] = E[2 * e + 1];
        return 2;
    }
    int64_t f = b - nV - nE;
    ids[0] = F[3 * f]; ids[1] = F[3 * f + 1]; ids[2] = F[3 * f + 2];
    return 3;
}

/* V0, V1: (nV, 3) row-major doubles.  Outputs (nB, 3) row-major. */
void oracle_boxes(int64_t nV, const double *V0, const double *V1,
                  int64_t nE, const int32_t *E, int64_t nF, const int32_t *F,
                  double *lo64, double *hi64, float *lo32, float *hi32)
{
    int64_t nB = nV + nE + nF;
    for (int64_t b = 0; b < nB; ++b) {
        int64_t ids[3];
        int n = box_vertices(b, nV, nE, E, F, ids);
        for (int a = 0; a < 3; ++a) {
            double lo = INFINITY, hi = -INFINITY;
            for (int k = 0; k < n; ++k) {
                double x0 = V0[3 * ids[k] + a], x1 = V1[3 * ids[k] + a];
                if (x0 < lo) lo = x0;
                if (x1 < lo) lo = x1;
                if (x0 > hi) hi = x0;
                if (x1 > hi) hi = x1;
            }
            lo64[3 * b + a] = lo;
            hi64[3 * b + a] = hi;
            if (lo32) lo32[3 * b + a] = f32_down(lo);
            if (hi32) hi32[3 * b + a] = f32_up(hi);
        }
    }
}

/* ------------------------------------------------------------------ */
/* 2. Broad phase                                                      */
/* ------------------------------------------------------------------ */

/* Closed-interval overlap on all three axes ("b_i ∩ b_j ≠ ∅"). */
static int overlap64(const double *lo, const double *hi, int64_t i, int64_t j)
{
    for (int a = 0; a < 3; ++a)
        if (lo[3 * i + a] > hi[3 * j + a] || lo[3 * j + a] > hi[3 * i + a]) return 0;
    return 1;
}

static int overlap32(const float *lo, const float *hi, int64_t i, int64_t j)
{
    for (int a = 0; a < 3; ++a)
        if (lo[3 * i + a] > hi[3 * j + a] || lo[3 * j + a] > hi[3 * i + a]) return 0;
    return 1;
}

static int shares_vertex(const int64_t *a, int na, const int64_t *b, int nb)
{
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j)
            if (a[i] == b[j]) return 1;
    return 0;
}

typedef struct { int64_t a, b; } pair64;

static int cmp_pair(const void *x, const void *y)
{
    const pair64 *p = x, *q = y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

typedef struct {
    pair64 *vf, *ee;
    int64_t nvf, nee, cap_vf, cap_ee;
} pairlist;

static int push(pair64 **arr, int64_t *n, int64_t *cap, int64_t a, int64_t b)
{
    if (*n == *cap) {
        int64_t nc = *cap ? 2 * *cap : 1024;
        pair64 *p = realloc(*arr, (size_t)nc * sizeof(pair64));
        if (!p) return -1;
        *arr = p; *cap = nc;
    }
    (*arr)[*n].a = a; (*arr)[*n].b = b; (*n)++;
    return 0;
}

/* Candidate rule for an unordered box pair (the dataset's rule, Section
 * "Dataset Generation"): only vertex-face and edge-edge, and no pair whose
 * primitives share a vertex.  Emits the canonical (v, f) or (e_lo, e_hi). */
static int emit_if_candidate(pairlist *out, int64_t bi, int64_t bj,
                             int64_t nV, int64_t nE, const int32_t *E, const int32_t *F)
{
    int ti = bi < nV ? 0 : (bi < nV + nE ? 1 : 2);
    int tj = bj < nV ? 0 : (bj < nV + nE ? 1 : 2);
    int vf = (ti == 0 && tj == 2) || (ti == 2 && tj == 0);
    int ee = (ti == 1 && tj == 1);
    if (!vf && !ee) return 0;
    int64_t a[3], b[3];
    int na = box_vertices(bi, nV, nE, E, F, a);
    int nb = box_vertices(bj, nV, nE, E, F, b);
    if (shares_vertex(a, na, b, nb)) return 0;
    if (vf) {
        int64_t v = ti == 0 ? bi : bj;
        int64_t f = (ti == 2 ? bi : bj) - nV - nE;
        return push(&out->vf, &out->nvf, &out->cap_vf, v, f);
    }
    int64_t e1 = bi - nV, e2 = bj - nV;
    if (e1 > e2) { int64_t t = e1; e1 = e2; e2 = t; }
    return push(&out->ee, &out->nee, &out->cap_ee, e1, e2);
}

static void finish_lists(pairlist *pl, int64_t *vf_out, int64_t vf_cap, int64_t *n_vf,
                         int64_t *ee_out, int64_t ee_cap, int64_t *n_ee)
{
    qsort(pl->vf, (size_t)pl->nvf, sizeof(pair64), cmp_pair);
    qsort(pl->ee, (size_t)pl->nee, sizeof(pair64), cmp_pair);
    *n_vf = pl->nvf;
    *n_ee = pl->nee;
    for (int64_t i = 0; i < pl->nvf && i < vf_cap; ++i) {
        vf_out[2 * i] = pl->vf[i].a; vf_out[2 * i + 1] = pl->vf[i].b;
    }
    for (int64_t i = 0; i < pl->nee && i < ee_cap; ++i) {
        ee_out[2 * i] = pl->ee[i].a; ee_out[2 * i + 1] = pl->ee[i].b;
    }
    free(pl->vf);
    free(pl->ee);
}

/* (i) O(n^2) brute force over every box pair.  use32 selects the FP32 boxes
 * (the paper's broad-phase set) instead of the FP64 extents.  Returns 0, or
 * -1 on allocation failure.  Output lists are sorted lexicographically; the
 * totals are always written, at most *_cap pairs are copied. */
int oracle_broad_brute(int64_t nV, int64_t nE, const int32_t *E, int64_t nF, const int32_t *F,
                       const double *lo64, const double *hi64, const float *lo32, const float *hi32,
                       int use32,
                       int64_t *vf_out, int64_t vf_cap, int64_t *n_vf,
                       int64_t *ee_out, int64_t ee_cap, int64_t *n_ee)
{
    pairlist pl = {0};
    int64_t nB = nV + nE + nF;
    for (int64_t i = 0; i < nB; ++i)
        for (int64_t j = i + 1; j < nB; ++j) {
            int ov = use32 ? overlap32(lo32, hi32, i, j) : overlap64(lo64, hi64, i, j);
            if (ov && emit_if_candidate(&pl, i, j, nV, nE, E, F)) return -1;
        }
    finish_lists(&pl, vf_out, vf_cap, n_vf, ee_out, ee_cap, n_ee);
    return 0;
}

/* (ii) Serial sweep (Algorithm 2 without its queue): sort by the minimum on
 * the axis of largest centre variance, then for each box scan forward while
 * the next minimum is <= this maximum, testing the other two axes. */
static const double *g_sort_lo;
static const float *g_sort_lo32;
static int g_sort_axis;

static int cmp_box64(const void *x, const void *y)
{
    int64_t i = *(const int64_t *)x, j = *(const int64_t *)y;
    double a = g_sort_lo[3 * i + g_sort_axis], b = g_sort_lo[3 * j + g_sort_axis];
    if (a != b) return a < b ? -1 : 1;
    return i < j ? -1 : (i > j);
}

static int cmp_box32(const void *x, const void *y)
{
    int64_t i = *(const int64_t *)x, j = *(const int64_t *)y;
    float a = g_sort_lo32[3 * i + g_sort_axis], b = g_sort_lo32[3 * j + g_sort_axis];
    if (a != b) return a < b ? -1 : 1;
    return i < j ? -1 : (i > j);
}

int oracle_broad_sweep(int64_t nV, int64_t nE, const int32_t *E, int64_t nF, const int32_t *F,
                       const double *lo64, const double *hi64, const float *lo32, const float *hi32,
                       int use32,
                       int64_t *vf_out, int64_t vf_cap, int64_t *n_vf,
                       int64_t *ee_out, int64_t ee_cap, int64_t *n_ee)
{
    int64_t nB = nV + nE + nF;
    /* Box centres and their variance per axis (Algorithm 2, first lines). */
    double mean[3] = {0, 0, 0}, var[3] = {0, 0, 0};
    for (int64_t i = 0; i < nB; ++i)
        for (int a = 0; a < 3; ++a) {
            double c = use32 ? 0.5 * ((double)lo32[3 * i + a] + (double)hi32[3 * i + a])
                             : 0.5 * (lo64[3 * i + a] + hi64[3 * i + a]);
            mean[a] += c;
        }
    for (int a = 0; a < 3; ++a) mean[a] /= (double)(nB > 0 ? nB : 1);
    for (int64_t i = 0; i < nB; ++i)
        for (int a = 0; a < 3; ++a) {
            double c = use32 ? 0.5 * ((double)lo32[3 * i + a] + (double)hi32[3 * i + a])
                             : 0.5 * (lo64[3 * i + a] + hi64[3 * i + a]);
            var[a] += (c - mean[a]) * (c - mean[a]);
        }
    int ax = 0;
    for (int a = 1; a < 3; ++a)
        if (var[a] > var[ax]) ax = a;

    int64_t *order = malloc((size_t)(nB > 0 ? nB : 1) * sizeof(int64_t));
    if (!order) return -1;
    for (int64_t i = 0; i < nB; ++i) order[i] = i;
    g_sort_axis = ax;
    g_sort_lo = lo64;
    g_sort_lo32 = lo32;
    qsort(order, (size_t)nB, sizeof(int64_t), use32 ? cmp_box32 : cmp_box64);

    /* The outer loop is split over OpenMP threads, each with its own list;
     * the lists are concatenated and sorted, so the result does not depend on
     * the thread count. */
    pairlist pl = {0};
    int failed = 0;
#pragma omp parallel
    {
        pairlist mine = {0};
#pragma omp for schedule(dynamic, 512)
        for (int64_t s = 0; s < nB; ++s) {
            int64_t i = order[s];
            for (int64_t r = s + 1; r < nB; ++r) {
                int64_t j = order[r];
                if (use32 ? (lo32[3 * j + ax] > hi32[3 * i + ax]) : (lo64[3 * j + ax] > hi64[3 * i + ax]))
                    break; /* sorted: no later box can overlap on the sweep axis */
                int ov = use32 ? overlap32(lo32, hi32, i, j) : overlap64(lo64, hi64, i, j);
                if (ov && emit_if_candidate(&mine, i, j, nV, nE, E, F)) failed = 1;
            }
        }
#pragma omp critical
        {
            for (int64_t k = 0; k < mine.nvf && !failed; ++k)
                if (push(&pl.vf, &pl.nvf, &pl.cap_vf, mine.vf[k].a, mine.vf[k].b)) failed = 1;
            for (int64_t k = 0; k < mine.nee && !failed; ++k)
                if (push(&pl.ee, &pl.nee, &pl.cap_ee, mine.ee[k].a, mine.ee[k].b)) failed = 1;
        }
        free(mine.vf);
        free(mine.ee);
    }
    free(order);
    if (failed) { free(pl.vf); free(pl.ee); return -1; }
    finish_lists(&pl, vf_out, vf_cap, n_vf, ee_out, ee_cap, n_ee);
    return 0;
}

/* ------------------------------------------------------------------ */
/* 3. Narrow phase                                                     */
/* ------------------------------------------------------------------ */

/* Interval I = I_t x I_u x I_v with dyadic ends: along axis k (0 = t, 1 = u,
 * 2 = v) it is [n_k / 2^l_k, (n_k + 1) / 2^l_k].  Midpoints are exact. */
typedef struct { uint64_t n[3]; int l[3]; } interval;

#define LEVEL_CAP 53   /* n / 2^l stays an exact double up to this level */

static double dyadic(uint64_t n, int l) { return ldexp((double)n, -l); }

typedef struct {
    int vf;            /* 1 = vertex-face, 0 = edge-edge */
    double c0[3][3];   /* c0[j][x]: vector j at t = 0, axis x */
    double dc[3][3];   /* c1 - c0 */
    double ebox[3];    /* half-width of C_eps enlarged by min_sep, per axis */
    double L[3];       /* split weights for t, u, v */
} query;

/*
 * Per-query set-up.  The four trajectories x(t) = x0 + t (x1 - x0).
 *   vertex-face (P; T0, T1, T2): F = w - u e1 - v e2 with w = P - T0,
 *                                e1 = T1 - T0, e2 = T2 - T0;
 *   edge-edge (A0, A1; B0, B1):  F = w + u ea - v eb with w = A0 - B0,
 *                                ea = A1 - A0, eb = B1 - B0.
 * Each vector j is stored by its rounded values c0 at t = 0 and the rounded
 * difference dc = fl(c1 - c0) to its value c1 at t = 1; at time t it is
 * evaluated as fma(t, dc, c0).
 *
 * Error box C_eps (the paper cites it, Wang et al. Eq. 5, without the
 * formula; this is the bound derived for the expression tree used here): every
 * computed corner value is within 46 u m_x of the exact one, u = 2^-53, m_x the
 * largest |coordinate| on axis x over the 8 input points (floored at 2^-960 to
 * cover gradual underflow).  eps_x = 48 u m_x leaves slack for second-order
 * terms and for the rounding of the product; min_sep enlarges the box
 * (Section "Avoiding Time of Impacts Equal to Zero"), and the sum is moved one
 * ulp up so that its rounding cannot shrink it.
 */
static void setup_query(query *q, int vf, const double *V0, const double *V1,
                        const int64_t ids[4], double min_sep)
{
    /* ids: VF (P, T0, T1, T2); EE (A0, A1, B0, B1). */
    int64_t x_of[3], y_of[3]; /* vector j = X - Y */
    q->vf = vf;
    if (vf) {
        x_of[0] = ids[0]; y_of[0] = ids[1];
        x_of[1] = ids[2]; y_of[1] = ids[1];
        x_of[2] = ids[3]; y_of[2] = ids[1];
    } else {
        x_of[0] = ids[0]; y_of[0] = ids[2];
        x_of[1] = ids[1]; y_of[1] = ids[0];
        x_of[2] = ids[3]; y_of[2] = ids[2];
    }
    for (int j = 0; j < 3; ++j)
        for (int x = 0; x < 3; ++x) {
            double a = V0[3 * x_of[j] + x] - V0[3 * y_of[j] + x];
            double b = V1[3 * x_of[j] + x] - V1[3 * y_of[j] + x];
            q->c0[j][x] = a;
            q->dc[j][x] = b - a;
        }
    for (int x = 0; x < 3; ++x) {
        double m = 0x1p-960;
        for (int k = 0; k < 4; ++k) {
            if (fabs(V0[3 * ids[k] + x]) > m) m = fabs(V0[3 * ids[k] + x]);
            if (fabs(V1[3 * ids[k] + x]) > m) m = fabs(V1[3 * ids[k] + x]);
        }
        double eps = m * 0x1.8p-48; /* 48 * 2^-53 */
        q->ebox[x] = nextafter(eps + min_sep, INFINITY);
    }
    /* Split weights (reading of "split", which the paper leaves open): bounds
     * on |dF/dt|, |dF/du|, |dF/dv| in the max-norm over the axes. */
    double Lt = 0, Lu = 0, Lv = 0;
    for (int x = 0; x < 3; ++x) {
        double st = fabs(q->dc[0][x]) + fabs(q->dc[1][x]);
        st = st + fabs(q->dc[2][x]);
        if (st > Lt) Lt = st;
        double c1u = q->c0[1][x] + q->dc[1][x], c1v = q->c0[2][x] + q->dc[2][x];
        double su = fmax(fabs(q->c0[1][x]), fabs(c1u));
        double sv = fmax(fabs(q->c0[2][x]), fabs(c1v));
        if (su > Lu) Lu = su;
        if (sv > Lv) Lv = sv;
    }
    q->L[0] = Lt < 0x1p-800 ? 0.0 : Lt;
    q->L[1] = Lu < 0x1p-800 ? 0.0 : Lu;
    q->L[2] = Lv < 0x1p-800 ? 0.0 : Lv;
}

/* B_F(I): the bounding box of F at the 8 corners of I.  F is affine in each
 * of t, u, v separately, so in exact arithmetic the corner hull is the exact
 * hull of F over I; the computed corners are each within eps of the exact. */
static void inclusion_box(const query *q, const interval *I, double bmin[3], double bmax[3])
{
    double ts[2] = {dyadic(I->n[0], I->l[0]), dyadic(I->n[0] + 1, I->l[0])};
    double us[2] = {dyadic(I->n[1], I->l[1]), dyadic(I->n[1] + 1, I->l[1])};
    double vs[2] = {dyadic(I->n[2], I->l[2]), dyadic(I->n[2] + 1, I->l[2])};
    for (int x = 0; x < 3; ++x) { bmin[x] = INFINITY; bmax[x] = -INFINITY; }
    for (int it = 0; it < 2; ++it) {
        double c[3][3];
        for (int j = 0; j < 3; ++j)
            for (int x = 0; x < 3; ++x)
                c[j][x] = fma(ts[it], q->dc[j][x], q->c0[j][x]);
        for (int iu = 0; iu < 2; ++iu)
            for (int iv = 0; iv < 2; ++iv)
                for (int x = 0; x < 3; ++x) {
                    double f;
                    if (q->vf) {
                        double g = fma(-vs[iv], c[2][x], c[0][x]);
                        f = fma(-us[iu], c[1][x], g);
                    } else {
                        double g = fma(us[iu], c[1][x], c[0][x]);
                        f = fma(-vs[iv], c[2][x], g);
                    }
                    if (f < bmin[x]) bmin[x] = f;
                    if (f > bmax[x]) bmax[x] = f;
                }
    }
}

/* Split axis (reading): the axis k with the largest L_k * width_k, ties in
 * the order t, u, v; axes at LEVEL_CAP or with L_k = 0 are never split.
 * Returns -1 when no axis can be split. */
static int split_axis(const query *q, const interval *I)
{
    int best = -1;
    double bestval = -1.0;
    for (int k = 0; k < 3; ++k) {
        if (q->L[k] == 0.0 || I->l[k] >= LEVEL_CAP) continue;
        double val = ldexp(q->L[k], -I->l[k]);
        if (val > bestval) { best = k; bestval = val; }
    }
    return best;
}

#define FLAG_ITER_CAP 1u
#define FLAG_LEVEL_CAP 2u
#define STACK_MAX 200

/*
 * ProcessInterval loop of Algorithm 3 for one query, depth first: the
 * children of a split are pushed right then left, so the left (earlier) half
 * is examined first.  tstar_in is the current t* (per-query: +inf; earliest
 * mode: the running global value).  Returns the query's t* (or tstar_in if
 * nothing earlier was found).
 *
 * Steps, in order, for each interval popped:
 *   - skip if I_t^l >= t*                      (Algorithm 3, TOI test)
 *   - vertex-face: skip if u_lo + v_lo > 1     (I_uv is the simplex)
 *   - count it; past max_iter: t* = min(t*, min I_t^l over the live
 *     intervals), set FLAG_ITER_CAP and stop  (reading of the iteration cap)
 *   - B = B_F(I); skip if B misses C_eps
 *   - collision if w(B) < delta (widest axis) or B inside C_eps: t* = I_t^l
 *   - otherwise split along split_axis(); if no axis can be split, accept as
 *     a collision and set FLAG_LEVEL_CAP.
 * no_zero (appendix "Zero time of impact and minimum separation"): an
 * interval with I_t^l = 0 is always split -- neither the stop rule, nor
 * containment in C_eps, nor the iteration cap applies to it; it is accepted
 * only when no axis can be split.
 */
static double process_query(const query *q, double delta, int64_t max_iter, double tstar_in,
                            const volatile uint64_t *global_bits, int no_zero,
                            uint8_t *flags, int64_t *iters)
{
    interval stack[STACK_MAX];
    int sp = 0;
    double tstar = tstar_in;
    int64_t count = 0;
    *flags = 0;
    memset(&stack[0], 0, sizeof(interval));
    sp = 1;
    while (sp > 0) {
        interval I = stack[--sp];
        if (global_bits) { /* earliest mode: follow the shared t* */
            uint64_t bits = __atomic_load_n(global_bits, __ATOMIC_RELAXED);
            double g;
            memcpy(&g, &bits, sizeof g);
            if (g < tstar) tstar = g;
        }
        double tl = dyadic(I.n[0], I.l[0]);
        if (tl >= tstar) continue;
        /* u_lo + v_lo > 1, decided exactly: 1 - v_lo is a dyadic of at most
         * 53 bits, so it and the comparison are exact in FP64 (the sum may
         * round at the deepest levels). */
        if (q->vf && dyadic(I.n[1], I.l[1]) > 1.0 - dyadic(I.n[2], I.l[2])) continue;
        int at_zero = no_zero && I.n[0] == 0;
        if (!at_zero && ++count > max_iter) {
            double m = tl;
            for (int s = 0; s < sp; ++s) {
                double ts = dyadic(stack[s].n[0], stack[s].l[0]);
                if (ts < m) m = ts;
            }
            if (m < tstar) tstar = m;
            *flags |= FLAG_ITER_CAP;
            break;
        }
        double bmin[3], bmax[3];
        inclusion_box(q, &I, bmin, bmax);
        int miss = 0, inside = 1;
        double w = 0.0;
        for (int x = 0; x < 3; ++x) {
            if (bmin[x] > q->ebox[x] || bmax[x] < -q->ebox[x]) miss = 1;
            if (bmin[x] < -q->ebox[x] || bmax[x] > q->ebox[x]) inside = 0;
            double wx = bmax[x] - bmin[x];
            if (wx > w) w = wx;
        }
        if (miss) continue;
        if (!at_zero && (w < delta || inside)) { tstar = tl; continue; }
        int k = split_axis(q, &I);
        if (k < 0) { tstar = tl; *flags |= FLAG_LEVEL_CAP; continue; }
        interval left = I, right = I;
        left.n[k] = 2 * I.n[k];
        right.n[k] = 2 * I.n[k] + 1;
        left.l[k] = right.l[k] = I.l[k] + 1;
        stack[sp++] = right;
        stack[sp++] = left;
    }
    *iters = count;
    return tstar;
}

static uint64_t bits_of(double d) { uint64_t b; memcpy(&b, &d, sizeof b); return b; }

/*
 * Narrow phase over nq queries.  qtype[i] = 1 vertex-face, 0 edge-edge;
 * qids[4 i .. 4 i + 3] the four vertex ids (VF: P, T0, T1, T2; EE: A0, A1,
 * B0, B1).  V0, V1: (nV, 3) row-major.
 *   mode 0: every query gets its own t* (toi[i], +inf if none), flags, iters.
 *   mode 1: earliest only: one t* shared by all queries (Algorithm 3 as
 *           printed); toi/flags/iters are still written but toi[i] is only an
 *           upper bound for pruned queries.
 * no_zero: the zero-TOI rule of process_query.  Returns the earliest t* over
 * all queries in *toi_min.  nthreads <= 0 uses the OpenMP default.
 */
void oracle_narrow(int64_t nq, const uint8_t *qtype, const int64_t *qids,
                   const double *V0, const double *V1,
                   double delta, double min_sep, int64_t max_iter, int mode, int no_zero, int nthreads,
                   double *toi, uint8_t *flags, int64_t *iters, double *toi_min)
{
    volatile uint64_t gbits = bits_of(INFINITY);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nq; ++i) {
        query q;
        setup_query(&q, qtype[i], V0, V1, &qids[4 * i], min_sep);
        double start = INFINITY;
        double t = process_query(&q, delta, max_iter, start, mode == 1 ? &gbits : NULL, no_zero,
                                 &flags[i], &iters[i]);
        toi[i] = t;
        if (t < INFINITY) { /* min into the shared value */
            uint64_t want = bits_of(t), cur = __atomic_load_n(&gbits, __ATOMIC_RELAXED);
            while (want < cur &&
                   !__atomic_compare_exchange_n(&gbits, &cur, want, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {
            }
        }
    }
    double g;
    uint64_t b = gbits;
    memcpy(&g, &b, sizeof g);
    *toi_min = g;
}

/* The inclusion box of one query over one interval, for the tests that check
 * the error bound against exact arithmetic: bmin/bmax = B_F(I) (corner hull of
 * the computed F), ebox = the per-axis half-width of C_eps enlarged by
 * min_sep.  n[k], l[k]: interval [n/2^l, (n+1)/2^l] on t, u, v. */
void oracle_inclusion(int vf, const int64_t ids[4], const double *V0, const double *V1,
                      double min_sep, const uint64_t n[3], const int32_t l[3],
                      double bmin[3], double bmax[3], double ebox[3])
{
    query q;
    interval I;
    setup_query(&q, vf, V0, V1, ids, min_sep);
    for (int k = 0; k < 3; ++k) { I.n[k] = n[k]; I.l[k] = l[k]; }
    inclusion_box(&q, &I, bmin, bmax);
    for (int x = 0; x < 3; ++x) ebox[x] = q.ebox[x];
}

/* The split weights L_t, L_u, L_v of one query (the reading of "split" that
 * the paper leaves open), so that the tests can check them against values
 * worked out by hand. */
void oracle_split_weights(int vf, const int64_t ids[4], const double *V0, const double *V1,
                          double L[3])
{
    query q;
    setup_query(&q, vf, V0, V1, ids, 0.0);
    for (int k = 0; k < 3; ++k) L[k] = q.L[k];
}

int oracle_has_openmp(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 0;
#endif
}
