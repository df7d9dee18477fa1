/*
 * lvb_oracle.c -- CPU oracle for the local Verlet buffer broad phase.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * It is deliberately plain and slow: every function is the definition it
 * cites, written out, with no blocking, fusion or reordering.
 *
 * Precision.  The broad-phase decisions (flags, pair set, contact set) are
 * defined on a fixed binary32 formula so that a GPU and a CPU evaluating the
 * same formula on the same inputs agree bit for bit: every + and * below
 * rounds to nearest-even in binary32.  This file MUST be compiled with
 * -ffp-contract=off and without -ffast-math (the build script does so); no
 * sqrt enters any comparison except the narrow-phase overlap, which uses the
 * correctly rounded sqrtf.  The DEM dynamics oracle is binary64.
 *
 * Formula (shared definition, written independently on each side):
 *   d      = a - b                      per component, binary32
 *   |d|^2  = ((dx*dx + dy*dy) + dz*dz)   each product and sum rounded
 *   flag   : |x - xref|^2 > skin*skin                      (Eq. update)
 *   R_NL   = r + skin                                      (Eq. bounding_sphere)
 *   pair   : |xref_i - xref_j|^2 <= (R_NL,i + R_NL,j)^2    (Def. verletlist,
 *                                                           Eq. broad_phase)
 *   delta  = (r_i + r_j) - sqrtf(|x_i - x_j|^2), contact iff delta > 0
 *                                                          (Eq. delta)
 *
 * Parity status per function is given in its comment; every function here is
 * pinned by a CPU test (closed forms, brute force, invariants), except
 * where a comment says "parity unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* Threads.  When built with OpenMP the flag test and the linked-cell   */
/* pair search split their loops over particles / cells across host    */
/* threads; every result is the same set in the same (sorted) order     */
/* whatever the thread count, since each decision is the fixed formula  */
/* on one particle or one pair.                                         */
/* ------------------------------------------------------------------ */
ORC_API void orc_set_threads(int t)
{
#ifdef _OPENMP
    omp_set_num_threads(t > 0 ? t : omp_get_num_procs());
#else
    (void)t;
#endif
}

ORC_API int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int thread_id(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

/* ------------------------------------------------------------------ */
/* binary32 building blocks                                            */
/* ------------------------------------------------------------------ */

/* Squared distance in the fixed association ((dx^2 + dy^2) + dz^2). */
static float sqdist_f32(const float *a, const float *b)
{
    float dx = a[0] - b[0];
    float dy = a[1] - b[1];
    float dz = a[2] - b[2];
    float xx = dx * dx;
    float yy = dy * dy;
    float zz = dz * dz;
    float s = xx + yy;
    s = s + zz;
    return s;
}

/* ------------------------------------------------------------------ */
/* Eq. update (Sec. "Automatic update and validity of the Verlet list"): */
/* particle p violates the validity condition when its linear          */
/* displacement since its last broad phase exceeds its skin.  The       */
/* displacement is the straight-line distance (Related work, where the  */
/* paper contrasts it with the accumulated path length).  Strict ">":  */
/* equality keeps the list (Eq. update uses <= for validity).          */
/* Pinned by: ballistic closed form, equality case, K = 0 case.        */
/* ------------------------------------------------------------------ */
ORC_API int64_t orc_flags(int64_t n, const float *pos4, const float *ref4,
                          uint8_t *flag)
{
    int64_t nf = 0;
#pragma omp parallel for reduction(+ : nf) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        float d2 = sqdist_f32(pos4 + 4 * i, ref4 + 4 * i);
        float s = ref4[4 * i + 3];
        float s2 = s * s;
        flag[i] = (uint8_t)(d2 > s2);
        nf += flag[i];
    }
    return nf;
}

/* The early trigger's set (an option of the partial trigger; the paper  */
/* has the per-particle violation of Eq. update and the global rebuild   */
/* of Def. autoverlet): the particles whose displacement exceeds beta    */
/* times their skin, |x - xref|^2 > t * t with t = beta * skin, every     */
/* product rounded to binary32 (beta itself a binary32 value).  Strict   */
/* ">" as in Eq. update.                                                 */
/* Pinned by: hand cases at and around the boundary (tests).             */
ORC_API int64_t orc_flags_beta(int64_t n, const float *pos4, const float *ref4, float beta,
                               uint8_t *flag)
{
    int64_t nf = 0;
    for (int64_t i = 0; i < n; ++i) {
        float d2 = sqdist_f32(pos4 + 4 * i, ref4 + 4 * i);
        float t = beta * ref4[4 * i + 3];
        float t2 = t * t;
        flag[i] = (uint8_t)(d2 > t2);
        nf += flag[i];
    }
    return nf;
}

/* ------------------------------------------------------------------ */
/* Skin policies.                                                       */
/*   kind 0  global skin s_g (the paper's constant-skin comparator,     */
/*           Sec. Results: skin equal to the particle radius)           */
/*   kind 1  diameter factor: skin = alpha * (2 r)                      */
/*   kind 2  the paper's rule skin_p = K * |v_p| * dt (Eq.              */
/*           skin_formulus1), evaluated as (K * |v|) * dt with |v| the  */
/*           correctly rounded sqrtf of ((vx^2 + vy^2) + vz^2)          */
/*   kind 3  an externally proposed skin (the learned network's output, */
/*           computed by the network oracle), taken as given            */
/* then the cap of Eq. skin_formulus_mincell, read as R_NL <= H with    */
/* H just under half a cell edge (so that every pair within             */
/* R_NL,i + R_NL,j is in adjacent cells):                               */
/*   skin = min(skin, max(0, H - r))                                    */
/* Pinned by: closed forms per kind and the cap boundary.               */
/* ------------------------------------------------------------------ */
static float skin_policy_one(int kind, float value, float dt, float H,
                             const float *p4, const float *v4, float proposal)
{
    float r = p4[3];
    float s;
    if (kind == 0) {
        s = value;
    } else if (kind == 1) {
        float d = 2.0f * r;
        s = value * d;
    } else if (kind == 2) {
        float vx = v4[0] * v4[0];
        float vy = v4[1] * v4[1];
        float vz = v4[2] * v4[2];
        float v2 = vx + vy;
        v2 = v2 + vz;
        float vm = sqrtf(v2);
        float kv = value * vm;
        s = kv * dt;
    } else {
        s = proposal;
    }
    float capv = H - r;
    if (!(capv > 0.0f)) capv = 0.0f;
    if (!(s >= 0.0f)) s = 0.0f;        /* negative or NaN proposals -> 0 */
    if (s > capv) s = capv;
    return s;
}

ORC_API void orc_skin(int64_t n, int kind, float value, float dt, float H,
                      const float *pos4, const float *vel4,
                      const float *proposal, float *skin_out)
{
    for (int64_t i = 0; i < n; ++i) {
        const float *v = vel4 ? vel4 + 4 * i : NULL;
        float prop = proposal ? proposal[i] : 0.0f;
        skin_out[i] = skin_policy_one(kind, value, dt, H, pos4 + 4 * i, v, prop);
    }
}

/* ------------------------------------------------------------------ */
/* Pair set by its definition (Def. verletlist; Eq. broad_phase; the    */
/* extended range R_NL = R_C + skin of Eq. bounding_sphere):            */
/*   P = { (i,j), i < j : |xref_i - xref_j|^2 <= (R_NL,i + R_NL,j)^2 }  */
/* evaluated on the reference positions.  Brute force over all pairs,   */
/* emitted in (i, j) lexicographic order.                               */
/* ref4 = (xref, yref, zref, skin), rad = radius.                       */
/* Returns the number of pairs; writes at most cap of them.             */
/* Pinned by: exact-cutoff and two-particle closed forms.               */
/* ------------------------------------------------------------------ */
static int pair_test(const float *ri4, float rad_i, const float *rj4, float rad_j)
{
    float rnl_i = rad_i + ri4[3];
    float rnl_j = rad_j + rj4[3];
    float c = rnl_i + rnl_j;
    float c2 = c * c;
    float d2 = sqdist_f32(ri4, rj4);
    return d2 <= c2;
}

ORC_API int64_t orc_pairs_brute(int64_t n, const float *ref4, const float *rad,
                                int32_t *pi, int32_t *pj, int64_t cap)
{
    int64_t np = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            if (pair_test(ref4 + 4 * i, rad[i], ref4 + 4 * j, rad[j])) {
                if (np < cap) { pi[np] = (int32_t)i; pj[np] = (int32_t)j; }
                ++np;
            }
        }
    }
    return np;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 (linked-cell algorithm, Sec. "Collision detection in     */
/* XDEM"): uniform cells no smaller than the largest bounding sphere;   */
/* every pair of neighbouring cells is visited once (the lower cell     */
/* index is the neighbour), and a pair is emitted when the bounding     */
/* spheres -- here the extended spheres of radius R_NL -- intersect.    */
/* The algorithm as printed skips same-cell pairs (it only visits       */
/* index(C_b) < index(C_a)); the pair set is defined by the distance    */
/* test, so pairs inside one cell (lower particle index first) are      */
/* visited too.                                                         */
/* The cell edge is the oracle's own: the largest 2 R_NL times          */
/* (1 + 2^-8), on a grid spanning the bounding box of the reference     */
/* positions.  The result is sorted into (i, j) order.                  */
/* Pinned by: equality with orc_pairs_brute on random polydisperse sets. */
/* ------------------------------------------------------------------ */
typedef struct { int32_t i, j; } ipair;

/* Cell grid over a set of points; counting sort of particle ids by cell. */
typedef struct {
    double lo[3];
    double edge;
    int64_t dim[3];
    int64_t ncell;
    int64_t *start;   /* ncell + 1 */
    int32_t *ids;     /* n */
} cellgrid;

static int64_t cell_coord(double x, double lo, double edge, int64_t dim)
{
    int64_t c = (int64_t)floor((x - lo) / edge);
    if (c < 0) c = 0;
    if (c >= dim) c = dim - 1;
    return c;
}

static int grid_build(cellgrid *g, int64_t n, const float *p4, double edge)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY};
    double hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            double x = p4[4 * i + k];
            if (x < lo[k]) lo[k] = x;
            if (x > hi[k]) hi[k] = x;
        }
    if (n == 0) { for (int k = 0; k < 3; ++k) { lo[k] = 0; hi[k] = 0; } }
    g->edge = edge;
    g->ncell = 1;
    for (int k = 0; k < 3; ++k) {
        g->lo[k] = lo[k];
        int64_t d = (int64_t)floor((hi[k] - lo[k]) / edge) + 1;
        if (d < 1) d = 1;
        g->dim[k] = d;
        g->ncell *= d;
    }
    g->start = (int64_t *)calloc((size_t)g->ncell + 1, sizeof(int64_t));
    g->ids = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int64_t *key = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!g->start || !g->ids || !key) { free(key); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        for (int k = 0; k < 3; ++k)
            c[k] = cell_coord(p4[4 * i + k], g->lo[k], edge, g->dim[k]);
        key[i] = (c[2] * g->dim[1] + c[1]) * g->dim[0] + c[0];
        g->start[key[i] + 1]++;
    }
    for (int64_t c = 0; c < g->ncell; ++c) g->start[c + 1] += g->start[c];
    int64_t *fill = (int64_t *)malloc((size_t)g->ncell * sizeof(int64_t));
    if (!fill) { free(key); return -1; }
    memcpy(fill, g->start, (size_t)g->ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) g->ids[fill[key[i]]++] = (int32_t)i;
    free(fill);
    free(key);
    return 0;
}

static void grid_free(cellgrid *g)
{
    free(g->start);
    free(g->ids);
}

/* Visit the 27-cell neighbourhood of every cell and call emit() on each
 * unordered particle pair exactly once (Algorithm 1 with same-cell pairs). */
typedef struct {
    ipair *buf;
    int64_t n, cap;
    int oom;
} pairbuf;

static void pb_push(pairbuf *pb, int32_t a, int32_t b)
{
    if (pb->n == pb->cap) {
        int64_t nc = pb->cap ? 2 * pb->cap : 1024;
        ipair *nb = (ipair *)realloc(pb->buf, (size_t)nc * sizeof(ipair));
        if (!nb) { pb->oom = 1; return; }
        pb->buf = nb;
        pb->cap = nc;
    }
    pb->buf[pb->n].i = a < b ? a : b;
    pb->buf[pb->n].j = a < b ? b : a;
    pb->n++;
}

ORC_API int64_t orc_pairs_cells(int64_t n, const float *ref4, const float *rad,
                                int32_t *pi, int32_t *pj, int64_t cap)
{
    double rmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double rnl = (double)rad[i] + (double)ref4[4 * i + 3];
        if (rnl > rmax) rmax = rnl;
    }
    double edge = 2.0 * rmax * (1.0 + 1.0 / 256.0);
    if (!(edge > 0.0)) edge = 1.0;
    cellgrid g;
    if (grid_build(&g, n, ref4, edge) != 0) { grid_free(&g); return -1; }
    /* one pair buffer per host thread; the cells are split among them */
    int nt = orc_threads();
    pairbuf *pbs = (pairbuf *)calloc((size_t)nt, sizeof(pairbuf));
    if (!pbs) { grid_free(&g); return -1; }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t ca = 0; ca < g.ncell; ++ca) {
        pairbuf *pb = &pbs[thread_id()];
        int64_t ax = ca % g.dim[0];
        int64_t ay = (ca / g.dim[0]) % g.dim[1];
        int64_t az = ca / (g.dim[0] * g.dim[1]);
        for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            int64_t bx = ax + dx, by = ay + dy, bz = az + dz;
            if (bx < 0 || by < 0 || bz < 0) continue;
            if (bx >= g.dim[0] || by >= g.dim[1] || bz >= g.dim[2]) continue;
            int64_t cb = (bz * g.dim[1] + by) * g.dim[0] + bx;
            if (cb > ca) continue;                 /* each cell pair once */
            for (int64_t s = g.start[ca]; s < g.start[ca + 1]; ++s) {
                int32_t a = g.ids[s];
                for (int64_t t = g.start[cb]; t < g.start[cb + 1]; ++t) {
                    int32_t b = g.ids[t];
                    if (cb == ca && b >= a) continue;   /* same cell: once */
                    if (pair_test(ref4 + 4 * (int64_t)a, rad[a],
                                  ref4 + 4 * (int64_t)b, rad[b]))
                        pb_push(pb, a, b);
                }
            }
        }
    }
    grid_free(&g);
    int64_t np = 0;
    int oom = 0;
    for (int t = 0; t < nt; ++t) { np += pbs[t].n; oom |= pbs[t].oom; }
    int64_t *start = oom ? NULL : (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *col = oom ? NULL : (int32_t *)malloc((size_t)(np > 0 ? np : 1) * sizeof(int32_t));
    if (oom || !start || !col) {
        for (int t = 0; t < nt; ++t) free(pbs[t].buf);
        free(pbs); free(start); free(col);
        return -1;
    }
    /* (i, j) order: bucket the pairs by i (counting sort), then sort each
     * bucket's j ascending */
    for (int t = 0; t < nt; ++t)
        for (int64_t k = 0; k < pbs[t].n; ++k) start[pbs[t].buf[k].i + 1]++;
    for (int64_t i = 0; i < n; ++i) start[i + 1] += start[i];
    for (int t = 0; t < nt; ++t) {
        for (int64_t k = 0; k < pbs[t].n; ++k) col[start[pbs[t].buf[k].i]++] = pbs[t].buf[k].j;
        free(pbs[t].buf);
    }
    free(pbs);
    for (int64_t i = n; i > 0; --i) start[i] = start[i - 1];   /* back to bucket starts */
    start[0] = 0;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t a = start[i] + 1; a < start[i + 1]; ++a) {   /* insertion sort */
            int32_t v = col[a];
            int64_t b = a;
            for (; b > start[i] && col[b - 1] > v; --b) col[b] = col[b - 1];
            col[b] = v;
        }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = start[i]; k < start[i + 1] && k < cap; ++k) {
            pi[k] = (int32_t)i;
            pj[k] = col[k];
        }
    free(start);
    free(col);
    return np;
}

/* ------------------------------------------------------------------ */
/* Narrow phase on a pair list, Eq. delta:                              */
/*   delta = (r_i + r_j) - ||X_i - X_j||, contact iff delta > 0         */
/* on the CURRENT positions (pos4 = x, y, z, r).  ||.|| is the          */
/* correctly rounded sqrtf of the fixed-association squared distance.   */
/* Pinned by: two-sphere closed forms and the touching (delta = 0) case. */
/* ------------------------------------------------------------------ */
static float overlap_f32(const float *a4, const float *b4)
{
    float R = a4[3] + b4[3];
    float d2 = sqdist_f32(a4, b4);
    float s = sqrtf(d2);
    return R - s;
}

ORC_API int64_t orc_contacts(int64_t npairs, const int32_t *pi, const int32_t *pj,
                             const float *pos4, int32_t *ci, int32_t *cj,
                             float *delta, int64_t cap)
{
    int64_t nc = 0;
    for (int64_t k = 0; k < npairs; ++k) {
        float dl = overlap_f32(pos4 + 4 * (int64_t)pi[k], pos4 + 4 * (int64_t)pj[k]);
        if (dl > 0.0f) {
            if (nc < cap) { ci[nc] = pi[k]; cj[nc] = pj[k]; delta[nc] = dl; }
            ++nc;
        }
    }
    return nc;
}

/* All overlapping pairs of a configuration, independent of any list:    */
/* brute force over every i < j (Eq. delta).  Used for the zero-missed- */
/* contact invariant of Theorem 1 on small inputs.                       */
ORC_API int64_t orc_contacts_brute(int64_t n, const float *pos4, int32_t *ci,
                                   int32_t *cj, float *delta, int64_t cap)
{
    int64_t nc = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            float dl = overlap_f32(pos4 + 4 * i, pos4 + 4 * j);
            if (dl > 0.0f) {
                if (nc < cap) { ci[nc] = (int32_t)i; cj[nc] = (int32_t)j; delta[nc] = dl; }
                ++nc;
            }
        }
    return nc;
}

/* Same set through a cell search on the current positions with skin 0   */
/* (cells of edge 2 r_max); for configurations too large for brute force. */
/* Pinned by: equality with orc_contacts_brute.                          */
ORC_API int64_t orc_contacts_cells(int64_t n, const float *pos4, int32_t *ci,
                                   int32_t *cj, float *delta, int64_t cap)
{
    float *ref0 = (float *)malloc((size_t)(n > 0 ? n : 1) * 4 * sizeof(float));
    float *rad = (float *)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
    if (!ref0 || !rad) { free(ref0); free(rad); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        ref0[4 * i + 0] = pos4[4 * i + 0];
        ref0[4 * i + 1] = pos4[4 * i + 1];
        ref0[4 * i + 2] = pos4[4 * i + 2];
        ref0[4 * i + 3] = 0.0f;
        rad[i] = pos4[4 * i + 3];
    }
    /* Candidate pairs at cutoff r_i + r_j (a superset of the overlaps up to
     * rounding of the squared cutoff), then the exact overlap test. */
    int64_t np = orc_pairs_cells(n, ref0, rad, NULL, NULL, 0);
    if (np < 0) { free(ref0); free(rad); return -1; }
    int32_t *pi = (int32_t *)malloc((size_t)(np > 0 ? np : 1) * sizeof(int32_t));
    int32_t *pj = (int32_t *)malloc((size_t)(np > 0 ? np : 1) * sizeof(int32_t));
    if (!pi || !pj) { free(pi); free(pj); free(ref0); free(rad); return -1; }
    orc_pairs_cells(n, ref0, rad, pi, pj, np);
    int64_t nc = orc_contacts(np, pi, pj, pos4, ci, cj, delta, cap);
    free(pi); free(pj); free(ref0); free(rad);
    return nc;
}

/* ------------------------------------------------------------------ */
/* DEM dynamics oracle, binary64.                                       */
/*                                                                      */
/* The paper's runs use velocity Verlet and a linear spring-dashpot     */
/* (Sec. Methodology); the contact law below is the normal-only linear  */
/* spring-dashpot without friction:                                     */
/*   F_i = (k_n delta - gamma_n v_n) n,   n = (x_i - x_j)/|x_i - x_j|    */
/*   v_n = (v_i - v_j) . n,  gamma_n = 2 zeta sqrt(m_eff k_n),          */
/*   zeta = -ln e / sqrt(pi^2 + ln^2 e),  m_eff = m_i m_j / (m_i + m_j)  */
/* with walls treated as bodies of infinite mass (m_eff = m_i).  The    */
/* velocity used for damping at the new positions is the predicted      */
/* v* = v + a dt.  No tensile clamp unless clamp_tensile != 0.          */
/* Inputs are the single-precision state of the code under test,        */
/* widened exactly to binary64.                                         */
/* Pinned by: free fall (exact for velocity Verlet), head-on            */
/* restitution and contact duration, energy with e = 1.                 */
/* ------------------------------------------------------------------ */

typedef struct {
    double kn;            /* spring stiffness [N/m] */
    double restitution;   /* e in (0, 1] */
    double rho;           /* density [kg/m^3] */
    double g[3];          /* gravity [m/s^2] */
    double lo[3], hi[3];  /* box walls (wall_kind 1) / end caps (kind 2) */
    int32_t wall_kind;    /* 0 none, 1 box, 2 drum (axis y) + caps, 3 specular box */
    int32_t clamp_tensile;
    double drum_center[2];/* (x, z) of the drum axis */
    double drum_radius;
    double drum_omega;    /* rad/s about +y; normal-only law ignores it */
    int32_t contacts_on;  /* 0: no particle contacts (ballistic) */
    int32_t pad;
} orc_dem_params;

static double mass_of(double r, double rho)
{
    return rho * (4.0 / 3.0) * M_PI * r * r * r;
}

static double zeta_of(double e)
{
    double le = log(e);
    return -le / sqrt(M_PI * M_PI + le * le);
}

/* Force on particle i from one contact of overlap dl along unit normal
 * nrm (pointing into i), relative normal velocity vn, effective mass m. */
static double lsd_force(const orc_dem_params *P, double dl, double vn, double meff)
{
    double gam = 2.0 * zeta_of(P->restitution) * sqrt(meff * P->kn);
    double f = P->kn * dl - gam * vn;
    if (P->clamp_tensile && f < 0.0) f = 0.0;
    return f;
}

/* Candidate pairs for the binary64 contact search: the binary32 pair search
 * at cutoff (r_i + r_j)(1 + 2^-20) on the positions rounded to binary32
 * (brute force when n <= 4096, the oracle's linked cells otherwise), far
 * above the binary32 rounding of any position.  *ci / *cj are malloc'd;
 * returns the count or -1. */
static int64_t contact_candidates(int64_t n, const double *x, const double *r, int32_t **ci_out,
                                  int32_t **cj_out)
{
    *ci_out = NULL;
    *cj_out = NULL;
    float *ref = (float *)malloc((size_t)(n > 0 ? n : 1) * 4 * sizeof(float));
    float *rad = (float *)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
    if (!ref || !rad) { free(ref); free(rad); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        ref[4 * i + 0] = (float)x[3 * i + 0];
        ref[4 * i + 1] = (float)x[3 * i + 1];
        ref[4 * i + 2] = (float)x[3 * i + 2];
        ref[4 * i + 3] = (float)(r[i] * (1.0 / 1048576.0));
        rad[i] = (float)r[i];
    }
    int64_t cap = 16 * n + 1024;
    int32_t *ci = NULL, *cj = NULL;
    int64_t np;
    for (;;) {
        ci = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
        cj = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
        if (!ci || !cj) { free(ci); free(cj); free(ref); free(rad); return -1; }
        np = (n <= 4096) ? orc_pairs_brute(n, ref, rad, ci, cj, cap)
                         : orc_pairs_cells(n, ref, rad, ci, cj, cap);
        if (np <= cap) break;
        cap = np;
        free(ci); free(cj);
    }
    free(ref); free(rad);
    if (np < 0) { free(ci); free(cj); return -1; }
    *ci_out = ci;
    *cj_out = cj;
    return np;
}

/* Every contact i < j (delta > 0 in binary64) of a configuration, sorted by
 * (i, j), with the force on i, f n (f = k_n delta - gamma_n v_n, n from j to
 * i, the law of orc_dem_forces64 below), the overlap, and the scale of the
 * terms of f, |k_n delta| + |gamma_n v_n|.  x, v: 3n; r: n.  Writes at
 * most cap contacts; returns their number or -1.
 * Pinned by: the head-on pair in closed form (tests). */
ORC_API int64_t orc_dem_contacts64(int64_t n, const double *x, const double *r, const double *v,
                                   const orc_dem_params *P, int32_t *oi, int32_t *oj,
                                   double *f3, double *delta, double *scale, int64_t cap)
{
    int32_t *ci, *cj;
    int64_t np = contact_candidates(n, x, r, &ci, &cj);
    if (np < 0) return -1;
    int64_t m = 0;
    for (int64_t k = 0; k < np; ++k) {
        int64_t i = ci[k], j = cj[k];
        double d[3], dist2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            d[c] = x[3 * i + c] - x[3 * j + c];
            dist2 += d[c] * d[c];
        }
        double dist = sqrt(dist2);
        double dl = (r[i] + r[j]) - dist;
        if (!(dl > 0.0) || !(dist > 0.0)) continue;
        double nrm[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
        double vn = 0.0;
        for (int c = 0; c < 3; ++c) vn += (v[3 * i + c] - v[3 * j + c]) * nrm[c];
        double mi = mass_of(r[i], P->rho), mj = mass_of(r[j], P->rho);
        double f = lsd_force(P, dl, vn, mi * mj / (mi + mj));
        if (m < cap) {
            oi[m] = (int32_t)i;
            oj[m] = (int32_t)j;
            for (int c = 0; c < 3; ++c) f3[3 * m + c] = f * nrm[c];
            delta[m] = dl;
            scale[m] = fabs(P->kn * dl) + fabs(f - P->kn * dl);
        }
        ++m;
    }
    free(ci); free(cj);
    return m;
}

/* Net force on every particle (binary64).  x: 3n positions, r: n radii,
 * v: 3n damping velocities.  Candidate pairs come from the binary32 pair
 * search at cutoff (r_i + r_j)(1 + 2^-20) on the positions rounded to
 * binary32 (brute force when n <= 4096, the oracle's linked cells
 * otherwise); the binary64 overlap then decides.  The 2^-20 inflation is
 * far above the binary32 rounding of any position.
 * force: 3n doubles (contact + wall forces, no gravity). */
ORC_API int orc_dem_forces64(int64_t n, const double *x, const double *r, const double *v,
                             const orc_dem_params *P, double *force, double *fmag)
{
    memset(force, 0, (size_t)n * 3 * sizeof(double));
    if (fmag) memset(fmag, 0, (size_t)n * sizeof(double));
    if (P->contacts_on && n > 1) {
        int32_t *ci, *cj;
        int64_t np = contact_candidates(n, x, r, &ci, &cj);
        if (np < 0) return -1;
        for (int64_t k = 0; k < np; ++k) {
            int64_t i = ci[k], j = cj[k];
            double d[3], dist2 = 0.0;
            for (int c = 0; c < 3; ++c) {
                d[c] = x[3 * i + c] - x[3 * j + c];
                dist2 += d[c] * d[c];
            }
            double dist = sqrt(dist2);
            double dl = (r[i] + r[j]) - dist;
            if (!(dl > 0.0) || !(dist > 0.0)) continue;
            double nrm[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
            double vn = 0.0;
            for (int c = 0; c < 3; ++c) vn += (v[3 * i + c] - v[3 * j + c]) * nrm[c];
            double mi = mass_of(r[i], P->rho), mj = mass_of(r[j], P->rho);
            double f = lsd_force(P, dl, vn, mi * mj / (mi + mj));
            for (int c = 0; c < 3; ++c) {
                force[3 * i + c] += f * nrm[c];
                force[3 * j + c] -= f * nrm[c];
            }
            if (fmag) {   /* scale of the terms summed into F_i, F_j */
                double sc = fabs(P->kn * dl) + fabs(f - P->kn * dl);
                fmag[i] += sc;
                fmag[j] += sc;
            }
        }
        free(ci); free(cj);
    }
    if (P->wall_kind == 1 || P->wall_kind == 2) {
        for (int64_t i = 0; i < n; ++i) {
            double ri = r[i];
            double m = mass_of(ri, P->rho);
            int first_axis = (P->wall_kind == 2) ? 1 : 0;
            int last_axis = (P->wall_kind == 2) ? 1 : 2;
            for (int c = first_axis; c <= last_axis; ++c) {
                double xc = x[3 * i + c];
                double vc = v[3 * i + c];
                double dlo = ri - (xc - P->lo[c]);     /* lower plane, normal +e_c */
                if (dlo > 0.0) {
                    double f = lsd_force(P, dlo, vc, m);
                    force[3 * i + c] += f;
                    if (fmag) fmag[i] += fabs(P->kn * dlo) + fabs(f - P->kn * dlo);
                }
                double dhi = ri - (P->hi[c] - xc);     /* upper plane, normal -e_c */
                if (dhi > 0.0) {
                    double f = lsd_force(P, dhi, -vc, m);
                    force[3 * i + c] -= f;
                    if (fmag) fmag[i] += fabs(P->kn * dhi) + fabs(f - P->kn * dhi);
                }
            }
            if (P->wall_kind == 2) {
                double ex = x[3 * i + 0] - P->drum_center[0];
                double ez = x[3 * i + 2] - P->drum_center[1];
                double rho_i = sqrt(ex * ex + ez * ez);
                double dl = ri + rho_i - P->drum_radius;
                if (dl > 0.0 && rho_i > 0.0) {
                    double nx = -ex / rho_i, nz = -ez / rho_i;   /* inward */
                    /* the wall moves tangentially: no normal component */
                    double vn = v[3 * i + 0] * nx + v[3 * i + 2] * nz;
                    double f = lsd_force(P, dl, vn, m);
                    force[3 * i + 0] += f * nx;
                    force[3 * i + 2] += f * nz;
                    if (fmag) fmag[i] += fabs(P->kn * dl) + fabs(f - P->kn * dl);
                }
            }
        }
    }
    return 0;
}

/* Binary32 records (x, y, z, r) and (vx, vy, vz, -) widened exactly. */
ORC_API int orc_dem_forces(int64_t n, const float *x4, const float *v4,
                           const orc_dem_params *P, double *force)
{
    double *x = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    double *v = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    double *r = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!x || !v || !r) { free(x); free(v); free(r); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < 3; ++c) {
            x[3 * i + c] = x4[4 * i + c];
            v[3 * i + c] = v4[4 * i + c];
        }
        r[i] = x4[4 * i + 3];
    }
    int rc = orc_dem_forces64(n, x, r, v, P, force, NULL);
    free(x); free(v); free(r);
    return rc;
}

/* One velocity-Verlet step in binary64 (Sec. Methodology names velocity
 * Verlet; the damping velocity at the new positions is the predicted
 * v* = v + a dt):
 *   x' = x + v dt + a dt^2 / 2,   v* = v + a dt,
 *   a' = F(x', v*)/m + g,         v' = v + (a + a') dt / 2.
 * With wall_kind 3 (specular box, meant for runs without contacts or
 * gravity) a coordinate that left [lo + r, hi - r] is mirrored back and its
 * velocity components v' and v* are negated (v* is the velocity the
 * particle has at its new, mirrored position).
 * xf / vf, when given (3n each), replace x' and v* as the state at which
 * forces are evaluated (the oracle "fed" the state of the code under test,
 * so that trajectories cannot drift apart).
 * fmag (n, optional): per particle, the sum over its contacts of
 * |k_n delta| + |damping term| -- the scale of the terms summed into F,
 * against which a binary32 evaluation's rounding is measured.
 * All arrays are binary64, 3n (r, fmag: n). */
static void half_step(int64_t n, const double *x, const double *v, const double *a, double dt,
                      double *x_out, double *vstar_out)
{
    for (int64_t k = 0; k < 3 * n; ++k) {
        x_out[k] = x[k] + v[k] * dt + 0.5 * a[k] * dt * dt;
        vstar_out[k] = v[k] + a[k] * dt;
    }
}

ORC_API int orc_dem_step64(int64_t n, const double *x, const double *v, const double *a,
                           const double *r, double dt, const orc_dem_params *P,
                           const double *xf, const double *vf,
                           double *x_out, double *vstar_out, double *a_out, double *v_out,
                           double *fmag)
{
    half_step(n, x, v, a, dt, x_out, vstar_out);
    double *F = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    if (!F) return -1;
    int rc = orc_dem_forces64(n, xf ? xf : x_out, r, vf ? vf : vstar_out, P, F, fmag);
    if (rc != 0) { free(F); return rc; }
    for (int64_t i = 0; i < n; ++i) {
        double m = mass_of(r[i], P->rho);
        for (int c = 0; c < 3; ++c) {
            double an = F[3 * i + c] / m + P->g[c];
            a_out[3 * i + c] = an;
            v_out[3 * i + c] = v[3 * i + c] + 0.5 * (a[3 * i + c] + an) * dt;
        }
    }
    if (P->wall_kind == 3) {
        for (int64_t i = 0; i < n; ++i) {
            for (int c = 0; c < 3; ++c) {
                double lo = P->lo[c] + r[i], hi = P->hi[c] - r[i];
                double xc = x_out[3 * i + c];
                if (xc < lo || xc > hi) {
                    x_out[3 * i + c] = 2.0 * (xc < lo ? lo : hi) - xc;
                    v_out[3 * i + c] = -v_out[3 * i + c];
                    vstar_out[3 * i + c] = -vstar_out[3 * i + c];
                }
            }
        }
    }
    free(F);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Friction with contact history, binary64 (the LSD model with static    */
/* friction named in Sec. Methodology; the paper gives no formula, so    */
/* this is the common linear tangential spring with a Coulomb cap):      */
/*   per particle also w (angular velocity) and al = T / I, I = 2/5 m r^2 */
/*   w* = w + al dt,  w' = w + (al + al') dt / 2  (velocity Verlet)       */
/* per contact i < j (delta > 0), n from j to i:                          */
/*   v_rel = (v*_i - v*_j) - (r_i w*_i + r_j w*_j) x n                   */
/*   v_t   = v_rel - (v_rel . n) n                                       */
/*   xi    = xi_prev - (xi_prev . n) n + v_t dt   (xi_prev = 0 for a     */
/*           pair that was not in contact at the previous step)           */
/*   F_t   = -k_t xi - gamma_t v_t,  k_t = kt_ratio k_n,                  */
/*           gamma_t = gt_ratio gamma_n(m_eff)                            */
/*   if |F_t| > mu max(F_n, 0): F_t *= mu max(F_n, 0) / |F_t| and         */
/*           xi = -(F_t + gamma_t v_t) / k_t                              */
/*   force on i F_n n + F_t (on j its negation); torque on i -r_i n x F_t, */
/*   on j -r_j n x F_t                                                    */
/* Walls: the normal law only.                                            */
/* History in: nh pairs (hi < hj, sorted by (i, j)) with xi (3 each, from */
/* i's side).  Out: every contact of the new state, sorted, with its xi,  */
/* the force on i and the scale of its terms |k_n delta| + |gamma_n v_n|  */
/* + |k_t xi| + |gamma_t v_t|; per particle the sums of those scales      */
/* (fmag) and of r times the tangential ones (tmag).  xf, vf, wf, when    */
/* given, replace x', v*, w* as the state of the force evaluation.        */
/* Returns the number of contacts (at most cap written) or -1.            */
/* Pinned by: a sphere sliding on a fixed one (Coulomb limit), a sticking */
/* pair's spring growing by v_t dt per step, the antisymmetry of forces   */
/* and the conservation of linear momentum (tests).                       */
/* ------------------------------------------------------------------ */
static int64_t find_pair(int64_t nh, const int32_t *hi, const int32_t *hj, int32_t i, int32_t j)
{
    int64_t lo = 0, up = nh;
    while (lo < up) {
        int64_t mid = lo + (up - lo) / 2;
        if (hi[mid] < i || (hi[mid] == i && hj[mid] < j)) lo = mid + 1;
        else up = mid;
    }
    return (lo < nh && hi[lo] == i && hj[lo] == j) ? lo : -1;
}

ORC_API int64_t orc_dem_step64f(int64_t n, const double *x, const double *v, const double *a,
                                const double *w, const double *al, const double *r, double dt,
                                const orc_dem_params *P, double mu, double kt_ratio,
                                double gt_ratio, const double *xf, const double *vf,
                                const double *wf, int64_t nh, const int32_t *hi,
                                const int32_t *hj, const double *hxi, double *x_out,
                                double *vstar_out, double *a_out, double *v_out,
                                double *wstar_out, double *al_out, double *w_out, int32_t *oi,
                                int32_t *oj, double *oxi, double *of3, double *oscale,
                                double *fmag, double *tmag, int64_t cap)
{
    half_step(n, x, v, a, dt, x_out, vstar_out);
    for (int64_t k = 0; k < 3 * n; ++k) wstar_out[k] = w[k] + al[k] * dt;
    const double *X = xf ? xf : x_out, *V = vf ? vf : vstar_out, *W = wf ? wf : wstar_out;
    double *F = (double *)calloc((size_t)(n > 0 ? n : 1) * 3, sizeof(double));
    double *T = (double *)calloc((size_t)(n > 0 ? n : 1) * 3, sizeof(double));
    if (!F || !T) { free(F); free(T); return -1; }
    memset(fmag, 0, (size_t)n * sizeof(double));
    memset(tmag, 0, (size_t)n * sizeof(double));
    int32_t *ci = NULL, *cj = NULL;
    int64_t np = P->contacts_on ? contact_candidates(n, X, r, &ci, &cj) : 0;
    if (np < 0) { free(F); free(T); return -1; }
    double kt = kt_ratio * P->kn;
    int64_t m = 0;
    for (int64_t k = 0; k < np; ++k) {
        int64_t i = ci[k], j = cj[k];
        double d[3], dist2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            d[c] = X[3 * i + c] - X[3 * j + c];
            dist2 += d[c] * d[c];
        }
        double dist = sqrt(dist2);
        double dl = (r[i] + r[j]) - dist;
        if (!(dl > 0.0) || !(dist > 0.0)) continue;
        double nr[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
        double s[3], u[3];
        for (int c = 0; c < 3; ++c) s[c] = r[i] * W[3 * i + c] + r[j] * W[3 * j + c];
        double sxn[3] = {s[1] * nr[2] - s[2] * nr[1], s[2] * nr[0] - s[0] * nr[2],
                         s[0] * nr[1] - s[1] * nr[0]};
        for (int c = 0; c < 3; ++c) u[c] = (V[3 * i + c] - V[3 * j + c]) - sxn[c];
        double vn = u[0] * nr[0] + u[1] * nr[1] + u[2] * nr[2];
        double vt[3] = {u[0] - vn * nr[0], u[1] - vn * nr[1], u[2] - vn * nr[2]};
        double mi = mass_of(r[i], P->rho), mj = mass_of(r[j], P->rho);
        double meff = mi * mj / (mi + mj);
        double fn = lsd_force(P, dl, vn, meff);
        double gam_n = 2.0 * zeta_of(P->restitution) * sqrt(meff * P->kn);
        double gt = gt_ratio * gam_n;
        double xi[3] = {0.0, 0.0, 0.0};
        int64_t h = nh > 0 ? find_pair(nh, hi, hj, (int32_t)i, (int32_t)j) : -1;
        if (h >= 0) for (int c = 0; c < 3; ++c) xi[c] = hxi[3 * h + c];
        double xn = xi[0] * nr[0] + xi[1] * nr[1] + xi[2] * nr[2];
        for (int c = 0; c < 3; ++c) xi[c] = xi[c] - xn * nr[c] + vt[c] * dt;
        double Ft[3], fm2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            Ft[c] = -kt * xi[c] - gt * vt[c];
            fm2 += Ft[c] * Ft[c];
        }
        double fm = sqrt(fm2), lim = mu * (fn > 0.0 ? fn : 0.0);
        if (fm > lim) {
            for (int c = 0; c < 3; ++c) {
                Ft[c] *= lim / fm;
                xi[c] = -(Ft[c] + gt * vt[c]) / kt;
            }
        }
        double nxf[3] = {nr[1] * Ft[2] - nr[2] * Ft[1], nr[2] * Ft[0] - nr[0] * Ft[2],
                         nr[0] * Ft[1] - nr[1] * Ft[0]};
        double sc_t = kt * sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]) +
                      gt * sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
        double sc = fabs(P->kn * dl) + fabs(fn - P->kn * dl) + sc_t;
        for (int c = 0; c < 3; ++c) {
            F[3 * i + c] += fn * nr[c] + Ft[c];
            F[3 * j + c] -= fn * nr[c] + Ft[c];
            T[3 * i + c] -= r[i] * nxf[c];
            T[3 * j + c] -= r[j] * nxf[c];
        }
        fmag[i] += sc;
        fmag[j] += sc;
        tmag[i] += r[i] * sc_t;
        tmag[j] += r[j] * sc_t;
        if (m < cap) {
            oi[m] = (int32_t)i;
            oj[m] = (int32_t)j;
            for (int c = 0; c < 3; ++c) {
                oxi[3 * m + c] = xi[c];
                of3[3 * m + c] = fn * nr[c] + Ft[c];
            }
            oscale[m] = sc;
        }
        ++m;
    }
    free(ci); free(cj);
    /* walls: the normal law (forces at the same state) */
    if (P->wall_kind == 1 || P->wall_kind == 2) {
        double *Fw = (double *)calloc((size_t)(n > 0 ? n : 1) * 3, sizeof(double));
        double *fw = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
        orc_dem_params Q = *P;
        Q.contacts_on = 0;
        if (!Fw || !fw || orc_dem_forces64(n, X, r, V, &Q, Fw, fw) != 0) {
            free(Fw); free(fw); free(F); free(T);
            return -1;
        }
        for (int64_t k = 0; k < 3 * n; ++k) F[k] += Fw[k];
        for (int64_t i = 0; i < n; ++i) fmag[i] += fw[i];
        free(Fw); free(fw);
    }
    for (int64_t i = 0; i < n; ++i) {
        double mi = mass_of(r[i], P->rho), Ii = 0.4 * mi * r[i] * r[i];
        for (int c = 0; c < 3; ++c) {
            double an = F[3 * i + c] / mi + P->g[c];
            a_out[3 * i + c] = an;
            v_out[3 * i + c] = v[3 * i + c] + 0.5 * (a[3 * i + c] + an) * dt;
            double aln = T[3 * i + c] / Ii;
            al_out[3 * i + c] = aln;
            w_out[3 * i + c] = w[3 * i + c] + 0.5 * (al[3 * i + c] + aln) * dt;
        }
    }
    free(F); free(T);
    return m;
}

/* ------------------------------------------------------------------ */
/* Multi-sphere clumps (the clump narrow phase that follows a broad      */
/* phase on bounding spheres, Sec. Background): sub-sphere a of clump i  */
/* at x_i + R(q_i) b_a, q = (w, x, y, z) a unit quaternion,              */
/*   R = [1-2(yy+zz)  2(xy-wz)  2(xz+wy)                                  */
/*        2(xy+wz)  1-2(xx+zz)  2(yz-wx)                                  */
/*        2(xz-wy)  2(yz+wx)  1-2(xx+yy)]                                 */
/* in binary32 with every operation rounded in the order written, each   */
/* component of R b as ((R_k0 b_x + R_k1 b_y) + R_k2 b_z), then added to  */
/* x_i.  A contact: a of i and b of j, i < j, delta = (r_a + r_b) -       */
/* sqrtf(|x_a - x_b|^2) > 0 (Eq. delta).  Brute force over every pair of  */
/* clumps and every pair of their sub-spheres, in (i, j, a, b) order.     */
/* Pinned by: a dumbbell turned by closed-form quaternions, and contacts  */
/* that appear and vanish with the turn (tests).                          */
/* ------------------------------------------------------------------ */
static void clump_rotmat(const float *q, float R[9])
{
    float w = q[0], x = q[1], y = q[2], z = q[3];
    float yy = y * y, zz = z * z, xx = x * x;
    float xy = x * y, wz = w * z, xz = x * z, wy = w * y, yz = y * z, wx = w * x;
    float t;
    t = yy + zz; t = 2.0f * t; R[0] = 1.0f - t;
    t = xy - wz; R[1] = 2.0f * t;
    t = xz + wy; R[2] = 2.0f * t;
    t = xy + wz; R[3] = 2.0f * t;
    t = xx + zz; t = 2.0f * t; R[4] = 1.0f - t;
    t = yz - wx; R[5] = 2.0f * t;
    t = xz - wy; R[6] = 2.0f * t;
    t = yz + wx; R[7] = 2.0f * t;
    t = xx + yy; t = 2.0f * t; R[8] = 1.0f - t;
}

static void clump_world(const float *c4, const float R[9], const float *b4, float out4[4])
{
    for (int k = 0; k < 3; ++k) {
        float p0 = R[3 * k + 0] * b4[0];
        float p1 = R[3 * k + 1] * b4[1];
        float p2 = R[3 * k + 2] * b4[2];
        float s = p0 + p1;
        s = s + p2;
        out4[k] = c4[k] + s;
    }
    out4[3] = b4[3];
}

ORC_API int64_t orc_clump_contacts(int64_t n, const float *pos4, const float *quat4,
                                   const int32_t *sub_off, const float *sub4, int32_t *ci,
                                   int32_t *ca, int32_t *cj, int32_t *cb, float *delta,
                                   int64_t cap)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        float Ri[9];
        clump_rotmat(quat4 + 4 * i, Ri);
        for (int64_t j = i + 1; j < n; ++j) {
            float Rj[9];
            clump_rotmat(quat4 + 4 * j, Rj);
            for (int32_t a = sub_off[i]; a < sub_off[i + 1]; ++a) {
                float wa[4];
                clump_world(pos4 + 4 * i, Ri, sub4 + 4 * (int64_t)a, wa);
                for (int32_t b = sub_off[j]; b < sub_off[j + 1]; ++b) {
                    float wb[4];
                    clump_world(pos4 + 4 * j, Rj, sub4 + 4 * (int64_t)b, wb);
                    float dl = overlap_f32(wa, wb);
                    if (dl > 0.0f) {
                        if (m < cap) {
                            ci[m] = (int32_t)i;
                            ca[m] = a - sub_off[i];
                            cj[m] = (int32_t)j;
                            cb[m] = b - sub_off[j];
                            delta[m] = dl;
                        }
                        ++m;
                    }
                }
            }
        }
    }
    return m;
}

/* Improvement of Eq. impr (Sec. Results):                               */
/*   Improvement = (T_without - T_case) / T_without * 100                */
/* Pinned by: the values printed in Table tab:summary.                   */
ORC_API double orc_improvement_pct(double t_without, double t_case)
{
    return (t_without - t_case) / t_without * 100.0;
}
