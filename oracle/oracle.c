/*
 * oracle.c -- plain FP64 CPU implementation of the TAGI convolution sums.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA library.
 *
 * What it computes (arXiv:2003.01833):
 *   - the discrete convolution sum of Eq. direct-sum, skipping r = 0, with
 *       Yukawa kernel  G_k(r) = exp(-k r) / (4 pi r)          (Eq. Hemlholtz_Greens_Function / 2)
 *       Coulomb kernel 1 / r                                    (Eq. Coulomb)
 *     and the singularity subtraction of Eq. yukawa-conv-ss (correction 4 pi f/k^2,
 *     i.e. f/k^2 for G_k) and Eq. coulomb-conv-ss / correction_term (2 pi alpha^2 f);
 *   - the barycentric Lagrange treecode of Section 5 / Algorithm 3:
 *       source-cluster tree (Section 5.1), Chebyshev points of the 2nd kind
 *       mapped to each cluster, barycentric Lagrange basis (Eq. Lagrange_polynomials,
 *       barycentric_weights), proxy weights of Eq. particle-cluster-approx-rearranged,
 *       MAC of Eq. MAC and the recursion ComputePotential of Algorithm 3.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   tree: root = minimal bounding box of the points; a cluster is a leaf iff
 *     it holds <= N_L points; split dimensions are those whose extent e_d
 *     satisfies e_d * sqrt(2) >= max extent; the cut is at the midpoint
 *     (lo+hi)*0.5 of the shrunk box and a point with x_d >= mid goes to the
 *     upper child; empty children are dropped; children are ordered by the
 *     code sum_d 2^d [x_d >= mid_d]; a box with zero extent in every
 *     dimension is a leaf.  Center = (lo+hi)*0.5, radius = half diagonal,
 *     R = distance between centers.
 *   MAC: (r_B + r_C) / R < theta (strict; R = 0 fails) and (n+1)^3 < N_S.
 *   SS in the far field: two charge sets, q = f w and w, are anterpolated;
 *     Yukawa far term G(x_i,s_k) (qh_k - f_i wh_k); Coulomb far term
 *     (qh_k - f_i wh_k exp(-r^2/alpha^2)) / r.
 *   Anterpolation: a source coordinate equal to a node takes the Kronecker
 *     delta; with zero extent every node coincides, the first one is taken.
 *
 * Built with -ffp-contract=off so that the geometric decisions (which points
 * go to which child, MAC outcomes) round exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846
#define ORACLE_SQRT2 1.4142135623730951

/* ------------------------------------------------------------------ */
/* Direct sums: Eq. direct-sum with the SS of Section 3.3              */
/* ------------------------------------------------------------------ */

/* u_i = sum_{j, r_ij != 0} exp(-k r)/(4 pi r) * (f_j - f_i) w_j + f_i / k^2   (ss = 1)
 * u_i = sum_{j, r_ij != 0} exp(-k r)/(4 pi r) * f_j w_j                        (ss = 0)
 * Targets are the points t (nt of them), sources the points s (ns). */
void oracle_direct_yukawa(int64_t nt, const double* tx, const double* ty, const double* tz,
                          const double* tf, int64_t ns, const double* sx, const double* sy,
                          const double* sz, const double* sw, const double* sf, double k,
                          int ss, double* u)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; i++) {
        double acc = 0.0;
        for (int64_t j = 0; j < ns; j++) {
            double dx = tx[i] - sx[j], dy = ty[i] - sy[j], dz = tz[i] - sz[j];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r == 0.0) continue; /* the singular r' = r term is skipped */
            double G = exp(-k * r) / (4.0 * ORACLE_PI * r);
            if (ss)
                acc += G * (sf[j] - tf[i]) * sw[j];
            else
                acc += G * sf[j] * sw[j];
        }
        u[i] = ss ? acc + tf[i] / (k * k) : acc;
    }
}

/* V_i = sum_{j, r != 0} (rho_j - rho_i exp(-r^2/alpha^2)) w_j / r + 2 pi alpha^2 rho_i  (ss = 1)
 * V_i = sum_{j, r != 0} rho_j w_j / r                                                   (ss = 0) */
void oracle_direct_coulomb(int64_t nt, const double* tx, const double* ty, const double* tz,
                           const double* trho, int64_t ns, const double* sx, const double* sy,
                           const double* sz, const double* sw, const double* srho, double alpha,
                           int ss, double* v)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nt; i++) {
        double acc = 0.0;
        for (int64_t j = 0; j < ns; j++) {
            double dx = tx[i] - sx[j], dy = ty[i] - sy[j], dz = tz[i] - sz[j];
            double r2 = dx * dx + dy * dy + dz * dz;
            double r = sqrt(r2);
            if (r == 0.0) continue;
            if (ss)
                acc += (srho[j] - trho[i] * exp(-r2 / (alpha * alpha))) * sw[j] / r;
            else
                acc += srho[j] * sw[j] / r;
        }
        v[i] = ss ? acc + 2.0 * ORACLE_PI * alpha * alpha * trho[i] : acc;
    }
}

/* ------------------------------------------------------------------ */
/* Source-cluster tree (Section 5.1)                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    int leaf_size;
    const double *x, *y, *z; /* borrowed: the caller keeps them alive */
    int64_t* idx;            /* point indices; cluster c owns idx[begin[c] .. end[c]) */
    int nc, cap;
    int64_t *begin, *end;
    double *lo, *hi; /* 3 per cluster */
    int *parent, *level, *nchild, *child; /* child: 8 per cluster */
} oracle_tree;

static int tree_new_cluster(oracle_tree* t)
{
    if (t->nc == t->cap) {
        int cap = t->cap ? 2 * t->cap : 64;
        t->begin = realloc(t->begin, sizeof(int64_t) * cap);
        t->end = realloc(t->end, sizeof(int64_t) * cap);
        t->lo = realloc(t->lo, sizeof(double) * 3 * cap);
        t->hi = realloc(t->hi, sizeof(double) * 3 * cap);
        t->parent = realloc(t->parent, sizeof(int) * cap);
        t->level = realloc(t->level, sizeof(int) * cap);
        t->nchild = realloc(t->nchild, sizeof(int) * cap);
        t->child = realloc(t->child, sizeof(int) * 8 * cap);
        t->cap = cap;
    }
    return t->nc++;
}

static double coord(const oracle_tree* t, int d, int64_t i)
{
    return d == 0 ? t->x[i] : (d == 1 ? t->y[i] : t->z[i]);
}

/* Build the cluster holding idx[b..e), then its children, depth first. */
static int tree_build_cluster(oracle_tree* t, int64_t b, int64_t e, int parent, int level,
                              int64_t* scratch)
{
    int c = tree_new_cluster(t);
    t->begin[c] = b;
    t->end[c] = e;
    t->parent[c] = parent;
    t->level[c] = level;
    t->nchild[c] = 0;
    /* the cluster is shrunk to the minimal bounding box of its points */
    double lo[3], hi[3];
    for (int d = 0; d < 3; d++) {
        lo[d] = coord(t, d, t->idx[b]);
        hi[d] = lo[d];
        for (int64_t p = b + 1; p < e; p++) {
            double v = coord(t, d, t->idx[p]);
            if (v < lo[d]) lo[d] = v;
            if (v > hi[d]) hi[d] = v;
        }
        t->lo[3 * c + d] = lo[d];
        t->hi[3 * c + d] = hi[d];
    }
    if (e - b <= t->leaf_size) return c; /* leaf: at most N_L points */
    double ext[3], emax = 0.0;
    for (int d = 0; d < 3; d++) {
        ext[d] = hi[d] - lo[d];
        if (ext[d] > emax) emax = ext[d];
    }
    if (emax == 0.0) return c; /* coincident points cannot be separated */
    int split[3];
    double mid[3];
    for (int d = 0; d < 3; d++) {
        /* bisect only the dimensions that keep the aspect ratio <= sqrt(2) */
        split[d] = ext[d] * ORACLE_SQRT2 >= emax;
        mid[d] = (lo[d] + hi[d]) * 0.5;
    }
    /* bucket the points by child code, keeping their relative order */
    int64_t count[8] = {0};
    for (int64_t p = b; p < e; p++) {
        int code = 0;
        for (int d = 0; d < 3; d++)
            if (split[d] && coord(t, d, t->idx[p]) >= mid[d]) code |= 1 << d;
        count[code]++;
    }
    int64_t start[8], fill[8];
    start[0] = b;
    for (int q = 1; q < 8; q++) start[q] = start[q - 1] + count[q - 1];
    for (int q = 0; q < 8; q++) fill[q] = start[q];
    for (int64_t p = b; p < e; p++) {
        int code = 0;
        for (int d = 0; d < 3; d++)
            if (split[d] && coord(t, d, t->idx[p]) >= mid[d]) code |= 1 << d;
        scratch[fill[code]++] = t->idx[p];
    }
    memcpy(t->idx + b, scratch + b, sizeof(int64_t) * (size_t)(e - b));
    for (int q = 0; q < 8; q++) {
        if (count[q] == 0) continue;
        int ch = tree_build_cluster(t, start[q], start[q] + count[q], c, level + 1, scratch);
        t->child[8 * c + t->nchild[c]] = ch;
        t->nchild[c]++;
    }
    return c;
}

oracle_tree* oracle_tree_build(int64_t n, const double* x, const double* y, const double* z,
                               int leaf_size)
{
    if (n <= 0 || leaf_size < 1) return NULL;
    oracle_tree* t = calloc(1, sizeof(oracle_tree));
    t->n = n;
    t->leaf_size = leaf_size;
    t->x = x;
    t->y = y;
    t->z = z;
    t->idx = malloc(sizeof(int64_t) * n);
    for (int64_t i = 0; i < n; i++) t->idx[i] = i;
    int64_t* scratch = malloc(sizeof(int64_t) * n);
    tree_build_cluster(t, 0, n, -1, 0, scratch);
    free(scratch);
    return t;
}

void oracle_tree_free(oracle_tree* t)
{
    if (!t) return;
    free(t->idx);
    free(t->begin);
    free(t->end);
    free(t->lo);
    free(t->hi);
    free(t->parent);
    free(t->level);
    free(t->nchild);
    free(t->child);
    free(t);
}

int oracle_tree_num_clusters(const oracle_tree* t) { return t->nc; }

/* Copy the tree out: idx[n], per cluster begin, end, lo[3], hi[3], parent,
 * level, nchild, child[8]. */
void oracle_tree_export(const oracle_tree* t, int64_t* idx, int64_t* begin, int64_t* end,
                        double* lo, double* hi, int* parent, int* level, int* nchild, int* child)
{
    memcpy(idx, t->idx, sizeof(int64_t) * t->n);
    memcpy(begin, t->begin, sizeof(int64_t) * t->nc);
    memcpy(end, t->end, sizeof(int64_t) * t->nc);
    memcpy(lo, t->lo, sizeof(double) * 3 * t->nc);
    memcpy(hi, t->hi, sizeof(double) * 3 * t->nc);
    memcpy(parent, t->parent, sizeof(int) * t->nc);
    memcpy(level, t->level, sizeof(int) * t->nc);
    memcpy(nchild, t->nchild, sizeof(int) * t->nc);
    memcpy(child, t->child, sizeof(int) * 8 * t->nc);
}

static void cluster_center_radius(const oracle_tree* t, int c, double* cen, double* rad)
{
    double e[3];
    for (int d = 0; d < 3; d++) {
        cen[d] = (t->lo[3 * c + d] + t->hi[3 * c + d]) * 0.5;
        e[d] = t->hi[3 * c + d] - t->lo[3 * c + d];
    }
    *rad = sqrt((e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]) * 0.5;
}

/* ------------------------------------------------------------------ */
/* Algorithm 3, ComputePotential: the list of batch-cluster interactions */
/* ------------------------------------------------------------------ */

/* kind: 0 = direct (Eq. direct-sum_2), 1 = approximation (Eq. particle-cluster-approx-rearranged) */
typedef void (*visit_fn)(void* ctx, int batch, int cluster, int kind);

static void compute_potential(const oracle_tree* t, int batch, int cluster, double theta,
                              int64_t np, visit_fn visit, void* ctx)
{
    double cb[3], rb, cc[3], rc;
    cluster_center_radius(t, batch, cb, &rb);
    cluster_center_radius(t, cluster, cc, &rc);
    double dx = cb[0] - cc[0], dy = cb[1] - cc[1], dz = cb[2] - cc[2];
    double R = sqrt((dx * dx + dy * dy) + dz * dz);
    int64_t ns = t->end[cluster] - t->begin[cluster];
    int theta_ok = (rb + rc) / R < theta;
    int size_ok = np < ns;
    if (theta_ok && size_ok) {
        visit(ctx, batch, cluster, 1);
    } else if (!theta_ok) {
        if (t->nchild[cluster] == 0)
            visit(ctx, batch, cluster, 0);
        else
            for (int q = 0; q < t->nchild[cluster]; q++)
                compute_potential(t, batch, t->child[8 * cluster + q], theta, np, visit, ctx);
    } else {
        visit(ctx, batch, cluster, 0); /* (n+1)^3 >= N_S: direct with the whole cluster */
    }
}

typedef struct {
    int64_t cap, cnt;
    int* batch;
    int* cluster;
    int* kind;
} list_ctx;

static void list_visit(void* vctx, int batch, int cluster, int kind)
{
    list_ctx* L = (list_ctx*)vctx;
    if (L->cnt < L->cap) {
        L->batch[L->cnt] = batch;
        L->cluster[L->cnt] = cluster;
        L->kind[L->cnt] = kind;
    }
    L->cnt++;
}

/* Every (batch, cluster, kind) triple Algorithm 3 visits, batches in cluster
 * order (the batches are the leaves, N_B = N_L).  Returns the total count; the
 * arrays are filled up to cap entries. */
int64_t oracle_tree_lists(const oracle_tree* t, double theta, int degree, int64_t cap,
                          int* batch, int* cluster, int* kind)
{
    list_ctx L = {cap, 0, batch, cluster, kind};
    int64_t np = (int64_t)(degree + 1) * (degree + 1) * (degree + 1);
    for (int b = 0; b < t->nc; b++)
        if (t->nchild[b] == 0) compute_potential(t, b, 0, theta, np, list_visit, &L);
    return L.cnt;
}

/* ------------------------------------------------------------------ */
/* Barycentric Lagrange interpolation (Section 5.2)                     */
/* ------------------------------------------------------------------ */

/* Chebyshev points of the second kind cos(pi k / n) mapped linearly to [a, b]. */
static void cluster_nodes(double a, double b, int n, double* s)
{
    double c = (a + b) * 0.5, h = (b - a) * 0.5;
    for (int k = 0; k <= n; k++) s[k] = c + h * cos(ORACLE_PI * k / n);
}

/* L_k(t) for k = 0..n (Eq. Lagrange_polynomials with b_k of Eq. barycentric_weights). */
static void lagrange_basis(double t, const double* s, int n, double* L)
{
    for (int k = 0; k <= n; k++)
        if (t == s[k]) {
            for (int m = 0; m <= n; m++) L[m] = (m == k) ? 1.0 : 0.0;
            return;
        }
    double den = 0.0;
    for (int k = 0; k <= n; k++) {
        double bk = ((k % 2) ? -1.0 : 1.0) * ((k == 0 || k == n) ? 0.5 : 1.0);
        L[k] = bk / (t - s[k]);
        den += L[k];
    }
    for (int k = 0; k <= n; k++) L[k] /= den;
}

/* Proxy positions of cluster c: px, py, pz each of length (n+1)^3, index
 * (k1 * (n+1) + k2) * (n+1) + k3. */
void oracle_cluster_proxies(const oracle_tree* t, int c, int n, double* px, double* py, double* pz)
{
    double s[3][64];
    for (int d = 0; d < 3; d++) cluster_nodes(t->lo[3 * c + d], t->hi[3 * c + d], n, s[d]);
    int m = n + 1;
    for (int k1 = 0; k1 < m; k1++)
        for (int k2 = 0; k2 < m; k2++)
            for (int k3 = 0; k3 < m; k3++) {
                int p = (k1 * m + k2) * m + k3;
                px[p] = s[0][k1];
                py[p] = s[1][k2];
                pz[p] = s[2][k3];
            }
}

/* Proxy weights of Eq. particle-cluster-approx-rearranged for nq charge
 * vectors q[iq * n_points + j] (caller's point order):
 *   qh[iq * P + k] = sum_{j in C} L_k1(x_j) L_k2(y_j) L_k3(z_j) q_j. */
void oracle_anterpolate(const oracle_tree* t, int c, int n, int nq, const double* q, double* qh)
{
    int m = n + 1, P = m * m * m;
    double s[3][64], Lx[64], Ly[64], Lz[64];
    for (int d = 0; d < 3; d++) cluster_nodes(t->lo[3 * c + d], t->hi[3 * c + d], n, s[d]);
    for (int i = 0; i < nq * P; i++) qh[i] = 0.0;
    for (int64_t p = t->begin[c]; p < t->end[c]; p++) {
        int64_t j = t->idx[p];
        lagrange_basis(t->x[j], s[0], n, Lx);
        lagrange_basis(t->y[j], s[1], n, Ly);
        lagrange_basis(t->z[j], s[2], n, Lz);
        for (int k1 = 0; k1 < m; k1++)
            for (int k2 = 0; k2 < m; k2++)
                for (int k3 = 0; k3 < m; k3++) {
                    double L = Lx[k1] * Ly[k2] * Lz[k3];
                    int k = (k1 * m + k2) * m + k3;
                    for (int iq = 0; iq < nq; iq++) qh[iq * P + k] += L * q[iq * t->n + j];
                }
    }
}

/* ------------------------------------------------------------------ */
/* Treecode (Algorithm 3) with the SS of Section 3.3                    */
/* ------------------------------------------------------------------ */

typedef struct {
    const oracle_tree* t;
    int n, P, kernel, ss; /* kernel 0 = Yukawa, 1 = Coulomb */
    double param;         /* k or alpha */
    const double *f, *w;  /* caller order */
    double** qh;          /* per cluster: 2*P values (qh of f w, then wh of w), or NULL */
    double* u;            /* output, caller order */
} tc_ctx;

static double kernel_yukawa(double r, double k) { return exp(-k * r) / (4.0 * ORACLE_PI * r); }

static void tc_visit(void* vctx, int batch, int cluster, int kind)
{
    tc_ctx* C = (tc_ctx*)vctx;
    const oracle_tree* t = C->t;
    double px[1000], py[1000], pz[1000];
    if (kind == 1) oracle_cluster_proxies(t, cluster, C->n, px, py, pz);
    for (int64_t pb = t->begin[batch]; pb < t->end[batch]; pb++) {
        int64_t i = t->idx[pb];
        double xi = t->x[i], yi = t->y[i], zi = t->z[i], fi = C->f[i];
        double acc = 0.0;
        if (kind == 0) { /* Eq. direct-sum_2 */
            for (int64_t ps = t->begin[cluster]; ps < t->end[cluster]; ps++) {
                int64_t j = t->idx[ps];
                double dx = xi - t->x[j], dy = yi - t->y[j], dz = zi - t->z[j];
                double r2 = dx * dx + dy * dy + dz * dz, r = sqrt(r2);
                if (r == 0.0) continue;
                if (C->kernel == 0) {
                    double G = kernel_yukawa(r, C->param);
                    acc += C->ss ? G * (C->f[j] - fi) * C->w[j] : G * C->f[j] * C->w[j];
                } else {
                    double a2 = C->param * C->param;
                    acc += C->ss ? (C->f[j] - fi * exp(-r2 / a2)) * C->w[j] / r
                                 : C->f[j] * C->w[j] / r;
                }
            }
        } else { /* Eq. particle-cluster-approx-rearranged */
            const double* qh = C->qh[cluster];
            const double* wh = qh + C->P;
            for (int k = 0; k < C->P; k++) {
                double dx = xi - px[k], dy = yi - py[k], dz = zi - pz[k];
                double r2 = dx * dx + dy * dy + dz * dz, r = sqrt(r2);
                if (C->kernel == 0) {
                    double G = kernel_yukawa(r, C->param);
                    acc += C->ss ? G * (qh[k] - fi * wh[k]) : G * qh[k];
                } else {
                    double a2 = C->param * C->param;
                    acc += C->ss ? (qh[k] - fi * wh[k] * exp(-r2 / a2)) / r : qh[k] / r;
                }
            }
        }
        C->u[i] += acc;
    }
}

/* One convolution by the treecode.  kernel 0: Yukawa with k = param,
 * kernel 1: Coulomb with alpha = param.  f, w and u in the caller's order. */
int oracle_treecode(const oracle_tree* t, double theta, int degree, int kernel, double param,
                    int ss, const double* f, const double* w, double* u)
{
    if (degree < 1 || degree > 9) return 1;
    int m = degree + 1, P = m * m * m;
    tc_ctx C0 = {t, degree, P, kernel, ss, param, f, w, NULL, u};
    C0.qh = calloc(t->nc, sizeof(double*));
    /* Algorithm 3 line 2: proxy weights of every cluster that may be approximated */
    double* q2 = malloc(sizeof(double) * 2 * t->n);
    for (int64_t j = 0; j < t->n; j++) {
        q2[j] = f[j] * w[j];
        q2[t->n + j] = w[j];
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < t->nc; c++) {
        if (t->end[c] - t->begin[c] <= P) continue;
        C0.qh[c] = malloc(sizeof(double) * 2 * P);
        oracle_anterpolate(t, c, degree, 2, q2, C0.qh[c]);
    }
    free(q2);
    for (int64_t i = 0; i < t->n; i++) u[i] = 0.0;
    /* Algorithm 3 line 3: every batch (leaf) walks the tree from the root */
    int nleaf = 0;
    int* leaves = malloc(sizeof(int) * t->nc);
    for (int c = 0; c < t->nc; c++)
        if (t->nchild[c] == 0) leaves[nleaf++] = c;
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nleaf; b++) {
        tc_ctx C = C0;
        compute_potential(t, leaves[b], 0, theta, P, tc_visit, &C);
    }
    free(leaves);
    /* SS corrections, Eq. yukawa-conv-ss (4 pi f / k^2 over 4 pi) and Eq. correction_term */
    if (ss)
        for (int64_t i = 0; i < t->n; i++)
            u[i] += kernel == 0 ? f[i] / (param * param) : 2.0 * ORACLE_PI * param * param * f[i];
    for (int c = 0; c < t->nc; c++) free(C0.qh[c]);
    free(C0.qh);
    return 0;
}

/* Treecode restricted to a subset of batches (used for bounded CPU timing).
 * batches: cluster ids of leaves; u accumulates their targets only. */
int oracle_treecode_batches(const oracle_tree* t, double theta, int degree, int kernel,
                            double param, int ss, const double* f, const double* w, int nb,
                            const int* batches, double* u)
{
    if (degree < 1 || degree > 9) return 1;
    int m = degree + 1, P = m * m * m;
    tc_ctx C0 = {t, degree, P, kernel, ss, param, f, w, NULL, u};
    C0.qh = calloc(t->nc, sizeof(double*));
    double* q2 = malloc(sizeof(double) * 2 * t->n);
    for (int64_t j = 0; j < t->n; j++) {
        q2[j] = f[j] * w[j];
        q2[t->n + j] = w[j];
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < t->nc; c++) {
        if (t->end[c] - t->begin[c] <= P) continue;
        C0.qh[c] = malloc(sizeof(double) * 2 * P);
        oracle_anterpolate(t, c, degree, 2, q2, C0.qh[c]);
    }
    free(q2);
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nb; b++) {
        tc_ctx C = C0;
        compute_potential(t, batches[b], 0, theta, P, tc_visit, &C);
        if (ss)
            for (int64_t p = t->begin[batches[b]]; p < t->end[batches[b]]; p++) {
                int64_t i = t->idx[p];
                u[i] += kernel == 0 ? f[i] / (param * param) : 2.0 * ORACLE_PI * param * param * f[i];
            }
    }
    for (int c = 0; c < t->nc; c++) free(C0.qh[c]);
    free(C0.qh);
    return 0;
}

/* Threads of the OpenMP loops above (the benchmark times the oracle on all
 * cores and on one); n < 1 leaves the setting alone.  Returns the count the
 * next parallel loop will use. */
int oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
