/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU reference for the element matrices of
 * Khodapanah, "A Product to Sum Approach for Matrix Filling in a Hierarchical
 * Finite-Element Method" (arXiv:1703.09619).  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load this library; the
 * product path (the CUDA library) never links, calls or reads it, and the two
 * share no source, header, table or constant generator.
 *
 * What it computes (Sec. II, Eq. (1)-(2)): for each element, each pair of
 * field components (gi, gj) and each product type t, the matrix entry
 *
 *   M_t[(gi,m1,n1,p1),(gj,m2,n2,p2)]
 *     = sum_{a,b,c} w_a w_b w_c  f_u(a) f_v(b) f_w(c)  alpha_{gi gj}(u_a,v_b,w_c)
 *
 * with f_u(a) = P^{(d1)}_{m1}(u_a) P^{(d2)}_{m2}(u_a) (same for v, w), Legendre
 * P, Gauss-Legendre nodes/weights (u_a, w_a), and (d1, d2) = (0,0), (1,0),
 * (0,1), (1,1) for t = vv, dv, vd, dd.  This is the "direct numerical
 * integration" the paper compares against (Sec. II, text after Eq. (2);
 * Sec. IV operation count); the product-to-sum method of Eq. (3)-(4) reaches
 * the same number up to rounding when it uses the same quadrature rule,
 * because the linearisation of Eq. (3) is an exact polynomial identity and
 * quadrature is linear.  Every entry is summed over all G^3 points in the
 * order written above with Neumaier-compensated summation.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - basis = plain Legendre P_m, P_m(1) = 1, m = 0..N-1 (Sec. II says
 *     "orthogonal polynomials");
 *   - reference element [-1,1]^3 (limits of Eq. (2));
 *   - the four product types use the same value/derivative choice on all
 *     three axes (one entry of each column vector of Eq. (2));
 *   - coupling factor of block (gi,gj) in the three-component case:
 *     alpha_{gi gj} = eps(x) * detJ * (J^{-1} J^{-T})_{gi gj}, J = dx/d(u,v,w),
 *     with a trilinear-plus-bulge geometry map (the Jacobian/material coupling
 *     of Sec. I and Eq. (2); Eq. (12)-(15) show its 2-D analogue);
 *   - one-component case: a scalar coupling factor given in reference
 *     coordinates.
 *
 * Output layout (shared by contract with the CUDA library's header, not by
 * code): per element, the selected types in the order vv, dv, vd, dd, each an
 * n x n row-major matrix, n = sum_g Nu_g Nv_g Nw_g; dof index = offset of
 * component g + (m*Nv_g + n)*Nw_g + p.
 *
 * Compile with -ffp-contract=off and without -ffast-math.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXG 128
#define OR_MAXN 32

/* ----------------------------------------------------------------------- */
/* 1-D Legendre polynomials (values and first derivatives).                 */
/* Values by the three-term recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1};
 * derivatives by (1 - x^2) P'_j = j (P_{j-1} - x P_j), valid for |x| < 1
 * (all Gauss-Legendre nodes are interior).  At |x| = 1 the closed form
 * P'_j(+-1) = (+-1)^{j-1} j (j+1) / 2 is used.                            */
void or_legendre(int n, double x, double* P, double* dP)
{
    if (n <= 0) return;
    P[0] = 1.0;
    if (n > 1) P[1] = x;
    for (int j = 1; j + 1 < n; ++j)
        P[j + 1] = ((2.0 * j + 1.0) * x * P[j] - j * P[j - 1]) / (j + 1.0);
    if (!dP) return;
    dP[0] = 0.0;
    for (int j = 1; j < n; ++j) {
        if (fabs(x) < 1.0) {
            dP[j] = j * (P[j - 1] - x * P[j]) / (1.0 - x * x);
        } else {
            double s = (x > 0 || (j - 1) % 2 == 0) ? 1.0 : -1.0;
            dP[j] = s * j * (j + 1.0) / 2.0;
        }
    }
}

/* Gauss-Legendre rule of G points on [-1,1]: nodes are the roots of P_G,
 * found by Newton's method from the usual cosine guesses; weights
 * w = 2 / ((1 - x^2) P'_G(x)^2).  Nodes are returned in ascending order.   */
int or_gauss_legendre(int G, double* x, double* w)
{
    if (G < 1 || G > OR_MAXG) return -1;
    double P[OR_MAXG + 2], dP[OR_MAXG + 2];
    for (int i = 0; i < G; ++i) {
        double z = cos(M_PI * (i + 0.75) / (G + 0.5));
        for (int it = 0; it < 100; ++it) {
            or_legendre(G + 1, z, P, dP);
            double dz = P[G] / dP[G];
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        or_legendre(G + 1, z, P, dP);
        /* descending z from the cosine guesses -> store ascending */
        x[G - 1 - i] = z;
        w[G - 1 - i] = 2.0 / ((1.0 - z * z) * dP[G] * dP[G]);
    }
    return 0;
}

/* ----------------------------------------------------------------------- */
/* Geometry: trilinear map of 8 nodes plus a bulge.                          */
/* nodes[8][3], node index = iu + 2 iv + 4 iw with iu = 0 at u = -1.
 * x(u,v,w) = sum_n N_n X_n + a b cos(pi u/2) cos(pi v/2) cos(pi w/2),
 * N_n = (1 + s_u u)(1 + s_v v)(1 + s_w w) / 8, s = -1 for i = 0, +1 for 1.
 * bulge = (a, b_x, b_y, b_z).  J[i][j] = d x_i / d xi_j, xi = (u,v,w).     */
void or_map(const double* nodes, const double* bulge, double u, double v, double w,
            double* x, double* J)
{
    double xi[3] = {u, v, w};
    for (int i = 0; i < 3; ++i) {
        x[i] = 0.0;
        for (int j = 0; j < 3; ++j) J[3 * i + j] = 0.0;
    }
    for (int n = 0; n < 8; ++n) {
        double s[3] = {(n & 1) ? 1.0 : -1.0, (n & 2) ? 1.0 : -1.0, (n & 4) ? 1.0 : -1.0};
        double f[3] = {1.0 + s[0] * xi[0], 1.0 + s[1] * xi[1], 1.0 + s[2] * xi[2]};
        double N = f[0] * f[1] * f[2] / 8.0;
        double dN[3] = {s[0] * f[1] * f[2] / 8.0, f[0] * s[1] * f[2] / 8.0, f[0] * f[1] * s[2] / 8.0};
        for (int i = 0; i < 3; ++i) {
            x[i] += N * nodes[3 * n + i];
            for (int j = 0; j < 3; ++j) J[3 * i + j] += dN[j] * nodes[3 * n + i];
        }
    }
    if (bulge) {
        double h = M_PI / 2.0;
        double c[3], sn[3];
        for (int j = 0; j < 3; ++j) { c[j] = cos(h * xi[j]); sn[j] = sin(h * xi[j]); }
        double beta = c[0] * c[1] * c[2];
        double dbeta[3] = {-h * sn[0] * c[1] * c[2], -h * c[0] * sn[1] * c[2], -h * c[0] * c[1] * sn[2]};
        for (int i = 0; i < 3; ++i) {
            x[i] += bulge[0] * bulge[1 + i] * beta;
            for (int j = 0; j < 3; ++j) J[3 * i + j] += bulge[0] * bulge[1 + i] * dbeta[j];
        }
    }
}

/* ----------------------------------------------------------------------- */
/* Coupling factors.                                                         */
enum { OR_ALPHA_SCALAR = 0, OR_ALPHA_METRIC_EPS = 1, OR_ALPHA_POLY = 2 };
#define OR_POLY_DEG 8 /* per-axis monomial count of the oracle-only POLY kind */

/* Number of parameters per element of each kind. */
int or_alpha_nparams(int kind)
{
    switch (kind) {
    case OR_ALPHA_SCALAR: return 4;
    case OR_ALPHA_METRIC_EPS: return 4;
    case OR_ALPHA_POLY: return OR_POLY_DEG * OR_POLY_DEG * OR_POLY_DEG;
    }
    return -1;
}

/* alpha at one reference point.  Writes n_comp*n_comp values, row-major
 * (gi, gj).  Returns detJ for the metric kind (1 otherwise).
 *   SCALAR (n_comp = 1): p = (A, phi, psi, c):
 *       alpha = 1 + A sin(pi (u + phi)) cos(pi (v + psi)) exp(c w)
 *   METRIC_EPS (n_comp = 3): p = (A, k_x, k_y, k_z):
 *       eps = 1 + A sin(k . x(u,v,w)),  alpha = eps detJ J^{-1} J^{-T}
 *   POLY (n_comp = 1, oracle only): alpha = sum c[i][j][k] u^i v^j w^k,
 *       c stored with k fastest.                                            */
double or_alpha(int kind, const double* p, const double* nodes, const double* bulge,
                double u, double v, double w, double* alpha)
{
    if (kind == OR_ALPHA_SCALAR) {
        alpha[0] = 1.0 + p[0] * sin(M_PI * (u + p[1])) * cos(M_PI * (v + p[2])) * exp(p[3] * w);
        return 1.0;
    }
    if (kind == OR_ALPHA_POLY) {
        double s = 0.0;
        double up = 1.0;
        for (int i = 0; i < OR_POLY_DEG; ++i) {
            double vp = 1.0;
            for (int j = 0; j < OR_POLY_DEG; ++j) {
                double wp = 1.0;
                for (int k = 0; k < OR_POLY_DEG; ++k) {
                    s += p[(i * OR_POLY_DEG + j) * OR_POLY_DEG + k] * up * vp * wp;
                    wp *= w;
                }
                vp *= v;
            }
            up *= u;
        }
        alpha[0] = s;
        return 1.0;
    }
    /* metric kind */
    double x[3], J[9];
    or_map(nodes, bulge, u, v, w, x, J);
    /* cofactor matrix C[i][j] = (-1)^{i+j} minor_ij, det = sum_j J[0][j] C[0][j] */
    double C[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            C[3 * i + j] = J[3 * i1 + j1] * J[3 * i2 + j2] - J[3 * i1 + j2] * J[3 * i2 + j1];
        }
    double det = J[0] * C[0] + J[1] * C[1] + J[2] * C[2];
    /* inverse: inv[i][j] = C[j][i] / det */
    double inv[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) inv[3 * i + j] = C[3 * j + i] / det;
    double kx = p[1] * x[0] + p[2] * x[1] + p[3] * x[2];
    double eps = 1.0 + p[0] * sin(kx);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double g = 0.0;
            for (int k = 0; k < 3; ++k) g += inv[3 * i + k] * inv[3 * j + k];
            alpha[3 * i + j] = eps * det * g;
        }
    return det;
}

/* ----------------------------------------------------------------------- */
/* Output bookkeeping.                                                        */
static int popcount4(uint32_t m) { return (int)((m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1)); }

static int64_t elem_ndof(int n_comp, const int32_t* ord)
{
    int64_t n = 0;
    for (int g = 0; g < n_comp; ++g) n += (int64_t)ord[3 * g] * ord[3 * g + 1] * ord[3 * g + 2];
    return n;
}

/* offsets[E+1] (entries); returns total entries. */
int64_t or_output_offsets(int64_t E, int n_comp, const int32_t* orders, uint32_t types_mask,
                          int64_t* offsets)
{
    int nt = popcount4(types_mask & 0xF);
    int64_t off = 0;
    for (int64_t e = 0; e < E; ++e) {
        if (offsets) offsets[e] = off;
        int64_t n = elem_ndof(n_comp, orders + 3 * n_comp * e);
        off += nt * n * n;
    }
    if (offsets) offsets[E] = off;
    return off;
}

/* ----------------------------------------------------------------------- */
/* Direct fill.                                                               */
typedef struct {
    int64_t E;
    int n_comp;
    const int32_t* orders;  /* [E][n_comp][3] */
    int kind;
    const double* params;   /* [E][nparams] */
    const double* nodes;    /* [E][8][3] */
    const double* bulge;    /* [E][4] or NULL */
    const int32_t* npts;    /* [E] */
    uint32_t types_mask;
    double* out;
    const int64_t* offsets;
    /* per-element precomputation, filled by a worker before its rows */
    int status;
    /* work distribution */
    int64_t next_task;
    int64_t n_tasks;
    pthread_mutex_t mu;
    int64_t* task_elem;     /* task -> element */
    int32_t* task_row;      /* task -> row within the element */
} or_job;

/* Neumaier-compensated accumulator */
typedef struct { double s, c; } or_acc;
static inline void acc_add(or_acc* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

/* Per-element cache: alpha at all G^3 points and 1-D polynomial tables.
 * Each worker builds it for the element it is working on (cheap compared
 * with the G^3 sums of every row).                                          */
typedef struct {
    int64_t e;
    int G;
    double xg[OR_MAXG], wg[OR_MAXG];
    double P[OR_MAXN][OR_MAXG], dP[OR_MAXN][OR_MAXG];
    double* alpha; /* [G^3][nc*nc], point index (c*G + b)*G + a */
    size_t alpha_cap;
    int bad_jac;
} or_cache;

static int build_cache(or_job* jb, or_cache* ch, int64_t e)
{
    int G = jb->npts[e];
    if (G < 1 || G > OR_MAXG) return -1;
    ch->e = e;
    ch->G = G;
    or_gauss_legendre(G, ch->xg, ch->wg);
    int nmax = 0;
    const int32_t* ord = jb->orders + 3 * jb->n_comp * e;
    for (int i = 0; i < 3 * jb->n_comp; ++i) if (ord[i] > nmax) nmax = ord[i];
    if (nmax < 1 || nmax > OR_MAXN) return -2;
    for (int a = 0; a < G; ++a) {
        double P[OR_MAXN], dP[OR_MAXN];
        or_legendre(nmax, ch->xg[a], P, dP);
        for (int j = 0; j < nmax; ++j) { ch->P[j][a] = P[j]; ch->dP[j][a] = dP[j]; }
    }
    int nc = jb->n_comp;
    size_t need = (size_t)G * G * G * nc * nc;
    if (need > ch->alpha_cap) {
        free(ch->alpha);
        ch->alpha = (double*)malloc(need * sizeof(double));
        if (!ch->alpha) { ch->alpha_cap = 0; return -4; }
        ch->alpha_cap = need;
    }
    int np = or_alpha_nparams(jb->kind);
    const double* p = jb->params + (size_t)np * e;
    const double* nodes = jb->nodes ? jb->nodes + 24 * e : NULL;
    const double* bulge = jb->bulge ? jb->bulge + 4 * e : NULL;
    ch->bad_jac = 0;
    for (int c = 0; c < G; ++c)
        for (int b = 0; b < G; ++b)
            for (int a = 0; a < G; ++a) {
                double al[9];
                double det = or_alpha(jb->kind, p, nodes, bulge, ch->xg[a], ch->xg[b], ch->xg[c], al);
                if (!(det > 0.0)) ch->bad_jac = 1;
                memcpy(ch->alpha + ((size_t)(c * G + b) * G + a) * nc * nc, al, sizeof(double) * nc * nc);
            }
    return 0;
}

static void fill_row(or_job* jb, or_cache* ch, int64_t e, int row)
{
    const int32_t* ord = jb->orders + 3 * jb->n_comp * e;
    int nc = jb->n_comp;
    int G = ch->G;
    int64_t n = elem_ndof(nc, ord);
    /* locate row -> (gi, m1, n1, p1) */
    int gi = 0, r = row;
    while (r >= ord[3 * gi] * ord[3 * gi + 1] * ord[3 * gi + 2]) {
        r -= ord[3 * gi] * ord[3 * gi + 1] * ord[3 * gi + 2];
        ++gi;
    }
    int Nv_i = ord[3 * gi + 1], Nw_i = ord[3 * gi + 2];
    int m1 = r / (Nv_i * Nw_i), n1 = (r / Nw_i) % Nv_i, p1 = r % Nw_i;
    int tslot = 0;
    for (int t = 0; t < 4; ++t) {
        if (!(jb->types_mask & (1u << t))) continue;
        int d1 = (t == 1 || t == 3), d2 = (t == 2 || t == 3);
        double* orow = jb->out + jb->offsets[e] + (int64_t)tslot * n * n + (int64_t)row * n;
        int64_t col = 0;
        for (int gj = 0; gj < nc; ++gj) {
            int Nu_j = ord[3 * gj], Nv_j = ord[3 * gj + 1], Nw_j = ord[3 * gj + 2];
            for (int m2 = 0; m2 < Nu_j; ++m2)
                for (int n2 = 0; n2 < Nv_j; ++n2)
                    for (int p2 = 0; p2 < Nw_j; ++p2) {
                        or_acc acc = {0.0, 0.0};
                        for (int c = 0; c < G; ++c) {
                            double fw = (d1 ? ch->dP[p1][c] : ch->P[p1][c]) * (d2 ? ch->dP[p2][c] : ch->P[p2][c]);
                            for (int b = 0; b < G; ++b) {
                                double fv = (d1 ? ch->dP[n1][b] : ch->P[n1][b]) * (d2 ? ch->dP[n2][b] : ch->P[n2][b]);
                                for (int a = 0; a < G; ++a) {
                                    double fu = (d1 ? ch->dP[m1][a] : ch->P[m1][a]) * (d2 ? ch->dP[m2][a] : ch->P[m2][a]);
                                    double al = ch->alpha[((size_t)(c * G + b) * G + a) * nc * nc + gi * nc + gj];
                                    acc_add(&acc, ch->wg[a] * ch->wg[b] * ch->wg[c] * fu * fv * fw * al);
                                }
                            }
                        }
                        orow[col++] = acc.s + acc.c;
                    }
        }
        ++tslot;
    }
}

static void* worker(void* arg)
{
    or_job* jb = (or_job*)arg;
    or_cache* ch = (or_cache*)calloc(1, sizeof(or_cache));
    if (!ch) { jb->status = -4; return NULL; }
    ch->e = -1;
    for (;;) {
        pthread_mutex_lock(&jb->mu);
        int64_t t = jb->next_task++;
        pthread_mutex_unlock(&jb->mu);
        if (t >= jb->n_tasks) break;
        int64_t e = jb->task_elem[t];
        if (ch->e != e) {
            int rc = build_cache(jb, ch, e);
            if (rc) { jb->status = rc; continue; }
            if (ch->bad_jac) jb->status = -3;
        }
        fill_row(jb, ch, e, jb->task_row[t]);
    }
    free(ch->alpha);
    free(ch);
    return NULL;
}

/* Direct fill of E elements.  out must hold or_output_offsets(...) doubles.
 * Returns 0, -1 (bad argument), -2 (order out of range), -3 (detJ <= 0 at a
 * quadrature point; the element is still written), -4 (out of memory).      */
int or_fill(int64_t E, int n_comp, const int32_t* orders, int kind, const double* params,
            const double* nodes, const double* bulge, const int32_t* npts, uint32_t types_mask,
            double* out, int nthreads)
{
    if (E < 0 || (n_comp != 1 && n_comp != 3) || !orders || !params || !npts || !out) return -1;
    if (kind == OR_ALPHA_METRIC_EPS && (n_comp != 3 || !nodes)) return -1;
    if (kind != OR_ALPHA_METRIC_EPS && n_comp != 1) return -1;
    if (kind < 0 || kind > 2) return -1;
    for (int64_t i = 0; i < E * 3 * n_comp; ++i)
        if (orders[i] < 1 || orders[i] > OR_MAXN) return -2;
    or_job jb;
    memset(&jb, 0, sizeof(jb));
    jb.E = E; jb.n_comp = n_comp; jb.orders = orders; jb.kind = kind; jb.params = params;
    jb.nodes = nodes; jb.bulge = bulge; jb.npts = npts; jb.types_mask = types_mask; jb.out = out;
    int64_t* offsets = (int64_t*)malloc(sizeof(int64_t) * (E + 1));
    if (!offsets) return -4;
    or_output_offsets(E, n_comp, orders, types_mask, offsets);
    jb.offsets = offsets;
    int64_t ntask = 0;
    for (int64_t e = 0; e < E; ++e) ntask += elem_ndof(n_comp, orders + 3 * n_comp * e);
    jb.task_elem = (int64_t*)malloc(sizeof(int64_t) * (ntask + 1));
    jb.task_row = (int32_t*)malloc(sizeof(int32_t) * (ntask + 1));
    if (!jb.task_elem || !jb.task_row) { free(offsets); free(jb.task_elem); free(jb.task_row); return -4; }
    int64_t t = 0;
    for (int64_t e = 0; e < E; ++e) {
        int64_t n = elem_ndof(n_comp, orders + 3 * n_comp * e);
        for (int64_t r = 0; r < n; ++r) { jb.task_elem[t] = e; jb.task_row[t] = (int32_t)r; ++t; }
    }
    jb.n_tasks = ntask;
    pthread_mutex_init(&jb.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 0; i < nthreads; ++i)
        if (pthread_create(&th[i], NULL, worker, &jb) == 0) ++started;
    if (started == 0) worker(&jb);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&jb.mu);
    free(offsets); free(jb.task_elem); free(jb.task_row);
    return jb.status;
}

/* ----------------------------------------------------------------------- */
/* Operators given as term lists (Eq. (2) in full generality).                */
/* A term adds to the block (gi, gj) of the element matrix
 *
 *   scale * sum_{a,b,c} w_a w_b w_c  f_u(a) f_v(b) f_w(c)  alpha_{sa sb}(u_a, v_b, w_c)
 *
 * with f_u(a) = P^{(du)}_{m1}(u_a) P^{(eu)}_{m2}(u_a), (du, eu) the term's derivative
 * orders of the test and trial functions on u (likewise v, w), so the value /
 * derivative choice may differ per axis.  alpha_{sa sb} is an entry of the coupling
 * factor matrix: for the metric kind eps detJ (J^{-1} J^{-T})_{sa sb} (sa, sb < 3, any
 * number of field components), for the scalar and POLY kinds the scalar (sa = sb = 0).
 * terms: n_terms rows of 10 ints (gi, gj, sa, sb, du, dv, dw, eu, ev, ew); scales[n_terms].
 * Output per element: one n x n row-major matrix, n = sum_g Nu_g Nv_g Nw_g, rows test
 * dofs, columns trial dofs (same dof numbering as or_fill); every entry is the sum over
 * the terms of its block, all terms and points in one Neumaier accumulator.          */
typedef struct {
    or_job jb;           /* elements, geometry, quadrature, output (types_mask unused) */
    int nalpha;          /* entries of the coupling factor matrix per side: 3 or 1 */
    int n_terms;
    const int32_t* terms;
    const double* scales;
} or_opjob;

static int build_cache_op(or_opjob* oj, or_cache* ch, int64_t e)
{
    or_job* jb = &oj->jb;
    int G = jb->npts[e];
    if (G < 1 || G > OR_MAXG) return -1;
    ch->e = e;
    ch->G = G;
    or_gauss_legendre(G, ch->xg, ch->wg);
    int nmax = 0;
    const int32_t* ord = jb->orders + 3 * jb->n_comp * e;
    for (int i = 0; i < 3 * jb->n_comp; ++i) if (ord[i] > nmax) nmax = ord[i];
    if (nmax < 1 || nmax > OR_MAXN) return -2;
    for (int a = 0; a < G; ++a) {
        double P[OR_MAXN], dP[OR_MAXN];
        or_legendre(nmax, ch->xg[a], P, dP);
        for (int j = 0; j < nmax; ++j) { ch->P[j][a] = P[j]; ch->dP[j][a] = dP[j]; }
    }
    int na = oj->nalpha;
    size_t need = (size_t)G * G * G * na * na;
    if (need > ch->alpha_cap) {
        free(ch->alpha);
        ch->alpha = (double*)malloc(need * sizeof(double));
        if (!ch->alpha) { ch->alpha_cap = 0; return -4; }
        ch->alpha_cap = need;
    }
    int np = or_alpha_nparams(jb->kind);
    const double* p = jb->params + (size_t)np * e;
    const double* nodes = jb->nodes ? jb->nodes + 24 * e : NULL;
    const double* bulge = jb->bulge ? jb->bulge + 4 * e : NULL;
    ch->bad_jac = 0;
    for (int c = 0; c < G; ++c)
        for (int b = 0; b < G; ++b)
            for (int a = 0; a < G; ++a) {
                double al[9];
                double det = or_alpha(jb->kind, p, nodes, bulge, ch->xg[a], ch->xg[b], ch->xg[c], al);
                if (!(det > 0.0)) ch->bad_jac = 1;
                memcpy(ch->alpha + ((size_t)(c * G + b) * G + a) * na * na, al, sizeof(double) * na * na);
            }
    return 0;
}

static double fac(const or_cache* ch, int d, int m, int a) { return d ? ch->dP[m][a] : ch->P[m][a]; }

static void fill_row_op(or_opjob* oj, or_cache* ch, int64_t e, int row)
{
    or_job* jb = &oj->jb;
    const int32_t* ord = jb->orders + 3 * jb->n_comp * e;
    int nc = jb->n_comp, na = oj->nalpha;
    int G = ch->G;
    int64_t n = elem_ndof(nc, ord);
    int gi = 0, r = row;
    while (r >= ord[3 * gi] * ord[3 * gi + 1] * ord[3 * gi + 2]) {
        r -= ord[3 * gi] * ord[3 * gi + 1] * ord[3 * gi + 2];
        ++gi;
    }
    int Nv_i = ord[3 * gi + 1], Nw_i = ord[3 * gi + 2];
    int m1 = r / (Nv_i * Nw_i);       /* row r of block gi = (m1 * Nv + n1) * Nw + p1 */
    int n1 = (r / Nw_i) % Nv_i;
    int p1 = r % Nw_i;
    double* orow = jb->out + jb->offsets[e] + (int64_t)row * n;
    int64_t col = 0;
    for (int gj = 0; gj < nc; ++gj) {
        int Nu_j = ord[3 * gj], Nv_j = ord[3 * gj + 1], Nw_j = ord[3 * gj + 2];
        for (int m2 = 0; m2 < Nu_j; ++m2)
            for (int n2 = 0; n2 < Nv_j; ++n2)
                for (int p2 = 0; p2 < Nw_j; ++p2) {
                    or_acc acc = {0.0, 0.0};
                    for (int k = 0; k < oj->n_terms; ++k) {
                        const int32_t* tm = oj->terms + 10 * k;
                        if (tm[0] != gi || tm[1] != gj) continue;
                        int sa = tm[2], sb = tm[3];
                        for (int c = 0; c < G; ++c) {
                            double fw = fac(ch, tm[6], p1, c) * fac(ch, tm[9], p2, c);
                            for (int b = 0; b < G; ++b) {
                                double fv = fac(ch, tm[5], n1, b) * fac(ch, tm[8], n2, b);
                                for (int a = 0; a < G; ++a) {
                                    double fu = fac(ch, tm[4], m1, a) * fac(ch, tm[7], m2, a);
                                    double al = ch->alpha[((size_t)(c * G + b) * G + a) * na * na + sa * na + sb];
                                    acc_add(&acc, oj->scales[k] * (ch->wg[a] * ch->wg[b] * ch->wg[c] * fu * fv * fw * al));
                                }
                            }
                        }
                    }
                    orow[col++] = acc.s + acc.c;
                }
    }
}

static void* worker_op(void* arg)
{
    or_opjob* oj = (or_opjob*)arg;
    or_job* jb = &oj->jb;
    or_cache* ch = (or_cache*)calloc(1, sizeof(or_cache));
    if (!ch) { jb->status = -4; return NULL; }
    ch->e = -1;
    for (;;) {
        pthread_mutex_lock(&jb->mu);
        int64_t t = jb->next_task++;
        pthread_mutex_unlock(&jb->mu);
        if (t >= jb->n_tasks) break;
        int64_t e = jb->task_elem[t];
        if (ch->e != e) {
            int rc = build_cache_op(oj, ch, e);
            if (rc) { jb->status = rc; continue; }
            if (ch->bad_jac) jb->status = -3;
        }
        fill_row_op(oj, ch, e, jb->task_row[t]);
    }
    free(ch->alpha);
    free(ch);
    return NULL;
}

/* Term-list fill of E elements; out holds sum_e n_e^2 doubles (or_output_offsets with
 * types_mask = 1).  Returns as or_fill; -1 also for a term out of range.             */
int or_fill_terms(int64_t E, int n_comp, const int32_t* orders, int kind, const double* params,
                  const double* nodes, const double* bulge, const int32_t* npts, int n_terms,
                  const int32_t* terms, const double* scales, double* out, int nthreads)
{
    if (E < 0 || n_comp < 1 || n_comp > 3 || !orders || !params || !npts || !out || n_terms < 0) return -1;
    if (n_terms > 0 && (!terms || !scales)) return -1;
    if (kind < 0 || kind > 2) return -1;
    if (kind == OR_ALPHA_METRIC_EPS && !nodes) return -1;
    int na = kind == OR_ALPHA_METRIC_EPS ? 3 : 1;
    for (int k = 0; k < n_terms; ++k) {
        const int32_t* tm = terms + 10 * k;
        if (tm[0] < 0 || tm[0] >= n_comp || tm[1] < 0 || tm[1] >= n_comp) return -1;
        if (tm[2] < 0 || tm[2] >= na || tm[3] < 0 || tm[3] >= na) return -1;
        for (int i = 4; i < 10; ++i) if (tm[i] != 0 && tm[i] != 1) return -1;
    }
    for (int64_t i = 0; i < E * 3 * n_comp; ++i)
        if (orders[i] < 1 || orders[i] > OR_MAXN) return -2;
    or_opjob oj;
    memset(&oj, 0, sizeof(oj));
    or_job* jb = &oj.jb;
    jb->E = E; jb->n_comp = n_comp; jb->orders = orders; jb->kind = kind; jb->params = params;
    jb->nodes = nodes; jb->bulge = bulge; jb->npts = npts; jb->types_mask = 1u; jb->out = out;
    oj.nalpha = na; oj.n_terms = n_terms; oj.terms = terms; oj.scales = scales;
    int64_t* offsets = (int64_t*)malloc(sizeof(int64_t) * (E + 1));
    if (!offsets) return -4;
    or_output_offsets(E, n_comp, orders, 1u, offsets);
    jb->offsets = offsets;
    int64_t ntask = 0;
    for (int64_t e = 0; e < E; ++e) ntask += elem_ndof(n_comp, orders + 3 * n_comp * e);
    jb->task_elem = (int64_t*)malloc(sizeof(int64_t) * (ntask + 1));
    jb->task_row = (int32_t*)malloc(sizeof(int32_t) * (ntask + 1));
    if (!jb->task_elem || !jb->task_row) { free(offsets); free(jb->task_elem); free(jb->task_row); return -4; }
    int64_t t = 0;
    for (int64_t e = 0; e < E; ++e) {
        int64_t n = elem_ndof(n_comp, orders + 3 * n_comp * e);
        for (int64_t r = 0; r < n; ++r) { jb->task_elem[t] = e; jb->task_row[t] = (int32_t)r; ++t; }
    }
    jb->n_tasks = ntask;
    pthread_mutex_init(&jb->mu, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 0; i < nthreads; ++i)
        if (pthread_create(&th[i], NULL, worker_op, &oj) == 0) ++started;
    if (started == 0) worker_op(&oj);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&jb->mu);
    free(offsets); free(jb->task_elem); free(jb->task_row);
    return jb->status;
}

/* ----------------------------------------------------------------------- */
/* Linearisation coefficients by projection (Eq. (3)).                       */
/* C[k] for k = 0..kmax, with P^{(d1)}_{m1} P^{(d2)}_{m2} = sum_k C[k] P_k:
 *   C[k] = (2k+1)/2 * int_{-1}^{1} P^{(d1)}_{m1} P^{(d2)}_{m2} P_k,
 * the integral taken with a Gauss-Legendre rule exact for the integrand's
 * degree (orthogonality of Legendre polynomials, int P_k^2 = 2/(2k+1)).     */
int or_linearisation(int d1, int d2, int m1, int m2, int kmax, double* C)
{
    if (m1 < 0 || m2 < 0 || kmax < 0 || m1 >= OR_MAXN || m2 >= OR_MAXN || kmax >= 2 * OR_MAXN) return -1;
    int deg = m1 + m2 + kmax;
    int G = deg / 2 + 2;
    if (G > OR_MAXG) return -1;
    double x[OR_MAXG], w[OR_MAXG];
    or_gauss_legendre(G, x, w);
    int nP = (m1 > m2 ? m1 : m2);
    if (kmax > nP) nP = kmax;
    nP += 1;
    double P[2 * OR_MAXN + 2], dP[2 * OR_MAXN + 2];
    for (int k = 0; k <= kmax; ++k) {
        or_acc acc = {0.0, 0.0};
        for (int a = 0; a < G; ++a) {
            or_legendre(nP, x[a], P, dP);
            double f = (d1 ? dP[m1] : P[m1]) * (d2 ? dP[m2] : P[m2]);
            acc_add(&acc, w[a] * f * P[k]);
        }
        C[k] = (2.0 * k + 1.0) / 2.0 * (acc.s + acc.c);
    }
    return 0;
}
