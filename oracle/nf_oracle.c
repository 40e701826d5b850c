/*
 * nf_oracle.c -- plain FP64 CPU oracle for the RBF neural-field method of
 * Shaw, Kilpatrick & Avitabile, "Radial Basis Function Techniques for Neural
 * Field Models on Surfaces".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with the
 * CUDA library: no headers, no helpers, no tables.
 *
 * Everything is double precision, compiled without floating-point contraction
 * (-ffp-contract=off), and written for clarity: full loops, textbook LU with
 * partial pivoting, no blocking or fusion.  OpenMP only distributes independent
 * elements / rows over threads; every reduction order is fixed.
 *
 * Contents, in the paper's order:
 *   stencils        §3.1  k nearest nodes to the element centre
 *   RBF-QF (flat)   §3.1-3.2, Eqs. (3.3)-(3.5): PHS r^3 + polynomials, analytic
 *                   integration of the basis over each element, saddle solve,
 *                   accumulation of element weights into node weights
 *   RBF-QF (surface) §3.3, Eq. (3.6): projection points, central projection maps,
 *                   their Jacobians, flat RBF-QF on the projected stencil
 *   nonlocal sum    §2.2, Eq. (2.9): I_i = sum_j w(x_i,x_j) mu_j f(u_j)
 *   time stepping   classical RK4 on Eq. (2.9) (the method of lines of §4)
 *   adjoint         discrete adjoint of that RK4 map (kernel-parameter and
 *                   initial-state gradients of a terminal loss)
 *   manufactured    the manufactured-solution technique of §4, Eq. (4.5), on the
 *   forcing         unit sphere (Funk-Hecke eigenvalues by numerical quadrature)
 *   §5 models       C^4 smooth-step firing rate, synaptic-depression two-field model,
 *                   Adams-Bashforth 5 (started by four RK4 steps)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_MAXK 128
#define OR_MAXP 28  /* (deg+1)(deg+2)/2 for deg <= 6 */

/* Threads of the OpenMP loops (timing only: every result is the same for any count,
 * each output being reduced in a fixed order).  n <= 0 restores the default. */
void or_set_threads(int n) {
#ifdef _OPENMP
    static int dflt = 0;
    if (!dflt) dflt = omp_get_max_threads();
    omp_set_num_threads(n > 0 ? n : dflt);
#else
    (void)n;
#endif
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ================================================================================
 * §3.1 stencils: S(E) = the k nodes nearest to the centre of element E.
 * Centre = centroid ((a+b)+c)/3, distance^2 = sum over coordinates in order,
 * ordering key (distance^2, node index) ascending.
 * ============================================================================== */

static void element_centroid(const double *nodes, int dim, const int32_t *tri, double *c) {
    for (int d = 0; d < dim; ++d) {
        double s = nodes[(int64_t)tri[0] * dim + d] + nodes[(int64_t)tri[1] * dim + d];
        s = s + nodes[(int64_t)tri[2] * dim + d];
        c[d] = s / 3.0;
    }
}

static double dist2(const double *x, const double *c, int dim) {
    double s = 0.0;
    for (int d = 0; d < dim; ++d) {
        double t = x[d] - c[d];
        s = s + t * t;
    }
    return s;
}

/* The k nodes nearest to the point c, in ascending (distance^2, index): every node is
 * compared with the current k-th entry and inserted in order (a full scan). */
static void knn_point(const double *nodes, int64_t n, int dim, const double *c, int k, int32_t *out) {
    double bd[OR_MAXK];
    int32_t bi[OR_MAXK];
    int cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
        double d2 = dist2(nodes + j * dim, c, dim);
        if (cnt == k && !(d2 < bd[k - 1] || (d2 == bd[k - 1] && j < bi[k - 1]))) continue;
        int pos = (cnt < k) ? cnt : k - 1;
        while (pos > 0 && (d2 < bd[pos - 1] || (d2 == bd[pos - 1] && j < bi[pos - 1]))) {
            bd[pos] = bd[pos - 1];
            bi[pos] = bi[pos - 1];
            --pos;
        }
        bd[pos] = d2;
        bi[pos] = (int32_t)j;
        if (cnt < k) ++cnt;
    }
    memcpy(out, bi, sizeof(int32_t) * k);
}

/* elems == NULL: all m elements, output row t = element t.
 * Otherwise: output row t = element elems[t]. */
int or_knn(const double *nodes, int64_t n, int dim, const int32_t *tris, int64_t m,
           const int64_t *elems, int64_t ne, int k, int32_t *stencils) {
    if (k < 1 || k > n || k > OR_MAXK || (dim != 2 && dim != 3)) return -1;
    if (!elems) ne = m;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t t = 0; t < ne; ++t) {
        int64_t e = elems ? elems[t] : t;
        if (e < 0 || e >= m) {
#pragma omp atomic write
            bad = 1;
            continue;
        }
        double c[3];
        element_centroid(nodes, dim, tris + 3 * e, c);
        knn_point(nodes, n, dim, c, k, stencils + t * k);
    }
    return bad ? -1 : 0;
}

/* The same selection around m given centres (m x dim), one output row per centre. */
int or_knn_at(const double *nodes, int64_t n, int dim, const double *centers, int64_t m, int k, int32_t *stencils) {
    if (k < 1 || k > n || k > OR_MAXK || (dim != 2 && dim != 3)) return -1;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t t = 0; t < m; ++t) knn_point(nodes, n, dim, centers + t * dim, k, stencils + t * k);
    return 0;
}

/* ================================================================================
 * §3.2 analytic integration of the basis over a (scaled, planar) triangle.
 * ============================================================================== */

/* d^5 * G(a/d) where G is the antiderivative of sec^5:
 *   G(s) = s (1+s^2)^{3/2} / 4 + 3 s (1+s^2)^{1/2} / 8 + 3 asinh(s) / 8. */
static double sec5_antideriv_scaled(double a, double d) {
    double rr = sqrt(a * a + d * d);
    return 0.25 * d * a * rr * rr * rr + 0.375 * d * d * d * a * rr
         + 0.375 * d * d * d * d * d * asinh(a / d);
}

/* Integral over triangle v (3 x 2, any orientation) of |x - p|^3 dx.
 * Signed fan from p over the three oriented edges; for an edge at distance d from p
 * the polar integral of r^3 * r dr dphi is (d^5/5)[G(phi_B) - G(phi_A)]. */
double or_tri_r3(const double *p, const double *v) {
    double area2 = (v[2] - v[0]) * (v[5] - v[1]) - (v[3] - v[1]) * (v[4] - v[0]);
    double orient = area2 > 0.0 ? 1.0 : -1.0;
    double total = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double *A = v + 2 * e, *B = v + 2 * ((e + 1) % 3);
        double ex = B[0] - A[0], ey = B[1] - A[1];
        double L = sqrt(ex * ex + ey * ey);
        double tx = ex / L, ty = ey / L;
        double ax = A[0] - p[0], ay = A[1] - p[1];
        double cr = ax * ty - ay * tx;        /* cross(A - p, t): sign of sub-triangle (p,A,B) */
        double d = fabs(cr);
        if (d == 0.0) continue;
        double aA = ax * tx + ay * ty;         /* position of A along t from the foot of p */
        double aB = aA + L;
        double part = (sec5_antideriv_scaled(aB, d) - sec5_antideriv_scaled(aA, d)) / 5.0;
        total += (cr > 0.0 ? 1.0 : -1.0) * part;
    }
    return orient * total;
}

static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

/* Integral over triangle v of x^a y^b: expand x = sum_i l_i x_i, y = sum_i l_i y_i in
 * barycentric coordinates and use  int_T l0^i l1^j l2^k = 2|T| i! j! k! / (i+j+k+2)!. */
double or_tri_mono(int a, int b, const double *v) {
    double area = 0.5 * fabs((v[2] - v[0]) * (v[5] - v[1]) - (v[3] - v[1]) * (v[4] - v[0]));
    double total = 0.0;
    for (int i0 = 0; i0 <= a; ++i0)
        for (int i1 = 0; i0 + i1 <= a; ++i1) {
            int i2 = a - i0 - i1;
            double cx = factorial(a) / (factorial(i0) * factorial(i1) * factorial(i2))
                      * pow(v[0], i0) * pow(v[2], i1) * pow(v[4], i2);
            for (int j0 = 0; j0 <= b; ++j0)
                for (int j1 = 0; j0 + j1 <= b; ++j1) {
                    int j2 = b - j0 - j1;
                    double cy = factorial(b) / (factorial(j0) * factorial(j1) * factorial(j2))
                              * pow(v[1], j0) * pow(v[3], j1) * pow(v[5], j2);
                    double mom = 2.0 * area * factorial(i0 + j0) * factorial(i1 + j1)
                               * factorial(i2 + j2) / factorial(a + b + 2);
                    total += cx * cy * mom;
                }
        }
    return total;
}

/* Number of monomials x^a y^b with a + b <= deg. */
static int n_poly(int deg) { return (deg + 1) * (deg + 2) / 2; }

/* Graded ordering: total degree t = 0..deg, then a = t..0 (b = t - a). */
static void poly_exponents(int deg, int *ea, int *eb) {
    int c = 0;
    for (int t = 0; t <= deg; ++t)
        for (int a = t; a >= 0; --a) { ea[c] = a; eb[c] = t - a; ++c; }
}

/* Dense LU with partial pivoting (Doolittle, first maximal pivot), solve in place.
 * Returns 0, or -1 if a pivot falls below tol * ||M||_inf. */
static int lu_solve(int N, double *M, double *x, double tol) {
    double anorm = 0.0;
    for (int r = 0; r < N; ++r) {
        double s = 0.0;
        for (int c = 0; c < N; ++c) s += fabs(M[r * N + c]);
        if (s > anorm) anorm = s;
    }
    for (int c = 0; c < N; ++c) {
        int piv = c;
        double best = fabs(M[c * N + c]);
        for (int r = c + 1; r < N; ++r)
            if (fabs(M[r * N + c]) > best) { best = fabs(M[r * N + c]); piv = r; }
        if (!(best > tol * anorm)) return -1;
        if (piv != c) {
            for (int cc = 0; cc < N; ++cc) {
                double t = M[c * N + cc]; M[c * N + cc] = M[piv * N + cc]; M[piv * N + cc] = t;
            }
            double t = x[c]; x[c] = x[piv]; x[piv] = t;
        }
        for (int r = c + 1; r < N; ++r) {
            double l = M[r * N + c] / M[c * N + c];
            M[r * N + c] = l;
            for (int cc = c + 1; cc < N; ++cc) M[r * N + cc] -= l * M[c * N + cc];
            x[r] -= l * x[c];
        }
    }
    for (int r = N - 1; r >= 0; --r) {
        double s = x[r];
        for (int cc = r + 1; cc < N; ++cc) s -= M[r * N + cc] * x[cc];
        x[r] = s / M[r * N + r];
    }
    return 0;
}

#define OR_PIVOT_TOL 1e-14

/* RBF-QF weights of one planar element (§3.2, Eq. (3.5)), in scaled local coordinates.
 * xi: k x 2 stencil points, tri: 3 x 2 triangle vertices, deg: appended polynomial
 * degree.  Interpolation matrix of Eq. (3.4): A_rs = |xi_r - xi_s|^3,
 * Pi_{r,alpha} = xi_r^alpha; right-hand side: integrals of each basis function over
 * the triangle.  The matrix is symmetric, so w_E = M^{-1} [L phi; L pi] is the
 * solution of M z = [L phi; L pi]; its first k entries are the element weights. */
int or_element_weights_local(const double *xi, int k, const double *tri, int deg, double *w) {
    int P = n_poly(deg);
    int N = k + P;
    int ea[OR_MAXP], eb[OR_MAXP];
    if (k > OR_MAXK || P > OR_MAXP) return -2;
    poly_exponents(deg, ea, eb);
    double *M = (double *)calloc((size_t)N * N, sizeof(double));
    double *z = (double *)calloc((size_t)N, sizeof(double));
    for (int r = 0; r < k; ++r) {
        for (int s = 0; s < k; ++s) {
            double dx = xi[2 * r] - xi[2 * s], dy = xi[2 * r + 1] - xi[2 * s + 1];
            double rr = sqrt(dx * dx + dy * dy);
            M[r * N + s] = rr * rr * rr;
        }
        for (int a = 0; a < P; ++a) {
            double pv = pow(xi[2 * r], ea[a]) * pow(xi[2 * r + 1], eb[a]);
            M[r * N + k + a] = pv;
            M[(k + a) * N + r] = pv;
        }
        z[r] = or_tri_r3(xi + 2 * r, tri);
    }
    for (int a = 0; a < P; ++a) z[k + a] = or_tri_mono(ea[a], eb[a], tri);
    int st = lu_solve(N, M, z, OR_PIVOT_TOL);
    if (st == 0) memcpy(w, z, sizeof(double) * k);
    free(M);
    free(z);
    return st;
}

/* ================================================================================
 * §3.3 surfaces: projection points, central projection, Jacobian of mu_j.
 * ============================================================================== */

static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* Unit normal of flat triangle e, oriented to agree with the mean of its vertex normals. */
static void tri_normal(const double *X, const double *NS, const int32_t *tri, double *nE) {
    const double *a = X + 3 * (int64_t)tri[0], *b = X + 3 * (int64_t)tri[1], *c = X + 3 * (int64_t)tri[2];
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    cross3(u, v, nE);
    double l = norm3(nE);
    for (int d = 0; d < 3; ++d) nE[d] /= l;
    double ref[3];
    for (int d = 0; d < 3; ++d)
        ref[d] = NS[3 * (int64_t)tri[0] + d] + NS[3 * (int64_t)tri[1] + d] + NS[3 * (int64_t)tri[2] + d];
    if (dot3(nE, ref) < 0.0)
        for (int d = 0; d < 3; ++d) nE[d] = -nE[d];
}

/* 3 x 3 solve by Gaussian elimination with partial pivoting; returns the infinity-norm
 * condition number estimate ||A|| ||A^{-1}|| (INFINITY if singular). */
static double solve3(const double *A_in, const double *b_in, double *x) {
    double A[9], Ainv[9];
    double anorm = 0.0;
    for (int r = 0; r < 3; ++r) {
        double s = fabs(A_in[3 * r]) + fabs(A_in[3 * r + 1]) + fabs(A_in[3 * r + 2]);
        if (s > anorm) anorm = s;
    }
    /* inverse by Gauss-Jordan on [A | I] */
    double W[18];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 6; ++c) W[6 * r + c] = (c < 3) ? A_in[3 * r + c] : (c - 3 == r ? 1.0 : 0.0);
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(W[6 * r + c]) > fabs(W[6 * piv + c])) piv = r;
        if (W[6 * piv + c] == 0.0) return INFINITY;
        if (piv != c)
            for (int cc = 0; cc < 6; ++cc) { double t = W[6 * c + cc]; W[6 * c + cc] = W[6 * piv + cc]; W[6 * piv + cc] = t; }
        double pv = W[6 * c + c];
        for (int cc = 0; cc < 6; ++cc) W[6 * c + cc] /= pv;
        for (int r = 0; r < 3; ++r) {
            if (r == c) continue;
            double l = W[6 * r + c];
            for (int cc = 0; cc < 6; ++cc) W[6 * r + cc] -= l * W[6 * c + cc];
        }
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Ainv[3 * r + c] = W[6 * r + 3 + c];
    double inorm = 0.0;
    for (int r = 0; r < 3; ++r) {
        double s = fabs(Ainv[3 * r]) + fabs(Ainv[3 * r + 1]) + fabs(Ainv[3 * r + 2]);
        if (s > inorm) inorm = s;
    }
    for (int r = 0; r < 3; ++r) x[r] = Ainv[3 * r] * b_in[0] + Ainv[3 * r + 1] * b_in[1] + Ainv[3 * r + 2] * b_in[2];
    (void)A;
    return anorm * inorm;
}

#define OR_PROJ_COND_MAX 1e10

/* Edge-adjacency: nbr[3e + k] = element sharing edge (tri[k], tri[(k+1)%3]) of e, or -1.
 * Plain O(m log m) edge sort. */
typedef struct { int32_t lo, hi; int64_t e; int k; } or_edge;
static int edge_cmp(const void *pa, const void *pb) {
    const or_edge *a = (const or_edge *)pa, *b = (const or_edge *)pb;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
    if (a->e != b->e) return a->e < b->e ? -1 : 1;
    return 0;
}
int or_tri_neighbors(const int32_t *tris, int64_t m, int64_t *nbr) {
    or_edge *E = (or_edge *)malloc(sizeof(or_edge) * (size_t)(3 * m));
    for (int64_t e = 0; e < m; ++e)
        for (int k = 0; k < 3; ++k) {
            int32_t a = tris[3 * e + k], b = tris[3 * e + (k + 1) % 3];
            or_edge x = {a < b ? a : b, a < b ? b : a, e, k};
            E[3 * e + k] = x;
            nbr[3 * e + k] = -1;
        }
    qsort(E, (size_t)(3 * m), sizeof(or_edge), edge_cmp);
    int nonmanifold = 0;
    for (int64_t i = 0; i < 3 * m;) {
        int64_t j = i + 1;
        while (j < 3 * m && E[j].lo == E[i].lo && E[j].hi == E[i].hi) ++j;
        if (j - i == 2) {
            nbr[3 * E[i].e + E[i].k] = E[i + 1].e;
            nbr[3 * E[i + 1].e + E[i + 1].k] = E[i].e;
        } else if (j - i > 2) {
            nonmanifold = 1;
        }
        i = j;
    }
    free(E);
    return nonmanifold ? -1 : 0;
}

/* Projection point p_E (§3.3): intersection of the three cutting planes, one per edge
 * (a, b) shared with neighbour E'.  Each cutting plane contains the edge and is
 * orthogonal to n_E - n_E', i.e. (p - a).(n_E - n_E') = 0.  Returns 1 and p when the
 * 3 x 3 system is well conditioned, 0 otherwise (then a parallel projection along n_E
 * is used: the limit of p at infinity). */
int or_projection_point(const double *X, const double *NS, const int32_t *tris, const int64_t *nbr,
                        int64_t e, double *p) {
    double nE[3], A[9], rhs[3];
    tri_normal(X, NS, tris + 3 * e, nE);
    for (int k = 0; k < 3; ++k) {
        int64_t f = nbr[3 * e + k];
        if (f < 0) return 0;
        double nF[3];
        tri_normal(X, NS, tris + 3 * f, nF);
        const double *a = X + 3 * (int64_t)tris[3 * e + k];
        for (int d = 0; d < 3; ++d) A[3 * k + d] = nE[d] - nF[d];
        rhs[k] = dot3(A + 3 * k, a);
    }
    double cond = solve3(A, rhs, p);
    return (isfinite(cond) && cond < OR_PROJ_COND_MAX) ? 1 : 0;
}

/* Element weights on a surface (§3.3): map the stencil to the plane of E by the
 * inverse of mu_E (central projection through p_E, or parallel projection along n_E),
 * apply flat RBF-QF there, and multiply each weight by the Jacobian of mu_E at the
 * projected node (the area factor of Eq. (3.6)):
 *   J = (|x - p|^2 / |xi - p|^2) |n_E . u| / |n_S(x) . u|,  u = (x - p)/|x - p|,
 *   parallel case J = 1 / |n_S(x) . n_E|.
 * Output w_out[k] (weights including J); jac_out (optional) the Jacobians. */
int or_surface_element_weights(const double *X, const double *NS, const int32_t *tris, const int64_t *nbr,
                               int64_t e, const int32_t *sten, int k, int deg,
                               double *w_out, double *jac_out, int *central_out) {
    const int32_t *tri = tris + 3 * e;
    const double *a = X + 3 * (int64_t)tri[0], *b = X + 3 * (int64_t)tri[1], *c = X + 3 * (int64_t)tri[2];
    double nE[3], cE[3], p[3], e1[3], e2[3];
    tri_normal(X, NS, tri, nE);
    for (int d = 0; d < 3; ++d) cE[d] = ((a[d] + b[d]) + c[d]) / 3.0;
    int central = or_projection_point(X, NS, tris, nbr, e, p);
    for (int d = 0; d < 3; ++d) e1[d] = b[d] - a[d];
    double l1 = norm3(e1);
    for (int d = 0; d < 3; ++d) e1[d] /= l1;
    cross3(nE, e1, e2);
    double xi3[OR_MAXK * 3], jac[OR_MAXK];
    for (int r = 0; r < k; ++r) {
        const double *x = X + 3 * (int64_t)sten[r];
        const double *ns = NS + 3 * (int64_t)sten[r];
        if (central) {
            double xp[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
            double cp[3] = {cE[0] - p[0], cE[1] - p[1], cE[2] - p[2]};
            double t = dot3(cp, nE) / dot3(xp, nE);
            double lx = norm3(xp);
            double u[3] = {xp[0] / lx, xp[1] / lx, xp[2] / lx};
            for (int d = 0; d < 3; ++d) xi3[3 * r + d] = p[d] + t * xp[d];
            jac[r] = (1.0 / (t * t)) * fabs(dot3(nE, u)) / fabs(dot3(ns, u));
        } else {
            double s = (x[0] - cE[0]) * nE[0] + (x[1] - cE[1]) * nE[1] + (x[2] - cE[2]) * nE[2];
            for (int d = 0; d < 3; ++d) xi3[3 * r + d] = x[d] - s * nE[d];
            jac[r] = 1.0 / fabs(dot3(ns, nE));
        }
    }
    double rho = 0.0;
    for (int r = 0; r < k; ++r) {
        double v[3] = {xi3[3 * r] - cE[0], xi3[3 * r + 1] - cE[1], xi3[3 * r + 2] - cE[2]};
        double l = norm3(v);
        if (l > rho) rho = l;
    }
    double xi[OR_MAXK * 2], tv[6];
    for (int r = 0; r < k; ++r) {
        double v[3] = {xi3[3 * r] - cE[0], xi3[3 * r + 1] - cE[1], xi3[3 * r + 2] - cE[2]};
        xi[2 * r] = dot3(v, e1) / rho;
        xi[2 * r + 1] = dot3(v, e2) / rho;
    }
    const double *vv[3] = {a, b, c};
    for (int i = 0; i < 3; ++i) {
        double v[3] = {vv[i][0] - cE[0], vv[i][1] - cE[1], vv[i][2] - cE[2]};
        tv[2 * i] = dot3(v, e1) / rho;
        tv[2 * i + 1] = dot3(v, e2) / rho;
    }
    double wl[OR_MAXK];
    int st = or_element_weights_local(xi, k, tv, deg, wl);
    if (st != 0) return st;
    for (int r = 0; r < k; ++r) w_out[r] = wl[r] * rho * rho * jac[r];
    if (jac_out) memcpy(jac_out, jac, sizeof(double) * k);
    if (central_out) *central_out = central;
    return 0;
}

/* Element weights on a flat domain (dim 2): local frame centred at the centroid,
 * scaled by rho = max stencil distance; weights scale back by rho^2. */
int or_flat_element_weights(const double *X2, const int32_t *tris, int64_t e, const int32_t *sten,
                            int k, int deg, double *w_out) {
    const int32_t *tri = tris + 3 * e;
    double cE[2];
    for (int d = 0; d < 2; ++d)
        cE[d] = ((X2[2 * (int64_t)tri[0] + d] + X2[2 * (int64_t)tri[1] + d]) + X2[2 * (int64_t)tri[2] + d]) / 3.0;
    double rho = 0.0;
    for (int r = 0; r < k; ++r) {
        double dx = X2[2 * (int64_t)sten[r]] - cE[0], dy = X2[2 * (int64_t)sten[r] + 1] - cE[1];
        double l = sqrt(dx * dx + dy * dy);
        if (l > rho) rho = l;
    }
    double xi[OR_MAXK * 2], tv[6];
    for (int r = 0; r < k; ++r) {
        xi[2 * r] = (X2[2 * (int64_t)sten[r]] - cE[0]) / rho;
        xi[2 * r + 1] = (X2[2 * (int64_t)sten[r] + 1] - cE[1]) / rho;
    }
    for (int i = 0; i < 3; ++i) {
        tv[2 * i] = (X2[2 * (int64_t)tri[i]] - cE[0]) / rho;
        tv[2 * i + 1] = (X2[2 * (int64_t)tri[i] + 1] - cE[1]) / rho;
    }
    double wl[OR_MAXK];
    int st = or_element_weights_local(xi, k, tv, deg, wl);
    if (st != 0) return st;
    for (int r = 0; r < k; ++r) w_out[r] = wl[r] * rho * rho;
    return 0;
}

/* Quadrature weights (§3.2 Eq. (3.5), §3.3): per element weights, then
 *   q_i = sum over (E, r) with S(E)_r = i of w_E[r],  summed in (E, r) ascending order.
 * X: n x dim; NS: n x 3 normals (surfaces) or NULL (dim 2).  elem_w (optional, m x k)
 * receives the element weights.  Returns 0, -1 on bad arguments, or 1 + the first
 * singular element index in *bad. */
int or_quad_weights(const double *X, const double *NS, int64_t n, int dim, const int32_t *tris, int64_t m,
                    const int32_t *stencils, int k, int deg, double *q, double *elem_w, int64_t *bad) {
    if ((dim == 3) != (NS != NULL) || k > OR_MAXK || n_poly(deg) > k) return -1;
    double *W = elem_w ? elem_w : (double *)malloc(sizeof(double) * (size_t)(m * k));
    int64_t *nbr = NULL;
    if (dim == 3) {
        nbr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(3 * m));
        or_tri_neighbors(tris, m, nbr);
    }
    int64_t first_bad = -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < m; ++e) {
        int st = (dim == 3)
            ? or_surface_element_weights(X, NS, tris, nbr, e, stencils + e * k, k, deg, W + e * k, NULL, NULL)
            : or_flat_element_weights(X, tris, e, stencils + e * k, k, deg, W + e * k);
        if (st != 0) {
#pragma omp critical
            { if (first_bad < 0 || e < first_bad) first_bad = e; }
        }
    }
    int rc = 0;
    if (first_bad >= 0) {
        rc = 1;
    } else {
        for (int64_t i = 0; i < n; ++i) q[i] = 0.0;
        for (int64_t e = 0; e < m; ++e)
            for (int r = 0; r < k; ++r) q[stencils[e * k + r]] += W[e * k + r];
    }
    if (bad) *bad = first_bad;
    if (!elem_w) free(W);
    free(nbr);
    return rc;
}

/* ================================================================================
 * §2.2 Eq. (2.9): the fully discrete nonlocal sum and the neural-field vector field.
 * Kernel: Mexican hat w(r) = A1 exp(-r^2/s1^2) - A2 exp(-r^2/s2^2) (Euclidean r).
 * Firing rate (§4, Eq. (4.4)): f(u) = 1 / (1 + exp(-beta (u - theta))).
 * ============================================================================== */

typedef struct { double A1, s1, A2, s2, period; } or_kernel;

static double kernel_w(const or_kernel *kp, double r2) {
    return kp->A1 * exp(-r2 / (kp->s1 * kp->s1)) - kp->A2 * exp(-r2 / (kp->s2 * kp->s2));
}
static double firing(double u, double beta, double theta) { return 1.0 / (1.0 + exp(-beta * (u - theta))); }

/* Squared distance.  period = 0: Euclidean.  period = L > 0: the doubly periodic distance of
 * §4, Eq. (dist), on the flat square of side L (z = 0): the minimum over the nine shifts
 * x - y + L (i, j), i, j in {-1, 0, 1}. */
static double dist2p(double dx, double dy, double dz, double period) {
    if (period <= 0.0) return dx * dx + dy * dy + dz * dz;
    double best = -1.0;
    for (int i = -1; i <= 1; ++i)
        for (int j = -1; j <= 1; ++j) {
            double ex = dx + period * i, ey = dy + period * j;
            double d = ex * ex + ey * ey + dz * dz;
            if (best < 0.0 || d < best) best = d;
        }
    return best;
}
static double pair_r2p(const double *X, int64_t i, int64_t j, double period) {
    return dist2p(X[3 * i] - X[3 * j], X[3 * i + 1] - X[3 * j + 1], X[3 * i + 2] - X[3 * j + 2], period);
}

/* I[b, rows[t]] = sum_j w(|x_i - x_j|) q_j f_b(u[b, j]).  X: n x 3.
 * rows == NULL: all rows, output I is B x n.  Otherwise output is B x nrows. */
void or_nonlocal(const double *X, const double *q, int64_t n, const double *u, int B, const double *kpar,
                 const double *beta, const double *theta, const int64_t *rows, int64_t nrows, double *I) {
    or_kernel kp = {kpar[0], kpar[1], kpar[2], kpar[3], kpar[4]};
    if (!rows) nrows = n;
    double *g = (double *)malloc(sizeof(double) * (size_t)(n * B));
    for (int b = 0; b < B; ++b)
        for (int64_t j = 0; j < n; ++j) g[b * n + j] = q[j] * firing(u[b * n + j], beta[b], theta[b]);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows ? rows[t] : t;
        for (int b = 0; b < B; ++b) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += kernel_w(&kp, pair_r2p(X, i, j, kp.period)) * g[b * n + j];
            I[b * nrows + t] = s;
        }
    }
    free(g);
}

/* ---------------------------------------------------------------------------------
 * Forcing gamma(t) of Eq. (2.9).  kind 0: none.  kind 1: manufactured solution on the
 * unit sphere (the technique of §4, Eq. (4.5)):
 *   f(u*) = z = c + a(t) Y(x),  a(t) = a0 cos t,  Y = Y1 + Y2,  Y1 = z/2 (degree 1),
 *   Y2 = x y (degree 2);   u* = theta + ln(z / (1 - z)) / beta.
 * Funk-Hecke: int_{S^2} w(|x-y|) Y_l(y) dS = lambda_l Y_l(x), so
 *   gamma = d/dt u* + u* - [lambda_0 c + a(t) (lambda_1 Y1 + lambda_2 Y2)].
 * --------------------------------------------------------------------------------- */
typedef struct {
    int kind;
    double c, a0, lam0, lam1, lam2;   /* kind 1 */
    double radius, sigma, scale;       /* kind 2 */
} or_forcing;

static void gauss_legendre(int N, double *x, double *w);

/* ---------------------------------------------------------------------------------
 * Forcing kind 2: the manufactured solution of the convergence study on the square (§4.3),
 * on the doubly periodic square of side L (the kernel's period), coordinates (x, y):
 *   z(t, x) = G(x, x0(t); sigma) + c,  x0(t) = radius (cos t, sin t),
 *   G(x, y; s) = exp(-dist^2(x, y) / (2 s^2)) / (2 pi s^2)   (dist: Eq. (dist)),
 *   u*(t, x) = theta + ln(z / (1 - z)) / beta,  so that f(u*) = z,
 *   gamma = d(u*)/dt + u* - scale * C(t, x),  C = int over one period cell of w(dist(x, y)) z(t, y) dy.
 * scale = 1 on the square.  On the torus of §4.4 the kernel is divided by R + r cos(theta)
 * of the source point and the surface element is r (R + r cos theta) dphi dtheta, which
 * leaves the same integral over the (phi, theta) square times scale = r.
 * d(u*)/dt = (dz/dt) / (beta z (1 - z)), dz/dt = G (x - x0) . x0'(t) / sigma^2 with the
 * minimum-image displacement x - x0.
 * C by quadrature over the displacement d = x - y, which runs over the square
 * [-L/2, L/2]^2 as y runs over a cell (so w(dist) = w(|d|)).  Where the kernel is negligible
 * (beyond 8 of its standard deviations) the square is cut down to that window.  z(x - d) is
 * smooth except on the lines where its nearest image of x0 changes (x - d - x0 = L/2 + kL in
 * a coordinate); those lines split the window into panels, each integrated by a 40 x 40
 * Gauss-Legendre product rule. */
static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

static double gauss2(double dx, double dy, double s) {
    return exp(-(dx * dx + dy * dy) / (2.0 * s * s)) / (2.0 * M_PI * s * s);
}

/* Breakpoints of one displacement coordinate: window ends and the cut points in between. */
static int conv_breaks(double xc, double x0c, double h, double L, double *bp) {
    int nb = 0;
    bp[nb++] = -h;
    for (int k = -3; k <= 3; ++k) {
        double d = xc - x0c - 0.5 * L - k * L;
        if (d > -h && d < h) bp[nb++] = d;
    }
    bp[nb++] = h;
    for (int i = 1; i < nb; ++i)  /* sort (at most a few entries) */
        for (int j = i; j > 0 && bp[j] < bp[j - 1]; --j) {
            double t = bp[j]; bp[j] = bp[j - 1]; bp[j - 1] = t;
        }
    return nb;
}

static double conv_window(const or_kernel *kp, double x, double y, double x0, double y0, double sigma, double c) {
    enum { NGL = 40 };
    static double gx[NGL], gw[NGL];
    static int init = 0;
    if (!init) {
#pragma omp critical(or_gl_init)
        {
            if (!init) { gauss_legendre(NGL, gx, gw); init = 1; }
        }
    }
    const double L = kp->period;
    double sd = kp->s1 / sqrt(2.0);
    if (kp->A2 != 0.0 && kp->s2 / sqrt(2.0) > sd) sd = kp->s2 / sqrt(2.0);
    double h = 8.0 * sd;
    if (h > 0.5 * L) h = 0.5 * L;
    double bx[10], by[10];
    int nbx = conv_breaks(x, x0, h, L, bx), nby = conv_breaks(y, y0, h, L, by);
    double acc = 0.0;
    for (int px = 0; px + 1 < nbx; ++px)
        for (int py = 0; py + 1 < nby; ++py) {
            double ax = bx[px], hx = 0.5 * (bx[px + 1] - ax), ay = by[py], hy = 0.5 * (by[py + 1] - ay);
            for (int i = 0; i < NGL; ++i) {
                double dx = ax + hx * (gx[i] + 1.0);
                for (int j = 0; j < NGL; ++j) {
                    double dy = ay + hy * (gx[j] + 1.0);
                    double w = kernel_w(kp, dx * dx + dy * dy);
                    double z = gauss2(min_image(x - dx - x0, L), min_image(y - dy - y0, L), sigma) + c;
                    acc += hx * hy * gw[i] * gw[j] * w * z;
                }
            }
        }
    return acc;
}

/* u*(t, x) and gamma of kind 2 at one node (x, y). */
static void mms_flat_point(const or_forcing *F, const or_kernel *kp, double x, double y, double t, double beta,
                           double theta, double *us, double *gam) {
    const double L = kp->period, s = F->sigma;
    double x0 = F->radius * cos(t), y0 = F->radius * sin(t);
    double dx = min_image(x - x0, L), dy = min_image(y - y0, L);
    double G = gauss2(dx, dy, s), z = G + F->c;
    double dz = G * (dx * (-F->radius * sin(t)) + dy * (F->radius * cos(t))) / (s * s);
    *us = theta + log(z / (1.0 - z)) / beta;
    if (gam) *gam = dz / (beta * z * (1.0 - z)) + *us - F->scale * conv_window(kp, x, y, x0, y0, s, F->c);
}

void or_mms_flat_solution(const double *X, int64_t n, double t, const double *kpar, double radius, double sigma,
                          double c, double beta, double theta, double *u) {
    or_kernel kp = {kpar[0], kpar[1], kpar[2], kpar[3], kpar[4]};
    or_forcing F = {2, c, 0, 0, 0, 0, radius, sigma, 1.0};
    for (int64_t i = 0; i < n; ++i) mms_flat_point(&F, &kp, X[3 * i], X[3 * i + 1], t, beta, theta, &u[i], NULL);
}

void or_mms_flat_forcing(const double *X, int64_t n, double t, const double *kpar, double radius, double sigma,
                         double c, double scale, double beta, double theta, double *gam) {
    or_kernel kp = {kpar[0], kpar[1], kpar[2], kpar[3], kpar[4]};
    or_forcing F = {2, c, 0, 0, 0, 0, radius, sigma, scale};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double us;
        mms_flat_point(&F, &kp, X[3 * i], X[3 * i + 1], t, beta, theta, &us, &gam[i]);
    }
}

static void forcing_eval(const or_forcing *F, const or_kernel *kp, const double *X, int64_t n, double t, double beta,
                         double theta, double *gam) {
    if (!F || F->kind == 0) {
        for (int64_t i = 0; i < n; ++i) gam[i] = 0.0;
        return;
    }
    if (F->kind == 2) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double us;
            mms_flat_point(F, kp, X[3 * i], X[3 * i + 1], t, beta, theta, &us, &gam[i]);
        }
        return;
    }
    double a = F->a0 * cos(t), da = -F->a0 * sin(t);
    for (int64_t i = 0; i < n; ++i) {
        double Y1 = 0.5 * X[3 * i + 2], Y2 = X[3 * i] * X[3 * i + 1];
        double Y = Y1 + Y2;
        double z = F->c + a * Y;
        double us = theta + log(z / (1.0 - z)) / beta;
        double dus = da * Y / (beta * z * (1.0 - z));
        gam[i] = dus + us - (F->lam0 * F->c + a * (F->lam1 * Y1 + F->lam2 * Y2));
    }
}

/* Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_N. */
static void gauss_legendre(int N, double *x, double *w) {
    for (int i = 0; i < N; ++i) {
        double z = cos(M_PI * (i + 0.75) / (N + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= N; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
            dp = N * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Funk-Hecke eigenvalues lambda_l = 2 pi int_{-1}^{1} w(sqrt(2 - 2t)) P_l(t) dt, l = 0,1,2,
 * by composite Gauss-Legendre quadrature (panels refined toward t = 1 where the
 * Gaussians concentrate). */
void or_mms_sphere_eigs(const double *kpar, double *lam) {
    or_kernel kp = {kpar[0], kpar[1], kpar[2], kpar[3], kpar[4]};
    enum { NG = 20, NPAN = 400 };
    double gx[NG], gw[NG];
    gauss_legendre(NG, gx, gw);
    double s[3] = {0, 0, 0};
    /* panels on u = 1 - t in [0, 2], geometrically graded near u = 0 */
    double edges[NPAN + 1];
    edges[0] = 0.0;
    for (int p = 1; p <= NPAN; ++p) edges[p] = 2.0 * pow((double)p / NPAN, 3.0);
    for (int p = 0; p < NPAN; ++p) {
        double lo = edges[p], hi = edges[p + 1], h = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
        for (int g = 0; g < NG; ++g) {
            double uu = mid + h * gx[g];
            double t = 1.0 - uu;
            double wr = kernel_w(&kp, 2.0 * uu);
            double P[3] = {1.0, t, 0.5 * (3.0 * t * t - 1.0)};
            for (int l = 0; l < 3; ++l) s[l] += h * gw[g] * wr * P[l];
        }
    }
    for (int l = 0; l < 3; ++l) lam[l] = 2.0 * M_PI * s[l];
}

/* Manufactured solution u*(t, x) on the unit sphere (for error measurement). */
void or_mms_sphere_solution(const double *X, int64_t n, double t, double c, double a0, double beta, double theta,
                            double *u) {
    double a = a0 * cos(t);
    for (int64_t i = 0; i < n; ++i) {
        double Y = 0.5 * X[3 * i + 2] + X[3 * i] * X[3 * i + 1];
        double z = c + a * Y;
        u[i] = theta + log(z / (1.0 - z)) / beta;
    }
}

/* Vector field N(t, U) = -U + I(U) + gamma(t) for B trajectories. */
static void vector_field(const double *X, const double *q, int64_t n, const double *U, int B, const double *kpar,
                         const double *beta, const double *theta, const or_forcing *F, double t, double *K) {
    or_nonlocal(X, q, n, U, B, kpar, beta, theta, NULL, 0, K);
    double *gam = (double *)malloc(sizeof(double) * (size_t)n);
    for (int b = 0; b < B; ++b) {
        or_kernel kp = {kpar[0], kpar[1], kpar[2], kpar[3], kpar[4]};
        forcing_eval(F, &kp, X, n, t, beta[b], theta[b], gam);
        for (int64_t i = 0; i < n; ++i) K[b * n + i] = -U[b * n + i] + K[b * n + i] + gam[i];
    }
    free(gam);
}

/* Classical RK4 for Eq. (2.9):
 *   k1 = N(t, u), k2 = N(t + dt/2, u + dt/2 k1), k3 = N(t + dt/2, u + dt/2 k2),
 *   k4 = N(t + dt, u + dt k3),  u <- u + dt/6 (k1 + 2 k2 + 2 k3 + k4).
 * u: B x n in/out.  stages (optional): nsteps x 4 x B x n stage inputs U_s. */
void or_rk4(const double *X, const double *q, int64_t n, double *u, int B, double t0, double dt, int nsteps,
            const double *kpar, const double *beta, const double *theta, const double *forcing,
            double *stages) {
    or_forcing F = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (forcing) {
        F.kind = (int)forcing[0];
        if (F.kind == 2) { F.c = forcing[1]; F.radius = forcing[2]; F.sigma = forcing[3]; F.scale = forcing[4]; }
        else { F.c = forcing[1]; F.a0 = forcing[2]; F.lam0 = forcing[3]; F.lam1 = forcing[4]; F.lam2 = forcing[5]; }
    }
    size_t sz = (size_t)(n * B);
    double *k1 = malloc(sizeof(double) * sz), *k2 = malloc(sizeof(double) * sz), *k3 = malloc(sizeof(double) * sz),
           *k4 = malloc(sizeof(double) * sz), *U = malloc(sizeof(double) * sz);
    for (int s = 0; s < nsteps; ++s) {
        double t = t0 + s * dt;
        double *st = stages ? stages + (size_t)s * 4 * sz : NULL;
        if (st) memcpy(st, u, sizeof(double) * sz);
        vector_field(X, q, n, u, B, kpar, beta, theta, &F, t, k1);
        for (size_t i = 0; i < sz; ++i) U[i] = u[i] + 0.5 * dt * k1[i];
        if (st) memcpy(st + sz, U, sizeof(double) * sz);
        vector_field(X, q, n, U, B, kpar, beta, theta, &F, t + 0.5 * dt, k2);
        for (size_t i = 0; i < sz; ++i) U[i] = u[i] + 0.5 * dt * k2[i];
        if (st) memcpy(st + 2 * sz, U, sizeof(double) * sz);
        vector_field(X, q, n, U, B, kpar, beta, theta, &F, t + 0.5 * dt, k3);
        for (size_t i = 0; i < sz; ++i) U[i] = u[i] + dt * k3[i];
        if (st) memcpy(st + 3 * sz, U, sizeof(double) * sz);
        vector_field(X, q, n, U, B, kpar, beta, theta, &F, t + dt, k4);
        for (size_t i = 0; i < sz; ++i) u[i] = u[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    free(k1); free(k2); free(k3); free(k4); free(U);
}

/* ================================================================================
 * Discrete adjoint of the RK4 map above.
 * For a loss L(u_N) with lambda_N = dL/du_N, one step backwards, with b = (1,2,2,1)/6:
 *   nu4 = dt b4 lam;              mu4 = J(U4)^T nu4
 *   nu3 = dt b3 lam + dt mu4;     mu3 = J(U3)^T nu3
 *   nu2 = dt b2 lam + dt/2 mu3;   mu2 = J(U2)^T nu2
 *   nu1 = dt b1 lam + dt/2 mu2;   mu1 = J(U1)^T nu1
 *   lam <- lam + mu1 + mu2 + mu3 + mu4
 * with J(U)^T nu = -nu + q o f'(U) o (W^T nu) and W symmetric (w is radial, §4 Eq. (4.2)
 * context), f' = beta f (1 - f).  Kernel-parameter gradients accumulate
 *   dL/dtheta += sum_s < nu_s, (d_theta W) (q o f(U_s)) >,
 *   d w/dA1 = e1, d w/ds1 = 2 A1 r^2 e1 / s1^3, d w/dA2 = -e2, d w/ds2 = -2 A2 r^2 e2 / s2^3.
 * Forcing (kind 1) depends on theta/beta only, not on kernel parameters.
 * lam_T: B x n, grad_u0: B x n, grad_k: B x 4.
 * ============================================================================== */
static void adj_stage(const double *X, const double *q, int64_t n, const double *U, const double *nu, int B,
                      const double *kpar, const double *beta, const double *theta, double *mu, double *gk) {
    or_kernel kp = {kpar[0], kpar[1], kpar[2], kpar[3], kpar[4]};
    double is1 = 1.0 / (kp.s1 * kp.s1), is2 = 1.0 / (kp.s2 * kp.s2);
    double *g = malloc(sizeof(double) * (size_t)n), *fp = malloc(sizeof(double) * (size_t)n);
    for (int b = 0; b < B; ++b) {
        for (int64_t j = 0; j < n; ++j) {
            double f = firing(U[b * n + j], beta[b], theta[b]);
            g[j] = q[j] * f;
            fp[j] = q[j] * beta[b] * f * (1.0 - f);
        }
        double tA1 = 0, tS1 = 0, tA2 = 0, tS2 = 0;
#pragma omp parallel for schedule(static) reduction(+ : tA1, tS1, tA2, tS2)
        for (int64_t i = 0; i < n; ++i) {
            double Wnu = 0, E1 = 0, R1 = 0, E2 = 0, R2 = 0;
            for (int64_t j = 0; j < n; ++j) {
                double r2 = pair_r2p(X, i, j, kp.period);
                double e1 = exp(-r2 * is1), e2 = exp(-r2 * is2);
                Wnu += (kp.A1 * e1 - kp.A2 * e2) * nu[b * n + j];
                E1 += e1 * g[j];
                R1 += r2 * e1 * g[j];
                E2 += e2 * g[j];
                R2 += r2 * e2 * g[j];
            }
            mu[b * n + i] = -nu[b * n + i] + fp[i] * Wnu;
            double v = nu[b * n + i];
            tA1 += v * E1;
            tS1 += v * 2.0 * kp.A1 * R1 / (kp.s1 * kp.s1 * kp.s1);
            tA2 += v * (-E2);
            tS2 += v * (-2.0 * kp.A2 * R2 / (kp.s2 * kp.s2 * kp.s2));
        }
        gk[4 * b + 0] += tA1;
        gk[4 * b + 1] += tS1;
        gk[4 * b + 2] += tA2;
        gk[4 * b + 3] += tS2;
    }
    free(g);
    free(fp);
}

void or_adjoint(const double *X, const double *q, int64_t n, const double *u0, int B, double t0, double dt,
                int nsteps, const double *kpar, const double *beta, const double *theta, const double *forcing,
                const double *lam_T, double *grad_u0, double *grad_k) {
    size_t sz = (size_t)(n * B);
    double *stages = malloc(sizeof(double) * sz * 4 * (size_t)nsteps);
    double *u = malloc(sizeof(double) * sz);
    memcpy(u, u0, sizeof(double) * sz);
    or_rk4(X, q, n, u, B, t0, dt, nsteps, kpar, beta, theta, forcing, stages);
    double *lam = grad_u0, *nu = malloc(sizeof(double) * sz), *mu = malloc(sizeof(double) * sz),
           *acc = malloc(sizeof(double) * sz);
    memcpy(lam, lam_T, sizeof(double) * sz);
    memset(grad_k, 0, sizeof(double) * 4 * B);
    const double bw[4] = {1.0 / 6.0, 2.0 / 6.0, 2.0 / 6.0, 1.0 / 6.0};
    const double cprev[4] = {0.0, 0.5, 0.5, 1.0}; /* U_s = u + cprev[s] dt k_{s-1} */
    for (int s = nsteps - 1; s >= 0; --s) {
        const double *st = stages + (size_t)s * 4 * sz;
        memset(acc, 0, sizeof(double) * sz);
        for (int i = 0; i < (int)sz; ++i) mu[i] = 0.0;
        for (int stg = 3; stg >= 0; --stg) {
            /* nu_stg = dt b_stg lam + cprev[stg+1] dt mu_{stg+1} */
            for (size_t i = 0; i < sz; ++i)
                nu[i] = dt * bw[stg] * lam[i] + (stg < 3 ? cprev[stg + 1] * dt * mu[i] : 0.0);
            adj_stage(X, q, n, st + (size_t)stg * sz, nu, B, kpar, beta, theta, mu, grad_k);
            for (size_t i = 0; i < sz; ++i) acc[i] += mu[i];
        }
        for (size_t i = 0; i < sz; ++i) lam[i] += acc[i];
    }
    free(stages); free(u); free(nu); free(mu); free(acc);
}

/* Terminal loss L = sum_b sum_i (u_N - target)^2 after nsteps RK4 steps (for finite
 * differences). */
double or_loss(const double *X, const double *q, int64_t n, const double *u0, int B, double t0, double dt,
               int nsteps, const double *kpar, const double *beta, const double *theta, const double *forcing,
               const double *target) {
    size_t sz = (size_t)(n * B);
    double *u = malloc(sizeof(double) * sz);
    memcpy(u, u0, sizeof(double) * sz);
    or_rk4(X, q, n, u, B, t0, dt, nsteps, kpar, beta, theta, forcing, NULL);
    double L = 0.0;
    for (size_t i = 0; i < sz; ++i) L += (u[i] - target[i]) * (u[i] - target[i]);
    free(u);
    return L;
}

/* ================================================================================
 * §5 examples: the C^4 smooth-step firing rate (labyrinth patterns, Eq. (smoothf)), the
 * synaptic-depression two-field model (travelling spots, Eq. (nfsyndep)) and the
 * Adams-Bashforth 5 integrator both examples use.
 *
 * model[] = {kind, rate, a, b, tau, beta_d}:
 *   kind 0: du/dt = -u + sum_j w_ij mu_j f(u_j)                       (Eq. (2.9), no forcing)
 *   kind 1: du/dt = -u + sum_j w_ij mu_j s_j f(u_j),
 *           tau ds/dt = 1 - s - beta_d s f(u)                           (s: synaptic efficacy)
 *   rate 0: f(u) = 1 / (1 + exp(-beta (u - theta)))   (per-trajectory beta, theta)
 *   rate 1: f = 0 for u < a, 1 for u >= b, p(u) in between, p the degree-9 polynomial with
 *           p(a) = 0, p(b) = 1 and its first four derivatives zero at a and at b.  With
 *           t = (u - a)/(b - a): p' is proportional to t^4 (1 - t)^4, so
 *           p = 630 int_0^t s^4 (1 - s)^4 ds = 126 t^5 - 420 t^6 + 540 t^7 - 315 t^8 + 70 t^9.
 * ============================================================================== */
static double smooth_step(double u, double a, double b) {
    if (u < a) return 0.0;
    if (u >= b) return 1.0;
    double t = (u - a) / (b - a);
    double t2 = t * t, t4 = t2 * t2, t5 = t4 * t;
    return t5 * (126.0 - 420.0 * t + 540.0 * t2 - 315.0 * t2 * t + 70.0 * t4);
}

double or_rate(const double *model, double u, double beta, double theta) {
    return (int)model[1] == 1 ? smooth_step(u, model[2], model[3]) : firing(u, beta, theta);
}

/* Vector field of the model for B trajectories: Fu (and Fs for kind 1). */
static void model_field(const double *X, const double *mu, int64_t n, const double *u, const double *s, int B,
                        const double *kpar, const double *beta, const double *theta, const double *model,
                        double *Fu, double *Fs) {
    or_kernel kp = {kpar[0], kpar[1], kpar[2], kpar[3], kpar[4]};
    int kind = (int)model[0];
    double *g = (double *)malloc(sizeof(double) * (size_t)(n * B));
    for (int b = 0; b < B; ++b)
        for (int64_t j = 0; j < n; ++j) {
            double f = or_rate(model, u[b * n + j], beta[b], theta[b]);
            g[b * n + j] = mu[j] * (kind == 1 ? s[b * n + j] : 1.0) * f;
            if (kind == 1) Fs[b * n + j] = (1.0 - s[b * n + j] - model[5] * s[b * n + j] * f) / model[4];
        }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int b = 0; b < B; ++b) {
            double acc = 0.0;
            for (int64_t j = 0; j < n; ++j) acc += kernel_w(&kp, pair_r2p(X, i, j, kp.period)) * g[b * n + j];
            Fu[b * n + i] = -u[b * n + i] + acc;
        }
    free(g);
}

/* Adams-Bashforth 5 weights from their definition: y_{n+1} = y_n + dt sum_m c_m F_{n-m},
 * c_m = int_0^1 L_m(s) ds with L_m the Lagrange basis polynomial through the nodes
 * s = 0, -1, -2, -3, -4 (times t_n, t_{n-1}, ...) that is 1 at s = -m.  5-point
 * Gauss-Legendre integrates the degree-4 integrands exactly. */
void or_ab5_weights(double *c) {
    double gx[5], gw[5];
    gauss_legendre(5, gx, gw);
    for (int m = 0; m < 5; ++m) {
        double acc = 0.0;
        for (int g = 0; g < 5; ++g) {
            double sv = 0.5 * (gx[g] + 1.0), L = 1.0;
            for (int k = 0; k < 5; ++k)
                if (k != m) L *= (sv + k) / (double)(k - m);
            acc += 0.5 * gw[g] * L;
        }
        c[m] = acc;
    }
}

/* Advance the model nsteps steps of dt from t0 (autonomous: t0 only labels time).
 * integrator 0: classical RK4 (tableau of or_rk4) on (u, s) together.
 * integrator 1: Adams-Bashforth 5; the paper does not say how it is started, and here the
 * first four steps are RK4 steps, each recording F at its start as AB5 history. */
void or_field_advance(const double *X, const double *mu, int64_t n, double *u, double *s, int B, double t0,
                      double dt, int nsteps, const double *kpar, const double *beta, const double *theta,
                      const double *model, int integrator) {
    (void)t0;
    int kind = (int)model[0];
    size_t sz = (size_t)(n * B);
    double *ku[4], *ks[4], *U = malloc(sizeof(double) * sz), *S = malloc(sizeof(double) * sz);
    for (int i = 0; i < 4; ++i) { ku[i] = malloc(sizeof(double) * sz); ks[i] = malloc(sizeof(double) * sz); }
    double *hu[5], *hs[5];
    for (int i = 0; i < 5; ++i) { hu[i] = malloc(sizeof(double) * sz); hs[i] = malloc(sizeof(double) * sz); }
    double c[5];
    or_ab5_weights(c);
    const double cs[4] = {0.0, 0.5, 0.5, 1.0};
    for (int step = 0; step < nsteps; ++step) {
        if (integrator == 1 && step >= 4) {
            /* history slot of F_step: step % 5; F_{step-m} in slot (step - m) % 5 */
            double *fu = hu[step % 5], *fs = hs[step % 5];
            model_field(X, mu, n, u, s, B, kpar, beta, theta, model, fu, fs);
            for (size_t i = 0; i < sz; ++i) {
                double du = 0.0, dsv = 0.0;
                for (int m = 0; m < 5; ++m) {
                    du += c[m] * hu[(step - m) % 5][i];
                    if (kind == 1) dsv += c[m] * hs[(step - m) % 5][i];
                }
                u[i] += dt * du;
                if (kind == 1) s[i] += dt * dsv;
            }
            continue;
        }
        for (int st = 0; st < 4; ++st) {
            for (size_t i = 0; i < sz; ++i) {
                U[i] = st == 0 ? u[i] : u[i] + cs[st] * dt * ku[st - 1][i];
                if (kind == 1) S[i] = st == 0 ? s[i] : s[i] + cs[st] * dt * ks[st - 1][i];
            }
            model_field(X, mu, n, U, kind == 1 ? S : NULL, B, kpar, beta, theta, model, ku[st], ks[st]);
        }
        if (integrator == 1) {
            memcpy(hu[step % 5], ku[0], sizeof(double) * sz);
            if (kind == 1) memcpy(hs[step % 5], ks[0], sizeof(double) * sz);
        }
        for (size_t i = 0; i < sz; ++i) {
            u[i] += dt / 6.0 * (ku[0][i] + 2.0 * ku[1][i] + 2.0 * ku[2][i] + ku[3][i]);
            if (kind == 1) s[i] += dt / 6.0 * (ks[0][i] + 2.0 * ks[1][i] + 2.0 * ks[2][i] + ks[3][i]);
        }
    }
    for (int i = 0; i < 4; ++i) { free(ku[i]); free(ks[i]); }
    for (int i = 0; i < 5; ++i) { free(hu[i]); free(hs[i]); }
    free(U); free(S);
}
