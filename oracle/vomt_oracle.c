/*
 * FP64 CPU oracle for vector / matrix / scalar L1 optimal mass transport
 * solved by PDHG (Ryu, Chen, Li, Osher, "Vector and Matrix Optimal Mass
 * Transport: Theory, Algorithm, and Applications", arXiv:1712.10279).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of the method that the CUDA library is checked against.  It is
 * compiled into its own shared object and loaded only by the tests, by the
 * smoke check and by the benchmark's CPU-baseline leg.  It shares no source,
 * header, table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Conventions (Appendix A, "Discretization"):
 *   - n x n grid on [0,1]^2, Delta x = h = 1/(n-1).
 *   - Every grid field is stored plane by plane, [c][j][i], with the x index i
 *     fastest: element (i, j) of plane c is at (c*n + j)*n + i, 0-based.
 *   - u_x and u_y are n x n with ghost entries u_x(n-1, j) = u_y(i, n-1) = 0
 *     (Appendix A, ghost cells); the iteration keeps them exactly zero.
 *   - Densities are cell masses (the finite-volume average of Appendix A).
 *
 * Everything is double precision, single threaded, in plain loops.  No
 * blocking, fusion or reordering beyond the order the paper's algorithm boxes
 * state: per iteration first the u-shrink for every point, then the w-shrink
 * for every point, then the extrapolated phi ascent for every point.
 *
 * Norm codes (Section 6.2):
 *   u: 0 = ||u||_{1,2} (per channel Euclidean in space, summed over channels;
 *          the reading of the garbled index ranges follows Section 8.3),
 *      1 = ||u||_2    (joint Euclidean over all channels and both directions),
 *      2 = ||u||_1    (entrywise).
 *   w: 0 = ||w||_1 (entrywise), 1 = ||w||_2 (joint Euclidean over the edges).
 * For matrices the same codes mean: u 1 = ||U||_2 (joint Frobenius over both
 * directions), 2 = ||U||_1 (entrywise), 3 = ||U||_{1,nuc} (nuclear norms of U_x
 * and U_y, summed); w 0 = ||W||_1 (entrywise), 1 = ||W||_2 (joint Frobenius over
 * the N components), 2 = ||W||_{1,nuc} (nuclear norms of the W_s, summed).
 *
 * Metrics written at every check (array of ORC_NMET doubles):
 *   [0] P   primal objective  sum_ij ||u_ij||_u + alpha sum_ij ||w_ij||_w
 *   [1] D   dual objective    sum <phi, rho1 - rho0>            (eq. vomt-dual)
 *   [2] rel_gap  |P - D| / |P|                                   (Section 8.1)
 *   [3] rel_res  ||div_x u + div_G w - (rho0 - rho1)|| / ||rho0 - rho1||
 *   [4] R   fixed-point residual ||s^t - s^{t-1}||^2_M             (Section 6.1)
 *   [5] dual_infeas  max_ij max(||grad phi||_{u*} - 1, ||grad_G phi||_{w*} - alpha, 0)
 *   [6] t   iteration index the metrics belong to
 *   [7] converged flag (1 if rel_gap <= tol_gap and rel_res <= tol_res)
 * Section 6.1 prints the y-block weight of R as 1/mu; the metric of the PDHG
 * proximal-point form makes it 1/nu, which is what is used here.
 *
 * Quadratic regularisation (the paper's concluding section): with eps > 0 the
 * objective gains eps (||u(x)||_2^2 + ||w(x)||_2^2) at every point, with
 * Euclidean norms (the reading under which the regularised problem is
 * strictly convex, as the paper states, for every choice of ||.||_u, ||.||_w).
 * P then includes that term, and D subtracts sum_x dist_2(grad phi(x), B_u*)^2
 * / (4 eps) + dist_2(grad_G phi(x), alpha B_w*)^2 / (4 eps), the conjugate of
 * ||.|| + eps ||.||_2^2 (B* the unit ball of the dual norm).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NMET 8

/* Built with -fopenmp -DORC_OPENMP (the benchmark's multi-core CPU baseline),
 * the loops over grid points of the iterations run on several threads.  Only
 * loops whose iterations are independent are split, and nothing inside a point
 * changes order, so the results are bit-identical to the one-thread build;
 * the reductions of the metrics stay serial. */
#ifdef ORC_OPENMP
#include <omp.h>
#define ORC_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")
#else
#define ORC_PARALLEL_FOR
#endif

/* Threads of the multi-core build (a no-op in the one-thread build). */
void orc_set_threads(int t)
{
#ifdef ORC_OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int orc_max_threads(void)
{
#ifdef ORC_OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define AT(c, j, i) (((size_t)(c) * (size_t)n + (size_t)(j)) * (size_t)n + (size_t)(i))

/* ------------------------------------------------------------------------ */
/* Shrink operators (Appendix B)                                             */
/* ------------------------------------------------------------------------ */

/* shrink_1(x; t) = argmin_z t|z| + (1/2)|z - x|^2 for real x. */
double orc_shrink1(double x, double t)
{
    double a = fabs(x);
    if (a <= t) return 0.0;
    return (1.0 - t / a) * x;
}

/* shrink_2(x; t) = argmin_z t||z||_2 + (1/2)||z - x||_2^2 for x in R^m. */
void orc_shrink2(int m, const double *x, double t, double *out)
{
    double s = 0.0;
    for (int q = 0; q < m; ++q) s += x[q] * x[q];
    s = sqrt(s);
    double f = (s <= t) ? 0.0 : (1.0 - t / s);
    for (int q = 0; q < m; ++q) out[q] = f * x[q];
}

/* ------------------------------------------------------------------------ */
/* Symmetric eigenvalues by the cyclic Jacobi method (used for the          */
/* "standard eigenvalue routine" of Sections 7.2 and 7.3).                   */
/* ------------------------------------------------------------------------ */

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Eigenvalues of the symmetric m x m row-major matrix A, ascending. */
int orc_jacobi_eigvals(int m, const double *A_in, double *ev)
{
    if (m <= 0) return -1;
    double *A = (double *)malloc(sizeof(double) * (size_t)m * (size_t)m);
    if (!A) return -1;
    memcpy(A, A_in, sizeof(double) * (size_t)m * (size_t)m);
    double scale = 0.0;
    for (int q = 0; q < m * m; ++q) scale += A[q] * A[q];
    for (int sweep = 0; sweep < 200; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) off += A[p * m + q] * A[p * m + q];
        if (off <= 1e-32 * scale || off == 0.0) break;
        for (int p = 0; p < m; ++p) {
            for (int q = p + 1; q < m; ++q) {
                double apq = A[p * m + q];
                if (apq == 0.0) continue;
                /* rotation angle that zeroes A[p][q]: cot(2 theta) = (aqq - app) / (2 apq) */
                double th = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < m; ++r) {
                    if (r == p || r == q) continue;
                    double arp = A[r * m + p], arq = A[r * m + q];
                    A[r * m + p] = A[p * m + r] = c * arp - s * arq;
                    A[r * m + q] = A[q * m + r] = s * arp + c * arq;
                }
                A[p * m + p] -= t * apq;
                A[q * m + q] += t * apq;
                A[p * m + q] = A[q * m + p] = 0.0;
            }
        }
    }
    for (int p = 0; p < m; ++p) ev[p] = A[p * m + p];
    qsort(ev, (size_t)m, sizeof(double), cmp_double);
    free(A);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Graph operators (Section 3.1)                                              */
/* ------------------------------------------------------------------------ */

/* Incidence matrix D (k x l, row-major).  Edge e = {a, b} is oriented from
 * the smaller node to the larger one: D[min][e] = +1, D[max][e] = -1. */
int orc_incidence(int k, int l, const int *ea, const int *eb, double *D)
{
    for (int q = 0; q < k * l; ++q) D[q] = 0.0;
    for (int e = 0; e < l; ++e) {
        int a = ea[e], b = eb[e];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b) return -1;
        int lo = a < b ? a : b, hi = a < b ? b : a;
        D[lo * l + e] = 1.0;
        D[hi * l + e] = -1.0;
    }
    return 0;
}

static double edge_cost(const double *cost, int e) { return cost ? cost[e] : 1.0; }

/* lambda_max(-Delta_G) with -Delta_G = D diag(1/c^2) D^T. */
double orc_graph_lmax(int k, int l, const int *ea, const int *eb, const double *cost)
{
    if (l == 0) return 0.0;
    double *D = (double *)malloc(sizeof(double) * (size_t)k * (size_t)l);
    double *M = (double *)calloc((size_t)k * (size_t)k, sizeof(double));
    double *ev = (double *)malloc(sizeof(double) * (size_t)k);
    orc_incidence(k, l, ea, eb, D);
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            double s = 0.0;
            for (int e = 0; e < l; ++e) {
                double c = edge_cost(cost, e);
                s += D[a * l + e] * D[b * l + e] / (c * c);
            }
            M[a * k + b] = s;
        }
    orc_jacobi_eigvals(k, M, ev);
    double lm = ev[k - 1];
    free(D); free(M); free(ev);
    return lm;
}

/* (grad_G phi)_e = (1/c_e) (D^T phi)_e at every grid point. g: [l][n][n]. */
void orc_grad_G(int n, int k, int l, const int *ea, const int *eb, const double *cost,
                const double *phi, double *g)
{
    (void)k;
    for (int e = 0; e < l; ++e) {
        int lo = ea[e] < eb[e] ? ea[e] : eb[e], hi = ea[e] < eb[e] ? eb[e] : ea[e];
        double ic = 1.0 / edge_cost(cost, e);
        ORC_PARALLEL_FOR
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                g[AT(e, j, i)] = ic * (phi[AT(lo, j, i)] - phi[AT(hi, j, i)]);
    }
}

/* div_G y = -D diag(1/c) y at every grid point. out: [k][n][n]. */
void orc_div_G(int n, int k, int l, const int *ea, const int *eb, const double *cost,
               const double *y, double *out)
{
    for (size_t q = 0; q < (size_t)k * n * n; ++q) out[q] = 0.0;
    for (int e = 0; e < l; ++e) {
        int lo = ea[e] < eb[e] ? ea[e] : eb[e], hi = ea[e] < eb[e] ? eb[e] : ea[e];
        double ic = 1.0 / edge_cost(cost, e);
        ORC_PARALLEL_FOR
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double v = ic * y[AT(e, j, i)];
                out[AT(lo, j, i)] -= v;   /* D[lo][e] = +1 */
                out[AT(hi, j, i)] += v;   /* D[hi][e] = -1 */
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Spatial operators with ghost cells (Appendix A)                            */
/* ------------------------------------------------------------------------ */

/* Forward-difference gradient; the ghost entries (i = n-1 for x, j = n-1 for
 * y) are zero.  planes: number of [n][n] planes (k for vectors, k*k for
 * matrices). */
void orc_grad(int n, int planes, const double *phi, double *gx, double *gy)
{
    double ih = (double)(n - 1);
    for (int c = 0; c < planes; ++c)
        ORC_PARALLEL_FOR
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                gx[AT(c, j, i)] = (i < n - 1) ? ih * (phi[AT(c, j, i + 1)] - phi[AT(c, j, i)]) : 0.0;
                gy[AT(c, j, i)] = (j < n - 1) ? ih * (phi[AT(c, j + 1, i)] - phi[AT(c, j, i)]) : 0.0;
            }
}

/* div_x(u)_ij = (1/h)(u_x,ij - u_x,(i-1)j + u_y,ij - u_y,i(j-1)), with
 * u_x,-1j = u_y,i-1 = 0 and the ghost entries taken as stored (zero). */
void orc_div(int n, int planes, const double *ux, const double *uy, double *out)
{
    double ih = (double)(n - 1);
    for (int c = 0; c < planes; ++c)
        ORC_PARALLEL_FOR
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double xl = (i > 0) ? ux[AT(c, j, i - 1)] : 0.0;
                double yl = (j > 0) ? uy[AT(c, j - 1, i)] : 0.0;
                out[AT(c, j, i)] = ih * (ux[AT(c, j, i)] - xl + uy[AT(c, j, i)] - yl);
            }
}

/* ------------------------------------------------------------------------ */
/* Quantum gradient / divergence (Section 4.1), real matrices               */
/* ------------------------------------------------------------------------ */

/* C = A B for k x k row-major. */
static void matmul(int k, const double *A, const double *B, double *C)
{
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            double s = 0.0;
            for (int q = 0; q < k; ++q) s += A[a * k + q] * B[q * k + b];
            C[a * k + b] = s;
        }
}

/* Z_s = L_s X - X L_s for one k x k matrix X; Z: N consecutive k x k blocks. */
void orc_grad_L_point(int k, int N, const double *L, const double *X, double *Z)
{
    double *t1 = (double *)malloc(sizeof(double) * (size_t)k * k);
    double *t2 = (double *)malloc(sizeof(double) * (size_t)k * k);
    for (int s = 0; s < N; ++s) {
        matmul(k, L + (size_t)s * k * k, X, t1);
        matmul(k, X, L + (size_t)s * k * k, t2);
        for (int q = 0; q < k * k; ++q) Z[(size_t)s * k * k + q] = t1[q] - t2[q];
    }
    free(t1); free(t2);
}

/* Y = sum_s (-L_s Z_s + Z_s L_s) for one point. */
void orc_div_L_point(int k, int N, const double *L, const double *Z, double *Y)
{
    double *t1 = (double *)malloc(sizeof(double) * (size_t)k * k);
    double *t2 = (double *)malloc(sizeof(double) * (size_t)k * k);
    for (int q = 0; q < k * k; ++q) Y[q] = 0.0;
    for (int s = 0; s < N; ++s) {
        matmul(k, L + (size_t)s * k * k, Z + (size_t)s * k * k, t1);
        matmul(k, Z + (size_t)s * k * k, L + (size_t)s * k * k, t2);
        for (int q = 0; q < k * k; ++q) Y[q] += -t1[q] + t2[q];
    }
    free(t1); free(t2);
}

/* Grid versions: X [k*k][n][n], Z [N*k*k][n][n] (component s, entry q at plane s*k*k+q). */
void orc_grad_L(int n, int k, int N, const double *L, const double *X, double *Z)
{
    int kk = k * k;
    ORC_PARALLEL_FOR
    for (int j = 0; j < n; ++j) {
        double *x = (double *)malloc(sizeof(double) * (size_t)kk);
        double *z = (double *)malloc(sizeof(double) * (size_t)kk * N);
        for (int i = 0; i < n; ++i) {
            for (int q = 0; q < kk; ++q) x[q] = X[AT(q, j, i)];
            orc_grad_L_point(k, N, L, x, z);
            for (int q = 0; q < kk * N; ++q) Z[AT(q, j, i)] = z[q];
        }
        free(x); free(z);
    }
}

void orc_div_L(int n, int k, int N, const double *L, const double *Z, double *Y)
{
    int kk = k * k;
    ORC_PARALLEL_FOR
    for (int j = 0; j < n; ++j) {
        double *z = (double *)malloc(sizeof(double) * (size_t)kk * N);
        double *y = (double *)malloc(sizeof(double) * (size_t)kk);
        for (int i = 0; i < n; ++i) {
            for (int q = 0; q < kk * N; ++q) z[q] = Z[AT(q, j, i)];
            orc_div_L_point(k, N, L, z, y);
            for (int q = 0; q < kk; ++q) Y[AT(q, j, i)] = y[q];
        }
        free(z); free(y);
    }
}

/* The k^2 x k^2 matrix of -Delta_L = -div_L grad_L acting on vec(X) (row-major
 * vec: index a*k+b), for real symmetric L_s:
 *   -Delta_L X = sum_s (L_s^2 X - 2 L_s X L_s + X L_s^2).
 * Section 7.3 forms exactly this matrix and takes its largest eigenvalue. */
void orc_neg_quantum_laplacian(int k, int N, const double *L, double *M)
{
    int kk = k * k;
    double *L2 = (double *)malloc(sizeof(double) * (size_t)kk);
    for (int q = 0; q < kk * kk; ++q) M[q] = 0.0;
    for (int s = 0; s < N; ++s) {
        const double *Ls = L + (size_t)s * kk;
        matmul(k, Ls, Ls, L2);
        /* row (a,b), column (c,d):  (L^2)_{ac} d_{bd} + d_{ac} (L^2)_{db} - 2 L_{ac} L_{db} */
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b)
                for (int c = 0; c < k; ++c)
                    for (int d = 0; d < k; ++d) {
                        double v = 0.0;
                        if (b == d) v += L2[a * k + c];
                        if (a == c) v += L2[d * k + b];
                        v -= 2.0 * Ls[a * k + c] * Ls[d * k + b];
                        M[(a * k + b) * kk + (c * k + d)] += v;
                    }
    }
    free(L2);
}

double orc_quantum_lmax(int k, int N, const double *L)
{
    int kk = k * k;
    double *M = (double *)malloc(sizeof(double) * (size_t)kk * kk);
    double *ev = (double *)malloc(sizeof(double) * (size_t)kk);
    orc_neg_quantum_laplacian(k, N, L, M);
    orc_jacobi_eigvals(kk, M, ev);
    double lm = ev[kk - 1];
    free(M); free(ev);
    return lm;
}

/* Second-smallest eigenvalue of -Delta_L restricted to symmetric matrices.
 * The standing assumption of Section 4.1 (ker grad_L = span{I}) holds iff it
 * is positive.  Orthonormal basis of Sym(k): E_aa and (E_ab + E_ba)/sqrt 2. */
double orc_quantum_sym_gap(int k, int N, const double *L)
{
    int kk = k * k, m = k * (k + 1) / 2;
    double *M = (double *)malloc(sizeof(double) * (size_t)kk * kk);
    double *B = (double *)calloc((size_t)kk * m, sizeof(double));
    double *S = (double *)malloc(sizeof(double) * (size_t)m * m);
    double *ev = (double *)malloc(sizeof(double) * (size_t)m);
    orc_neg_quantum_laplacian(k, N, L, M);
    int col = 0;
    for (int a = 0; a < k; ++a)
        for (int b = a; b < k; ++b, ++col) {
            if (a == b) B[(a * k + a) * m + col] = 1.0;
            else {
                B[(a * k + b) * m + col] = 1.0 / sqrt(2.0);
                B[(b * k + a) * m + col] = 1.0 / sqrt(2.0);
            }
        }
    for (int p = 0; p < m; ++p)
        for (int q = 0; q < m; ++q) {
            double s = 0.0;
            for (int r = 0; r < kk; ++r)
                for (int c = 0; c < kk; ++c) s += B[r * m + p] * M[r * kk + c] * B[c * m + q];
            S[p * m + q] = s;
        }
    orc_jacobi_eigvals(m, S, ev);
    double g = (m > 1) ? ev[1] : 0.0;
    free(M); free(B); free(S); free(ev);
    return g;
}

/* ------------------------------------------------------------------------ */
/* Step sizes (Sections 7.1-7.3)                                              */
/* ------------------------------------------------------------------------ */

/* mu = 1/(32 tau (n-1)^2), nu = 1/(4 tau lambda_max); with no second operator
 * (l = 0) the S-OMT rule mu = 1/(16 tau (n-1)^2) of Section 7.1 is used. */
void orc_step_sizes(int n, double tau, double lmax_second, int has_second, double *mu, double *nu)
{
    double n1 = (double)(n - 1);
    if (!has_second) {
        *mu = 1.0 / (16.0 * tau * n1 * n1);
        *nu = 0.0;
    } else {
        *mu = 1.0 / (32.0 * tau * n1 * n1);
        *nu = 1.0 / (4.0 * tau * lmax_second);
    }
}

/* ------------------------------------------------------------------------ */
/* Vector OMT (Section 7.2)                                                   */
/* ------------------------------------------------------------------------ */

/* u-shrink at one point for all channels (Section 7.2, first line of the
 * loop) given v = u + mu grad phi in vx[c], vy[c]. */
static void shrink_u_point(int k, int u_norm, double t, double *vx, double *vy)
{
    if (u_norm == 0) {              /* ||.||_{1,2}: shrink_2 on each channel's 2-vector */
        for (int c = 0; c < k; ++c) {
            double v[2] = {vx[c], vy[c]}, o[2];
            orc_shrink2(2, v, t, o);
            vx[c] = o[0]; vy[c] = o[1];
        }
    } else if (u_norm == 1) {       /* ||.||_2: shrink_2 on the whole 2k-vector */
        double v[64], o[64];
        for (int c = 0; c < k; ++c) { v[c] = vx[c]; v[k + c] = vy[c]; }
        orc_shrink2(2 * k, v, t, o);
        for (int c = 0; c < k; ++c) { vx[c] = o[c]; vy[c] = o[k + c]; }
    } else {                        /* ||.||_1: shrink_1 entry by entry */
        for (int c = 0; c < k; ++c) { vx[c] = orc_shrink1(vx[c], t); vy[c] = orc_shrink1(vy[c], t); }
    }
}

static void shrink_w_point(int l, int w_norm, double t, double *x)
{
    if (l == 0) return;
    if (w_norm == 0) {
        for (int e = 0; e < l; ++e) x[e] = orc_shrink1(x[e], t);
    } else {
        double o[64];
        orc_shrink2(l, x, t, o);
        for (int e = 0; e < l; ++e) x[e] = o[e];
    }
}

static double norm_u_point(int k, int u_norm, const double *ux, const double *uy)
{
    double s = 0.0;
    if (u_norm == 0) {
        for (int c = 0; c < k; ++c) s += sqrt(ux[c] * ux[c] + uy[c] * uy[c]);
    } else if (u_norm == 1) {
        for (int c = 0; c < k; ++c) s += ux[c] * ux[c] + uy[c] * uy[c];
        s = sqrt(s);
    } else {
        for (int c = 0; c < k; ++c) s += fabs(ux[c]) + fabs(uy[c]);
    }
    return s;
}

/* dual norm of ||.||_u at one point */
static double dualnorm_u_point(int k, int u_norm, const double *gx, const double *gy)
{
    double s = 0.0;
    if (u_norm == 0) {
        for (int c = 0; c < k; ++c) { double v = sqrt(gx[c] * gx[c] + gy[c] * gy[c]); if (v > s) s = v; }
    } else if (u_norm == 1) {
        for (int c = 0; c < k; ++c) s += gx[c] * gx[c] + gy[c] * gy[c];
        s = sqrt(s);
    } else {
        for (int c = 0; c < k; ++c) { if (fabs(gx[c]) > s) s = fabs(gx[c]); if (fabs(gy[c]) > s) s = fabs(gy[c]); }
    }
    return s;
}

static double norm_w_point(int l, int w_norm, const double *w)
{
    double s = 0.0;
    if (w_norm == 0) { for (int e = 0; e < l; ++e) s += fabs(w[e]); }
    else { for (int e = 0; e < l; ++e) s += w[e] * w[e]; s = sqrt(s); }
    return s;
}

static double dualnorm_w_point(int l, int w_norm, const double *g)
{
    double s = 0.0;
    if (w_norm == 0) { for (int e = 0; e < l; ++e) if (fabs(g[e]) > s) s = fabs(g[e]); }
    else { for (int e = 0; e < l; ++e) s += g[e] * g[e]; s = sqrt(s); }
    return s;
}

/* Squared Euclidean distance from g to the dual unit ball of ||.||_u at one
 * point (the ball is a product of per-channel discs for ||.||_{1,2}, one ball
 * for ||.||_2, a box for ||.||_1). */
static double dist2_dualball_u_point(int k, int u_norm, const double *gx, const double *gy)
{
    double s = 0.0;
    if (u_norm == 0) {
        for (int c = 0; c < k; ++c) {
            double v = sqrt(gx[c] * gx[c] + gy[c] * gy[c]) - 1.0;
            if (v > 0.0) s += v * v;
        }
    } else if (u_norm == 1) {
        double v = dualnorm_u_point(k, 1, gx, gy) - 1.0;
        if (v > 0.0) s = v * v;
    } else {
        for (int c = 0; c < k; ++c) {
            double v = fabs(gx[c]) - 1.0, q = fabs(gy[c]) - 1.0;
            if (v > 0.0) s += v * v;
            if (q > 0.0) s += q * q;
        }
    }
    return s;
}

/* Squared Euclidean distance from g to the dual ball of radius alpha of ||.||_w. */
static double dist2_dualball_w_point(int l, int w_norm, const double *g, double alpha)
{
    double s = 0.0;
    if (w_norm == 0) {
        for (int e = 0; e < l; ++e) { double v = fabs(g[e]) - alpha; if (v > 0.0) s += v * v; }
    } else {
        double v = dualnorm_w_point(l, 1, g) - alpha;
        if (v > 0.0) s = v * v;
    }
    return s;
}

/* Metrics of the state (ux, uy, w, phi) (see the header comment).  R is
 * computed from the previous state (pux, puy, pw, pphi) when those are given,
 * else set to 0.  out[6], out[7] are left to the caller. */
void orc_vomt_metrics(int n, int k, int l, const int *ea, const int *eb, const double *cost,
                      const double *rho0, const double *rho1, double alpha, int u_norm, int w_norm,
                      double mu, double nu, double tau,
                      const double *ux, const double *uy, const double *w, const double *phi,
                      const double *pux, const double *puy, const double *pw, const double *pphi,
                      double eps, double *out)
{
    size_t nk = (size_t)k * n * n, nl = (size_t)l * n * n, nn = (size_t)n * n;
    double *dv = (double *)malloc(sizeof(double) * nk);
    double *dg = (double *)malloc(sizeof(double) * nk);
    double *gx = (double *)malloc(sizeof(double) * nk);
    double *gy = (double *)malloc(sizeof(double) * nk);
    double *gg = (double *)malloc(sizeof(double) * (nl ? nl : 1));
    double a[32], b[32], c3[64];

    /* primal objective (with the regulariser eps (||u||_2^2 + ||w||_2^2) per point) */
    double P = 0.0;
    for (size_t p = 0; p < nn; ++p) {
        for (int c = 0; c < k; ++c) { a[c] = ux[c * nn + p]; b[c] = uy[c * nn + p]; }
        P += norm_u_point(k, u_norm, a, b);
        for (int e = 0; e < l; ++e) c3[e] = w[e * nn + p];
        P += alpha * norm_w_point(l, w_norm, c3);
        if (eps > 0.0) {
            double q2 = 0.0;
            for (int c = 0; c < k; ++c) q2 += a[c] * a[c] + b[c] * b[c];
            for (int e = 0; e < l; ++e) q2 += c3[e] * c3[e];
            P += eps * q2;
        }
    }
    /* dual objective; with eps > 0 the conjugate of ||.|| + eps ||.||_2^2 is
     * dist_2(., dual ball)^2 / (4 eps), subtracted at every point */
    double D = 0.0;
    for (size_t q = 0; q < nk; ++q) D += phi[q] * (rho1[q] - rho0[q]);
    /* constraint residual */
    orc_div(n, k, ux, uy, dv);
    orc_div_G(n, k, l, ea, eb, cost, w, dg);
    double rr = 0.0, bb = 0.0;
    for (size_t q = 0; q < nk; ++q) {
        double r = dv[q] + dg[q] - (rho0[q] - rho1[q]);
        rr += r * r;
        bb += (rho0[q] - rho1[q]) * (rho0[q] - rho1[q]);
    }
    /* dual infeasibility */
    orc_grad(n, k, phi, gx, gy);
    if (l) orc_grad_G(n, k, l, ea, eb, cost, phi, gg);
    double di = 0.0, dist2 = 0.0;
    for (size_t p = 0; p < nn; ++p) {
        for (int c = 0; c < k; ++c) { a[c] = gx[c * nn + p]; b[c] = gy[c * nn + p]; }
        double v = dualnorm_u_point(k, u_norm, a, b) - 1.0;
        if (v > di) di = v;
        if (eps > 0.0) dist2 += dist2_dualball_u_point(k, u_norm, a, b);
        if (l) {
            for (int e = 0; e < l; ++e) c3[e] = gg[e * nn + p];
            v = dualnorm_w_point(l, w_norm, c3) - alpha;
            if (v > di) di = v;
            if (eps > 0.0) dist2 += dist2_dualball_w_point(l, w_norm, c3, alpha);
        }
    }
    if (eps > 0.0) D -= dist2 / (4.0 * eps);
    /* fixed-point residual in the PDHG metric */
    double R = 0.0;
    if (pux) {
        double *dux = (double *)malloc(sizeof(double) * nk), *duy = (double *)malloc(sizeof(double) * nk);
        double *dw = (double *)malloc(sizeof(double) * (nl ? nl : 1));
        double su = 0.0, sw = 0.0, sp = 0.0, cr = 0.0;
        for (size_t q = 0; q < nk; ++q) {
            dux[q] = ux[q] - pux[q]; duy[q] = uy[q] - puy[q];
            su += dux[q] * dux[q] + duy[q] * duy[q];
            sp += (phi[q] - pphi[q]) * (phi[q] - pphi[q]);
        }
        for (size_t q = 0; q < nl; ++q) { dw[q] = w[q] - pw[q]; sw += dw[q] * dw[q]; }
        orc_div(n, k, dux, duy, dv);
        orc_div_G(n, k, l, ea, eb, cost, dw, dg);
        for (size_t q = 0; q < nk; ++q) cr += (phi[q] - pphi[q]) * (dv[q] + dg[q]);
        R = su / mu + (l ? sw / nu : 0.0) + sp / tau - 2.0 * cr;
        free(dux); free(duy); free(dw);
    }
    out[0] = P;
    out[1] = D;
    out[2] = fabs(P - D) / (fabs(P) > 1e-300 ? fabs(P) : 1e-300);
    out[3] = sqrt(rr) / (bb > 0.0 ? sqrt(bb) : 1.0);
    out[4] = R;
    out[5] = di;
    free(dv); free(dg); free(gx); free(gy); free(gg);
}

/*
 * V-OMT by PDHG (Section 7.2):
 *   u^{t+1}_ij = shrink_u(u^t_ij + mu (grad phi^t)_ij ; mu)
 *   w^{t+1}_ij = shrink_w(w^t_ij + nu (grad_G phi^t_ij) ; alpha nu)
 *   phi^{t+1}_ij = phi^t_ij + tau (div_x(2u^{t+1} - u^t)_ij + div_G(2w^{t+1} - w^t)_ij
 *                                 + rho1_ij - rho0_ij)
 * The state arrays hold the initial iterate on entry (zeros for a cold start)
 * and the last iterate on return.  A check runs after iteration t when
 * t % check_every == 0 or t == max_iters; it appends a metrics row to history
 * (up to hist_cap rows) and stops the loop when tol_gap > 0 and both relative
 * gap and relative residual are within tolerance.  Returns the number of
 * iterations run; metrics gets the last check row.
 */
int orc_vomt_solve(int n, int k, int l, const int *ea, const int *eb, const double *cost,
                   const double *rho0, const double *rho1, double alpha,
                   double tau, double mu, double nu, int u_norm, int w_norm,
                   int max_iters, int check_every, double tol_gap, double tol_res,
                   double *ux, double *uy, double *w, double *phi,
                   double *metrics, double *history, int hist_cap, double eps)
{
    size_t nk = (size_t)k * n * n, nl = (size_t)l * n * n, nn = (size_t)n * n;
    double *gx = (double *)malloc(sizeof(double) * nk), *gy = (double *)malloc(sizeof(double) * nk);
    double *nux = (double *)malloc(sizeof(double) * nk), *nuy = (double *)malloc(sizeof(double) * nk);
    double *gg = (double *)malloc(sizeof(double) * (nl ? nl : 1));
    double *nw = (double *)malloc(sizeof(double) * (nl ? nl : 1));
    double *bx = (double *)malloc(sizeof(double) * nk), *by = (double *)malloc(sizeof(double) * nk);
    double *bw = (double *)malloc(sizeof(double) * (nl ? nl : 1));
    double *dv = (double *)malloc(sizeof(double) * nk), *dg = (double *)malloc(sizeof(double) * nk);
    double *pphi = (double *)malloc(sizeof(double) * nk);
    int nh = 0, t = 0;
    if (check_every <= 0) check_every = max_iters > 0 ? max_iters : 1;
    /* With the regulariser eps ||.||_2^2 (conclusions of the paper), the primal
     * steps are the proximal maps of mu (||.||_u + eps ||.||_2^2) and of
     * nu (alpha ||.||_w + eps ||.||_2^2).  Completing the square,
     *   t ||z|| + t eps ||z||^2 + |z - v|^2 / 2
     *     = (1 + 2 t eps) (t' ||z|| + |z - v'|^2 / 2) + const,
     * with v' = v / (1 + 2 t eps) and t' = t / (1 + 2 t eps), so each step is the
     * shrink of v' with threshold t'.  eps = 0 gives the plain iteration. */
    const double su = 1.0 / (1.0 + 2.0 * mu * eps), sw = 1.0 / (1.0 + 2.0 * nu * eps);

    for (t = 1; t <= max_iters; ++t) {
        /* u-update: shrink of u + mu grad phi with threshold mu */
        orc_grad(n, k, phi, gx, gy);
        ORC_PARALLEL_FOR
        for (size_t p = 0; p < nn; ++p) {
            double a[32], b[32];
            for (int c = 0; c < k; ++c) {
                a[c] = (ux[c * nn + p] + mu * gx[c * nn + p]) * su;
                b[c] = (uy[c * nn + p] + mu * gy[c * nn + p]) * su;
            }
            shrink_u_point(k, u_norm, mu * su, a, b);
            for (int c = 0; c < k; ++c) { nux[c * nn + p] = a[c]; nuy[c * nn + p] = b[c]; }
        }
        /* w-update: shrink of w + nu grad_G phi with threshold alpha nu */
        if (l) {
            orc_grad_G(n, k, l, ea, eb, cost, phi, gg);
            ORC_PARALLEL_FOR
            for (size_t p = 0; p < nn; ++p) {
                double x[64];
                for (int e = 0; e < l; ++e) x[e] = (w[e * nn + p] + nu * gg[e * nn + p]) * sw;
                shrink_w_point(l, w_norm, alpha * nu * sw, x);
                for (int e = 0; e < l; ++e) nw[e * nn + p] = x[e];
            }
        }
        /* extrapolation and dual ascent */
        ORC_PARALLEL_FOR
        for (size_t q = 0; q < nk; ++q) { bx[q] = 2.0 * nux[q] - ux[q]; by[q] = 2.0 * nuy[q] - uy[q]; }
        for (size_t q = 0; q < nl; ++q) bw[q] = 2.0 * nw[q] - w[q];
        orc_div(n, k, bx, by, dv);
        if (l) orc_div_G(n, k, l, ea, eb, cost, bw, dg);
        else for (size_t q = 0; q < nk; ++q) dg[q] = 0.0;
        memcpy(pphi, phi, sizeof(double) * nk);
        ORC_PARALLEL_FOR
        for (size_t q = 0; q < nk; ++q) phi[q] = phi[q] + tau * (dv[q] + dg[q] + rho1[q] - rho0[q]);

        int check = (t % check_every == 0) || (t == max_iters);
        double m[ORC_NMET];
        if (check) {
            /* previous state: ux, uy, w (not yet overwritten), pphi */
            orc_vomt_metrics(n, k, l, ea, eb, cost, rho0, rho1, alpha, u_norm, w_norm, mu, nu, tau,
                             nux, nuy, nw, phi, ux, uy, w, pphi, eps, m);
            m[6] = (double)t;
            m[7] = (tol_gap > 0.0 && m[2] <= tol_gap && m[3] <= tol_res) ? 1.0 : 0.0;
            if (history && nh < hist_cap) { memcpy(history + (size_t)nh * ORC_NMET, m, sizeof m); ++nh; }
            if (metrics) memcpy(metrics, m, sizeof m);
        }
        memcpy(ux, nux, sizeof(double) * nk);
        memcpy(uy, nuy, sizeof(double) * nk);
        if (l) memcpy(w, nw, sizeof(double) * nl);
        if (check && m[7] != 0.0) break;
    }
    if (t > max_iters) t = max_iters;
    free(gx); free(gy); free(nux); free(nuy); free(gg); free(nw);
    free(bx); free(by); free(bw); free(dv); free(dg); free(pphi);
    return t;
}

/*
 * S-OMT by PDHG exactly as the box of Section 7.1 (scalar density, k = 1):
 *   u^{t+1}_ij = shrink(u^t_ij + mu (grad phi^t)_ij ; mu)
 *   phi^{t+1}_ij = phi^t_ij + tau (div_x(2u^{t+1} - u^t)_ij + rho1_ij - rho0_ij)
 * u_norm: 0 = isotropic ||u||_2 of the 2-vector, 2 = ||u||_1.
 */
int orc_somt_run(int n, const double *rho0, const double *rho1, double tau, double mu, int u_norm,
                 int iters, double *ux, double *uy, double *phi)
{
    size_t nn = (size_t)n * n;
    double *gx = (double *)malloc(sizeof(double) * nn), *gy = (double *)malloc(sizeof(double) * nn);
    double *nx = (double *)malloc(sizeof(double) * nn), *ny = (double *)malloc(sizeof(double) * nn);
    double *dv = (double *)malloc(sizeof(double) * nn);
    for (int t = 0; t < iters; ++t) {
        orc_grad(n, 1, phi, gx, gy);
        for (size_t p = 0; p < nn; ++p) {
            double v[2] = {ux[p] + mu * gx[p], uy[p] + mu * gy[p]}, o[2];
            if (u_norm == 2) { o[0] = orc_shrink1(v[0], mu); o[1] = orc_shrink1(v[1], mu); }
            else orc_shrink2(2, v, mu, o);
            nx[p] = o[0]; ny[p] = o[1];
        }
        for (size_t p = 0; p < nn; ++p) { gx[p] = 2.0 * nx[p] - ux[p]; gy[p] = 2.0 * ny[p] - uy[p]; }
        orc_div(n, 1, gx, gy, dv);
        for (size_t p = 0; p < nn; ++p) phi[p] += tau * (dv[p] + rho1[p] - rho0[p]);
        memcpy(ux, nx, sizeof(double) * nn);
        memcpy(uy, ny, sizeof(double) * nn);
    }
    free(gx); free(gy); free(nx); free(ny); free(dv);
    return iters;
}

/* ------------------------------------------------------------------------ */
/* Matrix OMT (Section 7.3), real symmetric densities, full k x k storage    */
/* ------------------------------------------------------------------------ */

/* Fields: Phi, Ux, Uy, Lam0, Lam1 [k*k][n][n]; W [N*k*k][n][n]. */
/* ------------------------------------------------------------------------ */
/* Nuclear norm (Section 6.2; shrink of Appendix B)                           */
/* ------------------------------------------------------------------------ */

/* Cyclic Jacobi eigen-decomposition of a symmetric m x m matrix A (row-major,
 * overwritten): on return ev holds the eigenvalues and column j of V the
 * eigenvector of ev[j].  Rotations as in Golub and Van Loan, Section 8.5. */
static void jacobi_eig_vectors(int m, double *A, double *V, double *ev)
{
    for (int i = 0; i < m * m; ++i) V[i] = 0.0;
    for (int i = 0; i < m; ++i) V[i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                tot += A[i * m + j] * A[i * m + j];
                if (i != j) off += A[i * m + j] * A[i * m + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                double apq = A[p * m + q];
                if (apq == 0.0) continue;
                double theta = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s_ = t * c;
                for (int r = 0; r < m; ++r) {           /* A <- A J */
                    double arp = A[r * m + p], arq = A[r * m + q];
                    A[r * m + p] = c * arp - s_ * arq;
                    A[r * m + q] = s_ * arp + c * arq;
                }
                for (int r = 0; r < m; ++r) {           /* A <- J^T A */
                    double apr = A[p * m + r], aqr = A[q * m + r];
                    A[p * m + r] = c * apr - s_ * aqr;
                    A[q * m + r] = s_ * apr + c * aqr;
                }
                for (int r = 0; r < m; ++r) {           /* V <- V J */
                    double vrp = V[r * m + p], vrq = V[r * m + q];
                    V[r * m + p] = c * vrp - s_ * vrq;
                    V[r * m + q] = s_ * vrp + c * vrq;
                }
            }
    }
    for (int i = 0; i < m; ++i) ev[i] = A[i * m + i];
}

/* Singular values of the k x k matrix X (k <= 8): square roots of the
 * eigenvalues of X^T X; V (optional) gets the right singular vectors. */
static void singular_values(int k, const double *X, double *sv, double *V)
{
    double A[64], Vl[64], ev[8];
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            double v = 0.0;
            for (int r = 0; r < k; ++r) v += X[r * k + i] * X[r * k + j];
            A[i * k + j] = v;
        }
    jacobi_eig_vectors(k, A, Vl, ev);
    for (int i = 0; i < k; ++i) sv[i] = ev[i] > 0.0 ? sqrt(ev[i]) : 0.0;
    if (V) memcpy(V, Vl, sizeof(double) * k * k);
}

/* ||X||_nuc, the sum of the singular values, and the spectral norm (its dual). */
double orc_nuc_norm(int k, const double *X)
{
    double sv[8], s = 0.0;
    singular_values(k, X, sv, NULL);
    for (int i = 0; i < k; ++i) s += sv[i];
    return s;
}

double orc_spectral_norm(int k, const double *X)
{
    double sv[8], s = 0.0;
    singular_values(k, X, sv, NULL);
    for (int i = 0; i < k; ++i) if (sv[i] > s) s = sv[i];
    return s;
}

/* shrink_nuc (Appendix B): argmin_Z t ||Z||_nuc + |Z - X|_F^2 / 2 = U diag((sigma - t)_+) V^T
 * for X = U diag(sigma) V^T; computed as X V diag((sigma_i - t)_+ / sigma_i) V^T. */
void orc_shrink_nuc(int k, const double *X, double t, double *out)
{
    double sv[8], V[64], f[8], XV[64];
    singular_values(k, X, sv, V);
    for (int i = 0; i < k; ++i) f[i] = sv[i] > t ? (sv[i] - t) / sv[i] : 0.0;
    for (int r = 0; r < k; ++r)
        for (int i = 0; i < k; ++i) {
            double v = 0.0;
            for (int m = 0; m < k; ++m) v += X[r * k + m] * V[m * k + i];
            XV[r * k + i] = v * f[i];
        }
    for (int r = 0; r < k; ++r)
        for (int c = 0; c < k; ++c) {
            double v = 0.0;
            for (int i = 0; i < k; ++i) v += XV[r * k + i] * V[c * k + i];
            out[r * k + c] = v;
        }
}

void orc_momt_metrics(int n, int k, int N, const double *L, const double *Lam0, const double *Lam1,
                      double alpha, int u_norm, int w_norm, double mu, double nu, double tau,
                      const double *Ux, const double *Uy, const double *W, const double *Phi,
                      const double *pUx, const double *pUy, const double *pW, const double *pPhi,
                      double *out)
{
    int kk = k * k;
    size_t nn = (size_t)n * n, nk = (size_t)kk * nn, nw = (size_t)N * kk * nn;
    double *dv = (double *)malloc(sizeof(double) * nk), *dl = (double *)malloc(sizeof(double) * nk);
    double *gx = (double *)malloc(sizeof(double) * nk), *gy = (double *)malloc(sizeof(double) * nk);
    double *gl = (double *)malloc(sizeof(double) * nw);
    double P = 0.0, D = 0.0, rr = 0.0, bb = 0.0, di = 0.0;
    double X[64];
    for (size_t p = 0; p < nn; ++p) {
        double su = 0.0, sw = 0.0;
        if (u_norm == 3) {              /* ||U||_{1,nuc} = ||U_x||_nuc + ||U_y||_nuc */
            for (int q = 0; q < kk; ++q) X[q] = Ux[q * nn + p];
            su = orc_nuc_norm(k, X);
            for (int q = 0; q < kk; ++q) X[q] = Uy[q * nn + p];
            su += orc_nuc_norm(k, X);
        } else {
            for (int q = 0; q < kk; ++q) {
                if (u_norm == 2) su += fabs(Ux[q * nn + p]) + fabs(Uy[q * nn + p]);
                else su += Ux[q * nn + p] * Ux[q * nn + p] + Uy[q * nn + p] * Uy[q * nn + p];
            }
            if (u_norm != 2) su = sqrt(su);
        }
        if (w_norm == 2) {              /* ||W||_{1,nuc} = sum_s ||W_s||_nuc */
            for (int s_ = 0; s_ < N; ++s_) {
                for (int q = 0; q < kk; ++q) X[q] = W[(s_ * kk + q) * nn + p];
                sw += orc_nuc_norm(k, X);
            }
        } else {
            for (int q = 0; q < N * kk; ++q) {
                if (w_norm == 0) sw += fabs(W[q * nn + p]);
                else sw += W[q * nn + p] * W[q * nn + p];
            }
            if (w_norm != 0) sw = sqrt(sw);
        }
        P += su + alpha * sw;
    }
    for (size_t q = 0; q < nk; ++q) D += Phi[q] * (Lam1[q] - Lam0[q]);
    orc_div(n, kk, Ux, Uy, dv);
    orc_div_L(n, k, N, L, W, dl);
    for (size_t q = 0; q < nk; ++q) {
        double r = dv[q] + dl[q] - (Lam0[q] - Lam1[q]);
        rr += r * r;
        bb += (Lam0[q] - Lam1[q]) * (Lam0[q] - Lam1[q]);
    }
    orc_grad(n, kk, Phi, gx, gy);
    orc_grad_L(n, k, N, L, Phi, gl);
    for (size_t p = 0; p < nn; ++p) {
        double s = 0.0, m = 0.0;
        if (u_norm == 3) {              /* dual of ||.||_{1,nuc}: the larger spectral norm */
            for (int q = 0; q < kk; ++q) X[q] = gx[q * nn + p];
            s = orc_spectral_norm(k, X);
            for (int q = 0; q < kk; ++q) X[q] = gy[q * nn + p];
            double s2 = orc_spectral_norm(k, X);
            if (s2 > s) s = s2;
        } else {
            for (int q = 0; q < kk; ++q) {
                if (u_norm == 2) { if (fabs(gx[q * nn + p]) > s) s = fabs(gx[q * nn + p]); if (fabs(gy[q * nn + p]) > s) s = fabs(gy[q * nn + p]); }
                else s += gx[q * nn + p] * gx[q * nn + p] + gy[q * nn + p] * gy[q * nn + p];
            }
            if (u_norm != 2) s = sqrt(s);
        }
        if (w_norm == 2) {
            for (int s_ = 0; s_ < N; ++s_) {
                for (int q = 0; q < kk; ++q) X[q] = gl[(s_ * kk + q) * nn + p];
                double v = orc_spectral_norm(k, X);
                if (v > m) m = v;
            }
        } else {
            for (int q = 0; q < N * kk; ++q) {
                if (w_norm == 0) { if (fabs(gl[q * nn + p]) > m) m = fabs(gl[q * nn + p]); }
                else m += gl[q * nn + p] * gl[q * nn + p];
            }
            if (w_norm != 0) m = sqrt(m);
        }
        if (s - 1.0 > di) di = s - 1.0;
        if (m - alpha > di) di = m - alpha;
    }
    double R = 0.0;
    if (pUx) {
        double *dUx = (double *)malloc(sizeof(double) * nk), *dUy = (double *)malloc(sizeof(double) * nk);
        double *dW = (double *)malloc(sizeof(double) * nw);
        double su = 0.0, sw = 0.0, sp = 0.0, cr = 0.0;
        for (size_t q = 0; q < nk; ++q) {
            dUx[q] = Ux[q] - pUx[q]; dUy[q] = Uy[q] - pUy[q];
            su += dUx[q] * dUx[q] + dUy[q] * dUy[q];
            sp += (Phi[q] - pPhi[q]) * (Phi[q] - pPhi[q]);
        }
        for (size_t q = 0; q < nw; ++q) { dW[q] = W[q] - pW[q]; sw += dW[q] * dW[q]; }
        orc_div(n, kk, dUx, dUy, dv);
        orc_div_L(n, k, N, L, dW, dl);
        for (size_t q = 0; q < nk; ++q) cr += (Phi[q] - pPhi[q]) * (dv[q] + dl[q]);
        R = su / mu + sw / nu + sp / tau - 2.0 * cr;
        free(dUx); free(dUy); free(dW);
    }
    out[0] = P;
    out[1] = D;
    out[2] = fabs(P - D) / (fabs(P) > 1e-300 ? fabs(P) : 1e-300);
    out[3] = sqrt(rr) / (bb > 0.0 ? sqrt(bb) : 1.0);
    out[4] = R;
    out[5] = di;
    free(dv); free(dl); free(gx); free(gy); free(gl);
}

/*
 * M-OMT by PDHG (Section 7.3):
 *   U^{t+1}_ij = shrink_u(U^t_ij + mu (grad Phi^t)_ij ; mu)
 *   W^{t+1}_ij = shrink_w(W^t_ij + nu (grad_L Phi^t_ij) ; alpha nu)
 *   Phi^{t+1}_ij = Phi^t_ij + tau (div_x(2U^{t+1} - U^t)_ij + div_L(2W^{t+1} - W^t)_ij
 *                                 + Lam1_ij - Lam0_ij)
 * on full k x k matrices; the Lemma of Appendix B (and its entrywise analogue
 * for ||.||_1) is why the shrinks can act on all of R^{k x k}.
 */
int orc_momt_solve(int n, int k, int N, const double *L, const double *Lam0, const double *Lam1,
                   double alpha, double tau, double mu, double nu, int u_norm, int w_norm,
                   int max_iters, int check_every, double tol_gap, double tol_res,
                   double *Ux, double *Uy, double *W, double *Phi,
                   double *metrics, double *history, int hist_cap)
{
    int kk = k * k;
    size_t nn = (size_t)n * n, nk = (size_t)kk * nn, nw = (size_t)N * kk * nn;
    double *gx = (double *)malloc(sizeof(double) * nk), *gy = (double *)malloc(sizeof(double) * nk);
    double *gl = (double *)malloc(sizeof(double) * nw);
    double *nUx = (double *)malloc(sizeof(double) * nk), *nUy = (double *)malloc(sizeof(double) * nk);
    double *nW = (double *)malloc(sizeof(double) * nw);
    double *bx = (double *)malloc(sizeof(double) * nk), *by = (double *)malloc(sizeof(double) * nk);
    double *bw = (double *)malloc(sizeof(double) * nw);
    double *dv = (double *)malloc(sizeof(double) * nk), *dl = (double *)malloc(sizeof(double) * nk);
    double *pPhi = (double *)malloc(sizeof(double) * nk);
    int nh = 0, t = 0;
    if (check_every <= 0) check_every = max_iters > 0 ? max_iters : 1;

    for (t = 1; t <= max_iters; ++t) {
        orc_grad(n, kk, Phi, gx, gy);
        ORC_PARALLEL_FOR
        for (size_t p = 0; p < nn; ++p) {
            double v[128], o[128];
            for (int q = 0; q < kk; ++q) {
                v[q] = Ux[q * nn + p] + mu * gx[q * nn + p];
                v[kk + q] = Uy[q * nn + p] + mu * gy[q * nn + p];
            }
            if (u_norm == 2) for (int q = 0; q < 2 * kk; ++q) o[q] = orc_shrink1(v[q], mu);
            else if (u_norm == 3) { orc_shrink_nuc(k, v, mu, o); orc_shrink_nuc(k, v + kk, mu, o + kk); }
            else orc_shrink2(2 * kk, v, mu, o);
            for (int q = 0; q < kk; ++q) { nUx[q * nn + p] = o[q]; nUy[q * nn + p] = o[kk + q]; }
        }
        orc_grad_L(n, k, N, L, Phi, gl);
        ORC_PARALLEL_FOR
        for (size_t p = 0; p < nn; ++p) {
            double xw[512], ow[512];
            for (int q = 0; q < N * kk; ++q) xw[q] = W[q * nn + p] + nu * gl[q * nn + p];
            if (w_norm == 0) for (int q = 0; q < N * kk; ++q) ow[q] = orc_shrink1(xw[q], alpha * nu);
            else if (w_norm == 2) for (int s_ = 0; s_ < N; ++s_) orc_shrink_nuc(k, xw + s_ * kk, alpha * nu, ow + s_ * kk);
            else orc_shrink2(N * kk, xw, alpha * nu, ow);
            for (int q = 0; q < N * kk; ++q) nW[q * nn + p] = ow[q];
        }
        for (size_t q = 0; q < nk; ++q) { bx[q] = 2.0 * nUx[q] - Ux[q]; by[q] = 2.0 * nUy[q] - Uy[q]; }
        for (size_t q = 0; q < nw; ++q) bw[q] = 2.0 * nW[q] - W[q];
        orc_div(n, kk, bx, by, dv);
        orc_div_L(n, k, N, L, bw, dl);
        memcpy(pPhi, Phi, sizeof(double) * nk);
        for (size_t q = 0; q < nk; ++q) Phi[q] = Phi[q] + tau * (dv[q] + dl[q] + Lam1[q] - Lam0[q]);

        int check = (t % check_every == 0) || (t == max_iters);
        double m[ORC_NMET];
        if (check) {
            orc_momt_metrics(n, k, N, L, Lam0, Lam1, alpha, u_norm, w_norm, mu, nu, tau,
                             nUx, nUy, nW, Phi, Ux, Uy, W, pPhi, m);
            m[6] = (double)t;
            m[7] = (tol_gap > 0.0 && m[2] <= tol_gap && m[3] <= tol_res) ? 1.0 : 0.0;
            if (history && nh < hist_cap) { memcpy(history + (size_t)nh * ORC_NMET, m, sizeof m); ++nh; }
            if (metrics) memcpy(metrics, m, sizeof m);
        }
        memcpy(Ux, nUx, sizeof(double) * nk);
        memcpy(Uy, nUy, sizeof(double) * nk);
        memcpy(W, nW, sizeof(double) * nw);
        if (check && m[7] != 0.0) break;
    }
    if (t > max_iters) t = max_iters;
    free(gx); free(gy); free(gl); free(nUx); free(nUy); free(nW); free(bx); free(by); free(bw);
    free(dv); free(dl); free(pPhi);
    return t;
}

/* ------------------------------------------------------------------------ */
/* Gradients of the transport cost                                            */
/* ------------------------------------------------------------------------ */

/*
 * Envelope gradient.  V(rho0, rho1) is the optimal value of the dual problem
 * (eq. vomt-dual), the maximum over the feasible phi of the linear function
 * <phi, rho1 - rho0>; the feasible set does not depend on the densities, so
 * dV/drho1 = phi* and dV/drho0 = -phi*, up to the constant that the dual
 * leaves free (grad and grad_G vanish on constants shared by all channels).
 * The constant is fixed by making phi* zero-mean over all cells and channels.
 * V is also the optimal value of the primal (eq. vomt), which is linear in
 * alpha for fixed (u, w), so dV/dalpha = sum_ij ||w*_ij||_w.
 */
void orc_envelope_grad(int n, int k, int l, int w_norm, const double *phi, const double *w,
                       double *g_rho1, double *g_rho0, double *g_alpha)
{
    size_t nk = (size_t)k * n * n, nn = (size_t)n * n;
    double mean = 0.0;
    for (size_t q = 0; q < nk; ++q) mean += phi[q];
    mean /= (double)nk;
    for (size_t q = 0; q < nk; ++q) { g_rho1[q] = phi[q] - mean; g_rho0[q] = -(phi[q] - mean); }
    double s = 0.0, x[64];
    for (size_t p = 0; p < nn; ++p) {
        for (int e = 0; e < l; ++e) x[e] = w[e * nn + p];
        s += norm_w_point(l, w_norm, x);
    }
    *g_alpha = s;
}

/* transpose of the Jacobian of shrink_2(.; t) at x, applied to g (symmetric):
 * (1 - t/s) g + t (x.g) x / s^3 for s = ||x|| > t, else 0.  Also returns the
 * derivative of the output with respect to the threshold t, dotted with g:
 * -(x.g)/s for s > t, else 0. */
static double shrink2_vjp(int m, const double *x, double t, const double *g, double *out)
{
    double s = 0.0, xg = 0.0;
    for (int q = 0; q < m; ++q) { s += x[q] * x[q]; xg += x[q] * g[q]; }
    s = sqrt(s);
    if (s <= t) { for (int q = 0; q < m; ++q) out[q] = 0.0; return 0.0; }
    for (int q = 0; q < m; ++q) out[q] = (1.0 - t / s) * g[q] + t * xg * x[q] / (s * s * s);
    return -xg / s;
}

static double shrink1_vjp(double x, double t, double g, double *out)
{
    if (fabs(x) <= t) { *out = 0.0; return 0.0; }
    *out = g;
    return -(x > 0 ? 1.0 : -1.0) * g;
}

/*
 * Unrolled gradient.  J_T = P(u^T, w^T), the primal objective after T
 * iterations of Section 7.2 from the zero iterate, is a piecewise-smooth
 * function of (rho0, rho1, alpha).  This routine stores every iterate and
 * applies the chain rule backwards through the T iterations, step by step:
 *   phi^{t+1} = phi^t + tau (div ubar + div_G wbar + rho1 - rho0)
 *   u^{t+1} = shrink_u(u^t + mu grad phi^t ; mu),  w^{t+1} = shrink_w(w^t + nu grad_G phi^t ; alpha nu)
 * using div_x^T = -grad_x (Appendix A) and div_G^T = -grad_G (Section 3.1).
 * Supports u_norm 0 (||.||_{1,2}) and w_norm 0 / 1.  Returns J_T.
 */
double orc_vomt_unrolled_grad(int n, int k, int l, const int *ea, const int *eb, const double *cost,
                              const double *rho0, const double *rho1, double alpha,
                              double tau, double mu, double nu, int w_norm, int T,
                              double *g_rho1, double *g_rho0, double *g_alpha)
{
    size_t nk = (size_t)k * n * n, nl = (size_t)l * n * n, nn = (size_t)n * n;
    size_t st = 3 * nk + nl;  /* ux, uy, phi, w */
    double *S = (double *)calloc(st * (size_t)(T + 1), sizeof(double));
    double met[ORC_NMET];
    /* forward, keeping every iterate */
    for (int t = 0; t < T; ++t) {
        double *cur = S + st * (size_t)t, *nxt = S + st * (size_t)(t + 1);
        memcpy(nxt, cur, sizeof(double) * st);
        orc_vomt_solve(n, k, l, ea, eb, cost, rho0, rho1, alpha, tau, mu, nu, 0, w_norm,
                       1, 1, 0.0, 0.0, nxt, nxt + nk, nxt + 3 * nk, nxt + 2 * nk, met, NULL, 0, 0.0);
    }
    double *fin = S + st * (size_t)T;
    double J = 0.0;
    /* adjoint of J wrt the final state */
    double *Gux = (double *)calloc(nk, sizeof(double)), *Guy = (double *)calloc(nk, sizeof(double));
    double *Gphi = (double *)calloc(nk, sizeof(double));
    double *Gw = (double *)calloc(nl ? nl : 1, sizeof(double));
    double ga = 0.0;
    for (size_t p = 0; p < nn; ++p) {
        for (int c = 0; c < k; ++c) {
            double x = fin[c * nn + p], y = fin[nk + c * nn + p], s = sqrt(x * x + y * y);
            J += s;
            if (s > 0) { Gux[c * nn + p] = x / s; Guy[c * nn + p] = y / s; }
        }
        double wv[64], ws = 0.0;
        for (int e = 0; e < l; ++e) wv[e] = fin[3 * nk + e * nn + p];
        ws = norm_w_point(l, w_norm, wv);
        J += alpha * ws;
        ga += ws;
        for (int e = 0; e < l; ++e) {
            double g;
            if (w_norm == 0) g = (wv[e] > 0) ? 1.0 : (wv[e] < 0 ? -1.0 : 0.0);
            else g = ws > 0 ? wv[e] / ws : 0.0;
            Gw[e * nn + p] = alpha * g;
        }
    }
    for (size_t q = 0; q < nk; ++q) { g_rho1[q] = 0.0; g_rho0[q] = 0.0; }

    double *gx = (double *)malloc(sizeof(double) * nk), *gy = (double *)malloc(sizeof(double) * nk);
    double *ggG = (double *)malloc(sizeof(double) * (nl ? nl : 1));
    double *Hx = (double *)malloc(sizeof(double) * nk), *Hy = (double *)malloc(sizeof(double) * nk);
    double *Hw = (double *)malloc(sizeof(double) * (nl ? nl : 1));
    double *gvx = (double *)malloc(sizeof(double) * nk), *gvy = (double *)malloc(sizeof(double) * nk);
    double *gxw = (double *)malloc(sizeof(double) * (nl ? nl : 1));
    double *dv = (double *)malloc(sizeof(double) * nk), *dg = (double *)malloc(sizeof(double) * nk);
    double *pgx = (double *)malloc(sizeof(double) * nk), *pgy = (double *)malloc(sizeof(double) * nk);
    double *pgG = (double *)malloc(sizeof(double) * (nl ? nl : 1));

    for (int t = T - 1; t >= 0; --t) {
        double *cur = S + st * (size_t)t;
        const double *ux = cur, *uy = cur + nk, *phi = cur + 2 * nk, *w = cur + 3 * nk;
        /* phi^{t+1} = phi^t + tau (div(2u' - u) + div_G(2w' - w) + rho1 - rho0) */
        for (size_t q = 0; q < nk; ++q) { g_rho1[q] += tau * Gphi[q]; g_rho0[q] -= tau * Gphi[q]; }
        orc_grad(n, k, Gphi, gx, gy);           /* div^T Gphi = -grad Gphi */
        if (l) orc_grad_G(n, k, l, ea, eb, cost, Gphi, ggG);
        for (size_t q = 0; q < nk; ++q) { Hx[q] = Gux[q] - 2.0 * tau * gx[q]; Hy[q] = Guy[q] - 2.0 * tau * gy[q]; }
        for (size_t q = 0; q < nl; ++q) Hw[q] = Gw[q] - 2.0 * tau * ggG[q];
        /* u' = shrink(u + mu grad phi; mu) per channel 2-vector */
        orc_grad(n, k, phi, pgx, pgy);
        for (size_t p = 0; p < nn; ++p)
            for (int c = 0; c < k; ++c) {
                size_t q = c * nn + p;
                double x[2] = {ux[q] + mu * pgx[q], uy[q] + mu * pgy[q]}, g[2] = {Hx[q], Hy[q]}, o[2];
                shrink2_vjp(2, x, mu, g, o);
                gvx[q] = o[0]; gvy[q] = o[1];
            }
        /* w' = shrink_w(w + nu grad_G phi; alpha nu) */
        if (l) {
            orc_grad_G(n, k, l, ea, eb, cost, phi, pgG);
            for (size_t p = 0; p < nn; ++p) {
                if (w_norm == 0) {
                    for (int e = 0; e < l; ++e) {
                        size_t q = e * nn + p;
                        double o;
                        double dt = shrink1_vjp(w[q] + nu * pgG[q], alpha * nu, Hw[q], &o);
                        gxw[q] = o;
                        ga += nu * dt;
                    }
                } else {
                    double x[64], g[64], o[64];
                    for (int e = 0; e < l; ++e) { x[e] = w[e * nn + p] + nu * pgG[e * nn + p]; g[e] = Hw[e * nn + p]; }
                    ga += nu * shrink2_vjp(l, x, alpha * nu, g, o);
                    for (int e = 0; e < l; ++e) gxw[e * nn + p] = o[e];
                }
            }
        }
        /* adjoints of the state at t */
        orc_div(n, k, gvx, gvy, dv);                       /* grad^T gv = -div gv */
        if (l) orc_div_G(n, k, l, ea, eb, cost, gxw, dg);  /* grad_G^T gx = -div_G gx */
        else for (size_t q = 0; q < nk; ++q) dg[q] = 0.0;
        for (size_t q = 0; q < nk; ++q) {
            Gux[q] = gvx[q] + tau * gx[q];
            Guy[q] = gvy[q] + tau * gy[q];
            Gphi[q] = Gphi[q] - mu * dv[q] - nu * dg[q];
        }
        for (size_t q = 0; q < nl; ++q) Gw[q] = gxw[q] + tau * ggG[q];
    }
    *g_alpha = ga;
    free(S); free(Gux); free(Guy); free(Gphi); free(Gw); free(gx); free(gy); free(ggG);
    free(Hx); free(Hy); free(Hw); free(gvx); free(gvy); free(gxw); free(dv); free(dg);
    free(pgx); free(pgy); free(pgG);
    return J;
}

/* ------------------------------------------------------------------------ */
/* 3-D grids (the extension to volumes the paper points to for 3-D DTI,       */
/* Section 8.2): the discretization of Appendix A with a third direction      */
/* ------------------------------------------------------------------------ */
/*
 * n x n x n cells on [0,1]^3, h = 1/(n-1); fields [c][z][y][x] with x fastest.
 * Flux components u_x, u_y, u_z per channel; u_x has its ghost entries at
 * x = n-1, u_y at y = n-1, u_z at z = n-1 (kept zero by the iteration).
 *   (grad phi)_d = (phi(. + e_d) - phi) / h, zero where . + e_d leaves the grid;
 *   div u = (u_x - u_x(x-1) + u_y - u_y(y-1) + u_z - u_z(z-1)) / h, with the
 *   terms before the first cell of a direction taken as zero.
 * Norms per point as in 2-D with three spatial components per channel:
 * ||u||_{1,2} = sum_c |(u_x, u_y, u_z)_c|_2, ||u||_2 joint, ||u||_1 entrywise.
 * Step rule (a reading: the paper states the 2-D rule only): ||grad||^2 <= 12 / h^2 in 3-D, so
 * mu = 1 / (48 tau (n-1)^2) keeps the 2-D rule's share of the bound
 * (8/32 = 12/48); nu as in 2-D.
 */
#define AT3(c, z, y, x) ((((size_t)(c) * (size_t)n + (size_t)(z)) * (size_t)n + (size_t)(y)) * (size_t)n + (size_t)(x))

void orc_grad3(int n, int planes, const double *phi, double *gx, double *gy, double *gz)
{
    double ih = (double)(n - 1);
    for (int c = 0; c < planes; ++c)
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    double p = phi[AT3(c, z, y, x)];
                    gx[AT3(c, z, y, x)] = (x < n - 1) ? ih * (phi[AT3(c, z, y, x + 1)] - p) : 0.0;
                    gy[AT3(c, z, y, x)] = (y < n - 1) ? ih * (phi[AT3(c, z, y + 1, x)] - p) : 0.0;
                    gz[AT3(c, z, y, x)] = (z < n - 1) ? ih * (phi[AT3(c, z + 1, y, x)] - p) : 0.0;
                }
}

void orc_div3(int n, int planes, const double *ux, const double *uy, const double *uz, double *out)
{
    double ih = (double)(n - 1);
    for (int c = 0; c < planes; ++c)
        for (int z = 0; z < n; ++z)
            for (int y = 0; y < n; ++y)
                for (int x = 0; x < n; ++x) {
                    double xl = (x > 0) ? ux[AT3(c, z, y, x - 1)] : 0.0;
                    double yl = (y > 0) ? uy[AT3(c, z, y - 1, x)] : 0.0;
                    double zl = (z > 0) ? uz[AT3(c, z - 1, y, x)] : 0.0;
                    out[AT3(c, z, y, x)] =
                        ih * (ux[AT3(c, z, y, x)] - xl + uy[AT3(c, z, y, x)] - yl + uz[AT3(c, z, y, x)] - zl);
                }
}

/* graph gradient and divergence at every one of m points (planes of m values) */
static void grad_G_pts(size_t m, int l, const int *ea, const int *eb, const double *cost, const double *phi,
                       double *g)
{
    for (int e = 0; e < l; ++e) {
        int lo = ea[e] < eb[e] ? ea[e] : eb[e], hi = ea[e] < eb[e] ? eb[e] : ea[e];
        double ic = 1.0 / edge_cost(cost, e);
        for (size_t p = 0; p < m; ++p) g[e * m + p] = ic * (phi[lo * m + p] - phi[hi * m + p]);
    }
}

static void div_G_pts(size_t m, int k, int l, const int *ea, const int *eb, const double *cost, const double *y,
                      double *out)
{
    for (size_t q = 0; q < (size_t)k * m; ++q) out[q] = 0.0;
    for (int e = 0; e < l; ++e) {
        int lo = ea[e] < eb[e] ? ea[e] : eb[e], hi = ea[e] < eb[e] ? eb[e] : ea[e];
        double ic = 1.0 / edge_cost(cost, e);
        for (size_t p = 0; p < m; ++p) {
            double v = ic * y[e * m + p];
            out[lo * m + p] -= v;
            out[hi * m + p] += v;
        }
    }
}

static void shrink_u3_point(int k, int u_norm, double t, double *vx, double *vy, double *vz)
{
    if (u_norm == 0) {
        for (int c = 0; c < k; ++c) {
            double v[3] = {vx[c], vy[c], vz[c]}, o[3];
            orc_shrink2(3, v, t, o);
            vx[c] = o[0]; vy[c] = o[1]; vz[c] = o[2];
        }
    } else if (u_norm == 1) {
        double v[96], o[96];
        for (int c = 0; c < k; ++c) { v[c] = vx[c]; v[k + c] = vy[c]; v[2 * k + c] = vz[c]; }
        orc_shrink2(3 * k, v, t, o);
        for (int c = 0; c < k; ++c) { vx[c] = o[c]; vy[c] = o[k + c]; vz[c] = o[2 * k + c]; }
    } else {
        for (int c = 0; c < k; ++c) {
            vx[c] = orc_shrink1(vx[c], t); vy[c] = orc_shrink1(vy[c], t); vz[c] = orc_shrink1(vz[c], t);
        }
    }
}

static double norm_u3_point(int k, int u_norm, const double *a, const double *b, const double *z)
{
    double s = 0.0;
    if (u_norm == 0) {
        for (int c = 0; c < k; ++c) s += sqrt(a[c] * a[c] + b[c] * b[c] + z[c] * z[c]);
    } else if (u_norm == 1) {
        for (int c = 0; c < k; ++c) s += a[c] * a[c] + b[c] * b[c] + z[c] * z[c];
        s = sqrt(s);
    } else {
        for (int c = 0; c < k; ++c) s += fabs(a[c]) + fabs(b[c]) + fabs(z[c]);
    }
    return s;
}

static double dualnorm_u3_point(int k, int u_norm, const double *a, const double *b, const double *z)
{
    double s = 0.0;
    if (u_norm == 0) {
        for (int c = 0; c < k; ++c) {
            double v = sqrt(a[c] * a[c] + b[c] * b[c] + z[c] * z[c]);
            if (v > s) s = v;
        }
    } else if (u_norm == 1) {
        for (int c = 0; c < k; ++c) s += a[c] * a[c] + b[c] * b[c] + z[c] * z[c];
        s = sqrt(s);
    } else {
        for (int c = 0; c < k; ++c) {
            if (fabs(a[c]) > s) s = fabs(a[c]);
            if (fabs(b[c]) > s) s = fabs(b[c]);
            if (fabs(z[c]) > s) s = fabs(z[c]);
        }
    }
    return s;
}

double orc_step_mu3(int n, double tau, int has_w)
{
    double n1 = (double)(n - 1);
    return has_w ? 1.0 / (48.0 * tau * n1 * n1) : 1.0 / (24.0 * tau * n1 * n1);
}

/* Metrics of a 3-D state (the same eight numbers as orc_vomt_metrics). */
void orc_vomt3_metrics(int n, int k, int l, const int *ea, const int *eb, const double *cost,
                       const double *rho0, const double *rho1, double alpha, int u_norm, int w_norm,
                       double mu, double nu, double tau,
                       const double *ux, const double *uy, const double *uz, const double *w, const double *phi,
                       const double *pux, const double *puy, const double *puz, const double *pw,
                       const double *pphi, double *out)
{
    size_t m = (size_t)n * n * n, nk = (size_t)k * m, nl = (size_t)l * m;
    double *dv = (double *)malloc(sizeof(double) * nk), *dg = (double *)malloc(sizeof(double) * nk);
    double *gx = (double *)malloc(sizeof(double) * nk), *gy = (double *)malloc(sizeof(double) * nk);
    double *gz = (double *)malloc(sizeof(double) * nk);
    double *gg = (double *)malloc(sizeof(double) * (nl ? nl : 1));
    double a[32], b[32], z[32], c3[64];
    double P = 0.0, D = 0.0, rr = 0.0, bb = 0.0, di = 0.0, R = 0.0;
    for (size_t p = 0; p < m; ++p) {
        for (int c = 0; c < k; ++c) { a[c] = ux[c * m + p]; b[c] = uy[c * m + p]; z[c] = uz[c * m + p]; }
        P += norm_u3_point(k, u_norm, a, b, z);
        for (int e = 0; e < l; ++e) c3[e] = w[e * m + p];
        P += alpha * norm_w_point(l, w_norm, c3);
    }
    for (size_t q = 0; q < nk; ++q) D += phi[q] * (rho1[q] - rho0[q]);
    orc_div3(n, k, ux, uy, uz, dv);
    div_G_pts(m, k, l, ea, eb, cost, w, dg);
    for (size_t q = 0; q < nk; ++q) {
        double r = dv[q] + dg[q] - (rho0[q] - rho1[q]);
        rr += r * r;
        bb += (rho0[q] - rho1[q]) * (rho0[q] - rho1[q]);
    }
    orc_grad3(n, k, phi, gx, gy, gz);
    if (l) grad_G_pts(m, l, ea, eb, cost, phi, gg);
    for (size_t p = 0; p < m; ++p) {
        for (int c = 0; c < k; ++c) { a[c] = gx[c * m + p]; b[c] = gy[c * m + p]; z[c] = gz[c * m + p]; }
        double v = dualnorm_u3_point(k, u_norm, a, b, z) - 1.0;
        if (v > di) di = v;
        if (l) {
            for (int e = 0; e < l; ++e) c3[e] = gg[e * m + p];
            v = dualnorm_w_point(l, w_norm, c3) - alpha;
            if (v > di) di = v;
        }
    }
    if (pux) {
        double *du[3], su = 0.0, sw = 0.0, sp = 0.0, cr = 0.0;
        double *dw = (double *)malloc(sizeof(double) * (nl ? nl : 1));
        const double *cu[3] = {ux, uy, uz}, *pu[3] = {pux, puy, puz};
        for (int d = 0; d < 3; ++d) {
            du[d] = (double *)malloc(sizeof(double) * nk);
            for (size_t q = 0; q < nk; ++q) { du[d][q] = cu[d][q] - pu[d][q]; su += du[d][q] * du[d][q]; }
        }
        for (size_t q = 0; q < nk; ++q) sp += (phi[q] - pphi[q]) * (phi[q] - pphi[q]);
        for (size_t q = 0; q < nl; ++q) { dw[q] = w[q] - pw[q]; sw += dw[q] * dw[q]; }
        orc_div3(n, k, du[0], du[1], du[2], dv);
        div_G_pts(m, k, l, ea, eb, cost, dw, dg);
        for (size_t q = 0; q < nk; ++q) cr += (phi[q] - pphi[q]) * (dv[q] + dg[q]);
        R = su / mu + (l ? sw / nu : 0.0) + sp / tau - 2.0 * cr;
        for (int d = 0; d < 3; ++d) free(du[d]);
        free(dw);
    }
    out[0] = P;
    out[1] = D;
    out[2] = fabs(P - D) / (fabs(P) > 1e-300 ? fabs(P) : 1e-300);
    out[3] = sqrt(rr) / (bb > 0.0 ? sqrt(bb) : 1.0);
    out[4] = R;
    out[5] = di;
    free(dv); free(dg); free(gx); free(gy); free(gz); free(gg);
}

/* V-OMT by PDHG on a 3-D grid: the loop of Section 7.2 with the 3-D operators. */
int orc_vomt3_solve(int n, int k, int l, const int *ea, const int *eb, const double *cost,
                    const double *rho0, const double *rho1, double alpha,
                    double tau, double mu, double nu, int u_norm, int w_norm,
                    int max_iters, int check_every, double tol_gap, double tol_res,
                    double *ux, double *uy, double *uz, double *w, double *phi,
                    double *metrics, double *history, int hist_cap)
{
    size_t m = (size_t)n * n * n, nk = (size_t)k * m, nl = (size_t)l * m;
    double *gx = (double *)malloc(sizeof(double) * nk), *gy = (double *)malloc(sizeof(double) * nk);
    double *gz = (double *)malloc(sizeof(double) * nk);
    double *nux = (double *)malloc(sizeof(double) * nk), *nuy = (double *)malloc(sizeof(double) * nk);
    double *nuz = (double *)malloc(sizeof(double) * nk);
    double *gg = (double *)malloc(sizeof(double) * (nl ? nl : 1)), *nw = (double *)malloc(sizeof(double) * (nl ? nl : 1));
    double *bx = (double *)malloc(sizeof(double) * nk), *by = (double *)malloc(sizeof(double) * nk);
    double *bz = (double *)malloc(sizeof(double) * nk), *bw = (double *)malloc(sizeof(double) * (nl ? nl : 1));
    double *dv = (double *)malloc(sizeof(double) * nk), *dg = (double *)malloc(sizeof(double) * nk);
    double *pphi = (double *)malloc(sizeof(double) * nk);
    double a[32], b[32], z[32], x[64];
    int nh = 0, t = 0;
    if (check_every <= 0) check_every = max_iters > 0 ? max_iters : 1;
    for (t = 1; t <= max_iters; ++t) {
        orc_grad3(n, k, phi, gx, gy, gz);
        for (size_t p = 0; p < m; ++p) {
            for (int c = 0; c < k; ++c) {
                a[c] = ux[c * m + p] + mu * gx[c * m + p];
                b[c] = uy[c * m + p] + mu * gy[c * m + p];
                z[c] = uz[c * m + p] + mu * gz[c * m + p];
            }
            shrink_u3_point(k, u_norm, mu, a, b, z);
            for (int c = 0; c < k; ++c) { nux[c * m + p] = a[c]; nuy[c * m + p] = b[c]; nuz[c * m + p] = z[c]; }
        }
        if (l) {
            grad_G_pts(m, l, ea, eb, cost, phi, gg);
            for (size_t p = 0; p < m; ++p) {
                for (int e = 0; e < l; ++e) x[e] = w[e * m + p] + nu * gg[e * m + p];
                shrink_w_point(l, w_norm, alpha * nu, x);
                for (int e = 0; e < l; ++e) nw[e * m + p] = x[e];
            }
        }
        for (size_t q = 0; q < nk; ++q) {
            bx[q] = 2.0 * nux[q] - ux[q]; by[q] = 2.0 * nuy[q] - uy[q]; bz[q] = 2.0 * nuz[q] - uz[q];
        }
        for (size_t q = 0; q < nl; ++q) bw[q] = 2.0 * nw[q] - w[q];
        orc_div3(n, k, bx, by, bz, dv);
        if (l) div_G_pts(m, k, l, ea, eb, cost, bw, dg);
        else for (size_t q = 0; q < nk; ++q) dg[q] = 0.0;
        memcpy(pphi, phi, sizeof(double) * nk);
        for (size_t q = 0; q < nk; ++q) phi[q] = phi[q] + tau * (dv[q] + dg[q] + rho1[q] - rho0[q]);
        int check = (t % check_every == 0) || (t == max_iters);
        double met[ORC_NMET];
        if (check) {
            orc_vomt3_metrics(n, k, l, ea, eb, cost, rho0, rho1, alpha, u_norm, w_norm, mu, nu, tau,
                              nux, nuy, nuz, nw, phi, ux, uy, uz, w, pphi, met);
            met[6] = (double)t;
            met[7] = (tol_gap > 0.0 && met[2] <= tol_gap && met[3] <= tol_res) ? 1.0 : 0.0;
            if (history && nh < hist_cap) { memcpy(history + (size_t)nh * ORC_NMET, met, sizeof met); ++nh; }
            if (metrics) memcpy(metrics, met, sizeof met);
        }
        memcpy(ux, nux, sizeof(double) * nk);
        memcpy(uy, nuy, sizeof(double) * nk);
        memcpy(uz, nuz, sizeof(double) * nk);
        if (l) memcpy(w, nw, sizeof(double) * nl);
        if (check && met[7] != 0.0) break;
    }
    if (t > max_iters) t = max_iters;
    free(gx); free(gy); free(gz); free(nux); free(nuy); free(nuz); free(gg); free(nw);
    free(bx); free(by); free(bz); free(bw); free(dv); free(dg); free(pphi);
    return t;
}

/* ------------------------------------------------------------------------ */
/* Matrix OMT on 3-D grids                                                    */
/* ------------------------------------------------------------------------ */

/*
 * The matrix problem of Sections 4-5 and the iteration of Section 7.3 on an
 * n x n x n grid: U has three directions U_x, U_y, U_z, each a full k x k
 * matrix per point ([k*k][n][n][n] planes, the 3-D gradient and divergence of
 * Appendix A applied entrywise), W and grad_L as in 2-D.  Norms:
 * u_norm 1: ||U||_2, the Frobenius norm over the three directions jointly;
 * 2: entrywise ||U||_1; 3: ||U||_{1,nuc} = sum_d ||U_d||_nuc.  w_norm as in
 * orc_momt_metrics.
 */
static double momt3_norm_u(int k, int u_norm, const double *a, const double *b, const double *c)
{
    int kk = k * k;
    double s = 0.0;
    if (u_norm == 3) return orc_nuc_norm(k, a) + orc_nuc_norm(k, b) + orc_nuc_norm(k, c);
    for (int q = 0; q < kk; ++q) {
        if (u_norm == 2) s += fabs(a[q]) + fabs(b[q]) + fabs(c[q]);
        else s += a[q] * a[q] + b[q] * b[q] + c[q] * c[q];
    }
    return u_norm == 2 ? s : sqrt(s);
}

static double momt3_dualnorm_u(int k, int u_norm, const double *a, const double *b, const double *c)
{
    int kk = k * k;
    double s = 0.0;
    if (u_norm == 3) {
        double v = orc_spectral_norm(k, a), v2 = orc_spectral_norm(k, b), v3 = orc_spectral_norm(k, c);
        if (v2 > v) v = v2;
        if (v3 > v) v = v3;
        return v;
    }
    for (int q = 0; q < kk; ++q) {
        if (u_norm == 2) {
            if (fabs(a[q]) > s) s = fabs(a[q]);
            if (fabs(b[q]) > s) s = fabs(b[q]);
            if (fabs(c[q]) > s) s = fabs(c[q]);
        } else {
            s += a[q] * a[q] + b[q] * b[q] + c[q] * c[q];
        }
    }
    return u_norm == 2 ? s : sqrt(s);
}

static double momt_norm_w(int k, int N, int w_norm, const double *w)
{
    int kk = k * k;
    double s = 0.0;
    if (w_norm == 2) {
        for (int s_ = 0; s_ < N; ++s_) s += orc_nuc_norm(k, w + s_ * kk);
        return s;
    }
    for (int q = 0; q < N * kk; ++q) s += w_norm == 0 ? fabs(w[q]) : w[q] * w[q];
    return w_norm == 0 ? s : sqrt(s);
}

static double momt_dualnorm_w(int k, int N, int w_norm, const double *g)
{
    int kk = k * k;
    double m = 0.0;
    if (w_norm == 2) {
        for (int s_ = 0; s_ < N; ++s_) {
            double v = orc_spectral_norm(k, g + s_ * kk);
            if (v > m) m = v;
        }
        return m;
    }
    for (int q = 0; q < N * kk; ++q) {
        if (w_norm == 0) { if (fabs(g[q]) > m) m = fabs(g[q]); }
        else m += g[q] * g[q];
    }
    return w_norm == 0 ? m : sqrt(m);
}

void orc_momt3_metrics(int n, int k, int N, const double *L, const double *Lam0, const double *Lam1,
                       double alpha, int u_norm, int w_norm, double mu, double nu, double tau,
                       const double *Ux, const double *Uy, const double *Uz, const double *W, const double *Phi,
                       const double *pUx, const double *pUy, const double *pUz, const double *pW,
                       const double *pPhi, double *out)
{
    int kk = k * k;
    size_t m = (size_t)n * n * n, nk = (size_t)kk * m, nw = (size_t)N * kk * m;
    double *dv = (double *)malloc(sizeof(double) * nk), *dl = (double *)malloc(sizeof(double) * nk);
    double *gx = (double *)malloc(sizeof(double) * nk), *gy = (double *)malloc(sizeof(double) * nk);
    double *gz = (double *)malloc(sizeof(double) * nk), *gl = (double *)malloc(sizeof(double) * nw);
    double A[64], B[64], C[64], X[8 * 64];
    double P = 0.0, D = 0.0, rr = 0.0, bb = 0.0, di = 0.0, R = 0.0;
    for (size_t p = 0; p < m; ++p) {
        for (int q = 0; q < kk; ++q) { A[q] = Ux[q * m + p]; B[q] = Uy[q * m + p]; C[q] = Uz[q * m + p]; }
        for (int q = 0; q < N * kk; ++q) X[q] = W[q * m + p];
        P += momt3_norm_u(k, u_norm, A, B, C) + alpha * momt_norm_w(k, N, w_norm, X);
    }
    for (size_t q = 0; q < nk; ++q) D += Phi[q] * (Lam1[q] - Lam0[q]);
    orc_div3(n, kk, Ux, Uy, Uz, dv);
    for (size_t p = 0; p < m; ++p) {            /* div_L per point on the 3-D grid */
        for (int q = 0; q < N * kk; ++q) X[q] = W[q * m + p];
        orc_div_L_point(k, N, L, X, A);
        for (int q = 0; q < kk; ++q) dl[q * m + p] = A[q];
    }
    for (size_t q = 0; q < nk; ++q) {
        double r = dv[q] + dl[q] - (Lam0[q] - Lam1[q]);
        rr += r * r;
        bb += (Lam0[q] - Lam1[q]) * (Lam0[q] - Lam1[q]);
    }
    orc_grad3(n, kk, Phi, gx, gy, gz);
    for (size_t p = 0; p < m; ++p) {
        for (int q = 0; q < kk; ++q) { A[q] = gx[q * m + p]; B[q] = gy[q * m + p]; C[q] = gz[q * m + p]; }
        double v = momt3_dualnorm_u(k, u_norm, A, B, C) - 1.0;
        if (v > di) di = v;
        for (int q = 0; q < kk; ++q) A[q] = Phi[q * m + p];
        orc_grad_L_point(k, N, L, A, X);
        v = momt_dualnorm_w(k, N, w_norm, X) - alpha;
        if (v > di) di = v;
    }
    if (pUx) {
        double su = 0.0, sw = 0.0, sp = 0.0, cr = 0.0;
        double *du[3];
        const double *cu[3] = {Ux, Uy, Uz}, *pu[3] = {pUx, pUy, pUz};
        for (int d = 0; d < 3; ++d) {
            du[d] = (double *)malloc(sizeof(double) * nk);
            for (size_t q = 0; q < nk; ++q) { du[d][q] = cu[d][q] - pu[d][q]; su += du[d][q] * du[d][q]; }
        }
        for (size_t q = 0; q < nk; ++q) sp += (Phi[q] - pPhi[q]) * (Phi[q] - pPhi[q]);
        for (size_t q = 0; q < nw; ++q) sw += (W[q] - pW[q]) * (W[q] - pW[q]);
        orc_div3(n, kk, du[0], du[1], du[2], dv);
        for (size_t p = 0; p < m; ++p) {
            for (int q = 0; q < N * kk; ++q) X[q] = W[q * m + p] - pW[q * m + p];
            orc_div_L_point(k, N, L, X, A);
            for (int q = 0; q < kk; ++q) dl[q * m + p] = A[q];
        }
        for (size_t q = 0; q < nk; ++q) cr += (Phi[q] - pPhi[q]) * (dv[q] + dl[q]);
        R = su / mu + sw / nu + sp / tau - 2.0 * cr;
        for (int d = 0; d < 3; ++d) free(du[d]);
    }
    out[0] = P;
    out[1] = D;
    out[2] = fabs(P - D) / (fabs(P) > 1e-300 ? fabs(P) : 1e-300);
    out[3] = sqrt(rr) / (bb > 0.0 ? sqrt(bb) : 1.0);
    out[4] = R;
    out[5] = di;
    free(dv); free(dl); free(gx); free(gy); free(gz); free(gl);
}

/* The M-OMT iteration of Section 7.3 on the 3-D grid (the steps of orc_momt_solve
 * with a third direction). */
int orc_momt3_solve(int n, int k, int N, const double *L, const double *Lam0, const double *Lam1,
                    double alpha, double tau, double mu, double nu, int u_norm, int w_norm,
                    int max_iters, int check_every, double tol_gap, double tol_res,
                    double *Ux, double *Uy, double *Uz, double *W, double *Phi,
                    double *metrics, double *history, int hist_cap)
{
    int kk = k * k;
    size_t m = (size_t)n * n * n, nk = (size_t)kk * m, nw = (size_t)N * kk * m;
    double *g[3], *nU[3], *bu[3];
    for (int d = 0; d < 3; ++d) {
        g[d] = (double *)malloc(sizeof(double) * nk);
        nU[d] = (double *)malloc(sizeof(double) * nk);
        bu[d] = (double *)malloc(sizeof(double) * nk);
    }
    double *U[3] = {Ux, Uy, Uz};
    double *nW = (double *)malloc(sizeof(double) * nw), *bw = (double *)malloc(sizeof(double) * nw);
    double *dv = (double *)malloc(sizeof(double) * nk), *dl = (double *)malloc(sizeof(double) * nk);
    double *pPhi = (double *)malloc(sizeof(double) * nk);
    double v[3 * 64], o[3 * 64], xw[8 * 64], ow[8 * 64], A[64];
    int nh = 0, t = 0;
    if (check_every <= 0) check_every = max_iters > 0 ? max_iters : 1;
    for (t = 1; t <= max_iters; ++t) {
        orc_grad3(n, kk, Phi, g[0], g[1], g[2]);
        for (size_t p = 0; p < m; ++p) {
            for (int d = 0; d < 3; ++d)
                for (int q = 0; q < kk; ++q) v[d * kk + q] = U[d][q * m + p] + mu * g[d][q * m + p];
            if (u_norm == 2) for (int q = 0; q < 3 * kk; ++q) o[q] = orc_shrink1(v[q], mu);
            else if (u_norm == 3) for (int d = 0; d < 3; ++d) orc_shrink_nuc(k, v + d * kk, mu, o + d * kk);
            else orc_shrink2(3 * kk, v, mu, o);
            for (int d = 0; d < 3; ++d)
                for (int q = 0; q < kk; ++q) nU[d][q * m + p] = o[d * kk + q];
        }
        for (size_t p = 0; p < m; ++p) {
            for (int q = 0; q < kk; ++q) A[q] = Phi[q * m + p];
            orc_grad_L_point(k, N, L, A, xw);
            for (int q = 0; q < N * kk; ++q) xw[q] = W[q * m + p] + nu * xw[q];
            if (w_norm == 0) for (int q = 0; q < N * kk; ++q) ow[q] = orc_shrink1(xw[q], alpha * nu);
            else if (w_norm == 2) for (int s_ = 0; s_ < N; ++s_) orc_shrink_nuc(k, xw + s_ * kk, alpha * nu, ow + s_ * kk);
            else orc_shrink2(N * kk, xw, alpha * nu, ow);
            for (int q = 0; q < N * kk; ++q) nW[q * m + p] = ow[q];
        }
        for (int d = 0; d < 3; ++d)
            for (size_t q = 0; q < nk; ++q) bu[d][q] = 2.0 * nU[d][q] - U[d][q];
        for (size_t q = 0; q < nw; ++q) bw[q] = 2.0 * nW[q] - W[q];
        orc_div3(n, kk, bu[0], bu[1], bu[2], dv);
        for (size_t p = 0; p < m; ++p) {
            for (int q = 0; q < N * kk; ++q) xw[q] = bw[q * m + p];
            orc_div_L_point(k, N, L, xw, A);
            for (int q = 0; q < kk; ++q) dl[q * m + p] = A[q];
        }
        memcpy(pPhi, Phi, sizeof(double) * nk);
        for (size_t q = 0; q < nk; ++q) Phi[q] = Phi[q] + tau * (dv[q] + dl[q] + Lam1[q] - Lam0[q]);
        int check = (t % check_every == 0) || (t == max_iters);
        double mm[ORC_NMET];
        if (check) {
            orc_momt3_metrics(n, k, N, L, Lam0, Lam1, alpha, u_norm, w_norm, mu, nu, tau, nU[0], nU[1], nU[2],
                              nW, Phi, Ux, Uy, Uz, W, pPhi, mm);
            mm[6] = (double)t;
            mm[7] = (tol_gap > 0.0 && mm[2] <= tol_gap && mm[3] <= tol_res) ? 1.0 : 0.0;
            if (history && nh < hist_cap) { memcpy(history + (size_t)nh * ORC_NMET, mm, sizeof mm); ++nh; }
            if (metrics) memcpy(metrics, mm, sizeof mm);
        }
        for (int d = 0; d < 3; ++d) memcpy(U[d], nU[d], sizeof(double) * nk);
        memcpy(W, nW, sizeof(double) * nw);
        if (check && mm[7] != 0.0) break;
    }
    if (t > max_iters) t = max_iters;
    for (int d = 0; d < 3; ++d) { free(g[d]); free(nU[d]); free(bu[d]); }
    free(nW); free(bw); free(dv); free(dl); free(pPhi);
    return t;
}

/* ------------------------------------------------------------------------ */
/* Complex Hermitian matrix OMT (Section 4 in the complex setting)           */
/* ------------------------------------------------------------------------ */

/*
 * Section 4 states matrix OMT for complex Hermitian densities: Lambda(x) is a
 * positive semidefinite Hermitian k x k matrix, U_x, U_y are Hermitian,
 * grad_L X = [L_l X - X L_l]_l with Hermitian L_l maps to skew-Hermitian
 * matrices, div_L Z = sum_s (-L_s Z_s + Z_s L_s), and every inner product is
 * the Hilbert-Schmidt one, <X, Y> = Re tr(X Y*) (the real inner product of
 * C^{k x k} seen as R^{2k^2}).  Norms here: ||U||_2 and ||W||_2, the Frobenius
 * norms (sum of |entry|^2 over everything, square root), whose shrink scales
 * the whole point's flux.  The iteration is that of Section 7.3.  Arrays are
 * complex planes [q][j][i] (q = a*k + b), C99 double complex.
 */
typedef double complex zdbl;

static void zmatmul(int k, const zdbl *A, const zdbl *B, zdbl *C)
{
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            zdbl s = 0.0;
            for (int q = 0; q < k; ++q) s += A[a * k + q] * B[q * k + b];
            C[a * k + b] = s;
        }
}

/* Z_s = L_s X - X L_s for one point. */
void orc_zgrad_L_point(int k, int N, const zdbl *L, const zdbl *X, zdbl *Z)
{
    zdbl t1[64], t2[64];
    for (int s = 0; s < N; ++s) {
        zmatmul(k, L + (size_t)s * k * k, X, t1);
        zmatmul(k, X, L + (size_t)s * k * k, t2);
        for (int q = 0; q < k * k; ++q) Z[(size_t)s * k * k + q] = t1[q] - t2[q];
    }
}

/* Y = sum_s (-L_s Z_s + Z_s L_s) for one point. */
void orc_zdiv_L_point(int k, int N, const zdbl *L, const zdbl *Z, zdbl *Y)
{
    zdbl t1[64], t2[64];
    for (int q = 0; q < k * k; ++q) Y[q] = 0.0;
    for (int s = 0; s < N; ++s) {
        zmatmul(k, L + (size_t)s * k * k, Z + (size_t)s * k * k, t1);
        zmatmul(k, Z + (size_t)s * k * k, L + (size_t)s * k * k, t2);
        for (int q = 0; q < k * k; ++q) Y[q] += -t1[q] + t2[q];
    }
}

/* Appendix A's forward-difference gradient and backward-difference divergence,
 * entrywise on complex planes (the same stencils as orc_grad / orc_div). */
static void zgrad(int n, int planes, const zdbl *phi, zdbl *gx, zdbl *gy)
{
    double ih = (double)(n - 1);
    for (int c = 0; c < planes; ++c)
        ORC_PARALLEL_FOR
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                gx[AT(c, j, i)] = (i < n - 1) ? ih * (phi[AT(c, j, i + 1)] - phi[AT(c, j, i)]) : 0.0;
                gy[AT(c, j, i)] = (j < n - 1) ? ih * (phi[AT(c, j + 1, i)] - phi[AT(c, j, i)]) : 0.0;
            }
}

static void zdiv(int n, int planes, const zdbl *ux, const zdbl *uy, zdbl *out)
{
    double ih = (double)(n - 1);
    for (int c = 0; c < planes; ++c)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                zdbl xl = (i > 0) ? ux[AT(c, j, i - 1)] : 0.0;
                zdbl yl = (j > 0) ? uy[AT(c, j - 1, i)] : 0.0;
                out[AT(c, j, i)] = ih * (ux[AT(c, j, i)] - xl + uy[AT(c, j, i)] - yl);
            }
}

/* lambda_max(-Delta_L) with -Delta_L X = sum_s [L_s, [L_s, X]] acting on all of
 * C^{k x k}, as a real symmetric 2k^2 x 2k^2 matrix (real parts, then imaginary
 * parts) assembled column by column. */
double orc_zquantum_lmax(int k, int N, const zdbl *L)
{
    int kk = k * k, m = 2 * kk;
    double *M = (double *)calloc((size_t)m * m, sizeof(double));
    double *ev = (double *)malloc(sizeof(double) * m);
    zdbl X[64], Z[8 * 64], Y[64];
    for (int col = 0; col < m; ++col) {
        for (int q = 0; q < kk; ++q) X[q] = 0.0;
        X[col % kk] = col < kk ? 1.0 : I;
        orc_zgrad_L_point(k, N, L, X, Z);
        orc_zdiv_L_point(k, N, L, Z, Y);            /* div grad = Delta_L */
        for (int q = 0; q < kk; ++q) {
            M[(size_t)q * m + col] = -creal(Y[q]);
            M[(size_t)(kk + q) * m + col] = -cimag(Y[q]);
        }
    }
    orc_jacobi_eigvals(m, M, ev);
    double mx = ev[0];
    for (int q = 1; q < m; ++q) if (ev[q] > mx) mx = ev[q];
    free(M); free(ev);
    return mx;
}

static double zsq(zdbl z) { return creal(z) * creal(z) + cimag(z) * cimag(z); }

/* Frobenius shrink of m complex entries jointly (Appendix B, shrink_2). */
static void zshrink2(int m, const zdbl *x, double t, zdbl *out)
{
    double s = 0.0;
    for (int q = 0; q < m; ++q) s += zsq(x[q]);
    s = sqrt(s);
    double f = (s > t) ? 1.0 - t / s : 0.0;
    for (int q = 0; q < m; ++q) out[q] = f * x[q];
}

/* Entrywise modulus shrink of m complex entries: the prox of t sum_q |z_q|, which
 * scales each entry by max(0, 1 - t / |z_q|) (shrink_2 of Appendix B on each entry
 * seen as a point of the plane). */
static void zshrink1(int m, const zdbl *x, double t, zdbl *out)
{
    for (int q = 0; q < m; ++q) {
        const double a = cabs(x[q]);
        out[q] = (a > t) ? (1.0 - t / a) * x[q] : 0.0;
    }
}

/* Norms of the complex setting (Section 6.2): the Frobenius norm ||.||_2 (square
 * root of the summed squared moduli) or, `entrywise`, ||.||_1 (the summed moduli of
 * the entries).  Their duals: the Frobenius norm and the largest modulus.  Codes as
 * for real matrices: u_norm 1 = ||U||_2, 2 = ||U||_1; w_norm 1 = ||W||_2, 0 = ||W||_1. */
static double znorm(int m, const zdbl *x, int entrywise)
{
    double s = 0.0;
    if (entrywise) { for (int q = 0; q < m; ++q) s += cabs(x[q]); return s; }
    for (int q = 0; q < m; ++q) s += zsq(x[q]);
    return sqrt(s);
}

static double zdualnorm(int m, const zdbl *x, int entrywise)
{
    double s = 0.0;
    if (entrywise) { for (int q = 0; q < m; ++q) if (cabs(x[q]) > s) s = cabs(x[q]); return s; }
    for (int q = 0; q < m; ++q) s += zsq(x[q]);
    return sqrt(s);
}

void orc_zmomt_metrics(int n, int k, int N, const zdbl *L, const zdbl *Lam0, const zdbl *Lam1, double alpha,
                       int u_norm, int w_norm, double mu, double nu, double tau, const zdbl *Ux, const zdbl *Uy,
                       const zdbl *W, const zdbl *Phi, const zdbl *pUx, const zdbl *pUy, const zdbl *pW,
                       const zdbl *pPhi, double *out)
{
    int kk = k * k;
    size_t nn = (size_t)n * n, nk = (size_t)kk * nn;
    zdbl *dv = (zdbl *)malloc(sizeof(zdbl) * nk), *dl = (zdbl *)malloc(sizeof(zdbl) * nk);
    zdbl *gx = (zdbl *)malloc(sizeof(zdbl) * nk), *gy = (zdbl *)malloc(sizeof(zdbl) * nk);
    zdbl X[64], Z[8 * 64], Y[64];
    double P = 0.0, D = 0.0, rr = 0.0, bb = 0.0, di = 0.0, R = 0.0;
    for (size_t p = 0; p < nn; ++p) {
        zdbl u2[128];                /* U_x and U_y of this point, side by side */
        for (int q = 0; q < kk; ++q) { u2[q] = Ux[q * nn + p]; u2[kk + q] = Uy[q * nn + p]; }
        for (int q = 0; q < N * kk; ++q) Z[q] = W[q * nn + p];
        P += znorm(2 * kk, u2, u_norm == 2) + alpha * znorm(N * kk, Z, w_norm == 0);
    }
    for (size_t q = 0; q < nk; ++q) D += creal(Phi[q] * conj(Lam1[q] - Lam0[q]));
    zdiv(n, kk, Ux, Uy, dv);
    for (size_t p = 0; p < nn; ++p) {
        for (int q = 0; q < N * kk; ++q) Z[q] = W[q * nn + p];
        orc_zdiv_L_point(k, N, L, Z, Y);
        for (int q = 0; q < kk; ++q) dl[q * nn + p] = Y[q];
    }
    for (size_t q = 0; q < nk; ++q) {
        rr += zsq(dv[q] + dl[q] - (Lam0[q] - Lam1[q]));
        bb += zsq(Lam0[q] - Lam1[q]);
    }
    zgrad(n, kk, Phi, gx, gy);
    for (size_t p = 0; p < nn; ++p) {
        zdbl g2[128];
        for (int q = 0; q < kk; ++q) { g2[q] = gx[q * nn + p]; g2[kk + q] = gy[q * nn + p]; X[q] = Phi[q * nn + p]; }
        orc_zgrad_L_point(k, N, L, X, Z);
        const double s = zdualnorm(2 * kk, g2, u_norm == 2), w2 = zdualnorm(N * kk, Z, w_norm == 0);
        if (s - 1.0 > di) di = s - 1.0;
        if (w2 - alpha > di) di = w2 - alpha;
    }
    if (pUx) {
        size_t nw = (size_t)N * kk * nn;
        zdbl *dUx = (zdbl *)malloc(sizeof(zdbl) * nk), *dUy = (zdbl *)malloc(sizeof(zdbl) * nk);
        zdbl *dW = (zdbl *)malloc(sizeof(zdbl) * nw);
        double su = 0.0, sw = 0.0, sp = 0.0, cr = 0.0;
        for (size_t q = 0; q < nk; ++q) {
            dUx[q] = Ux[q] - pUx[q]; dUy[q] = Uy[q] - pUy[q];
            su += zsq(dUx[q]) + zsq(dUy[q]);
            sp += zsq(Phi[q] - pPhi[q]);
        }
        for (size_t q = 0; q < nw; ++q) { dW[q] = W[q] - pW[q]; sw += zsq(dW[q]); }
        zdiv(n, kk, dUx, dUy, dv);
        for (size_t p = 0; p < nn; ++p) {
            for (int q = 0; q < N * kk; ++q) Z[q] = dW[q * nn + p];
            orc_zdiv_L_point(k, N, L, Z, Y);
            for (int q = 0; q < kk; ++q) dl[q * nn + p] = Y[q];
        }
        for (size_t q = 0; q < nk; ++q) cr += creal((Phi[q] - pPhi[q]) * conj(dv[q] + dl[q]));
        R = su / mu + sw / nu + sp / tau - 2.0 * cr;
        free(dUx); free(dUy); free(dW);
    }
    out[0] = P;
    out[1] = D;
    out[2] = fabs(P - D) / (fabs(P) > 1e-300 ? fabs(P) : 1e-300);
    out[3] = sqrt(rr) / (bb > 0.0 ? sqrt(bb) : 1.0);
    out[4] = R;
    out[5] = di;
    free(dv); free(dl); free(gx); free(gy);
}

/* The M-OMT iteration of Section 7.3 on complex Hermitian fields, with the
 * Frobenius norms or the entrywise ||.||_1 (whose shrink acts on each complex entry
 * by its modulus; Hermitian and skew-Hermitian structure is kept because an entry and
 * its mirror have the same modulus). */
int orc_zmomt_solve(int n, int k, int N, const zdbl *L, const zdbl *Lam0, const zdbl *Lam1, double alpha,
                    int u_norm, int w_norm, double tau, double mu, double nu, int max_iters, int check_every,
                    double tol_gap, double tol_res, zdbl *Ux, zdbl *Uy, zdbl *W, zdbl *Phi, double *metrics,
                    double *history, int hist_cap)
{
    int kk = k * k;
    size_t nn = (size_t)n * n, nk = (size_t)kk * nn, nw = (size_t)N * kk * nn;
    zdbl *gx = (zdbl *)malloc(sizeof(zdbl) * nk), *gy = (zdbl *)malloc(sizeof(zdbl) * nk);
    zdbl *nUx = (zdbl *)malloc(sizeof(zdbl) * nk), *nUy = (zdbl *)malloc(sizeof(zdbl) * nk);
    zdbl *nW = (zdbl *)malloc(sizeof(zdbl) * nw), *bw = (zdbl *)malloc(sizeof(zdbl) * nw);
    zdbl *bx = (zdbl *)malloc(sizeof(zdbl) * nk), *by = (zdbl *)malloc(sizeof(zdbl) * nk);
    zdbl *dv = (zdbl *)malloc(sizeof(zdbl) * nk), *dl = (zdbl *)malloc(sizeof(zdbl) * nk);
    zdbl *pPhi = (zdbl *)malloc(sizeof(zdbl) * nk);
    zdbl v[128], o[128], X[64], xw[8 * 64], ow[8 * 64], Y[64];
    int nh = 0, t = 0;
    if (check_every <= 0) check_every = max_iters > 0 ? max_iters : 1;
    for (t = 1; t <= max_iters; ++t) {
        zgrad(n, kk, Phi, gx, gy);
        for (size_t p = 0; p < nn; ++p) {
            for (int q = 0; q < kk; ++q) {
                v[q] = Ux[q * nn + p] + mu * gx[q * nn + p];
                v[kk + q] = Uy[q * nn + p] + mu * gy[q * nn + p];
            }
            if (u_norm == 2) zshrink1(2 * kk, v, mu, o);
            else zshrink2(2 * kk, v, mu, o);
            for (int q = 0; q < kk; ++q) { nUx[q * nn + p] = o[q]; nUy[q * nn + p] = o[kk + q]; }
        }
        for (size_t p = 0; p < nn; ++p) {
            for (int q = 0; q < kk; ++q) X[q] = Phi[q * nn + p];
            orc_zgrad_L_point(k, N, L, X, xw);
            for (int q = 0; q < N * kk; ++q) xw[q] = W[q * nn + p] + nu * xw[q];
            if (w_norm == 0) zshrink1(N * kk, xw, alpha * nu, ow);
            else zshrink2(N * kk, xw, alpha * nu, ow);
            for (int q = 0; q < N * kk; ++q) nW[q * nn + p] = ow[q];
        }
        for (size_t q = 0; q < nk; ++q) { bx[q] = 2.0 * nUx[q] - Ux[q]; by[q] = 2.0 * nUy[q] - Uy[q]; }
        for (size_t q = 0; q < nw; ++q) bw[q] = 2.0 * nW[q] - W[q];
        zdiv(n, kk, bx, by, dv);
        for (size_t p = 0; p < nn; ++p) {
            for (int q = 0; q < N * kk; ++q) xw[q] = bw[q * nn + p];
            orc_zdiv_L_point(k, N, L, xw, Y);
            for (int q = 0; q < kk; ++q) dl[q * nn + p] = Y[q];
        }
        memcpy(pPhi, Phi, sizeof(zdbl) * nk);
        for (size_t q = 0; q < nk; ++q) Phi[q] = Phi[q] + tau * (dv[q] + dl[q] + Lam1[q] - Lam0[q]);
        int check = (t % check_every == 0) || (t == max_iters);
        double m[ORC_NMET];
        if (check) {
            orc_zmomt_metrics(n, k, N, L, Lam0, Lam1, alpha, u_norm, w_norm, mu, nu, tau, nUx, nUy, nW, Phi, Ux, Uy,
                              W, pPhi, m);
            m[6] = (double)t;
            m[7] = (tol_gap > 0.0 && m[2] <= tol_gap && m[3] <= tol_res) ? 1.0 : 0.0;
            if (history && nh < hist_cap) { memcpy(history + (size_t)nh * ORC_NMET, m, sizeof m); ++nh; }
            if (metrics) memcpy(metrics, m, sizeof m);
        }
        memcpy(Ux, nUx, sizeof(zdbl) * nk);
        memcpy(Uy, nUy, sizeof(zdbl) * nk);
        memcpy(W, nW, sizeof(zdbl) * nw);
        if (check && m[7] != 0.0) break;
    }
    if (t > max_iters) t = max_iters;
    free(gx); free(gy); free(nUx); free(nUy); free(nW); free(bw); free(bx); free(by); free(dv); free(dl);
    free(pPhi);
    return t;
}
