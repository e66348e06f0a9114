// Host-side setup: channel-graph validation and the largest eigenvalues that
// fix the step sizes (Sections 7.2 and 7.3 ask for "a standard eigenvalue
// routine").  Here: Householder reduction to tridiagonal form, then bisection
// on the Sturm sequence of the tridiagonal matrix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "internal.h"

namespace vomt {

int graph_to_dev(const vomt_graph *g, GraphDev *out, std::string *err)
{
    if (!g || g->k < 1 || g->k > KVEC || g->n_edges < 0 || g->n_edges > LVEC) {
        *err = "graph: need 1 <= k <= 8 and 0 <= n_edges <= k(k-1)/2";
        return VOMT_ERR_BAD_ARG;
    }
    const int k = g->k, l = g->n_edges;
    if (l > 0 && (!g->tail || !g->head)) { *err = "graph: null edge arrays"; return VOMT_ERR_BAD_ARG; }
    memset(out, 0, sizeof(*out));
    out->k = k;
    out->l = l;
    bool seen[KMAX][KMAX] = {};
    int parent[KMAX];
    for (int a = 0; a < k; ++a) parent[a] = a;
    auto root = [&](int a) { while (parent[a] != a) a = parent[a] = parent[parent[a]]; return a; };
    for (int e = 0; e < l; ++e) {
        int a = g->tail[e], b = g->head[e];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b) { *err = "graph: edge endpoint out of range or self loop"; return VOMT_ERR_GRAPH; }
        int lo = a < b ? a : b, hi = a < b ? b : a;
        if (seen[lo][hi]) { *err = "graph: repeated edge"; return VOMT_ERR_GRAPH; }
        seen[lo][hi] = true;
        double c = g->cost ? g->cost[e] : 1.0;
        if (!(c > 0.0) || !isfinite(c)) { *err = "graph: edge cost must be positive and finite"; return VOMT_ERR_BAD_ARG; }
        out->lo[e] = (int8_t)lo;
        out->hi[e] = (int8_t)hi;
        out->inv_c[e] = (float)(1.0 / c);
        parent[root(lo)] = root(hi);
    }
    for (int a = 1; a < k; ++a)
        if (root(a) != root(0)) { *err = "graph: channel graph is not connected"; return VOMT_ERR_GRAPH; }
    return VOMT_OK;
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x.
static int sturm_count(int m, const double *d, const double *e, double x)
{
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < m; ++i) {
        double qq = (q == 0.0) ? 1e-300 : q;
        q = d[i] - x - e[i - 1] * e[i - 1] / qq;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// Householder reduction of a symmetric matrix to tridiagonal (d, e).
static void tridiagonalise(int m, const double *Ain, std::vector<double> &d, std::vector<double> &e);

double sym_lmax(int m, const double *Ain) { return sym_eig(m, Ain, m - 1); }

double sym_eig(int m, const double *Ain, int idx)
{
    if (m <= 0) return 0.0;
    std::vector<double> d, e;
    tridiagonalise(m, Ain, d, e);
    // Gershgorin interval, then bisection for the smallest x with more than idx
    // eigenvalues below it.
    double lo = d[0], hi = d[0];
    for (int i = 0; i < m; ++i) {
        double rad = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - rad);
        hi = std::max(hi, d[i] + rad);
    }
    double scale = std::max(fabs(lo), fabs(hi));
    lo -= 1e-12 * scale + 1e-300;
    hi += 1e-12 * scale + 1e-300;
    for (int it = 0; it < 400 && hi - lo > 1e-15 * scale; ++it) {
        double mid = 0.5 * (lo + hi);
        if (sturm_count(m, d.data(), e.data(), mid) > idx) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

static void tridiagonalise(int m, const double *Ain, std::vector<double> &d, std::vector<double> &e)
{
    std::vector<double> A(Ain, Ain + (size_t)m * m);
    std::vector<double> v(m), p(m);
    // Householder: zero column c below the sub-diagonal, for c = 0 .. m-3.
    for (int c = 0; c + 2 < m; ++c) {
        double nx = 0.0;
        for (int r = c + 1; r < m; ++r) nx += A[r * m + c] * A[r * m + c];
        nx = sqrt(nx);
        if (nx == 0.0) continue;
        double a0 = A[(c + 1) * m + c];
        double alpha = a0 > 0 ? -nx : nx;
        for (int r = 0; r < m; ++r) v[r] = 0.0;
        for (int r = c + 1; r < m; ++r) v[r] = A[r * m + c];
        v[c + 1] -= alpha;
        double nv = 0.0;
        for (int r = c + 1; r < m; ++r) nv += v[r] * v[r];
        nv = sqrt(nv);
        if (nv == 0.0) continue;
        for (int r = c + 1; r < m; ++r) v[r] /= nv;
        // A <- (I - 2vv^T) A (I - 2vv^T) = A - 2(v q^T + q v^T), q = Av - (v^T A v) v
        for (int r = 0; r < m; ++r) {
            double s = 0.0;
            for (int t = 0; t < m; ++t) s += A[r * m + t] * v[t];
            p[r] = s;
        }
        double K = 0.0;
        for (int r = 0; r < m; ++r) K += v[r] * p[r];
        for (int r = 0; r < m; ++r) p[r] -= K * v[r];
        for (int r = 0; r < m; ++r)
            for (int t = 0; t < m; ++t) A[r * m + t] -= 2.0 * (v[r] * p[t] + p[r] * v[t]);
    }
    d.assign(m, 0.0);
    e.assign(m > 1 ? m - 1 : 1, 0.0);
    for (int i = 0; i < m; ++i) d[i] = A[i * m + i];
    for (int i = 0; i + 1 < m; ++i) e[i] = 0.5 * (A[(i + 1) * m + i] + A[i * m + i + 1]);
}

// lambda_max(-Delta_G), -Delta_G = D diag(1/c^2) D^T (Section 3.1): entry (a, b)
// sums 1/c_e^2 over edges at a (a == b) or -1/c_e^2 over the edge {a, b}.
double graph_lmax(const GraphDev &g, const double *cost)
{
    if (g.l == 0) return 0.0;
    std::vector<double> M((size_t)g.k * g.k, 0.0);
    for (int e = 0; e < g.l; ++e) {
        double c = cost ? cost[e] : 1.0;
        double wgt = 1.0 / (c * c);
        int a = g.lo[e], b = g.hi[e];
        M[a * g.k + a] += wgt;
        M[b * g.k + b] += wgt;
        M[a * g.k + b] -= wgt;
        M[b * g.k + a] -= wgt;
    }
    return sym_lmax(g.k, M.data());
}

}  // namespace vomt

namespace vomt {

void graph_to_op(const GraphDev &g, OpDev *op)
{
    memset(op, 0, sizeof(*op));
    op->k = g.k;
    op->l = g.l;
    for (int c = 0; c < g.k; ++c) op->wc[c] = 1.0f;
    for (int e = 0; e < g.l; ++e) {
        op->we[e] = 1.0f;
        op->G[e][g.lo[e]] = g.inv_c[e];     // grad_G = diag(1/c) D^T, D[lo][e] = +1, D[hi][e] = -1
        op->G[e][g.hi[e]] = -g.inv_c[e];
        op->Dv[g.lo[e]][e] = g.inv_c[e];    // div_G = -D diag(1/c)
        op->Dv[g.hi[e]][e] = -g.inv_c[e];
    }
}

// compact index of the symmetric entry (a, b): the diagonal first, then the entries
// above it row by row ((0,1), (0,2), (1,2) for k = 3)
static int sym_index(int k, int a, int b)
{
    if (a == b) return a;
    if (a > b) { int t = a; a = b; b = t; }
    int idx = k;
    for (int r = 0; r < k; ++r)
        for (int c = r + 1; c < k; ++c) {
            if (r == a && c == b) return idx;
            ++idx;
        }
    return -1;
}

int quantum_to_op(int k, int N, const double *L, OpDev *op, double *lmax, double *sym_gap, std::string *err)
{
    if (k < 2 || k > 3 || N < 1 || !L) { *err = "matrix OMT: need 2 <= k <= 3, N >= 1, L given"; return VOMT_ERR_BAD_ARG; }
    const int K = k * (k + 1) / 2, ks = k * (k - 1) / 2;
    if (N * ks > K * (K - 1) / 2) { *err = "matrix OMT: too many L matrices for this k"; return VOMT_ERR_BAD_ARG; }
    double scale = 0.0;
    for (int q = 0; q < N * k * k; ++q) {
        if (!isfinite(L[q])) { *err = "matrix OMT: L has non-finite entries"; return VOMT_ERR_BAD_ARG; }
        scale = std::max(scale, fabs(L[q]));
    }
    for (int s = 0; s < N; ++s)
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b)
                if (fabs(L[(s * k + a) * k + b] - L[(s * k + b) * k + a]) > 1e-12 * std::max(scale, 1e-300)) {
                    *err = "matrix OMT: every L_s must be symmetric";
                    return VOMT_ERR_BAD_ARG;
                }
    memset(op, 0, sizeof(*op));
    op->k = K;
    op->l = N * ks;
    for (int c = 0; c < K; ++c) op->wc[c] = c < k ? 1.0f : 2.0f;
    // (grad_L Phi)_s = L_s Phi - Phi L_s; entry (a, b), a < b, of the skew result
    int e = 0;
    for (int s = 0; s < N; ++s) {
        const double *Ls = L + (size_t)s * k * k;
        for (int a = 0; a < k; ++a)
            for (int b = a + 1; b < k; ++b, ++e) {
                double row[KMAX] = {};
                for (int m = 0; m < k; ++m) {
                    row[sym_index(k, m, b)] += Ls[a * k + m];     // (L_s Phi)_ab
                    row[sym_index(k, a, m)] -= Ls[m * k + b];     // (Phi L_s)_ab
                }
                op->we[e] = 2.0f;
                for (int c = 0; c < K; ++c) {
                    op->G[e][c] = (float)row[c];
                    op->Dv[c][e] = (float)(2.0 / (c < k ? 1.0 : 2.0) * row[c]);
                }
            }
    }
    // -Delta_L X = sum_s [L_s, [L_s, X]] as a k^2 x k^2 matrix, column by column
    const int kk = k * k;
    std::vector<double> M((size_t)kk * kk, 0.0);
    for (int col = 0; col < kk; ++col) {
        double X[9] = {}, C1[9], C2[9];
        X[col] = 1.0;
        for (int s = 0; s < N; ++s) {
            const double *Ls = L + (size_t)s * kk;
            for (int a = 0; a < k; ++a)
                for (int b = 0; b < k; ++b) {
                    double v = 0.0;
                    for (int m = 0; m < k; ++m) v += Ls[a * k + m] * X[m * k + b] - X[a * k + m] * Ls[m * k + b];
                    C1[a * k + b] = v;
                }
            for (int a = 0; a < k; ++a)
                for (int b = 0; b < k; ++b) {
                    double v = 0.0;
                    for (int m = 0; m < k; ++m) v += Ls[a * k + m] * C1[m * k + b] - C1[a * k + m] * Ls[m * k + b];
                    C2[a * k + b] = v;
                }
            for (int r = 0; r < kk; ++r) M[(size_t)r * kk + col] += C2[r];
        }
    }
    if (lmax) *lmax = sym_lmax(kk, M.data());
    // restriction to symmetric matrices in an orthonormal basis (E_aa, (E_ab + E_ba)/sqrt 2)
    std::vector<double> B((size_t)kk * K, 0.0), Sm((size_t)K * K, 0.0);
    for (int a = 0; a < k; ++a)
        for (int b = a; b < k; ++b) {
            const int c = sym_index(k, a, b);
            if (a == b) B[(size_t)(a * k + a) * K + c] = 1.0;
            else {
                B[(size_t)(a * k + b) * K + c] = 1.0 / sqrt(2.0);
                B[(size_t)(b * k + a) * K + c] = 1.0 / sqrt(2.0);
            }
        }
    for (int p = 0; p < K; ++p)
        for (int q = 0; q < K; ++q) {
            double v = 0.0;
            for (int r = 0; r < kk; ++r)
                for (int c = 0; c < kk; ++c) v += B[(size_t)r * K + p] * M[(size_t)r * kk + c] * B[(size_t)c * K + q];
            Sm[(size_t)p * K + q] = v;
        }
    const double gap = sym_eig(K, Sm.data(), 1);
    if (sym_gap) *sym_gap = gap;
    const double lm = sym_lmax(kk, M.data());
    if (!(gap > 1e-8 * lm)) {
        *err = "matrix OMT: ker grad_L on symmetric matrices is larger than span{I}";
        return VOMT_ERR_L_KERNEL;
    }
    return VOMT_OK;
}

// Complex Hermitian fields (Section 4's complex setting) in real compact
// coordinates: a Hermitian k x k matrix X is its diagonal (real), then Re and Im
// of each entry above it (a, b), weights 1, 2, 2; a skew-Hermitian Z is Im of its
// diagonal, then Re and Im of each entry above it, weights 1, 2, 2.  Both
// reproduce Re tr(X Y*) exactly, so grad_L becomes a real-linear map G between
// the two coordinate spaces and div_L its weighted adjoint, as in the real case.
// The k * k real channels must fit KMAX (9), so k = 2 (4 channels, 4 flux entries
// per L_s) or k = 3 (9 channels, 9 flux entries per L_s); the channel count is
// padded to the smallest K >= k * k with K(K-1)/2 >= k * k * N, the flux bound of
// the kernels' templates (padding channels carry zero in every field and take no
// part in G): N <= 9 for k = 2, N <= 4 for k = 3.  The pairs (Re, Im) of the
// entries above the diagonal are marked in upair / wpair for the entrywise norm.
int hermitian_to_op(int k, int N, const double *L, OpDev *op, double *lmax, double *sym_gap, std::string *err)
{
    if (k < 2 || k > 3 || N < 1 || !L) {
        *err = "complex matrix OMT: k = 2 or 3 and N >= 1 with L given";
        return VOMT_ERR_BAD_ARG;
    }
    const int kk = k * k, ks = k * k;            // real coordinates of Hermitian / skew-Hermitian
    int K = kk;
    while (K * (K - 1) / 2 < N * ks) ++K;
    if (K > KMAX) {
        *err = k == 2 ? "complex matrix OMT: too many L matrices (N <= 9 for 2 x 2)"
                      : "complex matrix OMT: too many L matrices (N <= 4 for 3 x 3)";
        return VOMT_ERR_BAD_ARG;
    }
    typedef std::complex<double> cd;
    double scale = 0.0;
    for (int q = 0; q < 2 * N * kk; ++q) {
        if (!isfinite(L[q])) { *err = "complex matrix OMT: L has non-finite entries"; return VOMT_ERR_BAD_ARG; }
        scale = std::max(scale, fabs(L[q]));
    }
    auto Lz = [&](int s, int a, int b) { const double *p = L + 2 * ((size_t)(s * k + a) * k + b); return cd(p[0], p[1]); };
    for (int s = 0; s < N; ++s)
        for (int a = 0; a < k; ++a)
            for (int b = 0; b < k; ++b)
                if (std::abs(Lz(s, a, b) - std::conj(Lz(s, b, a))) > 1e-12 * std::max(scale, 1e-300)) {
                    *err = "complex matrix OMT: every L_s must be Hermitian";
                    return VOMT_ERR_BAD_ARG;
                }
    // basis X_c of the Hermitian coordinates, and the coordinate reader of skew-Hermitian matrices
    std::vector<std::vector<cd>> Xc;
    std::vector<double> wc;
    for (int a = 0; a < k; ++a) {
        std::vector<cd> X(kk, cd(0, 0));
        X[a * k + a] = 1.0;
        Xc.push_back(X);
        wc.push_back(1.0);
    }
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b) {
            std::vector<cd> Xr(kk, cd(0, 0)), Xi(kk, cd(0, 0));
            Xr[a * k + b] = 1.0;
            Xr[b * k + a] = 1.0;
            Xi[a * k + b] = cd(0, 1);
            Xi[b * k + a] = cd(0, -1);
            Xc.push_back(Xr);
            Xc.push_back(Xi);
            wc.push_back(2.0);
            wc.push_back(2.0);
        }
    auto skew_coords = [&](const std::vector<cd> &Z, double *out) {
        int e = 0;
        for (int a = 0; a < k; ++a) out[e++] = Z[a * k + a].imag();
        for (int a = 0; a < k; ++a)
            for (int b = a + 1; b < k; ++b) {
                out[e++] = Z[a * k + b].real();
                out[e++] = Z[a * k + b].imag();
            }
    };
    double we_one[64];
    {
        int e = 0;
        for (int a = 0; a < k; ++a) we_one[e++] = 1.0;
        for (int a = 0; a < k; ++a)
            for (int b = a + 1; b < k; ++b) { we_one[e++] = 2.0; we_one[e++] = 2.0; }
    }
    memset(op, 0, sizeof(*op));
    op->k = K;
    op->l = N * ks;
    for (int c = 0; c < K; ++c) op->wc[c] = c < kk ? (float)wc[c] : 1.0f;
    // (Re, Im) pairs: coordinates k, k+2, ... of every Hermitian / skew-Hermitian block
    for (int j = 0; j < k * (k - 1) / 2; ++j) {
        op->upair |= 1u << (k + 2 * j);
        for (int s = 0; s < N; ++s) {
            const int e = s * ks + k + 2 * j;
            op->wpair[e >> 5] |= 1u << (e & 31);
        }
    }
    std::vector<double> Gd((size_t)N * ks * kk, 0.0);
    for (int s = 0; s < N; ++s)
        for (int c = 0; c < kk; ++c) {
            std::vector<cd> Z(kk, cd(0, 0));          // L_s X_c - X_c L_s
            for (int a = 0; a < k; ++a)
                for (int b = 0; b < k; ++b) {
                    cd v(0, 0);
                    for (int m = 0; m < k; ++m) v += Lz(s, a, m) * Xc[c][m * k + b] - Xc[c][a * k + m] * Lz(s, m, b);
                    Z[a * k + b] = v;
                }
            double co[64];
            skew_coords(Z, co);
            for (int e = 0; e < ks; ++e) Gd[(size_t)(s * ks + e) * kk + c] = co[e];
        }
    for (int s = 0; s < N; ++s)
        for (int e = 0; e < ks; ++e) {
            const int ee = s * ks + e;
            op->we[ee] = (float)we_one[e];
            for (int c = 0; c < kk; ++c) {
                op->G[ee][c] = (float)Gd[(size_t)ee * kk + c];
                op->Dv[c][ee] = (float)(we_one[e] / wc[c] * Gd[(size_t)ee * kk + c]);
            }
        }
    // -Delta_L = div^* ... in these coordinates M = Dv G, self-adjoint for the weights wc;
    // its spectrum is that of W^(1/2) M W^(-1/2) (symmetric), the same on Hermitian
    // matrices as on all of C^{k x k} since -Delta_L is complex-linear
    std::vector<double> Sm((size_t)kk * kk, 0.0);
    for (int c = 0; c < kk; ++c)
        for (int d = 0; d < kk; ++d) {
            double v = 0.0;
            for (int e = 0; e < N * ks; ++e) v += (we_one[e % ks] / wc[c]) * Gd[(size_t)e * kk + c] * Gd[(size_t)e * kk + d];
            Sm[(size_t)c * kk + d] = sqrt(wc[c]) * v / sqrt(wc[d]);
        }
    const double lm = sym_lmax(kk, Sm.data());
    const double gap = sym_eig(kk, Sm.data(), 1);
    if (lmax) *lmax = lm;
    if (sym_gap) *sym_gap = gap;
    if (!(gap > 1e-8 * lm)) {
        *err = "complex matrix OMT: ker grad_L on Hermitian matrices is larger than span{I}";
        return VOMT_ERR_L_KERNEL;
    }
    return VOMT_OK;
}

}  // namespace vomt
