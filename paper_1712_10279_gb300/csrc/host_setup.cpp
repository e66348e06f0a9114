// Host-side setup: channel-graph validation and the largest eigenvalues that
// fix the step sizes (Sections 7.2 and 7.3 ask for "a standard eigenvalue
// routine").  Here: Householder reduction to tridiagonal form, then bisection
// on the Sturm sequence of the tridiagonal matrix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace vomt {

int graph_to_dev(const vomt_graph *g, GraphDev *out, std::string *err)
{
    if (!g || g->k < 1 || g->k > KMAX || g->n_edges < 0 || g->n_edges > LMAX) {
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

double sym_lmax(int m, const double *Ain)
{
    if (m <= 0) return 0.0;
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
    std::vector<double> d(m), e(m > 1 ? m - 1 : 1);
    for (int i = 0; i < m; ++i) d[i] = A[i * m + i];
    for (int i = 0; i + 1 < m; ++i) e[i] = 0.5 * (A[(i + 1) * m + i] + A[i * m + i + 1]);
    // Gershgorin interval, then bisection for the smallest x with all m eigenvalues below it.
    double lo = d[0], hi = d[0];
    for (int i = 0; i < m; ++i) {
        double rad = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - rad);
        hi = std::max(hi, d[i] + rad);
    }
    double scale = std::max(fabs(lo), fabs(hi));
    hi += 1e-12 * scale + 1e-300;
    for (int it = 0; it < 400 && hi - lo > 1e-15 * scale; ++it) {
        double mid = 0.5 * (lo + hi);
        if (sturm_count(m, d.data(), e.data(), mid) >= m) hi = mid; else lo = mid;
    }
    return hi;
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
