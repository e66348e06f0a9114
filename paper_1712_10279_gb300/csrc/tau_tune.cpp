// Tuner of the dual step tau (vomt_tune_tau, momt_tune_tau, vomt_batch_tune_tau).
//
// Sections 7.1-7.3 tie the primal steps to tau (mu = 1/(32 tau (n-1)^2),
// nu = 1/(4 tau lambda_max)), which keeps every tau > 0 inside the convergence
// condition, and tune tau per experiment for the fastest convergence (Tables 1
// and 3 print the values used).  The best tau depends on the scale of the
// densities and on how far mass moves, so the tuner measures it: short runs of
// the solve itself from the zero iterate over a geometric grid of tau, scored by
// max(relative gap, relative residual) after the run, with successive halving
// (the better candidates run longer) and one refinement around the winner.
// Host code only; every run is an ordinary solve through the C ABI.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <vector>

#include "internal.h"

namespace vomt {
namespace {

constexpr int kGrid = VOMT_TAU_GRID;

// tau of grid point j: the paper's value times 10^((j - 1) / 2), i.e. from a
// third of it to ten thousand times it
double grid_tau(double tau_paper, int j) { return tau_paper * pow(10.0, 0.5 * (j - 1)); }

double score_of(int rc, const vomt_result &r)
{
    if (rc < 0) return INFINITY;
    const double s = fmax(r.rel_gap, r.rel_res);
    return isfinite(s) ? s : INFINITY;
}

// Successive halving over the grid.  run(tau, iters) returns the score of a run.
double halving(double tau_paper, int s, const std::function<double(double, int)> &run, double *grid_scores,
               double *best_score)
{
    struct Cand {
        double tau, score;
    };
    std::vector<Cand> c(kGrid);
    for (int j = 0; j < kGrid; ++j) {
        c[j].tau = grid_tau(tau_paper, j);
        c[j].score = run(c[j].tau, s);
        if (grid_scores) grid_scores[j] = c[j].score;
    }
    auto better = [](const Cand &a, const Cand &b) { return a.score < b.score || (a.score == b.score && a.tau < b.tau); };
    int iters = s;
    for (int keep : {4, 2}) {
        std::sort(c.begin(), c.end(), better);
        c.resize(keep);
        iters *= 2;
        for (auto &x : c) x.score = run(x.tau, iters);
    }
    std::sort(c.begin(), c.end(), better);
    Cand best = c[0];
    for (double f : {pow(10.0, -0.25), pow(10.0, 0.25)}) {
        Cand x{best.tau * f, 0.0};
        x.score = run(x.tau, iters);
        if (better(x, best)) best = x;
    }
    if (best_score) *best_score = best.score;
    return best.tau;
}

}  // namespace
}  // namespace vomt

extern "C" int vomt_tune_tau(vomt_ctx *ctx, int n, const float *rho0, const float *rho1, const vomt_graph *g,
                             double alpha, const vomt_params *pin, int sample_iters, float *u, float *w,
                             float *phi, double *best_tau, double *best_score, double *grid_scores, void *stream)
{
    using namespace vomt;
    if (!ctx || sample_iters < 1 || !g) return VOMT_ERR_BAD_ARG;
    try {
        vomt_params p;
        vomt_default_params(&p);
        if (pin) p = *pin;
        double tau_paper = 0.0;
        int rc = vomt_step_sizes(n, g, 0.0, nullptr, nullptr, &tau_paper, nullptr);
        if (rc) return rc;
        int first_err = 0;
        auto run = [&](double tau, int iters) {
            vomt_params q = p;
            q.tau = tau;
            q.mu = q.nu = 0.0;
            q.max_iters = iters;
            q.check_every = iters;
            q.tol_gap = q.tol_res = 0.0;
            q.warm_start = 0;
            vomt_result r{};
            const int c = vomt_solve(ctx, n, rho0, rho1, g, alpha, &q, u, w, phi, &r, stream);
            // a diverging candidate (NONFINITE) is only a bad score; other errors end the search
            if (c < 0 && c != VOMT_ERR_NONFINITE && !first_err) first_err = c;
            return score_of(c, r);
        };
        double bs = 0.0;
        const double t = halving(tau_paper, sample_iters, run, grid_scores, &bs);
        if (first_err) return first_err;
        if (best_tau) *best_tau = t;
        if (best_score) *best_score = bs;
        return VOMT_OK;
    } catch (...) {
        return fail(ctx, VOMT_ERR_BAD_ARG, "internal exception");
    }
}

extern "C" int momt_tune_tau(vomt_ctx *ctx, int n, int k, const float *Lam0, const float *Lam1, int N,
                             const double *L, double alpha, const vomt_params *pin, int sample_iters, float *U,
                             float *W, float *Phi, double *best_tau, double *best_score, double *grid_scores,
                             void *stream)
{
    using namespace vomt;
    if (!ctx || sample_iters < 1) return VOMT_ERR_BAD_ARG;
    try {
        vomt_params p;
        vomt_default_params(&p);
        if (pin) p = *pin;
        double tau_paper = 0.0;
        int rc = momt_step_sizes(n, k, N, L, 0.0, nullptr, nullptr, &tau_paper, nullptr, nullptr);
        if (rc) return rc;
        int first_err = 0;
        auto run = [&](double tau, int iters) {
            vomt_params q = p;
            q.tau = tau;
            q.mu = q.nu = 0.0;
            q.max_iters = iters;
            q.check_every = iters;
            q.tol_gap = q.tol_res = 0.0;
            q.warm_start = 0;
            vomt_result r{};
            const int c = momt_solve(ctx, n, k, Lam0, Lam1, N, L, alpha, &q, U, W, Phi, &r, stream);
            if (c < 0 && c != VOMT_ERR_NONFINITE && !first_err) first_err = c;
            return score_of(c, r);
        };
        double bs = 0.0;
        const double t = halving(tau_paper, sample_iters, run, grid_scores, &bs);
        if (first_err) return first_err;
        if (best_tau) *best_tau = t;
        if (best_score) *best_score = bs;
        return VOMT_OK;
    } catch (...) {
        return fail(ctx, VOMT_ERR_BAD_ARG, "internal exception");
    }
}

extern "C" int vomt_batch_tune_tau(vomt_ctx *ctx, int count, const vomt_instance *inst, float *arena,
                                   const vomt_params *pin, int sample_iters, double *taus, double *scores)
{
    using namespace vomt;
    if (!ctx || count < 1 || !inst || !taus || sample_iters < 1) return VOMT_ERR_BAD_ARG;
    try {
        vomt_params p;
        vomt_default_params(&p);
        if (pin) p = *pin;
        p.max_iters = sample_iters;
        p.check_every = sample_iters;
        p.tol_gap = p.tol_res = 0.0;
        p.warm_start = 0;
        std::vector<vomt_instance> trial(inst, inst + count);
        std::vector<vomt_result> res(count);
        std::vector<double> paper(count), best(count, INFINITY);
        for (int q = 0; q < count; ++q) {
            int rc = vomt_step_sizes(inst[q].n, &inst[q].graph, 0.0, nullptr, nullptr, &paper[q], nullptr);
            if (rc) return rc;
            taus[q] = paper[q];
        }
        for (int j = 0; j < kGrid; ++j) {
            for (int q = 0; q < count; ++q) trial[q].tau = grid_tau(paper[q], j);
            const int rc = vomt_solve_batched(ctx, count, trial.data(), arena, &p, res.data(), nullptr);
            if (rc < 0 && rc != VOMT_ERR_NONFINITE) return rc;
            for (int q = 0; q < count; ++q) {
                const double s = rc == VOMT_ERR_NONFINITE ? INFINITY : score_of(0, res[q]);
                if (s < best[q]) {
                    best[q] = s;
                    taus[q] = trial[q].tau;
                }
            }
        }
        if (scores)
            for (int q = 0; q < count; ++q) scores[q] = best[q];
        return VOMT_OK;
    } catch (...) {
        return fail(ctx, VOMT_ERR_BAD_ARG, "internal exception");
    }
}
