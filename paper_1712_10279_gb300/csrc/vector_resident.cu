// Host side of the resident engine: the tile plan and the cooperative launch.
// The kernel (resident_kernel.cuh) is instantiated in the resident_k*.cu units,
// one group of channel counts per unit so that they compile in parallel.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "internal.h"
#include "resident_kernel.cuh"

namespace vomt {
namespace res {

ResKernel res_kernel_k12(int K, int P, int NM, int LB, int LF);
ResKernel res_kernel_k3(int K, int P, int NM, int LB, int LF);
ResKernel res_kernel_k45(int K, int P, int NM, int LB, int LF);
ResKernel res_kernel_k6(int K, int P, int NM, int LB, int LF);
ResKernel res_kernel_k78(int K, int P, int NM, int LB, int LF);
ResKernel res_kernel_k9(int K, int P, int NM, int LB, int LF);
MultiKernel res_multi_kernel_k12(int K, int P, int NM, int LB);
MultiKernel res_multi_kernel_k3(int K, int P, int NM, int LB);
MultiKernel res_multi_kernel_k45(int K, int P, int NM, int LB);
MultiKernel res_multi_kernel_k6(int K, int P, int NM, int LB);
MultiKernel res_multi_kernel_k78(int K, int P, int NM, int LB);

ResKernel res_kernel(int K, int P, int NM, int LB, int LF)
{
    if (K <= 2) return res_kernel_k12(K, P, NM, LB, LF);
    if (K == 3) return res_kernel_k3(K, P, NM, LB, LF);
    if (K <= 5) return res_kernel_k45(K, P, NM, LB, LF);
    if (K == 6) return res_kernel_k6(K, P, NM, LB, LF);
    if (K <= 8) return res_kernel_k78(K, P, NM, LB, LF);
    return res_kernel_k9(K, P, NM, LB, LF);
}

MultiKernel res_multi_kernel(int K, int P, int NM, int LB)
{
    if (K <= 2) return res_multi_kernel_k12(K, P, NM, LB);
    if (K == 3) return res_multi_kernel_k3(K, P, NM, LB);
    if (K <= 5) return res_multi_kernel_k45(K, P, NM, LB);
    if (K == 6) return res_multi_kernel_k6(K, P, NM, LB);
    if (K <= 8) return res_multi_kernel_k78(K, P, NM, LB);
    return nullptr;
}

}  // namespace res

namespace {

using res::RES_THREADS;
using res::HMAX;
constexpr int TMAX = 64;              // longest tile side
constexpr int SMEM_MAX = 227 * 1024;

// Largest extended tile of the 384-thread form of the two-point kernel (up to
// four channels; 170 registers a thread).
constexpr int kTwoPoint384Max = 768;

// Estimated nanoseconds per iteration (see resident_plan).  Constants fitted to
// GB300 measurements of this kernel at k = 3: 3.5 ns per point of the region a
// step updates (arithmetic, shared-memory traffic and the two barriers of a
// step at 16 warps per SM), 3.1 us per halo exchange (one L2 round trip plus
// the tagged stores and polls), and 30% more per point when a thread owns
// four points (register spills).  With five and more channels (`heavy`, 384
// threads) two points per thread already spill: 30% more there, 60% at four.
// With three or four channels (`k34`), two points per thread run in the
// 384-thread form up to 768 points and in 512-thread blocks at 128 registers
// beyond (at 256^2, k = 3 the two cost the same per iteration: H = 3 in the
// 384-thread form, 31.9 ms per 20,000 iterations, against H = 4 in the 512-thread
// form, 31.6 ms); four points per thread spill: 20,000 iterations at 256^2 took
// 45.7 ms against 33.0 at two (H = 4, 128 registers), the steps about 60% longer,
// so their steps are charged 65% more.  One point per thread stays
// the cheapest where it fits (128^2, k = 3: 0.92 us per iteration at one point
// against 1.23 at two).
double plan_cost(int TX, int TY, int H, int G, int rt = RES_THREADS, bool heavy = false, bool k34 = false)
{
    auto spill = [&](int ext) {
        if (k34 && ext > 2 * rt) return 1.65;
        if (ext <= (heavy ? rt : 2 * rt)) return 1.0;
        return heavy && ext > 2 * rt ? 1.6 : 1.3;
    };
    const double per_pt = 3.5;
    if (G == 1) return per_pt * TX * TY * spill(TX * TY);
    double pts = 0.0;
    for (int s = 1; s <= H; ++s) pts += (double)(TX + 2 * (H - s) + 1) * (TY + 2 * (H - s) + 1);
    const int ext = (TX + 2 * H) * (TY + 2 * H);
    return per_pt * spill(ext) * pts / H + 3100.0 / H;
}

}  // namespace

// Tile plan.  Tiles of at most 64 x 64 points, at most `max_blocks` of them; the
// ring width H is at most the narrowest tile side; the extended tile
// (TX + 2H) x (TY + 2H) holds at most four points per thread of res_threads(k)
// (2048 points; 1536 for five and more channels) and its shared-memory
// arrays fit one SM.
// Among those, the plan with the smallest estimated time per iteration
// (plan_cost) wins.  `force_H` > 0 pins the ring width.
bool resident_plan(int n, int k, int max_blocks, int force_H, ResidentPlan *out)
{
    auto smem_ok = [&](int EW, int EH, int G) {
        return res::smem_layout(k, res::row_stride(EW), EH, G).total <= SMEM_MAX;
    };
    const int RT = res::res_threads(k), max_points = 4 * RT;
    const bool heavy = RT < RES_THREADS, k34 = k >= 3 && k <= 4;
    double best = -1.0;
    for (int Gx = 1; Gx <= n && Gx <= max_blocks; ++Gx) {
        const int TX = (n + Gx - 1) / Gx, TXmin = n / Gx;
        if (TX > TMAX) continue;
        for (int Gy = 1; Gy <= n && Gx * Gy <= max_blocks; ++Gy) {
            const int TY = (n + Gy - 1) / Gy, TYmin = n / Gy;
            if (TY > TMAX) continue;
            const int G = Gx * Gy;
            if (G == 1) {
                if (TX * TY > max_points || !smem_ok(TX, TY, 1)) continue;
                const double cost = plan_cost(TX, TY, 0, 1, RT, heavy, k34);
                if (best < 0 || cost < best) {
                    best = cost;
                    *out = ResidentPlan{Gx, Gy, TX, TY, 0, 0, 0, cost};
                }
                continue;
            }
            for (int H = 1; H <= HMAX; ++H) {
                if (force_H > 0 && H != force_H) continue;
                if (H > TXmin || H > TYmin) break;
                const int EW = TX + 2 * H, EH = TY + 2 * H;
                if (EW * EH > max_points || !smem_ok(EW, EH, G)) break;
                const double cost = plan_cost(TX, TY, H, G, RT, heavy, k34);
                if (best < 0 || cost < best) {
                    best = cost;
                    *out = ResidentPlan{Gx, Gy, TX, TY, H, 0, 0, cost};
                }
            }
        }
    }
    if (best < 0) return false;
    const int EW = out->TXm + 2 * out->H, EH = out->TYm + 2 * out->H;
    // P points per thread, the fewest that fit RT threads, spread evenly over
    // round_up(ext / P, 32) threads; two points on at most 384 threads take the
    // 384-thread form (up to four channels)
    const int ext = EW * EH;
    out->P = ext <= RT ? 1 : (ext <= 2 * RT ? 2 : 4);
    out->threads = (((ext + out->P - 1) / out->P + 31) / 32) * 32;
    out->lb = (k <= 4 && out->P == 2 && ext <= kTwoPoint384Max) ? 384 : RT;
    return true;
}

// Tile plan for a wave of `count` problems of side n on `max_blocks` SMs (the
// grouped batch): each problem gets T = Gx x Gy tiles, floor(max_blocks / T)
// problems run side by side, and the plan minimises the estimated time of the
// whole wave (rounds of side-by-side problems x time per iteration of one).
// Same tile rules as resident_plan; P is 2 or 4 (the grouped kernels; two points
// in 384-thread blocks up to 768 points at up to four channels), or 1 for five
// channels when the extended tile fits one point per thread.
bool resident_plan_wave(int n, int k, int count, int max_blocks, ResidentPlan *out)
{
    auto smem_ok = [&](int EW, int EH, int G) {
        return res::smem_layout(k, res::row_stride(EW), EH, G).total <= SMEM_MAX - res::MULTI_STATIC_SMEM;
    };
    const int RT = res::res_threads(k), max_points = 4 * RT;
    const bool heavy = res::res_threads(k) < RES_THREADS, k34 = k >= 3 && k <= 4;
    double best = -1.0;
    for (int Gx = 1; Gx <= n && Gx <= max_blocks; ++Gx) {
        const int TX = (n + Gx - 1) / Gx, TXmin = n / Gx;
        if (TX > TMAX) continue;
        for (int Gy = 1; Gy <= n && Gx * Gy <= max_blocks; ++Gy) {
            const int TY = (n + Gy - 1) / Gy, TYmin = n / Gy;
            if (TY > TMAX) continue;
            const int G = Gx * Gy;
            const int side = std::min(count, max_blocks / G);
            const double rounds = (double)((count + side - 1) / side);
            if (G == 1) {
                if (TX * TY > max_points || !smem_ok(TX, TY, 1)) continue;
                const double cost = rounds * plan_cost(TX, TY, 0, 1, RT, heavy, k34);
                if (best < 0 || cost < best) {
                    best = cost;
                    *out = ResidentPlan{Gx, Gy, TX, TY, 0, 0, 0, cost};
                }
                continue;
            }
            for (int H = 1; H <= HMAX; ++H) {
                if (H > TXmin || H > TYmin) break;
                const int EW = TX + 2 * H, EH = TY + 2 * H;
                if (EW * EH > max_points || !smem_ok(EW, EH, G)) break;
                const double cost = rounds * plan_cost(TX, TY, H, G, RT, heavy, k34);
                if (best < 0 || cost < best) {
                    best = cost;
                    *out = ResidentPlan{Gx, Gy, TX, TY, H, 0, 0, cost};
                }
            }
        }
    }
    if (best < 0) return false;
    const int ext = (out->TXm + 2 * out->H) * (out->TYm + 2 * out->H);
    out->P = (k >= 5 && ext <= RT) ? 1 : (ext <= 2 * RT ? 2 : 4);
    out->threads = (((ext + out->P - 1) / out->P + 31) / 32) * 32;
    out->lb = (k <= 4 && out->P == 2 && ext <= kTwoPoint384Max) ? 384 : RT;
    return true;
}

int resident_solve(vomt_ctx *ctx, const OpDev &g, const StepDev &s, const SolveCfg &cfg, const vomt_params &p,
                   const ResidentPlan &plan, const float *rho0, const float *rho1, float *u, float *w, float *phi,
                   cudaStream_t st)
{
    const int K = g.k, F = 3 * K + g.l, F2 = (F + 1) / 2;
    const int G = plan.Gx * plan.Gy;
    const int EWm = plan.TXm + 2 * plan.H, EHm = plan.TYm + 2 * plan.H;
    const int EWs = res::row_stride(EWm);
    const res::SmemLayout SL = res::smem_layout(K, EWs, EHm, G);
    if (SL.total > SMEM_MAX) {
        ctx->err = "resident plan needs too much shared memory";
        return VOMT_ERR_TOO_LARGE;
    }
    const size_t xch_bytes = (size_t)G * 2 * F2 * plan.TXm * plan.TYm * 2 * sizeof(unsigned long long);
    const size_t rows_bytes = (size_t)2 * G * NRED * 2 * sizeof(unsigned long long);
    const size_t need = xch_bytes + rows_bytes + 256;
    int rc = ensure_buffer(ctx, &ctx->rscratch, &ctx->rscratch_bytes, need, "resident scratch");
    if (rc) return rc;
    unsigned char *base = (unsigned char *)ctx->rscratch;
    res::ResArgs a;
    memset(&a, 0, sizeof a);
    // a single tile never exchanges, so its blocks of iterations may be as long as a check interval
    const int H = G == 1 ? (1 << 30) : plan.H;
    a.geo = res::ResGeom{s.n, plan.Gx, plan.Gy, plan.TXm, plan.TYm, H, G == 1 ? 0 : plan.H, EWs, EHm};
    a.g = g;
    a.s = s;
    a.cfg = cfg;
    a.un = p.u_norm;
    a.wn = p.w_norm;
    a.max_iters = p.max_iters;
    a.check_every = p.check_every;
    a.warm = p.warm_start;
    a.rho0 = rho0;
    a.rho1 = rho1;
    a.u = u;
    a.w = w;
    a.phi = phi;
    a.xch = (unsigned long long *)base;
    a.rows = (unsigned long long *)(base + xch_bytes);
    a.ctl = (dev::ResCtl *)(base + xch_bytes + rows_bytes);
    a.st = ctx->dstatus;
    const int max_checks = p.max_iters / p.check_every + 2;
    if (ctx->hist_cap < max_checks) {
        if (ctx->dhist) cudaFree(ctx->dhist);
        ctx->dhist = nullptr;
        ctx->hist_cap = 0;
        cudaError_t e = cudaMalloc(&ctx->dhist, sizeof(double) * NMET * (size_t)max_checks);
        if (e != cudaSuccess) return set_cuda_error(ctx, e, "history");
        ctx->hist_cap = max_checks;
    }
    a.hist = ctx->dhist;
    a.hist_cap = ctx->hist_cap;
    ctx->hist_raw = true;            // the kernel's check rows hold raw sums (finish_raw_row)
    a.wait_ns = ctx->wait_ns ? ctx->wait_ns : dev::kWaitBudgetNs;
    a.drop_exch = ctx->drop_exchange;
    a.tag_hi = 0u;

    int nm = 0;
    if (p.u_norm == VOMT_U_L12 && p.w_norm == VOMT_W_L1) nm = 1;
    else if (p.u_norm == VOMT_U_L2 && p.w_norm == VOMT_W_L1 && (K == 3 || K == 6)) nm = 2;
    else if (p.u_norm == VOMT_U_NUC && p.w_norm == VOMT_W_NUC && K == 6) nm = 3;
    // 3 x 3 matrices with three L matrices: the flux count fixed at compile time
    const int lf = (K == 6 && g.l == 9 && (nm == 2 || nm == 3)) ? 9 : 0;
    res::ResKernel kern = res::res_kernel(K, plan.P, nm, plan.lb > 0 ? plan.lb : res::res_threads(K), lf);
    if (!kern) {
        ctx->err = "no resident kernel for this channel count and norm pair";
        return VOMT_ERR_TOO_LARGE;
    }
    cudaError_t e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SL.total);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "resident smem attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)kern, plan.threads, SL.total);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "resident occupancy");
    if (per_sm < 1 || G > per_sm * ctx->sm_count) {
        ctx->err = "resident plan does not fit on the device";
        return VOMT_ERR_TOO_LARGE;
    }
    e = cudaMemsetAsync(base, 0, need, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dstatus, 0, sizeof(DevStatus), st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "resident reset");
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(plan.threads), args, SL.total, st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "resident launch");
    ctx->launches += 1;
    ctx->last_blocks = G;
    ctx->last_halo = G > 1 ? plan.H : 0;
    e = cudaMemcpyAsync(&ctx->hstatus[0], ctx->dstatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error(ctx, e, "resident solve");
    return VOMT_OK;
}

}  // namespace vomt
