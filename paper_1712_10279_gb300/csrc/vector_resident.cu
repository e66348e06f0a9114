// Resident engine for vector OMT: one cooperative launch runs the whole PDHG
// solve (Section 7.2) with the iterate on chip, exchanging tile halos through
// L2 once every H iterations (temporal blocking).
//
// The n x n grid is cut into Gx x Gy rectangular tiles, one per thread block
// (one block per SM).  Each block works on its tile extended by a ring of
// width H on every side that has a neighbour tile.  After a halo exchange the
// block holds the full iterate (phi, u_x, u_y, w) on the extended region, and
// it can run H iterations without hearing from its neighbours: iteration s of
// a block updates the tile grown by H - s cells, because one iteration of
// Section 7.2 at a point reads the previous iterate only at that point and at
// neighbours one cell away (phi at (i+1,j), (i,j+1), (i-1,j+1), (i+1,j-1); u at
// (i-1,j), (i,j-1)).  After H iterations the tile itself is exact and the ring
// is refreshed from the neighbours.  The ring work is redundant arithmetic
// that buys H-fold fewer L2 round trips, which bound small grids.
//
// Points are owned by threads for the whole solve (up to P points per thread);
// each thread keeps its points' iterate and b = rho1 - rho0 in registers.  The
// stencils of Appendix A within a block read neighbouring phi and ubar through
// shared memory.  Between blocks, every iterate value a neighbour needs is
// written to L2 as a 64-bit word with the value in its low half and the
// exchange number in its high half; a reader polls the words themselves, so a
// halo exchange costs one L2 round trip and no fences or flags (aligned 64-bit
// accesses are single-copy atomic).
//
// Convergence checks (every check_every iterations and at the end; a block of
// iterations is cut short so that it ends on a check) reduce FP64 metric terms
// per thread block, publish one row per block as tagged word pairs, and every
// block sums all rows in the same fixed order, so all blocks take the same
// stopping decision.  Every wait is bounded in time; a wait that runs out
// raises a global abort word that makes every block return.
#include <math.h>
#include <string.h>

#include "internal.h"
#include "pdhg_device.cuh"

namespace vomt {
namespace {

using namespace dev;

constexpr int RES_THREADS = 512;      // most threads a block runs
constexpr int RES_P4_POINTS = 1024;   // extended tiles above this size: four points per thread
constexpr int RES_MAX_POINTS = 2048;  // largest extended tile (four points per thread, 512 threads)
constexpr int TMAX = 64;              // longest tile side
constexpr int HMAX = 16;              // widest halo ring

struct ResGeom {
    int n, Gx, Gy, TXm, TYm, H, EWm, EHm;
};

struct ResArgs {
    ResGeom geo;
    OpDev g;                   // per-point grad / div and inner-product weights
    StepDev s;
    SolveCfg cfg;
    int un, wn, max_iters, check_every, warm;
    const float *rho0, *rho1;
    float *u, *w, *phi;
    unsigned long long *xch;   // [G][2][F][TYm][TXm] tagged iterate words
    unsigned long long *rows;  // [2][G][NRED][2] tagged halves of the FP64 partial sums
    ResCtl *ctl;
    DevStatus *st;
    double *hist;
    int hist_cap;
};

template <int K>
struct LK {
    static constexpr int v = K * (K - 1) / 2 > 0 ? K * (K - 1) / 2 : 1;
};

struct SmemLayout {
    int red, S, dec, rtab, sphi, sux, suy, sdx, sdy, total;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline SmemLayout smem_layout(int K, int EWm, int EHm, int G)
{
    SmemLayout L;
    int o = 0;
    const int plane = K * EWm * EHm * 4;
    L.red = o; o += align16((RES_THREADS / 32) * NRED * 8);
    L.S = o; o += align16(NRED * 8);
    L.dec = o; o += 16;
    L.rtab = o; o += align16(G * NRED * 8);
    L.sphi = o; o += align16(plane);
    L.sux = o; o += align16(plane);
    L.suy = o; o += align16(plane);
    L.sdx = o; o += align16(plane);
    L.sdy = o; o += align16(plane);
    L.total = o;
    return L;
}

// Poll `cnt` tagged words (addresses from `addr(j)`), handing each value to
// `sink(j, bits)` once its tag matches.  All pending words of a batch are
// re-read every round.  Returns false on timeout or abort.
template <int BATCH, typename Addr, typename Sink>
__device__ __forceinline__ bool poll_words(int cnt, uint32_t tag, ResCtl *ctl, Addr addr, Sink sink)
{
    for (int base = 0; base < cnt; base += BATCH) {
        uint32_t pending = 0;
#pragma unroll
        for (int r = 0; r < BATCH; ++r)
            if (base + r < cnt) pending |= 1u << r;
        uint64_t t0 = 0;
        for (uint32_t round = 0; pending; ++round) {
            unsigned long long v[BATCH];
#pragma unroll
            for (int r = 0; r < BATCH; ++r) v[r] = (pending >> r & 1u) ? ld_relaxed64(addr(base + r)) : 0ull;
#pragma unroll
            for (int r = 0; r < BATCH; ++r) {
                if ((pending >> r & 1u) && (uint32_t)(v[r] >> 32) == tag) {
                    sink(base + r, (uint32_t)v[r]);
                    pending &= ~(1u << r);
                }
            }
            if (pending && (round & 63u) == 63u) {
                if (t0 == 0) t0 = global_ns();
                if (ld_relaxed32(&ctl->abort)) return false;
                if (global_ns() - t0 > kWaitBudgetNs) {
                    atomicExch(&ctl->abort, 1u);
                    atomicExch(&ctl->where, 1u);
                    return false;
                }
            }
        }
    }
    return true;
}

template <int K, int P>
__global__ void __launch_bounds__(RES_THREADS, 1) k_resident(ResArgs a)
{
    constexpr int LKv = LK<K>::v;
    constexpr int FMAX = 3 * K + LKv;
    extern __shared__ __align__(16) unsigned char smem[];
    const ResGeom G = a.geo;
    const int n = G.n, H = G.H;
    const size_t nn = (size_t)n * n;
    const int NT = (int)gridDim.x;
    const SmemLayout SL = smem_layout(K, G.EWm, G.EHm, NT);
    double *red = (double *)(smem + SL.red);
    double *S = (double *)(smem + SL.S);
    int *dec = (int *)(smem + SL.dec);
    double *rtab = (double *)(smem + SL.rtab);
    float *sphi = (float *)(smem + SL.sphi), *sux = (float *)(smem + SL.sux), *suy = (float *)(smem + SL.suy);
    float *sdx = (float *)(smem + SL.sdx), *sdy = (float *)(smem + SL.sdy);

    const int tile = blockIdx.x, gx = tile % G.Gx, gy = tile / G.Gx;
    const int x0 = gx * n / G.Gx, x1 = (gx + 1) * n / G.Gx;
    const int y0 = gy * n / G.Gy, y1 = (gy + 1) * n / G.Gy;
    const bool hasL = gx > 0, hasR = gx < G.Gx - 1, hasD = gy > 0, hasU = gy < G.Gy - 1;
    const int X0 = x0 - (hasL ? H : 0), X1 = x1 + (hasR ? H : 0);
    const int Y0 = y0 - (hasD ? H : 0), Y1 = y1 + (hasU ? H : 0);
    const int EW = X1 - X0, EH = Y1 - Y0, NP = EW * EH;
    const int PLANE = G.EWm * G.EHm;
#define SA(arr, c, ey, ex) arr[(c) * PLANE + (ey) * G.EWm + (ex)]

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int k = a.g.k, l = a.g.l, F = 3 * K + l;
    const float mu = a.s.mu, nu = a.s.nu, tau = a.s.tau, ih = a.s.ih, alpha = a.s.alpha;
    const float muih = mu * ih;
    const int T = a.max_iters, CE = a.check_every;
    const size_t TSZ = (size_t)G.TXm * G.TYm;
    auto xword = [&](int t_, int par, int f, int ly, int lx) -> unsigned long long * {
        return a.xch + (((size_t)t_ * 2 + par) * F + f) * TSZ + (size_t)ly * G.TXm + lx;
    };

    // ---- owned points: q = tid + r * nthreads over the extended region, x fastest
    int pex[P], pey[P];
    bool pv[P], ptile[P], pband[P];
#pragma unroll
    for (int r = 0; r < P; ++r) {
        const int q = tid + r * nthr;
        pv[r] = q < NP;
        pex[r] = pv[r] ? q % EW : 0;
        pey[r] = pv[r] ? q / EW : 0;
        const int x = X0 + pex[r], y = Y0 + pey[r];
        ptile[r] = pv[r] && x >= x0 && x < x1 && y >= y0 && y < y1;
        pband[r] = ptile[r] && ((hasL && x - x0 < H) || (hasR && x1 - 1 - x < H) || (hasD && y - y0 < H) ||
                                (hasU && y1 - 1 - y < H));
    }

    float ph[P][K], ux[P][K], uy[P][K], bb[P][K], w[P][LKv];
#pragma unroll
    for (int r = 0; r < P; ++r) {
        const int x = X0 + pex[r], y = Y0 + pey[r];
        const size_t p = (size_t)y * n + x;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            ph[r][c] = ux[r][c] = uy[r][c] = bb[r][c] = 0.0f;
            if (pv[r]) bb[r][c] = a.rho1[c * nn + p] - a.rho0[c * nn + p];
            if (ptile[r] && a.warm) {
                ph[r][c] = a.phi[c * nn + p];
                ux[r][c] = (x < n - 1) ? a.u[c * nn + p] : 0.0f;
                uy[r][c] = (y < n - 1) ? a.u[(k + c) * nn + p] : 0.0f;
            }
        }
#pragma unroll
        for (int e = 0; e < LKv; ++e) w[r][e] = (ptile[r] && a.warm && e < l) ? a.w[e * nn + p] : 0.0f;
    }
    if (tid == 0) { dec[0] = 0; dec[2] = 0; }

    // ---- halo exchange number e: publish the tile's band, receive the ring.  Before
    // a check, the ring points also record u_new - u_old in sdx / sdy.
    auto exchange = [&](int e, bool rec_delta) -> bool {
        const uint32_t tag = (uint32_t)e + 1u;
        const int par = e & 1;
#pragma unroll
        for (int r = 0; r < P; ++r) {
            if (!pband[r]) continue;
            const int lx = X0 + pex[r] - x0, ly = Y0 + pey[r] - y0;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                st_tagged(xword(tile, par, c, ly, lx), ph[r][c], tag);
                st_tagged(xword(tile, par, K + c, ly, lx), ux[r][c], tag);
                st_tagged(xword(tile, par, 2 * K + c, ly, lx), uy[r][c], tag);
            }
#pragma unroll
            for (int e2 = 0; e2 < LKv; ++e2)
                if (e2 < l) st_tagged(xword(tile, par, 3 * K + e2, ly, lx), w[r][e2], tag);
        }
        bool ok = true;
#pragma unroll
        for (int r = 0; r < P; ++r) {
            if (!pv[r] || ptile[r] || !ok) continue;
            const int x = X0 + pex[r], y = Y0 + pey[r];
            const int sgx = x < x0 ? gx - 1 : (x >= x1 ? gx + 1 : gx);
            const int sgy = y < y0 ? gy - 1 : (y >= y1 ? gy + 1 : gy);
            const int src = sgy * G.Gx + sgx;
            const int slx = x - sgx * n / G.Gx, sly = y - sgy * n / G.Gy;
            float vals[FMAX];
#pragma unroll
            for (int q = 0; q < FMAX; ++q) vals[q] = 0.0f;
            ok = poll_words<16>(
                F, tag, a.ctl, [&](int f) { return xword(src, par, f, sly, slx); },
                [&](int f, uint32_t bits) {
#pragma unroll
                    for (int q = 0; q < FMAX; ++q)
                        if (q == f) vals[q] = __uint_as_float(bits);
                });
            if (!ok) continue;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                if (rec_delta) {
                    SA(sdx, c, pey[r], pex[r]) = vals[K + c] - ux[r][c];
                    SA(sdy, c, pey[r], pex[r]) = vals[2 * K + c] - uy[r][c];
                }
                ph[r][c] = vals[c];
                ux[r][c] = vals[K + c];
                uy[r][c] = vals[2 * K + c];
                SA(sphi, c, pey[r], pex[r]) = ph[r][c];
            }
#pragma unroll
            for (int e2 = 0; e2 < LKv; ++e2)
                if (e2 < l) w[r][e2] = vals[3 * K + e2];
        }
        return ok;
    };

    // initial iterate: own phi to shared memory, then the first exchange
#pragma unroll
    for (int r = 0; r < P; ++r)
        if (ptile[r])
#pragma unroll
            for (int c = 0; c < K; ++c) SA(sphi, c, pey[r], pex[r]) = ph[r][c];
    if (!exchange(0, false)) dec[0] = 1;
    __syncthreads();
    bool aborted = dec[0] != 0;
    int nexch = 1, checks = 0, t = 0;
    bool stop = false;

    float dph[P][K], dgw[P][K], racc[P][K];
#pragma unroll
    for (int r = 0; r < P; ++r)
#pragma unroll
        for (int c = 0; c < K; ++c) { dph[r][c] = 0.0f; dgw[r][c] = 0.0f; racc[r][c] = 0.0f; }
    while (!aborted && !stop) {
        // a block of iterations runs to the next check (or the end) or H iterations
        int hb = 0;
        if (T > 0) {
            const int next_check = ((t / CE) + 1) * CE;
            hb = H;
            if (t + hb > next_check) hb = next_check - t;
            if (t + hb > T) hb = T - t;
        }
        const int t_end = t + hb;
        const bool check_after = (T == 0) || (t_end % CE == 0) || (t_end == T);
        double v[NRED];
#pragma unroll
        for (int q = 0; q < NRED; ++q) v[q] = 0.0;
        for (int s = 1; s <= hb; ++s) {
            const int rr = hb - s;                 // ring width of the region this step updates
            const bool last = (s == hb) && check_after;
            const int rl = hasL ? rr : 0, rrt = hasR ? rr : 0, rd = hasD ? rr : 0, ru = hasU ? rr : 0;
            const int rlp = hasL ? rr + 1 : 0, rdp = hasD ? rr + 1 : 0;
            // phase 1: u' on the region plus one column left and one row below (their
            // ubar enters the divergence); w' and the commit on the region itself
#pragma unroll
            for (int r = 0; r < P; ++r) {
                const int x = X0 + pex[r], y = Y0 + pey[r];
                const bool inRp = pv[r] && x >= x0 - rlp && x < x1 + rrt && y >= y0 - rdp && y < y1 + ru;
                if (!inRp) continue;
                const bool inR = x >= x0 - rl && y >= y0 - rd;
                const int ex = pex[r], ey = pey[r];
                float vx[K], vy[K];
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const float pc = ph[r][c];
                    vx[c] = ux[r][c] + ((x < n - 1) ? muih * (SA(sphi, c, ey, ex + 1) - pc) : 0.0f);
                    vy[c] = uy[r][c] + ((y < n - 1) ? muih * (SA(sphi, c, ey + 1, ex) - pc) : 0.0f);
                }
                shrink_u<K>(vx, vy, mu, a.un, a.g.wc);
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    SA(sux, c, ey, ex) = 2.0f * vx[c] - ux[r][c];
                    SA(suy, c, ey, ex) = 2.0f * vy[c] - uy[r][c];
                }
                if (!inR) continue;
                float wx[LKv];
#pragma unroll
                for (int e = 0; e < LKv; ++e) {
                    float ge = 0.0f;
#pragma unroll
                    for (int c = 0; c < K; ++c) ge += a.g.G[e][c] * ph[r][c];
                    wx[e] = (e < l) ? w[r][e] + nu * ge : 0.0f;
                }
                shrink_w<LKv>(wx, l, alpha * nu, a.wn, a.g.we);
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    float gw = 0.0f, gd = 0.0f;
#pragma unroll
                    for (int e = 0; e < LKv; ++e) {
                        gw -= a.g.Dv[c][e] * (2.0f * wx[e] - w[r][e]);
                        gd -= a.g.Dv[c][e] * (wx[e] - w[r][e]);
                    }
                    racc[r][c] = gw + bb[r][c];
                    if (last) dgw[r][c] = gd;
                }
                if (last) {
#pragma unroll
                    for (int c = 0; c < K; ++c) {
                        const float dux = vx[c] - ux[r][c], duy = vy[c] - uy[r][c];
                        SA(sdx, c, ey, ex) = dux;
                        SA(sdy, c, ey, ex) = duy;
                        v[RED_DU] += (double)(a.g.wc[c] * (dux * dux + duy * duy));
                    }
#pragma unroll
                    for (int e = 0; e < LKv; ++e) {
                        const float dw = wx[e] - w[r][e];
                        v[RED_DW] += (double)(a.g.we[e] * dw * dw);
                    }
                }
#pragma unroll
                for (int c = 0; c < K; ++c) { ux[r][c] = vx[c]; uy[r][c] = vy[c]; }
#pragma unroll
                for (int e = 0; e < LKv; ++e) w[r][e] = wx[e];
            }
            __syncthreads();
            // phase 2: phi' = phi + tau (div_x ubar + div_G wbar + rho1 - rho0) on the region
#pragma unroll
            for (int r = 0; r < P; ++r) {
                const int x = X0 + pex[r], y = Y0 + pey[r];
                const bool inR = pv[r] && x >= x0 - rl && x < x1 + rrt && y >= y0 - rd && y < y1 + ru;
                if (!inR) continue;
                const int ex = pex[r], ey = pey[r];
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const float xl = (x > 0) ? SA(sux, c, ey, ex - 1) : 0.0f;
                    const float yd = (y > 0) ? SA(suy, c, ey - 1, ex) : 0.0f;
                    const float d = ih * ((SA(sux, c, ey, ex) - xl) + (SA(suy, c, ey, ex) - yd)) + racc[r][c];
                    const float np = ph[r][c] + tau * d;
                    if (last) dph[r][c] = np - ph[r][c];
                    ph[r][c] = np;
                    SA(sphi, c, ey, ex) = np;
                }
            }
            __syncthreads();
        }
        t = t_end;
        // ---- refresh the ring (and, before a check, record u_new - u_old on it)
        if (hb > 0) {
            if (!exchange(nexch, check_after)) dec[0] = 1;
            ++nexch;
            __syncthreads();
            if (dec[0]) { aborted = true; break; }
        }
        if (!check_after) continue;

        // ---- FP64 convergence check of the iterate after iteration t
        if (T == 0) {
#pragma unroll
            for (int r = 0; r < P; ++r)
                if (pv[r])
#pragma unroll
                    for (int c = 0; c < K; ++c) { SA(sdx, c, pey[r], pex[r]) = 0.0f; SA(sdy, c, pey[r], pex[r]) = 0.0f; }
        }
#pragma unroll
        for (int r = 0; r < P; ++r) {
            if (!pv[r]) continue;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                SA(sux, c, pey[r], pex[r]) = ux[r][c];
                SA(suy, c, pey[r], pex[r]) = uy[r][c];
            }
        }
        __syncthreads();
        // Per-point terms in FP32, summed over this thread's few points in FP32
        // and then over the grid in FP64 (FP64 arithmetic is scarce on this GPU).
        // The constraint residual, which cancels several digits, is formed in FP64.
        float fs[NRED];
#pragma unroll
        for (int q = 0; q < NRED; ++q) fs[q] = 0.0f;
#pragma unroll
        for (int r = 0; r < P; ++r) {
            if (!ptile[r]) continue;
            const int x = X0 + pex[r], y = Y0 + pey[r], ex = pex[r], ey = pey[r];
            const double dih = (double)(n - 1);
            float nu_pt = 0.0f, dn_u = 0.0f;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const float uxc = ux[r][c], uyc = uy[r][c], phc = ph[r][c], bc = bb[r][c], wgt = a.g.wc[c];
                const float xl = (x > 0) ? SA(sux, c, ey, ex - 1) : 0.0f;
                const float yd = (y > 0) ? SA(suy, c, ey - 1, ex) : 0.0f;
                const float dxl = (x > 0) ? SA(sdx, c, ey, ex - 1) : 0.0f;
                const float dyd = (y > 0) ? SA(sdy, c, ey - 1, ex) : 0.0f;
                const float ddiv = ih * ((SA(sdx, c, ey, ex) - dxl) + (SA(sdy, c, ey, ex) - dyd)) + dgw[r][c];
                float gwb = bc;
#pragma unroll
                for (int e = 0; e < LKv; ++e) gwb -= a.g.Dv[c][e] * w[r][e];
                const double rc = dih * (((double)uxc - (double)xl) + ((double)uyc - (double)yd)) + (double)gwb;
                v[RED_RR] += (double)wgt * rc * rc;
                fs[RED_BB] += wgt * bc * bc;
                fs[RED_D] += wgt * phc * bc;
                fs[RED_DP] += wgt * dph[r][c] * dph[r][c];
                fs[RED_X] += wgt * dph[r][c] * ddiv;
                const float gxx = (x < n - 1) ? ih * (SA(sphi, c, ey, ex + 1) - phc) : 0.0f;
                const float gyy = (y < n - 1) ? ih * (SA(sphi, c, ey + 1, ex) - phc) : 0.0f;
                if (a.un == VOMT_U_L12) {
                    nu_pt += sqrtf(uxc * uxc + uyc * uyc);
                    dn_u = fmaxf(dn_u, sqrtf(gxx * gxx + gyy * gyy));
                } else if (a.un == VOMT_U_L2) {
                    nu_pt += a.g.wc[c] * (uxc * uxc + uyc * uyc);
                    dn_u += a.g.wc[c] * (gxx * gxx + gyy * gyy);
                } else {
                    nu_pt += a.g.wc[c] * (fabsf(uxc) + fabsf(uyc));
                    dn_u = fmaxf(dn_u, fmaxf(fabsf(gxx), fabsf(gyy)));
                }
            }
            if (a.un == VOMT_U_L2) { nu_pt = sqrtf(nu_pt); dn_u = sqrtf(dn_u); }
            float nw_pt = 0.0f, dn_w = 0.0f;
#pragma unroll
            for (int e = 0; e < LKv; ++e) {
                if (e < l) {
                    float ge = 0.0f;
#pragma unroll
                    for (int c = 0; c < K; ++c) ge += a.g.G[e][c] * ph[r][c];
                    const float we = w[r][e], wgt = a.g.we[e];
                    if (a.wn == VOMT_W_L1) { nw_pt += wgt * fabsf(we); dn_w = fmaxf(dn_w, fabsf(ge)); }
                    else { nw_pt += wgt * we * we; dn_w += wgt * ge * ge; }
                }
            }
            if (a.wn == VOMT_W_L2) { nw_pt = sqrtf(nw_pt); dn_w = sqrtf(dn_w); }
            fs[RED_P] += nu_pt + alpha * nw_pt;
            float di = fmaxf(dn_u - 1.0f, 0.0f);
            if (l > 0) di = fmaxf(di, dn_w - alpha);
            fs[RED_MAX] = fmaxf(fs[RED_MAX], di);
        }
        v[RED_P] += (double)fs[RED_P];
        v[RED_D] += (double)fs[RED_D];
        v[RED_BB] += (double)fs[RED_BB];
        v[RED_DP] += (double)fs[RED_DP];
        v[RED_X] += (double)fs[RED_X];
        v[RED_MAX] = fmax(v[RED_MAX], (double)fs[RED_MAX]);
        // block reduction (fixed order)
        const int lane = tid & 31, wid = tid >> 5, nw = (nthr + 31) >> 5;
#pragma unroll
        for (int q = 0; q < NRED; ++q) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double o = __shfl_down_sync(0xffffffffu, v[q], off);
                v[q] = (q == RED_MAX) ? fmax(v[q], o) : v[q] + o;
            }
        }
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < NRED; ++q) red[wid * NRED + q] = v[q];
        __syncthreads();
        const int cpar = checks & 1;
        const uint32_t ctag = (uint32_t)checks + 1u;
        const int words = NT * NRED * 2;
        if (tid < NRED) {
            double acc = red[tid];
            for (int q = 1; q < nw; ++q) acc = (tid == RED_MAX) ? fmax(acc, red[q * NRED + tid]) : acc + red[q * NRED + tid];
            unsigned long long *dst = a.rows + (size_t)cpar * words + ((size_t)tile * NRED + tid) * 2;
            st_tagged(dst, __int_as_float(__double2hiint(acc)), ctag);
            st_tagged(dst + 1, __int_as_float(__double2loint(acc)), ctag);
        }
        // every block gathers every row (one L2 round trip), then sums them in block order
        {
            const int mine = tid < words ? (words - tid + nthr - 1) / nthr : 0;
            const bool ok = poll_words<8>(
                mine, ctag, a.ctl, [&](int j) { return a.rows + (size_t)cpar * words + (size_t)tid + (size_t)j * nthr; },
                [&](int j, uint32_t bits) {
                    const int widx = tid + j * nthr;
                    ((uint32_t *)rtab)[(widx >> 1) * 2 + ((widx & 1) ? 0 : 1)] = bits;
                });
            if (!ok) dec[0] = 1;
        }
        __syncthreads();
        if (dec[0]) { aborted = true; break; }
        if (tid < NRED) {
            double acc = 0.0;
            for (int b = 0; b < NT; ++b) {
                const double x_ = rtab[b * NRED + tid];
                acc = (tid == RED_MAX) ? fmax(acc, x_) : acc + x_;
            }
            S[tid] = acc;
        }
        __syncthreads();
        if (tid == 0) {
            double m[NMET];
            m[0] = S[RED_P];
            m[1] = S[RED_D];
            m[2] = fabs(m[0] - m[1]) / fmax(fabs(m[0]), 1e-300);
            m[3] = sqrt(S[RED_RR]) / (S[RED_BB] > 0.0 ? sqrt(S[RED_BB]) : 1.0);
            m[4] = S[RED_DU] / a.cfg.mu + (a.cfg.has_w ? S[RED_DW] / a.cfg.nu : 0.0) + S[RED_DP] / a.cfg.tau -
                   2.0 * S[RED_X];
            m[5] = S[RED_MAX];
            m[6] = (double)t;
            bool finite = true;
            for (int q = 0; q < 6; ++q) finite = finite && isfinite(m[q]);
            const bool conv = a.cfg.tol_gap > 0.0 && m[2] <= a.cfg.tol_gap && m[3] <= a.cfg.tol_res;
            m[7] = conv ? 1.0 : 0.0;
            if (tile == 0) {
                for (int q = 0; q < NMET; ++q) a.st->met[q] = m[q];
                if (a.hist && checks < a.hist_cap)
                    for (int q = 0; q < NMET; ++q) a.hist[(size_t)checks * NMET + q] = m[q];
                a.st->checks = checks + 1;
                a.st->iter = t;
                if (!finite) a.st->error = VOMT_ERR_NONFINITE;
                if (conv || !finite) a.st->stop = 1;
            }
            dec[2] = (conv || !finite || t >= T) ? 1 : 0;
        }
        __syncthreads();
        ++checks;
        stop = dec[2] != 0;
    }
    if (aborted) {
        if (tid == 0 && tile == 0) {
            a.st->error = VOMT_ERR_BARRIER_TIMEOUT;
            a.st->stop = 1;
        }
        return;
    }
    // ---- final iterate of the tile to the caller's arrays
#pragma unroll
    for (int r = 0; r < P; ++r) {
        if (!ptile[r]) continue;
        const size_t p = (size_t)(Y0 + pey[r]) * n + (X0 + pex[r]);
#pragma unroll
        for (int c = 0; c < K; ++c) {
            a.phi[c * nn + p] = ph[r][c];
            a.u[c * nn + p] = ux[r][c];
            a.u[(k + c) * nn + p] = uy[r][c];
        }
#pragma unroll
        for (int e = 0; e < LKv; ++e)
            if (e < l) a.w[e * nn + p] = w[r][e];
    }
#undef SA
}

using ResKernel = void (*)(ResArgs);

template <int P>
ResKernel pick_k(int k)
{
    switch (k) {
        case 1: return k_resident<1, P>;
        case 2: return k_resident<2, P>;
        case 3: return k_resident<3, P>;
        case 4: return k_resident<4, P>;
        case 5: return k_resident<5, P>;
        case 6: return k_resident<6, P>;
        case 7: return k_resident<7, P>;
        default: return k_resident<8, P>;
    }
}

ResKernel pick_kernel(int k, int P) { return P == 1 ? pick_k<1>(k) : (P == 2 ? pick_k<2>(k) : pick_k<4>(k)); }

// Estimated nanoseconds per iteration (see resident_plan).  Constants fitted to
// GB300 measurements of this kernel at k = 3: 3.5 ns per point of the region a
// step updates (arithmetic, shared-memory traffic and the two barriers of a
// step at 16 warps per SM), 3.1 us per halo exchange (one L2 round trip plus
// the tagged stores and polls), and 30% more per point when a thread owns
// four points (register spills; extended tiles above RES_P4_POINTS).
double plan_cost(int TX, int TY, int H, int G)
{
    const double per_pt = 3.5;
    if (G == 1) return per_pt * TX * TY * (TX * TY > RES_P4_POINTS ? 1.3 : 1.0);
    double pts = 0.0;
    for (int s = 1; s <= H; ++s) pts += (double)(TX + 2 * (H - s) + 1) * (TY + 2 * (H - s) + 1);
    const int ext = (TX + 2 * H) * (TY + 2 * H);
    return per_pt * (ext > RES_P4_POINTS ? 1.3 : 1.0) * pts / H + 3100.0 / H;
}

}  // namespace

// Tile plan.  Tiles of at most 64 x 64 points, at most `max_blocks` of them; the
// ring width H is at most the narrowest tile side; the extended tile
// (TX + 2H) x (TY + 2H) holds at most RES_MAX_POINTS points.
// Among those, the plan with the smallest estimated time per iteration
// (plan_cost) wins.  `force_H` > 0 pins the ring width.
bool resident_plan(int n, int k, int max_blocks, int force_H, ResidentPlan *out)
{
    (void)k;
    double best = -1.0;
    for (int Gx = 1; Gx <= n && Gx <= max_blocks; ++Gx) {
        const int TX = (n + Gx - 1) / Gx, TXmin = n / Gx;
        if (TX > TMAX) continue;
        for (int Gy = 1; Gy <= n && Gx * Gy <= max_blocks; ++Gy) {
            const int TY = (n + Gy - 1) / Gy, TYmin = n / Gy;
            if (TY > TMAX) continue;
            const int G = Gx * Gy;
            if (G == 1) {
                if (TX * TY > RES_MAX_POINTS) continue;
                const double cost = plan_cost(TX, TY, 0, 1);
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
                if (EW * EH > RES_MAX_POINTS) break;
                const double cost = plan_cost(TX, TY, H, G);
                if (best < 0 || cost < best) {
                    best = cost;
                    *out = ResidentPlan{Gx, Gy, TX, TY, H, 0, 0, cost};
                }
            }
        }
    }
    if (best < 0) return false;
    const int EW = out->TXm + 2 * out->H, EH = out->TYm + 2 * out->H;
    // P points per thread, the fewest that fit 512 threads, spread evenly over
    // round_up(ext / P, 32) threads.
    const int ext = EW * EH;
    out->P = ext <= RES_THREADS ? 1 : (ext <= 2 * RES_THREADS ? 2 : 4);
    out->threads = (((ext + out->P - 1) / out->P + 31) / 32) * 32;
    return true;
}

int resident_solve(vomt_ctx *ctx, const OpDev &g, const StepDev &s, const SolveCfg &cfg, const vomt_params &p,
                   const ResidentPlan &plan, const float *rho0, const float *rho1, float *u, float *w, float *phi,
                   cudaStream_t st)
{
    const int K = g.k, F = 3 * K + g.l;
    const int G = plan.Gx * plan.Gy;
    const int EWm = plan.TXm + 2 * plan.H, EHm = plan.TYm + 2 * plan.H;
    const SmemLayout SL = smem_layout(K, EWm, EHm, G);
    if (SL.total > 227 * 1024) {
        ctx->err = "resident plan needs too much shared memory";
        return VOMT_ERR_TOO_LARGE;
    }
    const size_t xch_bytes = (size_t)G * 2 * F * plan.TXm * plan.TYm * sizeof(unsigned long long);
    const size_t rows_bytes = (size_t)2 * G * NRED * 2 * sizeof(unsigned long long);
    const size_t need = xch_bytes + rows_bytes + 256;
    int rc = ensure_buffer(ctx, &ctx->rscratch, &ctx->rscratch_bytes, need, "resident scratch");
    if (rc) return rc;
    unsigned char *base = (unsigned char *)ctx->rscratch;
    ResArgs a;
    memset(&a, 0, sizeof a);
    // a single tile never exchanges, so its blocks of iterations may be as long as a check interval
    const int H = G == 1 ? (1 << 30) : plan.H;
    a.geo = ResGeom{s.n, plan.Gx, plan.Gy, plan.TXm, plan.TYm, H, EWm, EHm};
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
    a.ctl = (ResCtl *)(base + xch_bytes + rows_bytes);
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

    ResKernel kern = pick_kernel(K, plan.P);
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
