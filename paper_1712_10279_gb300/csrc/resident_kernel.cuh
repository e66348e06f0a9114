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
// Points are owned by threads for the whole solve (up to P points per thread),
// numbered tile first and then ring by ring (resident_order.h), so that the
// shrinking region of every step is a prefix of the numbering: a step's idle
// points are whole idle warps.  Each thread keeps its points' iterate and
// b = rho1 - rho0 in registers.  The stencils of Appendix A within a block read
// neighbouring phi and ubar from shared memory, where a point's channels sit
// side by side (padded to 1, 2 or a multiple of 4 floats) so that one vector
// load fetches them all.  At the edges of the grid the neighbour offsets are
// zero (the forward difference then vanishes) and the backward neighbours are
// masked, so the stencil has no branches.
//
// Between blocks, every iterate value a neighbour needs is written to L2 as a
// 64-bit word with the value in its low half and the exchange number in its
// high half; words go in pairs (one 16-byte vector access per two fields).  A
// reader polls the words themselves, so a halo exchange costs one L2 round trip
// and no fences or flags (each aligned 64-bit element of a vector access is
// single-copy atomic).
//
// Convergence checks (every check_every iterations and at the end; a block of
// iterations is cut short so that it ends on a check) form the metric terms of
// each point in FP32 (the constraint residual with error-free transformations,
// to about twice FP32 precision), sum them per thread in FP32 and per block in
// FP64, publish one row per block as tagged word pairs, and every block sums
// all rows in the same fixed order, so all blocks take the same stopping
// decision.  Every wait is bounded in time; a wait that runs out raises a
// global abort word that makes every block return.
#pragma once

#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "internal.h"
#include "pdhg_device.cuh"
#include "resident_order.h"

namespace vomt {
namespace res {

using namespace dev;

constexpr int RES_THREADS = 512;      // most threads a block runs
// Five and more channels: at most 384 threads (12 warps, three per SM
// sub-partition), so that a thread may hold 170 registers; with 13 or more warps
// some sub-partition holds four and a thread gets 128, under which their
// per-point state spills.
__host__ __device__ constexpr int res_threads(int K) { return K >= 5 ? 384 : RES_THREADS; }
constexpr int HMAX = 16;              // widest halo ring

template <int K>
struct LK {
    static constexpr int v = K * (K - 1) / 2 > 0 ? K * (K - 1) / 2 : 1;
};

// floats per point in the shared-memory arrays: the channels padded to a vector width
__host__ __device__ constexpr int kv_of(int K) { return K == 1 ? 1 : (K == 2 ? 2 : ((K + 3) / 4) * 4); }

// padded row length (points) of the shared-memory arrays: odd, so that the
// column segments of the ring fall in distinct banks
__host__ __device__ inline int row_stride(int EWm) { return EWm | 1; }

struct ResGeom {
    int n, Gx, Gy, TXm, TYm;
    int H;         // iterations per block of steps between exchanges
    int R;         // ring width (H with neighbour tiles, 0 for a lone tile)
    int EWs, EHm;  // shared-memory array rows: padded length, count
};

struct ResArgs {
    ResGeom geo;
    OpDev g;                   // per-point grad / div and inner-product weights
    StepDev s;
    SolveCfg cfg;
    int un, wn, max_iters, check_every, warm;
    const float *rho0, *rho1;
    float *u, *w, *phi;
    unsigned long long *xch;   // [G][2][F2][TYm][TXm][2] tagged words, pair j = fields 2j, 2j+1
    unsigned long long *rows;  // [2][G][NRED][2] tagged halves of the FP64 partial sums
    ResCtl *ctl;
    DevStatus *st;
    double *hist;
    int hist_cap;
    unsigned long long wait_ns;  // time limit of one wait of a block on another
    int drop_exch;             // > 0: block 0 skips publishing this halo exchange (wait tests)
    uint32_t tag_hi;           // added to every tag of a grouped job: (instance + 1) << 20
};

struct SmemLayout {
    int red, S, dec, rtab, cnt, sphi, sux, suy, sdx, sdy, sdg, total;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }
__host__ __device__ inline int align128(int x) { return (x + 127) & ~127; }

__host__ __device__ inline SmemLayout smem_layout(int K, int EWs, int EHm, int G)
{
    SmemLayout L;
    int o = 0;
    const int plane = EWs * EHm * kv_of(K) * 4;
    L.red = o; o += align16((RES_THREADS / 32) * NRED * 8);
    L.S = o; o += align16(NRED * 8);
    L.dec = o; o += 16;
    L.rtab = o; o += align16(G * NRED * 8);
    L.cnt = o; o += align16(2 * (HMAX + 2) * 4);
    o = align128(o);           // the point arrays start on 128-byte boundaries (half_swap)
    L.sphi = o; o += align128(plane);
    L.sux = o; o += align128(plane);
    L.suy = o; o += align128(plane);
    L.sdx = o; o += align128(plane);
    L.sdy = o; o += align128(plane);
    L.sdg = o; o += align128(plane);
    L.total = o;
    return L;
}

// ---------------------------------------------------------------- small helpers
// A point's record of 8 floats (5 to 8 channels) holds two 16-byte halves.  Eight
// lanes of a warp reading the same half of eight consecutive records would touch
// every bank group twice; so the halves are swapped in every other group of four
// records (bit 2 of the record index, bit 7 of the shared-memory byte address with
// 128-byte aligned arrays), which spreads any eight consecutive records over all
// eight bank groups.
template <int KV>
__device__ __forceinline__ int half_swap(const float *p)
{
    if constexpr (KV == 8)
        return (int)((__cvta_generic_to_shared(p) >> 5) & 4u);   // 4 floats where the halves swap
    else
        return 0;
}

// K channel values of one point from / to a shared-memory array (vector accesses)
template <int K>
__device__ __forceinline__ void lds(const float *p, float (&v)[K])
{
    constexpr int KV = kv_of(K);
    float t[KV];
    if constexpr (KV == 1) {
        t[0] = p[0];
    } else if constexpr (KV == 2) {
        const float2 a = *reinterpret_cast<const float2 *>(p);
        t[0] = a.x;
        t[1] = a.y;
    } else {
        const int sw = half_swap<KV>(p);
#pragma unroll
        for (int j = 0; j < KV / 4; ++j) {
            const float4 a = *reinterpret_cast<const float4 *>(p + ((4 * j) ^ sw));
            t[4 * j] = a.x;
            t[4 * j + 1] = a.y;
            t[4 * j + 2] = a.z;
            t[4 * j + 3] = a.w;
        }
    }
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = t[c];
}

template <int K>
__device__ __forceinline__ void sts(float *p, const float (&v)[K])
{
    constexpr int KV = kv_of(K);
    float t[KV];
#pragma unroll
    for (int c = 0; c < KV; ++c) t[c] = 0.0f;
#pragma unroll
    for (int c = 0; c < K; ++c) t[c] = v[c];
    if constexpr (KV == 1) {
        p[0] = t[0];
    } else if constexpr (KV == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(t[0], t[1]);
    } else {
        const int sw = half_swap<KV>(p);
#pragma unroll
        for (int j = 0; j < KV / 4; ++j)
            *reinterpret_cast<float4 *>(p + ((4 * j) ^ sw)) =
                make_float4(t[4 * j], t[4 * j + 1], t[4 * j + 2], t[4 * j + 3]);
    }
}

// ih * ((ux - xl) + (uy - yd)) + gb with the rounding errors of the
// differences, their sum, the product and the final sum carried along (the
// compensated evaluation of Ogita, Rump and Oishi, "Accurate sum and dot
// product", 2005): about twice FP32 precision for the constraint residual,
// whose terms cancel as the iteration converges.
__device__ __forceinline__ float residual_c(float ih, float ux, float xl, float uy, float yd, float gb)
{
    float e1, e2, e3, e4;
    const float d1 = two_sum(ux, -xl, e1);
    const float d2 = two_sum(uy, -yd, e2);
    const float s = two_sum(d1, d2, e3);
    const float p = ih * s;
    const float pe = fmaf(ih, s, -p);
    const float r = two_sum(p, gb, e4);
    return r + (e4 + (pe + ih * ((e1 + e2) + e3)));
}

// Two tagged words (fields 2j and 2j+1 of one point) in one 16-byte access.
__device__ __forceinline__ void st_tagged2(unsigned long long *p, float v0, float v1, uint32_t tag)
{
    const unsigned long long w0 = ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v0);
    const unsigned long long w1 = ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v1);
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(w0), "l"(w1) : "memory");
}

__device__ __forceinline__ void ld_relaxed64x2(const unsigned long long *p, unsigned long long &w0,
                                               unsigned long long &w1)
{
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(w0), "=l"(w1) : "l"(p) : "memory");
}

// Poll `cnt` tagged words (addresses from `addr(j)`), handing each value to
// `sink(j, bits)` once its tag matches.  All pending words of a batch are
// re-read every round.  Returns false once the wait exceeds `budget` ns (raising
// the abort word) or another block has aborted.
template <int BATCH, typename Addr, typename Sink>
__device__ __forceinline__ bool poll_words(int cnt, uint32_t tag, ResCtl *ctl, uint64_t budget, Addr addr, Sink sink)
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
                if (global_ns() - t0 > budget) {
                    atomicExch(&ctl->abort, 1u);
                    atomicExch(&ctl->where, 1u);
                    return false;
                }
            }
        }
    }
    return true;
}

// Poll `cnt` <= NP2 tagged word pairs (addresses from `addr(j)`) until both
// tags of every pair match; the values land in vals[2j], vals[2j+1].  Pairs go
// in batches of up to 8: every round issues the batch's pending loads first
// (in-order issue would otherwise expose one L2 latency per pair), then checks
// the tags.  Returns false on timeout (`budget` ns) or abort.
template <int NP2, typename Addr>
__device__ __forceinline__ bool poll_pairs(int cnt, uint32_t tag, ResCtl *ctl, uint64_t budget, Addr addr,
                                           float (&vals)[2 * NP2])
{
    constexpr int B = NP2 < 8 ? NP2 : 8;
#pragma unroll
    for (int base = 0; base < NP2; base += B) {
        if (base >= cnt) break;
        uint32_t pending = 0;
#pragma unroll
        for (int j = 0; j < B; ++j)
            if (base + j < cnt && base + j < NP2) pending |= 1u << j;
        uint64_t t0 = 0;
        for (uint32_t round = 0; pending; ++round) {
            unsigned long long w0[B], w1[B];
#pragma unroll
            for (int j = 0; j < B; ++j) {
                w0[j] = w1[j] = 0ull;
                if (pending >> j & 1u) ld_relaxed64x2(addr(base + j), w0[j], w1[j]);
            }
#pragma unroll
            for (int j = 0; j < B; ++j) {
                if ((pending >> j & 1u) && (uint32_t)(w0[j] >> 32) == tag && (uint32_t)(w1[j] >> 32) == tag) {
                    if (base + j < NP2) {
                        vals[2 * (base + j)] = __uint_as_float((uint32_t)w0[j]);
                        vals[2 * (base + j) + 1] = __uint_as_float((uint32_t)w1[j]);
                    }
                    pending &= ~(1u << j);
                }
            }
            if (pending && (round & 63u) == 63u) {
                if (t0 == 0) t0 = global_ns();
                if (ld_relaxed32(&ctl->abort)) return false;
                if (global_ns() - t0 > budget) {
                    atomicExch(&ctl->abort, 1u);
                    atomicExch(&ctl->where, 2u);
                    return false;
                }
            }
        }
    }
    return true;
}

// ------------------------------------------------------------------ the kernel
// NM = 1: the norms are the vector default pair (||u||_{1,2}, ||w||_1), fixed at
// compile time; NM = 2: the matrix default pair (||U||_2, ||W||_1); NM = 3: both
// nuclear norms (||U||_{1,nuc}, ||W||_{1,nuc}; 3 x 3 matrices); NM = 0: the norms
// are read from the arguments.  LF > 0 fixes the number of flux entries per point
// at compile time (9 for 3 x 3 matrices with three L matrices: the flux loops then
// run over 9 entries instead of the 15 that a 3 x 3 problem may have); LF = 0
// reads it from the operator.
template <int K, int P, int NM, int LF = 0>
__device__ __forceinline__ void resident_body(const ResArgs &a, const int tile, const int NT, const uint32_t tag_hi)
{
    constexpr int LKv = LF > 0 ? LF : LK<K>::v;
    constexpr int FMAX = 3 * K + LKv;
    constexpr int F2MAX = (FMAX + 1) / 2;
    constexpr int KV = kv_of(K);
    extern __shared__ __align__(128) unsigned char smem[];
    const ResGeom G = a.geo;
    const int n = G.n, H = G.H, R = G.R;
    const size_t nn = (size_t)n * n;
    const SmemLayout SL = smem_layout(K, G.EWs, G.EHm, NT);
    double *red = (double *)(smem + SL.red);
    double *S = (double *)(smem + SL.S);
    int *dec = (int *)(smem + SL.dec);
    double *rtab = (double *)(smem + SL.rtab);
    int *cntR = (int *)(smem + SL.cnt), *cntRp = cntR + (HMAX + 2);
    float *sphi = (float *)(smem + SL.sphi), *sux = (float *)(smem + SL.sux), *suy = (float *)(smem + SL.suy);
    float *sdx = (float *)(smem + SL.sdx), *sdy = (float *)(smem + SL.sdy), *sdg = (float *)(smem + SL.sdg);

    const int gx = tile % G.Gx, gy = tile / G.Gx;
    TileFrame fr;
    fr.x0 = gx * n / G.Gx;
    fr.x1 = (gx + 1) * n / G.Gx;
    fr.y0 = gy * n / G.Gy;
    fr.y1 = (gy + 1) * n / G.Gy;
    fr.hL = gx > 0;
    fr.hR = gx < G.Gx - 1;
    fr.hD = gy > 0;
    fr.hU = gy < G.Gy - 1;
    fr.R = R;
    const int X0 = fr.x0 - fr.hL * R, Y0 = fr.y0 - fr.hD * R;
    const int NTILE = (fr.x1 - fr.x0) * (fr.y1 - fr.y0);
    const int NP = region_count(fr, R);
    const int RS = G.EWs * KV;             // one row of a shared array, in floats

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int k = a.g.k, l = LF > 0 ? LF : a.g.l, F = 3 * K + l, F2 = (F + 1) / 2;
    const int un = NM == 1 ? (int)VOMT_U_L12 : (NM == 2 ? (int)VOMT_U_L2 : (NM == 3 ? (int)VOMT_U_NUC : a.un));
    const int wn = NM == 3 ? (int)VOMT_W_NUC : (NM ? (int)VOMT_W_L1 : a.wn);
    const float mu = a.s.mu, nu = a.s.nu, tau = a.s.tau, ih = a.s.ih, alpha = a.s.alpha;
    const float muih = mu * ih;
    const int T = a.max_iters, CE = a.check_every;
    const size_t TSZ = (size_t)G.TXm * G.TYm;
    auto xpair = [&](int t_, int par, int j, int ly, int lx) -> unsigned long long * {
        return a.xch + ((((size_t)t_ * 2 + par) * F2 + j) * TSZ + (size_t)ly * G.TXm + lx) * 2;
    };

    // ---- owned points: number q = tid + r * nthreads in the tile-then-ring order
    int pxy[P];               // x | y << 16
    int sb[P];                // index of the point in the shared arrays
    int nbf[P];               // 1: x < n-1, 2: y < n-1, 4: x > 0, 8: y > 0
    bool pv[P], ptile[P], pband[P];
#pragma unroll
    for (int r = 0; r < P; ++r) {
        const int q = tid + r * nthr;
        int x = fr.x0, y = fr.y0;
        pv[r] = q < NP && onion_point(fr, q, x, y);
        ptile[r] = pv[r] && q < NTILE;
        pxy[r] = x | (y << 16);
        sb[r] = ((y - Y0) * G.EWs + (x - X0)) * KV;
        nbf[r] = (x < n - 1 ? 1 : 0) | (y < n - 1 ? 2 : 0) | (x > 0 ? 4 : 0) | (y > 0 ? 8 : 0);
        pband[r] = ptile[r] && R > 0 &&
                   ((fr.hL && x - fr.x0 < R) || (fr.hR && fr.x1 - 1 - x < R) || (fr.hD && y - fr.y0 < R) ||
                    (fr.hU && fr.y1 - 1 - y < R));
    }

    float ph[P][K], ux[P][K], uy[P][K], bb[P][K], w[P][LKv];
#pragma unroll
    for (int r = 0; r < P; ++r) {
        const int x = pxy[r] & 0xffff, y = pxy[r] >> 16;
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
    if (tid == 0) {
        dec[0] = 0;
        dec[2] = 0;
    }
    if (tid <= R) {
        cntR[tid] = region_count(fr, tid);
        cntRp[tid] = region_p_count(fr, tid);
    }
    __syncthreads();

    // ---- publish band point r for halo exchange number e (its tagged word pairs)
    auto publish_point = [&](int r, int e) {
        if (a.drop_exch > 0 && e == a.drop_exch && tile == 0) return;
        const uint32_t tag = tag_hi + (uint32_t)e + 1u;
        const int par = e & 1;
        const int lx = (pxy[r] & 0xffff) - fr.x0, ly = (pxy[r] >> 16) - fr.y0;
        float vals[2 * F2MAX];
#pragma unroll
        for (int q = 0; q < 2 * F2MAX; ++q) vals[q] = 0.0f;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            vals[c] = ph[r][c];
            vals[K + c] = ux[r][c];
            vals[2 * K + c] = uy[r][c];
        }
#pragma unroll
        for (int e2 = 0; e2 < LKv; ++e2) vals[3 * K + e2] = w[r][e2];
#pragma unroll
        for (int j = 0; j < F2MAX; ++j)
            if (j < F2) st_tagged2(xpair(tile, par, j, ly, lx), vals[2 * j], vals[2 * j + 1], tag);
    };

    // ---- halo exchange number e: publish the tile's band (unless the last step
    // already did), receive the ring
    auto exchange = [&](int e, bool published) -> bool {
        const uint32_t tag = tag_hi + (uint32_t)e + 1u;
        const int par = e & 1;
#pragma unroll
        for (int r = 0; r < P; ++r)
            if (pband[r] && !published) publish_point(r, e);
        bool ok = true;
#pragma unroll
        for (int r = 0; r < P; ++r) {
            if (!pv[r] || ptile[r] || !ok) continue;
            const int x = pxy[r] & 0xffff, y = pxy[r] >> 16;
            const int sgx = x < fr.x0 ? gx - 1 : (x >= fr.x1 ? gx + 1 : gx);
            const int sgy = y < fr.y0 ? gy - 1 : (y >= fr.y1 ? gy + 1 : gy);
            const int src = sgy * G.Gx + sgx;
            const int slx = x - sgx * n / G.Gx, sly = y - sgy * n / G.Gy;
            float vals[2 * F2MAX];
#pragma unroll
            for (int q = 0; q < 2 * F2MAX; ++q) vals[q] = 0.0f;
            ok = poll_pairs<F2MAX>(F2, tag, a.ctl, a.wait_ns, [&](int j) { return xpair(src, par, j, sly, slx); },
                                   vals);
            if (!ok) continue;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                ph[r][c] = vals[c];
                ux[r][c] = vals[K + c];
                uy[r][c] = vals[2 * K + c];
            }
#pragma unroll
            for (int e2 = 0; e2 < LKv; ++e2) w[r][e2] = (e2 < l) ? vals[3 * K + e2] : 0.0f;
            sts<K>(sphi + sb[r], ph[r]);
        }
        return ok;
    };

    // initial iterate: own phi to shared memory, then the first exchange
#pragma unroll
    for (int r = 0; r < P; ++r)
        if (ptile[r]) sts<K>(sphi + sb[r], ph[r]);
    if (!exchange(0, false)) dec[0] = 1;
    __syncthreads();
    bool aborted = dec[0] != 0;
    int nexch = 1, checks = 0, t = 0;
    bool stop = false;

    // reciprocals of the check's weights, once per solve (FP64 division is slow here)
    const double inv_mu = 1.0 / a.cfg.mu, inv_nu = a.cfg.has_w ? 1.0 / a.cfg.nu : 0.0;
    const double inv_tau = 1.0 / a.cfg.tau, inv4eps = a.cfg.eps > 0.0 ? 0.25 / a.cfg.eps : 0.0;
    const bool use_tol = a.cfg.tol_gap > 0.0;
    const double tol_g = a.cfg.tol_gap, tol_r2 = a.cfg.tol_res * a.cfg.tol_res;

    float racc[P][K];
#pragma unroll
    for (int r = 0; r < P; ++r)
#pragma unroll
        for (int c = 0; c < K; ++c) racc[r][c] = 0.0f;

    // ---- one PDHG step on the points q < nRp (phase 1: u, and ubar for the
    // divergence) and q < nR (w, the commit, phase 2: phi).  LAST: the step
    // before a check (its region is the tile), which also sums the terms of the
    // fixed-point residual R of Section 6.1: ||du||^2, ||dw||^2, ||dphi||^2 and
    // <dphi, div du + div_G dw>, where du on the points left of and below the tile
    // comes from the same phase-1 arithmetic their own tile does.
    float fdu = 0.0f, fdw = 0.0f, fdp = 0.0f, fdx = 0.0f;
    // pub_e >= 0: the last step before halo exchange pub_e.  With six and more
    // channels (EARLY) each band point publishes as soon as its phi is final, so
    // that its many stores drain while the rest of the tile finishes the step
    // (measured: 3 x 3 matrices at 128^2 gain 2-3%; at three channels the extra
    // code in the step costs more than the overlap gains)
    constexpr bool EARLY = K >= 6;
    auto step = [&](auto last_tag, int nR, int nRp, int pub_e) {
        constexpr bool LAST = decltype(last_tag)::value;
#pragma unroll
        for (int r = 0; r < P; ++r) {
            const int q = tid + r * nthr;
            if (q >= nRp) continue;
            const int b = sb[r], f = nbf[r];
            float fx[K], fy[K];
            lds<K>(sphi + b + ((f & 1) ? KV : 0), fx);
            lds<K>(sphi + b + ((f & 2) ? RS : 0), fy);
            float vx[K], vy[K];
#pragma unroll
            for (int c = 0; c < K; ++c) {
                vx[c] = ux[r][c] + muih * (fx[c] - ph[r][c]);
                vy[c] = uy[r][c] + muih * (fy[c] - ph[r][c]);
            }
            float tu = mu;
            if (a.s.reg) {          // regularised prox: shrink v / (1 + 2 mu eps) by mu / (1 + 2 mu eps)
                tu = mu * a.s.su;
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    vx[c] *= a.s.su;
                    vy[c] *= a.s.su;
                }
            }
            shrink_u<K>(vx, vy, tu, un, a.g.wc, NM ? 0u : a.g.upair);
            float ubx[K], uby[K];
#pragma unroll
            for (int c = 0; c < K; ++c) {
                ubx[c] = 2.0f * vx[c] - ux[r][c];
                uby[c] = 2.0f * vy[c] - uy[r][c];
            }
            sts<K>(sux + b, ubx);
            sts<K>(suy + b, uby);
            if constexpr (LAST) {
                float dux[K], duy[K];
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    dux[c] = vx[c] - ux[r][c];
                    duy[c] = vy[c] - uy[r][c];
                    if (q < nR) fdu += a.g.wc[c] * (dux[c] * dux[c] + duy[c] * duy[c]);
                }
                sts<K>(sdx + b, dux);
                sts<K>(sdy + b, duy);
            }
            if (q >= nR) continue;
            float wx[LKv];
#pragma unroll
            for (int e = 0; e < LKv; ++e) {
                float ge = 0.0f;
#pragma unroll
                for (int c = 0; c < K; ++c) ge += a.g.G[e][c] * ph[r][c];
                wx[e] = (e < l) ? w[r][e] + nu * ge : 0.0f;
            }
            float tw = alpha * nu;
            if (a.s.reg) {
                tw *= a.s.sw;
#pragma unroll
                for (int e = 0; e < LKv; ++e) wx[e] *= a.s.sw;
            }
            shrink_w<LKv>(wx, l, tw, wn, a.g.we, a.g.wpair);
#pragma unroll
            for (int c = 0; c < K; ++c) {
                float gw = 0.0f;
#pragma unroll
                for (int e = 0; e < LKv; ++e) gw -= a.g.Dv[c][e] * (2.0f * wx[e] - w[r][e]);
                racc[r][c] = gw + bb[r][c];
            }
            if constexpr (LAST) {
                float dg[K];
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    float gd = 0.0f;
#pragma unroll
                    for (int e = 0; e < LKv; ++e) gd -= a.g.Dv[c][e] * (wx[e] - w[r][e]);
                    dg[c] = gd;
                }
                sts<K>(sdg + b, dg);
#pragma unroll
                for (int e = 0; e < LKv; ++e) {
                    const float dw = wx[e] - w[r][e];
                    fdw += a.g.we[e] * dw * dw;
                }
            }
#pragma unroll
            for (int c = 0; c < K; ++c) {
                ux[r][c] = vx[c];
                uy[r][c] = vy[c];
            }
#pragma unroll
            for (int e = 0; e < LKv; ++e) w[r][e] = wx[e];
        }
        __syncthreads();
        // phase 2: phi' = phi + tau (div_x ubar + div_G wbar + rho1 - rho0); the
        // backward neighbours outside the grid are masked (ubar = 0 there)
#pragma unroll
        for (int r = 0; r < P; ++r) {
            const int q = tid + r * nthr;
            if (q >= nR) continue;
            const int b = sb[r], f = nbf[r];
            float bxo[K], bxl[K], byo[K], byd[K];
            lds<K>(sux + b, bxo);
            lds<K>(sux + b - ((f & 4) ? KV : 0), bxl);
            lds<K>(suy + b, byo);
            lds<K>(suy + b - ((f & 8) ? RS : 0), byd);
            const float mx = (f & 4) ? 1.0f : 0.0f, my = (f & 8) ? 1.0f : 0.0f;
            float dph[K];
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const float d = ih * ((bxo[c] - mx * bxl[c]) + (byo[c] - my * byd[c])) + racc[r][c];
                const float np = ph[r][c] + tau * d;
                dph[c] = np - ph[r][c];
                ph[r][c] = np;
            }
            sts<K>(sphi + b, ph[r]);
            if (EARLY && pub_e >= 0 && pband[r]) publish_point(r, pub_e);
            if constexpr (LAST) {
                float dxo[K], dxl[K], dyo[K], dyd[K], dg[K];
                lds<K>(sdx + b, dxo);
                lds<K>(sdx + b - ((f & 4) ? KV : 0), dxl);
                lds<K>(sdy + b, dyo);
                lds<K>(sdy + b - ((f & 8) ? RS : 0), dyd);
                lds<K>(sdg + b, dg);
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    const float ddiv = ih * ((dxo[c] - mx * dxl[c]) + (dyo[c] - my * dyd[c])) + dg[c];
                    fdp += a.g.wc[c] * dph[c] * dph[c];
                    fdx += a.g.wc[c] * dph[c] * ddiv;
                }
            }
        }
        __syncthreads();
    };

    // ---- the tile's iterate to the caller's arrays: at the end, and at every check
    // whose stop decision is deferred (the arrays then hold that check's iterate)
    auto write_out = [&]() {
#pragma unroll
        for (int r = 0; r < P; ++r) {
            if (!ptile[r]) continue;
            const int x = pxy[r] & 0xffff, y = pxy[r] >> 16;
            const size_t p = (size_t)y * n + x;
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
    };

    // ---- stop decision of check number idx (the iterate after iteration tc): every
    // block gathers every block's row (one L2 round trip), sums the rows in a fixed
    // order and decides; block 0 records the metric row.  dec[2] = 1 stops.  Returns
    // false if a wait ran out (the solve is then aborted).
    auto decide = [&](int idx, int tc) -> bool {
        const int cpar = idx & 1;
        const uint32_t ctag = tag_hi + (uint32_t)idx + 1u;
        const int words = NT * NRED * 2;
        const int lane = tid & 31, wid = tid >> 5, nw = (nthr + 31) >> 5;
        {
            const int mine = tid < words ? (words - tid + nthr - 1) / nthr : 0;
            const bool ok = poll_words<8>(
                mine, ctag, a.ctl, a.wait_ns,
                [&](int j) { return a.rows + (size_t)cpar * words + (size_t)tid + (size_t)j * nthr; },
                [&](int j, uint32_t bits) {
                    const int widx = tid + j * nthr;
                    ((uint32_t *)rtab)[(widx >> 1) * 2 + ((widx & 1) ? 0 : 1)] = bits;
                });
            if (!ok) dec[0] = 1;
        }
        __syncthreads();
        if (dec[0]) return false;
        // fixed-order sum: lane j takes rows j, j + 32, ..., then a butterfly over the
        // lanes (every lane ends with the same sum, in every block)
        for (int q = wid; q < NRED; q += nw) {
            double acc = 0.0;
            for (int b = lane; b < NT; b += 32) {
                const double x_ = rtab[b * NRED + q];
                acc = (q == RED_MAX) ? fmax(acc, x_) : acc + x_;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double o = __shfl_xor_sync(0xffffffffu, acc, off);
                acc = (q == RED_MAX) ? fmax(acc, o) : acc + o;
            }
            if (lane == 0) S[q] = acc;
        }
        __syncthreads();
        if (tid == 0) {
            // the stop decision with products and comparisons only: rel_gap <= tol_gap is
            // |P - D| <= tol_gap max(|P|, 1e-300), rel_res <= tol_res is
            // ||r||^2 <= tol_res^2 ||rho0 - rho1||^2; the ratios themselves are formed on
            // the host from the row (finish_raw_row)
            double m[NMET];
            m[0] = S[RED_P];
            m[1] = fma(-S[RED_DIST], inv4eps, S[RED_D]);
            m[2] = S[RED_RR];
            m[3] = S[RED_BB];
            m[4] = fma(S[RED_DU], inv_mu, fma(S[RED_DW], inv_nu, fma(S[RED_DP], inv_tau, -2.0 * S[RED_X])));
            m[5] = S[RED_MAX];
            m[6] = (double)tc;
            // finiteness, magnitudes and comparisons of non-negative values on the
            // bit patterns (integer instructions; IEEE order of non-negative doubles is
            // the order of their bits)
            bool finite = true;
#pragma unroll
            for (int q = 0; q < 6; ++q) finite = finite && (((uint32_t)__double2hiint(m[q]) & 0x7ff00000u) != 0x7ff00000u);
            const auto mag = [](double x) { return (long long)((unsigned long long)__double_as_longlong(x) << 1 >> 1); };
            const long long p_mag = mag(m[0]), tiny = mag(1e-300);
            const double scale = __longlong_as_double(p_mag > tiny ? p_mag : tiny);
            const double bb = mag(m[3]) > 0 ? m[3] : 1.0;
            const bool conv = use_tol && mag(m[0] - m[1]) <= mag(tol_g * scale) && mag(m[2]) <= mag(tol_r2 * bb);
            m[7] = conv ? 1.0 : 0.0;
            if (tile == 0) {
                for (int q = 0; q < NMET; ++q) a.st->met[q] = m[q];
                if (a.hist && idx < a.hist_cap)
                    for (int q = 0; q < NMET; ++q) a.hist[(size_t)idx * NMET + q] = m[q];
                a.st->raw = 1;
                a.st->checks = idx + 1;
                a.st->iter = tc;
                if (!finite) a.st->error = VOMT_ERR_NONFINITE;
                if (conv || !finite) a.st->stop = 1;
            }
            dec[2] = (conv || !finite || tc >= T) ? 1 : 0;
        }
        __syncthreads();
        return true;
    };

    // A check before the last iteration publishes its row and saves the iterate to
    // the caller's arrays, and the iteration runs on; the rows are gathered and the
    // stop decision taken after the next halo exchange, when every block's row has
    // long arrived, so that no block waits for the slowest one.  If that decision
    // stops, the solve ends with the saved iterate (the extra iterations are
    // discarded).  Rows alternate between two slots: a block publishes the row of
    // check c + 1 only after its decision of check c, which needed every row of c,
    // so no slot is overwritten before every block has read it.
    int pend = -1, pend_t = 0;
    bool saved = false;

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
        fdu = fdw = fdp = fdx = 0.0f;
        for (int s = 1; s <= hb; ++s) {
            const int rr = min(hb - s, R);      // ring width of the region this step updates
            const int nR = cntR[rr], nRp = cntRp[rr];
            const int pub_e = s == hb ? nexch : -1;
            if (s == hb && check_after)
                step(std::integral_constant<bool, true>(), nR, nRp, pub_e);
            else
                step(std::integral_constant<bool, false>(), nR, nRp, pub_e);
        }
        t = t_end;
        // ---- refresh the ring
        if (hb > 0) {
            if (!exchange(nexch, EARLY)) dec[0] = 1;
            ++nexch;
            __syncthreads();
            if (dec[0]) { aborted = true; break; }
        }
        if (pend >= 0) {
            if (!decide(pend, pend_t)) { aborted = true; break; }
            pend = -1;
            if (dec[2]) { saved = true; break; }
        }
        if (!check_after) continue;

        // ---- convergence check of the iterate after iteration t
#pragma unroll
        for (int r = 0; r < P; ++r)
            if (pv[r]) {
                sts<K>(sux + sb[r], ux[r]);
                sts<K>(suy + sb[r], uy[r]);
            }
        __syncthreads();
        // Per-point terms in FP32, summed over this thread's few points in FP32
        // and then over the grid in FP64 (FP64 arithmetic is scarce on this GPU).
        float fs[NRED];
#pragma unroll
        for (int q = 0; q < NRED; ++q) fs[q] = 0.0f;
        fs[RED_DU] = fdu;
        fs[RED_DW] = fdw;
        fs[RED_DP] = fdp;
        fs[RED_X] = fdx;
#pragma unroll
        for (int r = 0; r < P; ++r) {
            if (!ptile[r]) continue;
            const int b = sb[r], f = nbf[r];
            const int oxm = (f & 4) ? KV : 0, oym = (f & 8) ? RS : 0;
            const float mx = (f & 4) ? 1.0f : 0.0f, my = (f & 8) ? 1.0f : 0.0f;
            float uxl[K], uyd[K], fx[K], fy[K];
            lds<K>(sux + b - oxm, uxl);
            lds<K>(suy + b - oym, uyd);
            lds<K>(sphi + b + ((f & 1) ? KV : 0), fx);
            lds<K>(sphi + b + ((f & 2) ? RS : 0), fy);
            float nu_pt = 0.0f, dn_u = 0.0f, q2 = 0.0f, dist = 0.0f;
            float pux = 0.0f, puy = 0.0f, pgx = 0.0f, pgy = 0.0f;   // real parts of a complex pair
            float gxs[K], gys[K];
#pragma unroll
            for (int c = 0; c < K; ++c) {
                const float uxc = ux[r][c], uyc = uy[r][c], phc = ph[r][c], bc = bb[r][c], wgt = a.g.wc[c];
                q2 += wgt * (uxc * uxc + uyc * uyc);
                float gwb = bc;
#pragma unroll
                for (int e = 0; e < LKv; ++e) gwb -= a.g.Dv[c][e] * w[r][e];
                const float rc = residual_c(ih, uxc, mx * uxl[c], uyc, my * uyd[c], gwb);
                fs[RED_RR] += wgt * rc * rc;
                fs[RED_BB] += wgt * bc * bc;
                fs[RED_D] += wgt * phc * bc;
                const float gxx = ih * (fx[c] - phc), gyy = ih * (fy[c] - phc);
                gxs[c] = gxx;
                gys[c] = gyy;
                if (un == VOMT_U_NUC) {
                    // after the loop
                } else if (!NM && un == U_CL1) {
                    // complex entrywise: a pair's modulus (its weight 2 counts the mirror entry)
                    if (pair_first(a.g.upair, c)) {
                        pux = uxc; puy = uyc; pgx = gxx; pgy = gyy;
                    } else if (pair_second(a.g.upair, c)) {
                        nu_pt += wgt * (sqrtf(pux * pux + uxc * uxc) + sqrtf(puy * puy + uyc * uyc));
                        dn_u = fmaxf(dn_u, fmaxf(sqrtf(pgx * pgx + gxx * gxx), sqrtf(pgy * pgy + gyy * gyy)));
                    } else {
                        nu_pt += wgt * (fabsf(uxc) + fabsf(uyc));
                        dn_u = fmaxf(dn_u, fmaxf(fabsf(gxx), fabsf(gyy)));
                    }
                } else if (un == VOMT_U_L12) {
                    nu_pt += sqrtf(uxc * uxc + uyc * uyc);
                    const float gn = sqrtf(gxx * gxx + gyy * gyy);
                    dn_u = fmaxf(dn_u, gn);
                    const float o = fmaxf(gn - 1.0f, 0.0f);
                    dist += o * o;
                } else if (un == VOMT_U_L2) {
                    nu_pt += wgt * (uxc * uxc + uyc * uyc);
                    dn_u += wgt * (gxx * gxx + gyy * gyy);
                } else {
                    nu_pt += wgt * (fabsf(uxc) + fabsf(uyc));
                    dn_u = fmaxf(dn_u, fmaxf(fabsf(gxx), fabsf(gyy)));
                    const float ox = fmaxf(fabsf(gxx) - 1.0f, 0.0f), oy = fmaxf(fabsf(gyy) - 1.0f, 0.0f);
                    dist += wgt * (ox * ox + oy * oy);
                }
            }
            if (un == VOMT_U_L2) {
                nu_pt = sqrtf(nu_pt);
                dn_u = sqrtf(dn_u);
                const float o = fmaxf(dn_u - 1.0f, 0.0f);
                dist += o * o;
            }
            if (un == VOMT_U_NUC) {          // sum of the nuclear norms, larger spectral norm
                float n1, s1, n2, s2;
                mat::sym_nuc_spec<K>(ux[r], n1, s1);
                mat::sym_nuc_spec<K>(uy[r], n2, s2);
                nu_pt = n1 + n2;
                mat::sym_nuc_spec<K>(gxs, n1, s1);
                mat::sym_nuc_spec<K>(gys, n2, s2);
                dn_u = fmaxf(s1, s2);
            }
            float nw_pt = 0.0f, dn_w = 0.0f, wg2 = 0.0f, gg2 = 0.0f, pw_re = 0.0f, pg_re = 0.0f;
#pragma unroll
            for (int e = 0; e < LKv; ++e) {
                if (e < l) {
                    float ge = 0.0f;
#pragma unroll
                    for (int c = 0; c < K; ++c) ge += a.g.G[e][c] * ph[r][c];
                    const float we = w[r][e], wgt = a.g.we[e];
                    q2 += wgt * we * we;
                    if (wn == VOMT_W_L1) {
                        nw_pt += wgt * fabsf(we);
                        dn_w = fmaxf(dn_w, fabsf(ge));
                        const float o = fmaxf(fabsf(ge) - alpha, 0.0f);
                        dist += wgt * o * o;
                    } else if (!NM && wn == W_CL1) {
                        if (wpair_first(a.g.wpair, e)) {
                            pw_re = we;
                            pg_re = ge;
                        } else if (wpair_second(a.g.wpair, e)) {
                            nw_pt += wgt * sqrtf(pw_re * pw_re + we * we);
                            dn_w = fmaxf(dn_w, sqrtf(pg_re * pg_re + ge * ge));
                        } else {
                            nw_pt += wgt * fabsf(we);
                            dn_w = fmaxf(dn_w, fabsf(ge));
                        }
                    } else if (wn == VOMT_W_NUC) {
                        // 3 x 3 skew components (a, b, c): ||W_s||_nuc = 2 |(a,b,c)|, spectral |(a,b,c)|
                        wg2 += we * we;
                        gg2 += ge * ge;
                        if (e % 3 == 2) {
                            nw_pt += 2.0f * sqrtf(wg2);
                            dn_w = fmaxf(dn_w, sqrtf(gg2));
                            wg2 = gg2 = 0.0f;
                        }
                    } else {
                        nw_pt += wgt * we * we;
                        dn_w += wgt * ge * ge;
                    }
                }
            }
            if (wn == VOMT_W_L2) {
                nw_pt = sqrtf(nw_pt);
                dn_w = sqrtf(dn_w);
                const float o = fmaxf(dn_w - alpha, 0.0f);
                if (l > 0) dist += o * o;
            }
            fs[RED_P] += nu_pt + alpha * nw_pt;
            if (a.s.reg) {
                fs[RED_P] += a.s.eps * q2;
                fs[RED_DIST] += dist;
            }
            float di = fmaxf(dn_u - 1.0f, 0.0f);
            if (l > 0) di = fmaxf(di, dn_w - alpha);
            fs[RED_MAX] = fmaxf(fs[RED_MAX], di);
        }
        // warp sums in FP32 with the rounding error carried (TwoSum at every level,
        // fixed order), then the warps' (hi, lo) pairs summed in FP64 by one thread
        // per slot: the FP64 pipe sees a few dozen instructions per check
        const int lane = tid & 31, wid = tid >> 5, nw = (nthr + 31) >> 5;
        float lo[NRED];
#pragma unroll
        for (int q = 0; q < NRED; ++q) lo[q] = 0.0f;
#pragma unroll
        for (int q = 0; q < NRED; ++q) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float oh = __shfl_down_sync(0xffffffffu, fs[q], off);
                const float ol = __shfl_down_sync(0xffffffffu, lo[q], off);
                if (q == RED_MAX) {
                    fs[q] = fmaxf(fs[q], oh);
                } else {
                    float e;
                    fs[q] = two_sum(fs[q], oh, e);
                    lo[q] = lo[q] + (ol + e);
                }
            }
        }
        float *redf = reinterpret_cast<float *>(red);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < NRED; ++q) {
                redf[(wid * NRED + q) * 2] = fs[q];
                redf[(wid * NRED + q) * 2 + 1] = lo[q];
            }
        __syncthreads();
        const int cpar = checks & 1;
        const uint32_t ctag = tag_hi + (uint32_t)checks + 1u;
        const int words = NT * NRED * 2;
        // the block's row: warp q sums slot q over the warps' (hi, lo) pairs, lane j
        // taking warp j, then a butterfly over the lanes.  An FP64 instruction costs a
        // whole warp's issue on this GPU whatever its active lanes, so the few FP64
        // instructions are spread over the warps (the maximum stays in FP32: exact)
        for (int q = wid; q < NRED; q += nw) {
            double acc = 0.0;
            if (q == RED_MAX) {
                float mx = 0.0f;
                for (int j = lane; j < nw; j += 32) mx = fmaxf(mx, redf[(j * NRED + q) * 2]);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
                acc = (double)mx;
            } else {
                for (int j = lane; j < nw; j += 32)
                    acc += (double)redf[(j * NRED + q) * 2] + (double)redf[(j * NRED + q) * 2 + 1];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    if (off < nw) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            }
            if (lane == 0) {
                unsigned long long *dst = a.rows + (size_t)cpar * words + ((size_t)tile * NRED + q) * 2;
                st_tagged(dst, __int_as_float(__double2hiint(acc)), ctag);
                st_tagged(dst + 1, __int_as_float(__double2loint(acc)), ctag);
            }
        }
        if (R > 0 && t < T) {      // a halo exchange comes before the decision
            write_out();
            pend = checks++;
            pend_t = t;
            continue;
        }
        if (!decide(checks, t)) { aborted = true; break; }
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
    // ---- final iterate of the tile to the caller's arrays (unless a deferred
    // decision stopped the solve: its check's iterate is there already)
    if (!saved) write_out();
}

// One problem: the grid is its tiles.  Its tags carry the prefix a.tag_hi (0 for
// a lone solve; the grouped batch gives each problem its own).
// LB: the launch bound (most threads of a block).  A block of 384 threads (12
// warps, three per SM sub-partition) lets a thread hold 170 registers, 512 only
// 128 (four warps on some sub-partition): two points per thread need about 170
// to be processed side by side, so extended tiles of at most 768 points take the
// 384-thread form.
template <int K, int P, int NM, int LB = res_threads(K), int LF = 0>
__global__ void __launch_bounds__(LB, 1) k_resident(const __grid_constant__ ResArgs a)
{
    resident_body<K, P, NM, LF>(a, (int)blockIdx.x, (int)gridDim.x, a.tag_hi);
}

// Many problems of one shape (grouped batch): the grid is `groups` groups of T
// blocks; group g solves the problems of its job list one after the other, each
// on its T tiles.  A job's arguments (problem, exchange region, status) are
// copied to shared memory before the group starts it.  Consecutive jobs of a
// group use alternate exchange regions and distinct tag prefixes, so no block
// can mistake a word of the previous problem for one of the current problem.
struct MultiArgs {
    const ResArgs *jobs;       // [groups][per] arguments of each job
    const int *valid;          // [groups][per] 1 where the job exists
    int per, T;
    ResCtl *ctl;
};

template <int K, int P, int NM, int LB = res_threads(K)>
__global__ void __launch_bounds__(LB, 1) k_resident_multi(const __grid_constant__ MultiArgs m)
{
    __shared__ __align__(16) ResArgs sa;
    const int g = (int)blockIdx.x / m.T, t = (int)blockIdx.x % m.T;
    for (int j = 0; j < m.per; ++j) {
        if (!m.valid[g * m.per + j]) break;
        const int *src = reinterpret_cast<const int *>(&m.jobs[(size_t)g * m.per + j]);
        for (int q = threadIdx.x; q < (int)(sizeof(ResArgs) / sizeof(int)); q += blockDim.x)
            reinterpret_cast<int *>(&sa)[q] = src[q];
        __syncthreads();
        resident_body<K, P, NM>(sa, t, m.T, sa.tag_hi);
        __syncthreads();
        if (ld_relaxed32(&m.ctl->abort)) break;
    }
}

using ResKernel = void (*)(ResArgs);
using MultiKernel = void (*)(MultiArgs);

// Kernel for K channels, P points per thread, the norm mode NM, the launch bound
// LB and the fixed flux count LF (one per instantiation unit; the host picks
// through res_kernel).  LB = 384 with two points per thread exists for up to four
// channels; LF = 9 for 3 x 3 matrices with the matrix or the nuclear norms and one
// or two points per thread; every other request takes LB = res_threads(K), LF = 0.
template <int K>
ResKernel kernel_for(int P, int NM, int LB, int LF)
{
    if constexpr (K <= 4) {
        if (P == 2 && LB == 384) {
            if constexpr (K == 3) {
                if (NM == 2) return k_resident<K, 2, 2, 384>;
            }
            return NM == 1 ? k_resident<K, 2, 1, 384> : k_resident<K, 2, 0, 384>;
        }
    }
    if constexpr (K == 6) {
        if (LF == 9 && P <= 2) {
            if (NM == 2) return P == 1 ? k_resident<K, 1, 2, 384, 9> : k_resident<K, 2, 2, 384, 9>;
            if (NM == 3) return P == 1 ? k_resident<K, 1, 3, 384, 9> : k_resident<K, 2, 3, 384, 9>;
        }
    }
    (void)LB;
    (void)LF;
    if constexpr (K == 3 || K == 6) {     // compact 2 x 2 and 3 x 3 matrices
        if (NM == 2) return P == 1 ? k_resident<K, 1, 2> : (P == 2 ? k_resident<K, 2, 2> : k_resident<K, 4, 2>);
    }
    if constexpr (K == 6) {               // 3 x 3 matrices, both nuclear norms
        if (NM == 3) return P == 1 ? k_resident<K, 1, 3> : (P == 2 ? k_resident<K, 2, 3> : k_resident<K, 4, 3>);
    }
    if (NM == 1) return P == 1 ? k_resident<K, 1, 1> : (P == 2 ? k_resident<K, 2, 1> : k_resident<K, 4, 1>);
    return P == 1 ? k_resident<K, 1, 0> : (P == 2 ? k_resident<K, 2, 0> : k_resident<K, 4, 0>);
}

// Grouped-batch kernel for K <= 5 channels, P in {2, 4} (and P = 1 for five
// channels, whose per-point state spills at two points per thread), NM in {0, 1},
// and the 384-thread form of P = 2 (LB = 384) for up to four channels; nullptr
// otherwise.
template <int K>
MultiKernel multi_kernel_for(int P, int NM, int LB)
{
    if constexpr (K <= 5) {
        if constexpr (K <= 4) {
            if (P == 2 && LB == 384) return NM == 1 ? k_resident_multi<K, 2, 1, 384> : k_resident_multi<K, 2, 0, 384>;
        }
        if constexpr (K == 5) {
            if (P == 1) return NM == 1 ? k_resident_multi<K, 1, 1> : k_resident_multi<K, 1, 0>;
        }
        if (NM == 1) return P == 2 ? k_resident_multi<K, 2, 1> : k_resident_multi<K, 4, 1>;
        return P == 2 ? k_resident_multi<K, 2, 0> : k_resident_multi<K, 4, 0>;
    } else {
        (void)P;
        (void)NM;
        (void)LB;
        return nullptr;
    }
}

ResKernel res_kernel(int K, int P, int NM, int LB, int LF);
MultiKernel res_multi_kernel(int K, int P, int NM, int LB);

// Shared memory of the grouped kernel beyond the dynamic layout (the job copy).
constexpr int MULTI_STATIC_SMEM = (int)((sizeof(ResArgs) + 127) / 128 * 128);

}  // namespace res
}  // namespace vomt
