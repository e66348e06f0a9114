// Device helpers shared by the resident engines: the shrink operators of
// Appendix B with the norm picked at run time (the branch is uniform across a
// launch), tagged 64-bit exchange words and bounded waits.
#pragma once

#include <stdint.h>

#include "internal.h"
#include "matrix_norms.cuh"

namespace vomt {
namespace dev {

// factor of shrink_2 (Appendix B): 1 - t/s for s = sqrt(s2) > t, else 0, as
// max(1 - t / s, 0): the factor is positive exactly when s > t, and at s2 = 0 the
// reciprocal square root is +inf, so 1 - t/s is -inf (or NaN for t = 0, which
// fmaxf also maps to 0)
__device__ __forceinline__ float shrink2_factor(float s2, float t)
{
    return fmaxf(1.0f - t * rsqrtf(s2), 0.0f);
}

// shrink_1 (Appendix B): soft threshold sign(x) max(|x| - t, 0), as x minus x
// clamped to [-t, t] (the same single rounding of x -+ t where |x| > t, exactly 0
// elsewhere)
__device__ __forceinline__ float soft(float x, float t)
{
    return x - fminf(fmaxf(x, -t), t);
}

template <int K>
__device__ __forceinline__ float pick(const float (&a)[K], int idx)
{
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < K; ++c) r = (c == idx) ? a[c] : r;
    return r;
}

// shrink_u on one point (all channels), in place; un = VOMT_U_*; channel weights wc
// enter the joint norm (2 for an off-diagonal matrix entry)
// Is coordinate c the real part of a complex entry (bit c of `pairs`)?  The
// imaginary part is coordinate c + 1.
__device__ __forceinline__ bool pair_first(uint32_t pairs, int c) { return (pairs >> c) & 1u; }
__device__ __forceinline__ bool pair_second(uint32_t pairs, int c) { return c > 0 && ((pairs >> (c - 1)) & 1u); }
__device__ __forceinline__ bool wpair_first(const uint32_t (&wp)[2], int e) { return (wp[e >> 5] >> (e & 31)) & 1u; }
__device__ __forceinline__ bool wpair_second(const uint32_t (&wp)[2], int e)
{
    return e > 0 && ((wp[(e - 1) >> 5] >> ((e - 1) & 31)) & 1u);
}

template <int K>
__device__ __forceinline__ void shrink_u(float (&vx)[K], float (&vy)[K], float t, int un, const float *wc,
                                         uint32_t pairs = 0u)
{
    if (un == VOMT_U_L12) {
#pragma unroll
        for (int c = 0; c < K; ++c) {
            float f = shrink2_factor(vx[c] * vx[c] + vy[c] * vy[c], t);
            vx[c] *= f;
            vy[c] *= f;
        }
    } else if (un == VOMT_U_L2) {
        float s2 = 0.0f;
#pragma unroll
        for (int c = 0; c < K; ++c) s2 += wc[c] * (vx[c] * vx[c] + vy[c] * vy[c]);
        float f = shrink2_factor(s2, t);
#pragma unroll
        for (int c = 0; c < K; ++c) { vx[c] *= f; vy[c] *= f; }
    } else if (un == VOMT_U_NUC) {
        // ||U_x||_nuc + ||U_y||_nuc: each direction's symmetric matrix on its own
        mat::sym_shrink_nuc<K>(vx, t);
        mat::sym_shrink_nuc<K>(vy, t);
    } else if (un == U_CL1) {
        // complex entrywise ||.||_1 (sum of moduli) in each direction: the prox of t |z|
        // scales an (Re, Im) pair by its modulus (in the compact inner product the pair's
        // weight 2 multiplies both the norm and the distance, so the threshold stays t);
        // real coordinates (Hermitian diagonals) take the soft threshold
#pragma unroll
        for (int c = 0; c < K; ++c) {
            if (pair_first(pairs, c) && c + 1 < K) {
                const float fx = shrink2_factor(vx[c] * vx[c] + vx[c + 1] * vx[c + 1], t);
                const float fy = shrink2_factor(vy[c] * vy[c] + vy[c + 1] * vy[c + 1], t);
                vx[c] *= fx;
                vx[c + 1] *= fx;
                vy[c] *= fy;
                vy[c + 1] *= fy;
            } else if (!pair_second(pairs, c)) {
                vx[c] = soft(vx[c], t);
                vy[c] = soft(vy[c], t);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < K; ++c) { vx[c] = soft(vx[c], t); vy[c] = soft(vy[c], t); }
    }
}

// shrink_w on one point, l <= LK flux entries with weights we; wn = VOMT_W_*
template <int LK>
__device__ __forceinline__ void shrink_w(float (&x)[LK], int l, float t, int wn, const float *we,
                                         const uint32_t *wpairs = nullptr)
{
    if (wn == W_CL1) {
        // complex entrywise ||.||_1 of the skew-Hermitian components, as in shrink_u
        const uint32_t wp[2] = {wpairs ? wpairs[0] : 0u, wpairs ? wpairs[1] : 0u};
#pragma unroll
        for (int e = 0; e < LK; ++e) {
            if (e >= l) continue;
            if (wpair_first(wp, e) && e + 1 < LK) {
                const float f = shrink2_factor(x[e] * x[e] + x[e + 1] * x[e + 1], t);
                x[e] *= f;
                x[e + 1] *= f;
            } else if (!wpair_second(wp, e)) {
                x[e] = soft(x[e], t);
            }
        }
    } else if (wn == VOMT_W_L1) {
#pragma unroll
        for (int e = 0; e < LK; ++e)
            if (e < l) x[e] = soft(x[e], t);
    } else if (wn == VOMT_W_NUC) {
        // 3 x 3 skew components, entries (a, b, c) consecutive: Euclidean group shrink
        if constexpr (LK % 3 == 0) {
#pragma unroll
            for (int g = 0; g < LK; g += 3) {
                if (g < l) {
                    const float f = shrink2_factor(x[g] * x[g] + x[g + 1] * x[g + 1] + x[g + 2] * x[g + 2], t);
                    x[g] *= f;
                    x[g + 1] *= f;
                    x[g + 2] *= f;
                }
            }
        }
    } else {
        float s2 = 0.0f;
#pragma unroll
        for (int e = 0; e < LK; ++e)
            if (e < l) s2 += we[e] * x[e] * x[e];
        float f = shrink2_factor(s2, t);
#pragma unroll
        for (int e = 0; e < LK; ++e) x[e] *= f;
    }
}

// ---------------------------------------------------------------- check sums
// Error-free sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = a + b;
    const float bv = s - a;
    e = (a - (s - bv)) + (b - bv);
    return s;
}

// One thread's share of a convergence check: each sum slot is a pair of FP32
// numbers (hi, lo) that TwoSum keeps equal to the exact running sum up to the
// rounding of lo (about twice FP32 precision); the maximum slot is a plain FP32
// maximum (exact).  FP64 arithmetic runs at a small fraction of the FP32 rate on
// this GPU, so FP64 is kept for the sums across warps and blocks.
struct CheckAcc {
    float hi[NRED], lo[NRED];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int q = 0; q < NRED; ++q) hi[q] = lo[q] = 0.0f;
    }
    __device__ __forceinline__ void add(int q, float x)
    {
        float e;
        hi[q] = two_sum(hi[q], x, e);
        lo[q] += e;
    }
    // an FP64 term: its FP32 head through TwoSum, the remainder into lo
    __device__ __forceinline__ void add_d(int q, double x)
    {
        const float h = __double2float_rn(x);
        add(q, h);
        lo[q] += __double2float_rn(x - (double)h);
    }
    __device__ __forceinline__ void max(int q, float x) { hi[q] = fmaxf(hi[q], x); }
};

// The block's FP64 row of a check (NRED slots) from every thread's CheckAcc: warp
// sums of the (hi, lo) pairs in FP32 with TwoSum (fixed order), then the warps'
// pairs summed in FP64 by one thread per slot, in warp order.  NTH threads per
// block, numbered x fastest; every thread must call it.
template <int NTH>
__device__ __forceinline__ void block_sum_store(CheckAcc &a, double *dst)
{
    constexpr int NW = NTH / 32;
    __shared__ float sh[NW][NRED][2];
    const int tid = (int)(threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z));
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int q = 0; q < NRED; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float oh = __shfl_down_sync(0xffffffffu, a.hi[q], off);
            const float ol = __shfl_down_sync(0xffffffffu, a.lo[q], off);
            if (q == RED_MAX) {
                a.hi[q] = fmaxf(a.hi[q], oh);
            } else {
                float e;
                a.hi[q] = two_sum(a.hi[q], oh, e);
                a.lo[q] = a.lo[q] + (ol + e);
            }
        }
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NRED; ++q) {
            sh[wid][q][0] = a.hi[q];
            sh[wid][q][1] = a.lo[q];
        }
    __syncthreads();
    if (tid < NRED) {
        double s = 0.0;
        for (int w = 0; w < NW; ++w)
            s = (tid == RED_MAX) ? fmax(s, (double)sh[w][tid][0]) : s + ((double)sh[w][tid][0] + (double)sh[w][tid][1]);
        dst[tid] = s;
    }
}

// ---------------------------------------------------------------- exchange words
// A 64-bit word carries one FP32 value in its low half and a 32-bit tag (the
// iteration it belongs to, plus one) in its high half.  Aligned 64-bit stores
// and loads are single-copy atomic, so a reader that sees the expected tag also
// sees the value written with it: no separate flag, no fence.
__device__ __forceinline__ void st_tagged(unsigned long long *p, float v, uint32_t tag)
{
    unsigned long long w = ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v);
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p)
{
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

__device__ __forceinline__ uint32_t ld_relaxed32(const uint32_t *p)
{
    uint32_t w;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(w) : "l"(p) : "memory");
    return w;
}

__device__ __forceinline__ uint32_t ld_acquire32(const uint32_t *p)
{
    uint32_t w;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(w) : "l"(p) : "memory");
    return w;
}

__device__ __forceinline__ void st_release32(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ double ld_relaxed_f64(const double *p)
{
    double w;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(w) : "l"(p) : "memory");
    return w;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Control words of a resident launch (device memory, zeroed before the launch).
struct ResCtl {
    uint32_t abort;     // set by the first wait that runs out of time
    uint32_t where;     // which wait gave up (diagnostics)
};

constexpr uint64_t kWaitBudgetNs = 2000000000ull;   // default limit of one wait: 2 s


}  // namespace dev
}  // namespace vomt
