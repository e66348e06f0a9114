// Pieces shared by the two forms of the 3-D fused iteration (vector3d.cu,
// vector3d_tma.cu): the state views, the per-point shrinks and the tile shape.
// The shrinks cover vector OMT and, through the compact storage of symmetric /
// skew matrices, matrix OMT (K = k(k+1)/2 channels, off-diagonals weighted 2).
//
// A 3-D state is five runs of volumes, each n x n x n with x fastest:
// phi [k], u_x [k], u_y [k], u_z [k], w [l].  u_d's ghost face is the last index
// in direction d (kept zero).
#pragma once

#include "internal.h"
#include "pdhg_device.cuh"

namespace vomt {
namespace v3 {

using dev::shrink2_factor;
using dev::soft;
using dev::CheckAcc;
using dev::block_sum_store;

// a block owns an MX x MY column of the grid and marches through a chunk of z
constexpr int MX = 32, MY = 8, MT = MX * MY;

struct S3In {
    const float *phi, *ux, *uy, *uz, *w;
};
struct S3Out {
    float *phi, *ux, *uy, *uz, *w;
};

template <int K>
struct LK3 {
    static constexpr int v = K * (K - 1) / 2 > 0 ? K * (K - 1) / 2 : 1;
};

template <int K, int UN>
__device__ __forceinline__ void shrink_u3(float (&a)[K], float (&b)[K], float (&c)[K], float t, const float *wc)
{
    if (UN == VOMT_U_L12) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const float f = shrink2_factor(a[q] * a[q] + b[q] * b[q] + c[q] * c[q], t);
            a[q] *= f;
            b[q] *= f;
            c[q] *= f;
        }
    } else if (UN == VOMT_U_L2) {
        float s2 = 0.0f;
#pragma unroll
        for (int q = 0; q < K; ++q) s2 += wc[q] * (a[q] * a[q] + b[q] * b[q] + c[q] * c[q]);
        const float f = shrink2_factor(s2, t);
#pragma unroll
        for (int q = 0; q < K; ++q) { a[q] *= f; b[q] *= f; c[q] *= f; }
    } else if (UN == VOMT_U_NUC) {
        // matrix OMT, ||U||_{1,nuc} = sum_d ||U_d||_nuc: each direction's compact symmetric
        // matrix has its eigenvalues soft-thresholded (K = 3 or 6)
        mat::sym_shrink_nuc<K>(a, t);
        mat::sym_shrink_nuc<K>(b, t);
        mat::sym_shrink_nuc<K>(c, t);
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) { a[q] = soft(a[q], t); b[q] = soft(b[q], t); c[q] = soft(c[q], t); }
    }
}

template <int LK, int WN>
__device__ __forceinline__ void shrink_w3(float (&x)[LK], int l, float t, const float *we)
{
    if (WN == VOMT_W_L1) {
#pragma unroll
        for (int e = 0; e < LK; ++e)
            if (e < l) x[e] = soft(x[e], t);
    } else if (WN == VOMT_W_NUC) {
        // matrix OMT with 3 x 3 skew components (a, b, c): the prox of t ||W_s||_nuc is the
        // Euclidean group shrink of (a, b, c) by t
        if constexpr (LK % 3 == 0) {
#pragma unroll
            for (int g0 = 0; g0 < LK; g0 += 3) {
                if (g0 < l) {
                    const float f = shrink2_factor(x[g0] * x[g0] + x[g0 + 1] * x[g0 + 1] + x[g0 + 2] * x[g0 + 2], t);
                    x[g0] *= f;
                    x[g0 + 1] *= f;
                    x[g0 + 2] *= f;
                }
            }
        }
    } else {
        float s2 = 0.0f;
#pragma unroll
        for (int e = 0; e < LK; ++e)
            if (e < l) s2 += we[e] * x[e] * x[e];
        const float f = shrink2_factor(s2, t);
#pragma unroll
        for (int e = 0; e < LK; ++e) x[e] *= f;
    }
}

// u + mu grad phi along one direction (zero across a ghost face)
__device__ __forceinline__ float upre(float u0, float ahead, float here, bool inside, float mi)
{
    return inside ? u0 + mi * (ahead - here) : u0;
}

}  // namespace v3
}  // namespace vomt
