// Nuclear-norm pieces of matrix OMT on compact storage (Section 6.2 norms
// ||U||_{1,nuc} = ||U_x||_nuc + ||U_y||_nuc and ||W||_{1,nuc} = sum_s ||W_s||_nuc;
// the nuclear shrink of Appendix B: singular values soft-thresholded).
//
// Compact layouts (host_setup.cpp): a symmetric k x k matrix is K = k(k+1)/2
// floats, the diagonal first, then the entries above it row by row
// (k = 2: a00 a11 a01; k = 3: a00 a11 a22 a01 a02 a12); a skew matrix is its
// k(k-1)/2 entries above the diagonal.  K = 3 means k = 2 and K = 6 means
// k = 3 (the nuclear norms exist for matrix problems only).
//
// Symmetric: the singular values are |eigenvalues|, so the shrink keeps the
// eigenvectors and maps each eigenvalue l to sign(l) max(|l| - t, 0).  The
// eigen-decomposition is cyclic Jacobi (Golub and Van Loan, Section 8.5) in
// FP32: one rotation is exact for 2 x 2.  For 3 x 3 the rotations act on the
// six distinct entries only (a rotation in the (p, q) plane sets a_pq to 0,
// moves a_pp and a_qq by -+ tan(theta) a_pq and turns the pair (a_rp, a_rq) of
// the third index r), and four sweeps reach FP32 accuracy: cyclic Jacobi
// converges quadratically, and in FP32 the shrink of random, clustered and
// graded 3 x 3 matrices is within 3e-6 of the exact one after three sweeps and
// at the rounding floor (about 1e-6 relative) after four.
//
// Skew 3 x 3 with entries (a, b, c): the singular values are theta, theta, 0
// with theta = |(a, b, c)|, so ||W_s||_nuc = 2 theta, its dual (the spectral
// norm) is theta, and the shrink scales (a, b, c) by max(0, 1 - t / theta).
// In the compact inner product (off-diagonal weight 2) the prox of
// t ||W_s||_nuc is therefore the Euclidean group shrink of (a, b, c) by t.
// Skew 2 x 2 (one entry a): ||W_s||_nuc = 2 |a|, which is the weighted
// ||.||_1 of the compact storage, so W_NUC coincides with W_L1 there.
#pragma once

#include <math.h>

namespace vomt {
namespace mat {

template <int K>
struct Side {
    static constexpr int v = K == 3 ? 2 : (K == 6 ? 3 : 0);
};

// compact index of entry (a, b) of a symmetric M x M matrix
template <int M>
__host__ __device__ constexpr int sidx(int a, int b)
{
    return a == b ? a : (M == 2 ? 2 : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5)));
}

// In-place cyclic Jacobi on the symmetric M x M matrix A; V collects the
// rotations (columns: eigenvectors), A's diagonal ends as the eigenvalues.
template <int M, bool VEC>
__device__ __forceinline__ void jacobi(float (&A)[M][M], float (&V)[M][M])
{
    if constexpr (VEC) {
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = 0; j < M; ++j) V[i][j] = i == j ? 1.0f : 0.0f;
    }
    constexpr int SWEEPS = M == 2 ? 1 : 6;
#pragma unroll
    for (int sw = 0; sw < SWEEPS; ++sw) {
#pragma unroll
        for (int p = 0; p < M; ++p) {
#pragma unroll
            for (int q = p + 1; q < M; ++q) {
                const float apq = A[p][q];
                if (apq != 0.0f) {
                    const float theta = (A[q][q] - A[p][p]) / (2.0f * apq);
                    const float t = copysignf(1.0f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.0f));
                    const float c = rsqrtf(t * t + 1.0f), s = t * c;
#pragma unroll
                    for (int r = 0; r < M; ++r) {          // A <- A J
                        const float arp = A[r][p], arq = A[r][q];
                        A[r][p] = c * arp - s * arq;
                        A[r][q] = s * arp + c * arq;
                    }
#pragma unroll
                    for (int r = 0; r < M; ++r) {          // A <- J^T A
                        const float apr = A[p][r], aqr = A[q][r];
                        A[p][r] = c * apr - s * aqr;
                        A[q][r] = s * apr + c * aqr;
                    }
                    if constexpr (VEC) {
#pragma unroll
                        for (int r = 0; r < M; ++r) {      // V <- V J
                            const float vrp = V[r][p], vrq = V[r][q];
                            V[r][p] = c * vrp - s * vrq;
                            V[r][q] = s * vrp + c * vrq;
                        }
                    }
                }
            }
        }
    }
}

template <int M, int K>
__device__ __forceinline__ void unpack(const float (&x)[K], float (&A)[M][M])
{
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < M; ++b) A[a][b] = x[sidx<M>(a, b)];
}

// One Jacobi rotation of a symmetric 3 x 3 matrix held as its distinct entries:
// zeroes apq, updates app, aqq and the pair (arp, arq) of the third index r, and
// (VEC) the columns p, q of V.
template <bool VEC>
__device__ __forceinline__ void rot3(float &app, float &aqq, float &apq, float &arp, float &arq, float (&V)[3][3],
                                     int p, int q)
{
    if (apq == 0.0f) return;
    const float theta = (aqq - app) / (2.0f * apq);
    const float t = copysignf(1.0f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.0f)));
    const float c = rsqrtf(fmaf(t, t, 1.0f)), s = t * c;
    app = fmaf(-t, apq, app);
    aqq = fmaf(t, apq, aqq);
    apq = 0.0f;
    const float g = arp, h = arq;
    arp = c * g - s * h;
    arq = s * g + c * h;
    if constexpr (VEC) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float vp = V[r][p], vq = V[r][q];
            V[r][p] = c * vp - s * vq;
            V[r][q] = s * vp + c * vq;
        }
    }
}

// Cyclic Jacobi on the compact symmetric 3 x 3 matrix x = (a00 a11 a22 a01 a02 a12):
// on return d holds the eigenvalues and (VEC) V the eigenvectors as columns.
template <bool VEC>
__device__ __forceinline__ void jacobi3(const float (&x)[6], float (&d)[3], float (&V)[3][3])
{
    float a00 = x[0], a11 = x[1], a22 = x[2], a01 = x[3], a02 = x[4], a12 = x[5];
    if constexpr (VEC) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0f : 0.0f;
    }
#pragma unroll
    for (int sw = 0; sw < 4; ++sw) {
        rot3<VEC>(a00, a11, a01, a02, a12, V, 0, 1);   // (p, q) = (0, 1), r = 2: (a20, a21)
        rot3<VEC>(a00, a22, a02, a01, a12, V, 0, 2);   // (0, 2), r = 1: (a10, a12)
        rot3<VEC>(a11, a22, a12, a01, a02, V, 1, 2);   // (1, 2), r = 0: (a01, a02)
    }
    d[0] = a00;
    d[1] = a11;
    d[2] = a22;
}

// x <- shrink_nuc(x; t) for a compact symmetric matrix (K = 3 or 6)
template <int K>
__device__ __forceinline__ void sym_shrink_nuc(float (&x)[K], float t)
{
    constexpr int M = Side<K>::v;
    if constexpr (M > 0) {
        float d[M], V[M][M];
        if constexpr (M == 3) {
            jacobi3<true>(x, d, V);
        } else {
            float A[M][M];
            unpack<M>(x, A);
            jacobi<M, true>(A, V);
#pragma unroll
            for (int i = 0; i < M; ++i) d[i] = A[i][i];
        }
        float f[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const float l = d[i];
            f[i] = fabsf(l) > t ? l - copysignf(t, l) : 0.0f;
        }
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = a; b < M; ++b) {
                float v = 0.0f;
#pragma unroll
                for (int i = 0; i < M; ++i) v += V[a][i] * f[i] * V[b][i];
                x[sidx<M>(a, b)] = v;
            }
    }
}

// nuclear norm (sum |eigenvalues|) and spectral norm (max |eigenvalue|) of a
// compact symmetric matrix
template <int K>
__device__ __forceinline__ void sym_nuc_spec(const float (&x)[K], float &nuc, float &spec)
{
    constexpr int M = Side<K>::v;
    nuc = spec = 0.0f;
    if constexpr (M > 0) {
        float d[M], V[M][M];
        if constexpr (M == 3) {
            jacobi3<false>(x, d, V);
        } else {
            float A[M][M];
            unpack<M>(x, A);
            jacobi<M, false>(A, V);
#pragma unroll
            for (int i = 0; i < M; ++i) d[i] = A[i][i];
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
            nuc += fabsf(d[i]);
            spec = fmaxf(spec, fabsf(d[i]));
        }
    }
}

}  // namespace mat
}  // namespace vomt
