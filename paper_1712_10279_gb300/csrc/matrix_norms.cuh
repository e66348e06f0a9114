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
// eigenvectors and maps each eigenvalue l to sign(l) max(|l| - t, 0).  For
// 2 x 2 the eigen-decomposition is one Jacobi rotation (Golub and Van Loan,
// Section 8.5), which is exact.  For 3 x 3 it is closed form, in three steps:
// (1) the eigenvalue farthest from the other two from the trigonometric
// solution of the characteristic cubic (O. K. Smith, "Eigenvalues of a
// symmetric 3 x 3 matrix", Comm. ACM 4 (1961) 168); it lies at least
// sqrt(3) p from both others, p^2 = ||A - q I||_F^2 / 6, so (2) its
// eigenvector, the longest cross product of two rows of A - l I, is
// well conditioned; (3) the other two eigenpairs are those of the 2 x 2 block
// of A on the plane orthogonal to that vector, by one exact Jacobi rotation.
// The cubic alone would not do: near a double eigenvalue its two close roots
// carry errors of order sqrt(eps) p, and the deflation removes them.  Only v
// depends on the accuracy of l (an error d in l turns v by about d / (sqrt(3) p));
// the eigenvalues are Rayleigh quotients.  In FP32 the shrink of random,
// clustered, graded, near-scalar and exactly degenerate matrices is within
// 6e-7 (relative to ||A||_F) of the exact FP64 shrink, and within 8e-7 with l
// moved by 8e-7 p.
// The dependent chain is about a fifth of that of cyclic Jacobi (twelve
// rotations, each with two divisions and a square root).
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

// In-place Jacobi on the symmetric M x M matrix A (used for M = 2, where one
// rotation is exact); V collects the rotations (columns: eigenvectors), A's
// diagonal ends as the eigenvalues.
template <int M, bool VEC>
__device__ __forceinline__ void jacobi(float (&A)[M][M], float (&V)[M][M])
{
    if constexpr (VEC) {
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = 0; j < M; ++j) V[i][j] = i == j ? 1.0f : 0.0f;
    }
    static_assert(M == 2, "3 x 3 matrices take the closed form eig3");
    constexpr int SWEEPS = 1;
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

// Closed-form eigen-decomposition of the compact symmetric 3 x 3 matrix
// x = (a00 a11 a22 a01 a02 a12): d[0] is the eigenvalue farthest from the
// other two with unit eigenvector v; d[1], d[2] are the eigenvalues of the
// block of A on the plane orthogonal to v, with unit eigenvectors ga, gb
// (written when VEC).
template <bool VEC>
__device__ __forceinline__ void eig3(const float (&x)[6], float (&d)[3], float (&v)[3], float (&ga)[3],
                                     float (&gb)[3])
{
    // work on A / max |a_ij|: the cross products below are squares of entries
    // and their norms fourth powers, which would underflow in FP32 at the scale
    // of the primal steps (entries near 1e-10)
    const float sc = fmaxf(fmaxf(fmaxf(fabsf(x[0]), fabsf(x[1])), fmaxf(fabsf(x[2]), fabsf(x[3]))),
                           fmaxf(fabsf(x[4]), fabsf(x[5])));
    if (sc < 1e-30f) {      // A vanishes to FP32 range: eigenvalues 0, the unit axes as vectors
        d[0] = d[1] = d[2] = 0.0f;
        v[0] = 1.0f, v[1] = 0.0f, v[2] = 0.0f;
        if constexpr (VEC) {
            ga[0] = 0.0f, ga[1] = 1.0f, ga[2] = 0.0f;
            gb[0] = 0.0f, gb[1] = 0.0f, gb[2] = 1.0f;
        }
        return;
    }
    const float isc = __fdividef(1.0f, sc);
    const float a00 = x[0] * isc, a11 = x[1] * isc, a22 = x[2] * isc, a01 = x[3] * isc, a02 = x[4] * isc,
                a12 = x[5] * isc;
    const float q = (a00 + a11 + a22) * (1.0f / 3.0f);
    const float b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    const float off = fmaf(a01, a01, fmaf(a02, a02, a12 * a12));
    const float p2 = fmaf(2.0f, off, fmaf(b00, b00, fmaf(b11, b11, b22 * b22))) * (1.0f / 6.0f);
    // (1) the isolated eigenvalue: with B = (A - q I) / p, the eigenvalues are
    // q + 2 p cos(phi + 2 pi j / 3), phi = acos(det(B) / 2) / 3 in [0, pi / 3];
    // j = 0 (the largest) is isolated for phi <= pi / 6, else j = 1 (the smallest)
    float li = q;
    if (p2 > 0.0f) {
        const float ip = rsqrtf(p2), p = p2 * ip;
        const float c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip,
                    c12 = a12 * ip;
        const float det = c00 * fmaf(c11, c22, -c12 * c12) - c01 * fmaf(c01, c22, -c12 * c02) +
                          c02 * fmaf(c01, c12, -c11 * c02);
        const float r = fminf(fmaxf(0.5f * det, -1.0f), 1.0f);
        const float phi = acosf(r) * (1.0f / 3.0f);
        float sn, cs;
        __sincosf(phi, &sn, &cs);     // phi in [0, pi / 3]: the intrinsic's error moves li by < 1e-6 p
        li = phi <= 0.52359877f ? fmaf(2.0f * p, cs, q) : fmaf(-p, fmaf(1.7320508f, sn, cs), q);
    }
    // (2) its eigenvector: the longest cross product of two rows of A - li I
    const float r00 = a00 - li, r11 = a11 - li, r22 = a22 - li;
    const float w0x = fmaf(a01, a12, -a02 * r11), w0y = fmaf(a02, a01, -r00 * a12), w0z = fmaf(r00, r11, -a01 * a01);
    const float w1x = fmaf(a01, r22, -a02 * a12), w1y = fmaf(a02, a02, -r00 * r22), w1z = fmaf(r00, a12, -a01 * a02);
    const float w2x = fmaf(r11, r22, -a12 * a12), w2y = fmaf(a12, a02, -a01 * r22), w2z = fmaf(a01, a12, -r11 * a02);
    const float n0 = fmaf(w0x, w0x, fmaf(w0y, w0y, w0z * w0z));
    const float n1 = fmaf(w1x, w1x, fmaf(w1y, w1y, w1z * w1z));
    const float n2 = fmaf(w2x, w2x, fmaf(w2y, w2y, w2z * w2z));
    float vx = w0x, vy = w0y, vz = w0z, nn = n0;
    if (n1 > nn) vx = w1x, vy = w1y, vz = w1z, nn = n1;
    if (n2 > nn) vx = w2x, vy = w2y, vz = w2z, nn = n2;
    if (nn > 0.0f) {
        const float in = rsqrtf(nn);
        vx *= in, vy *= in, vz *= in;
    } else {    // A - li I vanishes to rounding: A is scalar, any unit vector will do
        vx = 1.0f, vy = 0.0f, vz = 0.0f;
    }
    // an orthonormal basis (e, g) of the plane orthogonal to v: e = v x (the axis
    // of v's smallest component), normalised; g = v x e
    const float ax = fabsf(vx), ay = fabsf(vy), az = fabsf(vz);
    float ex, ey, ez;
    if (ax <= ay && ax <= az) ex = 0.0f, ey = vz, ez = -vy;
    else if (ay <= az) ex = -vz, ey = 0.0f, ez = vx;
    else ex = vy, ey = -vx, ez = 0.0f;
    const float ie = rsqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
    ex *= ie, ey *= ie, ez *= ie;
    const float gx = fmaf(vy, ez, -vz * ey), gy = fmaf(vz, ex, -vx * ez), gz = fmaf(vx, ey, -vy * ex);
    // (3) the 2 x 2 block [[e.Ae, e.Ag], [e.Ag, g.Ag]] and v.Av
    const float Aex = fmaf(a00, ex, fmaf(a01, ey, a02 * ez)), Aey = fmaf(a01, ex, fmaf(a11, ey, a12 * ez)),
                Aez = fmaf(a02, ex, fmaf(a12, ey, a22 * ez));
    const float Agx = fmaf(a00, gx, fmaf(a01, gy, a02 * gz)), Agy = fmaf(a01, gx, fmaf(a11, gy, a12 * gz)),
                Agz = fmaf(a02, gx, fmaf(a12, gy, a22 * gz));
    const float Avx = fmaf(a00, vx, fmaf(a01, vy, a02 * vz)), Avy = fmaf(a01, vx, fmaf(a11, vy, a12 * vz)),
                Avz = fmaf(a02, vx, fmaf(a12, vy, a22 * vz));
    const float m00 = fmaf(ex, Aex, fmaf(ey, Aey, ez * Aez));
    const float m11 = fmaf(gx, Agx, fmaf(gy, Agy, gz * Agz));
    const float m01 = fmaf(ex, Agx, fmaf(ey, Agy, ez * Agz));
    d[0] = sc * fmaf(vx, Avx, fmaf(vy, Avy, vz * Avz));
    float t = 0.0f;
    if (fabsf(m01) > 1e-30f) {      // (entries are at most 1 here)
        const float theta = __fdividef(m11 - m00, 2.0f * m01);
        t = __fdividef(copysignf(1.0f, theta), fabsf(theta) + sqrtf(fmaf(theta, theta, 1.0f)));
    }
    d[1] = sc * fmaf(-t, m01, m00);
    d[2] = sc * fmaf(t, m01, m11);
    v[0] = vx, v[1] = vy, v[2] = vz;
    if constexpr (VEC) {
        const float c = rsqrtf(fmaf(t, t, 1.0f)), s = t * c;
        ga[0] = c * ex - s * gx, ga[1] = c * ey - s * gy, ga[2] = c * ez - s * gz;
        gb[0] = s * ex + c * gx, gb[1] = s * ey + c * gy, gb[2] = s * ez + c * gz;
    }
}

// x <- shrink_nuc(x; t) for a compact symmetric matrix (K = 3 or 6)
template <int K>
__device__ __forceinline__ void sym_shrink_nuc(float (&x)[K], float t)
{
    constexpr int M = Side<K>::v;
    if constexpr (M == 3) {
        float d[3], v[3], ga[3], gb[3];
        eig3<true>(x, d, v, ga, gb);
        float f[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) f[i] = fabsf(d[i]) > t ? d[i] - copysignf(t, d[i]) : 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b)
                x[sidx<3>(a, b)] = fmaf(f[0] * v[a], v[b], fmaf(f[1] * ga[a], ga[b], f[2] * gb[a] * gb[b]));
    } else if constexpr (M == 2) {
        float A[M][M], V[M][M];
        unpack<M>(x, A);
        jacobi<M, true>(A, V);
        float f[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const float l = A[i][i];
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
    float d[M > 0 ? M : 1];
    if constexpr (M == 3) {
        float v[3], ga[3], gb[3];
        eig3<false>(x, d, v, ga, gb);
    } else if constexpr (M == 2) {
        float A[M][M], V[M][M];
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

}  // namespace mat
}  // namespace vomt
