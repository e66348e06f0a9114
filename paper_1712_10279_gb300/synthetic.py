"""Seeded synthetic inputs shaped like the paper's experiments.

This module only draws data: densities, channel graphs and L matrices.  It
holds none of the transport method's arithmetic, so both the CUDA path and the
FP64 oracle can be fed from it.  The paper's own images (Section 8.1) and
tensor fields (Section 8.2) are not available; these recipes give inputs of the
same shapes and structure:

* ``blob_pair``          32 x 32 style colour densities: per channel three
                         isotropic Gaussian blobs (centres uniform on the grid,
                         sigma uniform in [2, 5] px, amplitude uniform in
                         [0.5, 1]) plus a 1e-3 floor; each density scaled to
                         total mass 1 over all channels.
* ``color_image_pair``   256 x 256 style colour image: per channel uniform noise
                         smoothed by a Gaussian (sigma 8 px, reflecting edges,
                         truncated at 4 sigma) plus 5 axis-aligned rectangles
                         (sides uniform in [8, 64] px, one amplitude per channel
                         uniform in [0.5, 1]); clipped at 0; total mass 1.
* ``tensor_field_pair``  real symmetric PSD k x k fields
                         R(theta) diag(lam) R(theta)^T with a smooth angle field
                         (sigma 10 px) and eigenvalues 0.05 + smooth
                         nonnegative fields; total trace 1.
* ``random_L``           N symmetric k x k matrices, Gaussian entries,
                         symmetrised and scaled to unit Frobenius norm.
* ``random_connected_graph``  G(k, p) redrawn until connected.
* ``hermitian_field_pair``, ``random_hermitian_L``  complex Hermitian positive
                         definite fields (the tensor-field recipe with a smooth
                         phase on the rotation's off-diagonal) and complex
                         Hermitian L matrices, for matrix OMT in the complex
                         setting of Section 4 (multivariate spectral densities).
* ``tensor_field_pair3`` the tensor-field recipe on an n x n x n grid (angle and
                         eigenvalue fields smoothed with sigma max(1, n/12) cells),
                         matrix densities of a 3-D DTI volume's shape.
* ``three_disk_pair``    the structure of the colour-disk example of Section 8.1
                         (Figure 3): three disks at the same places in both
                         images, each a pure colour, the colours permuted
                         between the two images (a pure recolouring); total
                         mass 1.
* ``blob_pair3``         the blob recipe on an n x n x n grid (three blobs per
                         channel, sigma uniform in [n/12, n/5] cells, amplitude
                         uniform in [0.5, 1], 1e-3 floor; total mass 1), the
                         shape of a 3-D DTI volume's scalar channels.

Densities come out as float64 arrays shaped [k, n, n] indexed [c, j, i] with the
x index i fastest; matrix fields as [k*k, n, n] with entry (a, b) at plane a*k+b.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import gaussian_filter

COMPLETE_K3 = [(0, 1), (0, 2), (1, 2)]


def complete_graph(k: int):
    return [(a, b) for a in range(k) for b in range(a + 1, k)]


def _blobs(rng, n, k, nblob=3, floor=1e-3):
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    out = np.zeros((k, n, n))
    for c in range(k):
        for _ in range(nblob):
            cx, cy = rng.uniform(0.0, n, size=2)
            s = rng.uniform(2.0, 5.0)
            a = rng.uniform(0.5, 1.0)
            out[c] += a * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2.0 * s * s))
    out += floor
    return out / out.sum()


def blob_pair(n: int = 32, k: int = 3, seed: int = 1001):
    rng = np.random.default_rng(seed)
    return _blobs(rng, n, k), _blobs(rng, n, k)


def _blobs3(rng, n, k, nblob=3, floor=1e-3):
    zz, yy, xx = np.mgrid[0:n, 0:n, 0:n].astype(np.float64)
    out = np.zeros((k, n, n, n))
    for c in range(k):
        for _ in range(nblob):
            cx, cy, cz = rng.uniform(0.0, n, size=3)
            s = rng.uniform(max(n / 12.0, 0.5), max(n / 5.0, 1.0))
            a = rng.uniform(0.5, 1.0)
            out[c] += a * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2 + (zz - cz) ** 2) / (2.0 * s * s))
    out += floor
    return out / out.sum()


def blob_pair3(n: int = 32, k: int = 3, seed: int = 1006):
    """[k, n, n, n] densities ([c, z, y, x], x fastest)."""
    rng = np.random.default_rng(seed)
    return _blobs3(rng, n, k), _blobs3(rng, n, k)


def _smooth_noise(rng, n, sigma):
    return gaussian_filter(rng.uniform(0.0, 1.0, size=(n, n)), sigma, mode="reflect", truncate=4.0)


def _color_image(rng, n, k, nrect=5, sigma=8.0):
    out = np.stack([_smooth_noise(rng, n, sigma) for _ in range(k)])
    lo, hi = min(8, n), min(64, n)
    for _ in range(nrect):
        w = int(rng.integers(lo, hi + 1))
        h = int(rng.integers(lo, hi + 1))
        x0 = int(rng.integers(0, n - w + 1))
        y0 = int(rng.integers(0, n - h + 1))
        amp = rng.uniform(0.5, 1.0, size=k)
        out[:, y0:y0 + h, x0:x0 + w] += amp[:, None, None]
    out = np.maximum(out, 0.0)
    return out / out.sum()


def color_image_pair(n: int = 256, k: int = 3, seed: int = 1002):
    rng = np.random.default_rng(seed)
    return _color_image(rng, n, k), _color_image(rng, n, k)


def _rot_z(theta, k):
    """Rotation about the last axis-pair (in-plane angle) for k x k, k >= 2."""
    R = np.zeros(theta.shape + (k, k))
    for a in range(k):
        R[..., a, a] = 1.0
    c, s = np.cos(theta), np.sin(theta)
    R[..., 0, 0] = c
    R[..., 0, 1] = -s
    R[..., 1, 0] = s
    R[..., 1, 1] = c
    return R


def _tensor_field(rng, n, k, sigma=10.0):
    t = _smooth_noise(rng, n, sigma)
    t = (t - t.min()) / max(t.max() - t.min(), 1e-300)
    theta = 2.0 * np.pi * t
    lam = np.stack([0.05 + _smooth_noise(rng, n, sigma) for _ in range(k)], axis=-1)  # [n, n, k]
    R = _rot_z(theta, k)                                                            # [n, n, k, k]
    M = np.einsum("jiab,jib,jicb->jiac", R, lam, R)
    M = M / np.trace(M, axis1=-2, axis2=-1).sum()
    return np.ascontiguousarray(M.reshape(n, n, k * k).transpose(2, 0, 1))


def tensor_field_pair(n: int = 128, k: int = 3, seed: int = 1003):
    rng = np.random.default_rng(seed)
    return _tensor_field(rng, n, k), _tensor_field(rng, n, k)


def _tensor_field3(rng, n, k, sigma):
    def smooth3():
        return gaussian_filter(rng.uniform(0.0, 1.0, size=(n, n, n)), sigma, mode="reflect", truncate=4.0)
    t = smooth3()
    t = (t - t.min()) / max(t.max() - t.min(), 1e-300)
    theta = 2.0 * np.pi * t
    lam = np.stack([0.05 + smooth3() for _ in range(k)], axis=-1)                  # [n, n, n, k]
    R = _rot_z(theta, k)                                                            # [n, n, n, k, k]
    M = np.einsum("zjiab,zjib,zjicb->zjiac", R, lam, R)
    M = M / np.trace(M, axis1=-2, axis2=-1).sum()
    return np.ascontiguousarray(M.reshape(n, n, n, k * k).transpose(3, 0, 1, 2))


def tensor_field_pair3(n: int = 32, k: int = 3, seed: int = 1009):
    """[k*k, n, n, n] symmetric positive definite fields (the 2-D recipe on a volume,
    smoothing sigma max(1, n/12) cells), total trace 1 each."""
    rng = np.random.default_rng(seed)
    sigma = max(1.0, n / 12.0)
    return _tensor_field3(rng, n, k, sigma), _tensor_field3(rng, n, k, sigma)


def _hermitian_field(rng, n, k, sigma=10.0):
    t = _smooth_noise(rng, n, sigma)
    t = (t - t.min()) / max(t.max() - t.min(), 1e-300)
    theta = 2.0 * np.pi * t
    s = _smooth_noise(rng, n, sigma)
    psi = 2.0 * np.pi * (s - s.min()) / max(s.max() - s.min(), 1e-300)
    lam = np.stack([0.05 + _smooth_noise(rng, n, sigma) for _ in range(k)], axis=-1)   # [n, n, k]
    Q = _rot_z(theta, k).astype(np.complex128)                                          # [n, n, k, k]
    Q[..., 0, 1] *= np.exp(1j * psi)
    Q[..., 1, 0] *= np.exp(-1j * psi)
    M = np.einsum("jiab,jib,jicb->jiac", Q, lam, Q.conj())
    M = M / np.trace(M, axis1=-2, axis2=-1).real.sum()
    return np.ascontiguousarray(M.reshape(n, n, k * k).transpose(2, 0, 1))


def hermitian_field_pair(n: int = 128, k: int = 2, seed: int = 1010):
    """[k*k, n, n] complex Hermitian positive definite fields Q diag(lam) Q*, Q a rotation of
    the first two coordinates by a smooth angle with a smooth phase on its off-diagonal
    (sigma 10 px), lam = 0.05 + smooth fields; total trace 1 each."""
    rng = np.random.default_rng(seed)
    return _hermitian_field(rng, n, k), _hermitian_field(rng, n, k)


def random_hermitian_L(k: int = 2, N: int = 3, seed: int = 1010):
    """N complex Hermitian k x k matrices (G + G*) / 2, G with N(0,1) real and imaginary
    parts, each scaled to unit Frobenius norm."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(N):
        G = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
        H = (G + G.conj().T) / 2.0
        out.append(H / np.linalg.norm(H))
    return np.array(out)


def random_L(k: int = 3, N: int = 3, seed: int = 1003):
    rng = np.random.default_rng(seed + 7919)
    out = []
    for _ in range(N):
        G = rng.standard_normal((k, k))
        S = 0.5 * (G + G.T)
        out.append(S / np.linalg.norm(S))
    return np.stack(out)


def paper_L():
    """The two L matrices printed in Section 8.2."""
    return np.array([[[1.0, 0, 0], [0, 2, 0], [0, 0, 0]],
                     [[1.0, 1, 1], [1, 0, 0], [1, 0, 0]]])


def _connected(k, edges):
    seen, stack = {0}, [0]
    adj = {a: [] for a in range(k)}
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    while stack:
        v = stack.pop()
        for u in adj[v]:
            if u not in seen:
                seen.add(u)
                stack.append(u)
    return len(seen) == k


def random_connected_graph(rng, k: int, p: float = 0.6):
    if k == 1:
        return []
    while True:
        edges = [(a, b) for a in range(k) for b in range(a + 1, k) if rng.uniform() < p]
        if _connected(k, edges):
            return edges


def batched_instances(count: int = 512, seed: int = 1004,
                      sides=(32, 64, 96, 128, 192, 256), ks=(1, 3, 5)):
    """Mixed-size vector OMT problems: side, channel count and graph drawn per instance."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(rng.choice(sides))
        k = int(rng.choice(ks))
        edges = random_connected_graph(rng, k)
        sub = np.random.default_rng(seed * 100003 + q)
        out.append(dict(n=n, k=k, edges=edges, rho0=_blobs(sub, n, k), rho1=_blobs(sub, n, k)))
    return out


def mass_preserving_directions(rho1, count: int, seed: int = 1005):
    """Directions delta = rho1 * xi with xi ~ N(0, 1), projected to sum(delta) = 0."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = rho1 * rng.standard_normal(rho1.shape)
        d -= rho1 * (d.sum() / rho1.sum())
        out.append(d)
    return out


def shifted_blob_pair(n: int, k: int, shift: int, sigma: float = 1.5, margin: int = 3, seed: int = 7):
    """A density and its copy moved by `shift` whole pixels in +x (support kept off the edge)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    base = np.zeros((k, n, n))
    lo, hi = margin, n - margin - shift
    for c in range(k):
        cx = rng.uniform(lo + 2 * sigma, hi - 2 * sigma) if hi - lo > 4 * sigma else 0.5 * (lo + hi)
        cy = rng.uniform(margin + 2 * sigma, n - margin - 2 * sigma)
        base[c] = rng.uniform(0.5, 1.0) * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sigma ** 2))
    base[:, :, :lo] = 0.0
    base[:, :, hi:] = 0.0
    base[:, :margin, :] = 0.0
    base[:, n - margin:, :] = 0.0
    base /= base.sum()
    moved = np.zeros_like(base)
    moved[:, :, shift:] = base[:, :, :n - shift]
    return base, moved


def three_disk_pair(n: int, radius: float = 0.12,
                    centres=((0.3, 0.3), (0.7, 0.35), (0.5, 0.7))):
    """Three disks (centres and radius in units of the unit square) that keep their place
    and change colour: disk d is channel d in rho0 and channel (d + 1) mod 3 in rho1."""
    x = np.arange(n) / (n - 1)
    X, Y = np.meshgrid(x, x)
    rho0 = np.zeros((3, n, n))
    rho1 = np.zeros((3, n, n))
    for d, (cx, cy) in enumerate(centres):
        m = (X - cx) ** 2 + (Y - cy) ** 2 <= radius ** 2
        rho0[d][m] += 1.0
        rho1[(d + 1) % 3][m] += 1.0
    return rho0 / rho0.sum(), rho1 / rho1.sum()
