"""FP64 CPU oracle for vector / matrix / scalar L1 optimal mass transport by PDHG.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports, links or calls it, and it shares no
code with the CUDA library: the two are independent restatements of the paper
(Ryu, Chen, Li, Osher, arXiv:1712.10279), checked against each other.

The arithmetic lives in ``vomt_oracle.c`` (plain C, double precision, one
thread); this module compiles it with gcc on first use and wraps it with
ctypes.  Grid fields are numpy float64 arrays shaped ``[planes, n, n]`` indexed
``[c, j, i]`` (x index i fastest), matching Appendix A's (i, j) grid.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vomt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libvomt_oracle.so")
_lib = None

NMET = 8
MET_NAMES = ("primal", "dual", "rel_gap", "rel_res", "fp_resid", "dual_infeas", "iter", "converged")

U_L12, U_L2, U_L1, U_NUC = 0, 1, 2, 3      # U_NUC: matrix OMT only (||U_x||_nuc + ||U_y||_nuc)
W_L1, W_L2, W_NUC = 0, 1, 2                # W_NUC: matrix OMT only (sum_s ||W_s||_nuc)


_OMP_LIB_PATH = os.path.join(_HERE, "libvomt_oracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle into ``libvomt_oracle.so`` (plain gcc, no fast-math).  With
    ``openmp`` the same source is built with -fopenmp into ``libvomt_oracle_omp.so``:
    the loops over grid points run on several threads, with bit-identical results."""
    path = _OMP_LIB_PATH if openmp else _LIB_PATH
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    extra = ["-fopenmp", "-DORC_OPENMP"] if openmp else []
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", *extra, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


_serial_lib = None
_omp_lib = None


def set_threads(threads: int) -> int:
    """Run the following oracle calls on `threads` host threads (1: the one-thread build,
    the default; more: the OpenMP build).  Returns the threads the library will use."""
    global _lib, _serial_lib, _omp_lib
    if threads <= 1:
        if _serial_lib is None:
            _lib = None
            _serial_lib = _load()
        _lib = _serial_lib
        return 1
    if _omp_lib is None:
        if _serial_lib is None:
            _serial_lib = _load()
        _lib = None
        _omp_lib = _load(openmp=True)
    _lib = _omp_lib
    _lib.orc_set_threads(int(threads))
    return int(_lib.orc_max_threads())


def _load(openmp: bool = False):
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build(openmp=openmp))
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        sig = {
            "orc_shrink1": (d, [d, d]),
            "orc_shrink2": (None, [i, p, d, p]),
            "orc_jacobi_eigvals": (i, [i, p, p]),
            "orc_incidence": (i, [i, i, p, p, p]),
            "orc_graph_lmax": (d, [i, i, p, p, p]),
            "orc_grad_G": (None, [i, i, i, p, p, p, p, p]),
            "orc_div_G": (None, [i, i, i, p, p, p, p, p]),
            "orc_grad": (None, [i, i, p, p, p]),
            "orc_div": (None, [i, i, p, p, p]),
            "orc_grad_L": (None, [i, i, i, p, p, p]),
            "orc_div_L": (None, [i, i, i, p, p, p]),
            "orc_neg_quantum_laplacian": (None, [i, i, p, p]),
            "orc_quantum_lmax": (d, [i, i, p]),
            "orc_quantum_sym_gap": (d, [i, i, p]),
            "orc_step_sizes": (None, [i, d, d, i, p, p]),
            "orc_vomt_metrics": (None, [i, i, i, p, p, p, p, p, d, i, i, d, d, d,
                                        p, p, p, p, p, p, p, p, d, p]),
            "orc_vomt_solve": (i, [i, i, i, p, p, p, p, p, d, d, d, d, i, i, i, i, d, d,
                                   p, p, p, p, p, p, i, d]),
            "orc_somt_run": (i, [i, p, p, d, d, i, i, p, p, p]),
            "orc_momt_metrics": (None, [i, i, i, p, p, p, d, i, i, d, d, d,
                                        p, p, p, p, p, p, p, p, p]),
            "orc_momt_solve": (i, [i, i, i, p, p, p, d, d, d, d, i, i, i, i, d, d,
                                   p, p, p, p, p, p, i]),
            "orc_envelope_grad": (None, [i, i, i, i, p, p, p, p, p]),
            "orc_nuc_norm": (d, [i, p]),
            "orc_grad3": (None, [i, i, p, p, p, p]),
            "orc_div3": (None, [i, i, p, p, p, p]),
            "orc_step_mu3": (d, [i, d, i]),
            "orc_vomt3_metrics": (None, [i, i, i, p, p, p, p, p, d, i, i, d, d, d,
                                         p, p, p, p, p, p, p, p, p, p, p]),
            "orc_vomt3_solve": (i, [i, i, i, p, p, p, p, p, d, d, d, d, i, i, i, i, d, d,
                                    p, p, p, p, p, p, p, i]),
            "orc_momt3_metrics": (None, [i, i, i, p, p, p, d, i, i, d, d, d,
                                         p, p, p, p, p, p, p, p, p, p, p]),
            "orc_momt3_solve": (i, [i, i, i, p, p, p, d, d, d, d, i, i, i, i, d, d,
                                    p, p, p, p, p, p, p, i]),
            "orc_zgrad_L_point": (None, [i, i, p, p, p]),
            "orc_zdiv_L_point": (None, [i, i, p, p, p]),
            "orc_zquantum_lmax": (d, [i, i, p]),
            "orc_zmomt_solve": (i, [i, i, i, p, p, p, d, i, i, d, d, d, i, i, d, d, p, p, p, p, p, p, i]),
            "orc_spectral_norm": (d, [i, p]),
            "orc_shrink_nuc": (None, [i, p, d, p]),
            "orc_vomt_unrolled_grad": (d, [i, i, i, p, p, p, p, p, d, d, d, d, i, i, p, p, p]),
            "orc_set_threads": (None, [i]),
            "orc_max_threads": (i, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _edges(edges):
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    return np.ascontiguousarray(e[:, 0]), np.ascontiguousarray(e[:, 1])


def _cost(cost, l):
    return None if cost is None else _f64(np.broadcast_to(np.asarray(cost, np.float64), (l,)))


# ---------------------------------------------------------------- building blocks
def shrink1(x: float, t: float) -> float:
    """Scalar soft threshold (Appendix B, shrink_1)."""
    return _load().orc_shrink1(float(x), float(t))


def shrink2(x, t: float):
    """Vector shrink (Appendix B, shrink_2)."""
    x = _f64(x).ravel()
    out = np.empty_like(x)
    _load().orc_shrink2(x.size, _ptr(x), float(t), _ptr(out))
    return out



def nuc_norm(X):
    """Sum of the singular values of the square matrix X."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    return float(_load().orc_nuc_norm(X.shape[0], _ptr(X)))


def spectral_norm(X):
    """Largest singular value of the square matrix X (the dual of the nuclear norm)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    return float(_load().orc_spectral_norm(X.shape[0], _ptr(X)))


def shrink_nuc(X, t: float):
    """argmin_Z t ||Z||_nuc + ||Z - X||_F^2 / 2 (singular values soft-thresholded by t)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros_like(X)
    _load().orc_shrink_nuc(X.shape[0], _ptr(X), float(t), _ptr(out))
    return out

def jacobi_eigvals(A):
    A = _f64(A)
    ev = np.empty(A.shape[0])
    _load().orc_jacobi_eigvals(A.shape[0], _ptr(A), _ptr(ev))
    return ev


def incidence(k: int, edges):
    """Incidence matrix D of Section 3.1 (edges oriented from smaller to larger node)."""
    a, b = _edges(edges)
    D = np.empty((k, a.size))
    if _load().orc_incidence(k, a.size, _ptr(a), _ptr(b), _ptr(D)) != 0:
        raise ValueError("bad edge list")
    return D


def graph_lmax(k: int, edges, cost=None) -> float:
    a, b = _edges(edges)
    c = _cost(cost, a.size)
    return _load().orc_graph_lmax(k, a.size, _ptr(a), _ptr(b), _ptr(c))


def grad(phi):
    phi = _f64(phi)
    gx, gy = np.empty_like(phi), np.empty_like(phi)
    _load().orc_grad(phi.shape[-1], phi.shape[0], _ptr(phi), _ptr(gx), _ptr(gy))
    return gx, gy


def div(ux, uy):
    ux, uy = _f64(ux), _f64(uy)
    out = np.empty_like(ux)
    _load().orc_div(ux.shape[-1], ux.shape[0], _ptr(ux), _ptr(uy), _ptr(out))
    return out


def grad_G(phi, edges, cost=None):
    phi = _f64(phi)
    a, b = _edges(edges)
    c = _cost(cost, a.size)
    n = phi.shape[-1]
    g = np.empty((a.size, n, n))
    _load().orc_grad_G(n, phi.shape[0], a.size, _ptr(a), _ptr(b), _ptr(c), _ptr(phi), _ptr(g))
    return g


def div_G(y, k: int, edges, cost=None):
    y = _f64(y)
    a, b = _edges(edges)
    c = _cost(cost, a.size)
    n = y.shape[-1]
    out = np.empty((k, n, n))
    _load().orc_div_G(n, k, a.size, _ptr(a), _ptr(b), _ptr(c), _ptr(y), _ptr(out))
    return out


def grad_L(X, L):
    """Quantum gradient (Section 4.1).  X: [k*k, n, n] full matrices; L: [N, k, k]."""
    X, L = _f64(X), _f64(L)
    N, k = L.shape[0], L.shape[1]
    n = X.shape[-1]
    Z = np.empty((N * k * k, n, n))
    _load().orc_grad_L(n, k, N, _ptr(L), _ptr(X), _ptr(Z))
    return Z


def div_L(Z, L):
    Z, L = _f64(Z), _f64(L)
    N, k = L.shape[0], L.shape[1]
    n = Z.shape[-1]
    Y = np.empty((k * k, n, n))
    _load().orc_div_L(n, k, N, _ptr(L), _ptr(Z), _ptr(Y))
    return Y


def neg_quantum_laplacian(L):
    L = _f64(L)
    N, k = L.shape[0], L.shape[1]
    M = np.empty((k * k, k * k))
    _load().orc_neg_quantum_laplacian(k, N, _ptr(L), _ptr(M))
    return M


def quantum_lmax(L) -> float:
    L = _f64(L)
    return _load().orc_quantum_lmax(L.shape[1], L.shape[0], _ptr(L))


def quantum_sym_gap(L) -> float:
    L = _f64(L)
    return _load().orc_quantum_sym_gap(L.shape[1], L.shape[0], _ptr(L))


def step_sizes(n: int, tau: float, lmax_second: float, has_second: bool):
    mu, nu = np.zeros(1), np.zeros(1)
    _load().orc_step_sizes(n, float(tau), float(lmax_second), int(has_second), _ptr(mu), _ptr(nu))
    return float(mu[0]), float(nu[0])


def default_tau_vector(n: int) -> float:
    """Table 1's tuned tau: 1 for the 32^2 and 64^2 grids, 3 for 128^2 and 256^2."""
    return 1.0 if n <= 64 else 3.0


def default_tau_matrix(n: int) -> float:
    """Table 3's tuned tau: 10 (32^2, 64^2), 30 (128^2), 60 (256^2)."""
    return 10.0 if n <= 64 else (30.0 if n <= 128 else 60.0)


# ---------------------------------------------------------------- solvers
def vomt_metrics(state, prev, rho0, rho1, edges, alpha, mu, nu, tau, cost=None,
                 u_norm=U_L12, w_norm=W_L1, eps=0.0):
    rho0, rho1 = _f64(rho0), _f64(rho1)
    k, n = rho0.shape[0], rho0.shape[-1]
    a, b = _edges(edges)
    c = _cost(cost, a.size)
    ux, uy, w, phi = (_f64(state[x]) for x in ("ux", "uy", "w", "phi"))
    if prev is not None:
        pux, puy, pw, pphi = (_f64(prev[x]) for x in ("ux", "uy", "w", "phi"))
    else:
        pux = puy = pw = pphi = None
    out = np.zeros(NMET)
    _load().orc_vomt_metrics(n, k, a.size, _ptr(a), _ptr(b), _ptr(c), _ptr(rho0), _ptr(rho1),
                             float(alpha), u_norm, w_norm, float(mu), float(nu), float(tau),
                             _ptr(ux), _ptr(uy), _ptr(w), _ptr(phi),
                             _ptr(pux), _ptr(puy), _ptr(pw), _ptr(pphi), float(eps), _ptr(out))
    return out


def vomt_solve(rho0, rho1, edges, alpha=1.0, tau=None, mu=None, nu=None, cost=None,
               u_norm=U_L12, w_norm=W_L1, max_iters=2000, check_every=100,
               tol_gap=0.0, tol_res=0.0, init=None, history=False, eps=0.0):
    """Run the V-OMT iteration of Section 7.2 in FP64.

    rho0, rho1: [k, n, n] cell masses.  edges: list of node pairs of the channel
    graph (empty for k = 1).  tau/mu/nu default to the paper's rules.  eps > 0 adds
    the quadratic regulariser eps (||u||_2^2 + ||w||_2^2) of the paper's conclusions
    (Euclidean norms per point).  Returns a
    dict with the final state (ux, uy, w, phi), the step sizes, the metrics of the
    last check and, if asked, every check row.
    """
    rho0, rho1 = _f64(rho0), _f64(rho1)
    k, n = rho0.shape[0], rho0.shape[-1]
    a, b = _edges(edges)
    l = a.size
    c = _cost(cost, l)
    if tau is None:
        tau = default_tau_vector(n)
    if mu is None or nu is None:
        lm = graph_lmax(k, edges, cost) if l else 0.0
        m0, n0 = step_sizes(n, tau, lm, l > 0)
        mu = m0 if mu is None else mu
        nu = n0 if nu is None else nu
    if init is None:
        ux = np.zeros((k, n, n)); uy = np.zeros((k, n, n))
        w = np.zeros((l, n, n)); phi = np.zeros((k, n, n))
    else:
        ux, uy, w, phi = (np.array(init[x], dtype=np.float64, copy=True) for x in ("ux", "uy", "w", "phi"))
    nchk = max_iters // max(check_every, 1) + 2
    hist = np.zeros((nchk, NMET))
    met = np.zeros(NMET)
    it = _load().orc_vomt_solve(n, k, l, _ptr(a), _ptr(b), _ptr(c), _ptr(rho0), _ptr(rho1),
                                float(alpha), float(tau), float(mu), float(nu), u_norm, w_norm,
                                int(max_iters), int(check_every), float(tol_gap), float(tol_res),
                                _ptr(ux), _ptr(uy), _ptr(w), _ptr(phi), _ptr(met), _ptr(hist), nchk, float(eps))
    out = dict(ux=ux, uy=uy, w=w, phi=phi, iters=it, mu=mu, nu=nu, tau=tau,
               metrics=dict(zip(MET_NAMES, met)))
    if history:
        rows = hist[hist[:, 6] > 0]
        out["history"] = rows
    return out


def somt_run(rho0, rho1, tau, mu=None, iters=100, u_norm=U_L12):
    """The S-OMT box of Section 7.1 (scalar densities [n, n])."""
    rho0, rho1 = _f64(rho0), _f64(rho1)
    n = rho0.shape[-1]
    if mu is None:
        mu = step_sizes(n, tau, 0.0, False)[0]
    ux = np.zeros((n, n)); uy = np.zeros((n, n)); phi = np.zeros((n, n))
    _load().orc_somt_run(n, _ptr(rho0), _ptr(rho1), float(tau), float(mu), int(u_norm), int(iters),
                         _ptr(ux), _ptr(uy), _ptr(phi))
    return dict(ux=ux, uy=uy, phi=phi, mu=mu, tau=tau)


def momt_metrics(state, prev, Lam0, Lam1, L, alpha, mu, nu, tau, u_norm=U_L2, w_norm=W_L1):
    Lam0, Lam1, L = _f64(Lam0), _f64(Lam1), _f64(L)
    N, k = L.shape[0], L.shape[1]
    n = Lam0.shape[-1]
    Ux, Uy, W, Phi = (_f64(state[x]) for x in ("Ux", "Uy", "W", "Phi"))
    if prev is not None:
        p = [_f64(prev[x]) for x in ("Ux", "Uy", "W", "Phi")]
    else:
        p = [None] * 4
    out = np.zeros(NMET)
    _load().orc_momt_metrics(n, k, N, _ptr(L), _ptr(Lam0), _ptr(Lam1), float(alpha), u_norm, w_norm,
                             float(mu), float(nu), float(tau), _ptr(Ux), _ptr(Uy), _ptr(W), _ptr(Phi),
                             *[_ptr(x) for x in p], _ptr(out))
    return out


def momt_solve(Lam0, Lam1, L, alpha=1.0, tau=None, mu=None, nu=None, u_norm=U_L2, w_norm=W_L1,
               max_iters=2000, check_every=100, tol_gap=0.0, tol_res=0.0, init=None, history=False):
    """Run the M-OMT iteration of Section 7.3 in FP64.

    Lam0, Lam1: [k*k, n, n] full real symmetric matrices per cell (entry (a, b)
    at plane a*k+b).  L: [N, k, k] real symmetric.
    """
    Lam0, Lam1, L = _f64(Lam0), _f64(Lam1), _f64(L)
    N, k = L.shape[0], L.shape[1]
    n = Lam0.shape[-1]
    if k > 8 or N * k * k > 512:
        raise ValueError("k <= 8 and N k^2 <= 512")
    if tau is None:
        tau = default_tau_matrix(n)
    if mu is None or nu is None:
        m0, n0 = step_sizes(n, tau, quantum_lmax(L), True)
        mu = m0 if mu is None else mu
        nu = n0 if nu is None else nu
    kk = k * k
    if init is None:
        Ux = np.zeros((kk, n, n)); Uy = np.zeros((kk, n, n))
        W = np.zeros((N * kk, n, n)); Phi = np.zeros((kk, n, n))
    else:
        Ux, Uy, W, Phi = (np.array(init[x], dtype=np.float64, copy=True) for x in ("Ux", "Uy", "W", "Phi"))
    nchk = max_iters // max(check_every, 1) + 2
    hist = np.zeros((nchk, NMET))
    met = np.zeros(NMET)
    it = _load().orc_momt_solve(n, k, N, _ptr(L), _ptr(Lam0), _ptr(Lam1), float(alpha), float(tau),
                                float(mu), float(nu), u_norm, w_norm, int(max_iters), int(check_every),
                                float(tol_gap), float(tol_res), _ptr(Ux), _ptr(Uy), _ptr(W), _ptr(Phi),
                                _ptr(met), _ptr(hist), nchk)
    out = dict(Ux=Ux, Uy=Uy, W=W, Phi=Phi, iters=it, mu=mu, nu=nu, tau=tau,
               metrics=dict(zip(MET_NAMES, met)))
    if history:
        out["history"] = hist[hist[:, 6] > 0]
    return out


def envelope_grad(phi, w, w_norm=W_L1):
    """dV/drho1, dV/drho0 (gauge-fixed phi*) and dV/dalpha from a converged state."""
    phi, w = _f64(phi), _f64(w)
    k, n = phi.shape[0], phi.shape[-1]
    l = w.shape[0]
    g1, g0 = np.empty_like(phi), np.empty_like(phi)
    ga = np.zeros(1)
    _load().orc_envelope_grad(n, k, l, w_norm, _ptr(phi), _ptr(w) if l else None,
                              _ptr(g1), _ptr(g0), _ptr(ga))
    return g1, g0, float(ga[0])


def unrolled_grad(rho0, rho1, edges, alpha, T, tau=None, mu=None, nu=None, cost=None, w_norm=W_L1):
    """J_T = P(u^T, w^T) after T iterations from zero, and its exact gradient."""
    rho0, rho1 = _f64(rho0), _f64(rho1)
    k, n = rho0.shape[0], rho0.shape[-1]
    a, b = _edges(edges)
    l = a.size
    c = _cost(cost, l)
    if tau is None:
        tau = default_tau_vector(n)
    if mu is None or nu is None:
        lm = graph_lmax(k, edges, cost) if l else 0.0
        m0, n0 = step_sizes(n, tau, lm, l > 0)
        mu = m0 if mu is None else mu
        nu = n0 if nu is None else nu
    g1, g0 = np.empty_like(rho0), np.empty_like(rho0)
    ga = np.zeros(1)
    J = _load().orc_vomt_unrolled_grad(n, k, l, _ptr(a), _ptr(b), _ptr(c), _ptr(rho0), _ptr(rho1),
                                       float(alpha), float(tau), float(mu), float(nu), int(w_norm),
                                       int(T), _ptr(g1), _ptr(g0), _ptr(ga))
    return J, g1, g0, float(ga[0])


# ---------------------------------------------------------------- 3-D grids
def grad3(phi):
    """Forward differences on an n x n x n grid, [planes, z, y, x]; ghost entries zero."""
    phi = _f64(phi)
    planes, n = phi.shape[0], phi.shape[-1]
    gx, gy, gz = (np.zeros_like(phi) for _ in range(3))
    _load().orc_grad3(n, planes, _ptr(phi), _ptr(gx), _ptr(gy), _ptr(gz))
    return gx, gy, gz


def div3(ux, uy, uz):
    ux, uy, uz = _f64(ux), _f64(uy), _f64(uz)
    planes, n = ux.shape[0], ux.shape[-1]
    out = np.zeros_like(ux)
    _load().orc_div3(n, planes, _ptr(ux), _ptr(uy), _ptr(uz), _ptr(out))
    return out


def vomt3_solve(rho0, rho1, edges, alpha=1.0, tau=None, mu=None, nu=None, cost=None, u_norm=U_L12, w_norm=W_L1,
                max_iters=2000, check_every=100, tol_gap=0.0, tol_res=0.0, init=None, history=False):
    """V-OMT by PDHG on an n x n x n grid (the 3-D extension of Section 7.2).  rho0, rho1:
    [k, n, n, n] cell masses.  mu defaults to 1/(48 tau (n-1)^2) (1/(24 ...) without edges)."""
    rho0, rho1 = _f64(rho0), _f64(rho1)
    k, n = rho0.shape[0], rho0.shape[-1]
    a, b = _edges(edges)
    l = a.size
    c = _cost(cost, l)
    if tau is None:
        tau = default_tau_vector(n)
    if mu is None:
        mu = float(_load().orc_step_mu3(n, float(tau), int(l > 0)))
    if nu is None:
        nu = 1.0 / (4.0 * tau * graph_lmax(k, edges, cost)) if l else 0.0
    if init is None:
        ux, uy, uz = (np.zeros((k, n, n, n)) for _ in range(3))
        w = np.zeros((l, n, n, n)); phi = np.zeros((k, n, n, n))
    else:
        ux, uy, uz, w, phi = (np.array(init[x], dtype=np.float64, copy=True) for x in ("ux", "uy", "uz", "w", "phi"))
    nchk = max_iters // max(check_every, 1) + 2
    hist = np.zeros((nchk, NMET))
    met = np.zeros(NMET)
    it = _load().orc_vomt3_solve(n, k, l, _ptr(a), _ptr(b), _ptr(c), _ptr(rho0), _ptr(rho1), float(alpha),
                                 float(tau), float(mu), float(nu), u_norm, w_norm, int(max_iters), int(check_every),
                                 float(tol_gap), float(tol_res), _ptr(ux), _ptr(uy), _ptr(uz), _ptr(w), _ptr(phi),
                                 _ptr(met), _ptr(hist), nchk)
    out = dict(ux=ux, uy=uy, uz=uz, w=w, phi=phi, iters=it, mu=mu, nu=nu, tau=tau,
               metrics=dict(zip(MET_NAMES, met)))
    if history:
        out["history"] = hist[hist[:, 6] > 0]
    return out


def momt3_solve(Lam0, Lam1, L, alpha=1.0, tau=None, mu=None, nu=None, u_norm=U_L2, w_norm=W_L1,
                max_iters=2000, check_every=100, tol_gap=0.0, tol_res=0.0, init=None, history=False):
    """The M-OMT iteration of Section 7.3 in FP64 on an n x n x n grid.

    Lam0, Lam1: [k*k, n, n, n] full real symmetric matrices per cell.  L: [N, k, k].  U has
    three directions Ux, Uy, Uz ([k*k, n, n, n] each); ||U||_2 is the Frobenius norm over the
    three directions jointly, ||U||_{1,nuc} the sum of the three directions' nuclear norms.
    mu defaults to 1/(48 tau (n-1)^2), nu to 1/(4 tau lambda_max(-Delta_L)).
    """
    Lam0, Lam1, L = _f64(Lam0), _f64(Lam1), _f64(L)
    N, k = L.shape[0], L.shape[1]
    n = Lam0.shape[-1]
    if k > 8 or N * k * k > 512:
        raise ValueError("k <= 8 and N k^2 <= 512")
    if tau is None:
        tau = default_tau_matrix(n)
    if mu is None:
        mu = float(_load().orc_step_mu3(n, float(tau), 1))
    if nu is None:
        nu = 1.0 / (4.0 * tau * quantum_lmax(L))
    kk = k * k
    if init is None:
        Ux, Uy, Uz = (np.zeros((kk, n, n, n)) for _ in range(3))
        W = np.zeros((N * kk, n, n, n)); Phi = np.zeros((kk, n, n, n))
    else:
        Ux, Uy, Uz, W, Phi = (np.array(init[x], dtype=np.float64, copy=True) for x in ("Ux", "Uy", "Uz", "W", "Phi"))
    nchk = max_iters // max(check_every, 1) + 2
    hist = np.zeros((nchk, NMET))
    met = np.zeros(NMET)
    it = _load().orc_momt3_solve(n, k, N, _ptr(L), _ptr(Lam0), _ptr(Lam1), float(alpha), float(tau),
                                 float(mu), float(nu), u_norm, w_norm, int(max_iters), int(check_every),
                                 float(tol_gap), float(tol_res), _ptr(Ux), _ptr(Uy), _ptr(Uz), _ptr(W), _ptr(Phi),
                                 _ptr(met), _ptr(hist), nchk)
    out = dict(Ux=Ux, Uy=Uy, Uz=Uz, W=W, Phi=Phi, iters=it, mu=mu, nu=nu, tau=tau,
               metrics=dict(zip(MET_NAMES, met)))
    if history:
        out["history"] = hist[hist[:, 6] > 0]
    return out


# ---------------------------------------------------------------- complex Hermitian matrix OMT
def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def zgrad_L_point(X, L):
    """[L_s X - X L_s]_s for one complex k x k X; L: [N, k, k] complex."""
    X, L = _c128(X), _c128(L)
    N, k = L.shape[0], L.shape[1]
    Z = np.zeros((N, k, k), np.complex128)
    _load().orc_zgrad_L_point(k, N, _ptr(L), _ptr(X), _ptr(Z))
    return Z


def zdiv_L_point(Z, L):
    """sum_s (-L_s Z_s + Z_s L_s) for one point."""
    Z, L = _c128(Z), _c128(L)
    N, k = L.shape[0], L.shape[1]
    Y = np.zeros((k, k), np.complex128)
    _load().orc_zdiv_L_point(k, N, _ptr(L), _ptr(Z), _ptr(Y))
    return Y


def zquantum_lmax(L) -> float:
    L = _c128(L)
    return float(_load().orc_zquantum_lmax(L.shape[1], L.shape[0], _ptr(L)))


def zmomt_solve(Lam0, Lam1, L, alpha=1.0, tau=None, mu=None, nu=None, max_iters=2000, check_every=100,
                tol_gap=0.0, tol_res=0.0, init=None, history=False, u_norm=U_L2, w_norm=W_L2):
    """The M-OMT iteration of Section 7.3 on complex Hermitian densities (Section 4's complex
    setting), FP64, with the Frobenius norms ||U||_2, ||W||_2 (u_norm U_L2, w_norm W_L2, the
    defaults) or the entrywise ||U||_1, ||W||_1 (U_L1, W_L1: sums of the entries' moduli).

    Lam0, Lam1: [k*k, n, n] complex Hermitian matrices per cell.  L: [N, k, k] complex
    Hermitian.  mu defaults to 1/(32 tau (n-1)^2), nu to 1/(4 tau lambda_max(-Delta_L)).
    """
    Lam0, Lam1, L = _c128(Lam0), _c128(Lam1), _c128(L)
    N, k = L.shape[0], L.shape[1]
    n = Lam0.shape[-1]
    if k > 8 or N * k * k > 512:
        raise ValueError("k <= 8 and N k^2 <= 512")
    if tau is None:
        tau = default_tau_matrix(n)
    if mu is None:
        mu = 1.0 / (32.0 * tau * (n - 1) ** 2)
    if nu is None:
        nu = 1.0 / (4.0 * tau * zquantum_lmax(L))
    kk = k * k
    if init is None:
        Ux = np.zeros((kk, n, n), np.complex128); Uy = np.zeros((kk, n, n), np.complex128)
        W = np.zeros((N * kk, n, n), np.complex128); Phi = np.zeros((kk, n, n), np.complex128)
    else:
        Ux, Uy, W, Phi = (np.array(init[x], dtype=np.complex128, copy=True) for x in ("Ux", "Uy", "W", "Phi"))
    nchk = max_iters // max(check_every, 1) + 2
    hist = np.zeros((nchk, NMET))
    met = np.zeros(NMET)
    if u_norm not in (U_L2, U_L1) or w_norm not in (W_L2, W_L1):
        raise ValueError("complex matrix OMT: Frobenius or entrywise norms")
    it = _load().orc_zmomt_solve(n, k, N, _ptr(L), _ptr(Lam0), _ptr(Lam1), float(alpha), int(u_norm), int(w_norm),
                                 float(tau), float(mu), float(nu), int(max_iters), int(check_every),
                                 float(tol_gap), float(tol_res),
                                 _ptr(Ux), _ptr(Uy), _ptr(W), _ptr(Phi), _ptr(met), _ptr(hist), nchk)
    out = dict(Ux=Ux, Uy=Uy, W=W, Phi=Phi, iters=it, mu=mu, nu=nu, tau=tau, metrics=dict(zip(MET_NAMES, met)))
    if history:
        out["history"] = hist[hist[:, 6] > 0]
    return out
