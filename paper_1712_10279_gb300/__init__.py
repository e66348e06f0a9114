"""GB300-native vector / matrix L1 optimal mass transport by PDHG.

Implements the primal-dual method of Ryu, Chen, Li and Osher, "Vector and
Matrix Optimal Mass Transport: Theory, Algorithm, and Applications"
(arXiv:1712.10279), Section 7, as hand-written sm_103a CUDA behind the C ABI in
``include/vomt.h``.  This package is the thin Python layer over that ABI:
torch provides device memory and streams, the library does all the work.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _native
from ._native import VomtError, ENGINES

U_L12, U_L2, U_L1, U_NUC = 0, 1, 2, 3    # U_NUC: matrix OMT, ||U_x||_nuc + ||U_y||_nuc
W_L1, W_L2, W_NUC = 0, 1, 2              # W_NUC: matrix OMT, sum_s ||W_s||_nuc

__all__ = ["solve", "solve_host", "solve3d", "step_sizes", "tune_tau", "momt_tune_tau", "history", "set_wait_policy", "VomtError", "U_L12", "U_L2", "U_L1", "U_NUC", "W_L1",
           "W_L2", "W_NUC"]


@dataclass
class Solution:
    u: object        # [2, k, n, n]: u_x planes then u_y planes
    w: object        # [l, n, n]
    phi: object      # [k, n, n]
    result: dict


def _params(tau, mu, nu, u_norm, w_norm, max_iters, check_every, tol_gap, tol_res, warm, engine, halo=0, eps=0.0,
            pitch=0):
    p = _native.Params()
    _native.load().vomt_default_params(ctypes.byref(p))
    p.tau = 0.0 if tau is None else float(tau)
    p.mu = 0.0 if mu is None else float(mu)
    p.nu = 0.0 if nu is None else float(nu)
    p.u_norm, p.w_norm = int(u_norm), int(w_norm)
    p.max_iters, p.check_every = int(max_iters), int(check_every)
    p.tol_gap, p.tol_res = float(tol_gap), float(tol_res)
    p.warm_start = int(bool(warm))
    p.engine = ENGINES[engine] if isinstance(engine, str) else int(engine)
    p.halo = int(halo)
    p.eps = float(eps)
    p.pitch = int(pitch)
    return p


def step_sizes(n: int, k: int, edges, tau=None, cost=None):
    """(mu, nu, tau, lambda_max(-Delta_G)) from the rules of Section 7.2."""
    g = _native.GraphArg(k, edges, cost)
    out = [ctypes.c_double() for _ in range(4)]
    _native.check(_native.load().vomt_step_sizes(int(n), g.ref, 0.0 if tau is None else float(tau),
                                                 *[ctypes.byref(x) for x in out]))
    return tuple(x.value for x in out)


def solve(rho0, rho1, edges, alpha: float = 1.0, *, tau=None, mu=None, nu=None, cost=None,
          u_norm: int = U_L12, w_norm: int = W_L1, max_iters: int = 2000, check_every: int = 100,
          tol_gap: float = 0.0, tol_res: float = 0.0, init=None, engine="auto", halo: int = 0,
          stream=None, eps: float = 0.0) -> Solution:
    """Vector OMT (Section 7.2) on the GPU.

    rho0, rho1: CUDA float32 tensors [k, n, n] (cell masses, [c, j, i], x fastest).
    edges: node pairs of the channel graph (empty for k = 1).  init: optional
    (u, w, phi) tensors to warm-start from.  Returns the final iterate and the
    metrics of the last FP64 convergence check.  eps > 0 solves the quadratically
    regularised problem of the paper's conclusions (eps (||u||_2^2 + ||w||_2^2)).
    """
    import torch
    if not (rho0.is_cuda and rho1.is_cuda):
        raise ValueError("rho0 and rho1 must be CUDA tensors")
    rho0 = rho0.contiguous().float()
    rho1 = rho1.contiguous().float()
    k, n = rho0.shape[0], rho0.shape[-1]
    dev = rho0.device
    g = _native.GraphArg(k, edges, cost)
    l = g.tail.size
    if init is not None:
        u = init[0].detach().clone().contiguous().float()
        w = init[1].detach().clone().contiguous().float()
        phi = init[2].detach().clone().contiguous().float()
    else:
        u = torch.empty((2, k, n, n), device=dev, dtype=torch.float32)
        w = torch.empty((max(l, 0), n, n), device=dev, dtype=torch.float32)
        phi = torch.empty((k, n, n), device=dev, dtype=torch.float32)
    p = _params(tau, mu, nu, u_norm, w_norm, max_iters, check_every, tol_gap, tol_res, init is not None, engine,
                halo, eps)
    res = _native.Result()
    st = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
    ctx = _native.context(dev.index if dev.index is not None else torch.cuda.current_device())
    rc = _native.load().vomt_solve(ctx, int(n), rho0.data_ptr(), rho1.data_ptr(), g.ref, float(alpha),
                                   ctypes.byref(p), u.data_ptr(), w.data_ptr() if l else None, phi.data_ptr(),
                                   ctypes.byref(res), ctypes.c_void_p(st))
    _native.check(rc, ctx)
    return Solution(u, w, phi, res.as_dict())


def tune_tau(rho0, rho1, edges, alpha: float = 1.0, *, cost=None, u_norm: int = U_L12, w_norm: int = W_L1,
             sample_iters: int = 1500, engine="auto", eps: float = 0.0, stream=None):
    """Measure the dual step tau for this problem (vomt_tune_tau): short GPU runs over the
    grid tau_paper * 10^((j-1)/2), successive halving, one refinement.  Sections 7.1-7.2
    tune tau per experiment; mu and nu follow from it by the paper's rule.  Returns
    (best tau, its score max(rel gap, rel res), scores of the grid after sample_iters)."""
    import torch
    rho0 = rho0.contiguous().float()
    rho1 = rho1.contiguous().float()
    k, n = rho0.shape[0], rho0.shape[-1]
    dev = rho0.device
    g = _native.GraphArg(k, edges, cost)
    l = g.tail.size
    u = torch.empty((2, k, n, n), device=dev, dtype=torch.float32)
    w = torch.empty((max(l, 1), n, n), device=dev, dtype=torch.float32)
    phi = torch.empty((k, n, n), device=dev, dtype=torch.float32)
    p = _params(None, None, None, u_norm, w_norm, sample_iters, sample_iters, 0.0, 0.0, False, engine, eps=eps)
    best, score = ctypes.c_double(), ctypes.c_double()
    grid = (ctypes.c_double * _native.TAU_GRID)()
    st = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
    ctx = _native.context(dev.index if dev.index is not None else torch.cuda.current_device())
    rc = _native.load().vomt_tune_tau(ctx, int(n), rho0.data_ptr(), rho1.data_ptr(), g.ref, float(alpha),
                                      ctypes.byref(p), int(sample_iters), u.data_ptr(), w.data_ptr() if l else None,
                                      phi.data_ptr(), ctypes.byref(best), ctypes.byref(score), grid,
                                      ctypes.c_void_p(st))
    _native.check(rc, ctx)
    return best.value, score.value, list(grid)


def solve3d(rho0, rho1, edges, alpha: float = 1.0, *, tau=None, mu=None, nu=None, cost=None,
            u_norm: int = U_L12, w_norm: int = W_L1, max_iters: int = 2000, check_every: int = 100,
            tol_gap: float = 0.0, tol_res: float = 0.0, init=None, stream=None, zc: int = 0) -> Solution:
    """Vector OMT on an n x n x n grid (Appendix A's discretization with a third direction).

    rho0, rho1: CUDA float32 tensors [k, n, n, n] (cell masses, [c, z, y, x]).  Returns u as
    [3, k, n, n, n] (u_x, u_y, u_z), w [l, n, n, n], phi [k, n, n, n] and the metrics of the
    last FP64 check.  Default mu = 1/(48 tau (n-1)^2) (1/(24 ...) without edges).  zc > 0
    sets the z planes each thread block marches through (0: the library's choice).
    """
    import torch
    if not (rho0.is_cuda and rho1.is_cuda):
        raise ValueError("rho0 and rho1 must be CUDA tensors")
    rho0 = rho0.contiguous().float()
    rho1 = rho1.contiguous().float()
    if rho0.dim() != 4 or rho0.shape != rho1.shape or not (rho0.shape[1] == rho0.shape[2] == rho0.shape[3]):
        raise ValueError("rho0 and rho1 must be [k, n, n, n] of one shape")
    k, n = rho0.shape[0], rho0.shape[-1]
    dev = rho0.device
    g = _native.GraphArg(k, edges, cost)
    l = g.tail.size
    if init is not None:
        u, w, phi = (x.detach().clone().contiguous().float() for x in init)
    else:
        u = torch.empty((3, k, n, n, n), device=dev, dtype=torch.float32)
        w = torch.empty((max(l, 0), n, n, n), device=dev, dtype=torch.float32)
        phi = torch.empty((k, n, n, n), device=dev, dtype=torch.float32)
    p = _params(tau, mu, nu, u_norm, w_norm, max_iters, check_every, tol_gap, tol_res, init is not None, "stream",
                halo=zc)
    res = _native.Result()
    st = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
    ctx = _native.context(dev.index if dev.index is not None else torch.cuda.current_device())
    rc = _native.load().vomt_solve3d(ctx, int(n), rho0.data_ptr(), rho1.data_ptr(), g.ref, float(alpha),
                                     ctypes.byref(p), u.data_ptr(), w.data_ptr() if l else None, phi.data_ptr(),
                                     ctypes.byref(res), ctypes.c_void_p(st))
    _native.check(rc, ctx)
    return Solution(u, w, phi, res.as_dict())


def solve_host(rho0, rho1, edges, alpha: float = 1.0, *, tau=None, mu=None, nu=None, cost=None,
               u_norm: int = U_L12, w_norm: int = W_L1, max_iters: int = 2000, check_every: int = 100,
               tol_gap: float = 0.0, tol_res: float = 0.0, engine="auto", halo: int = 0, device: int = 0,
               out=None, eps: float = 0.0) -> Solution:
    """The same solve through vomt_solve_host: numpy float32 inputs and outputs in host
    memory; the library copies them to and from the GPU inside the call."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float32)
    rho1 = np.ascontiguousarray(rho1, dtype=np.float32)
    k, n = rho0.shape[0], rho0.shape[-1]
    g = _native.GraphArg(k, edges, cost)
    l = g.tail.size
    if out is None:
        out = (np.empty((2, k, n, n), np.float32), np.empty((max(l, 0), n, n), np.float32),
               np.empty((k, n, n), np.float32))
    u, w, phi = out
    p = _params(tau, mu, nu, u_norm, w_norm, max_iters, check_every, tol_gap, tol_res, False, engine, halo, eps)
    res = _native.Result()
    ctx = _native.context(device)
    rc = _native.load().vomt_solve_host(ctx, int(n), rho0.ctypes.data, rho1.ctypes.data, g.ref, float(alpha),
                                        ctypes.byref(p), u.ctypes.data, w.ctypes.data if l else None,
                                        phi.ctypes.data, ctypes.byref(res), None)
    _native.check(rc, ctx)
    return Solution(u, w, phi, res.as_dict())


def momt_step_sizes(n: int, L, tau=None):
    """(mu, nu, tau, lambda_max(-Delta_L), second-smallest eigenvalue of -Delta_L on
    symmetric matrices) from the rules of Section 7.3; L: [N, k, k] real symmetric."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    N, k = L.shape[0], L.shape[1]
    out = [ctypes.c_double() for _ in range(5)]
    _native.check(_native.load().momt_step_sizes(int(n), int(k), int(N), L.ctypes.data,
                                                 0.0 if tau is None else float(tau),
                                                 *[ctypes.byref(x) for x in out]))
    return tuple(x.value for x in out)


@dataclass
class MatrixSolution:
    U: object        # [2, k*k, n, n]: U_x then U_y, full symmetric matrices
    W: object        # [N, k*k, n, n], full skew-symmetric matrices
    Phi: object      # [k*k, n, n], full symmetric matrices
    result: dict


def momt_solve(Lam0, Lam1, L, alpha: float = 1.0, *, tau=None, mu=None, nu=None, u_norm: int = U_L2,
               w_norm: int = W_L1, max_iters: int = 2000, check_every: int = 100, tol_gap: float = 0.0,
               tol_res: float = 0.0, init=None, engine="auto", halo: int = 0, stream=None) -> MatrixSolution:
    """Matrix OMT (Section 7.3) on the GPU.

    Lam0, Lam1: CUDA float32 tensors [k*k, n, n] of real symmetric matrices (entry (a, b)
    at plane a*k+b).  L: [N, k, k] real symmetric (numpy, host).  init: optional
    (U, W, Phi) tensors to warm-start from.
    """
    import torch
    Lam0 = Lam0.contiguous().float()
    Lam1 = Lam1.contiguous().float()
    Lh = np.ascontiguousarray(L, dtype=np.float64)
    N, k = Lh.shape[0], Lh.shape[1]
    kk, n = Lam0.shape[0], Lam0.shape[-1]
    if kk != k * k:
        raise ValueError("Lam0 must have k*k planes")
    dev = Lam0.device
    if init is not None:
        U, W, Phi = (x.detach().clone().contiguous().float() for x in init)
    else:
        U = torch.empty((2, kk, n, n), device=dev, dtype=torch.float32)
        W = torch.empty((N, kk, n, n), device=dev, dtype=torch.float32)
        Phi = torch.empty((kk, n, n), device=dev, dtype=torch.float32)
    p = _params(tau, mu, nu, u_norm, w_norm, max_iters, check_every, tol_gap, tol_res, init is not None, engine,
                halo)
    res = _native.Result()
    st = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
    ctx = _native.context(dev.index if dev.index is not None else torch.cuda.current_device())
    rc = _native.load().momt_solve(ctx, int(n), int(k), Lam0.data_ptr(), Lam1.data_ptr(), int(N), Lh.ctypes.data,
                                   float(alpha), ctypes.byref(p), U.data_ptr(), W.data_ptr(), Phi.data_ptr(),
                                   ctypes.byref(res), ctypes.c_void_p(st))
    _native.check(rc, ctx)
    return MatrixSolution(U, W, Phi, res.as_dict())


def momt_tune_tau(Lam0, Lam1, L, alpha: float = 1.0, *, u_norm: int = U_L2, w_norm: int = W_L1,
                  sample_iters: int = 1500, engine="auto", stream=None):
    """The tau search of tune_tau for matrix OMT (momt_tune_tau; Section 7.3, Table 3)."""
    import torch
    Lam0 = Lam0.contiguous().float()
    Lam1 = Lam1.contiguous().float()
    Lh = np.ascontiguousarray(L, dtype=np.float64)
    N, k = Lh.shape[0], Lh.shape[1]
    kk, n = Lam0.shape[0], Lam0.shape[-1]
    dev = Lam0.device
    U = torch.empty((2, kk, n, n), device=dev, dtype=torch.float32)
    W = torch.empty((N, kk, n, n), device=dev, dtype=torch.float32)
    Phi = torch.empty((kk, n, n), device=dev, dtype=torch.float32)
    p = _params(None, None, None, u_norm, w_norm, sample_iters, sample_iters, 0.0, 0.0, False, engine)
    best, score = ctypes.c_double(), ctypes.c_double()
    grid = (ctypes.c_double * _native.TAU_GRID)()
    st = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
    ctx = _native.context(dev.index if dev.index is not None else torch.cuda.current_device())
    rc = _native.load().momt_tune_tau(ctx, int(n), int(k), Lam0.data_ptr(), Lam1.data_ptr(), int(N), Lh.ctypes.data,
                                      float(alpha), ctypes.byref(p), int(sample_iters), U.data_ptr(), W.data_ptr(),
                                      Phi.data_ptr(), ctypes.byref(best), ctypes.byref(score), grid,
                                      ctypes.c_void_p(st))
    _native.check(rc, ctx)
    return best.value, score.value, list(grid)


def momt_solve_complex(Lam0, Lam1, L, alpha: float = 1.0, *, tau=None, mu=None, nu=None, max_iters: int = 2000,
                       check_every: int = 100, tol_gap: float = 0.0, tol_res: float = 0.0, init=None, engine="auto",
                       halo: int = 0, stream=None, u_norm: int = U_L2, w_norm: int = W_L2) -> MatrixSolution:
    """Complex Hermitian matrix OMT (Section 4's complex setting, Section 7.3 iteration) on
    the GPU, with the Frobenius norms ||U||_2, ||W||_2 (U_L2, W_L2) or the entrywise
    ||U||_1, ||W||_1 (U_L1, W_L1: sums of the entries' moduli).

    Lam0, Lam1: CUDA complex tensors [k*k, n, n] (k = 2 or 3) of Hermitian matrices.  L: [N, k, k]
    complex Hermitian (numpy, host).  Returns complex64 U [2, k*k, n, n], W [N, k*k, n, n],
    Phi [k*k, n, n].  The complex tensors are split into real and imaginary planes for the
    library and joined again on return (layout marshalling only).
    """
    import torch

    def planes(x):
        x = x.to(torch.complex64)
        return torch.stack([x.real, x.imag], dim=-4 if x.dim() >= 4 else 0).contiguous()

    def join(x):                                    # [..., 2, kk, n, n] -> complex [..., kk, n, n]
        return torch.complex(x.select(-4, 0), x.select(-4, 1))

    Lh = np.ascontiguousarray(np.asarray(L, dtype=np.complex128))
    N, k = Lh.shape[0], Lh.shape[1]
    kk, n = Lam0.shape[0], Lam0.shape[-1]
    if kk != k * k or Lam0.shape != Lam1.shape or Lam0.dim() != 3:
        raise ValueError("Lam0 and Lam1 must be [k*k, n, n] of one shape")
    dev = Lam0.device
    P0, P1 = planes(Lam0), planes(Lam1)
    if init is not None:
        U = torch.stack([planes(init[0][0]), planes(init[0][1])]).contiguous()
        W = torch.stack([planes(init[1][s]) for s in range(N)]).contiguous()
        Phi = planes(init[2])
    else:
        U = torch.empty((2, 2, kk, n, n), device=dev, dtype=torch.float32)
        W = torch.empty((N, 2, kk, n, n), device=dev, dtype=torch.float32)
        Phi = torch.empty((2, kk, n, n), device=dev, dtype=torch.float32)
    p = _params(tau, mu, nu, u_norm, w_norm, max_iters, check_every, tol_gap, tol_res, init is not None, engine, halo)
    res = _native.Result()
    st = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
    ctx = _native.context(dev.index if dev.index is not None else torch.cuda.current_device())
    Lri = np.ascontiguousarray(np.stack([Lh.real, Lh.imag], axis=-1))
    rc = _native.load().momt_solve_complex(ctx, int(n), int(k), P0.data_ptr(), P1.data_ptr(), int(N),
                                           Lri.ctypes.data, float(alpha), ctypes.byref(p), U.data_ptr(),
                                           W.data_ptr(), Phi.data_ptr(), ctypes.byref(res), ctypes.c_void_p(st))
    _native.check(rc, ctx)
    return MatrixSolution(join(U), join(W), join(Phi), res.as_dict())


def momt_solve3d(Lam0, Lam1, L, alpha: float = 1.0, *, tau=None, mu=None, nu=None, u_norm: int = U_L2,
                 w_norm: int = W_L1, max_iters: int = 2000, check_every: int = 100, tol_gap: float = 0.0,
                 tol_res: float = 0.0, init=None, stream=None, zc: int = 0) -> MatrixSolution:
    """Matrix OMT on an n x n x n grid (volumes of matrix densities, e.g. 3-D DTI).

    Lam0, Lam1: CUDA float32 tensors [k*k, n, n, n] of real symmetric matrices.  L: [N, k, k]
    (numpy, host).  Returns U [3, k*k, n, n, n] (U_x, U_y, U_z), W [N, k*k, n, n, n],
    Phi [k*k, n, n, n].  Default mu = 1/(48 tau (n-1)^2); zc > 0 sets the z planes per block.
    """
    import torch
    Lam0 = Lam0.contiguous().float()
    Lam1 = Lam1.contiguous().float()
    Lh = np.ascontiguousarray(L, dtype=np.float64)
    N, k = Lh.shape[0], Lh.shape[1]
    kk, n = Lam0.shape[0], Lam0.shape[-1]
    if kk != k * k or Lam0.dim() != 4 or Lam0.shape != Lam1.shape:
        raise ValueError("Lam0 and Lam1 must be [k*k, n, n, n] of one shape")
    dev = Lam0.device
    if init is not None:
        U, W, Phi = (x.detach().clone().contiguous().float() for x in init)
    else:
        U = torch.empty((3, kk, n, n, n), device=dev, dtype=torch.float32)
        W = torch.empty((N, kk, n, n, n), device=dev, dtype=torch.float32)
        Phi = torch.empty((kk, n, n, n), device=dev, dtype=torch.float32)
    p = _params(tau, mu, nu, u_norm, w_norm, max_iters, check_every, tol_gap, tol_res, init is not None, "stream",
                zc)
    res = _native.Result()
    st = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream.cuda_stream
    ctx = _native.context(dev.index if dev.index is not None else torch.cuda.current_device())
    rc = _native.load().momt_solve3d(ctx, int(n), int(k), Lam0.data_ptr(), Lam1.data_ptr(), int(N), Lh.ctypes.data,
                                     float(alpha), ctypes.byref(p), U.data_ptr(), W.data_ptr(), Phi.data_ptr(),
                                     ctypes.byref(res), ctypes.c_void_p(st))
    _native.check(rc, ctx)
    return MatrixSolution(U, W, Phi, res.as_dict())


def set_wait_policy(budget_ms: float = 0.0, drop_exchange: int = 0, device: int = 0):
    """Time limit of the resident engine's waits of one block on another (0: the
    default, 2 s) and, for tests, a halo exchange that block 0 skips on purpose
    (0: none); a wait that runs out ends the solve with BARRIER_TIMEOUT."""
    ctx = _native.context(device)
    _native.check(_native.load().vomt_set_wait_policy(ctx, float(budget_ms), int(drop_exchange)), ctx)


def history(device: int = 0):
    """Rows (primal, dual, rel_gap, rel_res, fp_resid, dual_infeas, iter, converged) of every
    convergence check of the last solve on `device`."""
    ctx = _native.context(device)
    lib = _native.load()
    rows = _native.check(lib.vomt_history(ctx, None, 0), ctx)
    out = np.zeros((rows, 8))
    if rows:
        _native.check(lib.vomt_history(ctx, out.ctypes.data_as(_native.P_double), rows), ctx)
    return out


class Batch:
    """A set of independent vector-OMT problems laid out in one device arena.

    problems: sequence of dicts with keys n, k, edges (node pairs), alpha, and
    optionally cost and tau.  `rho0`, `rho1`: per-problem arrays [k, n, n] (numpy or
    torch), copied into the arena.  After solve(), `u(q)`, `w(q)`, `phi(q)` are views
    of problem q's results in the arena.
    """

    def __init__(self, problems, rho0, rho1, device=0):
        import torch
        self.problems = list(problems)
        cnt = len(self.problems)
        self.graphs = [_native.GraphArg(p["k"], p.get("edges", []), p.get("cost")) for p in self.problems]
        self.inst = (_native.Instance * cnt)()
        for q, (p, g) in enumerate(zip(self.problems, self.graphs)):
            self.inst[q].n = int(p["n"])
            self.inst[q].graph = g.g
            self.inst[q].alpha = float(p.get("alpha", 1.0))
            self.inst[q].tau = float(p["tau"]) if p.get("tau") else 0.0
        total = ctypes.c_size_t()
        _native.check(_native.load().vomt_batch_layout(cnt, self.inst, ctypes.byref(total)))
        self.device = torch.device("cuda", device)
        self.arena = torch.zeros(int(total.value), dtype=torch.float32, device=self.device)
        for q, p in enumerate(self.problems):
            k, n = int(p["k"]), int(p["n"])
            nn = n * n
            off = int(self.inst[q].offset)
            r0 = torch.as_tensor(rho0[q], dtype=torch.float32).reshape(-1)
            r1 = torch.as_tensor(rho1[q], dtype=torch.float32).reshape(-1)
            self.arena[off:off + k * nn].copy_(r0)
            self.arena[off + k * nn:off + 2 * k * nn].copy_(r1)
        self.results = None

    def _view(self, q, start, planes):
        p = self.problems[q]
        n = int(p["n"])
        off = int(self.inst[q].offset) + start * n * n
        return self.arena[off:off + planes * n * n].view(planes, n, n)

    def u(self, q):
        k = int(self.problems[q]["k"])
        return self._view(q, 2 * k, 2 * k).view(2, k, *self._view(q, 0, 1).shape[1:])

    def w(self, q):
        k, l = int(self.problems[q]["k"]), self.graphs[q].tail.size
        return self._view(q, 4 * k, l)

    def phi(self, q):
        k, l = int(self.problems[q]["k"]), self.graphs[q].tail.size
        return self._view(q, 4 * k + l, k)

    def solve(self, *, max_iters=2000, check_every=100, tol_gap=0.0, tol_res=0.0, tau=None, u_norm=U_L12,
              w_norm=W_L1, warm_start=False, stream=None, path="auto", eps=0.0):
        """All problems through vomt_solve_batched.  path: "auto" (the tuned or
        estimated faster path), "queue" (one thread block per problem, one persistent
        launch, CUDA-graph captured on a non-default stream) or "grouped" (waves of
        equal-shape problems, each spread over a group of SMs).  Returns the overall
        status; per-problem results are in self.results."""
        import torch
        engine = {"auto": "batched", "queue": "stream", "grouped": "resident"}[path]
        p = _params(tau, None, None, u_norm, w_norm, max_iters, check_every, tol_gap, tol_res, warm_start, engine,
                    eps=eps)
        res = (_native.Result * len(self.problems))()
        st = (torch.cuda.current_stream(self.device) if stream is None else stream).cuda_stream
        ctx = _native.context(self.device.index)
        rc = _native.load().vomt_solve_batched(ctx, len(self.problems), self.inst, self.arena.data_ptr(),
                                               ctypes.byref(p), res, ctypes.c_void_p(st))
        _native.check(rc, ctx)
        self.results = [r.as_dict() for r in res]
        return rc

    def tune_tau(self, sample_iters=1000, **kw):
        """Per-problem dual step tau (vomt_batch_tune_tau): the whole batch runs once per
        grid point tau_paper(n) * 10^((j-1)/2); every problem keeps its best, which is
        stored as its tau for later solves.  Returns (taus, scores)."""
        p = _params(None, None, None, kw.get("u_norm", U_L12), kw.get("w_norm", W_L1), sample_iters, sample_iters,
                    0.0, 0.0, False, "batched", eps=kw.get("eps", 0.0))
        cnt = len(self.problems)
        taus = (ctypes.c_double * cnt)()
        scores = (ctypes.c_double * cnt)()
        ctx = _native.context(self.device.index)
        _native.check(_native.load().vomt_batch_tune_tau(ctx, cnt, self.inst, self.arena.data_ptr(), ctypes.byref(p),
                                                         int(sample_iters), taus, scores), ctx)
        for q in range(cnt):
            self.inst[q].tau = taus[q]
            self.problems[q]["tau"] = taus[q]
        return list(taus), list(scores)

    def tune(self, sample_iters=50, **kw):
        """Time the one-block-per-problem path with 128 / 256 / 512 threads per block and
        the grouped path on `sample_iters` iterations; keep the fastest on this device's
        context.  Returns (best thread count, {128: ms, 256: ms, 512: ms, "grouped": ms
        or -1 where that path does not apply})."""
        p = _params(kw.get("tau"), None, None, kw.get("u_norm", U_L12), kw.get("w_norm", W_L1), sample_iters,
                    sample_iters, 0.0, 0.0, False, "batched")
        best = ctypes.c_int()
        ms = (ctypes.c_double * 4)()
        ctx = _native.context(self.device.index)
        _native.check(_native.load().vomt_batch_tune(ctx, len(self.problems), self.inst, self.arena.data_ptr(),
                                                     ctypes.byref(p), int(sample_iters), ctypes.byref(best), ms), ctx)
        return best.value, dict(zip((128, 256, 512, "grouped"), list(ms)))


def set_batch_threads(threads: int, device: int = 0):
    ctx = _native.context(device)
    _native.check(_native.load().vomt_batch_set_threads(ctx, int(threads)), ctx)
