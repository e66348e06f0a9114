"""Differentiable transport costs (torch.autograd.Function wrappers).

``transport_cost`` is the optimal value V(rho0, rho1) of vector OMT (eq. vomt),
solved on the GPU; its backward is the envelope gradient computed by the CUDA
kernel behind ``vomt_backward`` (dV/drho1 = phi*, dV/drho0 = -phi*, centred;
dV/dalpha = sum ||w*||).  ``unrolled_cost`` is J_T, the primal objective after T
iterations from zero, whose backward runs the reverse-mode kernels behind
``vomt_unrolled_grad`` (checkpoints every ``ckpt`` iterations).  The Python
here only marshals tensors; every step runs in the library.
"""
from __future__ import annotations

import ctypes

import torch

from . import _native
from . import Batch, solve, _params, U_L12, W_L1


def _alpha_tensor(alpha, batch, device):
    if isinstance(alpha, torch.Tensor):
        a = alpha.detach().to(device=device, dtype=torch.float64).reshape(-1)
        return a.expand(batch) if a.numel() == 1 else a
    return torch.full((batch,), float(alpha), dtype=torch.float64, device=device)


class _TransportCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, rho1, alpha, edges, kw):
        squeeze = rho0.dim() == 3
        r0 = rho0.detach().reshape(-1, *rho0.shape[-3:]).float().contiguous()
        r1 = rho1.detach().reshape(-1, *rho1.shape[-3:]).float().contiguous()
        B, k, n = r0.shape[0], r0.shape[1], r0.shape[-1]
        alphas = _alpha_tensor(alpha, B, r0.device).cpu().tolist()
        w_norm = kw.get("w_norm", W_L1)
        taus = kw.get("taus")             # optional per-problem dual steps (e.g. from Batch.tune_tau)
        kw = {x: v for x, v in kw.items() if x != "taus"}
        if B == 1 or kw.get("engine") != "batched":
            costs, phis, ws = [], [], []
            for q in range(B):
                qkw = dict(kw, tau=taus[q]) if taus is not None else kw
                sol = solve(r0[q], r1[q], edges, alphas[q], **qkw)
                costs.append(sol.result["primal"])
                phis.append(sol.phi)
                ws.append(sol.w)
            phi = torch.stack(phis)
            w = torch.stack(ws)
        else:
            skw = {x: kw[x] for x in ("max_iters", "check_every", "tol_gap", "tol_res", "tau", "u_norm", "w_norm")
                   if x in kw}
            probs = [dict(n=n, k=k, edges=edges, alpha=alphas[q], tau=None if taus is None else taus[q])
                     for q in range(B)]
            bt = Batch(probs, list(r0), list(r1), device=r0.device.index or 0)
            bt.solve(**skw)
            costs = [r["primal"] for r in bt.results]
            phi = torch.stack([bt.phi(q) for q in range(B)])
            w = torch.stack([bt.w(q) for q in range(B)])
        ctx.save_for_backward(phi.contiguous(), w.contiguous())
        ashape = tuple(alpha.shape) if isinstance(alpha, torch.Tensor) else None
        ctx.meta = (B, n, k, len(edges), w_norm, squeeze, ashape, rho0.dtype)
        out = torch.tensor(costs, dtype=torch.float64, device=rho0.device)
        return out[0] if squeeze else out

    @staticmethod
    def backward(ctx, grad):
        phi, w = ctx.saved_tensors
        B, n, k, l, w_norm, squeeze, ashape, dtype = ctx.meta
        g = grad.detach().reshape(-1).to(torch.float32).expand(B).contiguous()
        d0 = torch.empty((B, k, n, n), device=phi.device, dtype=torch.float32)
        d1 = torch.empty_like(d0)
        da = torch.empty((B,), device=phi.device, dtype=torch.float32)
        cctx = _native.context(phi.device.index or 0)
        st = torch.cuda.current_stream(phi.device).cuda_stream
        rc = _native.load().vomt_backward(cctx, B, n, 0, k, l, w_norm, phi.data_ptr(), w.data_ptr() if l else None,
                                          g.data_ptr(), d0.data_ptr(), d1.data_ptr(), da.data_ptr(),
                                          ctypes.c_void_p(st))
        _native.check(rc, cctx)
        if squeeze:
            d0, d1 = d0[0], d1[0]
        dalpha = None
        if ashape is not None:
            # one alpha shared by the whole batch collects every problem's derivative
            dalpha = (da.double().sum() if int(torch.Size(ashape).numel()) == 1 else da.double()).reshape(ashape)
        return d0.to(dtype), d1.to(dtype), dalpha, None, None


def transport_cost(rho0, rho1, edges, alpha=1.0, **solve_kw):
    """V(rho0, rho1) by vomt_solve (or the batched engine for [B, k, n, n] inputs with
    engine="batched"); differentiable in rho0, rho1 and a tensor alpha."""
    return _TransportCost.apply(rho0, rho1, alpha, list(edges), dict(solve_kw))


class _UnrolledCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, rho1, alpha, edges, T, ckpt, kw):
        r0 = rho0.detach().float().contiguous()
        r1 = rho1.detach().float().contiguous()
        a = float(alpha.detach().reshape(-1)[0]) if isinstance(alpha, torch.Tensor) else float(alpha)
        sol = solve(r0, r1, edges, a, max_iters=T, check_every=T, engine="stream",
                    **{x: kw[x] for x in ("tau", "w_norm") if x in kw})
        ctx.save_for_backward(r0, r1)
        ctx.meta = (a, list(edges), T, ckpt, dict(kw), isinstance(alpha, torch.Tensor), rho0.dtype)
        return torch.tensor(sol.result["primal"], dtype=torch.float64, device=rho0.device)

    @staticmethod
    def backward(ctx, grad):
        r0, r1 = ctx.saved_tensors
        a, edges, T, ckpt, kw, alpha_is_tensor, dtype = ctx.meta
        k, n = r0.shape[0], r0.shape[-1]
        garg = _native.GraphArg(k, edges, kw.get("cost"))
        p = _params(kw.get("tau"), None, None, U_L12, kw.get("w_norm", W_L1), T, T, 0.0, 0.0, False, "stream")
        d0 = torch.empty_like(r0)
        d1 = torch.empty_like(r1)
        da, J = ctypes.c_double(), ctypes.c_double()
        cctx = _native.context(r0.device.index or 0)
        st = torch.cuda.current_stream(r0.device).cuda_stream
        rc = _native.load().vomt_unrolled_grad(cctx, int(n), r0.data_ptr(), r1.data_ptr(), garg.ref, a,
                                               ctypes.byref(p), int(T), int(ckpt), float(grad.item()),
                                               d0.data_ptr(), d1.data_ptr(), ctypes.byref(da), ctypes.byref(J),
                                               ctypes.c_void_p(st))
        _native.check(rc, cctx)
        dalpha = torch.tensor(da.value, dtype=torch.float64, device=r0.device) if alpha_is_tensor else None
        return d0.to(dtype), d1.to(dtype), dalpha, None, None, None, None


def unrolled_cost(rho0, rho1, edges, alpha=1.0, T=200, ckpt=20, **kw):
    """J_T = P(u^T, w^T) after T iterations from zero; backward by reverse mode with
    checkpoints every `ckpt` iterations (vomt_unrolled_grad)."""
    return _UnrolledCost.apply(rho0, rho1, alpha, list(edges), int(T), int(ckpt), dict(kw))


def unrolled_grad(rho0, rho1, edges, alpha=1.0, T=200, ckpt=20, tau=None, w_norm=W_L1, cost=None):
    """Direct call of vomt_unrolled_grad: returns (J_T, dJ/drho0, dJ/drho1, dJ/dalpha)."""
    r0 = rho0.detach().float().contiguous()
    r1 = rho1.detach().float().contiguous()
    k, n = r0.shape[0], r0.shape[-1]
    garg = _native.GraphArg(k, edges, cost)
    p = _params(tau, None, None, U_L12, w_norm, T, T, 0.0, 0.0, False, "stream")
    d0, d1 = torch.empty_like(r0), torch.empty_like(r1)
    da, J = ctypes.c_double(), ctypes.c_double()
    cctx = _native.context(r0.device.index or 0)
    st = torch.cuda.current_stream(r0.device).cuda_stream
    _native.check(_native.load().vomt_unrolled_grad(cctx, int(n), r0.data_ptr(), r1.data_ptr(), garg.ref,
                                                    float(alpha), ctypes.byref(p), int(T), int(ckpt), 1.0,
                                                    d0.data_ptr(), d1.data_ptr(), ctypes.byref(da),
                                                    ctypes.byref(J), ctypes.c_void_p(st)), cctx)
    return J.value, d0, d1, da.value
