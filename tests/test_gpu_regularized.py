"""GPU parity of the quadratically regularised problem (the paper's concluding section:
eps (||u||_2^2 + ||w||_2^2) added to the objective) against the FP64 oracle.

At a fixed iteration count the iterates match elementwise (relative L2 <= 1e-3, primal
<= 1e-4), for both engines and every norm pair.  Because the regularised problem has a
unique solution, converged GPU and oracle solutions are also compared elementwise."""
import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
V = pytest.importorskip("paper_1712_10279_gb300")
N = pytest.importorskip("paper_1712_10279_gb300._native")

K3 = S.COMPLETE_K3
ENGINES = ["resident", "stream"]


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _t(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(_dev())


def _f64(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("eps", [0.3, 5.0])
@pytest.mark.parametrize("u_norm,w_norm", [(0, 0), (1, 1), (2, 0)])
def test_fixed_iterations_match_oracle(engine, eps, u_norm, w_norm):
    r0, r1 = S.blob_pair(37, 3, seed=91)
    kw = dict(max_iters=600, check_every=200, u_norm=u_norm, w_norm=w_norm, eps=eps)
    sol = V.solve(_t(r0), _t(r1), K3, 0.8, engine=engine, **kw)
    ref = oracle.vomt_solve(_f64(r0), _f64(r1), K3, 0.8, **kw)
    assert sol.result["engine"] == engine
    u = sol.u.cpu().numpy().astype(np.float64)
    assert _rel(sol.phi.cpu().numpy().astype(np.float64), ref["phi"]) <= 1e-3
    assert _rel(u, np.stack([ref["ux"], ref["uy"]])) <= 1e-3
    assert _rel(sol.w.cpu().numpy().astype(np.float64), ref["w"]) <= 1e-3
    m = ref["metrics"]
    assert sol.result["primal"] == pytest.approx(m["primal"], rel=1e-4)
    assert sol.result["dual"] == pytest.approx(m["dual"], rel=1e-4, abs=1e-6 * abs(m["primal"]))
    assert sol.result["rel_res"] == pytest.approx(m["rel_res"], rel=1e-3)


@pytest.mark.parametrize("engine", ENGINES)
def test_converged_solution_is_the_oracle_solution(engine):
    """Unique optimum: the GPU stopped at gap and residual 1e-5 (about the FP32 floor) is
    close to the oracle's tightly converged solution.  (The oracle's own 1e-5 iterate is
    within 4e-6 of it, relative, on this case.)"""
    r0, r1 = S.blob_pair(20, 3, seed=92)
    kw = dict(tau=3.0, check_every=100, eps=2.0)
    sol = V.solve(_t(r0), _t(r1), K3, 1.0, engine=engine, max_iters=200000, tol_gap=1e-5, tol_res=1e-5, **kw)
    ref = oracle.vomt_solve(_f64(r0), _f64(r1), K3, 1.0, max_iters=100000, tol_gap=1e-9, tol_res=1e-9, **kw)
    assert sol.result["status"] == 0
    assert ref["metrics"]["rel_gap"] <= 1e-8 and ref["metrics"]["rel_res"] <= 1e-6
    u = sol.u.cpu().numpy().astype(np.float64)
    assert _rel(u, np.stack([ref["ux"], ref["uy"]])) <= 5e-4
    assert _rel(sol.w.cpu().numpy().astype(np.float64), ref["w"]) <= 5e-3
    assert sol.result["primal"] == pytest.approx(ref["metrics"]["primal"], rel=1e-5)


@pytest.mark.parametrize("path", ["queue", "grouped"])
def test_batched_regularised_matches_single_solves(path):
    d = _dev()
    insts = S.batched_instances(count=6, seed=93, sides=(24, 40, 64), ks=(1, 3))
    probs = [dict(n=p["n"], k=p["k"], edges=p["edges"], alpha=1.0) for p in insts]
    r0s = [p["rho0"].astype(np.float32) for p in insts]
    r1s = [p["rho1"].astype(np.float32) for p in insts]
    B = V.Batch(probs, r0s, r1s)
    B.solve(max_iters=300, check_every=100, path=path, eps=1.5)
    for q, p in enumerate(probs):
        ref = oracle.vomt_solve(_f64(r0s[q]), _f64(r1s[q]), p["edges"], 1.0, max_iters=300, check_every=100,
                                eps=1.5)
        assert _rel(B.phi(q).cpu().numpy().astype(np.float64), ref["phi"]) <= 1e-3
        assert B.results[q]["primal"] == pytest.approx(ref["metrics"]["primal"], rel=1e-4)
    assert d.type == "cuda"


def test_regularisation_arguments_are_checked():
    r0, r1 = S.blob_pair(12, 3, seed=94)
    with pytest.raises(N.VomtError) as e:
        V.solve(_t(r0), _t(r1), K3, 1.0, max_iters=10, eps=-1.0)
    assert e.value.status == -1
    A = pytest.importorskip("paper_1712_10279_gb300.autograd")
    lib = N.load()
    p = V._params(None, None, None, 0, 0, 10, 10, 0.0, 0.0, False, "stream", eps=1.0)
    g = N.GraphArg(3, K3)
    d0, d1 = _t(r0), _t(r1)
    out0, out1 = torch.empty_like(d0), torch.empty_like(d1)
    import ctypes
    da, J = ctypes.c_double(), ctypes.c_double()
    rc = lib.vomt_unrolled_grad(N.context(0), 12, d0.data_ptr(), d1.data_ptr(), g.ref, 1.0, ctypes.byref(p), 10, 5,
                                1.0, out0.data_ptr(), out1.data_ptr(), ctypes.byref(da), ctypes.byref(J), None)
    assert rc == -1
    assert A is not None
