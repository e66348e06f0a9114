"""GPU parity of the batched engine (many independent vector-OMT problems in one
persistent launch) against the FP64 oracle, problem by problem, and against the
single-problem GPU solver.  Tolerances as for vomt_solve: relative L2 <= 1e-3 on
phi and u, relative <= 1e-4 on the primal objective at a fixed iteration count."""
import numpy as np
import pytest

import oracle
from paper_1712_10279_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
V = pytest.importorskip("paper_1712_10279_gb300")


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _mixed(count, seed, sides=(2, 3, 5, 17, 32, 40), ks=(1, 2, 3, 5)):
    rng = np.random.default_rng(seed)
    probs, r0s, r1s = [], [], []
    for q in range(count):
        n = int(rng.choice(sides))
        k = int(rng.choice(ks))
        edges = S.random_connected_graph(rng, k, 0.6)
        r0 = rng.uniform(0.1, 1.0, (k, n, n)); r0 /= r0.sum()
        r1 = rng.uniform(0.1, 1.0, (k, n, n)); r1 /= r1.sum()
        if n >= 5:
            r0, r1 = S.blob_pair(n, k, seed=seed * 1000 + q)
        probs.append(dict(n=n, k=k, edges=edges, alpha=float(rng.uniform(0.3, 3.0))))
        r0s.append(r0.astype(np.float32))
        r1s.append(r1.astype(np.float32))
    return probs, r0s, r1s


def _check_against_oracle(B, probs, r0s, r1s, **kw):
    for q, p in enumerate(probs):
        ref = oracle.vomt_solve(r0s[q].astype(np.float64), r1s[q].astype(np.float64), p["edges"], p["alpha"], **kw)
        res = B.results[q]
        assert res["iters"] == ref["iters"], (q, res["iters"], ref["iters"])
        phi = B.phi(q).cpu().numpy().astype(np.float64)
        u = B.u(q).cpu().numpy().astype(np.float64)
        assert _rel(phi, ref["phi"]) <= 1e-3, q
        assert _rel(u, np.stack([ref["ux"], ref["uy"]])) <= 1e-3, q
        P = ref["metrics"]["primal"]
        if P > 0:
            assert abs(res["primal"] - P) <= 1e-4 * P, (q, res["primal"], P)
        else:
            assert res["primal"] == 0.0


PATHS = ["queue", "grouped"]


@pytest.mark.parametrize("path", PATHS)
def test_batched_mixed_problems_match_oracle(path):
    _dev()
    probs, r0s, r1s = _mixed(24, seed=1)
    B = V.Batch(probs, r0s, r1s)
    rc = B.solve(max_iters=300, check_every=100, path=path)
    assert rc == 0
    assert all(r["engine"] == "batched" for r in B.results)
    _check_against_oracle(B, probs, r0s, r1s, max_iters=300, check_every=100)


@pytest.mark.parametrize("path", PATHS)
def test_batched_per_instance_stopping(path):
    _dev()
    probs, r0s, r1s = _mixed(10, seed=2, sides=(12, 20, 28), ks=(1, 3))
    B = V.Batch(probs, r0s, r1s)
    B.solve(max_iters=20000, check_every=100, tol_gap=5e-3, tol_res=5e-3, path=path)
    for q, p in enumerate(probs):
        ref = oracle.vomt_solve(r0s[q].astype(np.float64), r1s[q].astype(np.float64), p["edges"], p["alpha"],
                                max_iters=20000, check_every=100, tol_gap=5e-3, tol_res=5e-3)
        r = B.results[q]
        assert abs(r["iters"] - ref["iters"]) <= 100, (q, r["iters"], ref["iters"])
        if ref["iters"] < 20000:
            assert r["status"] == 0 and r["rel_gap"] <= 5e-3 and r["rel_res"] <= 5e-3
    iters = {r["iters"] for r in B.results}
    assert len(iters) > 1          # instances stopped at different iterations


def test_batched_graph_replay_and_tuner():
    d = _dev()
    probs, r0s, r1s = _mixed(12, seed=3)
    B = V.Batch(probs, r0s, r1s)
    s = torch.cuda.Stream(device=d)
    B.solve(max_iters=200, check_every=50, stream=s, path="queue")          # captured
    first = [B.phi(q).clone() for q in range(len(probs))]
    B.solve(max_iters=200, check_every=50, stream=s, path="queue")          # replayed
    for q in range(len(probs)):
        assert torch.equal(first[q], B.phi(q))
    best, times = B.tune(sample_iters=30)
    assert best in (128, 256, 512) and all(t > 0 for t in times.values())
    B.solve(max_iters=200, check_every=50, stream=s, path="queue")          # new launch shape -> recaptured
    _check_against_oracle(B, probs, r0s, r1s, max_iters=200, check_every=50)


@pytest.mark.parametrize("on_side_stream", [False, True])
def test_grouped_path_runs_as_one_graph_replay(on_side_stream):
    """The grouped path's wave launches form one CUDA graph (captured on the caller's stream,
    or on the context's own stream when the caller uses the legacy default stream): every
    call reports the graph launch, the replay reproduces the captured solve bit for bit and
    equals the oracle, and new parameters recapture."""
    d = _dev()
    probs, r0s, r1s = _mixed(10, seed=8)
    B = V.Batch(probs, r0s, r1s)
    s = torch.cuda.Stream(device=d) if on_side_stream else None
    B.solve(max_iters=300, check_every=100, path="grouped", stream=s)        # captured
    assert all(r["variant"] == 1 for r in B.results)
    first = [B.phi(q).clone() for q in range(len(probs))]
    B.solve(max_iters=300, check_every=100, path="grouped", stream=s)        # replayed
    assert all(r["variant"] == 1 for r in B.results)
    for q in range(len(probs)):
        assert torch.equal(first[q], B.phi(q))
    _check_against_oracle(B, probs, r0s, r1s, max_iters=300, check_every=100)
    B.solve(max_iters=200, check_every=100, path="grouped", stream=s)        # new parameters
    assert all(r["variant"] == 1 and r["iters"] == 200 for r in B.results)
    _check_against_oracle(B, probs, r0s, r1s, max_iters=200, check_every=100)


@pytest.mark.parametrize("path", PATHS)
def test_batched_matches_single_solves_at_config_sizes(path):
    """Problems drawn like the 512-problem mixed configuration (sides up to 256, k in {1, 3, 5},
    G(k, 0.6) graphs): each result equals the single-problem streaming solve on the GPU."""
    d = _dev()
    insts = S.batched_instances(count=10, seed=1004)
    probs = [dict(n=p["n"], k=p["k"], edges=p["edges"], alpha=1.0) for p in insts]
    r0s = [p["rho0"].astype(np.float32) for p in insts]
    r1s = [p["rho1"].astype(np.float32) for p in insts]
    assert max(p["n"] for p in probs) >= 128
    B = V.Batch(probs, r0s, r1s)
    B.solve(max_iters=250, check_every=125, path=path)
    if path == "grouped":
        assert max(r["blocks"] for r in B.results) > 1      # the large problems span several SMs
    for q, p in enumerate(probs):
        sol = V.solve(torch.from_numpy(r0s[q]).to(d), torch.from_numpy(r1s[q]).to(d), p["edges"], 1.0,
                      max_iters=250, check_every=125, engine="stream")
        assert _rel(B.phi(q).cpu().numpy(), sol.phi.cpu().numpy()) <= 1e-5
        assert abs(B.results[q]["primal"] - sol.result["primal"]) <= 1e-6 * max(sol.result["primal"], 1e-30)


def test_batched_reports_bad_instance():
    _dev()
    probs, r0s, r1s = _mixed(6, seed=4)
    r1s[3] = 1.05 * r1s[3]
    B = V.Batch(probs, r0s, r1s)
    with pytest.raises(V.VomtError) as e:
        B.solve(max_iters=10)
    assert e.value.status == -2 and "instance 3" in str(e.value)
