"""Host-side tests of the C ABI: the library builds and loads, exports every
symbol include/vomt.h declares, and its host-only routines (step sizes,
argument checks) behave as documented.  No GPU needed."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_1712_10279_gb300 as V
from paper_1712_10279_gb300 import _native
from paper_1712_10279_gb300 import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.startswith("VOMT")))


def test_library_exports_every_declared_symbol():
    lib = _native.load()
    declared = _declared_functions()
    assert "vomt_solve" in declared and len(declared) >= 9
    out = subprocess.run(["nm", "-D", "--defined-only", _native.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    for n in declared:
        assert hasattr(lib, n)
        assert n in _native.SIGNATURES, "binding lacks a signature for %s" % n


@pytest.mark.parametrize("n,k,edges", [(32, 3, S.COMPLETE_K3), (256, 3, S.COMPLETE_K3), (64, 5, S.complete_graph(5)),
                                       (100, 4, [(0, 1), (1, 2), (2, 3)]), (17, 1, [])])
def test_step_sizes_match_oracle(n, k, edges):
    mu, nu, tau, lm = V.step_sizes(n, k, edges)
    lm_o = oracle.graph_lmax(k, edges) if edges else 0.0
    assert lm == pytest.approx(lm_o, rel=1e-12, abs=1e-14)
    mu_o, nu_o = oracle.step_sizes(n, tau, lm_o, bool(edges))
    assert mu == pytest.approx(mu_o, rel=1e-14)
    if edges:
        assert nu == pytest.approx(nu_o, rel=1e-12)
    assert tau == oracle.default_tau_vector(n)


def test_step_sizes_with_costs_and_random_graphs():
    rng = np.random.default_rng(0)
    for _ in range(20):
        k = int(rng.integers(2, 9))
        edges = S.random_connected_graph(rng, k, 0.5)
        cost = rng.uniform(0.3, 3.0, len(edges))
        _, _, _, lm = V.step_sizes(50, k, edges, cost=cost)
        assert lm == pytest.approx(oracle.graph_lmax(k, edges, cost), rel=1e-10)


def test_graph_errors_are_reported():
    with pytest.raises(V.VomtError) as e:
        V.step_sizes(32, 3, [(0, 1)])                    # node 2 unreachable
    assert e.value.status == -4
    with pytest.raises(V.VomtError) as e:
        V.step_sizes(32, 3, [(0, 1), (1, 1), (1, 2)])    # self loop
    assert e.value.status == -4
    with pytest.raises(V.VomtError) as e:
        V.step_sizes(32, 3, [(0, 1), (1, 0), (1, 2)])    # repeated edge
    assert e.value.status == -4
    with pytest.raises(V.VomtError) as e:
        V.step_sizes(32, 9, S.complete_graph(9))         # more channels than the limit
    assert e.value.status == -1
    with pytest.raises(V.VomtError):
        V.step_sizes(1, 3, S.COMPLETE_K3)


def test_status_strings():
    lib = _native.load()
    for code in list(_native.STATUS_NAMES):
        assert lib.vomt_status_str(code)
    p = _native.Params()
    lib.vomt_default_params(p)
    assert p.max_iters == 2000 and p.check_every == 100 and p.u_norm == 0 and p.w_norm == 0


def test_matrix_step_sizes_match_oracle():
    L = S.paper_L()
    mu, nu, tau, lm, gap = V.momt_step_sizes(128, L)
    assert lm == pytest.approx(oracle.quantum_lmax(L), rel=1e-10)
    assert gap == pytest.approx(oracle.quantum_sym_gap(L), rel=1e-8)
    assert tau == oracle.default_tau_matrix(128)
    mu_o, nu_o = oracle.step_sizes(128, tau, oracle.quantum_lmax(L), True)
    assert mu == pytest.approx(mu_o, rel=1e-14) and nu == pytest.approx(nu_o, rel=1e-10)
    for seed in range(5):
        Lr = S.random_L(3, 3, seed=seed)
        _, _, _, lm, gap = V.momt_step_sizes(64, Lr)
        assert lm == pytest.approx(oracle.quantum_lmax(Lr), rel=1e-10)
        assert gap == pytest.approx(oracle.quantum_sym_gap(Lr), rel=1e-7)
    L2 = S.random_L(2, 2, seed=3)
    _, _, _, lm, _ = V.momt_step_sizes(64, L2)
    assert lm == pytest.approx(oracle.quantum_lmax(L2), rel=1e-10)


def test_matrix_kernel_assumption_rejected():
    with pytest.raises(V.VomtError) as e:
        V.momt_step_sizes(32, np.diag([1.0, 1.0, 0.0])[None])
    assert e.value.status == -5
    with pytest.raises(V.VomtError) as e:
        V.momt_step_sizes(32, np.array([[[1.0, 2.0, 0], [0, 1, 0], [0, 0, 3]]]))   # not symmetric
    assert e.value.status == -1
