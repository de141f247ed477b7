"""Batched uneven circuits (one persistent launch per call) against the FP64
oracle and against single-circuit contexts."""
import numpy as np
import pytest

from common import oracle_parallel, rel
from oracle import oracle
from paper_2604_20384_gb300 import native
from paper_2604_20384_gb300.inputs import make_workload, uneven_batch_shapes

pytestmark = pytest.mark.gpu
TOL = 1e-5

SMALL = [(5, 4, 7), (9, 6, 19), (12, 5, 3), (13, 7, 5), (14, 9, 4), (8, 20, 33), (2, 1, 3), (16, 5, 2)]


def _small_batch():
    ws = [make_workload(n, L, ns, seed=100 + i) for i, (n, L, ns) in enumerate(SMALL)]
    return ws, [(w.n, w.n_layers, w.psi1q, w.Uref) for w in ws]


@pytest.mark.parametrize("riemannian,graphs", [(False, True), (True, False)])
def test_small_uneven_batch_matches_oracle(riemannian, graphs):
    ws, circuits = _small_batch()
    with native.BatchContext(circuits, riemannian=riemannian, graphs=graphs) as b:
        loss, grads, hvps = b.hvp([w.G for w in ws], [w.V for w in ws])
        T, Om = b.get("T"), b.get("Omega")
        l2, g2 = b.loss_grad([w.G for w in ws])
    for i, w in enumerate(ws):
        phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)
        o = oracle.evaluate(w.n, w.n_layers, w.G, w.V, w.psi1q, phi)
        kg, kh = ("grad_r", "hvp_r") if riemannian else ("grad", "hvp")
        assert abs((1 - loss[i]) - (1 - o["loss"])) <= TOL * (1 - o["loss"]) + 1e-13, i
        assert rel(grads[i], o[kg]) < TOL, (i, rel(grads[i], o[kg]))
        assert rel(hvps[i], o[kh]) < TOL, (i, rel(hvps[i], o[kh]))
        assert rel(T[i], o["T"]) < TOL and rel(Om[i], o["Omega"]) < TOL
        assert abs(l2[i] - loss[i]) < 1e-12
        assert rel(g2[i], o[kg]) < TOL


@pytest.mark.parametrize("window,autotune", [(10, False), (0, True)])
def test_batch_window_widths_and_autotune(window, autotune):
    # circuits above 12 qubits run window passes of `window` qubits (or the
    # autotuned width); results must not depend on it
    ws, circuits = _small_batch()
    with native.BatchContext(circuits, window=window, autotune=autotune) as b:
        info = b.plan_info()
        loss, grads, hvps = b.hvp([w.G for w in ws], [w.V for w in ws])
    if window:
        assert info["window"] == window
    else:
        assert info["window"] in (10, 11, 12)
    for i, w in enumerate(ws):
        phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)
        o = oracle.evaluate(w.n, w.n_layers, w.G, w.V, w.psi1q, phi)
        assert abs((1 - loss[i]) - (1 - o["loss"])) <= TOL * (1 - o["loss"]) + 1e-13, i
        assert rel(grads[i], o["grad"]) < TOL, (i, rel(grads[i], o["grad"]))
        assert rel(hvps[i], o["hvp"]) < TOL, (i, rel(hvps[i], o["hvp"]))


@pytest.mark.parametrize("count", [1, 3])
def test_odd_number_of_circuits(count):
    # the per-gate result blocks start after one loss per circuit: with an odd
    # count they must still be 16-byte aligned (double2 arrays)
    ws, circuits = _small_batch()
    ws, circuits = ws[:count], circuits[:count]
    with native.BatchContext(circuits) as b:
        loss, grads, hvps = b.hvp([w.G for w in ws], [w.V for w in ws])
    for i, w in enumerate(ws):
        phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)
        o = oracle.evaluate(w.n, w.n_layers, w.G, w.V, w.psi1q, phi)
        assert abs((1 - loss[i]) - (1 - o["loss"])) <= TOL * (1 - o["loss"]) + 1e-13, i
        assert rel(grads[i], o["grad"]) < TOL and rel(hvps[i], o["hvp"]) < TOL


def test_expired_chain_wait_is_reported_and_context_stays_usable():
    # every chain wait asks for a phase that never finishes: the first wait
    # gives up after 10^4 sleeps of 200 ns, the call reports HVP_ETIMEOUT, and
    # after restoring the normal waits the same context evaluates correctly
    ws, circuits = _small_batch()
    with native.BatchContext(circuits) as b:
        b.wait_test(1, 10000)
        with pytest.raises(native.HVPError) as e:
            b.hvp([w.G for w in ws], [w.V for w in ws])
        assert e.value.code == native.HVP_ETIMEOUT
        b.wait_test(0)
        loss, grads, hvps = b.hvp([w.G for w in ws], [w.V for w in ws])
    for i, w in enumerate(ws):
        phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)
        o = oracle.evaluate(w.n, w.n_layers, w.G, w.V, w.psi1q, phi)
        assert rel(hvps[i], o["hvp"]) < TOL, (i, rel(hvps[i], o["hvp"]))


def test_full_uneven_batch_matches_single_contexts_and_oracle():
    # 64 circuits, n ~ U{8..16}, L ~ U{4..20}, N_s log-uniform in [32, 512]
    shapes = uneven_batch_shapes(64, seed=0)
    ws = [make_workload(n, L, ns, s) for (n, L, ns, s) in shapes]
    with native.BatchContext([(w.n, w.n_layers, w.psi1q, w.Uref) for w in ws]) as b:
        info = b.plan_info()
        assert info["circuits"] == 64
        r1 = b.hvp([w.G for w in ws], [w.V for w in ws])
        r2 = b.hvp([w.G for w in ws], [w.V for w in ws])
    assert np.array_equal(r1[0], r2[0])
    assert all(np.array_equal(a, c) for a, c in zip(r1[2], r2[2]))
    assert np.all((r1[0] >= 0) & (r1[0] <= 1))
    # circuits checked against single-circuit contexts and against the FP64
    # oracle: the largest n, the smallest n, the largest N_s, and five more at
    # random among those the oracle evaluates in a few seconds on the host
    cost = [(1 << w.n) * w.n_samples * w.K for w in ws]
    light = [i for i in range(64) if cost[i] < 5e8]
    picks = sorted({int(np.argmax([w.n for w in ws])), int(np.argmin([w.n for w in ws])),
                    int(np.argmax([w.n_samples for w in ws]))} |
                   {int(i) for i in np.random.default_rng(3).choice(light, 5, replace=False)})
    for i in picks:
        w = ws[i]
        with native.Context(w.n, w.n_layers, w.psi1q, w.Uref) as c:
            loss, g, h = c.hvp(w.G, w.V)
        assert abs((1 - r1[0][i]) - (1 - loss)) <= TOL * (1 - loss) + 1e-13, i
        assert rel(r1[1][i], g) < TOL, (i, w.n)
        assert rel(r1[2][i], h) < TOL, (i, w.n)
        phi, o = oracle_parallel(w)
        assert abs((1 - r1[0][i]) - (1 - o["loss"])) <= TOL * (1 - o["loss"]) + 1e-13, i
        assert rel(r1[1][i], o["grad"]) < TOL, (i, w.n, rel(r1[1][i], o["grad"]))
        assert rel(r1[2][i], o["hvp"]) < TOL, (i, w.n, rel(r1[2][i], o["hvp"]))
