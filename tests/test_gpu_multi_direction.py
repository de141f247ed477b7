"""HVPs along several directions at the same gates (hvp_hvp_multi): with
HVP_MULTI_DIR the directions run through the sweep in pairs (states,
co-states and E shared, tangents per direction); checked against the FP64
oracle and against one-direction sweeps."""
import numpy as np
import pytest

from common import rel
from oracle import oracle
from paper_2604_20384_gb300 import native
from paper_2604_20384_gb300.inputs import make_workload, random_direction

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _dirs(w, count, seed):
    return np.stack([w.V] + [random_direction(w.K, w.G, seed=seed + i) for i in range(count - 1)])


@pytest.mark.parametrize("window,riemannian,frobenius", [(10, False, False), (11, False, False), (9, True, False),
                                                         (10, False, True)])
def test_direction_pairs_match_oracle(window, riemannian, frobenius):
    n, L, ns = 14, 8, 16
    w = make_workload(n, L, ns, seed=51)
    Vs = _dirs(w, 3, 90)                     # one pair and one single direction
    phi = oracle.reference_states(n, L, w.Uref, w.psi1q)
    key_g, key_h = ("grad_r", "hvp_r") if riemannian else ("grad", "hvp")
    if frobenius:
        key_g, key_h = "grad_f", "hvp_f"
    with native.Context(n, L, w.psi1q, w.Uref, window=window, riemannian=riemannian, multi_dir=True,
                        frobenius=frobenius) as ctx:
        info = ctx.plan_info()
        assert info["checkpoint_stride"] == 0 and info["window"] == window and info["passes"] > 1
        loss, grad, hv = ctx.hvp_multi(w.G, Vs)
        single = [ctx.hvp(w.G, V) for V in Vs]
    for d, V in enumerate(Vs):
        o = oracle.evaluate(n, L, w.G, V, w.psi1q, phi)
        if d == 0:
            lo = o["loss_f"] if frobenius else o["loss"]
            assert abs((1 - loss) - (1 - lo)) <= TOL * abs(1 - lo)
            assert rel(grad, o[key_g]) < TOL
        assert rel(hv[d], o[key_h]) < TOL, (d, rel(hv[d], o[key_h]))
        assert rel(hv[d], single[d][2]) < 2 * TOL
    assert np.array_equal(hv[2], single[2][2])   # the odd direction takes the one-direction sweep


def test_multi_direction_device_call_and_contexts_without_pairs():
    torch = pytest.importorskip("torch")
    n, L, ns = 12, 6, 8
    w = make_workload(n, L, ns, seed=52)
    Vs = _dirs(w, 4, 70)
    with native.Context(n, L, w.psi1q, w.Uref, multi_dir=True) as ctx:
        loss, grad, hv = ctx.hvp_multi(w.G, Vs)
        G_d = torch.from_numpy(w.G.view(np.float64).reshape(-1).copy()).cuda()
        V_d = torch.from_numpy(Vs.view(np.float64).reshape(-1).copy()).cuda()
        out = torch.zeros(4 * 32 * w.K, dtype=torch.float64, device="cuda")
        loss_d = torch.zeros(1, dtype=torch.float64, device="cuda")
        grad_d = torch.zeros(32 * w.K, dtype=torch.float64, device="cuda")
        ctx.hvp_multi_dev(G_d.data_ptr(), 4, V_d.data_ptr(), loss_d.data_ptr(), grad_d.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.complex128).reshape(4, w.K, 4, 4), hv)
        assert float(loss_d.cpu()[0]) == loss
        assert np.array_equal(grad_d.cpu().numpy().view(np.complex128).reshape(w.K, 4, 4), grad)
    # without HVP_MULTI_DIR every direction takes its own sweep: identical to hvp()
    with native.Context(n, L, w.psi1q, w.Uref) as ctx:
        loss1, grad1, hv1 = ctx.hvp_multi(w.G, Vs)
        for d, V in enumerate(Vs):
            assert np.array_equal(hv1[d], ctx.hvp(w.G, V)[2])
    for d in range(4):
        assert rel(hv[d], hv1[d]) < 2 * TOL


def test_direction_pairs_with_several_tiles_per_cta():
    # 16 qubits, 256 samples, 11-qubit windows: two tiles per CTA, so the
    # copy barriers' phases run on across tiles in the two-direction kernel
    n, L, ns = 16, 6, 256
    w = make_workload(n, L, ns, seed=53)
    Vs = _dirs(w, 2, 60)
    with native.Context(n, L, w.psi1q, w.Uref, multi_dir=True) as ctx:
        info = ctx.plan_info()
        assert info["tiles_per_cta"] > 1 and info["checkpoint_stride"] == 0
        r1 = ctx.hvp_multi(w.G, Vs)
        r2 = ctx.hvp_multi(w.G, Vs)
        single = [ctx.hvp(w.G, V) for V in Vs]
    assert r1[0] == r2[0] and np.array_equal(r1[2], r2[2])
    for d in range(2):
        assert rel(r1[2][d], single[d][2]) < 2 * TOL
    assert rel(r1[1], single[0][1]) < 2 * TOL


def test_expired_pair_copy_wait_is_reported():
    n, L, ns = 10, 6, 2
    w = make_workload(n, L, ns, seed=54)
    Vs = _dirs(w, 2, 40)
    phi = oracle.reference_states(n, L, w.Uref, w.psi1q)
    with native.Context(n, L, w.psi1q, w.Uref, window=8, multi_dir=True) as ctx:
        ctx.cache_wait_test(16, 1000)
        with pytest.raises(native.HVPError) as e:
            ctx.hvp_multi(w.G, Vs)
        assert e.value.code == native.HVP_ETIMEOUT
        ctx.cache_wait_test(0, 0)
        loss, grad, hv = ctx.hvp_multi(w.G, Vs)
    for d, V in enumerate(Vs):
        o = oracle.evaluate(n, L, w.G, V, w.psi1q, phi)
        assert rel(hv[d], o["hvp"]) < TOL
