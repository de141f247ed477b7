"""Fused-block tensor-core schedule (HVP_TENSOR) through the C ABI against the
FP64 oracle, element by element.

The schedule groups the gates into blocks of five neighbouring qubits (App.
D's block operator B and its tangent dB), applies each block as the real
GEMM [B ; dB] [psi | dpsi] on exact-integer bf16 slices of both operands on
tcgen05 (the block environments as a TF32 GEMM), and weights the co-states
by the overlaps so that block environments sum over samples. Bar: 1e-5 relative (Frobenius norm over all K blocks) for the
gradient and the HVP, the mean fidelity 1 - C relatively and C absolutely, as
for the other complex64 paths.
"""
import numpy as np
import pytest

from common import headline_oracle, rel
from oracle import oracle
from paper_2604_20384_gb300 import native
from paper_2604_20384_gb300.inputs import make_workload, random_direction

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _oracle(w, G=None, V=None, phi=None, threads=None):
    if phi is None:
        phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)
    o = oracle.evaluate(w.n, w.n_layers, w.G if G is None else G, w.V if V is None else V, w.psi1q, phi,
                        threads=threads)
    return o, phi


def _check(ctx, w, o, G=None, V=None, tol=TOL):
    loss, grad, hvp = ctx.hvp(w.G if G is None else G, w.V if V is None else V)
    F, Fo = 1 - loss, 1 - o["loss"]
    assert abs(F - Fo) <= tol * abs(Fo) + 1e-13, (F, Fo)
    assert abs(loss - o["loss"]) <= tol
    key_g, key_h = ("grad_r", "hvp_r") if ctx.riemannian else ("grad", "hvp")
    assert rel(grad, o[key_g]) < tol, rel(grad, o[key_g])
    assert rel(hvp, o[key_h]) < tol, rel(hvp, o[key_h])
    assert rel(ctx.get("T"), o["T"]) < tol
    assert rel(ctx.get("Omega"), o["Omega"]) < tol
    assert rel(ctx.get("grad_e"), o["grad"]) < tol
    assert rel(ctx.get("hvp_e"), o["hvp"]) < tol
    assert rel(ctx.get("grad_r"), o["grad_r"]) < tol
    assert rel(ctx.get("hvp_r"), o["hvp_r"]) < tol
    return loss, grad, hvp


@pytest.mark.parametrize("n,L,ns", [(5, 4, 3), (6, 3, 16), (7, 5, 2), (9, 6, 5), (10, 12, 9), (12, 8, 7),
                                    (13, 11, 3), (14, 7, 5), (16, 9, 3)])
def test_tensor_schedule_matches_oracle(n, L, ns):
    # one block (n = 5) up to many blocks at every block position; column
    # counts N_s * 2^(n-5) from 3 (a tile much wider than the data, tiles
    # spanning samples) to ragged multiples of the 64- and 128-column tiles
    w = make_workload(n, L, ns, seed=n * 7 + L)
    o, phi = _oracle(w)
    with native.Context(n, L, w.psi1q, w.Uref, tensor=True) as ctx:
        info = ctx.plan_info()
        assert info["window"] == 5 and info["passes"] == len(native.plan_blocks(n, L)[1])
        _check(ctx, w, o)


def test_tensor_loss_and_gradient_only_call():
    w = make_workload(11, 6, 4, seed=3)
    o, phi = _oracle(w)
    with native.Context(11, 6, w.psi1q, w.Uref, tensor=True) as ctx:
        loss, grad = ctx.loss_grad(w.G)
        assert abs(loss - o["loss"]) <= TOL
        assert rel(grad, o["grad"]) < TOL
        assert rel(ctx.get("T"), o["T"]) < TOL


def test_tensor_riemannian_and_near_solution():
    # near the solution every overlap is O(1) and the block environments'
    # diagonals are coherent sums over all amplitudes and samples (the case
    # where FP32 accumulation over long runs would lose digits)
    w = make_workload(13, 6, 8, seed=5, near_solution=0.1)
    o, phi = _oracle(w)
    with native.Context(13, 6, w.psi1q, w.Uref, tensor=True, riemannian=True) as ctx:
        _check(ctx, w, o)
    assert np.min(np.abs(o["T"])) > 0.3


def test_tensor_frobenius_cost():
    w = make_workload(12, 7, 6, seed=41)
    phi = oracle.reference_states(12, 7, w.Uref, w.psi1q)
    o = oracle.evaluate(12, 7, w.G, w.V, w.psi1q, phi)
    with native.Context(12, 7, w.psi1q, w.Uref, tensor=True, frobenius=True) as ctx:
        loss, grad, hvp = ctx.hvp(w.G, w.V)
        assert abs(loss - o["loss_f"]) <= TOL
        assert rel(grad, o["grad_f"]) < TOL and rel(hvp, o["hvp_f"]) < TOL
        assert rel(ctx.get("grad_r"), o["grad_fr"]) < TOL and rel(ctx.get("hvp_r"), o["hvp_fr"]) < TOL


def test_tensor_phi_given_and_non_unitary_gates():
    # finite differences evaluate G + h V (not unitary): the block recursion of
    # the environments uses G^-1, not G^dag
    w = make_workload(11, 5, 4, seed=9)
    phi = oracle.reference_states(11, 5, w.Uref, w.psi1q)
    G2 = w.G + 0.05 * w.V
    o = oracle.evaluate(11, 5, G2, w.V, w.psi1q, phi)
    with native.Context(11, 5, w.psi1q, phi, phi_given=True, tensor=True) as ctx:
        _check(ctx, w, o, G=G2)


def test_tensor_repeat_calls_graphs_and_hvp_symmetry():
    w = make_workload(12, 6, 5, seed=12)
    W = random_direction(w.K, w.G, seed=77)
    with native.Context(12, 6, w.psi1q, w.Uref, tensor=True) as a, \
            native.Context(12, 6, w.psi1q, w.Uref, tensor=True, graphs=False) as b:
        r1 = a.hvp(w.G, w.V)
        r2 = a.hvp(w.G, w.V)
        r3 = b.hvp(w.G, w.V)
        for x, y, z in zip(r1, r2, r3):   # fixed reduction order: bit-identical
            assert np.array_equal(np.asarray(x), np.asarray(y)) and np.array_equal(np.asarray(x), np.asarray(z))
        hv = r1[2]
        hw = a.hvp(w.G, W)[2]
        assert abs(np.real(np.vdot(W, hv)) - np.real(np.vdot(w.V, hw))) < 1e-5 * np.linalg.norm(hv) * np.linalg.norm(W)


def test_tensor_rejects_unsupported_configurations():
    w = make_workload(6, 3, 2, seed=0)
    for kw in (dict(precision="c128"), dict(multi_dir=True), dict(recompute=True), dict(unfused=True)):
        with pytest.raises(native.HVPError):
            native.Context(6, 3, w.psi1q, w.Uref, tensor=True, **kw)
    w4 = make_workload(4, 3, 2, seed=0)
    with pytest.raises(native.HVPError):
        native.Context(4, 3, w4.psi1q, w4.Uref, tensor=True)
    with native.Context(6, 3, w.psi1q, w.Uref, tensor=True) as ctx:
        ctx.hvp(w.G, w.V)
        with pytest.raises(native.HVPError):
            ctx.get("env")


def test_tensor_expired_wait_is_reported_and_context_stays_usable():
    # the waits for a tile's MMAs are bounded: with the tile barriers expecting
    # an arrival that never comes they give up after 1000 polls, the passes
    # stop (after their MMAs in flight complete) and the call reports
    # HVP_ETIMEOUT; restored, the same context evaluates correctly
    w = make_workload(12, 6, 8, seed=2)
    o, phi = _oracle(w)
    with native.Context(12, 6, w.psi1q, w.Uref, tensor=True) as ctx:
        ctx.cache_wait_test(16, 1000)
        with pytest.raises(native.HVPError) as e:
            ctx.hvp(w.G, w.V)
        assert e.value.code == native.HVP_ETIMEOUT
        ctx.cache_wait_test(0, 0)
        _check(ctx, w, o)


def test_tensor_headline_shape_against_oracle_on_all_samples():
    # n = 20, L = 16 (K = 152, 26 blocks), the benchmark's N_s = 64: the
    # sample-summed loss, gradient and HVP against the oracle run on all 64
    # samples
    w, phi, o = headline_oracle()
    with native.Context(20, 16, w.psi1q, w.Uref, tensor=True) as ctx:
        assert ctx.plan_info()["passes"] == 26
        _check(ctx, w, o)
        # the tangent-free kernels (a kernel of their own in the backward) at
        # 431 and 432 tiles per CTA: loss and gradient alone
        loss, grad = ctx.loss_grad(w.G)
        assert abs(loss - o["loss"]) <= TOL
        assert rel(grad, o["grad"]) < TOL
