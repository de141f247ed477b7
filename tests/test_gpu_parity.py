"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances (the bar of the benchmark plan): complex64 sweeps with FP64
accumulation within 1e-5 relative (Frobenius norm over all K blocks) for the
gradient and the HVP; the complex128 path within 1e-11. The loss is compared
as the mean fidelity F = 1 - C relatively (C is within 2^-n of 1 for random
circuits) and as C absolutely.
"""
import numpy as np
import pytest

from common import headline_oracle, rel
from oracle import oracle
from paper_2604_20384_gb300 import native
from paper_2604_20384_gb300.inputs import make_workload, random_direction

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c128": 1e-11}


def _oracle(w, G=None, V=None, phi=None, want_env=False):
    if phi is None:
        phi = oracle.reference_states(w.n, w.n_layers, w.Uref, w.psi1q)
    o = oracle.evaluate(w.n, w.n_layers, w.G if G is None else G, w.V if V is None else V, w.psi1q, phi,
                        want_env=want_env)
    return o, phi


def _check(ctx, w, o, tol, G=None, V=None):
    loss, grad, hvp = ctx.hvp(w.G if G is None else G, w.V if V is None else V)
    F, Fo = 1 - loss, 1 - o["loss"]
    assert abs(F - Fo) <= tol * abs(Fo) + 1e-13, (F, Fo)
    assert abs(loss - o["loss"]) <= max(tol, 1e-13)
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


@pytest.mark.parametrize("precision,unfused", [("c128", True), ("c64", False), ("c64", True)])
def test_small_brickwall_all_paths(precision, unfused):
    w = make_workload(6, 3, 16, seed=0)
    o, phi = _oracle(w)
    with native.Context(6, 3, w.psi1q, w.Uref, precision=precision, unfused=unfused) as ctx:
        _check(ctx, w, o, TOL[precision])


@pytest.mark.parametrize("precision", ["c128", "c64"])
def test_n12_precision_comparison(precision):
    w = make_workload(12, 8, 256, seed=0)
    o, phi = _oracle(w)
    with native.Context(12, 8, w.psi1q, w.Uref, precision=precision) as ctx:
        _check(ctx, w, o, TOL[precision])


@pytest.mark.parametrize("recompute", [False, True])
@pytest.mark.parametrize("n,L,ns,window", [(14, 7, 5, 10), (16, 9, 3, 12), (13, 11, 7, 8), (15, 6, 2, 9),
                                           (10, 12, 9, 6)])
def test_multi_pass_tiles_with_ragged_shapes(n, L, ns, window, recompute):
    # several passes, several tiles per sample, layouts permuted between
    # passes; both schedules (forward states cached before every gate, or
    # recomputed inside each pass from boundary checkpoints)
    w = make_workload(n, L, ns, seed=n + L)
    o, phi = _oracle(w)
    with native.Context(n, L, w.psi1q, w.Uref, window=window, recompute=recompute) as ctx:
        info = ctx.plan_info()
        assert info["passes"] > 1
        assert (info["checkpoint_stride"] == 0) == (not recompute)
        _check(ctx, w, o, TOL["c64"])


@pytest.mark.parametrize("threads,variant,recompute", [(256, 1, False), (256, 1, True), (256, 2, False),
                                                       (512, 1, False), (512, 2, False), (256, 3, False),
                                                       (512, 3, False), (128, 1, False), (128, 1, True)])
def test_kernel_variants_match_oracle(threads, variant, recompute):
    # every thread count and arithmetic form of the window-pass kernels (the
    # forward-cache schedule runs the scalar kernels at 128 and 256 threads;
    # the other forms recompute)
    w = make_workload(15, 9, 6, seed=44)
    o, phi = _oracle(w)
    with native.Context(15, 9, w.psi1q, w.Uref, window=11, threads=threads, variant=variant,
                        recompute=recompute) as ctx:
        info = ctx.plan_info()
        assert info["threads"] == threads and info["variant"] == variant and info["passes"] > 1
        cached = variant == 1 and threads in (128, 256) and not recompute
        assert (info["checkpoint_stride"] == 0) == cached
        _check(ctx, w, o, TOL["c64"])
        loss, grad = ctx.loss_grad(w.G)
        assert rel(grad, o["grad"]) < TOL["c64"]


def test_autotuned_context_matches_oracle():
    w = make_workload(14, 8, 6, seed=71)
    o, phi = _oracle(w)
    with native.Context(14, 8, w.psi1q, w.Uref, autotune=True) as ctx:
        info = ctx.plan_info()
        assert info["window"] in (10, 11, 12) and info["variant"] in (1, 2, 3) and info["threads"] in (128, 256)
        _check(ctx, w, o, TOL["c64"])


def test_loss_and_gradient_only_call():
    w = make_workload(14, 6, 4, seed=3)
    o, phi = _oracle(w)
    for prec, unf in (("c64", False), ("c128", True)):
        with native.Context(14, 6, w.psi1q, w.Uref, precision=prec, unfused=unf, window=10) as ctx:
            loss, grad = ctx.loss_grad(w.G)
            assert abs(loss - o["loss"]) <= TOL[prec]
            assert rel(grad, o["grad"]) < TOL[prec]
            assert rel(ctx.get("T"), o["T"]) < TOL[prec]


def test_riemannian_outputs_and_near_solution():
    w = make_workload(13, 6, 8, seed=5, near_solution=0.1)
    o, phi = _oracle(w)
    assert np.min(np.abs(o["T"])) > 0.3
    with native.Context(13, 6, w.psi1q, w.Uref, riemannian=True, window=10) as ctx:
        _check(ctx, w, o, TOL["c64"])


def test_phi_given_and_non_unitary_gates():
    w = make_workload(11, 5, 6, seed=8)
    rng = np.random.default_rng(1)
    Gn = w.G + 0.05 * (rng.standard_normal(w.G.shape) + 1j * rng.standard_normal(w.G.shape))
    o, phi = _oracle(w, G=Gn)
    for prec in ("c64", "c128"):
        with native.Context(11, 5, w.psi1q, phi, phi_given=True, precision=prec, window=8) as ctx:
            _check(ctx, w, o, TOL[prec], G=Gn)


def test_single_gate_and_single_sample():
    w = make_workload(2, 1, 1, seed=4)
    o, phi = _oracle(w)
    for prec in ("c64", "c128"):
        with native.Context(2, 1, w.psi1q, w.Uref, precision=prec) as ctx:
            _check(ctx, w, o, TOL[prec])


def test_checkpoint_stride_graphs_and_repeat_calls_are_bit_identical():
    w = make_workload(16, 14, 4, seed=9)
    o, phi = _oracle(w)
    results = []
    for stride, graphs in ((1, True), (2, True), (3, False), (100, True)):
        with native.Context(16, 14, w.psi1q, w.Uref, window=9, checkpoint_stride=stride, graphs=graphs) as ctx:
            info = ctx.plan_info()
            assert info["passes"] >= 4
            r1 = ctx.hvp(w.G, w.V)
            r2 = ctx.hvp(w.G, w.V)
            assert r1[0] == r2[0] and np.array_equal(r1[1], r2[1]) and np.array_equal(r1[2], r2[2])
            results.append(r1)
    for r in results[1:]:
        assert r[0] == results[0][0] and np.array_equal(r[1], results[0][1]) and np.array_equal(r[2], results[0][2])
    assert rel(results[0][2], o["hvp"]) < TOL["c64"]


def test_per_sample_environments_match_oracle():
    w = make_workload(12, 5, 3, seed=12)
    o, phi = _oracle(w, want_env=True)
    with native.Context(12, 5, w.psi1q, w.Uref, window=8) as ctx:
        ctx.hvp(w.G, w.V)
        E, DE = ctx.get("env")
    assert rel(E, o["E"]) < TOL["c64"]
    assert rel(DE, o["DE"]) < TOL["c64"]


def test_hvp_symmetry_on_gpu():
    w = make_workload(12, 6, 8, seed=21)
    W = random_direction(w.K, w.G, seed=5)
    with native.Context(12, 6, w.psi1q, w.Uref) as ctx:
        hv = ctx.hvp(w.G, w.V)[2]
        hw = ctx.hvp(w.G, W)[2]
    a = np.real(np.vdot(W.ravel(), hv.ravel()))
    b = np.real(np.vdot(w.V.ravel(), hw.ravel()))
    assert abs(a - b) < 1e-5 * max(abs(a), 1e-3)


def test_errors_are_reported_not_raised_on_device():
    w = make_workload(8, 3, 2, seed=2)
    with native.Context(8, 3, w.psi1q, w.Uref) as ctx:
        G = w.G.copy()
        G[1] = 0.0                               # singular gate: no inverse
        with pytest.raises(native.HVPError) as e:
            ctx.hvp(G, w.V)
        assert e.value.code == native.HVP_ENONFINITE
        G = w.G.copy()
        G[0, 0, 0] = np.nan
        with pytest.raises(native.HVPError) as e:
            ctx.loss_grad(G)
        assert e.value.code == native.HVP_ENONFINITE
        # the context stays usable
        o, phi = _oracle(w)
        _check(ctx, w, o, TOL["c64"])


def test_maximum_size_solution_point_and_directional_derivative():
    # n = 30, the largest register the library accepts (2^30 amplitudes,
    # 16 GiB per (psi, dpsi) state set), L = 3, one sample. The oracle cannot
    # run at this size, so the checks are what the paper fixes: at G = U_ref
    # the overlap is 1, the cost 0, the Riemannian gradient 0 (App. F) and
    # H_R positive semidefinite on tangent directions (a minimum); near it,
    # the derivative of the cost along the unit gradient direction equals
    # the gradient's norm (Eq. grad-real), checked by a central difference.
    n, L = 30, 3
    w = make_workload(n, L, 1, seed=30)
    V = random_direction(w.K, w.Uref, seed=31)
    with native.Context(n, L, w.psi1q, w.Uref, riemannian=True) as ctx:
        assert ctx.plan_info()["passes"] == 4
        loss, gr, hr = ctx.hvp(w.Uref, V)
        T, ge = ctx.get("T"), ctx.get("grad_e")
        assert abs(loss) < 1e-5 and abs(T[0] - 1) < 1e-5, (loss, T)
        assert np.linalg.norm(gr) < 1e-4 * np.linalg.norm(ge)
        q = np.real(np.vdot(V.ravel(), hr.ravel()))
        assert q > -1e-4 * np.linalg.norm(hr) * np.linalg.norm(V), q
        G1 = make_workload(n, L, 1, seed=30, near_solution=0.1).G
        ctx.loss_grad(G1)
        g1 = ctx.get("grad_e")
        d = g1 / np.linalg.norm(g1)

        def cdiff(h):
            return (ctx.loss_grad(G1 + h * d)[0] - ctx.loss_grad(G1 - h * d)[0]) / (2 * h)

        # Richardson extrapolation of two central differences: O(h^4) error
        fd = (4 * cdiff(5e-3) - cdiff(1e-2)) / 3
    an = np.linalg.norm(g1)
    assert abs(fd - an) < 1e-3 * an, (fd, an)


@pytest.mark.parametrize("threads,window,recompute", [(0, 0, False), (128, 11, False), (0, 0, True),
                                                      (128, 11, True)])
def test_headline_shape_sampled_against_oracle(threads, window, recompute):
    # n = 20, L = 16, N_s = 64 in the benchmark's launch configurations (12-
    # and 11-qubit windows; forward states cached before every gate, 152 GiB,
    # or recomputed inside each pass); the oracle checks eight of the samples,
    # spread over the 64, one by one (T_s, Omega_s and every per-sample
    # environment), and the sample-summed outputs are checked through
    # linearity in the samples (and against the oracle on all 64 samples in
    # test_headline_shape_sample_sums_against_oracle_on_all_samples).
    w = make_workload(20, 16, 64, seed=0)
    with native.Context(20, 16, w.psi1q, w.Uref, threads=threads, window=window, recompute=recompute) as ctx:
        info = ctx.plan_info()
        assert info["passes"] == (4 if window == 0 else 6)
        assert (info["checkpoint_stride"] == 0) == (not recompute)
        assert info["tiles_per_cta"] > 1
        r0 = ctx.hvp(w.G, w.V)
        loss, grad, hvp = ctx.hvp(w.G, w.V)
        assert r0[0] == loss and np.array_equal(r0[1], grad) and np.array_equal(r0[2], hvp)
        T, Om = ctx.get("T"), ctx.get("Omega")
        E, DE = ctx.get("env")
    import os

    pick = [0, 9, 18, 27, 37, 46, 55, 63]
    sub = w.psi1q[pick]
    phi = oracle.reference_states(20, 16, w.Uref, sub)
    o = oracle.evaluate(20, 16, w.G, w.V, sub, phi, threads=min(len(pick), os.cpu_count() or 1), ckpt_stride=12,
                        want_env=True)
    assert rel(T[pick], o["T"]) < TOL["c64"]
    assert rel(Om[pick], o["Omega"]) < TOL["c64"]
    for i, s in enumerate(pick):
        assert rel(E[s], o["E"][i]) < TOL["c64"]
        assert rel(DE[s], o["DE"][i]) < TOL["c64"]
    # sample sums from the per-sample pieces (Alg. 2 is linear in them)
    g = -(2 / 64) * np.einsum("s,skij->kij", T, E.conj())
    h = -(2 / 64) * (np.einsum("s,skij->kij", Om, E.conj()) + np.einsum("s,skij->kij", T, DE.conj()))
    assert rel(grad, g) < 1e-9 and rel(hvp, h) < 1e-9
    assert abs(loss - (1 - np.mean(np.abs(T) ** 2))) < 1e-12


def test_headline_shape_sample_sums_against_oracle_on_all_samples():
    # the benchmark workload in its default (autotuned-equivalent) window-pass
    # configuration: loss, gradient and HVP summed over all 64 samples against
    # the oracle run on all 64 samples
    w, phi, o = headline_oracle()
    with native.Context(20, 16, w.psi1q, w.Uref) as ctx:
        _check(ctx, w, o, TOL["c64"])


@pytest.mark.parametrize("threads", [256, 128])
def test_forward_cache_schedule_against_recompute_and_oracle(threads):
    # Several tiles per CTA (the copy barriers' phases run on across tiles),
    # several passes, both the tangent and the loss/gradient-only sweeps: the
    # cached schedule against the oracle, against the recomputing schedule
    # (same arithmetic except G^-1 recomputation, so close but not
    # identical) and against itself on a repeated call (bit-identical).
    n, L, ns = 14, 8, 256
    w = make_workload(n, L, ns, seed=140)
    o, phi = _oracle(w)
    res = {}
    for recompute in (False, True):
        with native.Context(n, L, w.psi1q, w.Uref, window=8, threads=threads, recompute=recompute) as ctx:
            info = ctx.plan_info()
            assert info["passes"] > 2 and info["tiles_per_cta"] > 1
            assert (info["checkpoint_stride"] == 0) == (not recompute)
            r1 = _check(ctx, w, o, TOL["c64"])
            r2 = ctx.hvp(w.G, w.V)
            assert r1[0] == r2[0] and np.array_equal(r1[1], r2[1]) and np.array_equal(r1[2], r2[2])
            lg = ctx.loss_grad(w.G)
            assert abs(lg[0] - o["loss"]) <= TOL["c64"] and rel(lg[1], o["grad"]) < TOL["c64"]
            res[recompute] = r1
    assert rel(res[False][1], res[True][1]) < 2 * TOL["c64"]
    assert rel(res[False][2], res[True][2]) < 2 * TOL["c64"]


def test_expired_cache_copy_wait_is_reported_and_context_stays_usable():
    # Every forward-cache copy barrier expects 16 bytes more than its copy
    # brings, so no wait completes: each gives up after 1000 polls, the call
    # reports HVP_ETIMEOUT, and after restoring normal operation the same
    # context evaluates correctly.
    w = make_workload(10, 6, 2, seed=13)
    o, phi = _oracle(w)
    with native.Context(10, 6, w.psi1q, w.Uref, window=8) as ctx:
        assert ctx.plan_info()["checkpoint_stride"] == 0
        ctx.cache_wait_test(16, 1000)
        with pytest.raises(native.HVPError) as e:
            ctx.hvp(w.G, w.V)
        assert e.value.code == native.HVP_ETIMEOUT
        ctx.cache_wait_test(0, 0)
        _check(ctx, w, o, TOL["c64"])
    with native.Context(10, 6, w.psi1q, w.Uref, window=8, recompute=True) as ctx:
        with pytest.raises(native.HVPError) as e:
            ctx.cache_wait_test(16, 1000)
        assert e.value.code == native.HVP_EINVAL
