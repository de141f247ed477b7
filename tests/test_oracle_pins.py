"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks the oracle against a fact that the paper or the mathematics
fixes: the dense brute force (oracle/dense.py), central finite differences of
the loss and of the gradient (Eq. grad-real, Eq. FoR), closed forms for a
single gate, the solution point G = U_ref, overlap invariance (Eq.
overlap-general), the identity for Omega (Eq. Omega, App. B), a second
derivation order of the HVP (App. C), and the projection identities of App. F.
"""
import numpy as np
import pytest

from common import expm_skew, grad_at, loss_at, oracle_case, re_inner, rel
from oracle import dense, oracle
from paper_2604_20384_gb300.inputs import (haar_unitary, make_workload, num_gates,
                                           random_direction)


# ---------------------------------------------------------------- layout / inputs

@pytest.mark.parametrize("n,L,K", [(6, 3, 8), (12, 8, 44), (20, 16, 152), (26, 24, 300), (2, 1, 1),
                                   (3, 2, 2), (7, 5, 15)])
def test_brickwall_gate_count(n, L, K):
    assert num_gates(n, L) == K
    fq = oracle.layout(n, L)
    assert len(fq) == K
    # every gate acts on (i, i+1) inside the chain, layers alternate offsets
    assert all(0 <= i and i + 1 <= n - 1 for i in fq)


def test_layout_matches_dense_independent_layout():
    for n, L in [(5, 4), (6, 3), (8, 6)]:
        a = list(oracle.layout(n, L))
        b = [i for (_, i, _) in dense.layer_gate_indices(n, L)]
        assert a == b


def test_inputs_are_unitary_and_normalised():
    w = make_workload(6, 3, 16, seed=3)
    eye = np.eye(4)
    for k in range(w.K):
        assert np.max(np.abs(w.G[k].conj().T @ w.G[k] - eye)) < 1e-14
        assert np.max(np.abs(w.Uref[k].conj().T @ w.Uref[k] - eye)) < 1e-14
        X = w.G[k].conj().T @ w.V[k]          # V = G X with X skew-Hermitian
        assert np.max(np.abs(X + X.conj().T)) < 1e-13
    assert np.max(np.abs(np.linalg.norm(w.psi1q, axis=-1) - 1)) < 1e-15
    phi = oracle.reference_states(6, 3, w.Uref, w.psi1q)
    assert np.max(np.abs(np.linalg.norm(phi, axis=1) - 1)) < 1e-14


def test_inputs_are_deterministic():
    a = make_workload(5, 3, 4, seed=11)
    b = make_workload(5, 3, 4, seed=11)
    c = make_workload(5, 3, 4, seed=12)
    assert np.array_equal(a.G, b.G) and np.array_equal(a.psi1q, b.psi1q) and np.array_equal(a.V, b.V)
    assert not np.array_equal(a.G, c.G)


# ---------------------------------------------------------------- dense brute force

@pytest.mark.parametrize("n,L,ns,seed", [(4, 3, 5, 0), (5, 4, 3, 1), (6, 3, 16, 0), (3, 5, 2, 7)])
def test_sweep_matches_dense_brute_force(n, L, ns, seed):
    w, phi, o = oracle_case(n, L, ns, seed, want_env=True)
    d = dense.evaluate(n, L, w.G, w.V, w.psi1q, w.Uref)
    assert abs(o["loss"] - d["loss"]) < 1e-13
    for key in ("T", "Omega", "E", "DE", "grad", "hvp"):
        assert rel(o[key], d[key]) < 1e-12, key
    assert rel(phi, d["phi"]) < 1e-13


def test_sweep_matches_dense_for_non_unitary_gates():
    # The oracle must not assume unitarity: finite differences evaluate G + hV.
    w = make_workload(5, 3, 4, seed=5)
    rng = np.random.default_rng(9)
    Gn = w.G + 0.2 * (rng.standard_normal(w.G.shape) + 1j * rng.standard_normal(w.G.shape))
    phi = oracle.reference_states(5, 3, w.Uref, w.psi1q)
    o = oracle.evaluate(5, 3, Gn, w.V, w.psi1q, phi, want_env=True)
    d = dense.evaluate(5, 3, Gn, w.V, w.psi1q, w.Uref)
    for key in ("T", "E", "DE", "grad", "hvp"):
        assert rel(o[key], d[key]) < 1e-12, key


# ---------------------------------------------------------------- finite differences

def _unit(K, k, i, j, val):
    e = np.zeros((K, 4, 4), complex)
    e[k, i, j] = val
    return e


def test_gradient_by_central_differences():
    # grad f = df/dx + i df/dy entry-wise (Eq. grad-real).
    w, phi, o = oracle_case(5, 4, 6, seed=2)
    h = 1e-5
    rng = np.random.default_rng(0)
    for _ in range(12):
        k, i, j = int(rng.integers(w.K)), int(rng.integers(4)), int(rng.integers(4))
        dx = (loss_at(w, phi, w.G + _unit(w.K, k, i, j, h)) - loss_at(w, phi, w.G - _unit(w.K, k, i, j, h))) / (2 * h)
        dy = (loss_at(w, phi, w.G + _unit(w.K, k, i, j, 1j * h)) - loss_at(w, phi, w.G - _unit(w.K, k, i, j, 1j * h))) / (2 * h)
        assert abs(o["grad"][k, i, j] - (dx + 1j * dy)) < 1e-9


def test_directional_derivative_matches_gradient():
    # D C[V] = Re<grad C, V> (Eq. directional-derivative-definition, App. A).
    w, phi, o = oracle_case(6, 3, 8, seed=4)
    h = 1e-5
    fd = (loss_at(w, phi, w.G + h * w.V) - loss_at(w, phi, w.G - h * w.V)) / (2 * h)
    assert abs(re_inner(o["grad"], w.V) - fd) < 1e-10


def test_hvp_by_central_differences_of_gradient():
    # H[V] = D(grad C)[V] (Eq. FoR); Richardson-extrapolated central differences.
    w, phi, o = oracle_case(5, 4, 6, seed=3)

    def cd(h):
        return (grad_at(w, phi, w.G + h * w.V) - grad_at(w, phi, w.G - h * w.V)) / (2 * h)

    h = 1e-3
    fd = (4 * cd(h / 2) - cd(h)) / 3
    assert rel(o["hvp"], fd) < 1e-8


def test_hvp_symmetry():
    # Re<W, H[V]> = Re<V, H[W]> (symmetry of mixed partials, Sec. 2.1).
    w, phi, o = oracle_case(6, 4, 8, seed=6)
    W = random_direction(w.K, w.G, seed=77)
    ow = oracle.evaluate(6, 4, w.G, W, w.psi1q, phi)
    a = re_inner(W, o["hvp"])
    b = re_inner(w.V, ow["hvp"])
    assert abs(a - b) < 1e-12 * max(1.0, abs(a))


def test_hvp_is_linear_in_direction():
    w, phi, o = oracle_case(5, 3, 4, seed=8)
    W = random_direction(w.K, w.G, seed=5)
    a = oracle.evaluate(5, 3, w.G, W, w.psi1q, phi)["hvp"]
    b = oracle.evaluate(5, 3, w.G, 2.0 * w.V - 3.0 * W, w.psi1q, phi)["hvp"]
    assert rel(b, 2.0 * o["hvp"] - 3.0 * a) < 1e-12


# ---------------------------------------------------------------- closed forms

def test_single_gate_closed_forms():
    # n = 2, one gate: dT/dG = conj(phi) psi^T, so grad C = -(2/N) sum T phi psi^dag,
    # DE = 0 (no other gate varies) and H = -(2/N) sum Omega phi psi^dag with
    # Omega = phi^dag V psi. A literal reading of Alg. 1's line order would give
    # DE = (V^dag phi)^* psi^T != 0 here.
    w, phi, o = oracle_case(2, 1, 7, seed=1, want_env=True)
    assert w.K == 1
    psi = np.stack([np.kron(w.psi1q[s, 0], w.psi1q[s, 1]) for s in range(7)])
    T = np.einsum("si,ij,sj->s", phi.conj(), w.G[0], psi)
    Om = np.einsum("si,ij,sj->s", phi.conj(), w.V[0], psi)
    grad = -(2 / 7) * np.einsum("s,si,sj->ij", T, phi, psi.conj())
    hvp = -(2 / 7) * np.einsum("s,si,sj->ij", Om, phi, psi.conj())
    assert rel(o["T"], T) < 1e-14
    assert rel(o["grad"][0], grad) < 1e-13
    assert rel(o["hvp"][0], hvp) < 1e-13
    assert np.max(np.abs(o["DE"])) == 0.0
    literal = np.einsum("si,sj->sij", (phi @ w.V[0].conj()).conj(), psi)   # (V^dag phi)^* psi^T
    assert np.max(np.abs(literal)) > 1e-3


def test_solution_point():
    # G = U_ref: T_s = 1, C = 0, Riemannian gradient 0, Euclidean gradient
    # G_k (Hermitian) (Sec. 4.1; App. F), Riemannian Hessian positive
    # semidefinite on tangent vectors (a minimum).
    w = make_workload(6, 4, 6, seed=9)
    phi = oracle.reference_states(6, 4, w.Uref, w.psi1q)
    o = oracle.evaluate(6, 4, w.Uref, w.V, w.psi1q, phi)
    assert np.max(np.abs(o["T"] - 1)) < 1e-13
    assert abs(o["loss"]) < 1e-13
    assert np.max(np.abs(o["grad_r"])) < 1e-13
    assert np.max(np.abs(o["grad"])) > 1e-3
    for k in range(w.K):
        H = w.Uref[k].conj().T @ o["grad"][k]
        assert np.max(np.abs(H - H.conj().T)) < 1e-13
    rng = np.random.default_rng(1)
    for t in range(4):
        X = rng.standard_normal((w.K, 4, 4)) + 1j * rng.standard_normal((w.K, 4, 4))
        Vt = np.stack([w.Uref[k] @ (0.5 * (X[k] - X[k].conj().T)) for k in range(w.K)])
        ot = oracle.evaluate(6, 4, w.Uref, Vt, w.psi1q, phi)
        assert re_inner(Vt, ot["hvp_r"]) >= -1e-12


def test_loss_bounds_random_circuit():
    w, phi, o = oracle_case(7, 5, 10, seed=2)
    assert np.all(np.abs(o["T"]) <= 1 + 1e-14)
    assert 0.0 <= o["loss"] <= 1.0


# ---------------------------------------------------------------- identities

def test_overlap_invariance_over_cuts():
    # T = phi^[K-k]^dag psi^[k] for every k (Eq. overlap-general).
    w, phi, o = oracle_case(6, 5, 4, seed=10, want_cuts=True)
    assert np.max(np.abs(o["cuts"] - o["T"][:, None])) < 1e-14


def test_overlap_from_environment():
    # T = sum_ij E_k[i][j] G_k[i][j] for every k (Eq. overlap-2).
    w, phi, o = oracle_case(6, 4, 5, seed=12, want_env=True)
    for k in range(w.K):
        Tk = np.einsum("sij,ij->s", o["E"][:, k], w.G[k])
        assert np.max(np.abs(Tk - o["T"])) < 1e-14


def test_omega_two_ways():
    # Omega = sum_k Tr(E_k^T V_k) (Eq. Omega) = phi^dag dpsi^[K] (Eq. dfis).
    w, phi, o = oracle_case(6, 4, 5, seed=13)
    assert np.max(np.abs(o["Omega"] - o["Omega_fwd"])) < 1e-13


def _apply(state, n, q, M):
    t = state.reshape([2] * n)
    t = np.moveaxis(t, (q, q + 1), (0, 1)).reshape(4, -1)
    t = (M @ t).reshape([2, 2] + [2] * (n - 2))
    return np.moveaxis(t, (0, 1), (q, q + 1)).reshape(-1)


def _pair(x, y, n, q):
    """sum_a x[m, a] y[n, a] over all qubits other than (q, q+1), no conjugation."""
    a = np.moveaxis(x.reshape([2] * n), (q, q + 1), (0, 1)).reshape(4, -1)
    b = np.moveaxis(y.reshape([2] * n), (q, q + 1), (0, 1)).reshape(4, -1)
    return a @ b.T


def test_reverse_over_reverse_order_agrees():
    # App. C: the HVP as the gradient of Omega, with dual tangent states obtained
    # by a backward recursion of transposes acting on conj(phi), and a forward
    # recursion for the other dual. Written here with numpy state vectors.
    n, L, ns = 5, 4, 3
    w, phi, o = oracle_case(n, L, ns, seed=14, want_env=True)
    fq = oracle.layout(n, L)
    K = w.K
    for s in range(ns):
        psi = [dense.product_state(w.psi1q[s])]
        for k in range(K):
            psi.append(_apply(psi[-1], n, fq[k], w.G[k]))
        phit = [phi[s].conj()]                               # conj(phi^[m]), m = 0..K
        for m in range(1, K + 1):
            phit.append(_apply(phit[-1], n, fq[K - m], w.G[K - m].T))
        bar_psi = [None] * (K + 1)                           # bar_psi_k, k = 0..K
        bar_psi[K] = np.zeros_like(psi[0])
        for k in range(K, 0, -1):
            bar_psi[k - 1] = _apply(phit[K - k], n, fq[k - 1], w.V[k - 1].T) + _apply(bar_psi[k], n, fq[k - 1], w.G[k - 1].T)
        beta = [None] * (K + 1)                              # beta_{K-k} = dpsi^[k]
        beta[K] = np.zeros_like(psi[0])
        for k in range(1, K + 1):
            beta[K - k] = _apply(psi[k - 1], n, fq[k - 1], w.V[k - 1]) + _apply(beta[K - k + 1], n, fq[k - 1], w.G[k - 1])
        for k in range(1, K + 1):
            H = _pair(bar_psi[k], psi[k - 1], n, fq[k - 1]) + _pair(phit[K - k], beta[K - k + 1], n, fq[k - 1])
            E = _pair(phit[K - k], psi[k - 1], n, fq[k - 1])
            assert np.max(np.abs(H - o["DE"][s, k - 1])) < 1e-13
            assert np.max(np.abs(E - o["E"][s, k - 1])) < 1e-13


def test_checkpoint_stride_and_threads_do_not_change_results():
    w, phi, o1 = oracle_case(6, 5, 6, seed=15, threads=1, want_env=True)
    for stride, threads in [(2, 3), (5, 6), (13, 2), (100, 4)]:
        o2 = oracle.evaluate(6, 5, w.G, w.V, w.psi1q, phi, threads=threads, ckpt_stride=stride, want_env=True)
        for key in ("T", "E", "DE", "grad", "hvp", "grad_r", "hvp_r"):
            assert np.array_equal(o1[key], o2[key]), (stride, key)


# ---------------------------------------------------------------- Riemannian (App. F)

def test_projection_identities():
    rng = np.random.default_rng(3)
    K = 5
    G = np.stack([haar_unitary(rng, 4) for _ in range(K)])
    X = rng.standard_normal((K, 4, 4)) + 1j * rng.standard_normal((K, 4, 4))
    P = oracle.project(G, X)
    assert rel(oracle.project(G, P), P) < 1e-14                   # idempotent
    for k in range(K):
        S = G[k].conj().T @ P[k]
        assert np.max(np.abs(S + S.conj().T)) < 1e-14             # G^dag P_G(X) skew
        skew = 0.5 * (X[k] - X[k].conj().T)
        assert np.max(np.abs(oracle.project(G[k:k + 1], (G[k] @ skew)[None])[0] - G[k] @ skew)) < 1e-14
    # orthogonality: Re<X - P(X), T> = 0 for tangent T
    Y = rng.standard_normal((K, 4, 4)) + 1j * rng.standard_normal((K, 4, 4))
    Tn = oracle.project(G, Y)
    assert abs(re_inner(X - P, Tn)) < 1e-13


def _geodesic_loss(w, phi, X, t):
    Gt = np.stack([w.G[k] @ expm_skew(t * X[k]) for k in range(w.K)])
    return loss_at(w, phi, Gt)


def test_riemannian_gradient_and_hvp_along_geodesics():
    # On U(4)^K with the metric Re Tr(A^dag B), t -> G exp(tX) is a geodesic, so
    # d/dt C = Re<grad_R, GX> and d^2/dt^2 C = Re<GX, H_R[GX]> at t = 0.
    w = make_workload(5, 4, 5, seed=16)
    phi = oracle.reference_states(5, 4, w.Uref, w.psi1q)
    X = np.stack([w.G[k].conj().T @ w.V[k] for k in range(w.K)])    # skew-Hermitian
    o = oracle.evaluate(5, 4, w.G, w.V, w.psi1q, phi)
    h = 1e-3
    c0 = _geodesic_loss(w, phi, X, 0.0)
    cp, cm = _geodesic_loss(w, phi, X, h), _geodesic_loss(w, phi, X, -h)
    cp2, cm2 = _geodesic_loss(w, phi, X, 2 * h), _geodesic_loss(w, phi, X, -2 * h)
    d1 = (8 * (cp - cm) - (cp2 - cm2)) / (12 * h)
    d2 = (-cp2 + 16 * cp - 30 * c0 + 16 * cm - cm2) / (12 * h * h)
    assert abs(re_inner(o["grad_r"], w.V) - d1) < 1e-9
    assert abs(re_inner(w.V, o["hvp_r"]) - d2) < 1e-6 * max(1.0, abs(d2))


def test_riemannian_hessian_self_adjoint():
    # <H_R u, v> = <u, H_R v> on tangent vectors (App. G).
    w = make_workload(6, 3, 6, seed=17)
    phi = oracle.reference_states(6, 3, w.Uref, w.psi1q)
    W = random_direction(w.K, w.G, seed=31)
    a = oracle.evaluate(6, 3, w.G, w.V, w.psi1q, phi)["hvp_r"]
    b = oracle.evaluate(6, 3, w.G, W, w.psi1q, phi)["hvp_r"]
    assert abs(re_inner(W, a) - re_inner(w.V, b)) < 1e-12


def test_near_solution_workload_has_order_one_overlaps():
    w, phi, o = oracle_case(6, 3, 8, seed=0, near_solution=0.1)
    assert np.min(np.abs(o["T"])) > 0.5


# ---------------------------------------------------------------- Frobenius cost (Eq. Frobenius)

def test_frobenius_cost_against_dense_and_differences():
    w, phi, o = oracle_case(5, 4, 6, seed=41)
    d = dense.evaluate(5, 4, w.G, w.V, w.psi1q, w.Uref)
    assert abs(o["loss_f"] - d["loss_f"]) < 1e-13
    assert rel(o["grad_f"], d["grad_f"]) < 1e-12 and rel(o["hvp_f"], d["hvp_f"]) < 1e-12

    def lf(G):
        return oracle.evaluate(5, 4, G, None, w.psi1q, phi)["loss_f"]

    h = 1e-5
    for (k, i, j) in [(0, 0, 0), (3, 2, 1), (w.K - 1, 3, 3)]:
        e = np.zeros_like(w.G)
        e[k, i, j] = h
        dx = (lf(w.G + e) - lf(w.G - e)) / (2 * h)
        dy = (lf(w.G + 1j * e) - lf(w.G - 1j * e)) / (2 * h)
        assert abs(o["grad_f"][k, i, j] - (dx + 1j * dy)) < 1e-9

    def gf(G):
        return oracle.evaluate(5, 4, G, None, w.psi1q, phi)["grad_f"]

    hh = 1e-3
    fd = (4 * (gf(w.G + hh / 2 * w.V) - gf(w.G - hh / 2 * w.V)) / hh - (gf(w.G + hh * w.V) - gf(w.G - hh * w.V)) / (2 * hh)) / 3
    assert rel(o["hvp_f"], fd) < 1e-8


def test_frobenius_solution_point():
    # G = U_ref: T_s = 1 so C_F = 0 and its Riemannian gradient vanishes.
    w = make_workload(6, 3, 5, seed=43)
    phi = oracle.reference_states(6, 3, w.Uref, w.psi1q)
    o = oracle.evaluate(6, 3, w.Uref, w.V, w.psi1q, phi)
    assert abs(o["loss_f"]) < 1e-13
    assert np.max(np.abs(o["grad_fr"])) < 1e-13



def _geodesic_loss_f(w, phi, X, t):
    Gt = np.stack([w.G[k] @ expm_skew(t * X[k]) for k in range(w.K)])
    return oracle.evaluate(w.n, w.n_layers, Gt, None, w.psi1q, phi)["loss_f"]


def test_frobenius_riemannian_gradient_and_hvp_along_geodesics():
    # App. F applied to Eq. Frobenius: along the geodesic t -> G exp(tX),
    # d/dt C_F = Re<grad_R, GX> and d^2/dt^2 C_F = Re<GX, H_R[GX]> at t = 0,
    # with H_R built from the Frobenius gradient (a slip to the HS gradient in
    # the -V grad^dag G / 2 terms changes the second derivative). Away from the
    # solution point, so that the gradient is not zero.
    w = make_workload(5, 4, 5, seed=18)
    phi = oracle.reference_states(5, 4, w.Uref, w.psi1q)
    X = np.stack([w.G[k].conj().T @ w.V[k] for k in range(w.K)])    # skew-Hermitian
    o = oracle.evaluate(5, 4, w.G, w.V, w.psi1q, phi)
    assert np.linalg.norm(o["grad_fr"]) > 1e-2
    h = 1e-3
    c0 = _geodesic_loss_f(w, phi, X, 0.0)
    cp, cm = _geodesic_loss_f(w, phi, X, h), _geodesic_loss_f(w, phi, X, -h)
    cp2, cm2 = _geodesic_loss_f(w, phi, X, 2 * h), _geodesic_loss_f(w, phi, X, -2 * h)
    d1 = (8 * (cp - cm) - (cp2 - cm2)) / (12 * h)
    d2 = (-cp2 + 16 * cp - 30 * c0 + 16 * cm - cm2) / (12 * h * h)
    assert abs(re_inner(o["grad_fr"], w.V) - d1) < 1e-9
    assert abs(re_inner(w.V, o["hvp_fr"]) - d2) < 1e-6 * max(1.0, abs(d2))
    # the Euclidean Frobenius HVP alone does not give the geodesic curvature:
    # the App. F correction terms are needed (checks that the pin can fail)
    assert abs(re_inner(w.V, o["hvp_f"]) - d2) > 1e-4 * max(1.0, abs(d2))


def test_frobenius_riemannian_gradient_per_gate_directions():
    # Re<grad_R, G_k X_k> for one gate at a time equals the first geodesic
    # derivative of C_F moving that gate alone (pins every gate's block of
    # grad_fr, not only its inner product with V).
    w = make_workload(4, 3, 4, seed=19)
    phi = oracle.reference_states(4, 3, w.Uref, w.psi1q)
    o = oracle.evaluate(4, 3, w.G, w.V, w.psi1q, phi)
    rng = np.random.default_rng(5)
    h = 1e-3
    for k in range(w.K):
        A = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
        Xk = 0.5 * (A - A.conj().T)
        X = np.zeros((w.K, 4, 4), complex)
        X[k] = Xk
        cp, cm = _geodesic_loss_f(w, phi, X, h), _geodesic_loss_f(w, phi, X, -h)
        cp2, cm2 = _geodesic_loss_f(w, phi, X, 2 * h), _geodesic_loss_f(w, phi, X, -2 * h)
        d1 = (8 * (cp - cm) - (cp2 - cm2)) / (12 * h)
        assert abs(np.real(np.vdot(o["grad_fr"][k], w.G[k] @ Xk)) - d1) < 1e-10
        S = w.G[k].conj().T @ o["grad_fr"][k]
        assert np.max(np.abs(S + S.conj().T)) < 1e-13                # tangent at G_k


def test_frobenius_riemannian_hessian_self_adjoint():
    # <H_R u, v> = <u, H_R v> on tangent vectors, for the Frobenius cost too.
    w = make_workload(6, 3, 6, seed=21)
    phi = oracle.reference_states(6, 3, w.Uref, w.psi1q)
    W = random_direction(w.K, w.G, seed=33)
    a = oracle.evaluate(6, 3, w.G, w.V, w.psi1q, phi)["hvp_fr"]
    b = oracle.evaluate(6, 3, w.G, W, w.psi1q, phi)["hvp_fr"]
    assert abs(re_inner(W, a) - re_inner(w.V, b)) < 1e-12


# ---------------------------------------------------------------- translation invariance (App. E)

def test_translation_invariant_chain_rule():
    # Layer-gate derivatives are the per-gate sums over the layer (App. E):
    # checked against central differences in the layer gates themselves.
    from common import contract, expand

    n, L, ns = 6, 4, 5
    w = make_workload(n, L, ns, seed=51)
    Gl = np.stack([w.G[0], w.G[3], w.G[5], w.G[8]])      # one gate of each layer
    Vl = np.stack([w.V[0], w.V[3], w.V[5], w.V[8]])
    phi = oracle.reference_states(n, L, w.Uref, w.psi1q)
    o = oracle.evaluate(n, L, expand(Gl, n, L), expand(Vl, n, L), w.psi1q, phi)
    g_l, h_l = contract(o["grad"], n, L), contract(o["hvp"], n, L)

    def loss_l(G):
        return oracle.evaluate(n, L, expand(G, n, L), None, w.psi1q, phi)["loss"]

    def grad_l(G):
        return contract(oracle.evaluate(n, L, expand(G, n, L), None, w.psi1q, phi)["grad"], n, L)

    h = 1e-5
    for (l, i, j) in [(0, 0, 1), (2, 3, 3), (3, 1, 2)]:
        e = np.zeros_like(Gl)
        e[l, i, j] = h
        dx = (loss_l(Gl + e) - loss_l(Gl - e)) / (2 * h)
        dy = (loss_l(Gl + 1j * e) - loss_l(Gl - 1j * e)) / (2 * h)
        assert abs(g_l[l, i, j] - (dx + 1j * dy)) < 1e-9
    hh = 1e-3
    fd = (4 * (grad_l(Gl + hh / 2 * Vl) - grad_l(Gl - hh / 2 * Vl)) / hh
          - (grad_l(Gl + hh * Vl) - grad_l(Gl - hh * Vl)) / (2 * hh)) / 3
    assert rel(h_l, fd) < 1e-8


# ---------------------------------------------------------------- dense Riemannian Hessian (App. G)

def test_pauli_tangent_basis_is_orthonormal_tangent():
    from paper_2604_20384_gb300.spectrum import tangent_basis

    w = make_workload(4, 2, 1, seed=3)
    B = tangent_basis(w.G)
    Bf = B.reshape(B.shape[0], -1)
    gram = np.real(Bf.conj() @ Bf.T)
    assert np.max(np.abs(gram - np.eye(B.shape[0]))) < 1e-13
    P = np.stack([oracle.project(w.G, B[j]) for j in range(B.shape[0])])   # already tangent
    assert np.max(np.abs(P - B)) < 1e-13


def test_riemannian_hessian_from_oracle_hvps():
    from paper_2604_20384_gb300.spectrum import riemannian_hessian, spectrum

    n, L, ns = 4, 3, 4
    w = make_workload(n, L, ns, seed=91)
    phi = oracle.reference_states(n, L, w.Uref, w.psi1q)
    H = riemannian_hessian(lambda G, V: oracle.evaluate(n, L, G, V, w.psi1q, phi)["hvp_r"], w.G)
    assert np.max(np.abs(H - H.T)) < 1e-12 * np.max(np.abs(H))
    # the quadratic form along a basis vector equals the second derivative along
    # its geodesic (App. F); check one diagonal entry
    from paper_2604_20384_gb300.spectrum import tangent_basis
    E = tangent_basis(w.G)[5]
    X = np.stack([w.G[k].conj().T @ E[k] for k in range(w.K)])
    h = 1e-3

    def c(t):
        return oracle.evaluate(n, L, np.stack([w.G[k] @ expm_skew(t * X[k]) for k in range(w.K)]), None,
                               w.psi1q, phi)["loss"]

    d2 = (-c(2 * h) + 16 * c(h) - 30 * c(0) + 16 * c(-h) - c(-2 * h)) / (12 * h * h)
    assert abs(H[5, 5] - d2) < 1e-6 * max(1.0, abs(d2))
    # at the solution G = U_ref the Riemannian Hessian is positive semidefinite
    H0 = riemannian_hessian(lambda G, V: oracle.evaluate(n, L, G, V, w.psi1q, phi)["hvp_r"], w.Uref)
    assert spectrum(H0)[0] > -1e-10
