"""Riemannian trust-region optimisation on U(4)^K with truncated conjugate
gradients: the optimiser the paper drives with its HVP kernel (Sec. 4, citing
Absil, Mahony and Sepulchre 2008, Algorithm 10 for the trust region and
Algorithm 11 for the truncated CG inner solver).

Every gradient and Hessian-vector product comes from a *problem* object: any
object with

    loss_grad(G) -> (loss, grad_R)
    hvp(G, V)    -> (loss, grad_R, H_R[V])

where grad_R and H_R[V] are the Riemannian forms (App. F), e.g. a
:class:`paper_2604_20384_gb300.native.Context` created with
``riemannian=True``. This module does only host-side bookkeeping on K 4x4
blocks: inner products with the metric Re Tr(A^dag B) of App. F, tangent
projections, the retraction and the radius logic. Each truncated-CG
iteration costs one HVP, i.e. one forward/backward sweep pair on the GPU.

The paper does not name a retraction; this module uses the polar retraction
R_G(xi) = U W^dag with G + xi = U S W^dag (SVD), gate by gate, which maps
G + xi to the nearest unitary and agrees with the exponential map to second
order.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def inner(a, b) -> float:
    """Re <A, B> = Re Tr(A^dag B), summed over the gates (App. F metric)."""
    return float(np.real(np.vdot(np.asarray(a).ravel(), np.asarray(b).ravel())))


def norm(a) -> float:
    return float(np.sqrt(max(inner(a, a), 0.0)))


def project(G, X):
    """P_G(X) = X/2 - G X^dag G/2 gate-wise (App. F, Eq. projec)."""
    G = np.asarray(G)
    X = np.asarray(X)
    return 0.5 * X - 0.5 * G @ np.conj(np.swapaxes(X, -1, -2)) @ G


def retract(G, xi):
    """Polar retraction: the unitary factor of G + xi, gate by gate."""
    U, _, Wh = np.linalg.svd(np.asarray(G) + np.asarray(xi))
    return U @ Wh


def _to_boundary(eta, d, delta) -> float:
    """tau >= 0 with ||eta + tau d|| = delta."""
    a = inner(d, d)
    b = 2.0 * inner(eta, d)
    c = inner(eta, eta) - delta * delta
    disc = max(b * b - 4.0 * a * c, 0.0)
    return (-b + np.sqrt(disc)) / (2.0 * a)


@dataclass
class TCGResult:
    eta: np.ndarray            # step (tangent at G)
    Heta: np.ndarray           # H_R[eta], kept by linearity (no extra HVP)
    iterations: int            # HVPs spent
    stop: str                  # "residual", "boundary", "negative curvature", "max iterations"


def truncated_cg(problem, G, grad, delta: float, kappa: float = 0.1, theta: float = 1.0,
                 max_iter: int = 50) -> TCGResult:
    """Truncated (Steihaug-Toint) CG for min m(eta) = <grad, eta> + <eta, H eta>/2
    over ||eta|| <= delta (Algorithm 11): stops on the residual criterion
    ||r|| <= ||r_0|| min(||r_0||^theta, kappa), at the trust-region boundary
    or on non-positive curvature."""
    eta = np.zeros_like(grad)
    Heta = np.zeros_like(grad)
    r = np.array(grad, copy=True)
    d = -r
    rr = inner(r, r)
    r0 = np.sqrt(rr)
    if r0 == 0.0:
        return TCGResult(eta, Heta, 0, "residual")
    for j in range(max_iter):
        Hd = project(G, problem.hvp(G, d)[2])
        curv = inner(d, Hd)
        if curv <= 0.0:
            tau = _to_boundary(eta, d, delta)
            return TCGResult(eta + tau * d, Heta + tau * Hd, j + 1, "negative curvature")
        alpha = rr / curv
        eta_next = eta + alpha * d
        if norm(eta_next) >= delta:
            tau = _to_boundary(eta, d, delta)
            return TCGResult(eta + tau * d, Heta + tau * Hd, j + 1, "boundary")
        eta = eta_next
        Heta = Heta + alpha * Hd
        r = r + alpha * Hd
        rr_next = inner(r, r)
        if np.sqrt(rr_next) <= r0 * min(r0 ** theta, kappa):
            return TCGResult(eta, Heta, j + 1, "residual")
        d = -r + (rr_next / rr) * d
        rr = rr_next
    return TCGResult(eta, Heta, max_iter, "max iterations")


@dataclass
class TRState:
    G: np.ndarray
    loss: float
    grad: np.ndarray
    delta: float
    history: list = field(default_factory=list)   # per step: loss, |grad|, rho, delta, HVPs, accepted, stop


def trust_region(problem, G0, steps: int = 10, delta0: float | None = None, delta_max: float | None = None,
                 rho_prime: float = 0.1, grad_tol: float = 1e-12, tcg_max_iter: int = 50) -> TRState:
    """Riemannian trust-region iterations (Algorithm 10) from unitary gates G0:
    truncated-CG step, polar retraction, acceptance on
    rho = (f(G) - f(R_G(eta))) / (m(0) - m(eta)) > rho_prime, radius quartered
    when rho < 1/4 and doubled (up to delta_max) when rho > 3/4 on the
    boundary. Stops after `steps` steps, when ||grad_R|| <= grad_tol, or when
    the model predicts no decrease above the rounding of the loss."""
    G = np.array(G0, dtype=np.complex128, copy=True)
    K = G.shape[0]
    if delta_max is None:
        delta_max = np.sqrt(4.0 * K)      # a gate's tangent vectors have norm <= 2
    delta = delta_max / 8.0 if delta0 is None else delta0
    loss, grad = problem.loss_grad(G)
    grad = project(G, grad)
    st = TRState(G, float(loss), grad, float(delta))
    for _ in range(steps):
        gnorm = norm(st.grad)
        if gnorm <= grad_tol:
            break
        res = truncated_cg(problem, st.G, st.grad, st.delta, max_iter=tcg_max_iter)
        model_decrease = -(inner(st.grad, res.eta) + 0.5 * inner(res.eta, res.Heta))
        if model_decrease <= 1e-15 * max(1.0, abs(st.loss)):
            st.history.append(dict(loss=st.loss, grad_norm=gnorm, rho=float("nan"), delta=st.delta,
                                   hvps=res.iterations, accepted=False, stop="no model decrease"))
            break
        G_new = retract(st.G, res.eta)
        loss_new, grad_new = problem.loss_grad(G_new)
        actual = st.loss - float(loss_new)
        rho = actual / model_decrease if model_decrease > 0 else -np.inf
        on_boundary = abs(norm(res.eta) - st.delta) <= 1e-12 * max(st.delta, 1.0)
        if rho < 0.25:
            new_delta = 0.25 * st.delta
        elif rho > 0.75 and on_boundary:
            new_delta = min(2.0 * st.delta, delta_max)
        else:
            new_delta = st.delta
        accepted = rho > rho_prime
        st.history.append(dict(loss=st.loss, grad_norm=gnorm, rho=float(rho), delta=st.delta,
                               hvps=res.iterations, accepted=accepted, stop=res.stop))
        if accepted:
            st.G, st.loss, st.grad = G_new, float(loss_new), project(G_new, grad_new)
        st.delta = new_delta
    return st
