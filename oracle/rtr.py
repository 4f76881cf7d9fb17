"""FP64 oracle for the paper's own J-update solvers: the Riemannian trust-region method (RTR) with
a truncated conjugate-gradient inner solver (Section 3, the minimisation of Eq. M1), and the SAGE
decomposition of the K-direction problem into K single-direction problems (step D1).

TEST INFRASTRUCTURE. Like oracle/admm.py (whose data-model, gradient, Hessian and Lagrangian
functions it calls), this module is the plain reference the CUDA path is checked against. Only the
test suite, the package smoke check and the benchmark's CPU legs may import it; the library never
does, and it shares no code with the CUDA sources.

Readings (the paper names the methods and cites their sources but prints no parameters):

* RTR runs in Euclidean space: the projection is the identity and the retraction is
  R(J, eta) = J + eta (Appendix A, last paragraph before the convergence section). The inner
  product is h (Eq. inprod), the gradient grad_i(L_i, J) (Eq. gradL), the Hessian the
  Gauss-Newton Hess_i(L_i, J) (Eq. HessL with the sign reading of oracle/admm.py).
* Outer iteration (trust-region rules of Absil, Baker and Gallivan, "Trust-region methods on
  Riemannian manifolds", 2007): ratio = (L(J) - L(J + eta)) / (m(0) - m(eta)) with the quadratic
  model m; the radius is quartered when ratio < 1/4, doubled (at most to Delta_bar) when
  ratio > 3/4 and the step reached the boundary, else kept; the step is accepted when
  ratio > 0.1. Delta_bar defaults to ||J0||_h and Delta_0 to Delta_bar / 8.
* Inner solver: truncated CG of Steihaug and Toint (the inner solver of the same paper), without a
  preconditioner, in the norm ||x||_h = sqrt(h(x, x)); it stops on the trust-region boundary, on
  non-positive curvature, when ||r_j|| <= ||r_0|| min(||r_0||^theta, kappa) with theta = 1 and
  kappa = 0.1, or after n_cg steps.
* SAGE (step D1): for each direction k in turn, the expectation step forms the conditional data
  V_k = V - sum_{l != k} J_pl C_pql J_ql^H (without the auxiliary variables or the penalty), and
  the maximisation step runs RTR on the single-direction Lagrangian of direction k,
  ||V_k - J_pk C_pqk J_qk^H||^2 + Re tr(Y_k^H (J_k - BZ_k)) + rho_k/2 ||J_k - BZ_k||^2 (full
  regularisation). One SAGE sweep visits k = 0 .. K-1; the paper's Simulation II uses 3 sweeps.
  With the other directions fixed this is L_i(J) up to a constant, so a sweep is block-coordinate
  descent on L_i.

Parity status: pinned by tests/test_oracle_rtr.py (closed-form Cauchy step, dense Newton solve,
Cauchy-decrease bound, monotone decrease, convergence to the known minimiser of noise-free data,
K = 1 reduction of SAGE to RTR).
"""
from __future__ import annotations

import math

import numpy as np

from oracle.admm import aug_lagrangian, grad_lagrangian, h_inner, hess_lagrangian, model_vis

RTR_ACCEPT = 0.1
TCG_THETA = 1.0
TCG_KAPPA = 0.1


def h_norm(x: np.ndarray) -> float:
    return math.sqrt(max(h_inner(x, x), 0.0))


def truncated_cg(J, C, pq, grad, rho, delta, n_cg, theta=TCG_THETA, kappa=TCG_KAPPA):
    """Approximate minimiser of m(eta) = h(grad, eta) + 1/2 h(eta, Hess L[eta]) over ||eta||_h <= delta
    (Steihaug-Toint truncated CG from eta = 0). Returns (eta, stop) with stop one of
    'boundary', 'curvature', 'residual', 'steps'."""
    eta = np.zeros_like(grad)
    r = grad.copy()
    d = -r
    rr = h_inner(r, r)
    r0 = math.sqrt(rr)
    if r0 == 0.0:
        return eta, "residual"
    for _ in range(n_cg):
        Hd = hess_lagrangian(J, d, C, pq, rho)
        dHd = h_inner(d, Hd)
        alpha = rr / dHd if dHd > 0.0 else 0.0
        nxt = eta + alpha * d
        if not dHd > 0.0 or h_norm(nxt) >= delta:
            # step to the boundary along d: ||eta + tau d|| = delta, tau >= 0
            ed, dd, ee = h_inner(eta, d), h_inner(d, d), h_inner(eta, eta)
            tau = (-ed + math.sqrt(ed * ed + dd * (delta * delta - ee))) / dd
            return eta + tau * d, ("curvature" if not dHd > 0.0 else "boundary")
        eta = nxt
        r = r + alpha * Hd
        rr_new = h_inner(r, r)
        if math.sqrt(rr_new) <= r0 * min(r0 ** theta, kappa):
            return eta, "residual"
        d = -r + (rr_new / rr) * d
        rr = rr_new
    return eta, "steps"


def model_decrease(J, C, pq, grad, rho, eta) -> float:
    """m(0) - m(eta) = -h(grad, eta) - 1/2 h(eta, Hess L[eta])."""
    return -(h_inner(grad, eta) + 0.5 * h_inner(eta, hess_lagrangian(J, eta, C, pq, rho)))


def rtr_jupdate(J0, V, C, pq, Y, BZ, rho, n_rtr, n_cg, delta_bar=None, delta0=None, trace=None):
    """Minimise L_i(J, Z, Y) over J (Eq. M1) by n_rtr Riemannian trust-region steps in Euclidean
    space (Section 3 and Appendix A; rules in the module docstring). trace, if a list, receives
    one (delta, ratio, accepted, stop, L after the step) tuple per step."""
    J = J0.copy()
    if delta_bar is None:
        delta_bar = h_norm(J0)
    delta = delta_bar / 8.0 if delta0 is None else delta0
    L = aug_lagrangian(J, V, C, pq, Y, BZ, rho)
    for _ in range(n_rtr):
        grad = grad_lagrangian(J, V, C, pq, Y, BZ, rho)
        eta, stop = truncated_cg(J, C, pq, grad, rho, delta, n_cg)
        pred = model_decrease(J, C, pq, grad, rho, eta)
        Lt = aug_lagrangian(J + eta, V, C, pq, Y, BZ, rho)
        ratio = (L - Lt) / pred if pred > 0.0 and math.isfinite(Lt) else -math.inf
        d_used = delta
        if ratio < 0.25:
            delta = delta / 4.0
        elif ratio > 0.75 and stop in ("boundary", "curvature"):
            delta = min(2.0 * delta, delta_bar)
        accepted = ratio > RTR_ACCEPT
        if accepted:
            J, L = J + eta, Lt
        if trace is not None:
            trace.append((d_used, ratio, accepted, stop, L))
    return J


def sage_jupdate(J0, V, C, pq, Y, BZ, rho, n_sage, n_rtr, n_cg, trace=None):
    """Step D1: n_sage SAGE sweeps over the directions; each direction's maximisation step is
    rtr_jupdate on its single-direction Lagrangian with the other directions' models removed from
    the data (expectation step). trace, if a list, receives L_i after every direction update."""
    J = J0.copy()
    K = J.shape[0]
    for _ in range(n_sage):
        for k in range(K):
            others = [l for l in range(K) if l != k]
            Vk = V - model_vis(J[others], C[:, :, others], pq) if others else V
            sl = slice(k, k + 1)
            J[sl] = rtr_jupdate(J[sl], Vk, C[:, :, sl], pq, Y[sl], BZ[sl], rho[sl], n_rtr, n_cg)
            if trace is not None:
                trace.append(aug_lagrangian(J, V, C, pq, Y, BZ, rho))
    return J
