"""Pins for the RTR and SAGE oracle (oracle/rtr.py): each checks it against something other than
itself - a closed-form boundary step, a dense Newton solve, the Cauchy-decrease bound of trust-region
theory, monotonicity, and the known minimiser of noise-free data - so that a wrong sign, a dropped
term or a mis-indexed direction in the solver fails at least one of them."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import admm as O
from oracle import rtr as R


def cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def agent(seed=0, N=4, K=2, T=3, noise=0.0, rho=None, at_truth=False):
    """One agent: noise-free (or noisy) data of known solutions Jt, Y = 0 and BZ = Jt, so the
    augmented Lagrangian's minimiser is Jt itself when the data are noise-free."""
    rng = np.random.default_rng(seed)
    pq = np.array([(p, q) for p in range(N) for q in range(p + 1, N)], dtype=np.int32)
    C = cn(rng, len(pq), T, K) * 2.0
    Jt = np.eye(2) + 0.3 * cn(rng, K, N, 2, 2)
    V = O.model_vis(Jt, C, pq) + noise * cn(rng, len(pq), T, 2, 2)
    J0 = Jt.copy() if at_truth else Jt + 0.15 * cn(rng, K, N, 2, 2)
    rho = np.full(K, 2.0) if rho is None else np.asarray(rho, float)
    return dict(pq=pq, C=C, V=V, Jt=Jt, J0=J0, Y=np.zeros_like(Jt), BZ=Jt.copy(), rho=rho)


def real_coords(x):
    return np.concatenate([x.real.ravel(), x.imag.ravel()])


def from_real(v, shape):
    n = int(np.prod(shape))
    return (v[:n] + 1j * v[n:]).reshape(shape)


def dense_hessian(J, C, pq, rho):
    """The real matrix of eta -> Hess L[eta], one column per real coordinate."""
    n = 2 * J.size
    A = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        A[:, i] = real_coords(O.hess_lagrangian(J, from_real(e, J.shape), C, pq, rho))
    return A


# ------------------------------------------------------------------ truncated CG

def test_tiny_radius_gives_the_boundary_step_along_minus_the_gradient():
    """With a radius smaller than the first CG step, tCG returns the Cauchy direction on the
    boundary: eta = -delta grad / ||grad||_h."""
    a = agent(1)
    grad = O.grad_lagrangian(a["J0"], a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"])
    delta = 1e-4
    eta, stop = R.truncated_cg(a["J0"], a["C"], a["pq"], grad, a["rho"], delta, n_cg=5)
    assert stop == "boundary"
    gnorm = math.sqrt(O.h_inner(grad, grad))
    np.testing.assert_allclose(eta, -delta * grad / gnorm, rtol=1e-12, atol=1e-15)


def test_large_radius_and_enough_steps_solve_the_newton_system():
    """Radius far outside the Newton step, kappa tiny, n_cg = dimension: tCG is plain CG on the
    positive-definite Hess L and returns the solution of Hess L[eta] = -grad (dense solve)."""
    a = agent(2, N=3, K=1, T=2)
    J, C, pq, rho = a["J0"], a["C"], a["pq"], a["rho"]
    grad = O.grad_lagrangian(J, a["V"], C, pq, a["Y"], a["BZ"], rho)
    A = dense_hessian(J, C, pq, rho)
    ref = from_real(np.linalg.solve(A, -real_coords(grad)), J.shape)
    eta, stop = R.truncated_cg(J, C, pq, grad, rho, delta=1e6, n_cg=2 * J.size, kappa=1e-14)
    assert stop in ("residual", "steps")
    np.testing.assert_allclose(eta, ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("delta", [1e-3, 3e-2, 0.3, 3.0])
def test_tcg_decrease_is_at_least_the_cauchy_decrease(delta):
    """Trust-region theory: the first tCG iterate is the Cauchy point and later iterates only
    lower the model, so m(0) - m(eta) >= the Cauchy decrease
    max over 0 <= t <= delta / ||g|| of t ||g||^2 - t^2/2 h(g, H g)."""
    a = agent(3, noise=0.3)
    J, C, pq, rho = a["J0"], a["C"], a["pq"], a["rho"]
    g = O.grad_lagrangian(J, a["V"], C, pq, a["Y"], a["BZ"], rho)
    eta, _ = R.truncated_cg(J, C, pq, g, rho, delta, n_cg=6)
    gg = O.h_inner(g, g)
    gHg = O.h_inner(g, O.hess_lagrangian(J, g, C, pq, rho))
    t = min(delta / math.sqrt(gg), gg / gHg)
    cauchy = t * gg - 0.5 * t * t * gHg
    assert R.model_decrease(J, C, pq, g, rho, eta) >= cauchy * (1 - 1e-12)
    assert R.h_norm(eta) <= delta * (1 + 1e-12)


# ------------------------------------------------------------------ RTR outer iteration

def test_rtr_never_increases_the_lagrangian_and_reaches_the_noise_free_minimiser():
    """Noise-free data of Jt with BZ = Jt and Y = 0: L = 0 only at Jt, so RTR converges to Jt;
    accepted steps never raise L, and rejected steps shrink the radius."""
    a = agent(4, N=5, K=2, T=3)
    args = (a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"])
    trace = []
    J = R.rtr_jupdate(a["J0"], *args, n_rtr=40, n_cg=20, trace=trace)
    assert np.abs(J - a["Jt"]).max() < 1e-8
    Ls = [O.aug_lagrangian(a["J0"], *args)] + [t[4] for t in trace]
    assert all(b <= x for x, b in zip(Ls, Ls[1:]))
    assert Ls[-1] == pytest.approx(O.aug_lagrangian(J, *args), rel=1e-12, abs=1e-300)
    for (delta, ratio, accepted, stop, _), nxt in zip(trace, trace[1:]):
        if not accepted:
            assert nxt[0] == pytest.approx(delta / 4)


def test_rtr_lagrangian_sequence_is_monotone_on_noisy_data():
    a = agent(5, N=5, K=2, T=4, noise=0.5)
    args = (a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"])
    J = a["J0"].copy()
    Ls = [O.aug_lagrangian(J, *args)]
    for _ in range(8):
        J = R.rtr_jupdate(J, *args, n_rtr=1, n_cg=4)
        Ls.append(O.aug_lagrangian(J, *args))
    assert all(b <= x * (1 + 1e-14) for x, b in zip(Ls, Ls[1:]))
    g0 = O.grad_lagrangian(a["J0"], *args)
    g = O.grad_lagrangian(J, *args)
    assert R.h_norm(g) < 0.1 * R.h_norm(g0)


def test_rtr_at_the_minimiser_stays_there():
    """Started at Jt with noise-free data: the gradient is zero, tCG returns a zero step."""
    a = agent(6, at_truth=True)
    J = R.rtr_jupdate(a["J0"], a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"], n_rtr=3, n_cg=4)
    assert np.abs(J - a["Jt"]).max() < 1e-14


# ------------------------------------------------------------------ SAGE (step D1)

def test_sage_with_one_direction_is_rtr():
    """K = 1: the expectation step removes nothing, so one SAGE sweep is one RTR solve."""
    a = agent(7, K=1, noise=0.2)
    args = (a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"])
    Js = R.sage_jupdate(a["J0"], *args, n_sage=1, n_rtr=5, n_cg=4)
    Jr = R.rtr_jupdate(a["J0"], *args, n_rtr=5, n_cg=4)
    np.testing.assert_array_equal(Js, Jr)


def test_sage_is_block_coordinate_descent_on_the_lagrangian():
    """Every direction update lowers (never raises) the full L_i, because with the other
    directions fixed the single-direction Lagrangian of the expectation-step data differs
    from L_i by a constant."""
    a = agent(8, N=5, K=3, T=3, noise=0.3)
    args = (a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"])
    trace = []
    R.sage_jupdate(a["J0"], *args, n_sage=3, n_rtr=4, n_cg=4, trace=trace)
    L0 = O.aug_lagrangian(a["J0"], *args)
    seq = [L0] + trace
    assert all(b <= x * (1 + 1e-13) for x, b in zip(seq, seq[1:]))
    assert seq[-1] < 0.5 * L0


def test_sage_reaches_the_noise_free_minimiser():
    """Block-coordinate descent over coupled directions converges linearly (about 0.7 per sweep
    here): 30 sweeps bring every direction to the noise-free minimiser Jt."""
    a = agent(9, N=5, K=3, T=3)
    args = (a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"])
    J = R.sage_jupdate(a["J0"], *args, n_sage=30, n_rtr=6, n_cg=12)
    assert np.abs(J - a["Jt"]).max() < 1e-4


def test_sage_expectation_step_uses_the_other_directions_only():
    """A SAGE sweep that starts at Jt for every direction but the first one visited recovers that
    direction alone: its expectation step leaves exactly its own model in the data, and the later
    directions, already at Jt, stay there. Removing the direction's own model too (or leaving
    another's in) would pull it away from Jt."""
    a = agent(10, N=5, K=3, T=3)
    J0 = a["Jt"].copy()
    J0[0] += 0.2 * cn(np.random.default_rng(11), 5, 2, 2)
    args = (a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"])
    J = R.sage_jupdate(J0, *args, n_sage=1, n_rtr=30, n_cg=20)
    assert np.abs(J - a["Jt"]).max() < 1e-8


# ------------------------------------------------------------------ in C-ADMM (steps D1-D3)

def test_admm_with_rtr_and_sage_j_updates_behaves_like_simulation_one():
    """C-ADMM on the tiny noise-free problem (K = 1) with the paper's inner solver (RTR, 10
    iterations per ADMM iteration as in Simulation I): the objective and, after the first
    iteration, the primal residual fall; with K = 1 SAGE and RTR give the same history. On a
    two-direction problem, C-ADMM over SAGE sweeps lowers the objective too."""
    from synth import make_problem
    prob = make_problem("tiny_n8_k1", noise=False)
    prob = dict(prob, basis=prob["basis"][:, :2], M=2)

    def rtr(J, V, C, pq, Y, BZ, rho):
        return R.rtr_jupdate(J, V, C, pq, Y, BZ, rho, n_rtr=10, n_cg=4)

    def sage(J, V, C, pq, Y, BZ, rho):
        return R.sage_jupdate(J, V, C, pq, Y, BZ, rho, n_sage=1, n_rtr=10, n_cg=4)

    h_rtr = O.admm(prob, 6, jupdate=rtr)["hist"]
    h_sage = O.admm(prob, 6, jupdate=sage)["hist"]
    assert h_rtr["objective"][-1] < h_rtr["objective"][0]
    assert np.all(np.diff(h_rtr["primal"][1:]) <= 1e-12)
    for key in h_rtr:
        np.testing.assert_array_equal(h_rtr[key], h_sage[key])
    prob2 = make_problem("adjoint_n16_k3", N=6, K=2, P=4, I=1, T=2, seed=3)
    h2 = O.admm(prob2, 4, jupdate=sage)["hist"]
    assert h2["objective"][-1] < h2["objective"][0]


def test_lm_rtr_and_sage_j_updates_reach_the_same_c_admm_objective():
    """Two independent inner solvers (the LM/PCG of the GPU path and the paper's RTR, with SAGE
    over RTR) driving the same C-ADMM reach the same objective and data residual after 10
    iterations on a three-direction problem (16 stations, 4 samples; agreement within 2e-4 there,
    while with fewer constraints per parameter the solvers' paths still differ by a few 1e-3 at
    iteration 10): a mistake in either solver's step or acceptance rule would leave it elsewhere."""
    from synth import make_problem
    prob = make_problem("adjoint_n16_k3", N=16, K=3, P=8, I=1, T=4, seed=3)

    def rtr(J, V, C, pq, Y, BZ, rho):
        return R.rtr_jupdate(J, V, C, pq, Y, BZ, rho, n_rtr=10, n_cg=4)

    def sage(J, V, C, pq, Y, BZ, rho):
        return R.sage_jupdate(J, V, C, pq, Y, BZ, rho, n_sage=1, n_rtr=10, n_cg=4)

    h_lm = O.admm(prob, 10)["hist"]
    for ju in (rtr, sage):
        h = O.admm(prob, 10, jupdate=ju)["hist"]
        assert h["objective"][-1] == pytest.approx(h_lm["objective"][-1], rel=1e-3)
        assert h["resid_norm"][-1] == pytest.approx(h_lm["resid_norm"][-1], rel=1e-3)
