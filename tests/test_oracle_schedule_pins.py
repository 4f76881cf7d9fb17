"""Pins for the two oracle parts that the other pins only touch at their first step:

* the Levenberg-Marquardt damping schedule of lm_jupdate (Madsen, Nielsen and Tingleff 2004,
  "Methods for non-linear least squares problems", Section 3.2: mu0 = tau max diag, the gain
  ratio, Nielsen's update mu <- mu max(1/3, 1 - (2 ratio - 1)^3), nu <- 2 on acceptance, and
  mu <- mu nu, nu <- 2 nu on rejection), followed over several steps with rejections;
* the per-iteration records of admm (Section 4: primal residual ||J_i - B_i Z|| / sqrt(4N)
  averaged over agents and directions, dual residual ||Z^{n+1} - Z^n|| / sqrt(4MN) averaged over
  directions, the objective after the Y-update of Eq. M3), on a case small enough to work out by hand.

The LM reference below is written independently of the oracle: it works in real coordinates,
builds the residual with explicit loops, takes its Jacobian by central differences (exact here,
since the model is bilinear in the Jones matrices) and solves the damped Gauss-Newton system
densely, which the oracle's PCG reaches when it is given more steps than unknowns.
"""
import math

import numpy as np
import pytest

from oracle import admm as O


# ------------------------------------------------------------------ LM damping schedule

def _cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def _lm_case(seed):
    """N=3 stations, K=1, T=3: noisy data of a random truth, started far from it."""
    rng = np.random.default_rng(seed)
    N, K, T = 3, 1, 3
    pq = np.array([(0, 1), (0, 2), (1, 2)], dtype=np.int32)
    C = 2.0 * _cn(rng, len(pq), T, K)
    Jtrue = np.eye(2) + 0.8 * _cn(rng, K, N, 2, 2)
    V = np.zeros((len(pq), T, 2, 2), dtype=complex)
    for b, (p, q) in enumerate(pq):
        for t in range(T):
            V[b, t] = C[b, t, 0] * Jtrue[0, p] @ Jtrue[0, q].conj().T
    V += 0.3 * _cn(rng, *V.shape)
    J0 = np.broadcast_to(np.eye(2, dtype=complex), (K, N, 2, 2)).copy() + 1.5 * _cn(rng, K, N, 2, 2)
    Y = 0.4 * _cn(rng, K, N, 2, 2)
    BZ = np.eye(2) + 0.2 * _cn(rng, K, N, 2, 2)
    rho = np.array([0.5])
    return dict(pq=pq, C=C, V=V, J0=J0, Y=Y, BZ=BZ, rho=rho, shape=(K, N, 2, 2))


def _theta(J):
    return np.ascontiguousarray(J).view(np.float64).ravel().copy()


def _jones(theta, shape):
    return theta.view(np.complex128).reshape(shape)


def _residual(theta, c):
    """Real vector of V_pq,t - sum_k c J_pk J_qk^H, explicit loops (Eq. vispq)."""
    J = _jones(theta, c["shape"])
    out = []
    for b, (p, q) in enumerate(c["pq"]):
        for t in range(c["V"].shape[1]):
            M = c["V"][b, t].copy()
            for k in range(J.shape[0]):
                M -= c["C"][b, t, k] * (J[k, p] @ J[k, q].conj().T)
            out.append(M)
    return np.ascontiguousarray(np.array(out)).view(np.float64).ravel()


def _lagrangian(theta, c):
    """L = r.r + y.(theta - b) + rho/2 |theta - b|^2 in real coordinates (Eq. sumtrace2, K = 1)."""
    r = _residual(theta, c)
    d = theta - _theta(c["BZ"])
    return float(r @ r + _theta(c["Y"]) @ d + 0.5 * c["rho"][0] * d @ d)


def _jacobian(theta, c):
    n = theta.size
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append((_residual(theta + e, c) - _residual(theta - e, c)) / 2.0)
    return np.stack(cols, axis=1)


def _dense_lm(c, n_lm):
    """The published LM iteration with the damped Gauss-Newton system solved densely.

    In the inner product h(a, b) = 2 a.b of real coordinates, the gradient is half the real
    one and the Gauss-Newton Hessian is Jr^T Jr + rho/2 (the real one halved). Returns one
    record per step (mu and nu the step was solved with, L, the trial L, pred, accepted)
    and the final point.
    """
    rho = c["rho"][0]
    th = _theta(c["J0"])
    y, b = _theta(c["Y"]), _theta(c["BZ"])
    L = _lagrangian(th, c)

    def model(th):
        Jr = _jacobian(th, c)
        r = _residual(th, c)
        g_h = 0.5 * (2.0 * Jr.T @ r + y + rho * (th - b))
        H_h = Jr.T @ Jr + 0.5 * rho * np.eye(th.size)
        return g_h, H_h

    g_h, H_h = model(th)
    mu = 1e-3 * float(np.max(np.diag(H_h)))
    nu = 2.0
    recs = []
    for _ in range(n_lm):
        x = np.linalg.solve(H_h + mu * np.eye(th.size), -g_h)
        pred = -(2.0 * x @ g_h + x @ H_h @ x)
        Lt = _lagrangian(th + x, c)
        acc = bool(pred > 0.0 and math.isfinite(Lt) and Lt < L)
        recs.append(dict(mu=mu, nu=nu, L=L, Lt=Lt, pred=pred, accepted=acc))
        if acc:
            ratio = (L - Lt) / pred
            th, L = th + x, Lt
            g_h, H_h = model(th)
            mu *= max(1.0 / 3.0, 1.0 - (2.0 * ratio - 1.0) ** 3)
            nu = 2.0
        else:
            mu *= nu
            nu *= 2.0
    return recs, _jones(th, c["shape"])


SEED, N_LM = 22, 10


def test_the_schedule_case_exercises_every_branch():
    """The fixed case rejects, accepts with a gain ratio where the cubic matters, and rejects
    again after an acceptance that followed a rejection (so nu must have been reset)."""
    recs, _ = _dense_lm(_lm_case(SEED), N_LM)
    acc = [r["accepted"] for r in recs]
    assert not acc[0] or any(not a for a in acc[1:])
    ratios = [(r["L"] - r["Lt"]) / r["pred"] for r in recs if r["accepted"]]
    # 1 - (2 ratio - 1)^3 > 1/3 and ratio not 1/2: another exponent gives another mu
    assert any(0.05 < q < 0.93 and abs(q - 0.5) > 0.02 for q in ratios)
    reset_seen = any(not acc[i] and acc[i + 1] and not acc[i + 2] for i in range(len(acc) - 2))
    assert reset_seen, acc


def test_lm_damping_sequence_matches_the_published_schedule():
    """mu, nu, the accept decisions, L and the final J of lm_jupdate equal those of the dense
    reference step by step (PCG given three times as many steps as there are unknowns)."""
    c = _lm_case(SEED)
    ref, J_ref = _dense_lm(c, N_LM)
    trace = []
    J = O.lm_jupdate(c["J0"], c["V"], c["C"], c["pq"], c["Y"], c["BZ"], c["rho"], N_LM, 72, trace=trace)
    assert len(trace) == N_LM
    for i, (t, r) in enumerate(zip(trace, ref)):
        assert t["accepted"] == r["accepted"], i
        assert t["mu"] == pytest.approx(r["mu"], rel=1e-7), i
        assert t["nu"] == r["nu"], i
        assert t["L"] == pytest.approx(r["L"], rel=1e-10), i
        assert t["pred"] == pytest.approx(r["pred"], rel=1e-6), i
    np.testing.assert_allclose(J, J_ref, rtol=0, atol=1e-7)


def test_first_damping_is_tau_times_the_largest_diagonal_by_hand():
    """mu0 = 1e-3 max_(p,k,j) (G_pk[j][j] + rho/2) with G_pk = sum_o s_po J_o^H J_o: for J = I
    every diagonal entry is sum_o s_po, the summed |c|^2 of station p's baselines."""
    c = _lm_case(SEED)
    c["J0"] = np.broadcast_to(np.eye(2, dtype=complex), c["shape"]).copy()
    s = np.sum(np.abs(c["C"][:, :, 0]) ** 2, axis=1)  # per baseline (0,1), (0,2), (1,2)
    per_station = [s[0] + s[1], s[0] + s[2], s[1] + s[2]]
    trace = []
    O.lm_jupdate(c["J0"], c["V"], c["C"], c["pq"], c["Y"], c["BZ"], c["rho"], 1, 4, trace=trace)
    assert trace[0]["mu"] == pytest.approx(1e-3 * (max(per_station) + 0.25), rel=1e-12)
    assert trace[0]["nu"] == 2.0


# ------------------------------------------------------------------ Section 4 records by hand

def _fixed_jupdate(alpha):
    """A J-update that returns alpha[i][k] * I for agent i, which it reads from its data
    (the first visibility entry of agent i is i + 1)."""
    def f(J, V, C, pq, Y, BZ, rho):
        i = int(round(V[0, 0, 0, 0].real)) - 1
        out = np.zeros_like(J)
        for k in range(J.shape[0]):
            out[k] = alpha[i][k] * np.eye(2)
        return out
    return f


def test_admm_records_follow_the_section_4_definitions_by_hand():
    """N=2, K=2, P=3 agents at x = -1, 0, 1, basis (1, x) (M=2), rho = (1, 2), coherencies zero,
    and a J-update that returns J_ik = alpha_ik I with alpha = [[1, 3], [2, 3], [4, 6]].

    Iteration 1 (Z = Y = 0): Z_k0 = mean_i alpha_ik I, Z_k1 = (alpha_3k - alpha_1k)/2 I, so
    B_i Z - J_i = -d_ik I with d = (1/6, -1/3, 1/6) for k=0 and (1/2, -1, 1/2) for k=1; a block
    d I over 2 stations has norm 2|d|.
      primal = mean_(i,k) 2|d_ik| / sqrt(4N)           = (16/3)/6 / sqrt(8)
      dual   = mean_k ||Z_k|| / sqrt(4MN), ||Z_k|| = 2 sqrt(z0^2 + z1^2)
             = (sqrt(277)/3 + sqrt(73)) / 2 / 4
      Y = rho d I, so each (i,k) adds Re tr(Y^H D) + rho/2 ||D||^2 = 4 rho d^2 + 2 rho d^2:
      objective = g + 1 + 18 with g = 1 + 4 + 9 (one visibility entry i+1 per agent).
    Iteration 2: the least-squares residual is orthogonal to the basis, so Z does not move
    (dual 0) and the primal is unchanged; Y = 2 rho d I gives 10 rho d^2 per (i,k).
    """
    N, K, P, M = 2, 2, 3, 2
    x = np.array([-1.0, 0.0, 1.0])
    basis = np.stack([np.ones(3), x], axis=1)
    V = np.zeros((P, 1, 1, 2, 2), dtype=complex)
    for i in range(P):
        V[i, 0, 0, 0, 0] = i + 1
    prob = dict(N=N, K=K, P=P, M=M, I=1, basis=basis, rho=np.array([1.0, 2.0]),
                pq=np.array([[0, 1]], dtype=np.int32), flags=np.zeros((P, 1), dtype=np.uint8),
                V=V, C=np.zeros((P, 1, 1, K), dtype=complex))
    alpha = [[1.0, 3.0], [2.0, 3.0], [4.0, 6.0]]
    h = O.admm(prob, 2, jupdate=_fixed_jupdate(alpha))["hist"]

    primal = (16.0 / 3.0) / 6.0 / math.sqrt(4 * N)
    dual = (math.sqrt(277.0) / 3.0 + math.sqrt(73.0)) / 2.0 / math.sqrt(4 * M * N)
    assert h["primal"][0] == pytest.approx(primal, rel=1e-12)
    assert h["dual"][0] == pytest.approx(dual, rel=1e-12)
    assert h["objective"][0] == pytest.approx(14.0 + 1.0 + 18.0, rel=1e-12)
    assert h["resid_norm"][0] == pytest.approx(math.sqrt(14.0), rel=1e-12)
    assert h["primal"][1] == pytest.approx(primal, rel=1e-12)
    assert h["dual"][1] == pytest.approx(0.0, abs=1e-14)
    assert h["objective"][1] == pytest.approx(14.0 + 10.0 / 6.0 + 30.0, rel=1e-12)
