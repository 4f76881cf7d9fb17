"""Pins for the FP64 oracle: each checks it against something other than itself
(finite differences, a closed form, a least-squares brute force, an invariant, a
hand-derived value), chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them."""
import json
import math
import os

import numpy as np
import pytest

from oracle import admm as O
from synth import make_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def small_agent(seed=0, N=5, K=2, T=3, noise=True):
    """A single random agent with a random (not identity) operating point."""
    rng = np.random.default_rng(seed)
    pq = np.array([(p, q) for p in range(N) for q in range(p + 1, N)], dtype=np.int32)
    C = cn(rng, len(pq), T, K) * 2.0
    Jt = np.eye(2) + 0.3 * cn(rng, K, N, 2, 2)
    V = O.model_vis(Jt, C, pq)
    if noise:
        V = V + 0.2 * cn(rng, *V.shape)
    J = Jt + 0.2 * cn(rng, K, N, 2, 2)
    Y = 0.5 * cn(rng, K, N, 2, 2)
    BZ = np.eye(2) + 0.1 * cn(rng, K, N, 2, 2)
    rho = np.array([3.0, 0.7][:K] + [1.0] * max(0, K - 2))
    return dict(pq=pq, C=C, V=V, Jt=Jt, J=J, Y=Y, BZ=BZ, rho=rho, rng=rng)


# ------------------------------------------------------------------ hand-derived values

def test_two_station_hand_example():
    """Hand-derived values for N=2, one baseline, K=1, T=1 (tests/golden/two_station.json)."""
    with open(os.path.join(GOLDEN, "two_station.json")) as fh:
        gold = json.load(fh)
    pq = np.array([[0, 1]], dtype=np.int32)
    C = np.ones((1, 1, 1), dtype=complex)
    J = np.broadcast_to(np.eye(2, dtype=complex), (1, 2, 2, 2)).copy()
    V = 2.0 * np.eye(2, dtype=complex)[None, None]
    rho = np.array([gold["rho"]])
    Y = np.zeros_like(J)
    BZ = np.zeros_like(J)
    assert O.data_cost(J, V, C, pq) == pytest.approx(gold["g"])
    assert O.aug_lagrangian(J, V, C, pq, Y, BZ, rho) == pytest.approx(gold["L"])
    gd = O.grad_data(J, V, C, pq)
    np.testing.assert_allclose(gd[0, 0], np.array(gold["grad_g_p"]))
    np.testing.assert_allclose(gd[0, 1], np.array(gold["grad_g_q"]))
    np.testing.assert_allclose(O.grad_lagrangian(J, V, C, pq, Y, BZ, rho), 0.0, atol=1e-15)
    eta = np.zeros_like(J)
    eta[0, 0, 0, 0] = 1.0
    H = O.hess_gn(J, eta, C, pq)
    np.testing.assert_allclose(H[0, 0], np.array(gold["hess_gn_p"]))
    np.testing.assert_allclose(H[0, 1], np.array(gold["hess_gn_q"]))


# ------------------------------------------------------------------ gradient (Eq. gradL)

@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    """h(xi, grad L) = D L[xi] for random complex directions xi (Eq. grad, Eq. gradL)."""
    a = small_agent(seed)
    args = (a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"])
    grad = O.grad_lagrangian(a["J"], *args)
    rng = a["rng"]
    eps = 1e-6
    for _ in range(4):
        xi = cn(rng, *a["J"].shape)
        fd = (O.aug_lagrangian(a["J"] + eps * xi, *args) - O.aug_lagrangian(a["J"] - eps * xi, *args)) / (2 * eps)
        assert O.h_inner(xi, grad) == pytest.approx(fd, rel=1e-7, abs=1e-7)


def test_gradient_elementwise_real_and_imaginary():
    """Each real coordinate: dL/dRe(J_e) = 2 Re grad_e and dL/dIm(J_e) = 2 Im grad_e
    (the factor 2 comes from h = trace(xi^H eta + eta^H xi))."""
    a = small_agent(3, N=3, K=1, T=2)
    args = (a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"])
    grad = O.grad_lagrangian(a["J"], *args)
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (0, 1, 0, 1), (0, 2, 1, 0), (0, 2, 1, 1)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            e = np.zeros_like(a["J"])
            e[idx] = unit
            fd = (O.aug_lagrangian(a["J"] + eps * e, *args) - O.aug_lagrangian(a["J"] - eps * e, *args)) / (2 * eps)
            assert fd == pytest.approx(2 * part(grad[idx]), rel=1e-7, abs=1e-7)


# ------------------------------------------------------------------ Hessian (Eq. HessL)

def test_gn_hessian_equals_fd_of_gradient_at_zero_residual():
    """At zero residual (noise-free data at the truth) the Gauss-Newton Hessian is the
    full Hessian (Eq. hess), so central differences of grad L equal Hess L[eta]."""
    a = small_agent(4, noise=False)
    J = a["Jt"]
    args = (a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"])
    assert O.data_cost(J, a["V"], a["C"], a["pq"]) < 1e-20
    rng = a["rng"]
    eps = 1e-6
    for _ in range(3):
        eta = cn(rng, *J.shape)
        fd = (O.grad_lagrangian(J + eps * eta, *args) - O.grad_lagrangian(J - eps * eta, *args)) / (2 * eps)
        np.testing.assert_allclose(O.hess_lagrangian(J, eta, a["C"], a["pq"], a["rho"]), fd, rtol=1e-6, atol=1e-7)


def test_gn_hessian_is_self_adjoint_and_psd():
    """h(xi, H eta) = h(H xi, eta) and h(eta, H eta) >= 0: the sign the printed Hess g
    would violate at zero residual."""
    a = small_agent(5)
    rng = a["rng"]
    for _ in range(3):
        xi, eta = cn(rng, *a["J"].shape), cn(rng, *a["J"].shape)
        Hx = O.hess_gn(a["J"], xi, a["C"], a["pq"])
        He = O.hess_gn(a["J"], eta, a["C"], a["pq"])
        assert O.h_inner(xi, He) == pytest.approx(O.h_inner(Hx, eta), rel=1e-10)
        assert O.h_inner(eta, He) > 0


def test_jacobi_blocks_are_the_diagonal_of_the_dense_gn_hessian():
    """G_pk reproduces the (p,k) diagonal block of H_GN: H_GN[e_pk X] restricted to (p,k)
    equals X G_pk for every 2x2 complex X."""
    a = small_agent(6, N=4, K=2, T=3)
    J, C, pq = a["J"], a["C"], a["pq"]
    G = O.jacobi_blocks(J, C, pq)
    rng = a["rng"]
    for k in range(2):
        for p in range(4):
            X = cn(rng, 2, 2)
            eta = np.zeros_like(J)
            eta[k, p] = X
            H = O.hess_gn(J, eta, C, pq)
            np.testing.assert_allclose(H[k, p], X @ G[k, p], rtol=1e-10, atol=1e-12)


def test_single_station_newton_step_equals_lstsq():
    """With every other station fixed and K=1, g is linear least squares in J_p. The block
    Newton step J_p - grad_p G_p^-1 equals numpy's lstsq solution of the stacked system."""
    a = small_agent(7, N=4, K=1, T=4)
    J, C, V, pq = a["J"].copy(), a["C"], a["V"], a["pq"]
    p0 = 2
    grad = O.grad_data(J, V, C, pq)
    G = O.jacobi_blocks(J, C, pq)
    newton = J[0, p0] - grad[0, p0] @ np.linalg.inv(G[0, p0])
    # Stack rows: for baselines (p0,q): V = c J_p0 J_q^H  ->  rows of (c J_q^H)^T acting on J_p0^T
    rows_A, rows_b = [], []
    for b, (p, q) in enumerate(pq):
        for t in range(C.shape[1]):
            c = C[b, t, 0]
            if p == p0:   # V = c X J_q^H  ->  V^T = c conj(J_q) X^T
                rows_A.append(c * np.conj(J[0, q]))
                rows_b.append(V[b, t].T)
            elif q == p0:  # V = c J_p X^H  ->  V^* = conj(c) conj(J_p) X^T
                rows_A.append(np.conj(c) * np.conj(J[0, p]))
                rows_b.append(np.conj(V[b, t]))
    A = np.concatenate(rows_A, axis=0)
    rhs = np.concatenate(rows_b, axis=0)
    XT, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    np.testing.assert_allclose(newton, XT.T, rtol=1e-9, atol=1e-10)


# ------------------------------------------------------------------ invariants of g

def test_gauge_invariance():
    """g(J U) = g(J) for a unitary U per direction, because C = c I_2 (Eq. coh)."""
    a = small_agent(8)
    rng = a["rng"]
    J = a["J"]
    JU = J.copy()
    for k in range(J.shape[0]):
        U, _ = np.linalg.qr(cn(rng, 2, 2))
        JU[k] = J[k] @ U
    assert O.data_cost(JU, a["V"], a["C"], a["pq"]) == pytest.approx(O.data_cost(J, a["V"], a["C"], a["pq"]), rel=1e-12)


def test_trace_form_of_g_matches_norm_form():
    """Eq. sumtrace1 (trace of R^H R) equals the sum of squared moduli (Eq. sum3)."""
    a = small_agent(9)
    R = O.residual(a["J"], a["V"], a["C"], a["pq"])
    tr = sum(np.trace(R[b, t].conj().T @ R[b, t]).real for b in range(R.shape[0]) for t in range(R.shape[1]))
    assert O.data_cost(a["J"], a["V"], a["C"], a["pq"]) == pytest.approx(tr, rel=1e-12)


def test_model_matches_explicit_selection_matrices():
    """model_vis equals A_p J_k C_pqk (A_q J_k)^H built with explicit selection matrices (Eq. Ap)."""
    a = small_agent(10, N=3, K=2, T=2)
    J, C, pq = a["J"], a["C"], a["pq"]
    N = 3
    M = O.model_vis(J, C, pq)
    for b, (p, q) in enumerate(pq):
        Ap = np.zeros((2, 2 * N)); Ap[:, 2 * p:2 * p + 2] = np.eye(2)
        Aq = np.zeros((2, 2 * N)); Aq[:, 2 * q:2 * q + 2] = np.eye(2)
        for t in range(2):
            ref = sum(Ap @ J[k].reshape(2 * N, 2) @ (C[b, t, k] * np.eye(2)) @ (Aq @ J[k].reshape(2 * N, 2)).conj().T
                      for k in range(2))
            np.testing.assert_allclose(M[b, t], ref, rtol=1e-12)


# ------------------------------------------------------------------ PCG / LM

def test_pcg_reaches_the_dense_solution():
    """With as many PCG steps as unknowns, PCG solves (Hess L + mu) x = -grad exactly:
    compare with a dense solve of the real 8NK x 8NK system assembled column by column."""
    a = small_agent(11, N=3, K=2, T=3)
    J, C, pq, rho = a["J"], a["C"], a["pq"], a["rho"]
    grad = O.grad_lagrangian(J, a["V"], C, pq, a["Y"], a["BZ"], rho)
    G = O.jacobi_blocks(J, C, pq)
    mu = 0.37
    n = J.size
    cols = []
    for i in range(2 * n):
        e = np.zeros(n, dtype=complex)
        e[i // 2] = 1.0 if i % 2 == 0 else 1j
        e = e.reshape(J.shape)
        Ae = O.hess_lagrangian(J, e, C, pq, rho) + mu * e
        cols.append(np.stack([Ae.real.ravel(), Ae.imag.ravel()], 1).ravel())
    A = np.array(cols).T
    b = -np.stack([grad.real.ravel(), grad.imag.ravel()], 1).ravel()
    xd = np.linalg.solve(A, b)
    x, steps = O.pcg(J, C, pq, grad, G, rho, mu, 6 * n)  # past 2n: round-off slows finite termination
    np.testing.assert_allclose(np.stack([x.real.ravel(), x.imag.ravel()], 1).ravel(), xd, rtol=1e-6, atol=1e-9)


def test_lm_never_increases_the_lagrangian():
    a = small_agent(12)
    args = (a["V"], a["C"], a["pq"], a["Y"], a["BZ"], a["rho"])
    L0 = O.aug_lagrangian(a["J"], *args)
    J1 = O.lm_jupdate(a["J"], *args, n_lm=5, n_cg=3)
    L1 = O.aug_lagrangian(J1, *args)
    assert L1 < L0
    J2 = O.lm_jupdate(J1, *args, n_lm=5, n_cg=3)
    assert O.aug_lagrangian(J2, *args) <= L1


def test_lm_single_step_by_hand():
    """n_lm = n_cg = 1 from J on N=3, K=1: one preconditioned steepest-descent step
    x = alpha z, z = M^-1 (-grad), alpha = h(r,z)/h(z,Az), written out with dense 2x2 algebra."""
    a = small_agent(13, N=3, K=1, T=2)
    J, C, V, pq, Y, BZ, rho = a["J"], a["C"], a["V"], a["pq"], a["Y"], a["BZ"], a["rho"]
    grad = O.grad_lagrangian(J, V, C, pq, Y, BZ, rho)
    G = O.jacobi_blocks(J, C, pq)
    diag = max(max(G[0, p, 0, 0].real, G[0, p, 1, 1].real) for p in range(3)) + rho[0] / 2
    mu = 1e-3 * diag
    lam = rho[0] / 2 + mu
    z = np.stack([(-grad[0, p]) @ np.linalg.inv(G[0, p] + lam * np.eye(2)) for p in range(3)])[None]
    Az = O.hess_lagrangian(J, z, C, pq, rho) + mu * z
    alpha = O.h_inner(-grad, z) / O.h_inner(z, Az)
    x = alpha * z
    L0 = O.aug_lagrangian(J, V, C, pq, Y, BZ, rho)
    Lx = O.aug_lagrangian(J + x, V, C, pq, Y, BZ, rho)
    expected = J + x if Lx < L0 else J
    np.testing.assert_allclose(O.lm_jupdate(J, V, C, pq, Y, BZ, rho, n_lm=1, n_cg=1), expected, rtol=1e-12)


# ------------------------------------------------------------------ consensus (Eq. Zest, M3)

def test_z_update_equals_bruteforce_least_squares():
    """Eq. Zest equals min_Z sum_i ||B_i Z - (J_i + Y_i/rho)||^2 solved by lstsq on the
    materialised Kronecker B_f = b_f^T (x) I_2N (Eq. hblock)."""
    rng = np.random.default_rng(14)
    P, M, N, K = 6, 3, 4, 2
    freqs = np.linspace(115e6, 185e6, P)
    basis = np.stack([((freqs - 150e6) / 150e6) ** l for l in range(M)], 1)
    rho = np.array([2.0, 7.0])
    Js = [cn(rng, K, N, 2, 2) for _ in range(P)]
    Ys = [cn(rng, K, N, 2, 2) for _ in range(P)]
    Z = O.z_update(Js, Ys, basis, rho)
    for k in range(K):
        Bbig = np.concatenate([np.kron(basis[i][None, :], np.eye(2 * N)) for i in range(P)], 0)
        rhs = np.concatenate([(Js[i][k] + Ys[i][k] / rho[k]).reshape(2 * N, 2) for i in range(P)], 0)
        Zls, *_ = np.linalg.lstsq(Bbig, rhs, rcond=None)
        np.testing.assert_allclose(Z[k].reshape(M * 2 * N, 2), Zls, rtol=1e-10, atol=1e-12)
        # and the gradient of Eq. gradZ vanishes there
        gz = sum(np.kron(basis[i][None, :], np.eye(2 * N)).T @ (-Ys[i][k].reshape(2 * N, 2)
                 + rho[k] * (-Js[i][k].reshape(2 * N, 2) + np.kron(basis[i][None, :], np.eye(2 * N)) @ Zls))
                 for i in range(P))
        assert np.abs(gz).max() < 1e-9


def test_z_update_split_rhs_sums_to_the_same_z():
    """The fusion centre only needs the sum of per-agent contributions (steps S1/S2):
    splitting the agents into two groups and adding their right-hand sums gives Z."""
    rng = np.random.default_rng(15)
    P, M, N, K = 8, 4, 3, 1
    x = np.linspace(0, 1, P)
    basis = np.stack([math.comb(3, l) * x ** l * (1 - x) ** (3 - l) for l in range(M)], 1)
    rho = np.array([10.0])
    Js = [cn(rng, K, N, 2, 2) for _ in range(P)]
    Ys = [cn(rng, K, N, 2, 2) for _ in range(P)]
    rhs = O.z_rhs(Js[:3], Ys[:3], basis[:3], rho) + O.z_rhs(Js[3:], Ys[3:], basis[3:], rho)
    np.testing.assert_allclose(O.z_from_rhs(rhs, basis, rho), O.z_update(Js, Ys, basis, rho), rtol=1e-12)


def test_consensus_exact_when_p_equals_m():
    """With P = M the basis interpolates any J exactly, so after every iteration
    J_i = B_i Z and the dual variables stay zero (primal residual 0)."""
    prob = make_problem("tiny_n8_k1", P=3, N=5)
    res = O.admm(prob, 3, n_lm=3, n_cg=3)
    assert np.all(res["hist"]["primal"] < 1e-12)
    for Y in res["Y"].values():
        assert np.abs(Y).max() < 1e-10


def test_fixed_point_noise_free():
    """Noise-free data with a truth inside the basis span: starting from the truth the
    data residual stays at round-off and the solution does not move (Section 3)."""
    prob = make_problem("tiny_n8_k1", noise=False)
    Zfit = O.z_update([prob["J_true"][f] for f in range(prob["P"])],
                      [np.zeros_like(prob["J_true"][0])] * prob["P"], prob["basis"], prob["rho"])
    np.testing.assert_allclose(O.bz(Zfit, prob["basis"][1]), prob["J_true"][1], atol=1e-12)
    res = O.admm(prob, 3, n_lm=3, n_cg=3, J0=prob["J_true"], Z0=[Zfit])
    assert res["hist"]["resid_norm"].max() < 1e-9
    for a, J in res["J"].items():
        np.testing.assert_allclose(J, prob["J_true"][a], atol=1e-9)


def test_procrustes_recovers_a_known_unitary():
    rng = np.random.default_rng(16)
    Jref = cn(rng, 6, 2, 2)
    U, _ = np.linalg.qr(cn(rng, 2, 2))
    Ja = Jref @ U.conj().T
    np.testing.assert_allclose(Ja @ O.procrustes_unitary(Ja, Jref), Jref, atol=1e-12)
    # and it beats random unitaries on noisy data
    Jn = Ja + 0.1 * cn(rng, 6, 2, 2)
    best = np.linalg.norm(Jref - Jn @ O.procrustes_unitary(Jn, Jref))
    for _ in range(50):
        W, _ = np.linalg.qr(cn(rng, 2, 2))
        assert np.linalg.norm(Jref - Jn @ W) >= best - 1e-12


def test_gauge_alignment_keeps_the_lagrangian_at_zero_consensus():
    """At the first iteration Z = Y = 0, so rotating J_k by a unitary leaves L_i unchanged."""
    a = small_agent(17)
    Z0 = np.zeros_like(a["J"])
    rho = a["rho"]
    L0 = O.aug_lagrangian(a["J"], a["V"], a["C"], a["pq"], Z0, Z0, rho)
    J2 = O.gauge_align([a["J"], a["Jt"]], 1)[0]
    assert O.aug_lagrangian(J2, a["V"], a["C"], a["pq"], Z0, Z0, rho) == pytest.approx(L0, rel=1e-12)


def test_admm_decreases_primal_and_objective_on_tiny_noise_free():
    """Noise-free, truth one degree above the basis: the primal residual and the
    objective fall over the iterations, and the dual residual falls after the first
    (Section 4: Simulation I behaviour)."""
    prob = make_problem("tiny_n8_k1", noise=False)
    prob = dict(prob, basis=prob["basis"][:, :2], M=2)
    res = O.admm(prob, 8, n_lm=5, n_cg=4)
    h = res["hist"]
    assert np.all(np.diff(h["primal"]) <= 1e-15)
    assert h["objective"][-1] < h["objective"][0]
    assert h["dual"][-1] < h["dual"][1]


# ------------------------------------------------------------------ predict (Eq. coh)

def _rand_geom(seed, T=3, N=4, K=2, S=3):
    rng = np.random.default_rng(seed)
    uvw = rng.normal(0, 2000.0, (T, N, 3))
    sky = np.zeros((K, S, 4))
    sky[..., 0] = rng.uniform(-0.05, 0.05, (K, S))
    sky[..., 1] = rng.uniform(-0.05, 0.05, (K, S))
    sky[..., 2] = rng.uniform(1, 10, (K, S))
    sky[..., 3] = rng.uniform(-1, 1, (K, S))
    pq = np.array([(p, q) for p in range(N) for q in range(p + 1, N)], dtype=np.int32)
    return uvw, sky, pq


def test_predict_phase_centre_and_zero_baseline_give_the_flux():
    uvw, sky, pq = _rand_geom(18)
    f, f0 = 140e6, 150e6
    flux = (sky[..., 2] * (f / f0) ** sky[..., 3]).sum(-1)
    sky0 = sky.copy(); sky0[..., :2] = 0.0
    C = O.predict_coherencies(uvw, sky0, f, f0, pq)
    np.testing.assert_allclose(C, np.broadcast_to(flux, C.shape), rtol=1e-13)
    uvw_same = np.broadcast_to(uvw[:, :1], uvw.shape).copy()
    C = O.predict_coherencies(uvw_same, sky, f, f0, pq)
    np.testing.assert_allclose(C, np.broadcast_to(flux, C.shape), rtol=1e-13)


def test_predict_reversed_baseline_conjugates():
    uvw, sky, pq = _rand_geom(19)
    C = O.predict_coherencies(uvw, sky, 160e6, 150e6, pq)
    Cr = O.predict_coherencies(uvw, sky, 160e6, 150e6, pq[:, ::-1].copy())
    np.testing.assert_allclose(Cr, np.conj(C), rtol=1e-12)


def test_predict_single_source_phase_is_linear_in_u_times_l():
    """One source, w = 0: the phase of c is -2 pi f/c (u l + v m) modulo 2 pi, so a shift of l
    by c/(f u) on a pure-u baseline leaves c unchanged, and half that shift flips its sign."""
    f = 150e6
    lam = 299792458.0 / f
    uvw = np.zeros((1, 2, 3))
    uvw[0, 0, 0] = 300.0 * lam  # 300 wavelengths
    pq = np.array([[0, 1]], dtype=np.int32)
    sky = np.array([[[0.01, 0.0, 2.0, 0.0]]])
    c0 = O.predict_coherencies(uvw, sky, f, f, pq)[0, 0, 0]
    sky1 = sky.copy(); sky1[0, 0, 0] += 1.0 / 300.0
    sky1[0, 0, 1] = 0.0
    # keep n fixed by compensating m is not needed: w = 0
    c1 = O.predict_coherencies(uvw, sky1, f, f, pq)[0, 0, 0]
    sky2 = sky.copy(); sky2[0, 0, 0] += 0.5 / 300.0
    c2 = O.predict_coherencies(uvw, sky2, f, f, pq)[0, 0, 0]
    assert c1 == pytest.approx(c0, rel=1e-9)
    assert c2 == pytest.approx(-c0, rel=1e-9)
    assert np.angle(c0) == pytest.approx(math.remainder(-2 * math.pi * 300.0 * 0.01, 2 * math.pi), abs=1e-9)


def test_predict_agrees_with_the_generator_s_factorised_simulation():
    """The oracle's per-baseline phase and the generator's per-station phasor product
    (written separately) agree: a transposed index or sign in either would show."""
    from synth.lofar import simulate_coherencies
    uvw, sky, pq = _rand_geom(20)
    f = 170e6
    a = O.predict_coherencies(uvw, sky, f, 150e6, pq)
    b = simulate_coherencies(uvw, sky, f, pq)
    np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-9)


# ------------------------------------------------------------------ residual and correction (Section 2)

def test_residual_of_noise_free_data_at_the_true_solutions_is_zero():
    """Subtracting every direction's model at the solutions that generated noise-free data
    leaves nothing; a transposed or unconjugated station product, or a dropped direction,
    leaves the model behind."""
    a = small_agent(40, N=5, K=3, T=2, noise=False)
    R = O.corrected_residual(a["Jt"], a["V"], a["C"], a["pq"])
    assert np.abs(R).max() < 1e-12 * np.abs(a["V"]).max()
    # the same with correction by any direction: J^-1 0 J^-H = 0
    R = O.corrected_residual(a["Jt"], a["V"], a["C"], a["pq"], correct=2)
    assert np.abs(R).max() < 1e-11 * np.abs(a["V"]).max()


def test_correcting_one_direction_s_data_returns_its_coherency():
    """K = 2, data of both directions, direction 1 subtracted, the rest corrected by
    direction 0: J_p0^-1 (J_p0 c_0 J_q0^H) J_q0^-H = c_0 I_2 for every baseline and sample.
    Subtracting the wrong direction, correcting by the wrong one, or applying the
    inverse on the wrong side fails."""
    a = small_agent(41, N=4, K=2, T=3, noise=False)
    R = O.corrected_residual(a["Jt"], a["V"], a["C"], a["pq"], subtract=[False, True], correct=0)
    ref = a["C"][:, :, 0, None, None] * np.eye(2)
    np.testing.assert_allclose(R, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    wrong = O.corrected_residual(a["Jt"], a["V"], a["C"], a["pq"], subtract=[True, False], correct=0)
    assert np.abs(wrong - ref).max() > 1e-3


def test_residual_with_identity_solutions_is_coherency_subtraction():
    """J = I: the model of direction k is c_k I_2, so the residual is V - sum_k c_k I_2 and the
    correction changes nothing."""
    a = small_agent(42, N=4, K=3, T=2)
    Jid = np.broadcast_to(np.eye(2), a["Jt"].shape).astype(complex)
    R = O.corrected_residual(Jid, a["V"], a["C"], a["pq"], subtract=[True, False, True], correct=1)
    ref = a["V"] - (a["C"][:, :, 0] + a["C"][:, :, 2])[..., None, None] * np.eye(2)
    np.testing.assert_allclose(R, ref, rtol=1e-13, atol=1e-13)


def test_correction_by_unitary_solutions_keeps_the_norm():
    """Unitary J: J^-1 = J^H, so the correction preserves each 2x2 block's Frobenius norm;
    with nothing subtracted, the corrected data of a unitary gauge equal the data rotated back."""
    a = small_agent(43, N=4, K=2, T=2)
    rng = np.random.default_rng(44)
    U = np.linalg.qr(cn(rng, 2, 4, 2, 2))[0]
    R = O.corrected_residual(U, a["V"], a["C"], a["pq"], subtract=[False, False], correct=1)
    np.testing.assert_allclose(np.linalg.norm(R, axis=(-2, -1)), np.linalg.norm(a["V"], axis=(-2, -1)), rtol=1e-12)
    p, q = a["pq"][:, 0], a["pq"][:, 1]
    back = np.einsum("bji,btjk,bkl->btil", U[1, p].conj(), a["V"], U[1, q])
    np.testing.assert_allclose(R, back, rtol=1e-12, atol=1e-12)
