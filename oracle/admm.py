"""FP64 CPU oracle for consensus-ADMM calibration across frequency (Yatawatta 2015).

TEST INFRASTRUCTURE. This module is the slow, plain reference that the CUDA path is
checked against. Only the test suite, the package smoke check and the benchmark's
CPU-baseline leg may import it; the library itself never does, and it shares no
code, constants or helpers with the CUDA sources.

Every function states the passage it follows. Where the paper is silent or garbled
the adopted reading is stated at the function:

* The augmented Lagrangian uses the appendix form (Eq. sumtrace2),
  Re tr(Y^H (J - BZ)) + rho/2 ||J - BZ||^2, not the norm printed in Eq. AugL.
* The printed Hess g (Section 3, the expression after Eq. HessL) has its overall
  sign flipped; the Gauss-Newton part used here is the R-free part of the
  derivative of grad g, following the Hessian definition of Eq. hess.
* The sum over p,q runs over unordered pairs p<q (N(N-1)/2 baselines, Section 3),
  and the sum over the samples of a solution interval is part of g (Section 2).
* All K directions are fitted jointly (M1 taken literally over the full model
  sum_k J_pk C_pqk J_qk^H); the inner solver is Levenberg-Marquardt with a
  preconditioned conjugate-gradient step in place of RTR.
* First C-ADMM iteration: each agent's J_k is rotated by the 2x2 Procrustes
  unitary towards the agent at the median frequency index before the Z average
  (Section 3, initialisation paragraph).

Parity status: all functions are pinned by tests in tests/test_oracle_pins.py
(finite differences, closed forms, least-squares brute force, invariants and
hand-derived values) and tests/test_oracle_schedule_pins.py (the LM damping
schedule over several steps against an independent dense LM, and the Section 4
records of admm worked out by hand), except the physical-accuracy claims of the
paper's figures, which print no numbers.

Shapes (per agent, complex128): J, Y, BZ [K,N,2,2]; V [B,T,2,2]; C [B,T,K] with the
coherency matrix c * I_2 (Eq. coh); pq int [B,2] with p<q.
"""
from __future__ import annotations

import math

import numpy as np

C_LIGHT = 299792458.0


def herm(X: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(X, -1, -2))


def h_inner(xi: np.ndarray, eta: np.ndarray) -> float:
    """Inner product h(xi, eta) = trace(xi^H eta + eta^H xi) (Appendix A, Eq. inprod)."""
    return 2.0 * float(np.real(np.vdot(xi, eta)))


# ----------------------------------------------------------------------------- data model

def predict_coherencies(uvw_t: np.ndarray, sky: np.ndarray, f: float, f0: float,
                        pq: np.ndarray) -> np.ndarray:
    """Scalar coherencies c[b,t,k] of unpolarised point-source clusters (Eq. coh).

    Reading of the phase the paper leaves unstated: for baseline pq with
    (u,v,w)_pq = (u,v,w)_p - (u,v,w)_q in metres,
    phi = -2 pi (f/c) (u_pq l + v_pq m + w_pq (sqrt(1-l^2-m^2) - 1)), and a source's
    intensity is I0 (f/f0)^alpha (Section 4). A cluster's c sums its sources.
    uvw_t: [T,N,3]; sky: [K,S,4] = (l, m, I0, alpha).
    """
    p, q = pq[:, 0], pq[:, 1]
    d = uvw_t[:, p, :] - uvw_t[:, q, :]  # [T,B,3]
    K = sky.shape[0]
    out = np.zeros((len(pq), uvw_t.shape[0], K), dtype=complex)
    for k in range(K):
        l, m, I0, alpha = sky[k, :, 0], sky[k, :, 1], sky[k, :, 2], sky[k, :, 3]
        nm1 = np.sqrt(1.0 - l * l - m * m) - 1.0
        phi = -2.0 * math.pi * (f / C_LIGHT) * (d[..., 0:1] * l + d[..., 1:2] * m + d[..., 2:3] * nm1)
        flux = I0 * (f / f0) ** alpha
        out[:, :, k] = np.sum(flux * np.exp(1j * phi), axis=-1).T
    return out


def model_vis(J: np.ndarray, C: np.ndarray, pq: np.ndarray) -> np.ndarray:
    """sum_k J_pk C_pqk J_qk^H for every baseline and sample (Eq. vispq without noise)."""
    p, q = pq[:, 0], pq[:, 1]
    P_k = np.matmul(J[:, p], herm(J[:, q]))  # [K,B,2,2]
    return np.einsum("btk,kbij->btij", C, P_k)


def residual(J, V, C, pq):
    return V - model_vis(J, C, pq)


def corrected_residual(J, V, C, pq, subtract=None, correct=None):
    """Residual visibilities after calibration, optionally corrected (Section 2: the solutions
    correct the data, and the residual is the data minus the predicted model).

    R_pq = V_pq - sum_{k in subtract} J_pk C_pqk J_qk^H, with subtract a boolean mask [K]
    (None: every direction). With correct = k0 the residual is then corrected by that
    direction's solutions, R_pq <- J_pk0^{-1} R_pq J_qk0^{-H}. Reading of the paper's order:
    correcting the data first and subtracting the corrected model gives the same matrix,
    because the correction is linear.
    """
    K = J.shape[0]
    sub = np.ones(K, dtype=bool) if subtract is None else np.asarray(subtract, dtype=bool)
    R = V - model_vis(J[sub], C[:, :, sub], pq)
    if correct is not None:
        p, q = pq[:, 0], pq[:, 1]
        left = np.linalg.inv(J[correct, p])           # [B,2,2]
        right = herm(np.linalg.inv(J[correct, q]))    # [B,2,2]
        R = np.einsum("bij,btjk,bkl->btil", left, R, right)
    return R


def data_cost(J, V, C, pq) -> float:
    """g(J) = sum_t sum_{p<q} ||V_pq - sum_k J_pk C_pqk J_qk^H||^2 (Eq. mltheta / Eq. sum3)."""
    return float(np.sum(np.abs(residual(J, V, C, pq)) ** 2))


def penalty(J, Y, BZ, rho) -> float:
    """0.5 tr(Y^H D + D^H Y) + rho/2 tr(D^H D), D = J - BZ, per direction (Eq. sumtrace2)."""
    total = 0.0
    for k in range(J.shape[0]):
        D = J[k] - BZ[k]
        total += 0.5 * (h_inner(Y[k], D)) + 0.5 * rho[k] * float(np.sum(np.abs(D) ** 2))
    return total


def aug_lagrangian(J, V, C, pq, Y, BZ, rho) -> float:
    """L_i(J, Z, Y) = g(J) + Re tr(Y^H (J - BZ)) + rho/2 ||J - BZ||^2 (Eq. sumtrace2)."""
    return data_cost(J, V, C, pq) + penalty(J, Y, BZ, rho)


def grad_data(J, V, C, pq) -> np.ndarray:
    """grad_i(g, J) of Section 3 (the expression after Eq. HessL), per station and direction:

    station p receives -sum_t conj(c) R_pq J_q   (the A_p^T (...) A_q J C^H term),
    station q receives -sum_t c R_pq^H J_p       (the A_q^T (...)^H A_p J C term),
    with R_pq = V_pq - sum_k J_pk C_pqk J_qk^H. Gradient w.r.t. the inner product h.
    """
    p, q = pq[:, 0], pq[:, 1]
    R = residual(J, V, C, pq)
    G = np.zeros_like(J)
    to_p = -np.einsum("btk,btij,kbjl->kbil", np.conj(C), R, J[:, q], optimize=True)
    to_q = -np.einsum("btk,btij,kbjl->kbil", C, herm(R), J[:, p], optimize=True)
    np.add.at(G, (slice(None), p), to_p)
    np.add.at(G, (slice(None), q), to_q)
    return G


def grad_lagrangian(J, V, C, pq, Y, BZ, rho) -> np.ndarray:
    """grad_i(L_i, J) = grad_i(g, J) + Y/2 + rho/2 (J - BZ) (Eq. gradL)."""
    r = rho[:, None, None, None]
    return grad_data(J, V, C, pq) + 0.5 * Y + 0.5 * r * (J - BZ)


def hess_gn(J, eta, C, pq) -> np.ndarray:
    """Gauss-Newton part of Hess g[eta] (Eq. hess applied to grad g, R-dependent terms dropped).

    With dM = sum_k c (eta_pk J_qk^H + J_pk eta_qk^H), station p receives
    sum_t conj(c) dM J_q and station q receives sum_t c dM^H J_p. This is the
    derivative of the expression for grad g with the residual's own change kept and
    the R eta terms removed; the printed Hess g carries the opposite overall sign.
    """
    p, q = pq[:, 0], pq[:, 1]
    Q = np.matmul(eta[:, p], herm(J[:, q])) + np.matmul(J[:, p], herm(eta[:, q]))  # [K,B,2,2]
    dM = np.einsum("btk,kbij->btij", C, Q)
    H = np.zeros_like(J)
    to_p = np.einsum("btk,btij,kbjl->kbil", np.conj(C), dM, J[:, q], optimize=True)
    to_q = np.einsum("btk,btij,kbjl->kbil", C, herm(dM), J[:, p], optimize=True)
    np.add.at(H, (slice(None), p), to_p)
    np.add.at(H, (slice(None), q), to_q)
    return H


def hess_lagrangian(J, eta, C, pq, rho) -> np.ndarray:
    """Hess_i(L_i, J, eta) = Hess g[eta] + rho/2 eta (Eq. HessL), with the GN Hess g."""
    return hess_gn(J, eta, C, pq) + 0.5 * rho[:, None, None, None] * eta


def jacobi_blocks(J, C, pq) -> np.ndarray:
    """Diagonal blocks of the GN Hessian: eta_pk -> eta_pk G_pk with
    G_pk = sum over baselines b incident on p of (sum_t |c_btk|^2) J_ok^H J_ok,
    o the other station of b. Returns G [K,N,2,2] (Hermitian)."""
    p, q = pq[:, 0], pq[:, 1]
    s = np.sum(np.abs(C) ** 2, axis=1).T  # [K,B]
    X = np.matmul(herm(J), J)  # [K,N,2,2]
    G = np.zeros(J.shape, dtype=complex)
    np.add.at(G, (slice(None), p), s[:, :, None, None] * X[:, q])
    np.add.at(G, (slice(None), q), s[:, :, None, None] * X[:, p])
    return G


# ----------------------------------------------------------------------------- J-update (M1)

def pcg(J, C, pq, grad, G, rho, mu, n_cg):
    """n_cg preconditioned CG steps on (Hess L + mu) x = -grad from x = 0.

    Preconditioner: x_pk -> x_pk (G_pk + (rho_k/2 + mu) I)^-1. Inner products use h.
    Stops updating when r^T z <= 0 or p^T A p <= 0. Returns (x, steps_taken).
    """
    lam = 0.5 * rho + mu
    Minv = np.linalg.inv(G + lam[:, None, None, None] * np.eye(2))

    def apply_A(v):
        return hess_lagrangian(J, v, C, pq, rho) + mu * v

    def apply_M(v):
        return np.matmul(v, Minv)

    b = -grad
    x = np.zeros_like(grad)
    r = b.copy()
    z = apply_M(r)
    d = z.copy()
    rz = h_inner(r, z)
    steps = 0
    for _ in range(n_cg):
        if not rz > 0.0:
            break
        Ad = apply_A(d)
        dAd = h_inner(d, Ad)
        if not dAd > 0.0:
            break
        alpha = rz / dAd
        x = x + alpha * d
        r = r - alpha * Ad
        z = apply_M(r)
        rz_new = h_inner(r, z)
        d = z + (rz_new / rz) * d
        rz = rz_new
        steps += 1
    return x, steps


LM_TAU = 1e-3


def lm_jupdate(J0, V, C, pq, Y, BZ, rho, n_lm, n_cg, stats=None, trace=None):
    """Minimise L_i(J, Z^n, Y^n) over J (Eq. M1) by n_lm Levenberg-Marquardt steps.

    Each step: PCG solve of the damped GN system, predicted decrease from the
    undamped quadratic model -h(x, grad) - 1/2 h(x, Hess L[x]), gain ratio
    (L(J) - L(J+x)) / pred, accept when pred > 0 and L(J+x) < L(J) (finite),
    Nielsen damping update mu *= max(1/3, 1-(2 ratio-1)^3) on accept, mu *= nu,
    nu *= 2 on reject. mu0 = 1e-3 * max_{p,k} max diag(G_pk + rho_k/2 I).
    trace, if a list, receives one record per step (recording only): the damping
    (mu, nu) the step was solved with, L at the current point and at the trial
    point, pred, and whether the step was accepted.
    """
    J = J0.copy()
    L = aug_lagrangian(J, V, C, pq, Y, BZ, rho)
    grad = grad_lagrangian(J, V, C, pq, Y, BZ, rho)
    G = jacobi_blocks(J, C, pq)
    diag = np.real(np.stack([G[..., 0, 0], G[..., 1, 1]], -1)) + 0.5 * rho[:, None, None]
    mu = LM_TAU * float(diag.max())
    nu = 2.0
    accepted = 0
    for _ in range(n_lm):
        x, _ = pcg(J, C, pq, grad, G, rho, mu, n_cg)
        pred = -(h_inner(x, grad) + 0.5 * h_inner(x, hess_lagrangian(J, x, C, pq, rho)))
        Jt = J + x
        Lt = aug_lagrangian(Jt, V, C, pq, Y, BZ, rho)
        if trace is not None:
            trace.append(dict(mu=mu, nu=nu, L=L, Lt=Lt, pred=pred,
                              accepted=bool(pred > 0.0 and math.isfinite(Lt) and Lt < L)))
        if pred > 0.0 and math.isfinite(Lt) and Lt < L:
            ratio = (L - Lt) / pred
            J, L = Jt, Lt
            grad = grad_lagrangian(J, V, C, pq, Y, BZ, rho)
            G = jacobi_blocks(J, C, pq)
            mu *= max(1.0 / 3.0, 1.0 - (2.0 * ratio - 1.0) ** 3)
            nu = 2.0
            accepted += 1
        else:
            mu *= nu
            nu *= 2.0
    if stats is not None:
        stats["accepted"] = stats.get("accepted", 0) + accepted
    return J


# ----------------------------------------------------------------------------- consensus (M2, M3)

def procrustes_unitary(Ja: np.ndarray, Jref: np.ndarray) -> np.ndarray:
    """Unitary U minimising ||Jref - Ja U|| for stacked [N,2,2] Jones (matrix Procrustes,
    Section 4): U = W V^H from the SVD Ja^H Jref = W S V^H."""
    Mx = np.einsum("nji,njk->ik", np.conj(Ja), Jref)  # (2N x 2)^H (2N x 2)
    W, _, Vh = np.linalg.svd(Mx)
    return W @ Vh


def gauge_align(Js: list[np.ndarray], ref: int) -> list[np.ndarray]:
    """First-iteration projection of every agent's J_k onto the reference agent's gauge
    (Section 3, initialisation): J_ak <- J_ak U_ak, U_ak the Procrustes unitary."""
    out = []
    for J in Js:
        Jn = J.copy()
        for k in range(J.shape[0]):
            U = procrustes_unitary(J[k], Js[ref][k])
            Jn[k] = np.matmul(J[k], U)
        out.append(Jn)
    return out


def z_update(Js, Ys, basis, rho) -> np.ndarray:
    """Closed-form Z (Eq. Zest), per direction k:
    Z_k = (1/rho_k) ((sum_i b_i b_i^T)^dagger (x) I_2N) (sum_i b_i (x) (Y_ik + rho_k J_ik)).
    Returns Z [K,M,N,2,2] (block l is Z_l)."""
    Pm = np.linalg.pinv(basis.T @ basis)
    K = Js[0].shape[0]
    M = basis.shape[1]
    Z = np.zeros((K, M) + Js[0].shape[1:], dtype=complex)
    for k in range(K):
        Rt = sum(basis[i][:, None, None, None] * (Ys[i][k] + rho[k] * Js[i][k]) for i in range(len(Js)))
        Z[k] = np.einsum("lm,mnij->lnij", Pm, Rt) / rho[k]
    return Z


def z_rhs(Js, Ys, basis_rows, rho) -> np.ndarray:
    """The right-hand sum of Eq. Zest over a subset of agents, [K,M,N,2,2]
    (what each agent contributes in step S1/D1)."""
    K = Js[0].shape[0]
    out = np.zeros((K, basis_rows.shape[1]) + Js[0].shape[1:], dtype=complex)
    for i in range(len(Js)):
        for k in range(K):
            out[k] += basis_rows[i][:, None, None, None] * (Ys[i][k] + rho[k] * Js[i][k])
    return out


def z_from_rhs(rhs, basis, rho) -> np.ndarray:
    Pm = np.linalg.pinv(basis.T @ basis)
    return np.stack([np.einsum("lm,mnij->lnij", Pm, rhs[k]) / rho[k] for k in range(rhs.shape[0])])


def bz(Z, b_row) -> np.ndarray:
    """B_f Z = sum_l b_l(f) Z_l (Eq. hidden / Eq. hblock), per direction: [K,N,2,2]."""
    return np.einsum("l,klnij->knij", b_row, Z)


# ----------------------------------------------------------------------------- driver

def agent_data(prob: dict, a: int):
    """The unflagged baselines of agent a: (V [B_a,T,2,2], C [B_a,T,K], pq [B_a,2])."""
    keep = prob["flags"][a] == 0
    return prob["V"][a][keep], prob["C"][a][keep], prob["pq"][keep]


def admm(prob: dict, n_iter: int, n_lm: int = 10, n_cg: int = 4, C_list=None, J0=None,
         Z0=None, intervals=None, jupdate=None) -> dict:
    """C-ADMM (Eq. M1, M2, M3; steps D1-D3) for every solution interval independently.

    jupdate, if given, replaces the LM J-update: a callable (J, V, C, pq, Y, BZ, rho) -> J,
    e.g. the RTR or SAGE solvers of oracle/rtr.py (Section 3 uses RTR, step D1 uses SAGE).

    Initialisation: J = identity blocks (or J0), Z = Y = 0 (Section 3). A warm start may
    also pass Z0 [I][K,M,N,2,2]; the first-iteration gauge projection is only applied
    when Z starts at zero, since it exists to remove the ambiguity that Z = Y = 0 leaves.
    History per iteration n (after the Y-update):
      primal = mean over agents and directions of ||J_ik - B_i Z_k|| / sqrt(4N)
      dual   = mean over directions of ||Z_k^{n+1} - Z_k^n|| / sqrt(4MN)   (Section 4)
      objective = sum_i L_i(J_i^{n+1}, Z^{n+1}, Y_i^{n+1})
      resid_norm = sqrt(sum_i g_i(J_i^{n+1}))
    Means and sums run over all intervals processed.
    """
    N, K, P, M = prob["N"], prob["K"], prob["P"], prob["M"]
    basis, rho = prob["basis"], prob["rho"]
    ivs = list(range(prob["I"])) if intervals is None else list(intervals)
    hist = {k: np.zeros(n_iter) for k in ("primal", "dual", "objective", "resid_norm")}
    J_out, Y_out, Z_out, L_out, g_out = {}, {}, {}, {}, {}
    n_prim = 0
    per_iv = []
    for iv in ivs:
        agents = [iv * P + f for f in range(P)]
        data = []
        for a in agents:
            V, C, pq = agent_data(prob, a)
            if C_list is not None:
                C = C_list[a][prob["flags"][a] == 0]
            data.append((V, C, pq))
        eye = np.broadcast_to(np.eye(2, dtype=complex), (K, N, 2, 2))
        Js = [eye.copy() if J0 is None else J0[a].copy() for a in agents]
        Ys = [np.zeros((K, N, 2, 2), dtype=complex) for _ in agents]
        Z = np.zeros((K, M, N, 2, 2), dtype=complex) if Z0 is None else Z0[iv].copy()
        BZs = [bz(Z, basis[i]) for i in range(P)]
        rec = []
        for n in range(n_iter):
            if jupdate is None:
                Js = [lm_jupdate(Js[i], *data[i], Ys[i], BZs[i], rho, n_lm, n_cg) for i in range(P)]
            else:
                Js = [jupdate(Js[i], *data[i], Ys[i], BZs[i], rho) for i in range(P)]
            if n == 0 and Z0 is None:
                Js = gauge_align(Js, P // 2)
            Zn = z_update(Js, Ys, basis, rho)
            BZs = [bz(Zn, basis[i]) for i in range(P)]
            Ys = [Ys[i] + rho[:, None, None, None] * (Js[i] - BZs[i]) for i in range(P)]
            prim = sum(np.linalg.norm(Js[i][k] - BZs[i][k]) for i in range(P) for k in range(K))
            dual = sum(np.linalg.norm(Zn[k] - Z[k]) for k in range(K))
            gs = [data_cost(Js[i], *data[i]) for i in range(P)]
            Ls = [gs[i] + penalty(Js[i], Ys[i], BZs[i], rho) for i in range(P)]
            rec.append((prim / math.sqrt(4 * N), dual / math.sqrt(4 * M * N), sum(Ls), sum(gs)))
            Z = Zn
        per_iv.append(rec)
        n_prim += 1
        for i, a in enumerate(agents):
            J_out[a], Y_out[a] = Js[i], Ys[i]
            L_out[a] = Ls[i]
            g_out[a] = gs[i]
        Z_out[iv] = Z
    nI = len(ivs)
    for n in range(n_iter):
        hist["primal"][n] = sum(r[n][0] for r in per_iv) / (nI * P * K)
        hist["dual"][n] = sum(r[n][1] for r in per_iv) / (nI * K)
        hist["objective"][n] = sum(r[n][2] for r in per_iv)
        hist["resid_norm"][n] = math.sqrt(sum(r[n][3] for r in per_iv))
    return dict(hist=hist, J=J_out, Y=Y_out, Z=Z_out, L=L_out, g=g_out)
