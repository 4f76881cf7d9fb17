"""Simulation I of the paper (Section 4) on the GPU library.

One direction (K = 1), 47 stations, 32 channels over 115-185 MHz, 20 samples of 10 s, Jones
matrices varying in time and frequency, 300 weak background sources left out of the sky model,
noise power 10 % of the signal power (the `sim1_n47_k1` problem of the synthetic generator).

* Normal calibration: every channel alone (rho -> 1e-6, no consensus), 30 LM steps.
* Distributed calibration: 50 C-ADMM iterations of 10 LM steps, for F in {2, 5} terms of the
  ordinary polynomial basis (Eq. poly) and rho in {0.5, 5, 50}.

For each run it records the primal and dual residuals per iteration (Section 4 definitions) and
the per-parameter error per channel, (1/sqrt(4N)) ||J_f(t) - J^_f U|| with U the Procrustes
unitary between the estimate and the truth, averaged over the samples t. It then checks the
section's qualitative claims: the primal residual falls further for larger rho, the dual residual
is lower for F = 2, distributed calibration has a lower error than normal calibration, the lowest
error is at rho = 50, and F = 5 has higher error at the edge channels.

    python -m experiments.sim1 [--seed S] [--out FILE.json]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

F_VALUES = (2, 5)
RHO_VALUES = (0.5, 5.0, 50.0)
N_ADMM, N_LM_DIST, N_LM_NORMAL, N_CG = 50, 10, 30, 4
RHO_NORMAL = 1e-6


def poly_basis(freqs: np.ndarray, F: int, f0: float) -> np.ndarray:
    """Ordinary polynomial basis b_l(f) = ((f - f0)/f0)^l, l < F (Eq. poly), [P,F]."""
    x = (np.asarray(freqs) - f0) / f0
    return np.stack([x ** l for l in range(F)], axis=1)


def procrustes(J_hat: np.ndarray, J: np.ndarray) -> np.ndarray:
    """The 2x2 unitary U minimising ||J - J_hat U|| over the stacked station blocks [N,2,2]:
    U = W V^H from the SVD W S V^H of J_hat^H J (orthogonal Procrustes)."""
    A = J_hat.reshape(-1, 2)
    Bm = J.reshape(-1, 2)
    w, _, vh = np.linalg.svd(A.conj().T @ Bm)
    return w @ vh


def jones_error(J_hat: np.ndarray, J: np.ndarray) -> float:
    """Per-parameter error (1/sqrt(4N)) ||J - J_hat U|| after the Procrustes unitary (Section 4)."""
    U = procrustes(J_hat, J)
    return float(np.linalg.norm(J - J_hat @ U) / math.sqrt(4 * J.shape[0]))


def channel_errors(J_hat: np.ndarray, J_true_t: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Error per channel, averaged over its samples: J_hat [P,N,2,2] (direction 0), J_true_t
    [P,Tmax,N,2,2]."""
    return np.array([np.mean([jones_error(J_hat[f], J_true_t[f, t]) for t in range(int(T[f]))])
                     for f in range(J_hat.shape[0])])


def check_claims(res: dict) -> dict:
    """The qualitative claims of Simulation I as booleans, from run results keyed 'normal' and
    'F{F}_rho{rho}' (each with final 'primal', 'dual' and per-channel 'error')."""
    def run(F, rho):
        return res[f"F{F}_rho{rho:g}"]

    out = {}
    out["primal_lower_for_larger_rho"] = all(
        run(F, 50.0)["primal"] < run(F, 5.0)["primal"] < run(F, 0.5)["primal"] for F in F_VALUES)
    out["dual_lower_for_F2"] = all(run(2, rho)["dual"] < run(5, rho)["dual"] for rho in RHO_VALUES)
    normal = float(np.mean(res["normal"]["error"]))
    out["distributed_beats_normal"] = all(float(np.mean(run(F, rho)["error"])) < normal
                                          for F in F_VALUES for rho in RHO_VALUES)
    out["lowest_error_at_rho50"] = all(
        min(RHO_VALUES, key=lambda r: float(np.mean(run(F, r)["error"]))) == 50.0 for F in F_VALUES)
    e5 = np.asarray(run(5, 50.0)["error"])
    edge = np.concatenate([e5[:2], e5[-2:]])
    out["edge_error_higher_for_F5"] = bool(edge.mean() > np.median(e5[2:-2]))
    return out


def calibrate(prob: dict, ul: dict, basis: np.ndarray, rho: float, n_admm: int, n_lm: int):
    """One calibration of all channels through the library; returns (history, J [P,N,2,2])."""
    from paper_1502_00858_gb300 import Calibrator

    cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], basis, np.full(prob["K"], rho),
                     n_intervals=prob["I"], samples=prob["T"], n_lm=n_lm, n_cg=N_CG)
    try:
        cal.set_data(ul["vis"], ul["coh"])
        hist = cal.iterate(n_admm)
        J, _, _ = cal.solutions()
    finally:
        cal.close()
    return hist, J[:, 0].astype(np.complex128)


def main(argv=None) -> dict:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--out", default=None, help="write the results as JSON")
    args = ap.parse_args(argv)

    from synth import make_problem, user_layout

    prob = make_problem("sim1_n47_k1", seed=args.seed)
    ul = user_layout(prob)
    J_true_t = prob["J_true_t"][:, :, 0]  # [P,T,N,2,2]
    res = {}
    hist, J = calibrate(prob, ul, np.ones((prob["P"], 1)), RHO_NORMAL, 1, N_LM_NORMAL)
    res["normal"] = {"error": channel_errors(J, J_true_t, prob["T"]).tolist()}
    for F in F_VALUES:
        basis = poly_basis(prob["freqs"], F, prob["f0"])
        for rho in RHO_VALUES:
            hist, J = calibrate(prob, ul, basis, rho, N_ADMM, N_LM_DIST)
            res[f"F{F}_rho{rho:g}"] = {
                "primal": float(hist["primal"][-1]), "dual": float(hist["dual"][-1]),
                "primal_curve": [float(v) for v in hist["primal"]],
                "dual_curve": [float(v) for v in hist["dual"]],
                "error": channel_errors(J, J_true_t, prob["T"]).tolist()}
    out = {"problem": "sim1_n47_k1", "seed": args.seed, "n_admm": N_ADMM, "n_lm": N_LM_DIST,
           "n_lm_normal": N_LM_NORMAL, "results": res, "claims": check_claims(res)}
    summary = {k: (float(np.mean(v["error"])), v.get("primal"), v.get("dual")) for k, v in res.items()}
    print(json.dumps({"mean_error_primal_dual": summary, "claims": out["claims"]}))
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(out, fh)
    return out


if __name__ == "__main__":
    main()
