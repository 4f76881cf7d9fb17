"""Simulation I (Section 4) through the float64 oracle at reduced size: the qualitative behaviour the
section reports, checked on the oracle's C-ADMM with the Simulation I problem generator. Reduced
problem: 10 stations, 8 channels, 20 samples, 20 C-ADMM iterations of 10 LM steps; normal
calibration is each channel alone (rho 1e-6) with 30 LM steps. Three claims hold at this size: the
lowest error is at rho = 50 for both F, the dual residual is lower for F = 2 than for F = 5, and F = 5
has the higher error at the edge channels. The primal-residual ordering and distributed-beats-normal
at every rho need more stations and iterations, and are left to the full-size run on the GPU."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import admm as O
from paper_1502_00858_gb300 import sim1
from synth import make_problem


@pytest.fixture(scope="module")
def results():
    N, P, n_iter = 10, 8, 20
    prob = make_problem("sim1_n47_k1", N=N, P=P, seed=5)
    Jt = prob["J_true_t"][:, :, 0]
    zero = np.zeros((1, N, 2, 2), complex)
    eye = np.broadcast_to(np.eye(2, dtype=complex), (1, N, 2, 2))
    Jn = [O.lm_jupdate(eye.copy(), *O.agent_data(prob, a), zero, zero, np.array([sim1.RHO_NORMAL]),
                       sim1.N_LM_NORMAL, sim1.N_CG)[0] for a in range(P)]
    res = {"normal": {"error": sim1.channel_errors(np.array(Jn), Jt, prob["T"])}}
    for F in sim1.F_VALUES:
        basis = sim1.poly_basis(prob["freqs"], F, prob["f0"])
        for rho in sim1.RHO_VALUES:
            out = O.admm(dict(prob, basis=basis, M=F, rho=np.array([rho])), n_iter, n_lm=sim1.N_LM_DIST,
                         n_cg=sim1.N_CG)
            J = np.array([out["J"][a][0] for a in range(P)])
            res[f"F{F}_rho{rho:g}"] = {"primal": float(out["hist"]["primal"][-1]),
                                       "dual": float(out["hist"]["dual"][-1]),
                                       "error": sim1.channel_errors(J, Jt, prob["T"])}
    return res


def test_simulation_one_behaviour_on_the_oracle(results):
    claims = sim1.check_claims(results)
    assert claims["lowest_error_at_rho50"]
    assert claims["dual_lower_for_F2"]
    assert claims["edge_error_higher_for_F5"]
    # rho = 50 beats normal calibration for both F
    normal = float(np.mean(results["normal"]["error"]))
    for F in sim1.F_VALUES:
        assert float(np.mean(results[f"F{F}_rho50"]["error"])) < normal
