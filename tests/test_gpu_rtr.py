"""The paper's own J-update solver on the GPU: Riemannian trust region with truncated CG
(Section 3 and Appendix A; CALIB_JUPDATE_RTR), against the float64 oracle's rtr_jupdate inside
the same C-ADMM (oracle/rtr.py), on the same seeded inputs, in both formulations of the sweeps.

The bar is the one of the LM J-update: objective and data residual norm of every iteration at
1e-4 relative, primal residual at 1e-3. The trust-region decisions (accept, radius, boundary)
are taken in float64 from float32 dot products on both sides of a threshold only by chance; the
cases are small enough that none sits on one. The dual residual (differences of consecutive Z)
gets the LM test's relative band but an absolute floor of 2e-3 of its first record instead of
1e-5: unpreconditioned truncated CG resolves the gauge mode of each direction (curved only by
rho/2) less than the block-Jacobi PCG does, so float32 round-off there moves Z by about 1e-3 of
its first change once the iteration has settled; on the tiny case's ordinary-polynomial basis
(amplification 20.7 from J to Z) that is 4e-4 of a 0.43 first record.
"""
import math

import numpy as np
import pytest

from oracle import admm as O
from oracle import rtr as R
from paper_1502_00858_gb300 import Calibrator, capi
from synth import make_problem, user_layout

pytestmark = pytest.mark.gpu

FORMS = {"statistics": capi.CALIB_FORM_STATISTICS, "direct": capi.CALIB_FORM_DIRECT}
N_RTR, N_CG = 10, 4
CASES = {
    "tiny_n8_k1": lambda: make_problem("tiny_n8_k1"),
    "ragged_n13_k3": lambda: make_problem("adjoint_n16_k3", seed=5, N=13, K=3, P=5, I=2, T=(3, 5, 7), flag_max=0.25),
    "n10_k10_flagged": lambda: make_problem("adjoint_n16_k3", N=10, K=10, P=4, I=1, T=(2, 3), flag_max=0.1, seed=21),
}
_ORACLE = {}


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def oracle_history(case, prob, n_iter):
    if case not in _ORACLE:
        pr = dict(prob, V=[c64(v) for v in prob["V"]], C=[c64(c) for c in prob["C"]])
        upd = lambda J, V, C, pq, Y, BZ, rho: R.rtr_jupdate(J, V, C, pq, Y, BZ, rho, N_RTR, N_CG)  # noqa: E731
        _ORACLE[case] = O.admm(pr, n_iter, jupdate=upd)["hist"]
    return _ORACLE[case]


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("case", sorted(CASES))
def test_rtr_admm_history_matches_the_oracle(lib, case, form):
    prob = CASES[case]()
    n_iter = 6 if case == "tiny_n8_k1" else 4
    cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                     n_intervals=prob["I"], samples=prob["T"], n_lm=N_RTR, n_cg=N_CG, formulation=FORMS[form],
                     jupdate=capi.CALIB_JUPDATE_RTR)
    ul = user_layout(prob)
    cal.set_data(ul["vis"], ul["coh"], ul["flags"] if ul["flags"].any() else None)
    hist = cal.iterate(n_iter)
    cal.close()
    ref = oracle_history(case, prob, n_iter)
    np.testing.assert_allclose(hist["objective"], ref["objective"], rtol=1e-4)
    np.testing.assert_allclose(hist["resid_norm"], ref["resid_norm"], rtol=1e-4)
    np.testing.assert_allclose(hist["primal"], ref["primal"], rtol=1e-3, atol=1e-7)
    basis = prob["basis"]
    amp = np.linalg.norm(np.linalg.pinv(basis.T @ basis) @ basis.T, 2)
    np.testing.assert_allclose(hist["dual"], ref["dual"], rtol=max(0.15, 0.015 * amp), atol=2e-3 * ref["dual"][0])


def test_rtr_and_lm_reach_the_same_consensus_objective(lib):
    """Both inner solvers minimise the same L_i (Eq. M1): after 6 C-ADMM iterations on the tiny case
    their objectives agree to 1e-3 (the iterates differ; the minimisers they approach do not)."""
    prob = CASES["tiny_n8_k1"]()
    out = {}
    for name, ju in (("lm", capi.CALIB_JUPDATE_LM), ("rtr", capi.CALIB_JUPDATE_RTR)):
        cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                         n_intervals=prob["I"], samples=prob["T"], n_lm=N_RTR, n_cg=N_CG, jupdate=ju)
        ul = user_layout(prob)
        cal.set_data(ul["vis"], ul["coh"])
        out[name] = cal.iterate(6)
        cal.close()
    assert math.isclose(out["lm"]["objective"][-1], out["rtr"]["objective"][-1], rel_tol=1e-3)


N_SAGE, N_RTR_SAGE = 2, 5
_ORACLE_SAGE = {}


def oracle_sage_history(case, prob, n_iter):
    if case not in _ORACLE_SAGE:
        pr = dict(prob, V=[c64(v) for v in prob["V"]], C=[c64(c) for c in prob["C"]])
        upd = lambda J, V, C, pq, Y, BZ, rho: R.sage_jupdate(J, V, C, pq, Y, BZ, rho, N_SAGE, N_RTR_SAGE, N_CG)  # noqa: E731
        _ORACLE_SAGE[case] = O.admm(pr, n_iter, jupdate=upd)["hist"]
    return _ORACLE_SAGE[case]


@pytest.mark.parametrize("case", sorted(CASES))
def test_sage_admm_history_matches_the_oracle(lib, case):
    """SAGE over the directions (step D1; 2 sweeps of 5 RTR steps per direction), its expectation
    step taken on the per-baseline statistics, against the oracle's sage_jupdate, which removes the
    other directions' models from the visibilities themselves."""
    prob = CASES[case]()
    n_iter = 4
    cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                     n_intervals=prob["I"], samples=prob["T"], n_lm=N_RTR_SAGE, n_cg=N_CG,
                     jupdate=capi.CALIB_JUPDATE_SAGE, n_sage=N_SAGE)
    ul = user_layout(prob)
    cal.set_data(ul["vis"], ul["coh"], ul["flags"] if ul["flags"].any() else None)
    hist = cal.iterate(n_iter)
    cal.close()
    ref = oracle_sage_history(case, prob, n_iter)
    np.testing.assert_allclose(hist["objective"], ref["objective"], rtol=1e-4)
    np.testing.assert_allclose(hist["resid_norm"], ref["resid_norm"], rtol=1e-4)
    np.testing.assert_allclose(hist["primal"], ref["primal"], rtol=1e-3, atol=1e-7)


def test_sage_needs_the_statistics_formulation(lib):
    prob = CASES["tiny_n8_k1"]()
    with pytest.raises(capi.CalibError) as e:
        Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                   n_intervals=prob["I"], samples=prob["T"], formulation=capi.CALIB_FORM_DIRECT,
                   jupdate=capi.CALIB_JUPDATE_SAGE)
    assert e.value.code == capi.CALIB_EINVAL
