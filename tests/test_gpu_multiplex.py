"""Frequency multiplexing (Section 3: with more frequencies than agents, a subset of P
frequencies is calibrated and the selection repeated until every frequency is done).

calib_options.freq_groups = G splits each interval's frequencies into G interleaved subsets
(g, g+G, g+2G, ...), each its own C-ADMM problem with its own Z; the library runs all of them in
one batch. The oracle runs each subset as a separate problem (oracle.admm on the subset's agents
and basis rows), which is the paper's sequential repetition; the records of the batch are the
sums (objective, squared residual norm) and means (primal over agents, dual over problems) of
the subsets' records.
"""
import math

import numpy as np
import pytest

from oracle import admm as O
from paper_1502_00858_gb300 import Calibrator, capi
from synth import make_problem, user_layout

pytestmark = pytest.mark.gpu

FORMS = {"statistics": capi.CALIB_FORM_STATISTICS, "direct": capi.CALIB_FORM_DIRECT}


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def problem():
    """13 stations, 3 directions, 12 frequencies (2 groups of 6 > M = 4), 2 intervals, 3/5/7 samples, flags."""
    return make_problem("adjoint_n16_k3", seed=31, N=13, K=3, P=12, I=2, T=(3, 5, 7), flag_max=0.2)


def subset(prob, G, g):
    """The consensus problem of frequency group g: agents iv * P + g + G j, basis rows g, g+G, ..."""
    P, I = prob["P"], prob["I"]
    agents = [iv * P + g + G * j for iv in range(I) for j in range(P // G)]
    return dict(prob, P=P // G, A=len(agents), basis=prob["basis"][g::G], freqs=prob["freqs"][g::G],
                V=[c64(prob["V"][a]) for a in agents], C=[c64(prob["C"][a]) for a in agents],
                flags=prob["flags"][agents], T=prob["T"][agents]), agents


@pytest.mark.parametrize("form", sorted(FORMS))
def test_grouped_batch_matches_the_oracle_run_group_by_group(lib, form):
    prob = problem()
    G, n_iter = 2, 4
    cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                     n_intervals=prob["I"], samples=prob["T"], formulation=FORMS[form], freq_groups=G)
    ul = user_layout(prob)
    cal.set_data(ul["vis"], ul["coh"], ul["flags"])
    hist = cal.iterate(n_iter)
    J, Z, _ = cal.solutions()
    cal.close()
    assert Z.shape == (prob["I"] * G, prob["K"], prob["M"], prob["N"], 2, 2)
    refs = []
    for g in range(G):
        sub, agents = subset(prob, G, g)
        out = O.admm(sub, n_iter)
        refs.append((out, agents))
        for iv in range(prob["I"]):  # this group's Z of interval iv is problem iv * G + g
            assert np.abs(Z[iv * G + g] - out["Z"][iv]).max() <= 5e-3 * np.abs(out["Z"][iv]).max()
    obj = sum(r[0]["hist"]["objective"] for r in refs)
    res = np.sqrt(sum(r[0]["hist"]["resid_norm"] ** 2 for r in refs))
    prim = sum(r[0]["hist"]["primal"] for r in refs) / G
    np.testing.assert_allclose(hist["objective"], obj, rtol=1e-4)
    np.testing.assert_allclose(hist["resid_norm"], res, rtol=1e-4)
    np.testing.assert_allclose(hist["primal"], prim, rtol=1e-3, atol=1e-7)


def test_group_count_must_divide_the_frequencies_and_leave_enough_per_problem(lib):
    prob = problem()
    for G, code in ((5, capi.CALIB_EINVAL), (4, capi.CALIB_ERANK)):  # 12 % 5 != 0; 12 / 4 = 3 < M = 4
        with pytest.raises(capi.CalibError) as e:
            Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                       n_intervals=prob["I"], samples=prob["T"], freq_groups=G)
        assert e.value.code == code, G


def test_one_group_is_the_plain_batch(lib):
    """freq_groups = 1 is the default path bit for bit."""
    prob = problem()
    ul = user_layout(prob)
    out = []
    for kw in ({}, {"freq_groups": 1}):
        cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                         n_intervals=prob["I"], samples=prob["T"], **kw)
        cal.set_data(ul["vis"], ul["coh"], ul["flags"])
        out.append(cal.iterate(2))
        cal.close()
    for key in ("objective", "primal", "dual", "resid_norm"):
        assert np.array_equal(out[0][key], out[1][key])
    assert math.isfinite(out[0]["objective"][-1])
