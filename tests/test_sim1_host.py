"""Host-side parts of the Simulation I driver (Section 4) and the generator paths it uses: the
Procrustes error metric, the claim checks, the time-and-frequency Jones model, the uncorrupted
background sources and the noise level. No GPU: the calibrations themselves run on the GPU machine."""
from __future__ import annotations

import math

import numpy as np
import pytest

from experiments import sim1
from synth import make_problem
from synth.lofar import simulate_visibilities


def cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def test_error_is_blind_to_the_unitary_ambiguity():
    """J and J U (U unitary) are the same solution up to the ambiguity of Section 3: zero error."""
    rng = np.random.default_rng(0)
    J = cn(rng, 9, 2, 2)
    U = np.linalg.qr(cn(rng, 2, 2))[0]
    assert sim1.jones_error(J @ U, J) < 1e-12
    np.testing.assert_allclose(sim1.procrustes(J @ U, J), U.conj().T, atol=1e-12)


def test_error_of_a_perturbation_is_its_norm_per_parameter():
    """Without ambiguity (perturbation small and J far from any rotation of itself), the error is
    ||dJ|| / sqrt(4N) to first order, and never more than that."""
    rng = np.random.default_rng(1)
    J = np.eye(2) + 0.3 * cn(rng, 12, 2, 2)
    dJ = 1e-6 * cn(rng, 12, 2, 2)
    e = sim1.jones_error(J + dJ, J)
    bound = np.linalg.norm(dJ) / math.sqrt(4 * 12)
    assert e <= bound * (1 + 1e-9)
    assert e > 0.5 * bound


def test_channel_errors_average_over_the_samples():
    rng = np.random.default_rng(2)
    Jt = cn(rng, 3, 4, 5, 2, 2)  # [P,T,N,2,2]
    Jh = Jt[:, 0]
    T = np.array([1, 2, 4])
    e = sim1.channel_errors(Jh, Jt, T)
    assert e[0] == pytest.approx(0.0, abs=1e-12)
    ref = np.mean([sim1.jones_error(Jh[2], Jt[2, t]) for t in range(4)])
    assert e[2] == pytest.approx(ref)


def _results(normal=1.0, errs=None, primal=None, dual=None):
    res = {"normal": {"error": [normal] * 8}}
    for F in sim1.F_VALUES:
        for rho in sim1.RHO_VALUES:
            e = errs[(F, rho)] if errs else [0.5 / rho ** 0.1] * 8
            res[f"F{F}_rho{rho:g}"] = {"error": e, "primal": primal[(F, rho)] if primal else 1.0 / rho,
                                       "dual": dual[(F, rho)] if dual else 0.1 * F}
    return res


def test_claims_hold_on_results_shaped_like_the_paper_s_figures():
    errs = {(F, rho): [0.6] * 2 + [0.5 / rho ** 0.1] * 4 + [0.6] * 2 if F == 5 else [0.5 / rho ** 0.1] * 8
            for F in sim1.F_VALUES for rho in sim1.RHO_VALUES}
    claims = sim1.check_claims(_results(errs=errs))
    assert all(claims.values()), claims


def test_claims_fail_where_the_results_contradict_them():
    primal = {(F, rho): rho for F in sim1.F_VALUES for rho in sim1.RHO_VALUES}  # rises with rho
    claims = sim1.check_claims(_results(normal=0.1, primal=primal))
    assert not claims["primal_lower_for_larger_rho"]
    assert not claims["distributed_beats_normal"]
    assert not claims["edge_error_higher_for_F5"]


def test_poly_basis_is_the_ordinary_polynomial():
    f = np.array([140e6, 150e6, 165e6])
    B = sim1.poly_basis(f, 3, 150e6)
    x = (f - 150e6) / 150e6
    np.testing.assert_allclose(B, np.stack([np.ones(3), x, x * x], 1))


# ------------------------------------------------------------------ generator paths of Simulation I

@pytest.fixture(scope="module")
def sim_small():
    return make_problem("sim1_n47_k1", N=6, P=5, T=4, seed=9)


def test_jones_elements_are_a_time_factor_times_a_frequency_factor(sim_small):
    """Every element is a product T(t) F(f) (Section 4), so for any two samples and two
    channels J(t1,f1) J(t2,f2) = J(t1,f2) J(t2,f1) element-wise; and the time factor of element
    e is sin(a1 t' + 2 pi b1) + i sin(a2 t' + 2 pi b2), whose real and imaginary parts lie in [-1, 1]."""
    Jt = sim_small["J_true_t"]  # [A,T,K,N,2,2]
    lhs = Jt[0, 0] * Jt[3, 2]
    rhs = Jt[3, 0] * Jt[0, 2]
    np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-12)
    # the reported J_true is the mean over the samples
    np.testing.assert_allclose(sim_small["J_true"][2], Jt[2, :4].mean(axis=0))


def test_background_sources_are_not_corrupted(sim_small):
    """Noise-free data minus the calibrated direction's model (with the per-sample Jones) is
    c_bg I_2: zero off the diagonal, equal on it."""
    p = make_problem("sim1_n47_k1", N=6, P=5, T=4, seed=9, noise=False)
    for a in (0, 4):
        R = p["V"][a] - np.concatenate(
            [simulate_visibilities(p["J_true_t"][a, t], p["C"][a][:, t:t + 1], p["pq"]) for t in range(4)], axis=1)
        assert np.abs(R[..., 0, 1]).max() < 1e-12 and np.abs(R[..., 1, 0]).max() < 1e-12
        np.testing.assert_allclose(R[..., 0, 0], R[..., 1, 1], atol=1e-12)
        assert np.abs(R[..., 0, 0]).max() > 0  # the background is there
        assert np.abs(R[..., 0, 0]).max() <= 300 * 0.1 * (1 + 1e-12)  # at most 300 sources below 0.1 Jy


def test_noise_power_is_a_tenth_of_the_signal_power(sim_small):
    p0 = make_problem("sim1_n47_k1", N=6, P=5, T=4, seed=9, noise=False)
    sig = sum(float(np.sum(np.abs(v) ** 2)) for v in p0["V"])
    noise = sum(float(np.sum(np.abs(v - v0) ** 2)) for v, v0 in zip(sim_small["V"], p0["V"]))
    assert noise / sig == pytest.approx(0.1, rel=0.15)
