"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: the hot path computes in float32 with float64 cost, dot products and
consensus (Z) accumulation, so single-pass quantities are compared at 2e-5..1e-4 of
their scale, and whole C-ADMM runs at 1e-4 relative on the consensus objective and
the data residual norm (the parity bar for the iteration).

The dual residual ||Z^{n+1} - Z^n|| is dominated by the slow drift of the common unitary
gauge of each direction: the data term is exactly flat along it (C = c I_2, Eq. coh) and
only the penalty curves it, with Hessian rho/2 against ~sum_t |c|^2 |J|^2 for the data.
Float32 residuals carry an error ~eps |V| per element, so the gauge component of the
gradient is known to ~eps |V| |J| sum(T) / (rho/2 |dJ_gauge|), a few per cent on these
inputs. Z is the least-squares fit of Eq. Zest, so differences in J reach Z amplified by
||(sum_i b_i b_i^T)^-1 B^T||_2: 1.9 for the Bernstein basis of the LOFAR-shaped case but 20.7
for the ordinary polynomial over the narrow band of the tiny case. The dual is therefore
compared at max(15 %, 1.5 % x that amplification) relative, with an absolute floor of 1e-5 of
the solution scale ||Z^1|| / sqrt(4MN) (the first record) where the iteration has converged
and float32 stops resolving the difference of consecutive Z. With one LM step per J-update
the gauge mode is not resolved on either side and all four records agree at 1e-4.
"""
import math

import numpy as np
import pytest

from oracle import admm as O
from paper_1502_00858_gb300 import Calibrator, capi
from synth import make_problem, user_layout

pytestmark = pytest.mark.gpu

REL_ADMM = 1e-4
FORMS = {"statistics": capi.CALIB_FORM_STATISTICS, "direct": capi.CALIB_FORM_DIRECT}
_ORACLE_CACHE = {}


def cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def rounded(prob):
    """The problem with V and C rounded to complex64, as the GPU sees them."""
    return dict(prob, V=[c64(v) for v in prob["V"]], C=[c64(c) for c in prob["C"]])


def calibrator(lib, prob, **kw):
    cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                     n_intervals=prob["I"], samples=prob["T"], **kw)
    ul = user_layout(prob)
    cal.set_data(ul["vis"], ul["coh"], ul["flags"] if ul["flags"].any() else None)
    return cal


def ragged_problem(seed=5):
    """Odd N, three directions, two intervals, uneven sample counts and flagged baselines."""
    return make_problem("adjoint_n16_k3", seed=seed, N=13, K=3, P=5, I=2, T=(3, 5, 7), flag_max=0.25)


CASES = {
    "tiny_n8_k1": lambda: make_problem("tiny_n8_k1"),
    "ragged_n13_k3": ragged_problem,
    "n2_single_baseline": lambda: make_problem("tiny_n8_k1", N=2, P=3, seed=7),
    "n3_k2": lambda: make_problem("adjoint_n16_k3", N=3, K=2, P=4, I=1, T=1, seed=8),
    # ten directions (the batched workload's K: exact register bucket, shared-memory-limited sweeps)
    "n10_k10_flagged": lambda: make_problem("adjoint_n16_k3", N=10, K=10, P=4, I=1, T=(2, 3), flag_max=0.1, seed=21),
    # seven directions: a register bucket larger than K
    "n9_k7": lambda: make_problem("adjoint_n16_k3", N=9, K=7, P=4, I=1, T=2, seed=22),
    # 700 samples per interval: the statistics pass's per-(agent, diagonal) block exceeds what it
    # stages in shared memory and it reads global memory directly
    "n8_t700": lambda: make_problem("tiny_n8_k1", N=8, P=3, T=700, seed=23),
    # more than 64 stations (a 96-thread Hessian sweep, 3 warps) and four directions
    "n66_k4": lambda: make_problem("adjoint_n16_k3", N=66, K=4, P=4, I=1, T=2, flag_max=0.05, seed=24),
    # the largest register buckets of the statistics sweeps (K = 12 and K = 16)
    "n12_k12": lambda: make_problem("adjoint_n16_k3", N=12, K=12, P=4, I=1, T=2, flag_max=0.1, seed=25),
    "n10_k16": lambda: make_problem("adjoint_n16_k3", N=10, K=16, P=4, I=1, T=2, seed=26),
    # the largest station count (8128 baselines; 256-thread trial sweep, 128-thread Hessian sweep)
    "n128_k2": lambda: make_problem("adjoint_n16_k3", N=128, K=2, P=4, I=1, T=1, seed=27),
    # the paper's 47-station array with 16 directions (the trial pass reads U from global memory)
    "n47_k16": lambda: make_problem("adjoint_n16_k3", N=47, K=16, P=4, I=1, T=2, seed=28),
}
DIRECT_ONLY = set()


def form_kw(case):
    """Options of a case's context for the single-pass tests (the direct form where the statistics
    sweeps do not take the shape)."""
    return {"formulation": capi.CALIB_FORM_DIRECT} if case in DIRECT_ONLY else {}


def random_state(prob, seed):
    rng = np.random.default_rng(seed)
    A, K, N, M, I = prob["A"], prob["K"], prob["N"], prob["M"], prob["I"]
    J = (prob["J_true"] + 0.05 * cn(rng, A, K, N, 2, 2)).astype(np.complex64)
    Z = 0.1 * cn(rng, I, K, M, N, 2, 2)
    Y = (0.3 * cn(rng, A, K, N, 2, 2)).astype(np.complex64)
    return J, Z, Y


@pytest.mark.parametrize("case", sorted(CASES))
def test_eval_matches_oracle(lib, case):
    prob = CASES[case]()
    pr = rounded(prob)
    cal = calibrator(lib, prob, **form_kw(case))
    J, Z, Y = random_state(prob, 11)
    cal.set_consensus(Z, Y)
    L, g, grad = cal.eval(J)
    P = prob["P"]
    for a in range(prob["A"]):
        V, C, pq = O.agent_data(pr, a)
        BZ = c64(O.bz(Z[a // P], prob["basis"][a % P]))
        Ja, Ya = J[a].astype(np.complex128), Y[a].astype(np.complex128)
        go = O.data_cost(Ja, V, C, pq)
        Lo = O.aug_lagrangian(Ja, V, C, pq, Ya, BZ, prob["rho"])
        gro = O.grad_lagrangian(Ja, V, C, pq, Ya, BZ, prob["rho"])
        assert g[a] == pytest.approx(go, rel=2e-5, abs=1e-6)
        assert L[a] == pytest.approx(Lo, rel=2e-5, abs=1e-6)
        scale = np.abs(gro).max()
        assert np.abs(grad[a] - gro).max() <= 1e-4 * scale + 1e-6


@pytest.mark.parametrize("case", sorted(CASES))
def test_hessvec_matches_oracle(lib, case):
    prob = CASES[case]()
    pr = rounded(prob)
    cal = calibrator(lib, prob, **form_kw(case))
    J, _, _ = random_state(prob, 12)
    rng = np.random.default_rng(13)
    eta = cn(rng, *J.shape).astype(np.complex64)
    Hv = cal.hessvec(J, eta)
    for a in range(prob["A"]):
        V, C, pq = O.agent_data(pr, a)
        ref = O.hess_lagrangian(J[a].astype(np.complex128), eta[a].astype(np.complex128), C, pq, prob["rho"])
        assert np.abs(Hv[a] - ref).max() <= 1e-4 * np.abs(ref).max() + 1e-6


@pytest.mark.parametrize("case", ["tiny_n8_k1", "ragged_n13_k3", "n10_k10_flagged", "n66_k4"])
def test_residual_matches_oracle(lib, case):
    """Residual visibilities after two C-ADMM iterations, a subset of directions subtracted and
    the rest corrected by the last direction's solutions, element by element against the oracle
    at the GPU's J; flagged baselines are zero. Tolerance: float32 rounding of the sum of the
    K model terms (u ~ 6e-8 times about 10 K operations on terms up to the scale M = |V| +
    sum_k |c_k| |J_pk| |J_qk|), amplified by the correction's ||J_p^-1|| ||J_q^-1||."""
    prob = CASES[case]()
    pr = rounded(prob)
    cal = calibrator(lib, prob)
    cal.iterate(2)
    J, _, _ = cal.solutions()
    K, B = prob["K"], prob["B"]
    rng = np.random.default_rng(51)
    sub = rng.random(K) < 0.7
    sub[0] = True
    corr = K - 1
    for subtract, correct in ((None, None), (sub, corr)):
        out = cal.residual(subtract=subtract, correct=correct)
        off = 0
        for a in range(prob["A"]):
            Ta = int(prob["T"][a])
            blk = out[off: off + B * Ta * 4].reshape(B, Ta, 2, 2)
            off += B * Ta * 4
            keep = prob["flags"][a] == 0
            V, C, pq = O.agent_data(pr, a)
            Ja = J[a].astype(np.complex128)
            ref = O.corrected_residual(Ja, V, C, pq, subtract=subtract, correct=correct)
            nj = np.linalg.norm(Ja, ord=2, axis=(-2, -1))  # [K,N] spectral norms
            scale = np.abs(V).max() + np.max(np.abs(C).sum(-1)) * nj.max() ** 2
            amp = 1.0
            if correct is not None:
                amp = np.linalg.norm(np.linalg.inv(Ja[correct]), ord=2, axis=(-2, -1)).max() ** 2
            tol = 10 * K * 6e-8 * scale * amp * 10
            err = np.abs(blk[keep] - ref).max()
            assert err <= tol, (a, err, tol)
            assert np.all(blk[~keep] == 0)


def test_eval_is_bitwise_reproducible(lib):
    prob = ragged_problem()
    cal = calibrator(lib, prob)
    J, Z, Y = random_state(prob, 14)
    cal.set_consensus(Z, Y)
    r1 = cal.eval(J)
    r2 = cal.eval(J)
    for x, y in zip(r1, r2):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("case", ["tiny_n8_k1", "ragged_n13_k3"])
def test_predict_matches_oracle(lib, case):
    prob = CASES[case]()
    cal = calibrator(lib, prob)
    cal.predict(prob["uvw"], prob["sky"], prob["f0"])
    got = cal.coherencies()
    off = 0
    P, B, K = prob["P"], prob["B"], prob["K"]
    for a in range(prob["A"]):
        iv, f = divmod(a, P)
        Ta = int(prob["T"][a])
        blk = got[off: off + B * Ta * K].reshape(B, Ta, K)
        off += B * Ta * K
        ref = O.predict_coherencies(prob["uvw"][iv, :Ta], prob["sky"], prob["freqs"][f], prob["f0"], prob["pq"])
        flux = (prob["sky"][..., 2] * (prob["freqs"][f] / prob["f0"]) ** prob["sky"][..., 3]).sum(-1)
        keep = prob["flags"][a] == 0
        err = np.abs(blk[keep] - ref[keep]).max(axis=(0, 1))
        assert np.all(err <= 2e-5 * flux), (a, err / flux)
        assert np.all(blk[~keep] == 0)


def test_predict_full_size_lofar_sample(lib):
    """calib_predict on the whole LOFAR-shaped batch (320 agents, 1891 baselines, 10 samples, 5
    clusters of 20 sources): agents at both band edges and in the middle, of the first and last
    intervals, every baseline (the longest reach about 80 km, thousands of turns), element by
    element against the float64 oracle. The turns are formed in float64 and reduced to [-1/2, 1/2)
    before float32 sincospi, so each source's term is off by a few float32 ulps of its flux; the
    bound 2e-5 of the cluster's summed flux covers the 20-term sum."""
    prob = make_problem("lofar_n62_k5")
    cal = calibrator(lib, prob)
    cal.predict(prob["uvw"], prob["sky"], prob["f0"])
    got = cal.coherencies()
    P, B, K, T = prob["P"], prob["B"], prob["K"], 10
    longest = np.argmax(np.linalg.norm(prob["uvw"][0, 0, prob["pq"][:, 0]] - prob["uvw"][0, 0, prob["pq"][:, 1]], axis=1))
    for a in (0, P // 2, P - 1, prob["A"] - P, prob["A"] - 1):
        iv, f = divmod(a, P)
        blk = got[a * B * T * K: (a + 1) * B * T * K].reshape(B, T, K)
        ref = O.predict_coherencies(prob["uvw"][iv], prob["sky"], prob["freqs"][f], prob["f0"], prob["pq"])
        flux = (prob["sky"][..., 2] * (prob["freqs"][f] / prob["f0"]) ** prob["sky"][..., 3]).sum(-1)
        err = np.abs(blk - ref).max(axis=(0, 1))
        assert np.all(err <= 2e-5 * flux), (a, err / flux)
        assert np.abs(blk[longest] - ref[longest]).max() <= 2e-5 * flux.max()
    cal.close()


def test_statistics_form_rejects_shapes_beyond_its_shared_memory(lib):
    """64 stations x 16 directions need more shared memory than the statistics sweeps have:
    calib_init refuses that formulation with CALIB_EINVAL and names the direct one, which takes it."""
    prob = make_problem("adjoint_n16_k3", N=64, K=16, P=4, I=1, T=1, seed=29)
    with pytest.raises(capi.CalibError) as e:
        Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                   n_intervals=prob["I"], samples=prob["T"], formulation=capi.CALIB_FORM_STATISTICS)
    assert e.value.code == capi.CALIB_EINVAL and "CALIB_FORM_DIRECT" in str(e.value)
    cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                     n_intervals=prob["I"], samples=prob["T"], formulation=capi.CALIB_FORM_DIRECT)
    cal.close()


def test_full_size_uneven_first_jupdate_sample(lib):
    """The batched uneven workload at full size (2560 agents: 256 subbands x 10 intervals, 62
    stations, K = 10, 5/10/20 samples per subband, 0-15 % of baselines flagged) in its own launch
    configuration (autotuned statistics sweeps). From the cold start (Z = Y = 0) the first J-update
    of every agent is independent of the others and the gauge projection leaves g unchanged, so the
    oracle's LM J-update of single agents gives their g after one C-ADMM iteration."""
    prob = make_problem("uneven_n62_k10")
    cal = calibrator(lib, prob)
    cal.iterate(1)
    _, g = cal.agent_objective()
    cal.close()
    T, flags = prob["T"], prob["flags"]
    P = prob["P"]
    picks = [int(np.argmax(T[:P] == t)) for t in (5, 10, 20)]
    picks.append(int(np.argmax(flags[:P].mean(axis=1))))
    pr_rho = prob["rho"]
    for a in picks:
        keep = flags[a] == 0
        V, C, pq = c64(prob["V"][a][keep]), c64(prob["C"][a][keep]), prob["pq"][keep]
        J0 = np.broadcast_to(np.eye(2, dtype=complex), (prob["K"], prob["N"], 2, 2)).copy()
        zero = np.zeros_like(J0)
        J = O.lm_jupdate(J0, V, C, pq, zero, zero, pr_rho, 10, 4)
        assert g[a] == pytest.approx(O.data_cost(J, V, C, pq), rel=REL_ADMM), (a, int(T[a]), float(flags[a].mean()))


def run_both(lib, prob, n_iter, n_lm=10, n_cg=4, form="statistics"):
    cal = calibrator(lib, prob, n_lm=n_lm, n_cg=n_cg, formulation=FORMS[form])
    hist = cal.iterate(n_iter)
    ref = O.admm(rounded(prob), n_iter, n_lm=n_lm, n_cg=n_cg)["hist"]
    return cal, hist, ref


HISTORY_CASES = ["tiny_n8_k1", "ragged_n13_k3", "n2_single_baseline", "n10_k10_flagged", "n9_k7", "n8_t700", "n66_k4",
                 "n12_k12", "n10_k16", "n128_k2", "n47_k16"]


@pytest.mark.parametrize("case,form", [(c, f) for c in HISTORY_CASES for f in sorted(FORMS)
                                       if not (c in DIRECT_ONLY and f == "statistics")])
def test_admm_history_matches_oracle(lib, case, form):
    """Whole C-ADMM histories. The dual residual (differences of consecutive Z) is held at 1e-3
    where the basis amplifies J into Z by less than 10 (measured: 2e-4 at most, on the ragged
    case; 7e-6 or less on the others), with an absolute floor of 1e-5 of its first record where it
    has fallen to round-off. The tiny case's ordinary-polynomial basis amplifies by 20.7: there the
    float32 round-off in the weakly curved gauge mode of its direction moves Z once the iteration
    has settled, and the dual, which measures exactly that motion, differs by up to 24 % (band
    0.015 x amplification). The dual's definition and normalisation (Section 4) are held at 1e-4 by
    test_admm_one_lm_step_matches_all_records, where the gauge mode is not yet resolved, and pinned
    by hand in tests/test_oracle_schedule_pins.py."""
    prob = CASES[case]()
    n_iter = 10 if case == "tiny_n8_k1" else 4
    _, hist, ref = run_both(lib, prob, n_iter, form=form)
    np.testing.assert_allclose(hist["objective"], ref["objective"], rtol=REL_ADMM)
    np.testing.assert_allclose(hist["resid_norm"], ref["resid_norm"], rtol=REL_ADMM)
    np.testing.assert_allclose(hist["primal"], ref["primal"], rtol=1e-3, atol=1e-7)
    basis = prob["basis"]
    amp = np.linalg.norm(np.linalg.pinv(basis.T @ basis) @ basis.T, 2)
    band = 1e-3 if amp < 10 else max(0.15, 0.015 * amp)
    np.testing.assert_allclose(hist["dual"], ref["dual"], rtol=band, atol=1e-5 * ref["dual"][0])


@pytest.mark.parametrize("degree", [5, 9])
def test_admm_history_with_a_larger_basis(lib, degree):
    """Basis sizes M = 6 and 10 over 12 frequencies run the fusion-centre kernel's 8- and 16-term
    buckets; the records follow the oracle as in the history test. The basis is the orthonormalised
    span of the Bernstein polynomials of degree 5 and 9 (QR): the same fit space, well conditioned
    (amplification 1 from J to Z), so the dual is held at 1e-3."""
    from synth.lofar import basis_matrix

    prob = make_problem("tiny_n8_k1", P=12, seed=24)
    basis = np.linalg.qr(basis_matrix("bernstein", degree, prob["freqs"]))[0]
    prob = dict(prob, basis=basis, M=basis.shape[1])
    _, hist, ref = run_both(lib, prob, 4)
    np.testing.assert_allclose(hist["objective"], ref["objective"], rtol=REL_ADMM)
    np.testing.assert_allclose(hist["resid_norm"], ref["resid_norm"], rtol=REL_ADMM)
    np.testing.assert_allclose(hist["primal"], ref["primal"], rtol=1e-3, atol=1e-7)
    amp = np.linalg.norm(np.linalg.pinv(basis.T @ basis) @ basis.T, 2)
    band = 1e-3 if amp < 10 else max(0.15, 0.015 * amp)
    np.testing.assert_allclose(hist["dual"], ref["dual"], rtol=band, atol=1e-5 * ref["dual"][0])


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("case,n_cg", [("n3_k2", 1), ("tiny_n8_k1", 4), ("ragged_n13_k3", 4)])
def test_admm_one_lm_step_matches_all_records(lib, case, n_cg, form):
    """n_lm = 1 (and n_cg = 1: one preconditioned steepest-descent step): the gauge mode is
    not resolved, so primal and dual residuals agree at 1e-4 as well. The dual residual is the
    norm of a difference of consecutive Z (Section 4): its float32 round-off is absolute, of the
    order of Z's own, so it gets the floor 1e-5 x its first record (as in the full history test)."""
    prob = CASES[case]()
    _, hist, ref = run_both(lib, prob, 3, n_lm=1, n_cg=n_cg, form=form)
    for key in ("objective", "resid_norm", "primal", "dual"):
        atol = 1e-5 * ref[key][0] if key == "dual" else 1e-9
        np.testing.assert_allclose(hist[key], ref[key], rtol=REL_ADMM, atol=atol, err_msg=key)


def test_admm_solutions_match_oracle_after_gauge(lib):
    """J after 5 iterations agrees with the oracle's up to float32 round-off; the gauge is
    fixed by the first-iteration projection and Z, so no Procrustes is needed here."""
    prob = CASES["tiny_n8_k1"]()
    cal = calibrator(lib, prob)
    cal.iterate(5)
    J, Z, Y = cal.solutions()
    ref = O.admm(rounded(prob), 5)
    for a in range(prob["A"]):
        assert np.abs(J[a] - ref["J"][a]).max() < 5e-4
    assert np.abs(Z[0] - ref["Z"][0]).max() < 5e-3


@pytest.mark.parametrize("form", sorted(FORMS))
def test_full_size_lofar_interval_sample(lib, form):
    """The full LOFAR-shaped batch (62 stations, 5 directions, 32 subbands, 10 intervals,
    10 samples) in the benchmark's launch configuration; the oracle recomputes interval 0."""
    prob = make_problem("lofar_n62_k5")
    n_iter = 2
    cal = calibrator(lib, prob, formulation=FORMS[form])
    hist = cal.iterate(n_iter)
    L, g = cal.agent_objective()
    if "lofar" not in _ORACLE_CACHE:  # the oracle's interval 0 serves both formulations
        _ORACLE_CACHE["lofar"] = O.admm(rounded(prob), n_iter, intervals=[0])
    ref = _ORACLE_CACHE["lofar"]
    P = prob["P"]
    assert float(np.sum(L[:P])) == pytest.approx(sum(ref["L"][a] for a in range(P)), rel=REL_ADMM)
    assert float(np.sum(g[:P])) == pytest.approx(sum(ref["g"][a] for a in range(P)), rel=REL_ADMM)
    assert np.all(np.isfinite(hist["objective"]))
    # every interval converges to the noise floor: g ~ noise power x (data - parameters)
    sig2 = 2 * prob["sigma"] ** 2
    n_data = prob["B"] * 10 * 4
    n_par = prob["K"] * prob["N"] * 8 / 2
    assert np.all(g / (sig2 * (n_data - n_par)) < 1.5)


def test_autotuner_picks_a_measured_split_and_results_do_not_depend_on_it(lib):
    """The autotuner times candidate splits of the sweeps and keeps the fastest; the C-ADMM
    history with any fixed split agrees with the tuned one (only summation order changes)."""
    prob = CASES["ragged_n13_k3"]()
    cal = calibrator(lib, prob)
    chosen, chosen_tr, table = capi.calib_autotune(cal.ctx)
    assert chosen in table and table[chosen][0] == min(v[0] for v in table.values())
    assert chosen_tr in table and table[chosen_tr][1] == min(v[1] for v in table.values())
    h_tuned = cal.iterate(3)
    for m in (1, 5):  # CTAs per SM of the statistics sweeps
        other = calibrator(lib, prob, ctas_per_sm=m)
        h = other.iterate(3)
        for key in ("objective", "resid_norm"):
            np.testing.assert_allclose(h[key], h_tuned[key], rtol=1e-5)
