"""Checkpoint and resume of the C-ADMM iteration state (calib_get_state / calib_set_state).

The paper restarts a calibration from the previous time slot's solutions (Section 3,
initialisation); the state blob keeps everything a following iteration reads (J, Y, B_i Z, Z,
the previous Z, the projected data gradient and Jacobi blocks, the LM scalars and the pending
gauge projection). The library's reductions run in a fixed order, so a resumed run must repeat
the uninterrupted one bit for bit, in the same context or in a new one of the same problem.
"""
import numpy as np
import pytest

from paper_1502_00858_gb300 import Calibrator, capi
from synth import make_problem, user_layout

pytestmark = pytest.mark.gpu

FORMS = {"statistics": capi.CALIB_FORM_STATISTICS, "direct": capi.CALIB_FORM_DIRECT}


def ragged():
    """13 stations, 3 directions, 2 intervals, 3/5/7 samples, up to 25 % of baselines flagged."""
    return make_problem("adjoint_n16_k3", seed=5, N=13, K=3, P=5, I=2, T=(3, 5, 7), flag_max=0.25)


def calibrator(prob, form):
    cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                     n_intervals=prob["I"], samples=prob["T"], formulation=FORMS[form])
    ul = user_layout(prob)
    cal.set_data(ul["vis"], ul["coh"], ul["flags"])
    return cal


def run(cal, n):
    h = cal.iterate(n)
    J, Z, Y = cal.solutions()
    return h, J, Z, Y


def assert_same(a, b):
    ha, *xa = a
    hb, *xb = b
    for key in ("primal", "dual", "objective", "resid_norm"):
        assert np.array_equal(ha[key], hb[key]), key
    for u, v in zip(xa, xb):
        assert np.array_equal(u.view(np.uint8), v.view(np.uint8))


@pytest.mark.parametrize("form", sorted(FORMS))
def test_resume_repeats_the_uninterrupted_run_bit_for_bit(lib, form):
    """3 iterations, save, 2 more; restore, the same 2 again: identical records and solutions;
    restored into a new context of the same problem: identical again."""
    prob = ragged()
    cal = calibrator(prob, form)
    run(cal, 3)
    blob = cal.get_state()
    first = run(cal, 2)
    cal.set_state(blob)
    again = run(cal, 2)
    assert_same(first, again)
    other = calibrator(prob, form)
    other.set_state(blob)
    assert_same(first, run(other, 2))
    other.close()
    cal.close()


def test_a_cold_blob_keeps_the_pending_gauge_projection(lib):
    """A blob saved before the first iteration restores the cold start: the next iteration still
    applies the first-iteration gauge projection (Section 3, initialisation)."""
    prob = ragged()
    cal = calibrator(prob, "statistics")
    cold = cal.get_state()
    ref = run(cal, 2)
    run(cal, 1)
    cal.set_state(cold)
    assert_same(ref, run(cal, 2))
    cal.close()


def test_blobs_of_another_problem_or_damaged_blobs_are_rejected(lib):
    prob = ragged()
    cal = calibrator(prob, "statistics")
    blob = cal.get_state()
    small = prob.copy()
    other = Calibrator(prob["N"], prob["pq"], 2, prob["freqs"], prob["basis"], prob["rho"][:2],
                       n_intervals=prob["I"], samples=prob["T"])
    with pytest.raises(capi.CalibError) as e:
        other.set_state(blob)
    assert e.value.code == capi.CALIB_EINVAL
    bad = bytearray(blob)
    bad[0:8] = b"NOTSTATE"
    with pytest.raises(capi.CalibError) as e:
        cal.set_state(bytes(bad))
    assert e.value.code == capi.CALIB_EINVAL
    with pytest.raises(capi.CalibError) as e:
        cal.set_state(blob[:-64])
    assert e.value.code == capi.CALIB_EINVAL
    # flags differ: the data layout the blob belongs to is not this one
    unflagged = calibrator(dict(small, flags=np.zeros_like(prob["flags"])), "statistics")
    with pytest.raises(capi.CalibError) as e:
        unflagged.set_state(blob)
    assert e.value.code == capi.CALIB_EINVAL
    unflagged.close()
    other.close()
    cal.close()


@pytest.mark.parametrize("form", sorted(FORMS))
def test_dependent_launch_changes_no_result(lib, form):
    """In the timed graph the LM chain's kernels run under programmatic dependent launch: each may
    start while the one before it is still running and waits (griddepcontrol.wait) before it touches
    that kernel's outputs. With per-kernel profiling on, the graph has event records between the
    kernels and runs them strictly one after another. Both give the same records and solutions bit
    for bit."""
    prob = ragged()
    out = []
    for profiling in (False, True):
        cal = calibrator(prob, form)
        capi.calib_profile_enable(cal.ctx, profiling)
        out.append(run(cal, 4))
        cal.close()
    assert_same(out[0], out[1])
