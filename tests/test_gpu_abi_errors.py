"""The C ABI rejects invalid problems and out-of-order calls with the documented error codes and
a message, and a rejected call leaves the library usable (a valid context still calibrates)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1502_00858_gb300 import capi
from paper_1502_00858_gb300.capi import CalibError
from synth import make_problem, user_layout

pytestmark = pytest.mark.gpu

EINVAL, ERANK, ENUMERIC, ESTATE = -1, -2, -6, -7


def all_pairs(N):
    return np.array([(p, q) for p in range(N) for q in range(p + 1, N)], dtype=np.int32)


def valid(N=4, K=1, P=3, M=2):
    freqs = np.linspace(115e6, 185e6, P)
    x = (freqs - freqs[P // 2]) / freqs[P // 2]
    basis = np.stack([x ** l for l in range(M)], axis=1)
    return dict(N=N, pq=all_pairs(N), K=K, freqs_hz=freqs, basis=basis, rho=np.full(K, 5.0))


def init(**over):
    kw = valid()
    opt = {k: over.pop(k) for k in list(over) if k in ("n_lm", "n_cg", "formulation", "n_intervals")}
    kw.update(over)
    return capi.calib_init(kw["N"], kw["pq"], kw["K"], kw["freqs_hz"], kw["basis"], kw["rho"], **opt)


@pytest.mark.parametrize("over,code,text", [
    (dict(N=1, pq=np.zeros((1, 2), np.int32)), EINVAL, "n_stations"),
    (dict(N=129, pq=all_pairs(129)), EINVAL, "n_stations"),
    (dict(K=0, rho=np.ones(1)), EINVAL, "n_dirs"),
    (dict(K=17, rho=np.ones(17)), EINVAL, "n_dirs"),
    (dict(pq=np.array([[0, 1], [0, 1]], np.int32)), EINVAL, "duplicate"),
    (dict(pq=np.array([[2, 2]], np.int32)), EINVAL, "0 <= p < q < N"),
    (dict(pq=np.array([[0, 4]], np.int32)), EINVAL, "0 <= p < q < N"),
    (dict(rho=np.array([0.0])), EINVAL, "rho"),
    (dict(rho=np.array([np.nan])), EINVAL, "rho"),
    (dict(basis=np.array([[1.0, np.inf]] * 3)), EINVAL, "basis"),
    (dict(basis=np.ones((3, 4))), ERANK, "P >= M"),
    (dict(basis=np.array([[1.0, 2.0], [1.0, 2.0], [2.0, 4.0]])), ERANK, "singular"),
    (dict(n_lm=0), EINVAL, "n_lm"),
    (dict(n_cg=0), EINVAL, "n_cg"),
    (dict(formulation=7), EINVAL, "formulation"),
    (dict(n_intervals=0), EINVAL, "n_intervals"),
])
def test_init_rejects_invalid_problems(over, code, text):
    with pytest.raises(CalibError) as err:
        init(**over)
    assert err.value.code == code
    assert text in str(err.value)


def test_calls_out_of_order_and_bad_data_are_rejected_and_the_library_stays_usable():
    ctx = init()
    try:
        with pytest.raises(CalibError) as err:
            capi.calib_admm_iter(ctx, 1)
        assert err.value.code == ESTATE
        A, B = 3, 6
        vis = np.zeros(A * B * 1 * 4, np.complex64)
        coh = np.ones(A * B * 1 * 1, np.complex64)
        vis[5] = np.nan
        with pytest.raises(CalibError) as err:
            capi.calib_set_data(ctx, vis, coh)
        assert err.value.code == ENUMERIC
        with pytest.raises(CalibError) as err:
            capi.calib_admm_iter(ctx, 0)
        assert err.value.code == EINVAL
        out = np.zeros(A * B * 1 * 4, np.complex64)
        with pytest.raises(CalibError) as err:  # no coherencies yet
            capi.calib_residual(ctx, out)
        assert err.value.code == ESTATE
        capi.calib_set_data(ctx, np.zeros(A * B * 4, np.complex64), coh)
        with pytest.raises(CalibError) as err:
            capi.calib_residual(ctx, out, correct=1)  # K = 1
        assert err.value.code == EINVAL
        capi.calib_residual(ctx, out, correct=0)  # J = I, V = 0: R = -c I
        np.testing.assert_array_equal(out.reshape(-1, 2, 2), np.broadcast_to(-np.eye(2, dtype=np.complex64), (A * B, 2, 2)))
    finally:
        capi.calib_destroy(ctx)

    # a valid problem after the rejected calls calibrates and lowers the data residual
    prob = make_problem("tiny_n8_k1", P=3, seed=31)
    ul = user_layout(prob)
    ctx = capi.calib_init(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                          n_intervals=prob["I"], n_samples=int(prob["T"][0]))
    try:
        capi.calib_set_data(ctx, ul["vis"], ul["coh"])
        hist = capi.calib_admm_iter(ctx, 3)
        assert np.all(np.isfinite(hist["objective"]))
        assert hist["resid_norm"][-1] < hist["resid_norm"][0]
    finally:
        capi.calib_destroy(ctx)


def test_bounded_wait_gives_up_reports_timeout_and_leaves_the_device_usable():
    # control: the barrier phase completes, the wait returns at once
    ms = capi.calib_selftest_bounded_wait(True)
    assert ms < 50.0
    # a phase nothing completes: the wait gives up after its budget (about one second of SM
    # clock), the call reports CALIB_ETIMEOUT, and the device's context stays usable
    with pytest.raises(CalibError) as err:
        capi.calib_selftest_bounded_wait(False)
    assert err.value.code == capi.CALIB_ETIMEOUT
    assert "gave up" in str(err.value)
    assert capi.calib_selftest_bounded_wait(True) < 50.0
    prob = make_problem("tiny_n8_k1", P=3, seed=32)
    ul = user_layout(prob)
    ctx = capi.calib_init(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                          n_intervals=prob["I"], n_samples=int(prob["T"][0]))
    try:
        capi.calib_set_data(ctx, ul["vis"], ul["coh"])
        hist = capi.calib_admm_iter(ctx, 2)
        assert np.all(np.isfinite(hist["objective"]))
    finally:
        capi.calib_destroy(ctx)
