"""Learned warm start: the network kernels against the float64 oracle (oracle/mlp.py), training,
the never-worse selection rule, and time to the plain method's residual on a small sequence."""
import math

import numpy as np
import pytest

from oracle import mlp as OM
from paper_1502_00858_gb300 import Calibrator, capi
from paper_1502_00858_gb300 import warmstart as W
from synth import make_problem

pytestmark = pytest.mark.gpu


def bf16(x):
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


def unpack(flat, width, depth):
    dims_in = [17] + [width] * depth
    dims_out = [width] * depth + [8]
    params, off = [], 0
    for i, o in zip(dims_in, dims_out):
        Wm = flat[off: off + i * o].reshape(o, i).astype(np.float64)
        off += i * o
        b = flat[off: off + o].astype(np.float64)
        off += o
        params.append((Wm, b))
    return params


@pytest.fixture
def small_net(lib):
    width, depth = 48, 2
    h = capi.calib_mlp_create(width, depth)
    rng = np.random.default_rng(5)
    n = capi.calib_mlp_num_params(h)
    w = bf16(0.2 * rng.standard_normal(n).astype(np.float32))
    capi.calib_mlp_set_weights(h, w)
    yield h, w, width, depth, rng
    capi.calib_mlp_destroy(h)


def test_forward_and_gradient_match_the_oracle(small_net):
    h, w, width, depth, rng = small_net
    n_rows = 300  # spans several 64-row tiles and a ragged tail
    X = rng.standard_normal((n_rows, 17)).astype(np.float32)
    T = rng.standard_normal((n_rows, 8)).astype(np.float32)
    params = unpack(w, width, depth)
    Y = np.zeros((n_rows, 8), dtype=np.float32)
    capi.calib_mlp_forward(h, X, Y)
    ref, _ = OM.forward(params, X.astype(np.float64))
    assert np.abs(Y - ref).max() <= 1e-4 * np.abs(ref).max()
    g = np.zeros(len(w), dtype=np.float32)
    loss = np.zeros(1)
    capi.calib_mlp_grad(h, X, T, g, loss)
    lref, gref = OM.loss_and_grads(params, X.astype(np.float64), T.astype(np.float64))
    assert loss[0] == pytest.approx(lref, rel=1e-5)
    flat_ref = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in gref])
    assert np.abs(g - flat_ref).max() <= 1e-4 * np.abs(flat_ref).max()


def test_adamw_step_matches_the_oracle(small_net):
    h, w, width, depth, rng = small_net
    X = rng.standard_normal((130, 17)).astype(np.float32)
    T = rng.standard_normal((130, 8)).astype(np.float32)
    params = unpack(w, width, depth)
    _, gref = OM.loss_and_grads(params, X.astype(np.float64), T.astype(np.float64))
    m = [[np.zeros_like(gw), np.zeros_like(gb)] for gw, gb in gref]
    v = [[np.zeros_like(gw), np.zeros_like(gb)] for gw, gb in gref]
    new = OM.adamw_step(params, gref, m, v, 1, lr=1e-3, wd=1e-2)
    capi.calib_mlp_train_step(h, X, T, 1e-3, 1e-2)
    got = capi.calib_mlp_get_weights(h)
    flat_new = np.concatenate([np.concatenate([a.ravel(), b]) for a, b in new])
    # first step moves each weight by about lr; compare the moves
    assert np.abs((got - w) - (flat_new - w)).max() <= 2e-5


@pytest.fixture(scope="module")
def small_sequence(lib):
    return make_problem("warm_n62_k5", N=16, K=2, P=8, I=8, T=4, seed=41)


def test_training_lowers_the_loss_and_the_start_is_never_worse(small_sequence):
    prob = small_sequence
    X, T = W.training_pairs(prob, n_transitions=3, n_iter=10)
    net = W.WarmStartNet(width=64, depth=3, seed=1)
    l0 = net.loss(X, T)
    hist = net.fit(X, T, epochs=80, batch=256, lr=1e-3)
    assert hist[-1] < hist[0] and net.loss(X, T) < l0
    # selection rule: the kept start never has a larger L_i than the previous solution
    calp, Jp, Zp, _ = W.solve_intervals(prob, [4, 5], 10)
    calp.close()
    vis, coh, Ts = W._interval_slice(prob, [5, 6])
    cal = W._context(prob, 2, Ts)
    cal.set_data(vis, coh)
    chose = np.zeros(cal.A, dtype=np.int32)
    capi.calib_warm_start(cal.ctx, net.h, Jp, Zp, chose)
    J0, _, _ = cal.solutions()
    L_kept, _, _ = cal.eval(J0)
    L_prev, _, _ = cal.eval(Jp.astype(np.complex64))
    assert np.all(L_kept <= L_prev * (1 + 1e-7))
    assert np.array_equal(chose == 1, np.any(J0 != Jp.astype(np.complex64), axis=(1, 2, 3, 4)))
    net.close()
    cal.close()


def test_warm_starts_reach_the_cold_residual_sooner(small_sequence):
    prob = small_sequence
    X, T = W.training_pairs(prob, n_transitions=3, n_iter=10)
    net = W.WarmStartNet(width=64, depth=3, seed=2)
    net.fit(X, T, epochs=80, batch=256, lr=1e-3)
    res = W.time_to_residual(prob, net, n_eval=4, n_iter=10)
    for name in ("previous", "network"):
        assert res[name]["reached"] == res[name]["of"]
        assert res[name]["iters_max"] <= res["plain"]["iters"]
    # the network's start is kept only where it lowers L_i, so the summed starting objective is never
    # higher; on this sequence it also starts closer to the target data cost
    assert res["network"]["start_objective"] <= res["previous"]["start_objective"] * (1 + 1e-9)
    assert res["network"]["start_data_cost_over_target"] < res["previous"]["start_data_cost_over_target"]
    # counted in single LM steps, the network's start stays closer after the first step too
    res1 = W.time_to_residual(prob, net, n_eval=4, n_iter=10, eval_n_lm=1)
    assert res1["network"]["mean_excess_after"][0] < res1["previous"]["mean_excess_after"][0]
    net.close()
