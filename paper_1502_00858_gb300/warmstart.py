"""Learned warm start of the calibration (driver; marshalling and orchestration only).

The paper starts a calibration from the previous time slot's solution (Section 3,
initialisation). Here a small network, trained on pairs the library's own C-ADMM produced,
refines that start: J_init = J_prev + net(J_prev, B_f Z_prev, f). Where the refined start does
not lower the augmented Lagrangian L_i it is discarded in favour of J_prev (calib_warm_start).

Everything numeric runs in libcalib.so: feature rows (calib_get_features), the forward and
backward passes and AdamW (calib_mlp_*), and the ADMM itself. Python draws the initial weights
and the mini-batch order (random numbers passed in as inputs) and moves arrays.
"""
from __future__ import annotations

import time

import numpy as np

from . import capi
from .calibrator import Calibrator


def init_weights(width: int = 256, depth: int = 3, seed: int = 0) -> np.ndarray:
    """Flat float32 weights in the library's layout: He-uniform hidden layers, zero biases, and a
    zero last layer, so an untrained network reproduces the previous-solution start exactly."""
    rng = np.random.default_rng(seed)
    dims_in = [17] + [width] * depth
    dims_out = [width] * depth + [8]
    parts = []
    for l, (i, o) in enumerate(zip(dims_in, dims_out)):
        if l == depth:
            W = np.zeros((o, i))
        else:
            bound = np.sqrt(6.0 / i)
            W = rng.uniform(-bound, bound, (o, i))
        parts += [W.ravel(), np.zeros(o)]
    return np.concatenate(parts).astype(np.float32)


class WarmStartNet:
    def __init__(self, width: int = 256, depth: int = 3, seed: int = 0):
        import torch

        self.width, self.depth = width, depth
        # One stream for the network and for the torch ops that feed it: batches are built and
        # consumed in stream order, so the caching allocator cannot recycle a batch still in use.
        self.stream = torch.cuda.Stream()
        self.h = capi.calib_mlp_create(width, depth, cuda_stream=self.stream.cuda_stream)
        capi.calib_mlp_set_weights(self.h, init_weights(width, depth, seed))

    def fit(self, X, T, epochs: int = 20, batch: int = 2048, lr: float = 1e-3, weight_decay: float = 1e-4,
            seed: int = 0, device: str = "cuda"):
        """Mini-batch AdamW on rows X [n,17] -> targets T [n,8] (host arrays). Returns the mean
        loss of each epoch (before each step's update)."""
        import torch

        n = X.shape[0]
        rng = np.random.default_rng(seed)
        history = []
        with torch.cuda.stream(self.stream):
            Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(device)
            Td = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).to(device)
            losses = torch.zeros((n + batch - 1) // batch, dtype=torch.float64, device=device)
            for _ in range(epochs):
                order = torch.from_numpy(rng.permutation(n)).to(device)
                weights = []
                for bi, s in enumerate(range(0, n, batch)):
                    idx = order[s:s + batch]
                    xb = Xd.index_select(0, idx).contiguous()
                    tb = Td.index_select(0, idx).contiguous()
                    capi.calib_mlp_train_step(self.h, xb, tb, lr, weight_decay, losses[bi:bi + 1])
                    weights.append(xb.shape[0])
                w = torch.tensor(weights, dtype=torch.float64, device=device)
                history.append(float((losses[:len(weights)] * w).sum().item() / n))
        return history

    def loss(self, X, T) -> float:
        out = np.zeros(1)
        capi.calib_mlp_grad(self.h, np.ascontiguousarray(X, np.float32), np.ascontiguousarray(T, np.float32), None, out)
        return float(out[0])

    def close(self):
        if self.h:
            capi.calib_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- data and evaluation

def _interval_slice(prob, ivs):
    """User-layout arrays (vis, coh) of the agents of the given intervals, in order."""
    P = prob["P"]
    agents = [iv * P + f for iv in ivs for f in range(P)]
    vis = np.concatenate([prob["V"][a].reshape(-1) for a in agents]).astype(np.complex64)
    coh = np.concatenate([prob["C"][a].reshape(-1) for a in agents]).astype(np.complex64)
    T = np.asarray(prob["T"])[agents]
    return vis, coh, T


def _context(prob, n_intervals, T, **kw):
    return Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                      n_intervals=n_intervals, samples=T, **kw)


def interval_g(cal, P):
    """Data cost g summed per solution interval (from the per-agent values)."""
    _, g = cal.agent_objective()
    return g.reshape(-1, P).sum(axis=1)


def solve_intervals(prob, ivs, n_iter, warm=None, mlp=None):
    """Calibrate the given intervals in one batched context. warm = (J_prev, Z_prev) starts
    each interval from its predecessor's solution (network-refined when mlp is given).
    Returns (calibrator, J, Z, features of the final state)."""
    vis, coh, T = _interval_slice(prob, ivs)
    cal = _context(prob, len(ivs), T)
    cal.set_data(vis, coh)
    if warm is not None:
        capi.calib_warm_start(cal.ctx, mlp.h if mlp is not None else None, warm[0], warm[1])
    cal.iterate(n_iter, want_hist=False)
    J, Z, _ = cal.solutions()
    X = np.zeros((cal.A * cal.K * cal.N, 17), dtype=np.float32)
    capi.calib_get_features(cal.ctx, X)
    return cal, J, Z, X


def training_pairs(prob, n_transitions, n_iter=30):
    """(features of interval iv's cold solution) -> (interval iv+1's solution warm-started from it)."""
    ivs = list(range(n_transitions + 1))
    cal0, J0, Z0, X0 = solve_intervals(prob, ivs[:-1], n_iter)
    cal0.close()
    cal1, J1, _, _ = solve_intervals(prob, ivs[1:], n_iter, warm=(J0, Z0))
    cal1.close()
    T = np.ascontiguousarray(J1).view(np.float32).reshape(-1, 8)
    return X0, T


# Relative tolerances of the steps-to-target table: g <= (1 + eps) x the cold start's n_iter-iteration cost.
TOLERANCES = (0.0, 1e-5, 3e-5, 1e-4, 3e-4, 1e-3)


def time_to_residual(prob, net, n_eval, n_iter=30, eval_n_lm=10):
    """For intervals 1..n_eval of a drifting sequence: the plain cold start's residual after n_iter
    iterations (10 LM steps each) is the target; report the iterations and wall time the
    previous-solution start and the network start need to reach it (per interval), plus the
    fraction of agents where the network's start was kept. eval_n_lm sets the LM steps per C-ADMM
    iteration of the two warm starts (1 counts single LM steps: a finer measure of the start).
    Also, per warm start, the iterations each interval needs to come within a relative tolerance of
    the target (TOLERANCES) and the mean excess data cost after each of the first iterations."""
    import torch

    P = prob["P"]
    prev = list(range(n_eval))
    cur = list(range(1, n_eval + 1))
    calp, Jp, Zp, _ = solve_intervals(prob, prev, n_iter)
    calp.close()
    vis, coh, T = _interval_slice(prob, cur)
    out = {}
    # plain: cold start
    cal = _context(prob, len(cur), T)
    cal.set_data(vis, coh)
    cal.iterate(1, want_hist=False)  # warm the graph cache and the autotuner
    cal.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cal.iterate(n_iter, want_hist=False)
    t_plain = time.perf_counter() - t0
    target = interval_g(cal, P) * (1 + 1e-9)
    out["plain"] = dict(iters=n_iter, seconds=t_plain)
    if eval_n_lm != 10:
        cal.close()
        cal = _context(prob, len(cur), T, n_lm=eval_n_lm)
        cal.set_data(vis, coh)
        n_iter = n_iter * 10 // eval_n_lm
    out["eval_n_lm"] = eval_n_lm
    for name, use_net in (("previous", False), ("network", True)):
        chose = np.zeros(cal.A, dtype=np.int32)
        capi.calib_warm_start(cal.ctx, net.h if use_net else None, Jp, Zp, chose)
        J0, _, _ = cal.solutions()
        L0, g0, _ = cal.eval(J0)  # objective and data cost at the start
        need = np.full(len(cur), -1)
        g_first = None
        ratio = []  # per iteration: each interval's data cost / target
        for it in range(1, n_iter + 1):
            cal.iterate(1, want_hist=False)
            g = interval_g(cal, P)
            ratio.append(g / target)
            if it == 1:
                g_first = g.copy()
            need[(need < 0) & (g <= target)] = it
        ratio = np.array(ratio)
        within = {}
        for eps in TOLERANCES:  # iterations until g <= (1 + eps) target, per interval
            hit = ratio <= 1.0 + eps
            steps = np.where(hit.any(0), hit.argmax(0) + 1, n_iter + 1)
            within[f"{eps:g}"] = dict(median=float(np.median(steps)), mean=float(steps.mean()), max=int(steps.max()))
        reached = need[need > 0]
        n_max = int(reached.max()) if reached.size else n_iter
        # wall time of a batched run of that many iterations from the same start
        capi.calib_warm_start(cal.ctx, net.h if use_net else None, Jp, Zp, None)
        cal.iterate(n_max, want_hist=False)  # cache the graph for n_max
        capi.calib_warm_start(cal.ctx, net.h if use_net else None, Jp, Zp, None)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cal.iterate(n_max, want_hist=False)
        secs = time.perf_counter() - t0
        out[name] = dict(iters_median=float(np.median(np.where(need > 0, need, n_iter + 1))),
                         iters_max=n_max, reached=int(reached.size), of=len(cur), seconds=secs,
                         network_kept=float(chose.mean()) if use_net else 0.0,
                         start_objective=float(L0.sum()), start_data_cost_over_target=float(g0.sum() / target.sum()),
                         after_one_iter_data_cost_over_target=float(g_first.sum() / target.sum()),
                         iters_to_within=within,
                         mean_excess_after=[float(ratio[i].mean() - 1.0) for i in range(min(5, n_iter))])
    cal.close()
    return out


def main(argv=None):
    """Train on ~20k rows from one interval transition of the 62-station, 5-direction, 64-subband
    sequence, then report time to the plain method's residual on n_eval new seeded intervals."""
    import argparse
    import json

    import torch

    from synth import make_problem

    ap = argparse.ArgumentParser()
    ap.add_argument("--n-eval", type=int, default=200)
    ap.add_argument("--transitions", type=int, default=1)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--width", type=int, default=256)
    ap.add_argument("--depth", type=int, default=3)
    ap.add_argument("--iters", type=int, default=30)
    ap.add_argument("--eval-lm", type=int, default=10, help="LM steps per C-ADMM iteration of the warm starts")
    args = ap.parse_args(argv)
    t0 = time.perf_counter()
    train = make_problem("warm_n62_k5", I=args.transitions + 1, seed=4, dtype=np.complex64)
    X, T = training_pairs(train, args.transitions, args.iters)
    del train
    net = WarmStartNet(args.width, args.depth, seed=0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = net.fit(X, T, epochs=args.epochs, batch=2048, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    ev = make_problem("warm_n62_k5", I=args.n_eval + 1, seed=1000, dtype=np.complex64)
    res = time_to_residual(ev, net, args.n_eval, args.iters, args.eval_lm)
    print(json.dumps({"workload": "warm_n62_k5 (N=62, K=5, 64 subbands, T=10)", "train_rows": int(X.shape[0]),
                      "epochs": args.epochs, "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                      "train_seconds": round(t_train, 3), "eval_intervals": args.n_eval, "admm_iters": args.iters,
                      "result": res, "total_seconds": round(time.perf_counter() - t0, 1)}), flush=True)
    net.close()


if __name__ == "__main__":
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main()
