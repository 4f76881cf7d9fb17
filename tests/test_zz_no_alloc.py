"""calib_eval_noalloc: the allocation-free variant of calib_eval.

It serves callers that cannot call cudaMalloc - applications whose device memory belongs to
their own pool allocator, and latency-critical pipelines that must avoid the implicit
synchronisation of cudaMalloc/cudaFree. Its output must equal calib_eval's and the oracle's on
the same inputs, call after call, although every call reuses the same fixed scratch array
(per-chunk partial sums of 256 baselines). This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

from oracle import admm as O
from paper_1502_00858_gb300 import Calibrator, capi
from synth import make_problem, user_layout


def cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def test_noalloc_rejects_a_problem_larger_than_its_scratch():
    """Checked on the host before anything touches a device (the pointers are never read)."""
    capi.load()
    fake = 16  # non-null placeholders
    rho = np.ones(5)
    rc = capi.load().calib_eval_noalloc(4096, 62, 1891, 5, 10, fake, fake, fake, fake, None, None,
                                        rho.ctypes.data, None, None, fake, None)
    assert rc == capi.CALIB_EINVAL
    assert "scratch" in capi.load().calib_last_error().decode()


@pytest.mark.gpu
def test_noalloc_matches_calib_eval_on_two_calls_in_a_row(lib):
    torch = pytest.importorskip("torch")
    prob = make_problem("adjoint_n16_k3", N=20, K=3, P=4, I=1, T=6, seed=21)
    A, N, K, P, B, T = prob["A"], prob["N"], prob["K"], prob["P"], prob["B"], 6
    ul = user_layout(prob)
    cal = Calibrator(N, prob["pq"], K, prob["freqs"], prob["basis"], prob["rho"], n_intervals=1, samples=T)
    cal.set_data(ul["vis"], ul["coh"])
    rng = np.random.default_rng(22)
    Z = 0.1 * cn(rng, 1, K, prob["M"], N, 2, 2)
    Y = (0.3 * cn(rng, A, K, N, 2, 2)).astype(np.complex64)
    cal.set_consensus(Z, Y)
    BZ = np.stack([np.einsum("l,klnij->knij", prob["basis"][a % P], Z[0]) for a in range(A)]).astype(np.complex64)

    dev = torch.device("cuda", 0)

    def d(x, dtype):
        return torch.from_numpy(np.ascontiguousarray(x).view(dtype)).to(dev)

    pq_d = d(prob["pq"].astype(np.int32), np.int32)
    vis_d = d(ul["vis"], np.float32)
    coh_d = d(ul["coh"], np.float32)
    Y_d = d(Y, np.float32)
    BZ_d = d(BZ, np.float32)
    L_d = torch.zeros(A, dtype=torch.float64, device=dev)
    g_d = torch.zeros(A, dtype=torch.float64, device=dev)
    grad_d = torch.zeros(A * K * N * 8, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    for call in range(2):
        J = (prob["J_true"] + 0.05 * (call + 1) * cn(rng, A, K, N, 2, 2)).astype(np.complex64)
        L_ref, g_ref, grad_ref = cal.eval(J)
        J_d = d(J, np.float32)
        torch.cuda.synchronize()
        capi.calib_eval_noalloc(A, N, B, K, T, pq_d, vis_d, coh_d, J_d, Y_d, BZ_d, prob["rho"],
                                L_d, g_d, grad_d, None)
        torch.cuda.synchronize()
        L = L_d.cpu().numpy()
        g = g_d.cpu().numpy()
        grad = grad_d.cpu().numpy().view(np.complex64).reshape(A, K, N, 2, 2)
        np.testing.assert_allclose(g, g_ref, rtol=2e-5, err_msg=f"call {call}")
        np.testing.assert_allclose(L, L_ref, rtol=2e-5, err_msg=f"call {call}")
        scale = np.abs(grad_ref).max()
        assert np.abs(grad - grad_ref).max() <= 1e-4 * scale, f"call {call}"
    cal.close()


def _random_agents(seed, A, N, K, T):
    """Seeded synthetic agents: noisy data of a random truth, evaluated near it (complex64)."""
    rng = np.random.default_rng(seed)
    pq = np.array([(p, q) for p in range(N) for q in range(p + 1, N)], dtype=np.int32)
    B = len(pq)
    C = (cn(rng, A, B, T, K) * 1.5).astype(np.complex64)
    Jt = np.eye(2) + 0.2 * cn(rng, A, K, N, 2, 2)
    V = np.stack([O.model_vis(Jt[a], C[a].astype(np.complex128), pq) for a in range(A)])
    V = (V + 0.2 * cn(rng, *V.shape)).astype(np.complex64)
    J = (Jt + 0.05 * cn(rng, A, K, N, 2, 2)).astype(np.complex64)
    Y = (0.3 * cn(rng, A, K, N, 2, 2)).astype(np.complex64)
    BZ = (np.eye(2) + 0.1 * cn(rng, A, K, N, 2, 2)).astype(np.complex64)
    rho = np.linspace(2.0, 9.0, K)
    return dict(pq=pq, B=B, C=C, V=V, J=J, Y=Y, BZ=BZ, rho=rho, A=A, N=N, K=K, T=T)


def _run_noalloc(torch, c, with_consensus=True, with_scalars=True, pq=None):
    dev = torch.device("cuda", 0)

    def d(x, dtype):
        return torch.from_numpy(np.ascontiguousarray(x).view(dtype)).to(dev)

    A, N, K = c["A"], c["N"], c["K"]
    L_d = torch.full((A,), -1.0, dtype=torch.float64, device=dev) if with_scalars else None
    g_d = torch.full((A,), -1.0, dtype=torch.float64, device=dev) if with_scalars else None
    grad_d = torch.zeros(A * K * N * 8, dtype=torch.float32, device=dev)
    ins = [d(c["pq"] if pq is None else pq, np.int32), d(c["V"], np.float32), d(c["C"], np.float32),
           d(c["J"], np.float32)]
    Y_d = d(c["Y"], np.float32) if with_consensus else None
    BZ_d = d(c["BZ"], np.float32) if with_consensus else None
    torch.cuda.synchronize()
    capi.calib_eval_noalloc(A, N, c["B"], K, c["T"], *ins, Y_d, BZ_d, c["rho"], L_d, g_d, grad_d, None)
    torch.cuda.synchronize()
    grad = grad_d.cpu().numpy().view(np.complex64).reshape(A, K, N, 2, 2)
    return (L_d.cpu().numpy() if with_scalars else None), (g_d.cpu().numpy() if with_scalars else None), grad


def _oracle(c, with_consensus=True):
    """Per agent (L, g, grad) of the float64 oracle on the same complex64 inputs (Eq. gradL, Eq. sumtrace2)."""
    L, g, grad = [], [], []
    for a in range(c["A"]):
        J = c["J"][a].astype(np.complex128)
        V = c["V"][a].astype(np.complex128)
        C = c["C"][a].astype(np.complex128)
        Y = c["Y"][a].astype(np.complex128) if with_consensus else np.zeros_like(J)
        BZ = c["BZ"][a].astype(np.complex128) if with_consensus else np.zeros_like(J)
        g.append(O.data_cost(J, V, C, c["pq"]))
        L.append(O.aug_lagrangian(J, V, C, c["pq"], Y, BZ, c["rho"]))
        grad.append(O.grad_lagrangian(J, V, C, c["pq"], Y, BZ, c["rho"]))
    return np.array(L), np.array(g), np.stack(grad)


def _check(c, got, ref, label):
    L, g, grad = got
    L_ref, g_ref, grad_ref = ref
    if L is not None:
        np.testing.assert_allclose(g, g_ref, rtol=1e-4, err_msg=label)
        np.testing.assert_allclose(L, L_ref, rtol=1e-4, err_msg=label)
    scale = np.abs(grad_ref).max()
    assert np.abs(grad - grad_ref).max() <= 1e-4 * scale, label


@pytest.mark.gpu
def test_noalloc_with_several_chunks_matches_the_oracle_and_a_smaller_call_after_it(lib):
    """62 stations (1891 baselines, 8 chunks of 256) and then 24 stations (276 baselines, 2 chunks)
    with another K: the second call reads only slots it wrote, so stale partial sums of the larger
    first call cannot leak into it. The second call also takes Y = BZ = NULL (zero)."""
    torch = pytest.importorskip("torch")
    big = _random_agents(31, A=2, N=62, K=5, T=3)
    _check(big, _run_noalloc(torch, big), _oracle(big), "N=62, 8 chunks")
    small = _random_agents(32, A=3, N=24, K=3, T=4)
    _check(small, _run_noalloc(torch, small, with_consensus=False), _oracle(small, with_consensus=False),
           "N=24, 2 chunks, Y = BZ = NULL")
    # L and g may be NULL: only grad is written
    _, _, grad = _run_noalloc(torch, small, with_scalars=False)
    _check(small, (None, None, grad), _oracle(small), "L = g = NULL")


@pytest.mark.gpu
def test_noalloc_at_its_largest_shared_memory_shape_matches_the_oracle(lib):
    """K=16 directions and N=128 stations: 2 K N 32 B = 128 KiB of shared memory per CTA (J and the
    station sums), 8128 baselines in 32 chunks."""
    torch = pytest.importorskip("torch")
    c = _random_agents(33, A=1, N=128, K=16, T=2)
    _check(c, _run_noalloc(torch, c), _oracle(c), "N=128, K=16")


@pytest.mark.gpu
def test_noalloc_marks_every_result_invalid_for_a_station_pair_out_of_range(lib):
    """A pair with q = N is skipped on the device (never used as an index) and makes L, g and
    grad NaN; the next call with valid pairs is correct again."""
    torch = pytest.importorskip("torch")
    c = _random_agents(34, A=2, N=24, K=3, T=2)
    bad = c["pq"].copy()
    bad[100] = (5, c["N"])
    L, g, grad = _run_noalloc(torch, c, pq=bad)
    assert np.all(np.isnan(L)) and np.all(np.isnan(g)) and np.all(np.isnan(grad))
    _check(c, _run_noalloc(torch, c), _oracle(c), "valid pairs after an invalid call")
