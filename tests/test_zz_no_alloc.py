"""calib_eval_noalloc: the allocation-free variant of calib_eval.

It serves callers that cannot call cudaMalloc - work enqueued during a global-mode stream
capture, applications whose device memory belongs to their own pool allocator, and
latency-critical pipelines that must avoid the implicit synchronisation of cudaMalloc/cudaFree.
Its output must equal calib_eval's on the same inputs, call after call, although every call
reuses the same fixed scratch array. This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

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
