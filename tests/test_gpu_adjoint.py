"""Adjoint (torch.autograd.Function over the library's gradient sweep) on the adjoint-check
workload: 16 stations, 3 directions, 8 frequencies, 2 samples. Checked against central finite
differences of the same forward in float32 (step 1e-3) and against the oracle's float64
gradient (Eq. gradL; PyTorch's convention is twice the h-gradient)."""
import math

import numpy as np
import pytest

from oracle import admm as O
from paper_1502_00858_gb300 import Calibrator
from synth import make_problem, user_layout

pytestmark = pytest.mark.gpu


def cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


@pytest.fixture(scope="module")
def setup(lib):
    torch = pytest.importorskip("torch")
    prob = make_problem("adjoint_n16_k3")
    ul = user_layout(prob)
    cal = Calibrator(prob["N"], prob["pq"], prob["K"], prob["freqs"], prob["basis"], prob["rho"],
                     n_intervals=prob["I"], samples=prob["T"])
    cal.set_data(ul["vis"], ul["coh"])
    rng = np.random.default_rng(31)
    Z = 0.1 * cn(rng, prob["I"], prob["K"], prob["M"], prob["N"], 2, 2)
    Y = (0.3 * cn(rng, prob["A"], prob["K"], prob["N"], 2, 2)).astype(np.complex64)
    cal.set_consensus(Z, Y)
    J0 = (prob["J_true"] + 0.05 * cn(rng, *prob["J_true"].shape)).astype(np.complex64)
    return torch, prob, cal, Z, Y, J0, rng


def test_adjoint_matches_the_oracle_gradient(setup):
    from paper_1502_00858_gb300.adjoint import admm_loss
    torch, prob, cal, Z, Y, J0, rng = setup
    J = torch.tensor(J0, device="cuda", requires_grad=True)
    L = admm_loss(J, cal)
    L.sum().backward()
    G = J.grad.cpu().numpy()
    pr = dict(prob, V=[c64(v) for v in prob["V"]], C=[c64(c) for c in prob["C"]])
    P = prob["P"]
    for a in range(prob["A"]):
        V, C, pq = O.agent_data(pr, a)
        BZ = c64(O.bz(Z[a // P], prob["basis"][a % P]))
        ref = 2.0 * O.grad_lagrangian(J0[a].astype(np.complex128), V, C, pq, Y[a].astype(np.complex128), BZ, prob["rho"])
        assert np.abs(G[a] - ref).max() <= 1e-4 * np.abs(ref).max()
        Lo = O.aug_lagrangian(J0[a].astype(np.complex128), V, C, pq, Y[a].astype(np.complex128), BZ, prob["rho"])
        assert float(L[a].detach()) == pytest.approx(Lo, rel=2e-5)


def test_adjoint_matches_central_differences(setup):
    from paper_1502_00858_gb300.adjoint import admm_loss
    torch, prob, cal, Z, Y, J0, rng = setup
    J = torch.tensor(J0, device="cuda", requires_grad=True)
    w = torch.tensor(rng.uniform(0.5, 1.5, prob["A"]), device="cuda")  # weights: backward scales per agent
    (admm_loss(J, cal) * w).sum().backward()
    G = J.grad
    eps = 1e-3
    for _ in range(4):
        xi = torch.tensor(cn(rng, *J0.shape).astype(np.complex64), device="cuda")
        with torch.no_grad():
            lp = float((admm_loss(J.detach() + eps * xi, cal) * w).sum())
            lm = float((admm_loss(J.detach() - eps * xi, cal) * w).sum())
        fd = (lp - lm) / (2 * eps)
        ad = float(torch.real(torch.sum(torch.conj(G) * xi)))
        assert fd == pytest.approx(ad, rel=1e-2)
