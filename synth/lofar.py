"""Seeded, LOFAR-shaped synthetic calibration problems.

What this module does: it draws random numbers (station layout, sky model, true
Jones matrices, noise, flags, per-subband sample counts), builds the observing
geometry (station uvw tracks for a north-celestial-pole pointing), and synthesises
noisy visibilities from them by a forward simulation of the data model of
Section 2 (Eq. vispq with the unpolarised coherency of Eq. coh).

What it does not do: any calibration arithmetic. There is no cost, gradient,
Hessian, damping, consensus (Z) or dual (Y) step here. Both the CUDA path and the
CPU oracle take the arrays produced here as plain inputs; neither imports the
other.

Shapes follow the simulation section (Section 4: 115-185 MHz, LOFAR-like array at
the NCP, 10 s samples, point-source clusters inside a 7x7 degree field).

Array conventions (all float64 / complex128):
  pq      int32 [B,2]          every station pair p<q, row-major over p
  freqs   [P] Hz               one per frequency agent
  basis   [P,M]                b_l(f_i), the smoothness basis rows (Eq. hidden/poly)
  rho     [K]                  per-direction regularisation
  T       int [A]              samples in each agent's solution interval, A = I*P,
                               agent a = interval*P + frequency index
  flags   uint8 [A,B]          1 = baseline flagged (excluded) for that agent
  uvw     [I,Tmax,N,3] metres  per-station (u,v,w) for each interval and sample
  sky     [K,S,4]              per cluster: l, m (direction cosines), I0 (Jy at f0), alpha
  J_true  [A,K,N,2,2]          true Jones matrices
  V       list of A arrays [B,T_a,2,2]   noisy visibilities (flagged rows still present)
  C       list of A arrays [B,T_a,K]     scalar coherencies c with C = c * I_2
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import math
import os
from typing import Sequence

import numpy as np

C_LIGHT = 299792458.0
SIDEREAL_RATE = 2.0 * math.pi / 86164.0905  # rad / s
LOFAR_LAT = math.radians(52.9)
SAMPLE_SECONDS = 10.0
F0_HZ = 150e6


@dataclasses.dataclass(frozen=True)
class ProblemSpec:
    name: str
    N: int
    K: int
    P: int
    I: int
    T: int | tuple[int, ...]  # int = every agent; tuple = per-subband choice set
    n_src: int  # sources per cluster
    sky_kind: str  # "uniform_small" or "clusters"
    basis_kind: str  # "poly" or "bernstein"
    degree: int
    rho: float
    snr: float
    n_admm: int
    jones_kind: str  # "poly_deg2" or "smooth_deg3"
    flag_max: float = 0.0
    fmin: float = 115e6
    fmax: float = 185e6
    seed: int = 0
    n_bg: int = 0            # weak background sources, not corrupted by any Jones matrix
    bg_flux_max: float = 0.1  # their peak flux (Jy), flat spectrum

    @property
    def M(self) -> int:
        return self.degree + 1

    @property
    def B(self) -> int:
        return self.N * (self.N - 1) // 2


SPECS: dict[str, ProblemSpec] = {
    # plain ADMM, 8 stations (28 baselines), one direction of 4 sources, 4 frequencies.
    "tiny_n8_k1": ProblemSpec("tiny_n8_k1", N=8, K=1, P=4, I=1, T=10, n_src=4,
                              sky_kind="uniform_small", basis_kind="poly", degree=2,
                              rho=5.0, snr=50.0, n_admm=10, jones_kind="poly_deg2", seed=0),
    # LOFAR-shaped: 62 stations (1891 baselines), 5 clusters x 20 sources, 32 subbands,
    # 10 solution intervals of 10 samples, Bernstein degree 3, rho 10, SNR 10, 30 iterations.
    "lofar_n62_k5": ProblemSpec("lofar_n62_k5", N=62, K=5, P=32, I=10, T=10, n_src=20,
                                sky_kind="clusters", basis_kind="bernstein", degree=3,
                                rho=10.0, snr=10.0, n_admm=30, jones_kind="smooth_deg3", seed=1),
    # uneven batch: 256 subbands with 5/10/20 samples each and 0-15 % flagged baselines.
    "uneven_n62_k10": ProblemSpec("uneven_n62_k10", N=62, K=10, P=256, I=10, T=(5, 10, 20), n_src=20,
                                  sky_kind="clusters", basis_kind="bernstein", degree=3,
                                  rho=10.0, snr=10.0, n_admm=50, jones_kind="smooth_deg3",
                                  flag_max=0.15, seed=2),
    # learned warm start: 62 stations, 5 directions, 64 subbands, drifting consecutive intervals.
    "warm_n62_k5": ProblemSpec("warm_n62_k5", N=62, K=5, P=64, I=3, T=10, n_src=20,
                               sky_kind="clusters", basis_kind="bernstein", degree=3,
                               rho=10.0, snr=10.0, n_admm=30, jones_kind="smooth_deg3", seed=4),
    # Simulation I (Section 4): one direction, 47 stations, 32 channels over 115-185 MHz, 20
    # samples, Jones varying in time and frequency (G = 4), 300 weak uncorrupted background
    # sources, noise power 10 % of the signal power; ordinary polynomial basis.
    "sim1_n47_k1": ProblemSpec("sim1_n47_k1", N=47, K=1, P=32, I=1, T=20, n_src=1,
                               sky_kind="clusters", basis_kind="poly", degree=1,
                               rho=5.0, snr=10.0, n_admm=50, jones_kind="sim1_time", seed=5,
                               n_bg=300),
    # adjoint check size: 16 stations, 3 directions, 8 frequencies, 2 samples.
    "adjoint_n16_k3": ProblemSpec("adjoint_n16_k3", N=16, K=3, P=8, I=1, T=2, n_src=5,
                                  sky_kind="clusters", basis_kind="bernstein", degree=3,
                                  rho=10.0, snr=10.0, n_admm=5, jones_kind="smooth_deg3", seed=3),
}


# ----------------------------------------------------------------------------- geometry

def station_layout(rng: np.random.Generator, N: int) -> np.ndarray:
    """Equatorial XYZ (m) of N stations: log-uniform radius 50 m..40 km, uniform azimuth,
    N(0, 10 m) height, rotated from the local horizon frame at latitude 52.9 deg."""
    r = np.exp(rng.uniform(math.log(50.0), math.log(40e3), N))
    az = rng.uniform(0.0, 2 * math.pi, N)
    e, n, u = r * np.sin(az), r * np.cos(az), rng.normal(0.0, 10.0, N)
    s, c = math.sin(LOFAR_LAT), math.cos(LOFAR_LAT)
    return np.stack([-s * n + c * u, e, c * n + s * u], axis=1)


def station_uvw(xyz: np.ndarray, I: int, Tmax: int, h0: float = 0.3) -> np.ndarray:
    """Per-station (u,v,w) in metres for a pointing at declination 90 deg (the NCP):
    the textbook rotation of equatorial XYZ by hour angle H; samples SAMPLE_SECONDS apart."""
    n_samp = I * Tmax
    H = h0 + SIDEREAL_RATE * SAMPLE_SECONDS * np.arange(n_samp)
    sH, cH = np.sin(H)[:, None], np.cos(H)[:, None]
    X, Y, Z = xyz[:, 0][None, :], xyz[:, 1][None, :], xyz[:, 2][None, :]
    u = sH * X + cH * Y
    v = -cH * X + sH * Y
    w = np.broadcast_to(Z, u.shape)
    return np.stack([u, v, w], axis=-1).reshape(I, Tmax, xyz.shape[0], 3)


def all_pairs(N: int) -> np.ndarray:
    return np.array([(p, q) for p in range(N) for q in range(p + 1, N)], dtype=np.int32).reshape(-1, 2)


def basis_matrix(kind: str, degree: int, freqs: np.ndarray) -> np.ndarray:
    """Rows b(f_i). 'poly': ((f-f0)/f0)^l with f0 = 150 MHz (Eq. hidden);
    'bernstein': C(d,l) x^l (1-x)^(d-l), x = (f-fmin)/(fmax-fmin)."""
    if kind == "poly":
        x = (freqs - F0_HZ) / F0_HZ
        return np.stack([x ** l for l in range(degree + 1)], axis=1)
    if kind == "bernstein":
        x = (freqs - freqs.min()) / (freqs.max() - freqs.min())
        return np.stack([math.comb(degree, l) * x ** l * (1 - x) ** (degree - l)
                         for l in range(degree + 1)], axis=1)
    raise ValueError(kind)


def make_sky(rng: np.random.Generator, spec: ProblemSpec) -> np.ndarray:
    """[K,S,4] = (l, m, I0 at 150 MHz, spectral index)."""
    K, S = spec.K, spec.n_src
    sky = np.zeros((K, S, 4))
    if spec.sky_kind == "uniform_small":
        sky[..., 0] = rng.uniform(-0.05, 0.05, (K, S))
        sky[..., 1] = rng.uniform(-0.05, 0.05, (K, S))
        sky[..., 2] = rng.uniform(1.0, 10.0, (K, S))
        sky[..., 3] = 0.0
        return sky
    half = math.radians(3.5)
    centres = rng.uniform(-half, half, (K, 2))
    rad = math.radians(0.5) * np.sqrt(rng.uniform(0, 1, (K, S)))
    ang = rng.uniform(0, 2 * math.pi, (K, S))
    sky[..., 0] = np.sin(centres[:, 0:1] + rad * np.cos(ang))
    sky[..., 1] = np.sin(centres[:, 1:2] + rad * np.sin(ang))
    sky[..., 2] = 1.0 * (1.0 + rng.pareto(1.5, (K, S)))  # Pareto, minimum 1 Jy, index 1.5
    sky[..., 3] = rng.uniform(-1.0, 1.0, (K, S))
    return sky


def make_jones(rng: np.random.Generator, spec: ProblemSpec, freqs: np.ndarray) -> np.ndarray:
    """True Jones [I,P,K,N,2,2]: identity plus a smooth polynomial in x=(f-f0)/f0."""
    I, P, K, N = spec.I, spec.P, spec.K, spec.N
    x = (freqs - F0_HZ) / F0_HZ
    eye = np.eye(2)

    def cn(*shape):
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)

    if spec.jones_kind == "poly_deg2":
        G = cn(K, N, 3, 2, 2)
        Jf = eye + 0.1 * np.einsum("knlij,fl->fknij", G, np.stack([x ** l for l in range(3)], 1))
        return np.broadcast_to(Jf, (I,) + Jf.shape).copy()
    if spec.jones_kind == "smooth_deg3":
        A0 = cn(K, N, 4, 2, 2)
        D = 0.3 * cn(K, N, 4, 2, 2)
        al = rng.uniform(0, 1, (K, N, 4, 1, 1))
        be = rng.uniform(0, 1, (K, N, 4, 1, 1))
        xs = np.stack([x ** l for l in range(4)], 1)  # [P,4]
        out = np.empty((I, P, K, N, 2, 2), dtype=complex)
        for iv in range(I):
            G = A0 + D * np.sin(al * iv + 2 * math.pi * be)  # drifts between intervals
            out[iv] = eye + 0.1 * np.einsum("knlij,fl->fknij", G, xs)
        out += 0.01 * cn(I, P, K, N, 2, 2)  # 1 % per-channel perturbation
        return out
    raise ValueError(spec.jones_kind)


def make_jones_time(rng: np.random.Generator, spec: ProblemSpec, freqs: np.ndarray, Tmax: int) -> np.ndarray:
    """Simulation I Jones matrices [I,P,Tmax,K,N,2,2] (Section 4): every element is the product of a
    time factor sin(a1 t' + 2 pi b1) + i sin(a2 t' + 2 pi b2) and a frequency polynomial
    sum_{l=1..4} (g_l + i d_l) ((f - f0)/f0)^(l-1), with a1, a2, b1, b2, g_l, d_l ~ U(0,1) drawn per
    station, direction and element. t' is the sample's time in hours since the start of the
    observation (10 s samples; solution interval iv starts at iv * T samples)."""
    I, P, K, N = spec.I, spec.P, spec.K, spec.N
    G = 4
    a = rng.uniform(0, 1, (4, K, N, 2, 2))       # a1, a2, b1, b2
    gd = rng.uniform(0, 1, (2, G, K, N, 2, 2))   # g_l, d_l
    x = (freqs - F0_HZ) / F0_HZ
    xs = np.stack([x ** l for l in range(G)], 0)  # [G,P]
    freq = np.einsum("lknij,lf->fknij", gd[0] + 1j * gd[1], xs)  # [P,K,N,2,2]
    out = np.empty((I, P, Tmax, K, N, 2, 2), dtype=complex)
    for iv in range(I):
        tp = (iv * Tmax + np.arange(Tmax)) * SAMPLE_SECONDS / 3600.0  # hours
        tm = (np.sin(a[0][None] * tp[:, None, None, None, None] + 2 * math.pi * a[2][None])
              + 1j * np.sin(a[1][None] * tp[:, None, None, None, None] + 2 * math.pi * a[3][None]))  # [T,K,N,2,2]
        out[iv] = freq[:, None] * tm[None]
    return out


# ----------------------------------------------------------------------------- forward simulation

def simulate_coherencies(uvw_t: np.ndarray, sky: np.ndarray, f: float, pq: np.ndarray) -> np.ndarray:
    """Scalar coherencies [B,T,K] at frequency f for per-station uvw [T,N,3].

    Unpolarised point sources give C = c I_2 (Eq. coh). The baseline phase factorises
    into per-station phasors because u_pq = u_p - u_q; each cluster's c is
    sum_s I_s(f) E_ps conj(E_qs) with E_ps = exp(-2 pi i f/c (u_p l + v_p m + w_p (n-1))).
    """
    l, m = sky[..., 0], sky[..., 1]
    n1 = np.sqrt(1.0 - l * l - m * m) - 1.0
    flux = sky[..., 2] * (f / F0_HZ) ** sky[..., 3]  # [K,S]
    K = sky.shape[0]
    T, N = uvw_t.shape[0], uvw_t.shape[1]
    out = np.empty((len(pq), T, K), dtype=complex)
    for k in range(K):
        turns = (f / C_LIGHT) * (uvw_t[..., 0:1] * l[k] + uvw_t[..., 1:2] * m[k] + uvw_t[..., 2:3] * n1[k])
        E = np.exp(-2j * math.pi * turns)  # [T,N,S]
        G = np.matmul(E * flux[k], np.conj(E).transpose(0, 2, 1))  # [T,N,N]
        out[:, :, k] = G[:, pq[:, 0], pq[:, 1]].T
    return out


def simulate_visibilities(Jt: np.ndarray, C: np.ndarray, pq: np.ndarray) -> np.ndarray:
    """Noise-free sum_k c_k J_pk J_qk^H, [B,T,2,2], from Jones [K,N,2,2] and c [B,T,K]."""
    Jp = Jt[:, pq[:, 0]]  # [K,B,2,2]
    JqH = np.conj(Jt[:, pq[:, 1]]).transpose(0, 1, 3, 2)
    A = np.matmul(Jp, JqH)  # [K,B,2,2]
    return np.einsum("btk,kbij->btij", C, A)


# ----------------------------------------------------------------------------- top level

def make_problem(spec: ProblemSpec | str, seed: int | None = None, *, I: int | None = None,
                 P: int | None = None, N: int | None = None, K: int | None = None,
                 T: int | Sequence[int] | None = None, flag_max: float | None = None,
                 noise: bool = True, dtype=complex, coherencies: bool = True) -> dict:
    """Build a seeded problem. Keyword overrides shrink or reshape a named spec.
    coherencies=False drops the simulated coherencies from the result (C is None) for callers
    that predict them from uvw and sky; every other array is unchanged."""
    if isinstance(spec, str):
        spec = SPECS[spec]
    kw = {}
    for key, val in (("I", I), ("P", P), ("N", N), ("K", K), ("flag_max", flag_max)):
        if val is not None:
            kw[key] = val
    if T is not None:
        kw["T"] = tuple(T) if not isinstance(T, int) else T
    if seed is not None:
        kw["seed"] = seed
    spec = dataclasses.replace(spec, **kw)
    rng = np.random.default_rng(spec.seed)

    N, K, P, I = spec.N, spec.K, spec.P, spec.I
    A = I * P
    pq = all_pairs(N)
    B = len(pq)
    freqs = np.linspace(spec.fmin, spec.fmax, P) if P > 1 else np.array([F0_HZ])
    basis = basis_matrix(spec.basis_kind, spec.degree, freqs) if P > 1 else np.ones((1, spec.M))
    rho = np.full(K, spec.rho)
    if isinstance(spec.T, int):
        T_sub = np.full(P, spec.T, dtype=np.int32)
    else:
        T_sub = rng.choice(np.array(spec.T, dtype=np.int32), size=P)
    T_agent = np.tile(T_sub, I).astype(np.int32)
    Tmax = int(T_sub.max())

    xyz = station_layout(rng, N)
    uvw = station_uvw(xyz, I, Tmax)
    sky = make_sky(rng, spec)
    J_true_t = None
    if spec.jones_kind == "sim1_time":
        J_true_t = make_jones_time(rng, spec, freqs, Tmax).reshape(A, Tmax, K, N, 2, 2)
        J_true = np.stack([J_true_t[a, :int(T_agent[a])].mean(axis=0) for a in range(A)])
    else:
        J_true = make_jones(rng, spec, freqs).reshape(A, K, N, 2, 2)

    flags = np.zeros((A, B), dtype=np.uint8)
    if spec.flag_max > 0:
        frac = rng.uniform(0.0, spec.flag_max, A)
        flags = (rng.uniform(0, 1, (A, B)) < frac[:, None]).astype(np.uint8)
    sky_bg = None
    if spec.n_bg > 0:  # weak background sources over the 7 x 7 degree field, flat spectrum
        half = math.radians(3.5)
        sky_bg = np.zeros((1, spec.n_bg, 4))
        sky_bg[0, :, 0] = np.sin(rng.uniform(-half, half, spec.n_bg))
        sky_bg[0, :, 1] = np.sin(rng.uniform(-half, half, spec.n_bg))
        sky_bg[0, :, 2] = rng.uniform(0.0, spec.bg_flux_max, spec.n_bg)

    def agent(a):  # deterministic (no random draws): safe to run agents concurrently
        iv, fi = divmod(a, P)
        Ta = int(T_agent[a])
        C = simulate_coherencies(uvw[iv, :Ta], sky, float(freqs[fi]), pq)
        if J_true_t is None:
            V = simulate_visibilities(J_true[a], C, pq)
        else:  # Jones matrices of every sample
            V = np.concatenate([simulate_visibilities(J_true_t[a, t], C[:, t:t + 1], pq) for t in range(Ta)], axis=1)
        if sky_bg is not None:  # uncorrupted: c_bg I_2
            cb = simulate_coherencies(uvw[iv, :Ta], sky_bg, float(freqs[fi]), pq)[:, :, 0]
            V = V + cb[:, :, None, None] * np.eye(2)
        s_a = float(np.sum(np.abs(V[flags[a] == 0]) ** 2))
        C_out = C.astype(dtype, copy=False) if coherencies else None
        return C_out, V.astype(dtype, copy=False), s_a, int(np.sum(flags[a] == 0)) * Ta * 4

    workers = min(A, os.cpu_count() or 1) if A >= 64 else 1
    if workers > 1:
        with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
            per_agent = list(ex.map(agent, range(A)))
    else:
        per_agent = [agent(a) for a in range(A)]
    Cs = [r[0] for r in per_agent] if coherencies else None
    Vs = [r[1] for r in per_agent]
    sig, cnt = 0.0, 0
    for r in per_agent:  # summed in agent order: the same noise level however the agents ran
        sig += r[2]
        cnt += r[3]
    del per_agent
    # Noise: total noise power = total signal power / SNR over all unflagged data
    # (equal variance in real and imaginary parts, Section 2 and Section 4).
    sigma = math.sqrt(sig / cnt / (2.0 * spec.snr)) if (noise and cnt) else 0.0
    if sigma > 0:
        for a in range(A):
            shape = Vs[a].shape
            Vs[a] = Vs[a] + (sigma * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))).astype(dtype, copy=False)
    out = dict(spec=spec, N=N, K=K, P=P, I=I, M=spec.M, B=B, A=A, pq=pq, freqs=freqs, basis=basis,
               rho=rho, T=T_agent, flags=flags, uvw=uvw, sky=sky, f0=F0_HZ, J_true=J_true,
               V=Vs, C=Cs, sigma=sigma, n_admm=spec.n_admm)
    if J_true_t is not None:
        out["J_true_t"] = J_true_t  # [A,Tmax,K,N,2,2]; J_true is its mean over each agent's samples
    if sky_bg is not None:
        out["sky_bg"] = sky_bg
    return out


def agent_slices(T: np.ndarray, B: int) -> np.ndarray:
    """Start offsets (in visibilities) of each agent's [B,T_a] block in the packed layout."""
    off = np.zeros(len(T) + 1, dtype=np.int64)
    off[1:] = np.cumsum(B * np.asarray(T, dtype=np.int64))
    return off


def pack_uniform(arrs: list[np.ndarray], dtype=np.complex64) -> np.ndarray:
    """Concatenate per-agent blocks (agent-major) into one contiguous array."""
    return np.ascontiguousarray(np.concatenate([a.reshape(-1) for a in arrs]).astype(dtype))


def user_layout(prob: dict) -> dict:
    """The problem's arrays in the C-ABI input layout (complex64, agent-major packed):
    vis [A][B][T_a][2][2], coh [A][B][T_a][K], flags [A][B], plus T [A]."""
    vis = np.concatenate([V.reshape(-1) for V in prob["V"]]).astype(np.complex64)
    coh = np.concatenate([C.reshape(-1) for C in prob["C"]]).astype(np.complex64)
    return dict(vis=vis, coh=coh, flags=np.ascontiguousarray(prob["flags"]), T=prob["T"].astype(np.int32))
