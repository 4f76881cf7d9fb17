"""A context object over the C ABI (include/calib.h); marshalling only."""
from __future__ import annotations

import numpy as np

from . import capi


class Calibrator:
    """One calibration problem shape: N stations, baselines pq, K directions, P frequencies,
    basis [P,M], rho [K], I solution intervals, samples per agent."""

    def __init__(self, N, pq, K, freqs_hz, basis, rho, *, n_intervals=1, samples=1, n_lm=10, n_cg=4,
                 chunk_diagonals=0, cuda_stream=None, formulation=capi.CALIB_FORM_STATISTICS, ctas_per_sm=0,
                 jupdate=capi.CALIB_JUPDATE_LM, n_sage=1, freq_groups=1):
        spa = None if np.isscalar(samples) else np.asarray(samples, dtype=np.int32)
        self.N, self.K, self.P = int(N), int(K), len(freqs_hz)
        self.M = int(np.asarray(basis).shape[1])
        self.I = int(n_intervals)
        self.A = self.I * self.P
        self.G = int(freq_groups)
        self.B = int(np.asarray(pq).shape[0])
        self.T = spa if spa is not None else np.full(self.A, int(samples), dtype=np.int32)
        self.ctx = capi.calib_init(N, pq, K, freqs_hz, basis, rho, n_intervals=n_intervals,
                                   n_samples=int(samples) if spa is None else 1, samples_per_agent=spa,
                                   n_lm=n_lm, n_cg=n_cg, chunk_diagonals=chunk_diagonals, cuda_stream=cuda_stream,
                                   formulation=formulation, ctas_per_sm=ctas_per_sm, jupdate=jupdate,
                                   n_sage=n_sage, freq_groups=freq_groups)

    # shapes of the public arrays
    @property
    def jones_shape(self):
        return (self.A, self.K, self.N, 2, 2)

    @property
    def z_shape(self):
        """Z per consensus problem (interval * G + frequency group), [I*G][K][M][N][2][2]."""
        return (self.I * self.G, self.K, self.M, self.N, 2, 2)

    def set_data(self, vis, coh=None, flags=None):
        capi.calib_set_data(self.ctx, vis, coh, flags)

    def predict(self, uvw_m, sky, f0_hz):
        capi.calib_predict(self.ctx, uvw_m, sky, f0_hz)

    def coherencies(self):
        out = np.zeros(int(self.B * self.T.sum() * self.K), dtype=np.complex64)
        return capi.calib_get_coherencies(self.ctx, out)

    def residual(self, subtract=None, correct=None):
        """V - the model of the subtracted directions (all by default), corrected by direction
        `correct`'s solutions if given; visibility layout [A][B][T_a][2][2] flattened."""
        if subtract is not None and np.asarray(subtract).shape != (self.K,):
            raise ValueError(f"subtract must have one entry per direction ({self.K})")
        out = np.zeros(int(self.B * self.T.sum() * 4), dtype=np.complex64)
        return capi.calib_residual(self.ctx, out, subtract, -1 if correct is None else int(correct))

    def reset(self):
        capi.calib_reset(self.ctx)

    def set_initial(self, J0):
        capi.calib_set_initial(self.ctx, J0)

    def set_consensus(self, Z=None, Y=None):
        capi.calib_set_consensus(self.ctx, Z, Y)

    def iterate(self, n, want_hist=True):
        return capi.calib_admm_iter(self.ctx, n, want_hist)

    def solutions(self):
        J = np.zeros(self.jones_shape, dtype=np.complex64)
        Z = np.zeros(self.z_shape, dtype=np.complex128)
        Y = np.zeros(self.jones_shape, dtype=np.complex64)
        capi.calib_get_solutions(self.ctx, J, Z, Y)
        return J, Z, Y

    def get_state(self) -> bytes:
        """Opaque checkpoint of the whole iteration state (calib_get_state)."""
        return capi.calib_get_state(self.ctx)

    def set_state(self, blob: bytes):
        capi.calib_set_state(self.ctx, blob)

    def agent_objective(self):
        return capi.calib_get_agent_objective(self.ctx, self.A)

    def eval(self, J):
        L = np.zeros(self.A)
        g = np.zeros(self.A)
        grad = np.zeros(self.jones_shape, dtype=np.complex64)
        capi.calib_eval(self.ctx, np.ascontiguousarray(J, dtype=np.complex64), L, g, grad)
        return L, g, grad

    def hessvec(self, J, eta):
        out = np.zeros(self.jones_shape, dtype=np.complex64)
        capi.calib_hessvec(self.ctx, np.ascontiguousarray(J, dtype=np.complex64),
                           np.ascontiguousarray(eta, dtype=np.complex64), out)
        return out

    def close(self):
        if self.ctx:
            capi.calib_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
