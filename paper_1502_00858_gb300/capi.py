"""Python binding of libcalib.so (include/calib.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. Functions carry the C names; arrays
may be NumPy arrays (host, ptr_kind 0) or CUDA torch tensors (device, ptr_kind 1). The
loader raises if the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcalib.so")

CALIB_FORM_STATISTICS, CALIB_FORM_DIRECT = 0, 1
CALIB_JUPDATE_LM, CALIB_JUPDATE_RTR, CALIB_JUPDATE_SAGE = 0, 1, 2
CALIB_OK, CALIB_EINVAL, CALIB_ERANK, CALIB_ENOMEM, CALIB_ECUDA, CALIB_ETIMEOUT, CALIB_ENUMERIC, CALIB_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7

EXPORTED = [
    "calib_default_options", "calib_init", "calib_set_data", "calib_predict", "calib_get_coherencies",
    "calib_reset", "calib_set_initial", "calib_set_consensus", "calib_admm_iter", "calib_get_solutions",
    "calib_get_agent_objective", "calib_eval", "calib_hessvec", "calib_sync", "calib_profile_enable",
    "calib_profile_read", "calib_launch_count", "calib_last_error", "calib_destroy", "calib_eval_noalloc",
    "calib_autotune", "calib_mlp_create", "calib_mlp_num_params", "calib_mlp_set_weights", "calib_mlp_get_weights",
    "calib_mlp_forward", "calib_mlp_grad", "calib_mlp_train_step", "calib_mlp_destroy", "calib_get_features",
    "calib_warm_start", "calib_selftest_bounded_wait", "calib_residual", "calib_get_state", "calib_set_state",
]


class CalibOptions(C.Structure):
    _fields_ = [("n_intervals", C.c_int), ("n_samples", C.c_int), ("samples_per_agent", C.POINTER(C.c_int32)),
                ("n_lm", C.c_int), ("n_cg", C.c_int), ("chunk_diagonals", C.c_int), ("cuda_stream", C.c_void_p),
                ("formulation", C.c_int), ("ctas_per_sm", C.c_int), ("jupdate", C.c_int), ("n_sage", C.c_int),
                ("freq_groups", C.c_int)]


class CalibStats(C.Structure):
    _fields_ = [("primal", C.c_double), ("dual", C.c_double), ("objective", C.c_double), ("resid_norm", C.c_double)]


class CalibError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"calib error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libcalib.so and declare the signatures. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1502_00858_gb300.build.build() "
                           "(the CUDA path has no CPU fallback)")
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    sig = {
        "calib_default_options": (None, [C.POINTER(CalibOptions)]),
        "calib_init": (i, [C.POINTER(vp), i, i, vp, i, i, vp, i, vp, vp, C.POINTER(CalibOptions)]),
        "calib_set_data": (i, [vp, vp, vp, vp, i]),
        "calib_predict": (i, [vp, vp, vp, i, d, i]),
        "calib_get_coherencies": (i, [vp, vp, i]),
        "calib_reset": (i, [vp]),
        "calib_set_initial": (i, [vp, vp, i]),
        "calib_set_consensus": (i, [vp, vp, vp, i]),
        "calib_admm_iter": (i, [vp, i, vp]),
        "calib_get_solutions": (i, [vp, vp, vp, vp, i]),
        "calib_get_agent_objective": (i, [vp, vp, vp]),
        "calib_eval": (i, [vp, vp, vp, vp, vp, i]),
        "calib_hessvec": (i, [vp, vp, vp, vp, i]),
        "calib_sync": (i, [vp]),
        "calib_profile_enable": (i, [vp, i]),
        "calib_profile_read": (i, [vp, i, vp, vp, vp, vp, vp]),
        "calib_launch_count": (C.c_longlong, [vp]),
        "calib_last_error": (C.c_char_p, []),
        "calib_destroy": (None, [vp]),
        "calib_eval_noalloc": (i, [i, i, i, i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "calib_autotune": (i, [vp, vp, vp, i, vp, vp, vp, vp]),
        "calib_mlp_create": (i, [C.POINTER(vp), i, i, i, i, vp]),
        "calib_mlp_num_params": (C.c_longlong, [vp]),
        "calib_mlp_set_weights": (i, [vp, vp, i]),
        "calib_mlp_get_weights": (i, [vp, vp, i]),
        "calib_mlp_forward": (i, [vp, vp, vp, i, i]),
        "calib_mlp_grad": (i, [vp, vp, vp, i, vp, vp, i]),
        "calib_mlp_train_step": (i, [vp, vp, vp, i, C.c_float, C.c_float, vp, i]),
        "calib_mlp_destroy": (None, [vp]),
        "calib_get_features": (i, [vp, vp, i]),
        "calib_warm_start": (i, [vp, vp, vp, vp, vp, i]),
        "calib_selftest_bounded_wait": (i, [i, vp, vp]),
        "calib_residual": (i, [vp, vp, i, vp, i]),
        "calib_get_state": (i, [vp, vp, C.POINTER(C.c_size_t)]),
        "calib_set_state": (i, [vp, vp, C.c_size_t]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int) -> None:
    if rc != CALIB_OK:
        raise CalibError(rc, load().calib_last_error().decode())


def _ptr(x, dtype=None):
    """(address, ptr_kind, keepalive) for a NumPy array or a torch tensor; None -> NULL."""
    if x is None:
        return None, 0, None
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (1 if x.is_cuda else 0), x
    arr = np.ascontiguousarray(x, dtype=dtype) if dtype is not None else np.ascontiguousarray(x)
    return arr.ctypes.data, 0, arr


def _kind(*ks) -> int:
    ks = [k for k in ks if k is not None]
    if not ks:
        return 0
    if len(set(ks)) != 1:
        raise ValueError("mix of host and device arrays in one call")
    return ks[0]


# ----------------------------------------------------------------------------- C names

def calib_default_options() -> CalibOptions:
    opt = CalibOptions()
    load().calib_default_options(C.byref(opt))
    return opt


def calib_init(N, pq, K, freqs_hz, basis, rho, *, n_intervals=1, n_samples=1, samples_per_agent=None,
               n_lm=10, n_cg=4, chunk_diagonals=0, cuda_stream=None, formulation=CALIB_FORM_STATISTICS,
               ctas_per_sm=0, jupdate=CALIB_JUPDATE_LM, n_sage=1, freq_groups=1):
    lib = load()
    pq_a = np.ascontiguousarray(pq, dtype=np.int32)
    fr = np.ascontiguousarray(freqs_hz, dtype=np.float64)
    ba = np.ascontiguousarray(basis, dtype=np.float64)
    rh = np.ascontiguousarray(rho, dtype=np.float64)
    opt = calib_default_options()
    opt.n_intervals, opt.n_samples, opt.n_lm, opt.n_cg = n_intervals, n_samples, n_lm, n_cg
    opt.chunk_diagonals = chunk_diagonals
    opt.formulation = formulation
    opt.ctas_per_sm = ctas_per_sm
    opt.jupdate = jupdate
    opt.n_sage = n_sage
    opt.freq_groups = freq_groups
    spa = None
    if samples_per_agent is not None:
        spa = np.ascontiguousarray(samples_per_agent, dtype=np.int32)
        opt.samples_per_agent = spa.ctypes.data_as(C.POINTER(C.c_int32))
    opt.cuda_stream = cuda_stream
    h = C.c_void_p()
    _check(lib.calib_init(C.byref(h), int(N), int(pq_a.shape[0]), pq_a.ctypes.data, int(K), int(fr.shape[0]),
                          fr.ctypes.data, int(ba.shape[1]), ba.ctypes.data, rh.ctypes.data, C.byref(opt)))
    del spa
    return h


def calib_set_data(ctx, vis, coh=None, flags=None):
    pv, kv, a = _ptr(vis, np.complex64)
    pc, kc, b = _ptr(coh, np.complex64)
    pf, kf, c = _ptr(flags, np.uint8)
    _check(load().calib_set_data(ctx, pv, pc, pf, _kind(kv, kc if coh is not None else None,
                                                        kf if flags is not None else None)))


def calib_predict(ctx, uvw_m, sky, f0_hz):
    pu, ku, a = _ptr(uvw_m, np.float64)
    ps, ks, b = _ptr(sky, np.float64)
    n_src = int(sky.shape[1])
    _check(load().calib_predict(ctx, pu, ps, n_src, float(f0_hz), _kind(ku, ks)))


def calib_get_coherencies(ctx, out):
    p, k, _ = _ptr(out)
    _check(load().calib_get_coherencies(ctx, p, k))
    return out


def calib_residual(ctx, out, subtract=None, correct: int = -1):
    """Residual (optionally corrected) visibilities into out (user visibility layout)."""
    sub = None if subtract is None else np.ascontiguousarray(np.asarray(subtract).astype(np.int32))
    sp = None if sub is None else sub.ctypes.data
    p, k, _ = _ptr(out)
    _check(load().calib_residual(ctx, sp, int(correct), p, k))
    return out


def calib_get_state(ctx) -> bytes:
    """The context's opaque iteration-state blob (host bytes)."""
    n = C.c_size_t(0)
    _check(load().calib_get_state(ctx, None, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(load().calib_get_state(ctx, buf, C.byref(n)))
    return buf.raw[:n.value]


def calib_set_state(ctx, blob: bytes) -> None:
    buf = C.create_string_buffer(bytes(blob), len(blob))
    _check(load().calib_set_state(ctx, buf, len(blob)))


def calib_reset(ctx):
    _check(load().calib_reset(ctx))


def calib_set_initial(ctx, J0):
    p, k, a = _ptr(J0, np.complex64)
    _check(load().calib_set_initial(ctx, p, k))


def calib_set_consensus(ctx, Z=None, Y=None):
    pz, kz, a = _ptr(Z, np.complex128)
    py, ky, b = _ptr(Y, np.complex64)
    _check(load().calib_set_consensus(ctx, pz, py, _kind(kz if Z is not None else None, ky if Y is not None else None)))


def calib_admm_iter(ctx, n_iters: int, want_hist: bool = True):
    hist = (CalibStats * n_iters)() if want_hist else None
    _check(load().calib_admm_iter(ctx, int(n_iters), C.cast(hist, C.c_void_p) if hist is not None else None))
    if hist is None:
        return None
    return {k: np.array([getattr(h, k) for h in hist]) for k in ("primal", "dual", "objective", "resid_norm")}


def calib_get_solutions(ctx, J=None, Z=None, Y=None):
    pj, kj, _ = _ptr(J)
    pz, kz, _ = _ptr(Z)
    py, ky, _ = _ptr(Y)
    k = _kind(kj if J is not None else None, kz if Z is not None else None, ky if Y is not None else None)
    _check(load().calib_get_solutions(ctx, pj, pz, py, k))


def calib_get_agent_objective(ctx, A: int):
    L = np.zeros(A)
    g = np.zeros(A)
    _check(load().calib_get_agent_objective(ctx, L.ctypes.data, g.ctypes.data))
    return L, g


def calib_eval(ctx, J, L=None, g=None, grad=None):
    pj, kj, a = _ptr(J, np.complex64)
    pl, _, _ = _ptr(L)
    pg, _, _ = _ptr(g)
    pgr, _, _ = _ptr(grad)
    _check(load().calib_eval(ctx, pj, pl, pg, pgr, kj))


def calib_hessvec(ctx, J, eta, out):
    pj, kj, a = _ptr(J, np.complex64)
    pe, ke, b = _ptr(eta, np.complex64)
    po, ko, _ = _ptr(out)
    _check(load().calib_hessvec(ctx, pj, pe, po, _kind(kj, ke, ko)))


def calib_sync(ctx):
    _check(load().calib_sync(ctx))


def calib_profile_enable(ctx, on: bool):
    _check(load().calib_profile_enable(ctx, int(bool(on))))


def calib_profile_read(ctx):
    cap = 16
    names = (C.c_char_p * cap)()
    ms = np.zeros(cap)
    n = np.zeros(cap, dtype=np.int64)
    by = np.zeros(cap)
    fl = np.zeros(cap)
    cnt = load().calib_profile_read(ctx, cap, C.cast(names, C.c_void_p), ms.ctypes.data, n.ctypes.data,
                                    by.ctypes.data, fl.ctypes.data)
    return {names[i].decode(): dict(total_ms=float(ms[i]), launches=int(n[i]), bytes_per_launch=float(by[i]),
                                    flops_per_launch=float(fl[i]))
            for i in range(cnt)}


def calib_launch_count(ctx) -> int:
    return int(load().calib_launch_count(ctx))


def calib_selftest_bounded_wait(complete_phase: bool, stream: int = 0) -> float:
    """Runs the bounded-wait self-test; returns the kernel's duration in ms, raises CalibError
    (code CALIB_ETIMEOUT) when the wait gave up."""
    ms = C.c_double(0.0)
    _check(load().calib_selftest_bounded_wait(int(bool(complete_phase)), C.byref(ms), C.c_void_p(stream)))
    return ms.value


def calib_destroy(ctx):
    if ctx:
        load().calib_destroy(ctx)


def calib_eval_noalloc(n_agents, n_stations, n_baselines, n_dirs, n_samples, pq, vis, coh, J, Y, BZ, rho,
                       L, g, grad, cuda_stream=None):
    """Device tensors in, device tensors out; rho is a host array. Allocates nothing."""
    rh = np.ascontiguousarray(rho, dtype=np.float64)
    ptrs = [_ptr(x)[0] for x in (pq, vis, coh, J, Y, BZ)]
    _check(load().calib_eval_noalloc(int(n_agents), int(n_stations), int(n_baselines), int(n_dirs),
                                     int(n_samples), *ptrs, rh.ctypes.data, _ptr(L)[0], _ptr(g)[0],
                                     _ptr(grad)[0], cuda_stream))


def calib_autotune(ctx):
    """Re-measure the sweep split. Returns (split of the Hessian pass, split of the trial pass,
    {candidate: (ms of n_cg Hessian passes with PCG steps, ms of the trial pass with its reduction)}).
    The split is CTAs per SM (statistics form) or diagonals per CTA (direct form, one value)."""
    cap = 64
    chosen, chosen_tr = C.c_int(), C.c_int()
    cand = np.zeros(cap, dtype=np.int32)
    ms_hv, ms_tr = np.zeros(cap), np.zeros(cap)
    n = C.c_int()
    _check(load().calib_autotune(ctx, C.byref(chosen), C.byref(chosen_tr), cap, cand.ctypes.data, ms_hv.ctypes.data,
                                 ms_tr.ctypes.data, C.byref(n)))
    return chosen.value, chosen_tr.value, {int(cand[i]): (float(ms_hv[i]), float(ms_tr[i])) for i in range(n.value)}


# ----------------------------------------------------------------------------- warm-start network

def calib_mlp_create(width=256, depth=3, cuda_stream=None):
    h = C.c_void_p()
    _check(load().calib_mlp_create(C.byref(h), 17, int(width), int(depth), 8, cuda_stream))
    return h


def calib_mlp_num_params(h) -> int:
    return int(load().calib_mlp_num_params(h))


def calib_mlp_set_weights(h, w):
    p, k, keep = _ptr(w, np.float32)
    _check(load().calib_mlp_set_weights(h, p, k))


def calib_mlp_get_weights(h, out=None):
    if out is None:
        out = np.zeros(calib_mlp_num_params(h), dtype=np.float32)
    p, k, _ = _ptr(out)
    _check(load().calib_mlp_get_weights(h, p, k))
    return out


def calib_mlp_forward(h, X, Y):
    px, kx, a = _ptr(X, np.float32)
    py, ky, _ = _ptr(Y)
    _check(load().calib_mlp_forward(h, px, py, int(X.shape[0]), _kind(kx, ky)))
    return Y


def calib_mlp_grad(h, X, T, grad=None, loss=None):
    px, kx, a = _ptr(X, np.float32)
    pt, kt, b = _ptr(T, np.float32)
    pg, _, _ = _ptr(grad)
    pl, _, _ = _ptr(loss)
    _check(load().calib_mlp_grad(h, px, pt, int(X.shape[0]), pg, pl, _kind(kx, kt)))


def calib_mlp_train_step(h, X, T, lr, weight_decay, loss=None):
    px, kx, a = _ptr(X, np.float32)
    pt, kt, b = _ptr(T, np.float32)
    pl, _, _ = _ptr(loss)
    _check(load().calib_mlp_train_step(h, px, pt, int(X.shape[0]), C.c_float(lr), C.c_float(weight_decay), pl,
                                       _kind(kx, kt)))


def calib_mlp_destroy(h):
    if h:
        load().calib_mlp_destroy(h)


def calib_get_features(ctx, X):
    p, k, _ = _ptr(X)
    _check(load().calib_get_features(ctx, p, k))
    return X


def calib_warm_start(ctx, mlp, J_prev, Z_prev, chose=None):
    pj, kj, a = _ptr(J_prev, np.complex64)
    pz, kz, b = _ptr(Z_prev, np.complex128)
    pc, _, _ = _ptr(chose)
    _check(load().calib_warm_start(ctx, mlp, pj, pz, pc, _kind(kj, kz)))
