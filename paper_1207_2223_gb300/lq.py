"""ctypes binding of the C interface in include/lq.h (argument marshalling only).

Buffers may be torch tensors (CUDA or CPU) or numpy arrays; their data
pointers go straight to the library, which stages host buffers itself.
Complex fields use the canonical layouts of lq.h:
  gauge  complex128 (V, 4, 3, 3)   spinor complex128 (V, 4, 3)
  momentum / force float64 (V, 4, 8)
Every non-zero status raises LQError with the library's message.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblq.so")

LQ_OK, LQ_ERR_ARG, LQ_ERR_SHAPE, LQ_ERR_CUDA, LQ_ERR_NOT_CONVERGED, LQ_ERR_NAN, LQ_ERR_STATE, LQ_ERR_TIMEOUT = range(8)
LQ_F64, LQ_F32, LQ_F32_12, LQ_F16_12, LQ_BF16_12, LQ_DF64, LQ_I16_12 = range(7)
PRECISIONS = {"f64": LQ_F64, "f32": LQ_F32, "f32_12": LQ_F32_12, "f16_12": LQ_F16_12, "bf16_12": LQ_BF16_12,
              "df64": LQ_DF64, "i16_12": LQ_I16_12}


class LQError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("lq status %d: %s" % (status, msg))
        self.status = status


class lq_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("restarts", ctypes.c_int),
                ("converged", ctypes.c_int), ("true_rel_resid", ctypes.c_double), ("seconds", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("escalations", ctypes.c_int), ("stage_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("deliver_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lq_hmc_params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("kappa", ctypes.c_double), ("tau", ctypes.c_double),
                ("n_steps", ctypes.c_int), ("tol", ctypes.c_double), ("maxiter", ctypes.c_int),
                ("inner_prec", ctypes.c_int), ("reliable_every", ctypes.c_int)]


class lq_traj_result(ctypes.Structure):
    _fields_ = [("dH", ctypes.c_double), ("dK", ctypes.c_double), ("dSg", ctypes.c_double),
                ("dSf", ctypes.c_double), ("accepted", ctypes.c_int), ("plaquette", ctypes.c_double),
                ("solves", ctypes.c_int), ("cg_iterations", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("seconds", ctypes.c_double), ("seconds_solve", ctypes.c_double),
                ("seconds_gauge_force", ctypes.c_double), ("seconds_fermion_force", ctypes.c_double),
                ("seconds_link_update", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int

# name -> (restype, argtypes); the C declarations are in include/lq.h
SIGNATURES = {
    "lq_version": (ctypes.c_char_p, []),
    "lq_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_I), _I, _P]),
    "lq_destroy": (_I, [_P]),
    "lq_last_error": (ctypes.c_char_p, [_P]),
    "lq_set_stream": (_I, [_P, _P]),
    "lq_volume": (ctypes.c_int64, [_P]),
    "lq_set_option": (_I, [_P, _I, _I]),
    "lq_gauge_set": (_I, [_P, _P]),
    "lq_gauge_get": (_I, [_P, _P]),
    "lq_apply_M": (_I, [_P, _P, _P, _D, _I, _I]),
    "lq_apply_MdagM": (_I, [_P, _P, _P, _D, _I]),
    "lq_solve_MdagM": (_I, [_P, _P, _P, _D, _D, _I, _I, _I, _P, _I, ctypes.POINTER(lq_solve_stats)]),
    "lq_time_dslash": (_I, [_P, _P, _D, _I, _I, _I, _I, ctypes.POINTER(_D)]),
    "lq_apply_MdagM_static": (_I, [_P, _P, _P, ctypes.POINTER(_I), _I, _D, _P]),
    "lq_time_cg_kernel": (_I, [_P, _P, _D, _I, _I, _I, ctypes.POINTER(_D)]),
    "lq_solve_batch": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_D), _I,
                            _D, _I, _I, _I, _P, _I, _P, _P, ctypes.POINTER(lq_solve_stats)]),
    "lq_apply_M_naive": (_I, [_P, _P, _P, _D, _I, _I, ctypes.POINTER(_D)]),
    "lq_fermion_force_naive": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(_D)]),
    "lq_time_fermion_force": (_I, [_P, _P, _D, _I, ctypes.POINTER(_D)]),
    "lq_plaquette": (_I, [_P, ctypes.POINTER(_D)]),
    "lq_gauge_action": (_I, [_P, _D, ctypes.POINTER(_D)]),
    "lq_gauge_force": (_I, [_P, _P, _D]),
    "lq_fermion_force": (_I, [_P, _P, _P, _D]),
    "lq_link_update": (_I, [_P, _P, _D]),
    "lq_fermion_grad": (_I, [_P, _P, _P, _D]),
    "lq_pseudofermion_action": (_I, [_P, _P, _D, _D, _I, _I, _I, ctypes.POINTER(_D), _P]),
    "lq_hmc_trajectory": (_I, [_P, ctypes.POINTER(lq_hmc_params), _P, _P, _D, ctypes.POINTER(lq_traj_result)]),
    "lq_hmc_trajectory_seeded": (_I, [_P, ctypes.POINTER(lq_hmc_params), ctypes.c_uint64, ctypes.c_uint64, _P,
                                      ctypes.POINTER(lq_traj_result)]),
    "lq_heatbath_draw": (_I, [_P, ctypes.c_uint64, ctypes.c_uint64, _P, _P, ctypes.POINTER(_D)]),
    "lq_philox4x32_10": (_I, [_P, _P, _P, _I]),
    "lq_time_fma_peak": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "lq_batch_tuning": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), _P,
                            _I]),
}

_lib = None


def load(path=LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("CUDA library %s not built: run paper_1207_2223_gb300.build.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(buf):
    if buf is None:
        return None
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return buf.data_ptr()
    if hasattr(buf, "ctypes"):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be C-contiguous")
        return buf.ctypes.data
    return int(buf)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


def _check(ctx, status):
    if status != LQ_OK:
        msg = load().lq_last_error(ctx)
        raise LQError(status, msg.decode() if msg else "")


def lq_version():
    return load().lq_version().decode()


def lq_create(dims, t_antiperiodic=True, stream=None):
    lib = load()
    out = _P()
    d = (_I * 4)(*[int(v) for v in dims])
    st = _current_stream() if stream is None else stream
    _check(None, lib.lq_create(ctypes.byref(out), d, 1 if t_antiperiodic else 0, st))
    return out


def lq_destroy(ctx):
    _check(ctx, load().lq_destroy(ctx))


def lq_last_error(ctx):
    return load().lq_last_error(ctx).decode()


def lq_set_stream(ctx, stream):
    _check(ctx, load().lq_set_stream(ctx, stream))


LQ_OPT_CUDA_GRAPHS, LQ_OPT_DF64_UPDATES, LQ_OPT_PAIR_SITES, LQ_OPT_STAGED = 1, 2, 3, 4
LQ_OPT_BATCH_RHS_PER_THREAD, LQ_OPT_BATCH_PERSISTENT, LQ_OPT_BATCH_BARRIER_TEST = 5, 6, 7
LQ_OPT_BATCH_DEVICE_LOOP = 8
LQ_OPT_HOST_DIRECT = 9
LQ_OPT_BATCH_TILE_ORDER = 10
LQ_OPT_DF64_PREFETCH = 11


def lq_set_option(ctx, option, value):
    _check(ctx, load().lq_set_option(ctx, int(option), int(value)))


def lq_volume(ctx):
    return int(load().lq_volume(ctx))


def lq_gauge_set(ctx, U):
    _check(ctx, load().lq_gauge_set(ctx, _ptr(U)))


def lq_gauge_get(ctx, U):
    _check(ctx, load().lq_gauge_get(ctx, _ptr(U)))


def lq_apply_M(ctx, out, inp, kappa, dagger=False, prec=LQ_F64):
    _check(ctx, load().lq_apply_M(ctx, _ptr(out), _ptr(inp), float(kappa), 1 if dagger else 0, int(prec)))


def lq_apply_MdagM(ctx, out, inp, kappa, prec=LQ_F64):
    _check(ctx, load().lq_apply_MdagM(ctx, _ptr(out), _ptr(inp), float(kappa), int(prec)))


def lq_solve_MdagM(ctx, x, phi, kappa, tol=1e-10, maxiter=100000, inner_prec=LQ_F64, reliable_every=50,
                   hist=None, raise_on_error=True):
    """Returns (status, stats dict); raises on errors other than NOT_CONVERGED unless told not to."""
    st = lq_solve_stats()
    n = 0 if hist is None else len(hist)
    status = load().lq_solve_MdagM(ctx, _ptr(x), _ptr(phi), float(kappa), float(tol), int(maxiter),
                                   int(inner_prec), int(reliable_every), _ptr(hist), n, ctypes.byref(st))
    if raise_on_error and status not in (LQ_OK, LQ_ERR_NOT_CONVERGED):
        _check(ctx, status)
    return status, st.as_dict()


def lq_time_dslash(ctx, inp, kappa, dagger=False, prec=LQ_F64, n=20, flush_l2=False):
    """Average device milliseconds of one application of M (or M^dag)."""
    ms = _D()
    _check(ctx, load().lq_time_dslash(ctx, _ptr(inp), float(kappa), 1 if dagger else 0, int(prec), int(n),
                                      1 if flush_l2 else 0, ctypes.byref(ms)))
    return ms.value


def lq_time_cg_kernel(ctx, inp, kappa, which=0, prec=LQ_F64, n=20):
    """Average device milliseconds of a CG iteration (which=0) or one of its passes (1, 2, 3)."""
    ms = _D()
    _check(ctx, load().lq_time_cg_kernel(ctx, _ptr(inp), float(kappa), int(which), int(prec), int(n),
                                         ctypes.byref(ms)))
    return ms.value


def lq_solve_batch(ctxs, xs, phis, kappas, nrhs=1, tol=1e-10, maxiter=100000, inner_prec=LQ_F32_12,
                   reliable_every=50, hist_len=0):
    """Solve n systems together.  Returns (status, stats, iters[n*nrhs], resid[n*nrhs], hist or None)."""
    import numpy as np
    n = len(ctxs)
    c_arr = (_P * n)(*[c.value if hasattr(c, "value") else c for c in ctxs])
    x_arr = (_P * n)(*[_ptr(x) for x in xs])
    p_arr = (_P * n)(*[_ptr(p) for p in phis])
    k_arr = (_D * n)(*[float(k) for k in kappas])
    iters = np.zeros(n * nrhs, dtype=np.int32)
    resid = np.zeros(n * nrhs)
    hist = np.zeros((n * nrhs, hist_len)) if hist_len > 0 else None
    st = lq_solve_stats()
    status = load().lq_solve_batch(c_arr, n, x_arr, p_arr, k_arr, int(nrhs), float(tol), int(maxiter),
                                   int(inner_prec), int(reliable_every), _ptr(hist), int(hist_len),
                                   iters.ctypes.data, resid.ctypes.data, ctypes.byref(st))
    if status not in (LQ_OK, LQ_ERR_NOT_CONVERGED):
        _check(ctxs[0], status)
    return status, st.as_dict(), iters, resid, hist


def lq_batch_tuning(ctx):
    """The autotuner's choice for the last batched solve on ctx: dict with tile (threads per
    block), rhs_per_thread, blocks_per_sm (0: all that fit), site_major (tile order) and the
    per-candidate ms."""
    import numpy as np
    t, rb, bps, sm = _I(), _I(), _I(), _I()
    ms = np.full(64, np.nan)
    _check(ctx, load().lq_batch_tuning(ctx, ctypes.byref(t), ctypes.byref(rb), ctypes.byref(bps), ctypes.byref(sm),
                                       ms.ctypes.data, 64))
    return {"tile": t.value, "rhs_per_thread": rb.value, "blocks_per_sm": bps.value, "site_major": sm.value,
            "candidate_ms": [float(v) for v in ms if v == v]}


def lq_apply_M_naive(ctx, out, inp, kappa, dagger=False, n=0):
    """Naive-kernel M (ablation); with n > 0 returns its average device ms over n launches."""
    ms = _D(0.0)
    _check(ctx, load().lq_apply_M_naive(ctx, _ptr(out), _ptr(inp), float(kappa), 1 if dagger else 0, int(n),
                                        ctypes.byref(ms)))
    return ms.value


def lq_fermion_force_naive(ctx, F, X, kappa, n=0):
    """Naive-kernel fermion force (ablation) into F (device, (V, 4, 8)); with n > 0 returns
    the force kernel's average device ms over n launches."""
    ms = _D(0.0)
    _check(ctx, load().lq_fermion_force_naive(ctx, _ptr(F), _ptr(X), float(kappa), int(n), ctypes.byref(ms)))
    return ms.value


def lq_time_fermion_force(ctx, X, kappa, n=20):
    """Average device ms of the optimised fermion-force kernel (Y = M X formed beforehand)."""
    ms = _D()
    _check(ctx, load().lq_time_fermion_force(ctx, _ptr(X), float(kappa), int(n), ctypes.byref(ms)))
    return ms.value


def lq_time_fma_peak(ctx, prec=LQ_F64):
    """Measured fused multiply-add rate of the GPU (TFLOP/s) in FP64 or FP32."""
    v = _D()
    _check(ctx, load().lq_time_fma_peak(ctx, int(prec), ctypes.byref(v)))
    return v.value


def lq_plaquette(ctx):
    v = _D()
    _check(ctx, load().lq_plaquette(ctx, ctypes.byref(v)))
    return v.value


def lq_gauge_action(ctx, beta):
    v = _D()
    _check(ctx, load().lq_gauge_action(ctx, float(beta), ctypes.byref(v)))
    return v.value


def lq_gauge_force(ctx, F, beta):
    _check(ctx, load().lq_gauge_force(ctx, _ptr(F), float(beta)))


def lq_fermion_force(ctx, F, X, kappa):
    _check(ctx, load().lq_fermion_force(ctx, _ptr(F), _ptr(X), float(kappa)))


def lq_fermion_grad(ctx, G, X, kappa):
    _check(ctx, load().lq_fermion_grad(ctx, _ptr(G), _ptr(X), float(kappa)))


def lq_pseudofermion_action(ctx, phi, kappa, tol=1e-10, maxiter=100000, inner_prec=LQ_F64, reliable_every=50,
                            X=None):
    v = _D()
    _check(ctx, load().lq_pseudofermion_action(ctx, _ptr(phi), float(kappa), float(tol), int(maxiter),
                                               int(inner_prec), int(reliable_every), ctypes.byref(v), _ptr(X)))
    return v.value


def lq_link_update(ctx, p, eps):
    _check(ctx, load().lq_link_update(ctx, _ptr(p), float(eps)))


def lq_hmc_trajectory(ctx, p, chi, u, beta, kappa, n_steps, tau=1.0, tol=1e-10, maxiter=100000,
                      inner_prec=LQ_F64, reliable_every=50):
    """One trajectory; p is updated in place.  Returns the result as a dict."""
    hp = lq_hmc_params(float(beta), float(kappa), float(tau), int(n_steps), float(tol), int(maxiter),
                       int(inner_prec), int(reliable_every))
    res = lq_traj_result()
    _check(ctx, load().lq_hmc_trajectory(ctx, ctypes.byref(hp), _ptr(p), _ptr(chi), float(u), ctypes.byref(res)))
    return res.as_dict()


def lq_hmc_trajectory_seeded(ctx, seed, traj_index, beta, kappa, n_steps, tau=1.0, tol=1e-10, maxiter=100000,
                             inner_prec=LQ_F64, reliable_every=50, p_out=None):
    """One trajectory with the heat bath (momenta, chi, Metropolis uniform) drawn on the
    device from (seed, traj_index).  Returns the result as a dict."""
    hp = lq_hmc_params(float(beta), float(kappa), float(tau), int(n_steps), float(tol), int(maxiter),
                       int(inner_prec), int(reliable_every))
    res = lq_traj_result()
    _check(ctx, load().lq_hmc_trajectory_seeded(ctx, ctypes.byref(hp), int(seed), int(traj_index), _ptr(p_out),
                                                ctypes.byref(res)))
    return res.as_dict()


def lq_heatbath_draw(ctx, seed, traj_index, p=None, chi=None):
    """The device heat-bath draws of (seed, traj_index) into p (V, 4, 8) and chi (V, 4, 3)
    (either may be None); returns the Metropolis uniform."""
    u = _D()
    _check(ctx, load().lq_heatbath_draw(ctx, int(seed), int(traj_index), _ptr(p), _ptr(chi), ctypes.byref(u)))
    return u.value


def lq_philox4x32_10(ctx, inp, out):
    """Philox4x32-10 words on the device: inp int32/uint32 (n, 6) counters and keys, out (n, 4)."""
    _check(ctx, load().lq_philox4x32_10(ctx, _ptr(inp), _ptr(out), int(inp.shape[0])))


def lq_apply_MdagM_static(out, U, inp, dims, kappa, t_antiperiodic=True, stream=None):
    """out = M^dag M inp on caller device buffers, with no device allocation.

    For callers that cannot let the library allocate GPU memory (all memory
    owned by their own pool, or a fixed budget); at most 65,536 sites.
    Asynchronous on `stream` (the current torch stream by default).

    The C side cannot see buffer sizes, so they are checked here: out, U and
    inp must be CUDA tensors of dtype complex128 (or float64 holding twice as
    many reals) with 12 V (spinors) and 36 V (links) complex entries for
    V = prod(dims); anything else raises ValueError before the call."""
    V = 1
    for v in dims:
        V *= int(v)
    for name, buf, n in (("out", out, 12 * V), ("U", U, 36 * V), ("inp", inp, 12 * V)):
        if not (hasattr(buf, "is_cuda") and buf.is_cuda):
            raise ValueError("%s must be a CUDA tensor" % name)
        dt = str(buf.dtype)
        if dt.endswith("complex128"):
            count = buf.numel()
        elif dt.endswith("float64"):
            if buf.numel() % 2:
                raise ValueError("%s: odd number of float64 entries" % name)
            count = buf.numel() // 2
        else:
            raise ValueError("%s must be complex128 (or float64), not %s" % (name, dt))
        if count != n:
            raise ValueError("%s holds %d complex entries; the %s lattice needs %d" % (name, count, tuple(dims), n))
    d = (_I * 4)(*[int(v) for v in dims])
    st = _current_stream() if stream is None else stream
    _check(None, load().lq_apply_MdagM_static(_ptr(out), _ptr(U), _ptr(inp), d, 1 if t_antiperiodic else 0,
                                              float(kappa), st))


__all__ = [n for n in list(globals()) if n.startswith(("lq_", "LQ_"))] + ["LQError", "PRECISIONS", "load"]
