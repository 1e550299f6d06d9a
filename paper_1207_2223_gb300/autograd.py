"""The pseudofermion action S_f = phi^dag (M^dag M)^{-1} phi as a torch.autograd.Function.

Forward solves M^dag M X = phi and reduces phi^dag X in the CUDA library;
backward recomputes X (it is not stored), then the library's adjoint
kernel returns dS_f / dU in torch's complex-gradient convention, and
dS_f / dphi = 2 X.  Every step runs in the library; this module only
passes tensors through the C interface.

Contexts are cached, one per (lattice extents, time boundary, device), so
a training or HMC loop allocates device memory on its first call only:
later calls reuse the context's fields and replay the CUDA graphs it
recorded for the same kappa.  The links are loaded into the context
(lq_gauge_set: one device-side pack, no allocation) on every forward and
backward call, so any change to the tensor, by any route, is seen.
``release_contexts()`` frees the device memory of the cached contexts.
"""
import atexit
import threading

import torch

from . import lq


class _CachedContext:
    def __init__(self, dims, t_antiperiodic):
        self.ctx = lq.lq_create(dims, t_antiperiodic)
        self.lock = threading.Lock()
        self.gauge_loads = 0         # links loaded so far (for tests and reports)

    def bind(self, U):
        """Issue work on the current stream of U's device and load the links U."""
        lq.lq_set_stream(self.ctx, torch.cuda.current_stream(U.device).cuda_stream)
        lq.lq_gauge_set(self.ctx, U)
        self.gauge_loads += 1


_CACHE = {}
_CACHE_LOCK = threading.Lock()


def _context(U, dims, t_antiperiodic):
    key = (tuple(int(d) for d in dims), bool(t_antiperiodic), U.device.index)
    with _CACHE_LOCK:
        c = _CACHE.get(key)
        if c is None:
            with torch.cuda.device(U.device):
                c = _CachedContext(dims, t_antiperiodic)
            _CACHE[key] = c
    return c


def release_contexts():
    """Destroy every cached context (frees their device memory)."""
    with _CACHE_LOCK:
        items = list(_CACHE.values())
        _CACHE.clear()
    for c in items:
        with c.lock:
            try:
                lq.lq_destroy(c.ctx)
            except lq.LQError:
                pass


def cached_context_stats():
    """{(dims, t_antiperiodic, device): number of link loads} of the cached contexts."""
    with _CACHE_LOCK:
        return {k: c.gauge_loads for k, c in _CACHE.items()}


atexit.register(release_contexts)


class PseudofermionAction(torch.autograd.Function):
    """S_f(U, phi) for U complex128 (V, 4, 3, 3) and phi complex128 (V, 4, 3) on the GPU."""

    @staticmethod
    def forward(fctx, U, phi, dims, kappa, tol, inner_prec, t_antiperiodic):
        U = U.contiguous()
        phi = phi.contiguous()
        c = _context(U, dims, t_antiperiodic)
        with c.lock:
            c.bind(U)
            S = lq.lq_pseudofermion_action(c.ctx, phi, kappa, tol, 100000, inner_prec)
        fctx.save_for_backward(U, phi)
        fctx.args = (dims, kappa, tol, inner_prec, t_antiperiodic)
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(fctx, gS):
        U, phi = fctx.saved_tensors
        dims, kappa, tol, inner_prec, t_antiperiodic = fctx.args
        c = _context(U, dims, t_antiperiodic)
        X = torch.empty_like(phi)
        G = torch.empty_like(U)
        with c.lock:
            c.bind(U)
            lq.lq_solve_MdagM(c.ctx, X, phi, kappa, tol, 100000, inner_prec, 50)
            lq.lq_fermion_grad(c.ctx, G, X, kappa)
        g = gS.to(torch.float64)
        gU = G * g if fctx.needs_input_grad[0] else None
        gphi = 2.0 * X * g if fctx.needs_input_grad[1] else None
        return gU, gphi, None, None, None, None, None


def pseudofermion_action(U, phi, dims, kappa, tol=1e-10, inner_prec=lq.LQ_F64, t_antiperiodic=True):
    """Differentiable S_f = phi^dag (M^dag M)^{-1} phi."""
    return PseudofermionAction.apply(U, phi, tuple(dims), float(kappa), float(tol), int(inner_prec),
                                     bool(t_antiperiodic))
