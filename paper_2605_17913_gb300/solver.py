"""PyTorch-facing API: batched solves, gradients and a torch.autograd.Function.

Tensors must be float32, contiguous and on the CUDA device current when the
solver is created (``solve_backward_host``: in host memory).  PyTorch only
allocates memory and supplies the stream; the arithmetic is in libqpgpu's
kernels.
"""
from __future__ import annotations

import ctypes
from typing import Dict, Optional

import numpy as np
import torch

from . import _lib
from ._lib import QPError, check, default_settings, ptr


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class QPSolver:
    """Handle for batches of ``batch`` QPs with ``n`` variables, ``n_eq``
    equality rows and ``n_ineq`` inequality rows (eq. 1).  ``threads_per_qp``:
    0 chooses by size and batch; 32 (one warp per QP, n <= 32) or 128 force
    a width (qp_handle_create_threads)."""

    def __init__(self, batch: int, n: int, n_eq: int, n_ineq: int, threads_per_qp: int = 0):
        self.batch, self.n, self.n_eq, self.n_ineq = int(batch), int(n), int(n_eq), int(n_ineq)
        self._dims = _lib.Dims(self.batch, self.n, self.n_eq, self.n_ineq)
        h = ctypes.c_void_p()
        check(_lib.lib().qp_handle_create_threads(ctypes.byref(self._dims), int(threads_per_qp),
                                                  ctypes.byref(h)), "qp_handle_create_threads")
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().qp_handle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        """The launch configuration this handle chose (qp_handle_query)."""
        out = _lib.HandleInfo()
        check(_lib.lib().qp_handle_query(self._h, ctypes.byref(out)), "qp_handle_query")
        return {k: getattr(out, k) for k, _ in _lib.HandleInfo._fields_}

    def set_diag(self, diag: Optional[torch.Tensor]) -> None:
        """Register an int32 CUDA tensor of shape [batch] that later solves and
        backward passes through this handle fill with per-instance
        diagnostics words (qp_handle_set_diag); None turns them off."""
        if diag is not None:
            if diag.dtype != torch.int32 or not diag.is_cuda or not diag.is_contiguous() \
                    or tuple(diag.shape) != (self.batch,):
                raise QPError(f"diag must be a contiguous int32 CUDA tensor of shape ({self.batch},)")
        self._diag = diag  # keep it alive while registered
        check(_lib.lib().qp_handle_set_diag(self._h, ptr(diag) if diag is not None else None),
              "qp_handle_set_diag")

    @property
    def grad_cache_bytes(self) -> int:
        return int(_lib.lib().qp_grad_cache_bytes(ctypes.byref(self._dims)))

    def new_grad_cache(self) -> torch.Tensor:
        nfl = max(4, self.grad_cache_bytes // 4)
        return torch.empty(nfl, dtype=torch.float32, device=self.device)

    def _check(self, name, t, shape):
        if t is None:
            if int(torch.tensor(shape).prod()) == 0:
                return None
            raise QPError(f"{name} is required")
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise QPError(f"{name} must be a contiguous float32 CUDA tensor")
        if tuple(t.shape) != tuple(shape):
            raise QPError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
        return t

    def _host(self, name, t, shape):
        if t is None:
            if int(torch.tensor(shape).prod()) == 0:
                return None
            raise QPError(f"{name} is required")
        if not isinstance(t, torch.Tensor):
            t = torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32))
        if t.dtype != torch.float32 or t.is_cuda or not t.is_contiguous():
            raise QPError(f"{name} must be a contiguous float32 host tensor or array")
        if tuple(t.shape) != tuple(shape):
            raise QPError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
        return t

    def solve_backward_host(self, Q, q, A, b, G, h, dl_dx=None,
                            settings: Optional[_lib.Settings] = None, out: Optional[Dict] = None,
                            **overrides) -> Dict[str, torch.Tensor]:
        """Solve, relax and backward pass of a batch in host memory in one
        call (qp_solve_backward_host): the library moves chunks of the batch
        to the device and back on two streams, overlapping the copies with
        the kernels when the host tensors are page-locked (``pin_memory()``).
        Without ``dl_dx``: the solve only.  Returns host tensors (``out``,
        if given, is filled instead)."""
        B, n, p, m = self.batch, self.n, self.n_eq, self.n_ineq
        Q = self._host("Q", Q, (B, n, n))
        q = self._host("q", q, (B, n))
        A = self._host("A", A, (B, p, n))
        b = self._host("b", b, (B, p))
        G = self._host("G", G, (B, m, n))
        h = self._host("h", h, (B, m))
        g = self._host("dl_dx", dl_dx, (B, n)) if dl_dx is not None else None
        st = settings if settings is not None else default_settings(**overrides)
        if out is None:
            out = dict(x=torch.empty(B, n), y=torch.empty(B, p), z=torch.empty(B, m),
                       s=torch.empty(B, m), status=torch.empty(B, dtype=torch.int32),
                       iters=torch.empty(B, dtype=torch.int32), kkt=torch.empty(B))
            if g is not None:
                out.update(dQ=torch.empty(B, n, n), dq=torch.empty(B, n), dA=torch.empty(B, p, n),
                           db=torch.empty(B, p), dG=torch.empty(B, m, n), dh=torch.empty(B, m))
        o = lambda k: ptr(out.get(k))  # noqa: E731
        rc = _lib.lib().qp_solve_backward_host(
            self._h, ctypes.byref(st), ptr(Q), ptr(q), ptr(A), ptr(b), ptr(G), ptr(h), ptr(g),
            o("x"), o("y"), o("z"), o("s"), o("status"), o("iters"), o("kkt"), o("dQ"), o("dq"),
            o("dA"), o("db"), o("dG"), o("dh"))
        check(rc, "qp_solve_backward_host")
        return out

    def solve(self, Q, q, A, b, G, h, settings: Optional[_lib.Settings] = None,
              grad_cache: Optional[torch.Tensor] = None, out: Optional[Dict] = None,
              stream: Optional[torch.cuda.Stream] = None, **overrides) -> Dict[str, torch.Tensor]:
        """Alg. 1 (and Alg. 2 + factor caching when ``grad_cache`` is given)."""
        B, n, p, m = self.batch, self.n, self.n_eq, self.n_ineq
        Q = self._check("Q", Q, (B, n, n))
        q = self._check("q", q, (B, n))
        A = self._check("A", A, (B, p, n))
        b = self._check("b", b, (B, p))
        G = self._check("G", G, (B, m, n))
        h = self._check("h", h, (B, m))
        st = settings if settings is not None else default_settings(**overrides)
        dev = self.device
        if out is None:
            out = dict(x=torch.empty(B, n, device=dev), y=torch.empty(B, p, device=dev),
                       z=torch.empty(B, m, device=dev), s=torch.empty(B, m, device=dev),
                       status=torch.empty(B, dtype=torch.int32, device=dev),
                       iters=torch.empty(B, dtype=torch.int32, device=dev),
                       kkt=torch.empty(B, device=dev))
        rc = _lib.lib().qp_solve_batch(
            self._h, ctypes.byref(st), ptr(Q), ptr(q), ptr(A), ptr(b), ptr(G), ptr(h),
            ptr(out["x"]), ptr(out["y"]), ptr(out["z"]), ptr(out["s"]), ptr(out["status"]),
            ptr(out["iters"]), ptr(out["kkt"]), ptr(grad_cache), _stream_handle(stream))
        check(rc, "qp_solve_batch")
        return out

    def backward(self, grad_cache: torch.Tensor, Q, A, G, dl_dx, out: Optional[Dict] = None,
                 stream: Optional[torch.cuda.Stream] = None) -> Dict[str, torch.Tensor]:
        """Alg. 3: gradients of <dl_dx, x(kappa_relax)> w.r.t. Q, q, A, b, G, h.
        Q, A, G are the data of the solve that filled ``grad_cache``."""
        B, n, p, m = self.batch, self.n, self.n_eq, self.n_ineq
        Q = self._check("Q", Q, (B, n, n))
        A = self._check("A", A, (B, p, n))
        G = self._check("G", G, (B, m, n))
        dl_dx = self._check("dl_dx", dl_dx, (B, n))
        dev = self.device
        if out is None:
            out = dict(dQ=torch.empty(B, n, n, device=dev), dq=torch.empty(B, n, device=dev),
                       dA=torch.empty(B, p, n, device=dev), db=torch.empty(B, p, device=dev),
                       dG=torch.empty(B, m, n, device=dev), dh=torch.empty(B, m, device=dev))
        rc = _lib.lib().qp_backward_batch(
            self._h, ptr(grad_cache), ptr(Q), ptr(A), ptr(G), ptr(dl_dx), ptr(out["dQ"]),
            ptr(out["dq"]),
            ptr(out["dA"]), ptr(out["db"]), ptr(out["dG"]), ptr(out["dh"]),
            _stream_handle(stream))
        check(rc, "qp_backward_batch")
        return out


_SOLVERS: Dict[tuple, QPSolver] = {}


def get_solver(batch: int, n: int, n_eq: int, n_ineq: int) -> QPSolver:
    key = (torch.cuda.current_device(), batch, n, n_eq, n_ineq)
    s = _SOLVERS.get(key)
    if s is None:
        s = _SOLVERS[key] = QPSolver(batch, n, n_eq, n_ineq)
    return s


class QPFunction(torch.autograd.Function):
    """x = argmin 1/2 x'Qx + q'x s.t. Ax = b, Gx <= h, batched; backward gives
    the gradients at the relaxed point kappa_relax (Alg. 2, Alg. 3)."""

    @staticmethod
    def forward(ctx, Q, q, A, b, G, h, settings: Optional[dict] = None):
        settings = dict(settings or {})
        B, n = q.shape
        p, m = A.shape[1], G.shape[1]
        solver = get_solver(B, n, p, m)
        cache = solver.new_grad_cache() if any(ctx.needs_input_grad[:6]) else None
        out = solver.solve(Q.contiguous(), q.contiguous(), A.contiguous(), b.contiguous(),
                           G.contiguous(), h.contiguous(), grad_cache=cache, **settings)
        ctx.solver = solver
        ctx.cache = cache
        ctx.save_for_backward(Q, A, G)
        ctx.mark_non_differentiable(out["status"])
        return out["x"], out["status"]

    @staticmethod
    def backward(ctx, gx, _gstatus):
        Q, A, G = ctx.saved_tensors
        g = ctx.solver.backward(ctx.cache, Q.contiguous(), A.contiguous(), G.contiguous(),
                                gx.contiguous())
        # with no equalities (inequalities) dA, db (dG, dh) are empty, like A, b (G, h)
        return g["dQ"], g["dq"], g["dA"], g["db"], g["dG"], g["dh"], None


def qp_layer(Q, q, A, b, G, h, **settings):
    """Differentiable batched QP solve; returns (x, status)."""
    return QPFunction.apply(Q, q, A, b, G, h, settings)
