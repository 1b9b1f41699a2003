"""Continuous-batching QP server (qp_serve_* in include/qp.h): marshalling only.

Requests are host (numpy) arrays of one instance each; the library's
scheduler thread batches them onto the GPU.  Output arrays are allocated by
this binding at submit and handed back when the request is collected.
"""
from __future__ import annotations

import ctypes
from typing import Dict, Optional

import numpy as np

from . import _lib
from ._lib import QP_ETIMEOUT, QP_PENDING, QPError, check


def footprint_bytes(n: int, n_eq: int, n_ineq: int, want_grad: bool) -> int:
    """Arena bytes one request occupies while resident (0: unsupported size)."""
    return int(_lib.lib().qp_serve_footprint_bytes(n, n_eq, n_ineq, int(bool(want_grad))))


def _host(a, shape) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if a.size != int(np.prod(shape)):
        raise QPError(f"array of {a.size} values, expected shape {shape}")
    return a


def _p(a: Optional[np.ndarray]):
    return None if a is None or a.size == 0 else a.ctypes.data


class QPServer:
    """One server per device: ``submit`` single QPs, collect them with
    ``poll``, ``poll_any`` or ``wait``.  ``mode``: "launches" (ragged launches
    per kernel class) or "persistent" (resident CTAs that claim requests as
    they arrive; every size at 512 threads per QP)."""

    def __init__(self, hbm_budget_bytes: int = 1 << 30, max_inflight: int = 8,
                 max_batch: int = 1024, max_queue: int = 1 << 20, mode: str = "persistent",
                 idle_ms: int = 50, **settings):
        L = _lib.lib()
        cfg = _lib.ServeConfig()
        L.qp_serve_config_default(ctypes.byref(cfg))
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.max_inflight, cfg.max_batch, cfg.max_queue = max_inflight, max_batch, max_queue
        if mode not in _lib.SERVE_MODES:
            raise QPError(f"unknown serving mode {mode!r}")
        cfg.mode = _lib.SERVE_MODES[mode]
        cfg.idle_ms = int(idle_ms)
        self.mode = mode
        cfg.settings = _lib.default_settings(**settings)
        h = ctypes.c_void_p()
        check(L.qp_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "qp_serve_create")
        self._h = h
        self._out: Dict[int, dict] = {}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().qp_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, Q, q, A, b, G, h, dl_dx=None) -> int:
        """Queue one QP (host arrays, copied before returning); returns its
        ticket.  Raises QPError (QP_EAGAIN) when the queue is full."""
        n = int(np.asarray(q).size)
        p = int(np.asarray(b).size)
        m = int(np.asarray(h).size)
        grad = dl_dx is not None
        arrs = dict(Q=_host(Q, (n, n)), q=_host(q, (n,)), A=_host(A, (p, n)), b=_host(b, (p,)),
                    G=_host(G, (m, n)), h=_host(h, (m,)))
        if grad:
            arrs["dl_dx"] = _host(dl_dx, (n,))
        out = dict(x=np.empty(n, np.float32), y=np.empty(p, np.float32),
                   z=np.empty(m, np.float32), s=np.empty(m, np.float32))
        if grad:
            out.update(dQ=np.empty((n, n), np.float32), dq=np.empty(n, np.float32),
                       dA=np.empty((p, n), np.float32), db=np.empty(p, np.float32),
                       dG=np.empty((m, n), np.float32), dh=np.empty(m, np.float32))
        r = _lib.Request(n, p, m, int(grad))
        for k, v in list(arrs.items()) + list(out.items()):
            setattr(r, k, _p(v))
        t = ctypes.c_uint64()
        check(_lib.lib().qp_serve_submit(self._h, ctypes.byref(r), ctypes.byref(t)),
              "qp_serve_submit")
        self._out[t.value] = out
        return t.value

    def _collect(self, rc: int, res: "_lib.Result") -> Optional[dict]:
        if rc == QP_PENDING:
            return None
        out = self._out.pop(res.ticket, {})
        check(rc, f"qp_serve (ticket {res.ticket})")
        d = dict(out)
        d.update(ticket=res.ticket, status=res.status, iters=res.iters, kkt=res.kkt_res,
                 t_submit_ms=res.t_submit_ms, t_launch_ms=res.t_launch_ms,
                 t_done_ms=res.t_done_ms)
        return d

    def poll(self, ticket: int) -> Optional[dict]:
        """The request's result, or None while it is queued or running."""
        res = _lib.Result()
        return self._collect(_lib.lib().qp_serve_poll(self._h, ticket, ctypes.byref(res)), res)

    def poll_any(self) -> Optional[dict]:
        """The earliest completed request not yet collected, or None."""
        res = _lib.Result()
        return self._collect(_lib.lib().qp_serve_poll_any(self._h, ctypes.byref(res)), res)

    def wait(self, ticket: int, timeout_ms: int = 60000) -> dict:
        """Wait (bounded) for one request; raises QPError on QP_ETIMEOUT."""
        res = _lib.Result()
        rc = _lib.lib().qp_serve_wait(self._h, ticket, int(timeout_ms), ctypes.byref(res))
        if rc == QP_ETIMEOUT:
            raise QPError(f"qp_serve_wait: ticket {ticket} not done after {timeout_ms} ms")
        return self._collect(rc, res)
