"""ctypes binding of the FP64 CPU oracle (``qp_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use it to check the CUDA path.  Nothing in the product
package imports it, and it imports nothing from the product package.

Functions follow the paper: ``solve`` runs Alg. 1 (implicit complementarity,
predictor-corrector sigma), optionally Alg. 2 (relax to kappa_relax) and
Alg. 3 (gradients at the relaxed point); ``formulation="standard"`` runs the
explicit-complementarity ablation (eq. 6 / eq. 8, Mehrotra).
Parity status: pinned (closed forms, brute-force active sets, known optima,
central-path invariants, the linearisation that one direction solves and
central finite differences in tests/; mistakes planted in copies of the C
source fail those pins).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

SOLVED, MAX_ITER, STALLED, NUMERICAL, BAD_INPUT = 0, 1, 2, 3, 4


class _Settings(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("sigma_mode", ctypes.c_int),
        ("sigma", ctypes.c_double),
        ("kappa_min", ctypes.c_double),
        ("scaled", ctypes.c_int),
        ("step_frac", ctypes.c_double),
    ]


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("p", ctypes.c_int), ("m", ctypes.c_int),
        ("Q", ctypes.c_void_p), ("q", ctypes.c_void_p), ("A", ctypes.c_void_p),
        ("b", ctypes.c_void_p), ("G", ctypes.c_void_p), ("h", ctypes.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
               _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    """The oracle library: ``liboracle.so`` (built on first use), or the build
    that ``QP_ORACLE_LIB`` names -- a separately compiled copy of
    ``qp_oracle.c``, used by the test that plants mistakes in the oracle and
    checks that its pins catch them."""
    global _lib
    if _lib is None:
        other = os.environ.get("QP_ORACLE_LIB")
        L = ctypes.CDLL(other if other else build())
        d, vp, i = ctypes.c_double, ctypes.c_void_p, ctypes.c_int
        L.oqp_retract.restype = d
        L.oqp_retract.argtypes = [d, d]
        L.oqp_retract_dv.restype = d
        L.oqp_retract_dv.argtypes = [d, d]
        L.oqp_retract_dk.restype = d
        L.oqp_retract_dk.argtypes = [d, d]
        L.oqp_kkt_measure.restype = d
        L.oqp_kkt_measure.argtypes = [ctypes.POINTER(_Problem), vp, vp, vp, vp, i]
        L.oqp_newton_direction.restype = i
        L.oqp_newton_direction.argtypes = [ctypes.POINTER(_Problem)] + [vp] * 4 + [d] + [vp] * 6
        L.oqp_batch.restype = i
        L.oqp_batch.argtypes = ([i, i, i, i, i] + [vp] * 7 + [ctypes.POINTER(_Settings), d]
                                + [vp] * 8 + [vp] * 4 + [vp] * 6 + [i])
        _lib = L
    return _lib


def retract(v: float, kappa: float) -> float:
    """b_kappa(v), eq. 11 in the cancellation-free form of App. C."""
    return lib().oqp_retract(float(v), float(kappa))


def retract_dv(v: float, kappa: float) -> float:
    """d/dv b_kappa(v), App. C."""
    return lib().oqp_retract_dv(float(v), float(kappa))


def retract_dk(v: float, kappa: float) -> float:
    """d/dkappa b_kappa(v) = 1/sqrt(v^2 + 4 kappa)."""
    return lib().oqp_retract_dk(float(v), float(kappa))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _as_batch(Q, q, A, b, G, h):
    Q = _f64(Q)
    single = Q.ndim == 2
    if single:
        Q = Q[None]
    B, n = Q.shape[0], Q.shape[1]
    q = _f64(q).reshape(B, n)
    A = _f64(A).reshape(B, -1, n) if np.size(A) else np.zeros((B, 0, n))
    b = _f64(b).reshape(B, A.shape[1])
    G = _f64(G).reshape(B, -1, n) if np.size(G) else np.zeros((B, 0, n))
    h = _f64(h).reshape(B, G.shape[1])
    return single, Q, q, A, b, G, h


def kkt_measure(Q, q, A, b, G, h, x, y, z, s, scaled: bool = True) -> float:
    """Scaled (or absolute) infinity-norm KKT measure of one iterate, in FP64."""
    _, Qb, qb, Ab, bb, Gb, hb = _as_batch(Q, q, A, b, G, h)
    n, p, m = Qb.shape[1], Ab.shape[1], Gb.shape[1]
    arrs = [Qb[0], qb[0], Ab[0], bb[0], Gb[0], hb[0]]
    P = _Problem(n, p, m, *[_ptr(a) for a in arrs])
    xs = [_f64(v) for v in (x, y, z, s)]
    return lib().oqp_kkt_measure(ctypes.byref(P), *[_ptr(v) for v in xs], int(scaled))


def newton_direction(Q, q, A, b, G, h, x, y, z, s, kappa_target: float) -> dict:
    """One Alg. 1 direction at (x, y, z, s) toward ``kappa_target``: eq. 14
    solved at v = z - s, kappa = s'z/m, then dz, ds, dkappa from eq. 13.
    Returns dx, dy, dv, dz, ds, dkappa and the status."""
    _, Qb, qb, Ab, bb, Gb, hb = _as_batch(Q, q, A, b, G, h)
    n, p, m = Qb.shape[1], Ab.shape[1], Gb.shape[1]
    arrs = [Qb[0], qb[0], Ab[0], bb[0], Gb[0], hb[0]]
    P = _Problem(n, p, m, *[_ptr(a) for a in arrs])
    xs = [_f64(v) for v in (x, y, z, s)]
    out = dict(dx=np.zeros(n), dy=np.zeros(p), dv=np.zeros(m), dz=np.zeros(m), ds=np.zeros(m))
    dk = ctypes.c_double(0.0)
    st = lib().oqp_newton_direction(ctypes.byref(P), *[_ptr(v) for v in xs], float(kappa_target),
                                    *[_ptr(out[k]) for k in ("dx", "dy", "dv", "dz", "ds")],
                                    ctypes.byref(dk))
    out["dkappa"] = dk.value
    out["status"] = st
    return out


def solve(Q, q, A, b, G, h, *, tol: float = 1e-12, max_iter: int = 100, sigma_mode: int = 0,
          sigma: float = 0.1, kappa_min: Optional[float] = None, scaled: bool = True,
          step_frac: float = 1.0, formulation: str = "implicit",
          kappa_relax: Optional[float] = None, g=None, nthreads: int = 1) -> dict:
    """Run the oracle on one problem (2-D Q) or a batch (3-D Q) of one size.

    Returns a dict with the solution x, y, z, s of Alg. 1, the relaxed point
    xr, yr, zr, sr of Alg. 2 (equal to the solution without ``kappa_relax``),
    status, iters, relax_iters, res and, when ``g`` is given, the gradients
    dQ, dq, dA, db, dG, dh of <g, x> at the relaxed point.
    """
    single, Q, q, A, b, G, h = _as_batch(Q, q, A, b, G, h)
    B, n, p, m = Q.shape[0], Q.shape[1], A.shape[1], G.shape[1]
    if kappa_min is None:
        kappa_min = 1e-2 * tol
    S = _Settings(tol, max_iter, sigma_mode, sigma, kappa_min, int(scaled), step_frac)
    mode = 1
    if kappa_relax is not None:
        mode |= 2
    if g is not None:
        mode |= 4
        g = _f64(g).reshape(B, n)
    if formulation == "standard":
        mode |= 8
    elif formulation != "implicit":
        raise ValueError(formulation)
    out = {k: np.zeros((B,) + shp) for k, shp in
           dict(x=(n,), y=(p,), z=(m,), s=(m,), res=(), xr=(n,), yr=(p,), zr=(m,),
                sr=(m,)).items()}
    out["status"] = np.zeros(B, dtype=np.int32)
    out["iters"] = np.zeros(B, dtype=np.int32)
    out["relax_iters"] = np.zeros(B, dtype=np.int32)
    grads = [None] * 6
    if g is not None:
        for k, shp in dict(dQ=(n, n), dq=(n,), dA=(p, n), db=(p,), dG=(m, n), dh=(m,)).items():
            out[k] = np.zeros((B,) + shp)
        grads = [out[k] for k in ("dQ", "dq", "dA", "db", "dG", "dh")]
    lib().oqp_batch(B, n, p, m, mode, *[_ptr(a) for a in (Q, q, A, b, G, h, g)],
                    ctypes.byref(S), float(kappa_relax or 0.0),
                    *[_ptr(out[k]) for k in ("x", "y", "z", "s", "res", "status", "iters",
                                             "relax_iters", "xr", "yr", "zr", "sr")],
                    *[_ptr(a) for a in grads], int(nthreads))
    if single:
        out = {k: v[0] for k, v in out.items()}
    return out
