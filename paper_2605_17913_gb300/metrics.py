"""Host-side accuracy report of returned solutions, in FP64 (numpy).

For each instance, from the FP32 outputs and the FP32 data:
  r_t = Qx + q + G'z + A'y,  r_e = Ax - b,  r_i = Gx + s - h   (eq. 4)
  scaled measure = max( |r_t| / max(1, |Qx|, |q|, |A'y|, |G'z|),
                        |r_e| / max(1, |Ax|, |b|),
                        |r_i| / max(1, |Gx|, |h|, |s|),
                        max_i z_i s_i )                     (infinity norms)
and the absolute measure max(|r_t|, |r_e|, |r_i|, max z.*s).  This is the
number the solver's tolerance is checked against when results are counted.
"""
from __future__ import annotations

import numpy as np


def _amax(a, axis):
    return np.abs(a).max(axis=axis) if a.shape[axis] > 0 else np.zeros(a.shape[0])


def kkt_report(Q, q, A, b, G, h, x, y, z, s) -> dict:
    f = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731
    Q, q, A, b, G, h, x, y, z, s = map(f, (Q, q, A, b, G, h, x, y, z, s))
    Qx = np.einsum("bij,bj->bi", Q, x)
    Gtz = np.einsum("bki,bk->bi", G, z)
    Aty = np.einsum("bki,bk->bi", A, y)
    Ax = np.einsum("bkj,bj->bk", A, x)
    Gx = np.einsum("bkj,bj->bk", G, x)
    rt = Qx + q + Gtz + Aty
    re = Ax - b
    ri = Gx + s - h
    zs = (z * s).max(axis=1) if z.shape[1] else np.zeros(x.shape[0])
    one = np.ones(x.shape[0])
    dt = np.maximum.reduce([one, _amax(Qx, 1), _amax(q, 1), _amax(Aty, 1), _amax(Gtz, 1)])
    de = np.maximum.reduce([one, _amax(Ax, 1), _amax(b, 1)])
    di = np.maximum.reduce([one, _amax(Gx, 1), _amax(h, 1), _amax(s, 1)])
    et, ee, ei = _amax(rt, 1), _amax(re, 1), _amax(ri, 1)
    scaled = np.maximum.reduce([et / dt, ee / de, ei / di, zs])
    absolute = np.maximum.reduce([et, ee, ei, zs])
    obj = 0.5 * np.einsum("bi,bi->b", x, Qx) + np.einsum("bi,bi->b", q, x)
    bad = ~np.isfinite(scaled)
    scaled[bad] = np.inf
    absolute[bad] = np.inf
    return dict(scaled=scaled, absolute=absolute, objective=obj, min_z=z.min(axis=1) if z.shape[1]
                else one, min_s=s.min(axis=1) if s.shape[1] else one)


def rel_err_inf(a, ref) -> np.ndarray:
    """Per-instance |a - ref|_inf / max(1, |ref|_inf)."""
    a = np.asarray(a, dtype=np.float64).reshape(a.shape[0], -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(ref.shape[0], -1)
    if a.shape[1] == 0:
        return np.zeros(a.shape[0])
    return np.abs(a - ref).max(axis=1) / np.maximum(1.0, np.abs(ref).max(axis=1))


def rel_err_2(a, ref, floor: float = 1e-6) -> np.ndarray:
    """Per-instance |a - ref|_2 / max(|ref|_2, floor)."""
    a = np.asarray(a, dtype=np.float64).reshape(a.shape[0], -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(ref.shape[0], -1)
    if a.shape[1] == 0:
        return np.zeros(a.shape[0])
    return np.linalg.norm(a - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), floor)
