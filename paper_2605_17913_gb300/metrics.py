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

# Bars of gradient_report under which an instance's gradients count as
# consistent with Alg. 3: exact gradients rounded to FP32 give ~1e-7, exact
# gradients with 1e-3 relative noise in every entry ~2e-3; a dropped term, a
# sign slip or a swapped operand gives 0.5 or more.
GRAD_CONSISTENCY_BAR = 1e-3
GRAD_POINT_BAR = 1e-2


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


def gradient_report(Q, q, A, b, G, g, dQ, dq, dA, db, dG, dh) -> dict:
    """Per-instance FP64 consistency of returned gradients with Alg. 3.

    With dx = dq, dy = -db, dz = -dh (Alg. 3 returns grad_q = dx,
    grad_b = -dy, grad_h = -dz):
      adjoint:   r1 = Q dx + A'dy + G'dz + g   (first block row of the adjoint
                 system at any point, = 0),  r2 = A dx (= 0);
                 relative: |r1| / max(|g|, |Q dx|, |A'dy|, |G'dz|),
                 |r2| / (|A| |dx|)                          (infinity norms);
      structure: grad_Q = (dx x' + x dx')/2, grad_A = dy x' + y dx',
                 grad_G = dz x' + z dx' for one point (x, y, z) (the relaxed
                 point): x, y, z are recovered from the blocks themselves
                 (c = dx' grad_Q dx / |dx|^2 = x'dx; x = (2 grad_Q dx - c dx) / |dx|^2;
                 y = (grad_A dx - c dy) / |dx|^2; z likewise) and the fit's
                 residual is reported relative to each block's norm;
      point:     the recovered (x, y, z) is the relaxed central-path point, so
                 it is stationary, Qx + q + G'z + A'y = 0 and Ax = b (scaled as
                 in kkt_report), with z > 0 (reported: max(0, -min z) / max z).
    The adjoint and structure values are ~1e-7 for FP32-rounded exact
    gradients and the point's residual ~1e-5 (it inherits the gradients' own
    error); a dropped term, a sign slip or a transposed block gives O(1).
    """
    f = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731
    Q, q, A, b, G, g, dQ, dq, dA, db, dG, dh = map(f, (Q, q, A, b, G, g, dQ, dq, dA, db, dG, dh))
    B = dq.shape[0]
    dx, dy, dz = dq, -db, -dh
    Qdx = np.einsum("bij,bj->bi", Q, dx)
    Atdy = np.einsum("bki,bk->bi", A, dy)
    Gtdz = np.einsum("bki,bk->bi", G, dz)
    r1 = Qdx + Atdy + Gtdz + g
    den1 = np.maximum.reduce([_amax(g, 1), _amax(Qdx, 1), _amax(Atdy, 1), _amax(Gtdz, 1),
                              np.full(B, 1e-300)])
    adj1 = _amax(r1, 1) / den1
    if A.shape[1]:
        Adx = np.einsum("bkj,bj->bk", A, dx)
        adj2 = _amax(Adx, 1) / np.maximum(np.abs(A).sum(axis=2).max(axis=1) * _amax(dx, 1),
                                          1e-300)
    else:
        adj2 = np.zeros(B)
    nn = np.maximum(np.einsum("bi,bi->b", dx, dx), 1e-300)
    c = np.einsum("bi,bij,bj->b", dx, dQ, dx) / nn
    x = (2.0 * np.einsum("bij,bj->bi", dQ, dx) - c[:, None] * dx) / nn[:, None]

    def fit(M, Mhat):
        if M.shape[1] == 0:
            return np.zeros(B)
        den = np.maximum(np.linalg.norm(M.reshape(B, -1), axis=1), 1e-300)
        return np.linalg.norm((M - Mhat).reshape(B, -1), axis=1) / den

    sQ = fit(dQ, 0.5 * (dx[:, :, None] * x[:, None, :] + x[:, :, None] * dx[:, None, :]))
    y = (np.einsum("bkj,bj->bk", dA, dx) - c[:, None] * dy) / nn[:, None]
    sA = fit(dA, dy[:, :, None] * x[:, None, :] + y[:, :, None] * dx[:, None, :])
    z = (np.einsum("bkj,bj->bk", dG, dx) - c[:, None] * dz) / nn[:, None]
    sG = fit(dG, dz[:, :, None] * x[:, None, :] + z[:, :, None] * dx[:, None, :])
    # the recovered point: stationarity, equality feasibility, z > 0
    Qx = np.einsum("bij,bj->bi", Q, x)
    Gtz = np.einsum("bki,bk->bi", G, z)
    Aty = np.einsum("bki,bk->bi", A, y)
    one = np.ones(B)
    dt = np.maximum.reduce([one, _amax(Qx, 1), _amax(q, 1), _amax(Aty, 1), _amax(Gtz, 1)])
    pt = _amax(Qx + q + Gtz + Aty, 1) / dt
    if A.shape[1]:
        Ax = np.einsum("bkj,bj->bk", A, x)
        pt = np.maximum(pt, _amax(Ax - b, 1) / np.maximum.reduce([one, _amax(Ax, 1), _amax(b, 1)]))
    if G.shape[1]:
        pz = np.maximum(-z.min(axis=1), 0.0) / np.maximum(z.max(axis=1), 1e-300)
    else:
        pz = np.zeros(B)
    worst = np.maximum.reduce([adj1, adj2, sQ, sA, sG])
    worst[~np.isfinite(worst)] = np.inf
    point = np.maximum(pt, pz)
    point[~np.isfinite(point)] = np.inf
    return dict(adjoint=adj1, adjoint_eq=adj2, structure_Q=sQ, structure_A=sA,
                structure_G=sG, worst=worst, point=point)
