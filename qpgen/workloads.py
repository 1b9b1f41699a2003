"""Seeded synthetic inputs for batches of dense convex QPs.

    minimise  1/2 x^T Q x + q^T x   subject to  A x = b,  G x <= h        (eq. 1)

Sizes use the build's names: ``n`` variables, ``m`` inequality rows (G, h)
and ``p`` equality rows (A, b).  (The paper's own letters swap m and p.)

Every instance is drawn from its own counter-based Philox stream keyed by
(seed, workload, instance index), so instance ``i`` is the same whether it is
drawn alone or inside a batch of any size.  Data are drawn in FP64; callers
that feed the FP32 solver round them with ``dtype=np.float32`` and hand the
same rounded numbers to every checker.

Workloads (one per named configuration):

``small``       n=10,  m=20,  p=2.   Q = M M^T + 1e-2 I, M ~ N(0,1);
                q ~ N(0,1); G, A ~ N(0,1); x0 ~ N(0,1); s0 ~ U(0.1, 1);
                h = G x0 + s0; b = A x0.  Strictly feasible at x0.
``degenerate``  n=50,  m=100, p=10.  As ``small`` but s0 = 0 on a random half
                of the rows, and q is built so that x0 is optimal:
                z0 ~ U(0.1,1) on the rows with s0 = 0 (0 elsewhere),
                y0 ~ N(0,1), q = -(Q x0 + A^T y0 + G^T z0).  Then exactly m/2
                inequalities are active at the optimum x* = x0 and, with
                m/2 + p > n, the active rows are linearly dependent.
                ``q_mode="gauss"`` gives the literal q ~ N(0,1) variant.
``diff``        n=100, m=200, p=20.  As ``small``; also draws the upstream
                gradient g = dL/dx ~ N(0,1).
``precision``   n=256, m=512, p=32.  Q = U diag(logspace(0, 4, n)) U^T with U
                Haar-orthogonal (QR of a Gaussian, signs fixed), cond(Q)=1e4;
                otherwise as ``small``.  ``Q_mode="mmt"`` gives the literal
                Q = M M^T + 1e-3 I variant.
``serving``     n = round(exp(U(ln 8, ln 256))), m = 2n, p = floor(n/10);
                data as ``small``; 30% of requests want gradients.
``projection``  Euclidean projection onto a polytope with a prescribed active
                face: Q = I, q = -x_query, no equalities, G rows ~ N(0, I)
                normalised to unit length, y0 ~ N(0, I), the first ``m_act``
                rows active at y0 (h = G y0 there), the others inactive with
                h = G y0 + U(0.1, 1); x_query = y0 + G_A^T (d * xi),
                xi ~ U(0.5, 1.5).  Then the projection of x_query is y0.
``safety``      the centralised CBF safety-filter QP of k planar agents (the
                paper's App. E shapes; default k = 7: n = 14, m = 70, p = 0).
                u in R^{2k}; Q = I, q = -u_nom; rows: the box -u_max <= u_c
                <= u_max (4k rows, u_max = 2), one zeroing-CBF row per agent
                and obstacle (3 obstacles: -2 (p_i - c_o)' u_i <= alpha h_obs,
                h_obs = |p_i - c_o|^2 - r_o^2) and one per agent pair
                (-2 (p_i - p_j)' (u_i - u_j) <= alpha h_pair, h_pair =
                |p_i - p_j|^2 - (2 r_agent)^2, r_agent = 0.35).  Positions,
                goals and obstacle centres ~ U(-3, 3)^2, radii ~ U(0.3, 0.8),
                each agent redrawn until it is safe (every h >= 0.05); gains
                alpha ~ U(0.5, 2); u_nom = 3 (g_i - p_i) / max(|g_i - p_i|, 0.1)
                (the goal-seeking law, not clipped, so box rows can bind).
                u = 0 is strictly feasible (x0 = 0).  Shapes and structure
                only: no rollouts, no learned gains.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional

import numpy as np

# Stable integer codes that key the per-instance random streams.
_WORKLOAD_CODE = {
    "small": 1,
    "degenerate": 2,
    "diff": 3,
    "precision": 4,
    "serving": 5,
    "projection": 6,
    "custom": 7,
    "safety": 8,
}

CONFIGS: Dict[str, dict] = {
    "small": dict(n=10, m=20, p=2, batch=64, Q_mode="mmt", reg=1e-2,
                  q_mode="gauss", s0_mode="uniform"),
    "degenerate": dict(n=50, m=100, p=10, batch=4096, Q_mode="mmt", reg=1e-2,
                       q_mode="optimal_x0", s0_mode="half_zero"),
    "diff": dict(n=100, m=200, p=20, batch=1024, Q_mode="mmt", reg=1e-2,
                 q_mode="gauss", s0_mode="uniform"),
    "precision": dict(n=256, m=512, p=32, batch=256, Q_mode="logspec", reg=1e-3,
                      cond=1e4, q_mode="gauss", s0_mode="uniform"),
    "safety": dict(n=14, m=70, p=0, batch=65536, agents=7),
}


def safety_size(agents: int):
    """(n, m, p) of the k-agent safety-filter QP: 2k, 4k + 3k + k(k-1)/2, 0."""
    k = int(agents)
    return 2 * k, 4 * k + 3 * k + k * (k - 1) // 2, 0


@dataclasses.dataclass
class QPBatch:
    """A uniform-size batch, batch-major and row-major per instance."""

    Q: np.ndarray  # [B, n, n]
    q: np.ndarray  # [B, n]
    A: np.ndarray  # [B, p, n]
    b: np.ndarray  # [B, p]
    G: np.ndarray  # [B, m, n]
    h: np.ndarray  # [B, m]
    x0: np.ndarray  # [B, n]  point used to build the data (optimal for "degenerate")
    g: np.ndarray  # [B, n]  upstream gradient dL/dx
    workload: str = "custom"
    seed: int = 0
    start: int = 0

    @property
    def batch(self) -> int:
        return self.Q.shape[0]

    @property
    def n(self) -> int:
        return self.Q.shape[1]

    @property
    def m(self) -> int:
        return self.G.shape[1]

    @property
    def p(self) -> int:
        return self.A.shape[1]

    def astype(self, dtype) -> "QPBatch":
        f = lambda a: np.ascontiguousarray(a, dtype=dtype)  # noqa: E731
        return dataclasses.replace(
            self, Q=f(self.Q), q=f(self.q), A=f(self.A), b=f(self.b), G=f(self.G),
            h=f(self.h), x0=f(self.x0), g=f(self.g))

    def instance(self, i: int) -> dict:
        return dict(Q=self.Q[i], q=self.q[i], A=self.A[i], b=self.b[i],
                    G=self.G[i], h=self.h[i])


def instance_rng(seed: int, workload: str, index: int) -> np.random.Generator:
    """Counter-based Philox stream for one instance."""
    ss = np.random.SeedSequence([int(seed), _WORKLOAD_CODE[workload], int(index)])
    return np.random.Generator(np.random.Philox(ss))


def _sym(M: np.ndarray) -> np.ndarray:
    return 0.5 * (M + M.T)


def _haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    Z = rng.standard_normal((n, n))
    Qm, R = np.linalg.qr(Z)
    return Qm * np.sign(np.diag(R))[None, :]


def make_instance(workload: str, index: int, seed: int = 0, *, n: Optional[int] = None,
                  m: Optional[int] = None, p: Optional[int] = None, **overrides) -> dict:
    """Draw one instance (FP64).  Returns dict(Q,q,A,b,G,h,x0,g)."""
    if workload == "serving":
        rng = instance_rng(seed, workload, index)
        n_, m_, p_, _ = _serving_size(rng)
        cfg = dict(CONFIGS["small"])
        cfg.update(n=n_, m=m_, p=p_)
    elif workload == "projection":
        return _projection_instance(index, seed, n=n, m=m, **overrides)
    elif workload == "safety":
        return _safety_instance(index, seed, **overrides)
    else:
        cfg = dict(CONFIGS.get(workload, CONFIGS["small"]))
        rng = instance_rng(seed, workload, index)
    cfg.update(overrides)
    if n is not None:
        cfg["n"] = n
    if m is not None:
        cfg["m"] = m
    if p is not None:
        cfg["p"] = p
    n_, m_, p_ = int(cfg["n"]), int(cfg["m"]), int(cfg["p"])

    if cfg["Q_mode"] == "mmt":
        M = rng.standard_normal((n_, n_))
        Q = _sym(M @ M.T) + cfg["reg"] * np.eye(n_)
    elif cfg["Q_mode"] == "logspec":
        U = _haar_orthogonal(rng, n_)
        lam = np.logspace(0.0, math.log10(cfg.get("cond", 1e4)), n_)
        Q = _sym((U * lam[None, :]) @ U.T)
    elif cfg["Q_mode"] == "identity":
        Q = np.eye(n_)
    else:
        raise ValueError(cfg["Q_mode"])
    q = rng.standard_normal(n_)
    G = rng.standard_normal((m_, n_))
    A = rng.standard_normal((p_, n_))
    x0 = rng.standard_normal(n_)
    s0 = rng.uniform(0.1, 1.0, m_)
    if cfg["s0_mode"] == "half_zero":
        active = rng.permutation(m_)[: m_ // 2]
        s0[active] = 0.0
    h = G @ x0 + s0
    b = A @ x0
    if cfg["q_mode"] == "optimal_x0":
        z0 = np.zeros(m_)
        z0[s0 == 0.0] = rng.uniform(0.1, 1.0, int(np.count_nonzero(s0 == 0.0)))
        y0 = rng.standard_normal(p_)
        q = -(Q @ x0 + A.T @ y0 + G.T @ z0)
    g = rng.standard_normal(n_)
    return dict(Q=Q, q=q, A=A, b=b, G=G, h=h, x0=x0, g=g)


def make_batch(workload: str, batch: Optional[int] = None, seed: int = 0, start: int = 0,
               dtype=np.float32, **overrides) -> QPBatch:
    """Stack instances start..start+batch-1 of a uniform-size workload."""
    if workload == "serving":
        raise ValueError("serving requests have uneven sizes; use make_instance per request")
    if batch is None:
        batch = CONFIGS[workload]["batch"]
    insts = [make_instance(workload, start + i, seed, **overrides) for i in range(batch)]
    if batch == 0:
        probe = make_instance(workload, 0, seed, **overrides)
        insts, zero = [probe], True
    else:
        zero = False
    stack = lambda k: np.stack([d[k] for d in insts])  # noqa: E731
    out = QPBatch(Q=stack("Q"), q=stack("q"), A=stack("A"), b=stack("b"), G=stack("G"),
                  h=stack("h"), x0=stack("x0"), g=stack("g"), workload=workload,
                  seed=seed, start=start)
    if zero:
        out = dataclasses.replace(out, **{k: getattr(out, k)[:0] for k in
                                          ("Q", "q", "A", "b", "G", "h", "x0", "g")})
    return out.astype(dtype)


def _serving_size(rng: np.random.Generator):
    n = int(round(math.exp(rng.uniform(math.log(8.0), math.log(256.0)))))
    want_grad = bool(rng.uniform() < 0.3)
    return n, 2 * n, n // 10, want_grad


def serving_sizes(count: int, seed: int = 0, start: int = 0):
    """(n, m, p, want_grad) of serving requests start..start+count-1."""
    out = []
    for i in range(start, start + count):
        out.append(_serving_size(instance_rng(seed, "serving", i)))
    return out


def _projection_instance(index: int, seed: int, *, n=None, m=None, m_act=None, d=1.0,
                         **_):
    n_ = 20 if n is None else int(n)
    m_ = int(round(1.25 * n_)) if m is None else int(m)
    ma = (m_ // 2) if m_act is None else int(m_act)
    rng = instance_rng(seed, "projection", index)
    G = rng.standard_normal((m_, n_))
    G /= np.linalg.norm(G, axis=1, keepdims=True)
    y0 = rng.standard_normal(n_)
    slack = np.zeros(m_)
    slack[ma:] = rng.uniform(0.1, 1.0, m_ - ma)
    h = G @ y0 + slack
    xi = rng.uniform(0.5, 1.5, ma)
    xq = y0 + G[:ma].T @ (d * xi)
    probe = rng.standard_normal(n_)
    return dict(Q=np.eye(n_), q=-xq, A=np.zeros((0, n_)), b=np.zeros(0), G=G, h=h,
                x0=y0, g=probe, x_query=xq, n_active=ma)


def _safety_instance(index: int, seed: int, *, agents: int = 7, u_max: float = 2.0,
                     n_obs: int = 3, r_agent: float = 0.35, **_):
    k = int(agents)
    n_, m_, _p = safety_size(k)
    rng = instance_rng(seed, "safety", index)
    c = rng.uniform(-3.0, 3.0, (n_obs, 2))
    r = rng.uniform(0.3, 0.8, n_obs)
    pos = np.zeros((k, 2))
    for i in range(k):
        for _try in range(1000):
            pi = rng.uniform(-3.0, 3.0, 2)
            ok = np.all(np.sum((pi - c) ** 2, axis=1) - r ** 2 >= 0.05)
            ok = ok and all(np.sum((pi - pos[j]) ** 2) - (2 * r_agent) ** 2 >= 0.05
                            for j in range(i))
            if ok:
                break
        pos[i] = pi
    goal = rng.uniform(-3.0, 3.0, (k, 2))
    d = goal - pos
    u_nom = (3.0 * d / np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 0.1)).reshape(-1)
    G = np.zeros((m_, n_))
    h = np.zeros(m_)
    row = 0
    for cc in range(n_):                     # box
        G[row, cc], h[row] = 1.0, u_max
        G[row + 1, cc], h[row + 1] = -1.0, u_max
        row += 2
    for i in range(k):                       # obstacles
        for o in range(n_obs):
            dp = pos[i] - c[o]
            G[row, 2 * i:2 * i + 2] = -2.0 * dp
            h[row] = rng.uniform(0.5, 2.0) * (dp @ dp - r[o] ** 2)
            row += 1
    for i in range(k):                       # agent pairs
        for j in range(i + 1, k):
            dp = pos[i] - pos[j]
            G[row, 2 * i:2 * i + 2] = -2.0 * dp
            G[row, 2 * j:2 * j + 2] = 2.0 * dp
            h[row] = rng.uniform(0.5, 2.0) * (dp @ dp - (2 * r_agent) ** 2)
            row += 1
    assert row == m_
    g = rng.standard_normal(n_)
    return dict(Q=np.eye(n_), q=-u_nom, A=np.zeros((0, n_)), b=np.zeros(0), G=G, h=h,
                x0=np.zeros(n_), g=g)
