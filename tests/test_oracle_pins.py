"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formulas: each compares it with a
closed form, an exact high-precision value, a different algorithm (brute-force
active-set enumeration, a plain KKT solve, finite differences) or an
invariant the paper states.
"""
import itertools

import mpmath
import numpy as np
import pytest

from oracle import oracle as O
from qpgen import make_instance

mpmath.mp.dps = 60


# ---------------------------------------------------------------- retraction
V_GRID = [s * 10.0 ** e for e in range(-20, 7, 2) for s in (1.0, -1.0)] + [0.0, 0.37, -0.37]
K_GRID = [1e-30, 1e-20, 1e-12, 1e-8, 1e-4, 1e-2, 1.0]


def _b_exact(v, k):
    v, k = mpmath.mpf(v), mpmath.mpf(k)
    return (v + mpmath.sqrt(v * v + 4 * k)) / 2


@pytest.mark.parametrize("kappa", K_GRID)
def test_retraction_matches_exact_value(kappa):
    """eq. 11 evaluated in 60-digit arithmetic; App. C's form must be accurate
    to a few ulp even where the naive form cancels (v < 0, v^2 >> kappa)."""
    for v in V_GRID:
        ex = _b_exact(v, kappa)
        got = O.retract(v, kappa)
        assert abs(mpmath.mpf(got) - ex) <= 4e-16 * abs(ex), (v, kappa, got, ex)


@pytest.mark.parametrize("kappa", K_GRID)
def test_retraction_identities(kappa):
    """eq. 10/12: b(v) b(-v) = kappa, b(v) - b(-v) = v, b'(v) + b'(-v) = 1, 0 < b' <= 1."""
    for v in V_GRID:
        bp, bm = O.retract(v, kappa), O.retract(-v, kappa)
        assert bp > 0 and bm > 0
        assert abs(bp * bm - kappa) <= 1e-15 * kappa * 4
        assert abs((bp - bm) - v) <= 9e-16 * max(abs(v), bp, bm)
        dp, dm = O.retract_dv(v, kappa), O.retract_dv(-v, kappa)
        assert 0.0 < dp <= 1.0 and 0.0 < dm <= 1.0
        assert abs(dp + dm - 1.0) <= 4e-16


@pytest.mark.parametrize("kappa", [1e-12, 1e-4, 1.0])
def test_retraction_derivatives_exact(kappa):
    """d/dv and d/dkappa of eq. 11, by 60-digit numerical differentiation."""
    for v in [-1e3, -3.0, -1e-3, 0.0, 1e-3, 2.5, 1e3]:
        dv = mpmath.diff(lambda t: _b_exact(t, kappa), v)
        dk = mpmath.diff(lambda t: _b_exact(v, t), kappa)
        assert abs(mpmath.mpf(O.retract_dv(v, kappa)) - dv) <= 1e-14 * abs(dv)
        assert abs(mpmath.mpf(O.retract_dk(v, kappa)) - dk) <= 1e-14 * abs(dk)


# ---------------------------------------------------------------- helpers
def _solve(d, **kw):
    return O.solve(d["Q"], d["q"], d["A"], d["b"], d["G"], d["h"], **kw)


def _rand_qp(rng, n, m, p, feasible_margin=True):
    M = rng.standard_normal((n, n))
    Q = M @ M.T + 0.1 * np.eye(n)
    Q = 0.5 * (Q + Q.T)
    q = rng.standard_normal(n)
    G = rng.standard_normal((m, n))
    A = rng.standard_normal((p, n))
    x0 = rng.standard_normal(n)
    h = G @ x0 + rng.uniform(0.1, 1.0, m)
    b = A @ x0
    return dict(Q=Q, q=q, A=A, b=b, G=G, h=h)


def _brute_force(d):
    """Enumerate active sets: for each subset S of inequalities solve the
    equality-constrained QP with rows [A; G_S]; keep the feasible, dual-
    feasible one.  Q > 0 makes the minimiser unique."""
    Q, q, A, b, G, h = (d[k] for k in ("Q", "q", "A", "b", "G", "h"))
    n, m, p = Q.shape[0], G.shape[0], A.shape[0]
    best = None
    for r in range(0, min(m, n - p) + 1):
        for S in itertools.combinations(range(m), r):
            E = np.vstack([A, G[list(S)]]) if (p + r) else np.zeros((0, n))
            e = np.concatenate([b, h[list(S)]])
            K = np.block([[Q, E.T], [E, np.zeros((p + r, p + r))]])
            try:
                sol = np.linalg.solve(K, np.concatenate([-q, e]))
            except np.linalg.LinAlgError:
                continue
            x, lam = sol[:n], sol[n:]
            zS = lam[p:]
            if np.all(G @ x <= h + 1e-9) and np.all(zS >= -1e-9):
                f = 0.5 * x @ Q @ x + q @ x
                if best is None or f < best[0] - 1e-12:
                    best = (f, x)
    return best[1]


# ---------------------------------------------------------------- forward pins
def test_unconstrained_closed_form():
    rng = np.random.default_rng(1)
    for n in (1, 3, 10):
        M = rng.standard_normal((n, n))
        Q = M @ M.T + np.eye(n)
        q = rng.standard_normal(n)
        r = O.solve(Q, q, np.zeros((0, n)), np.zeros(0), np.zeros((0, n)), np.zeros(0))
        assert r["status"] == O.SOLVED
        np.testing.assert_allclose(r["x"], -np.linalg.solve(Q, q), rtol=0, atol=1e-12)


def test_equality_only_kkt_solve():
    rng = np.random.default_rng(2)
    n, p = 6, 2
    d = _rand_qp(rng, n, 0, p)
    r = _solve(d)
    K = np.block([[d["Q"], d["A"].T], [d["A"], np.zeros((p, p))]])
    sol = np.linalg.solve(K, np.concatenate([-d["q"], d["b"]]))
    np.testing.assert_allclose(r["x"], sol[:n], atol=1e-12)
    np.testing.assert_allclose(r["y"], sol[n:], atol=1e-11)


def test_box_projection_clip():
    """Q = I, G = [I; -I], h = [u; -l]: x* = clip(-q, l, u)."""
    rng = np.random.default_rng(3)
    n = 7
    for _ in range(5):
        q = 2.0 * rng.standard_normal(n)
        lo, hi = -rng.uniform(0.2, 1.0, n), rng.uniform(0.2, 1.0, n)
        G = np.vstack([np.eye(n), -np.eye(n)])
        h = np.concatenate([hi, -lo])
        r = O.solve(np.eye(n), q, np.zeros((0, n)), np.zeros(0), G, h)
        assert r["status"] == O.SOLVED
        np.testing.assert_allclose(r["x"], np.clip(-q, lo, hi), atol=1e-10)


@pytest.mark.parametrize("formulation", ["implicit", "standard"])
def test_brute_force_active_sets(formulation):
    rng = np.random.default_rng(4)
    count = 0
    for trial in range(200):
        n = int(rng.integers(1, 5))
        m = int(rng.integers(1, 9))
        p = int(rng.integers(0, min(2, n)))
        d = _rand_qp(rng, n, m, p)
        d["q"] = 3.0 * d["q"]  # push the optimum onto the boundary more often
        r = _solve(d, formulation=formulation)
        assert r["status"] == O.SOLVED, (trial, r["status"])
        xb = _brute_force(d)
        np.testing.assert_allclose(r["x"], xb, atol=1e-8, err_msg=f"trial {trial}")
        count += int(np.any(np.abs(d["G"] @ xb - d["h"]) < 1e-9))
    assert count > 50  # many instances have active inequalities


def test_known_optimum_degenerate_construction():
    """Degenerate workload: x* = x0 by construction (m/2 + p > n active rows)."""
    for i in range(3):
        d = make_instance("degenerate", i)
        r = _solve(d, tol=1e-12)
        assert r["status"] == O.SOLVED
        np.testing.assert_allclose(r["x"], d["x0"], atol=1e-10)
        rs = _solve(d, tol=1e-12, formulation="standard")
        np.testing.assert_allclose(rs["x"], d["x0"], atol=1e-9)


def test_kkt_conditions_at_solution_small():
    """eq. 4 at the returned point, recomputed with numpy."""
    for i in range(8):
        d = make_instance("small", i)
        r = _solve(d, tol=1e-12)
        x, y, z, s = r["x"], r["y"], r["z"], r["s"]
        Q, q, A, b, G, h = (d[k] for k in ("Q", "q", "A", "b", "G", "h"))
        assert np.abs(Q @ x + q + G.T @ z + A.T @ y).max() < 1e-10
        assert np.abs(A @ x - b).max() < 1e-11
        assert np.abs(G @ x + s - h).max() < 1e-11
        assert z.min() > 0 and s.min() > 0 and (z * s).max() < 1e-12
        assert abs(O.kkt_measure(Q, q, A, b, G, h, x, y, z, s, scaled=False)
                   - max(np.abs(Q @ x + q + G.T @ z + A.T @ y).max(), np.abs(A @ x - b).max(),
                         np.abs(G @ x + s - h).max(), (z * s).max())) < 1e-12


def test_batch_matches_single_and_threads():
    ds = [make_instance("small", i) for i in range(6)]
    st = {k: np.stack([d[k] for d in ds]) for k in ("Q", "q", "A", "b", "G", "h", "g")}
    rb = O.solve(st["Q"], st["q"], st["A"], st["b"], st["G"], st["h"], kappa_relax=1e-4,
                 g=st["g"], nthreads=3)
    for i, d in enumerate(ds):
        r1 = _solve(d, kappa_relax=1e-4, g=d["g"])
        for k in ("x", "y", "z", "s", "xr", "zr", "dQ", "dG", "dh"):
            np.testing.assert_array_equal(rb[k][i], r1[k])


# ---------------------------------------------------------------- relaxation
def test_relaxed_point_is_central_path_point():
    """Alg. 2 output: z.*s = kappa_relax and r_t = r_e = r_i = 0 (invariant)."""
    for kr in (1e-2, 1e-4, 1e-6):
        d = make_instance("small", 3)
        r = _solve(d, tol=1e-13, kappa_relax=kr)
        assert r["status"] == O.SOLVED
        x, y, z, s = r["xr"], r["yr"], r["zr"], r["sr"]
        Q, q, A, b, G, h = (d[k] for k in ("Q", "q", "A", "b", "G", "h"))
        np.testing.assert_allclose(z * s, kr, rtol=1e-10)
        assert np.abs(Q @ x + q + G.T @ z + A.T @ y).max() < 1e-10
        assert np.abs(G @ x + s - h).max() < 1e-11
        assert np.abs(A @ x - b).max() < 1e-11


def test_relaxed_point_tends_to_optimum():
    d = make_instance("small", 5)
    x_star = _solve(d, tol=1e-13)["x"]
    errs = [np.abs(_solve(d, tol=1e-13, kappa_relax=kr)["xr"] - x_star).max()
            for kr in (1e-2, 1e-4, 1e-6, 1e-8)]
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-6


# ---------------------------------------------------------------- gradients
def test_gradient_unconstrained_closed_form():
    rng = np.random.default_rng(7)
    n = 5
    M = rng.standard_normal((n, n))
    Q = M @ M.T + np.eye(n)
    q, g = rng.standard_normal(n), rng.standard_normal(n)
    e0 = np.zeros((0, n))
    r = O.solve(Q, q, e0, np.zeros(0), e0, np.zeros(0), g=g)
    x = -np.linalg.solve(Q, q)
    dx = -np.linalg.solve(Q, g)
    np.testing.assert_allclose(r["dq"], dx, atol=1e-12)
    np.testing.assert_allclose(r["dQ"], 0.5 * (np.outer(dx, x) + np.outer(x, dx)), atol=1e-12)


def _relaxed_x(d, kr, **over):
    e = dict(d)
    e.update(over)
    r = O.solve(e["Q"], e["q"], e["A"], e["b"], e["G"], e["h"], tol=1e-13, kappa_relax=kr)
    assert r["status"] == O.SOLVED
    return r["xr"]


@pytest.mark.parametrize("index", [0, 1])
def test_gradient_central_finite_differences(index):
    """<g, x(kappa_relax; theta)> differentiated by central differences (h = 1e-6)
    along random directions per block (symmetric directions for Q)."""
    kr = 1e-3
    d = make_instance("small", index)
    g = d["g"]
    r = _solve(d, tol=1e-13, kappa_relax=kr, g=g)
    rng = np.random.default_rng(11 + index)
    hstep = 1e-6
    for key, gk in (("Q", "dQ"), ("q", "dq"), ("A", "dA"), ("b", "db"), ("G", "dG"),
                    ("h", "dh")):
        for _ in range(4):
            E = rng.standard_normal(d[key].shape)
            if key == "Q":
                E = 0.5 * (E + E.T)
            fp = g @ _relaxed_x(d, kr, **{key: d[key] + hstep * E})
            fm = g @ _relaxed_x(d, kr, **{key: d[key] - hstep * E})
            fd = (fp - fm) / (2 * hstep)
            an = float(np.sum(r[gk] * E))
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (key, fd, an)


def test_gradient_matches_hard_projection_jacobian():
    """App. D: projection onto a polytope with a known active face; as
    kappa_relax -> 0, d<v, Pi(x)>/dx -> J_hard v with
    J_hard = I - G_A^T (G_A G_A^T)^{-1} G_A (eq. 21)."""
    errs = []
    for kr in (1e-4, 1e-6, 1e-8):
        d = make_instance("projection", 0, n=20, m=25, m_act=10, d=1.0)
        r = O.solve(d["Q"], d["q"], d["A"], d["b"], d["G"], d["h"], tol=1e-13,
                    kappa_relax=kr, g=d["g"])
        np.testing.assert_allclose(r["xr"], d["x0"], atol=50 * kr + 1e-9)
        GA = d["G"][: d["n_active"]]
        J = np.eye(20) - GA.T @ np.linalg.solve(GA @ GA.T, GA)
        g_hard = J @ d["g"]
        g_qp = -r["dq"]  # q = -x_query
        errs.append(np.linalg.norm(g_qp - g_hard) / np.linalg.norm(g_hard))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5


def test_gradient_equality_constrained_closed_form():
    """Equality-only QP: x = solution of [Q A';A 0]; the IFT gives
    [Q A';A 0](dx, dy) = (-g, 0) and the Alg. 3 formulas."""
    rng = np.random.default_rng(9)
    n, p = 6, 2
    d = _rand_qp(rng, n, 0, p)
    g = rng.standard_normal(n)
    r = O.solve(d["Q"], d["q"], d["A"], d["b"], d["G"], d["h"], g=g)
    K = np.block([[d["Q"], d["A"].T], [d["A"], np.zeros((p, p))]])
    sol = np.linalg.solve(K, np.concatenate([-d["q"], d["b"]]))
    x, y = sol[:n], sol[n:]
    adj = np.linalg.solve(K, np.concatenate([-g, np.zeros(p)]))
    dx, dy = adj[:n], adj[n:]
    np.testing.assert_allclose(r["dq"], dx, atol=1e-11)
    np.testing.assert_allclose(r["db"], -dy, atol=1e-11)
    np.testing.assert_allclose(r["dA"], np.outer(dy, x) + np.outer(y, dx), atol=1e-10)


def test_absolute_kkt_measure_at_arbitrary_points():
    """The absolute measure is the largest infinity norm among eq. 4's r_t, r_e,
    r_i and the complementarity z.*s, at any point, not only near a solution
    (where every term is tiny)."""
    rng = np.random.default_rng(12)
    for trial in range(20):
        n, m, p = 6, 9, 2
        d = _rand_qp(rng, n, m, p)
        x, y = rng.standard_normal(n), rng.standard_normal(p)
        z, s = rng.uniform(0.01, 3.0, m), rng.uniform(0.01, 3.0, m)
        if trial % 2:
            z *= 10.0  # complementarity the largest term
        Q, q, A, b, G, h = (d[k] for k in ("Q", "q", "A", "b", "G", "h"))
        want = max(np.abs(Q @ x + q + G.T @ z + A.T @ y).max(), np.abs(A @ x - b).max(),
                   np.abs(G @ x + s - h).max(), (z * s).max())
        got = O.kkt_measure(Q, q, A, b, G, h, x, y, z, s, scaled=False)
        assert abs(got - want) <= 1e-13 * want, (trial, got, want)


# ---------------------------------------------------------------- Newton direction
def _b_directional(v, k, dv, dk):
    """d/dt b_{k + t dk}(v + t dv) at t = 0 (eq. 11), by 60-digit central
    differences of the exact formula."""
    t = mpmath.mpf("1e-25")
    v, k, dv, dk = (mpmath.mpf(a) for a in (v, k, dv, dk))
    return (_b_exact(v + t * dv, k + t * dk) - _b_exact(v - t * dv, k - t * dk)) / (2 * t)


@pytest.mark.parametrize("on_manifold", [True, False])
@pytest.mark.parametrize("target", [0.0, 0.2])
def test_newton_direction_solves_the_linearised_conditions(on_manifold, target):
    """One Alg. 1 direction is Newton's step for eq. 4 with z = b_k(v),
    s = b_k(-v) (eq. 11) in the coordinates (x, y, v, kappa):
      Q dx + G'dz + A'dy = -r_t,  A dx = -r_e,  G dx + ds = -r_i,
      dkappa = kappa_target - kappa,
      dz = b_k(v) - z + Db_k(v)[dv, dkappa],  ds = b_k(-v) - s + Db_k(-v)[-dv, dkappa].
    Residuals in numpy, the retraction's derivative by 60-digit differences:
    this fixes eq. 13 and eq. 14 (matrix, right-hand side and recovery)."""
    rng = np.random.default_rng(21 + int(on_manifold) + int(10 * target))
    n, m, p = 5, 8, 2
    for _ in range(4):
        d = _rand_qp(rng, n, m, p)
        Q, q, A, b, G, h = (d[k] for k in ("Q", "q", "A", "b", "G", "h"))
        x, y = rng.standard_normal(n), rng.standard_normal(p)
        if on_manifold:
            kap, v = 0.3, rng.standard_normal(m)
            z = np.array([float(_b_exact(a, kap)) for a in v])
            s = np.array([float(_b_exact(-a, kap)) for a in v])
        else:
            z, s = rng.uniform(0.05, 2.0, m), rng.uniform(0.05, 2.0, m)
        v, kap = z - s, float(s @ z) / m
        kt = target * kap
        r = O.newton_direction(Q, q, A, b, G, h, x, y, z, s, kt)
        assert r["status"] == O.SOLVED
        dx, dy, dv, dz, ds, dk = (r[k] for k in ("dx", "dy", "dv", "dz", "ds", "dkappa"))
        rt, re, ri = Q @ x + q + G.T @ z + A.T @ y, A @ x - b, G @ x + s - h
        scale = max(1.0, np.abs(rt).max(), np.abs(ri).max(), np.abs(dx).max(), np.abs(dz).max())
        assert np.abs(Q @ dx + G.T @ dz + A.T @ dy + rt).max() <= 1e-11 * scale
        assert np.abs(A @ dx + re).max() <= 1e-11 * scale
        assert np.abs(G @ dx + ds + ri).max() <= 1e-11 * scale
        assert abs(dk - (kt - kap)) <= 1e-15 * kap
        for i in range(m):
            want_z = _b_exact(v[i], kap) - z[i] + _b_directional(v[i], kap, dv[i], dk)
            want_s = _b_exact(-v[i], kap) - s[i] + _b_directional(-v[i], kap, -dv[i], dk)
            assert abs(dz[i] - float(want_z)) <= 1e-12 * scale, (i, dz[i], want_z)
            assert abs(ds[i] - float(want_s)) <= 1e-12 * scale, (i, ds[i], want_s)
