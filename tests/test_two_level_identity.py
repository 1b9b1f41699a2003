"""The two-level bounded elimination that the CUDA path factors (reading R9)
solves eq. 14 exactly: checked in FP64 on the CPU, against the oracle's
Newton direction (which its own pin holds to the linearisation of eq. 4 and
eq. 11), for random iterates on and off the central path and for any
activity threshold tau.

Rows with W = B_k(v) / B_k(-v) <= tau are eliminated into
K_I = Q + G_I' W_I G_I; the others stay as lambda = dv_A - G_A dx beside the
equality rows, giving the saddle-point system
    [ K_I  F' ] [dx]   [ rhs1 ]      F = [G_A; A],  D = diag(B_-/B_+ on A, 0)
    [ F   -D  ] [mu] = [ rhs2 ]
solved by K_I = L L', Y = F L^-T, C = D + Y Y', u = L^-1 rhs1,
C mu = Y u - rhs2, dx = L^-T (u - Y' mu).  Every pivot of that route is
bounded: B_- >= 1 / (1 + tau) on the eliminated rows (1/2 at the default
tau = 1), D < 1 / tau on the kept ones.
The right-hand sides are affine in r_kappa, so the two columns r_kappa = 0
and d/dr_kappa give every kappa_target.  The adjoint solve of Alg. 3 takes
the same route (eq. 14 is symmetric) and gives the oracle's gradients.
"""
import numpy as np
import pytest

from oracle import oracle as O


def _b(v, k):
    """b_k(v), eq. 11, in the cancellation-free form of App. C."""
    r = np.sqrt(v * v + 4.0 * k)
    return np.where(v >= 0, 0.5 * (v + r), 2.0 * k / (r - v))


def _db(v, k):
    """d/dv b_k(v) = b_k(v) / sqrt(v^2 + 4k) (from eq. 11)."""
    return _b(v, k) / np.sqrt(v * v + 4.0 * k)


def _two_level(Q, G, A, v, k, rt, re, ri, rz, rs, rk, tau):
    n, m, p = Q.shape[0], G.shape[0], A.shape[0]
    Bp, Bm, c = _db(v, k), _db(-v, k), 1.0 / np.sqrt(v * v + 4.0 * k)
    W = Bp / Bm
    I, Aa = np.where(W <= tau)[0], np.where(W > tau)[0]
    rho1 = rt - G.T @ (ri + rz - rs)
    rho2 = ri - rs - c * rk
    GI, GA = G[I], G[Aa]
    KI = Q + GI.T @ (W[I][:, None] * GI)
    F = np.vstack([GA, A])
    D = np.concatenate([Bm[Aa] / Bp[Aa], np.zeros(p)])
    rhs1 = -rho1 - GI.T @ (rho2[I] / Bm[I])
    rhs2 = np.concatenate([-rho2[Aa] / Bp[Aa], -re])
    L = np.linalg.cholesky(KI)
    Y = np.linalg.solve(L, F.T).T                      # F L^-T
    C = np.diag(D) + Y @ Y.T
    u = np.linalg.solve(L, rhs1)
    mu = np.linalg.solve(C, Y @ u - rhs2) if C.size else np.zeros(0)
    dx = np.linalg.solve(L.T, u - Y.T @ mu)
    lam, dy = mu[:len(Aa)], mu[len(Aa):]
    dv = np.empty(m)
    dv[I] = (GI @ dx + rho2[I]) / Bm[I]
    dv[Aa] = lam + GA @ dx
    dz = -rz + Bp * dv - c * rk
    ds = -rs - Bm * dv - c * rk
    return dict(dx=dx, dy=dy, dv=dv, dz=dz, ds=ds, Bm_I=Bm[I], D_A=D[:len(Aa)],
                n_active=len(Aa))


def _rand(rng, n, m, p, scale_v):
    M = rng.standard_normal((n, n))
    Q = M @ M.T / n + 0.1 * np.eye(n)
    G = rng.standard_normal((m, n))
    A = rng.standard_normal((p, n))
    q, h, b = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(p)
    x, y = rng.standard_normal(n), rng.standard_normal(p)
    v = scale_v * rng.standard_normal(m)
    return Q, q, A, b, G, h, x, y, v


@pytest.mark.parametrize("tau", [1.0, 4.0, 1e3])
@pytest.mark.parametrize("on_path", [True, False])
def test_two_level_elimination_solves_eq14(tau, on_path):
    rng = np.random.default_rng(5 + int(tau) + 7 * int(on_path))
    kept = eliminated = 0
    for trial in range(6):
        n, m, p = 7, 12, 2
        kappa0 = 10.0 ** rng.uniform(-6, -1)
        # |v| large against sqrt(kappa): W spans many decades, as near a solution
        Q, q, A, b, G, h, x, y, v = _rand(rng, n, m, p, scale_v=1.0)
        if on_path:
            z, s = _b(v, kappa0), _b(-v, kappa0)
        else:
            z = _b(v, kappa0) * rng.uniform(0.5, 2.0, m)
            s = _b(-v, kappa0) * rng.uniform(0.5, 2.0, m)
        v, k = z - s, float(z @ s) / m
        kt = 0.1 * k
        ref = O.newton_direction(Q, q, A, b, G, h, x, y, z, s, kt)
        assert ref["status"] == O.SOLVED
        rt, re, ri = Q @ x + q + G.T @ z + A.T @ y, A @ x - b, G @ x + s - h
        rz, rs = z - _b(v, k), s - _b(-v, k)
        got = _two_level(Q, G, A, v, k, rt, re, ri, rz, rs, k - kt, tau)
        for key in ("dx", "dy", "dv", "dz", "ds"):
            scale = max(1.0, np.abs(ref[key]).max()) if ref[key].size else 1.0
            err = np.abs(got[key] - ref[key]).max() / scale if ref[key].size else 0.0
            assert err <= 1e-8, (trial, key, err)
        # the pivots of the route stay bounded whatever kappa is: W <= tau
        # means B_- >= 1 / (1 + tau) (B_+ + B_- = 1, eq. 12), and D = 1 / W
        assert np.all(got["Bm_I"] >= 1.0 / (1.0 + tau) - 1e-15)
        assert np.all(got["D_A"] < 1.0 / tau + 1e-15)
        kept += got["n_active"]
        eliminated += m - got["n_active"]
    assert kept > 0 and eliminated > 0  # both routes of the split were taken


def test_two_columns_give_every_kappa_target():
    """The right-hand sides are affine in r_kappa: the solution for any
    kappa_target is col0 + r_kappa * col1 (r_kappa = kappa - kappa_target)."""
    rng = np.random.default_rng(3)
    n, m, p = 6, 10, 1
    Q, q, A, b, G, h, x, y, v = _rand(rng, n, m, p, scale_v=0.3)
    kappa = 1e-3
    z, s = _b(v, kappa), _b(-v, kappa)
    rt, re, ri = Q @ x + q + G.T @ z + A.T @ y, A @ x - b, G @ x + s - h
    zero = np.zeros(m)
    col0 = _two_level(Q, G, A, v, kappa, rt, re, ri, zero, zero, 0.0, 1.0)
    col1 = _two_level(Q, G, A, v, kappa, 0 * rt, 0 * re, 0 * ri, zero, zero, 1.0, 1.0)
    for kt in (0.0, 0.3 * kappa, kappa, 2.0 * kappa):
        ref = O.newton_direction(Q, q, A, b, G, h, x, y, z, s, kt)
        rk = kappa - kt
        for key in ("dx", "dv", "dz", "ds"):
            np.testing.assert_allclose(col0[key] + rk * col1[key], ref[key], rtol=0,
                                       atol=1e-9 * max(1.0, np.abs(ref[key]).max()))


@pytest.mark.parametrize("workload", ["small", "degenerate"])
def test_two_level_adjoint_gives_the_oracle_gradients(workload):
    """Alg. 3 through the same route: eq. 14 is symmetric, so the adjoint is
    the route with right-hand side (-g, 0, 0) (rho1 = g, everything else 0) at
    the relaxed point, dz = B_k(v) dv, and the gradient blocks of Alg. 3
    follow; they equal the oracle's, which solves the full system."""
    from qpgen import make_instance

    kr = 1e-4
    for i in range(3):
        d = make_instance(workload, i)
        Q, q, A, b, G, h, g = (d[k] for k in ("Q", "q", "A", "b", "G", "h", "g"))
        r = O.solve(Q, q, A, b, G, h, tol=1e-12, kappa_relax=kr, g=g)
        assert r["status"] == O.SOLVED
        x, y, z, s = r["xr"], r["yr"], r["zr"], r["sr"]
        v = z - s
        n, m, p = Q.shape[0], G.shape[0], A.shape[0]
        adj = _two_level(Q, G, A, v, kr, g, np.zeros(p), np.zeros(m), np.zeros(m),
                         np.zeros(m), 0.0, 1.0)
        dx, dy, dz = adj["dx"], adj["dy"], _db(v, kr) * adj["dv"]
        got = dict(dq=dx, db=-dy, dh=-dz, dQ=0.5 * (np.outer(dx, x) + np.outer(x, dx)),
                   dA=np.outer(dy, x) + np.outer(y, dx), dG=np.outer(dz, x) + np.outer(z, dx))
        for key, val in got.items():
            ref = r[key]
            err = np.abs(val - ref).max() / max(1.0, np.abs(ref).max())
            assert err <= 1e-7, (workload, i, key, err)
