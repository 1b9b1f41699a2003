"""Closed-form fixtures of tests/golden/ (written by tests/golden/make_golden.py
from hand-derived formulas, no solver involved) against the FP64 oracle and
the GPU path.

central_path_separable: Q = I, G = I, h = u, no equalities, so every
coordinate is a 1-D problem whose relaxed point (z s = kappa_relax, Alg. 2) is
s = b_k(u + q), z = b_k(-(u + q)) (App. C) and whose gradients (Alg. 3) follow
by differentiating the KKT conditions of eq. 1 by hand; these fix every entry
of dG and dQ, including the off-diagonal ones that couple coordinates.
equality_projection: one equality, no inequalities, derivatives of the
explicit solution.
"""
import importlib.util
import json
import os

import numpy as np
import pytest

from oracle import oracle as O

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
GRAD_TOL = 1e-3   # relative 2-norm per gradient block (FP32 path)
X_TOL = 1e-4      # relative infinity norm of x (FP32 path)


def _cases(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)["cases"]


def _arrays(c):
    n, p, m = c["n"], c["n_eq"], c["n_ineq"]
    A = np.array(c["A"], dtype=np.float64).reshape(p, n)
    G = np.array(c["G"], dtype=np.float64).reshape(m, n)
    return (np.array(c["Q"]), np.array(c["q"]), A, np.array(c["b"]).reshape(p), G,
            np.array(c["h"]).reshape(m), np.array(c["g"]))


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-6)


def test_fixtures_are_what_the_script_writes():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    for name, content in mg.fixtures().items():
        with open(os.path.join(HERE, name)) as f:
            assert f.read() == mg.dumps(content), name


@pytest.mark.parametrize("idx", [0, 1])
def test_oracle_central_path_closed_form(idx):
    c = _cases("central_path_separable.json")[idx]
    Q, q, A, b, G, h, g = _arrays(c)
    r = O.solve(Q, q, A, b, G, h, tol=1e-13, kappa_relax=c["kappa_relax"], g=g)
    assert r["status"] == O.SOLVED
    for k, key in (("xr", "x_relaxed"), ("sr", "s_relaxed"), ("zr", "z_relaxed")):
        np.testing.assert_allclose(r[k], c[key], rtol=1e-12, atol=1e-13, err_msg=k)
    np.testing.assert_allclose(r["x"], c["x_optimum"], atol=1e-11)
    for k in ("dQ", "dq", "dG", "dh"):
        np.testing.assert_allclose(r[k], c[k], rtol=1e-11, atol=1e-13, err_msg=k)


@pytest.mark.parametrize("idx", [0, 1])
def test_oracle_standard_formulation_reaches_the_same_optimum(idx):
    """The explicit-complementarity ablation (eq. 6 / eq. 8) solves the same
    problem: x* = min(-q, u) coordinate-wise."""
    c = _cases("central_path_separable.json")[idx]
    Q, q, A, b, G, h, g = _arrays(c)
    r = O.solve(Q, q, A, b, G, h, tol=1e-12, formulation="standard")
    assert r["status"] == O.SOLVED
    np.testing.assert_allclose(r["x"], c["x_optimum"], atol=1e-10)


@pytest.mark.parametrize("idx", [0, 1])
def test_oracle_equality_closed_form(idx):
    c = _cases("equality_projection.json")[idx]
    Q, q, A, b, G, h, g = _arrays(c)
    r = O.solve(Q, q, A, b, G, h, tol=1e-13, g=g)
    assert r["status"] == O.SOLVED
    for k in ("x", "y", "dq", "dA", "db"):
        np.testing.assert_allclose(r[k], c[k], rtol=1e-12, atol=1e-13, err_msg=k)


def _gpu(c, kappa_relax):
    import torch

    from paper_2605_17913_gb300.solver import QPSolver

    arrs = _arrays(c)
    # a batch of 3 copies: instances are independent, so all three must agree
    T = [torch.from_numpy(np.ascontiguousarray(np.broadcast_to(a, (3,) + a.shape),
                                               dtype=np.float32)).cuda() for a in arrs]
    Q, q, A, b, G, h, g = T
    slv = QPSolver(3, c["n"], c["n_eq"], c["n_ineq"])
    cache = slv.new_grad_cache()
    out = slv.solve(Q, q, A, b, G, h, grad_cache=cache, tol=5e-6, kappa_relax=kappa_relax)
    grads = slv.backward(cache, Q, A, G, g)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res.update({k: v.cpu().numpy() for k, v in grads.items()})
    return res


@pytest.mark.gpu
@pytest.mark.parametrize("idx", [0, 1])
def test_gpu_central_path_closed_form(idx):
    c = _cases("central_path_separable.json")[idx]
    res = _gpu(c, c["kappa_relax"])
    assert np.all(res["status"] == 0)
    for i in range(3):
        x = res["x"][i]
        assert np.abs(x - c["x_optimum"]).max() / max(1.0, np.abs(c["x_optimum"]).max()) <= X_TOL
        for k in ("dQ", "dq", "dG", "dh"):
            assert _rel(res[k][i], c[k]) <= GRAD_TOL, (k, i, _rel(res[k][i], c[k]))


@pytest.mark.gpu
@pytest.mark.parametrize("idx", [0, 1])
def test_gpu_equality_closed_form(idx):
    c = _cases("equality_projection.json")[idx]
    res = _gpu(c, 1e-4)
    assert np.all(res["status"] == 0)
    for i in range(3):
        assert np.abs(res["x"][i] - c["x"]).max() / max(1.0, np.abs(c["x"]).max()) <= X_TOL
        for k in ("dq", "dA", "db"):
            assert _rel(res[k][i], c[k]) <= GRAD_TOL, (k, i, _rel(res[k][i], c[k]))


def test_fixtures_reject_planted_mistakes():
    """The fixtures are sharp enough to catch the plausible slips in Alg. 3:
    each variant below, built from the fixture's own dx = dq, dz = -dh and the
    relaxed point, misses the stored gradient by far more than the FP32 bar."""
    c = _cases("central_path_separable.json")[0]
    x, z = np.array(c["x_relaxed"]), np.array(c["z_relaxed"])
    dx, dz = np.array(c["dq"]), -np.array(c["dh"])
    dG, dQ = np.array(c["dG"]), np.array(c["dQ"])
    # the correct formulas reproduce the fixture (so the variants differ only by the slip)
    assert _rel(np.outer(dz, x) + np.outer(z, dx), dG) < 1e-12
    assert _rel(0.5 * (np.outer(dx, x) + np.outer(x, dx)), dQ) < 1e-12
    planted = {
        "dG without z dx'": np.outer(dz, x),
        "dG without dz x'": np.outer(z, dx),
        "dG transposed": (np.outer(dz, x) + np.outer(z, dx)).T,
        "dG with dz sign flipped": np.outer(-dz, x) + np.outer(z, dx),
        "dQ unsymmetrised": np.outer(dx, x),
        "dQ doubled": np.outer(dx, x) + np.outer(x, dx),
    }
    for name, wrong in planted.items():
        ref = dQ if name.startswith("dQ") else dG
        assert _rel(wrong, ref) > 50 * GRAD_TOL, name
