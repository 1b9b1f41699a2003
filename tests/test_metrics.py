"""The FP64 gradient-consistency report the bench counts instances with
(metrics.gradient_report): exact gradients of the FP64 oracle and their FP32
roundings pass its bars; planted slips in the Alg. 3 gradient blocks fail them
by orders of magnitude."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_17913_gb300.metrics import GRAD_CONSISTENCY_BAR, GRAD_POINT_BAR, gradient_report
from qpgen import make_batch

KEYS = ("dQ", "dq", "dA", "db", "dG", "dh")


@pytest.fixture(scope="module", params=["small", "degenerate"])
def case(request):
    B = 6 if request.param == "small" else 3
    d = make_batch(request.param, B, seed=0)
    r = O.solve(d.Q, d.q, d.A, d.b, d.G, d.h, tol=1e-12, kappa_relax=1e-4, g=d.g, nthreads=6)
    return d, r


def _rep(d, grads):
    return gradient_report(d.Q, d.q, d.A, d.b, d.G, d.g, *(grads[k] for k in KEYS))


def test_exact_gradients_are_consistent(case):
    d, r = case
    rep = _rep(d, r)
    assert rep["worst"].max() < 1e-11
    assert rep["point"].max() < 1e-9


def test_fp32_rounded_gradients_pass_the_bars(case):
    d, r = case
    f32 = {k: r[k].astype(np.float32) for k in KEYS}
    rep = _rep(d, f32)
    assert rep["worst"].max() < GRAD_CONSISTENCY_BAR / 10
    assert rep["point"].max() < GRAD_POINT_BAR / 10


def test_recovered_point_is_the_relaxed_point(case):
    d, r = case
    f = {k: r[k] for k in KEYS}
    dx = f["dq"]
    nn = (dx * dx).sum(1)
    c = np.einsum("bi,bij,bj->b", dx, f["dQ"], dx) / nn
    x = (2 * np.einsum("bij,bj->bi", f["dQ"], dx) - c[:, None] * dx) / nn[:, None]
    assert np.abs(x - r["xr"]).max() < 1e-9


@pytest.mark.parametrize("slip", ["dh_sign", "dG_dropped_z_term", "dA_transposed_roles",
                                  "dQ_unsymmetrised", "dx_without_GtWG", "db_sign"])
def test_planted_slips_fail(case, slip):
    d, r = case
    f = {k: r[k].astype(np.float32).astype(np.float64) for k in KEYS}
    x, y, z = r["xr"], r["yr"], r["zr"]
    if slip == "dh_sign":
        f["dh"] = -f["dh"]
    elif slip == "dG_dropped_z_term":
        f["dG"] = f["dG"] - z[:, :, None] * f["dq"][:, None, :]
    elif slip == "dA_transposed_roles":
        # y x' in place of dy x' (a swapped operand)
        f["dA"] = y[:, :, None] * x[:, None, :] + y[:, :, None] * f["dq"][:, None, :]
    elif slip == "dQ_unsymmetrised":
        f["dQ"] = f["dq"][:, :, None] * x[:, None, :]
    elif slip == "dx_without_GtWG":
        # the adjoint solved with Q alone (G'WG dropped from the Newton matrix)
        f["dq"] = np.linalg.solve(d.Q.astype(np.float64), -d.g.astype(np.float64)[:, :, None])[:, :, 0]
    elif slip == "db_sign":
        f["db"] = -f["db"]
    rep = _rep(d, f)
    bad = (rep["worst"] > 100 * GRAD_CONSISTENCY_BAR) | (rep["point"] > 10 * GRAD_POINT_BAR)
    assert bad.all(), {k: v.tolist() for k, v in rep.items()}
