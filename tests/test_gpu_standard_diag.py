"""The standard formulation with eq. 8's matrix factored as it stands
(QP_STANDARD_SCHUR) against the FP64 oracle, and the per-instance
diagnostics words (qp_handle_set_diag): first non-finite stage, failed
factorisations, tensor-core and bulk-copy fallbacks."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_17913_gb300 import _lib
from paper_2605_17913_gb300.metrics import kkt_report, rel_err_inf
from paper_2605_17913_gb300.solver import QPSolver
from qpgen import make_batch

pytestmark = pytest.mark.gpu

STAGE = _lib.QP_STAGE_MASK


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g

    g.build()
    torch.cuda.set_device(0)


def _run(batch, grad=False, diag=True, **settings):
    T = {k: torch.from_numpy(np.ascontiguousarray(getattr(batch, k))).cuda()
         for k in ("Q", "q", "A", "b", "G", "h", "g")}
    slv = QPSolver(batch.batch, batch.n, batch.p, batch.m)
    dg = torch.full((batch.batch,), -1, dtype=torch.int32, device="cuda") if diag else None
    if diag:
        slv.set_diag(dg)
    cache = slv.new_grad_cache() if grad else None
    out = slv.solve(T["Q"], T["q"], T["A"], T["b"], T["G"], T["h"], grad_cache=cache, **settings)
    res = {k: v.cpu().numpy() for k, v in out.items()}
    if grad:
        res.update({k: v.cpu().numpy() for k, v in
                    slv.backward(cache, T["Q"], T["A"], T["G"], T["g"]).items()})
    torch.cuda.synchronize()
    if diag:
        res["diag"] = dg.cpu().numpy()
    return res, slv, T, cache, dg


def test_standard_schur_matches_oracle_where_it_solves():
    """Where FP32 Cholesky of Q + G' diag(z/s) G succeeds, the solution is the
    unique optimum (the oracle's), at the same bars as the implicit method."""
    batch = make_batch("small", 64, seed=11)
    res, *_ = _run(batch, formulation="standard_schur", tol=1e-4)
    ref = O.solve(batch.Q, batch.q, batch.A, batch.b, batch.G, batch.h, tol=1e-12, nthreads=8)
    ok = res["status"] == 0
    assert ok.mean() >= 0.5, np.unique(res["status"], return_counts=True)
    rep = kkt_report(batch.Q, batch.q, batch.A, batch.b, batch.G, batch.h, res["x"], res["y"],
                     res["z"], res["s"])
    assert rep["scaled"][ok].max() <= 2e-4
    assert rel_err_inf(res["x"][ok], ref["x"][ok]).max() <= 1e-3
    # failures are numerical and carry their first stage
    bad = res["status"] == _lib.QP_NUMERICAL
    assert np.all((res["diag"][bad] & STAGE) != 0)


def test_diag_words_implicit_clean():
    """The implicit method records no non-finite stage and no fallback."""
    batch = make_batch("small", 32, seed=12)
    res, *_ = _run(batch, grad=True, tol=5e-6)
    assert np.all(res["status"] == 0)
    assert np.all(res["diag"] == 0), res["diag"]


def test_diag_standard_schur_tight_tolerance():
    """At a tolerance below FP32's reach the plain Schur form breaks down on
    the degenerate workload; every instance that ends QP_NUMERICAL names its
    first non-finite stage, and a failed pivot carries the factor flag with
    the predictor stage (the factorisation's first use)."""
    batch = make_batch("degenerate", 128, seed=0)
    res, *_ = _run(batch, formulation="standard_schur", tol=1e-8, max_iter=60)
    st, dg = res["status"], res["diag"]
    assert np.all(dg >= 0)
    numerical = st == _lib.QP_NUMERICAL
    assert np.all((dg[numerical] & STAGE) != 0)
    failed = (dg & _lib.QP_DIAG_FACTOR_FAILED) != 0
    assert np.all((dg[failed] & STAGE) == 2)
    assert np.all((dg[st == 0] & STAGE) == 0)


def test_diag_backward_stage():
    """A cache whose factors are not finite: the backward pass records its
    own stage for an instance the solve left clean."""
    batch = make_batch("small", 4, seed=13)
    res, slv, T, cache, dg = _run(batch, grad=True, tol=5e-6)
    assert np.all(res["diag"] == 0)
    stride = cache.numel() // batch.batch
    cache.view(batch.batch, stride)[0, 4:] = float("nan")  # keep instance 0's header
    g = slv.backward(cache, T["Q"], T["A"], T["G"], T["g"])
    torch.cuda.synchronize()
    d = dg.cpu().numpy()
    assert (d[0] & STAGE) == 7, d
    assert np.all(d[1:] == 0)
    assert not torch.isfinite(g["dq"][0]).all()


@pytest.mark.parametrize("gwg", ["fp32", "tf32", "bf16"])
def test_large_variant_no_fallback(gwg):
    """The large variant's staged and tensor-core G'WG finish within their
    bounded waits: no fallback bit on any instance."""
    batch = make_batch("precision", 4, seed=0)
    res, *_ = _run(batch, grad=True, tol=5e-6, gwg_precision=gwg)
    assert np.all(res["status"] == 0)
    assert np.all(res["diag"] == 0), res["diag"]
