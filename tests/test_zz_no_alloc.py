"""qp_solve_backward_static (solve + relax + backward with the factor cache in
the library's fixed device array) against the two-call path qp_solve_batch +
qp_backward_batch with a caller-owned cache, through the C ABI.

The file name sorts last so that the suite also exercises the fixed array
after every other test has run; it passes on its own in a fresh process too.
"""
import ctypes

import numpy as np
import pytest
import torch

from qpgen import make_batch

pytestmark = pytest.mark.gpu

SOLVER_TOL = 5e-6
GRAD_KEYS = ("dQ", "dq", "dA", "db", "dG", "dh")
OUT_KEYS = ("x", "y", "z", "s", "status", "iters", "kkt")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g

    g.build()
    torch.cuda.set_device(0)


def _device_data(batch):
    return {k: torch.from_numpy(np.ascontiguousarray(getattr(batch, k))).cuda()
            for k in ("Q", "q", "A", "b", "G", "h", "g")}


def _outputs(B, n, p, m, fill=0.0):
    f = dict(device="cuda")
    out = dict(x=torch.full((B, n), fill, **f), y=torch.full((B, p), fill, **f),
               z=torch.full((B, m), fill, **f), s=torch.full((B, m), fill, **f),
               status=torch.full((B,), -9, dtype=torch.int32, **f),
               iters=torch.zeros(B, dtype=torch.int32, **f), kkt=torch.zeros(B, **f))
    out.update(dQ=torch.full((B, n, n), fill, **f), dq=torch.full((B, n), fill, **f),
               dA=torch.full((B, p, n), fill, **f), db=torch.full((B, p), fill, **f),
               dG=torch.full((B, m, n), fill, **f), dh=torch.full((B, m), fill, **f))
    return out


def _static_call(slv, T, out, settings):
    from paper_2605_17913_gb300 import _lib
    from paper_2605_17913_gb300._lib import ptr

    return _lib.lib().qp_solve_backward_static(
        slv._h, ctypes.byref(settings), *(ptr(T[k]) for k in ("Q", "q", "A", "b", "G", "h", "g")),
        *(ptr(out[k]) for k in OUT_KEYS), *(ptr(out[k]) for k in GRAD_KEYS),
        torch.cuda.current_stream().cuda_stream)


def _two_call_path(slv, T, settings):
    cache = slv.new_grad_cache()
    out = slv.solve(T["Q"], T["q"], T["A"], T["b"], T["G"], T["h"], settings=settings,
                    grad_cache=cache)
    out.update(slv.backward(cache, T["Q"], T["A"], T["G"], T["g"]))
    return out


def test_static_cache_matches_caller_cache_on_consecutive_calls():
    from paper_2605_17913_gb300 import _lib
    from paper_2605_17913_gb300.solver import QPSolver

    B = 96
    first = make_batch("degenerate", B, seed=0)
    second = make_batch("degenerate", B, seed=1)
    # the second call has one instance with non-finite data; its slot of the
    # fixed array still holds the first call's factor, which must not leak
    # into the second call's gradients
    second.q[5, 0] = np.nan
    slv = QPSolver(B, first.n, first.p, first.m)
    assert slv.grad_cache_bytes <= _lib.QP_STATIC_CACHE_BYTES
    settings = _lib.default_settings(tol=SOLVER_TOL)
    for data in (first, second):
        T = _device_data(data)
        out = _outputs(B, data.n, data.p, data.m)
        rc = _static_call(slv, T, out, settings)
        assert rc == _lib.QP_OK, _lib.status_string(rc)
        ref = _two_call_path(slv, T, settings)
        torch.cuda.synchronize()
        st = out["status"].cpu().numpy()
        np.testing.assert_array_equal(st, ref["status"].cpu().numpy())
        good = np.flatnonzero(st == _lib.QP_SOLVED)
        bad = np.flatnonzero(st == _lib.QP_BAD_INPUT)
        assert len(good) + len(bad) == B
        assert (len(bad) == 0) if data is first else (bad.tolist() == [5])
        for k in OUT_KEYS[:4] + GRAD_KEYS:
            a = out[k].cpu().numpy()[good]
            r = ref[k].cpu().numpy()[good]
            np.testing.assert_allclose(a, r, rtol=0, atol=1e-6, err_msg=k)
        for k in GRAD_KEYS:
            assert np.all(np.isnan(out[k].cpu().numpy()[bad])), k
            assert np.all(np.isnan(ref[k].cpu().numpy()[bad])), k


def test_oversized_batch_refused_without_side_effects():
    from paper_2605_17913_gb300 import _lib
    from paper_2605_17913_gb300.solver import QPSolver

    B, n, p, m = 1024, 50, 10, 100
    slv = QPSolver(B, n, p, m)
    assert slv.grad_cache_bytes > _lib.QP_STATIC_CACHE_BYTES
    T = {k: torch.zeros(shape, device="cuda") for k, shape in
         dict(Q=(B, n, n), q=(B, n), A=(B, p, n), b=(B, p), G=(B, m, n), h=(B, m),
              g=(B, n)).items()}
    out = _outputs(B, n, p, m, fill=7.0)
    rc = _static_call(slv, T, out, _lib.default_settings())
    assert rc == _lib.QP_ENOTSUP
    torch.cuda.synchronize()
    assert torch.all(out["x"] == 7.0) and torch.all(out["dQ"] == 7.0)
    assert torch.all(out["status"] == -9)
