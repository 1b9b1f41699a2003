"""Serving (qp_serve_*): continuous batching of single requests of uneven
sizes.  Each served result must equal the same request solved alone
(qp_solve_batch / qp_backward_batch of batch 1) bit for bit; requests that
arrive while others run must start and finish without waiting for them;
admission must respect the device arena."""
import time

import numpy as np
import pytest
import torch

from qpgen import make_instance

pytestmark = pytest.mark.gpu

SOLVER_TOL = 5e-6
GRAD_KEYS = ("dQ", "dq", "dA", "db", "dG", "dh")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g

    g.build()
    torch.cuda.set_device(0)


def _inst(i, n, m, p, seed=3):
    d = make_instance("small", i, seed=seed, n=n, m=m, p=p)
    return {k: np.asarray(v, dtype=np.float32) for k, v in d.items()}


def _solo(d, grad):
    from paper_2605_17913_gb300.solver import QPSolver

    n, p, m = d["q"].size, d["b"].size, d["h"].size
    T = {k: torch.from_numpy(d[k].reshape((1,) + d[k].shape)).cuda() for k in
         ("Q", "q", "A", "b", "G", "h", "g")}
    slv = QPSolver(1, n, p, m)
    cache = slv.new_grad_cache() if grad else None
    out = slv.solve(T["Q"], T["q"], T["A"], T["b"], T["G"], T["h"], grad_cache=cache,
                    tol=SOLVER_TOL)
    res = {k: v.cpu().numpy()[0] for k, v in out.items()}
    if grad:
        g = slv.backward(cache, T["Q"], T["A"], T["G"], T["g"])
        res.update({k: v.cpu().numpy()[0] for k, v in g.items()})
    torch.cuda.synchronize()
    return res


def _submit(srv, d, grad):
    return srv.submit(d["Q"], d["q"], d["A"], d["b"], d["G"], d["h"],
                      dl_dx=d["g"] if grad else None)


def test_served_results_equal_solo_bitwise():
    from paper_2605_17913_gb300.serve import QPServer

    sizes = [(8, 16, 0, False), (10, 20, 1, True), (33, 66, 3, True), (50, 100, 5, False),
             (72, 144, 7, True), (90, 180, 9, False), (130, 260, 13, True),
             (200, 400, 20, False), (256, 512, 25, True)]
    inst = [_inst(i, n, m, p) for i, (n, m, p, _) in enumerate(sizes)]
    srv = QPServer(hbm_budget_bytes=512 << 20, tol=SOLVER_TOL)
    try:
        tickets = [_submit(srv, d, g) for d, (_, _, _, g) in zip(inst, sizes)]
        got = [srv.wait(t, 120000) for t in tickets]
    finally:
        srv.close()
    for d, (n, m, p, grad), r in zip(inst, sizes, got):
        ref = _solo(d, grad)
        assert r["status"] == 0 and ref["status"] == 0, (n, r["status"])
        assert r["iters"] == ref["iters"]
        for k in ("x", "y", "z", "s") + (GRAD_KEYS if grad else ()):
            np.testing.assert_array_equal(r[k], ref[k], err_msg=f"{k} at n={n}")


def test_requests_arriving_later_start_while_others_run():
    from paper_2605_17913_gb300.serve import QPServer

    big = [_inst(100 + i, 256, 512, 25) for i in range(4)]
    small = [_inst(200 + i, 10, 20, 1) for i in range(24)]
    srv = QPServer(hbm_budget_bytes=512 << 20, max_inflight=4, tol=SOLVER_TOL)
    try:
        tb = [_submit(srv, d, True) for d in big]
        time.sleep(0.02)
        ts = [_submit(srv, d, i % 3 == 0) for i, d in enumerate(small)]
        rs = [srv.wait(t, 120000) for t in ts]
        rb = [srv.wait(t, 120000) for t in tb]
    finally:
        srv.close()
    assert all(r["status"] == 0 for r in rs + rb)
    # the small requests arrived after the large ones, were launched while
    # those were still on the GPU, and most came back before them
    big_done = min(r["t_done_ms"] for r in rb)
    assert min(r["t_submit_ms"] for r in rs) > max(r["t_submit_ms"] for r in rb)
    assert min(r["t_launch_ms"] for r in rs) < big_done
    assert sum(r["t_done_ms"] < big_done for r in rs) >= 18


def test_admission_by_arena_memory():
    from paper_2605_17913_gb300 import _lib
    from paper_2605_17913_gb300.serve import QPServer, footprint_bytes

    budget = 16 << 20
    n, m, p = 150, 300, 15
    each = footprint_bytes(n, p, m, True)
    count = 40
    assert count * each > 2 * budget  # needs several rounds of admission
    srv = QPServer(hbm_budget_bytes=budget, max_inflight=2, tol=SOLVER_TOL)
    try:
        inst = [_inst(300 + i, n, m, p) for i in range(count)]
        tickets = [_submit(srv, d, True) for d in inst]
        got = [srv.wait(t, 300000) for t in tickets]
    finally:
        srv.close()
    assert all(r["status"] == 0 for r in got)
    # a request larger than the whole arena is refused at submit
    tiny = QPServer(hbm_budget_bytes=1 << 20, tol=SOLVER_TOL)
    try:
        assert each > 1 << 20
        with pytest.raises(_lib.QPError, match="QP_ENOTSUP"):
            _submit(tiny, inst[0], True)
    finally:
        tiny.close()
    ref = _solo(inst[7], True)
    for k in ("x",) + GRAD_KEYS:
        np.testing.assert_array_equal(got[7][k], ref[k])
