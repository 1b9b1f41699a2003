"""Serving (qp_serve_*): continuous batching of single requests of uneven
sizes.  Each served result must equal the same request solved alone
(qp_solve_batch / qp_backward_batch of batch 1) bit for bit and meet the
FP64 oracle's bars (x, KKT, every gradient block); requests that arrive
while others run must start and finish without waiting for them; admission
must respect the device arena; a wait that runs out, a client that stops
collecting and a request whose Q is not positive definite must leave every
other request untouched."""
import time

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2605_17913_gb300.metrics import kkt_report, rel_err_2, rel_err_inf
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


def _solo(d, grad, threads=0):
    """The request solved alone: a batch-1 qp_solve_batch (forward width
    `threads`, 0 = the size's default) and qp_backward_batch."""
    from paper_2605_17913_gb300.solver import QPSolver

    n, p, m = d["q"].size, d["b"].size, d["h"].size
    T = {k: torch.from_numpy(d[k].reshape((1,) + d[k].shape)).cuda() for k in
         ("Q", "q", "A", "b", "G", "h", "g")}
    slv = QPSolver(1, n, p, m, threads_per_qp=threads)
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


# every kernel class: one warp / 128 / 512 threads on chip, the large variant;
# with and without gradients
SIZES = [(8, 16, 0, False), (10, 20, 1, True), (33, 66, 3, True), (50, 100, 5, False),
         (72, 144, 7, True), (90, 180, 9, False), (90, 180, 9, True), (130, 260, 13, True),
         (200, 400, 20, False), (200, 400, 20, True), (256, 512, 25, True)]


MODES = ["launches", "persistent"]
# the forward width a served request runs at: the size's default in launches,
# 512 for every size in the persistent loop
SOLO_THREADS = {"launches": 0, "persistent": 512}


@pytest.fixture(scope="module", params=MODES)
def served(request):
    from paper_2605_17913_gb300.serve import QPServer

    inst = [_inst(i, n, m, p) for i, (n, m, p, _) in enumerate(SIZES)]
    srv = QPServer(hbm_budget_bytes=512 << 20, tol=SOLVER_TOL, mode=request.param)
    try:
        tickets = [_submit(srv, d, g) for d, (_, _, _, g) in zip(inst, SIZES)]
        got = [srv.wait(t, 120000) for t in tickets]
    finally:
        srv.close()
    return inst, got, request.param


def test_served_results_match_oracle(served):
    """Every served result against the FP64 oracle at the method's bars:
    scaled KKT <= 1e-5, x <= 1e-4, and (requests with gradients) every
    gradient block <= 1e-3 at the relaxed point."""
    inst, got, _ = served
    for d, (n, m, p, grad), r in zip(inst, SIZES, got):
        assert r["status"] == 0, (n, r["status"])
        one = lambda k: d[k][None]  # noqa: E731
        ref = O.solve(one("Q"), one("q"), one("A"), one("b"), one("G"), one("h"), tol=1e-12,
                      kappa_relax=1e-4 if grad else None, g=one("g") if grad else None)
        rep = kkt_report(one("Q"), one("q"), one("A"), one("b"), one("G"), one("h"),
                         r["x"][None], r["y"][None], r["z"][None], r["s"][None])
        assert rep["scaled"][0] <= 1e-5, (n, rep["scaled"][0])
        assert rel_err_inf(r["x"][None], ref["x"])[0] <= 1e-4, n
        if grad:
            for k in GRAD_KEYS:
                if ref[k].size:
                    e = rel_err_2(r[k][None], ref[k])[0]
                    assert e <= 1e-3, (n, k, e)


def test_served_results_equal_solo_bitwise(served):
    inst, got, mode = served
    for d, (n, m, p, grad), r in zip(inst, SIZES, got):
        ref = _solo(d, grad, SOLO_THREADS[mode])
        assert r["status"] == 0 and ref["status"] == 0, (n, r["status"])
        assert r["iters"] == ref["iters"]
        for k in ("x", "y", "z", "s") + (GRAD_KEYS if grad else ()):
            np.testing.assert_array_equal(r[k], ref[k], err_msg=f"{k} at n={n}")


@pytest.mark.parametrize("mode", MODES)
def test_requests_arriving_later_start_while_others_run(mode):
    from paper_2605_17913_gb300.serve import QPServer

    big = [_inst(100 + i, 256, 512, 25) for i in range(8)]
    small = [_inst(200 + i, 10, 20, 1) for i in range(24)]
    srv = QPServer(hbm_budget_bytes=512 << 20, max_inflight=4, tol=SOLVER_TOL, mode=mode)
    try:
        tb = [_submit(srv, d, True) for d in big]
        # the large requests take ~20 ms on the GPU: the small ones arrive
        # well within that
        time.sleep(0.003)
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


@pytest.mark.parametrize("mode", MODES)
def test_admission_by_arena_memory(mode):
    from paper_2605_17913_gb300 import _lib
    from paper_2605_17913_gb300.serve import QPServer, footprint_bytes

    budget = 16 << 20
    n, m, p = 150, 300, 15
    each = footprint_bytes(n, p, m, True)
    count = 40
    assert count * each > 2 * budget  # needs several rounds of admission
    srv = QPServer(hbm_budget_bytes=budget, max_inflight=2, tol=SOLVER_TOL, mode=mode)
    try:
        inst = [_inst(300 + i, n, m, p) for i in range(count)]
        tickets = [_submit(srv, d, True) for d in inst]
        got = [srv.wait(t, 300000) for t in tickets]
    finally:
        srv.close()
    assert all(r["status"] == 0 for r in got)
    # a request larger than the whole arena is refused at submit
    tiny = QPServer(hbm_budget_bytes=1 << 20, tol=SOLVER_TOL, mode=mode)
    try:
        assert each > 1 << 20
        with pytest.raises(_lib.QPError, match="QP_ENOTSUP"):
            _submit(tiny, inst[0], True)
    finally:
        tiny.close()
    ref = _solo(inst[7], True, SOLO_THREADS[mode])
    for k in ("x",) + GRAD_KEYS:
        np.testing.assert_array_equal(got[7][k], ref[k])


@pytest.mark.parametrize("mode", MODES)
def test_wait_times_out_and_the_request_survives(mode):
    """qp_serve_wait returns QP_ETIMEOUT when its bound runs out before the
    request completes; the request is still collected afterwards, intact."""
    from paper_2605_17913_gb300.serve import QPServer

    d = _inst(400, 256, 512, 25)
    srv = QPServer(hbm_budget_bytes=256 << 20, tol=SOLVER_TOL, mode=mode)
    try:
        t = _submit(srv, d, True)
        with pytest.raises(Exception, match="not done after 0 ms"):
            srv.wait(t, 0)
        r = srv.wait(t, 120000)
    finally:
        srv.close()
    assert r["status"] == 0
    ref = _solo(d, True, SOLO_THREADS[mode])
    for k in ("x",) + GRAD_KEYS:
        np.testing.assert_array_equal(r[k], ref[k])


@pytest.mark.parametrize("mode", MODES)
def test_client_that_stops_collecting_does_not_block_others(mode):
    """Requests a client never collects stay completed on the host side;
    another client's requests, submitted after them, run and are collected
    as usual (results bit for bit those of solo runs)."""
    from paper_2605_17913_gb300.serve import QPServer

    idle = [_inst(500 + i, 40, 80, 4) for i in range(24)]
    busy = [_inst(600 + i, 40, 80, 4) for i in range(24)]
    srv = QPServer(hbm_budget_bytes=64 << 20, max_inflight=2, tol=SOLVER_TOL, mode=mode)
    try:
        for d in idle:
            _submit(srv, d, True)  # never collected
        tb = [_submit(srv, d, i % 2 == 0) for i, d in enumerate(busy)]
        rb = [srv.wait(t, 120000) for t in tb]
    finally:
        srv.close()  # drops the uncollected tickets
    assert all(r["status"] == 0 for r in rb)
    for i in (0, 1, 23):
        ref = _solo(busy[i], i % 2 == 0, SOLO_THREADS[mode])
        for k in ("x", "z") + (GRAD_KEYS if i % 2 == 0 else ()):
            np.testing.assert_array_equal(rb[i][k], ref[k])


@pytest.mark.parametrize("mode", MODES)
def test_non_positive_definite_request_is_isolated(mode):
    """A request whose Q is not positive definite (K = Q + G'G indefinite at
    the start) ends QP_NUMERICAL; the requests around it, in the same
    launches, are solved exactly as alone."""
    from paper_2605_17913_gb300 import _lib
    from paper_2605_17913_gb300.serve import QPServer

    good = [_inst(700 + i, 10, 20, 1) for i in range(6)]
    bad = dict(_inst(710, 10, 20, 1))
    bad["Q"] = (-10.0 * np.eye(10)).astype(np.float32)
    srv = QPServer(hbm_budget_bytes=64 << 20, max_inflight=1, tol=SOLVER_TOL, mode=mode)
    try:
        tg = [_submit(srv, d, True) for d in good[:3]]
        tbad = _submit(srv, bad, True)
        tg += [_submit(srv, d, True) for d in good[3:]]
        rg = [srv.wait(t, 60000) for t in tg]
        rbad = srv.wait(tbad, 60000)
    finally:
        srv.close()
    assert rbad["status"] == _lib.QP_NUMERICAL
    for d, r in zip(good, rg):
        assert r["status"] == 0
        ref = _solo(d, True, SOLO_THREADS[mode])
        for k in ("x", "y", "z", "s") + GRAD_KEYS:
            np.testing.assert_array_equal(r[k], ref[k])


def test_persistent_ctas_leave_when_idle_and_come_back():
    """Resident CTAs that find no request for idle_ms leave their loop; a
    request submitted afterwards starts new ones and is solved as alone."""
    from paper_2605_17913_gb300.serve import QPServer

    a, b = _inst(800, 40, 80, 4), _inst(801, 150, 300, 15)
    srv = QPServer(hbm_budget_bytes=64 << 20, tol=SOLVER_TOL, mode="persistent", idle_ms=5)
    try:
        ra = srv.wait(_submit(srv, a, True), 60000)
        time.sleep(0.2)  # every CTA has left by now
        rb = srv.wait(_submit(srv, b, True), 60000)
    finally:
        srv.close()
    for d, r in ((a, ra), (b, rb)):
        assert r["status"] == 0
        ref = _solo(d, True, 512)
        for k in ("x", "y", "z", "s") + GRAD_KEYS:
            np.testing.assert_array_equal(r[k], ref[k])


def test_persistent_server_tensor_core_gwg():
    """Resident CTAs with TF32 G'WG on the tensor cores (TMEM held for the
    CTA's life): large requests equal batch-1 solves of width 512 with the
    same setting bit for bit, and meet the oracle's bars."""
    from paper_2605_17913_gb300.serve import QPServer
    from paper_2605_17913_gb300.solver import QPSolver

    inst = [_inst(900 + i, 200, 400, 20) for i in range(2)]
    srv = QPServer(hbm_budget_bytes=256 << 20, tol=SOLVER_TOL, mode="persistent",
                   gwg_precision="tf32")
    try:
        got = [srv.wait(_submit(srv, d, True), 60000) for d in inst]
    finally:
        srv.close()
    for d, r in zip(inst, got):
        assert r["status"] == 0
        n, p, m = d["q"].size, d["b"].size, d["h"].size
        T = {k: torch.from_numpy(d[k].reshape((1,) + d[k].shape)).cuda() for k in
             ("Q", "q", "A", "b", "G", "h", "g")}
        slv = QPSolver(1, n, p, m, threads_per_qp=512)
        cache = slv.new_grad_cache()
        out = slv.solve(T["Q"], T["q"], T["A"], T["b"], T["G"], T["h"], grad_cache=cache,
                        tol=SOLVER_TOL, gwg_precision="tf32")
        g = slv.backward(cache, T["Q"], T["A"], T["G"], T["g"])
        torch.cuda.synchronize()
        ref = {k: v.cpu().numpy()[0] for k, v in list(out.items()) + list(g.items())}
        for k in ("x", "y", "z", "s") + GRAD_KEYS:
            np.testing.assert_array_equal(r[k], ref[k], err_msg=k)
        one = lambda k: d[k][None]  # noqa: E731
        orc = O.solve(one("Q"), one("q"), one("A"), one("b"), one("G"), one("h"), tol=1e-12,
                      kappa_relax=1e-4, g=one("g"))
        assert rel_err_inf(r["x"][None], orc["x"])[0] <= 1e-4
        for k in GRAD_KEYS:
            if orc[k].size:
                assert rel_err_2(r[k][None], orc[k])[0] <= 1e-3, k
