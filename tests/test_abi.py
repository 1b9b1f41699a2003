"""The C ABI library loads and exports every function include/qp.h declares;
host-side argument validation works without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(qp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g

    g.build()
    from paper_2605_17913_gb300 import _lib

    return _lib.lib()


def test_header_declares_api():
    names = _declared_functions()
    for required in ("qp_handle_create", "qp_handle_destroy", "qp_solve_batch",
                     "qp_backward_batch", "qp_grad_cache_bytes", "qp_settings_default",
                     "qp_status_string", "qp_smem_bytes"):
        assert required in names, names


def test_library_exports_every_declared_symbol(L):
    for name in _declared_functions():
        assert hasattr(L, name), f"{name} declared in include/ but not exported"


def test_settings_defaults(L):
    from paper_2605_17913_gb300 import _lib

    s = _lib.default_settings()
    assert abs(s.tol - 1e-5) < 1e-12 and s.max_iter == 100
    assert abs(s.kappa_relax - 1e-4) < 1e-10 and s.formulation == 0


def test_host_validation_without_gpu(L):
    from paper_2605_17913_gb300 import _lib

    h = ctypes.c_void_p()
    bad = [(-1, 4, 0, 2), (1, 0, 0, 2), (1, 3, 4, 2), (1, 3, 0, -1)]
    for d in bad:
        dims = _lib.Dims(*d)
        assert L.qp_handle_create(ctypes.byref(dims), ctypes.byref(h)) == _lib.QP_EINVAL
        assert L.qp_grad_cache_bytes(ctypes.byref(dims)) == 0
    assert L.qp_handle_create(None, ctypes.byref(h)) == _lib.QP_EINVAL
    assert L.qp_solve_batch(None, None, *([None] * 15)) == _lib.QP_EINVAL
    assert L.qp_backward_batch(*([None] * 13)) == _lib.QP_EINVAL
    assert L.qp_handle_destroy(None) == _lib.QP_EINVAL


def test_sizes(L):
    from paper_2605_17913_gb300 import _lib

    assert _lib.smem_bytes(50, 10, 100) > 0
    assert _lib.smem_bytes(100, 20, 200) > 0
    assert _lib.smem_bytes(300, 10, 10) == 0  # beyond the shared-memory kernel
    assert _lib.smem_bytes(4, 5, 2) == 0  # n_eq > n
    dims = _lib.Dims(3, 10, 2, 20)
    # padded blocks: header, L (55), Y (12 x 10: amax = min(m, n) = 10 plus p = 2 rows),
    # L_C (78), W, row map, x, y, z
    per = (4 + 56 + 120 + 80 + 20 + 20 + 12 + 4 + 20 + 20) * 4
    assert L.qp_grad_cache_bytes(ctypes.byref(dims)) == 3 * per
    for c in (0, 1, 2, 3, 4, -1, -6):
        assert isinstance(_lib.status_string(c), str)


def test_serve_footprint_and_config_validation(L):
    from paper_2605_17913_gb300 import _lib

    f0 = L.qp_serve_footprint_bytes(50, 5, 100, 0)
    f1 = L.qp_serve_footprint_bytes(50, 5, 100, 1)
    assert 0 < f0 < f1 and f0 % 256 == 0
    # data + outputs at least, gradients and the factor cache on top
    assert f0 >= 4 * (50 * 50 + 50 + 5 * 50 + 5 + 100 * 50 + 100)
    assert f1 - f0 >= 4 * (50 * 50 + 100 * 50)
    assert L.qp_serve_footprint_bytes(300, 5, 10, 0) == 0  # beyond n = 256
    assert L.qp_serve_footprint_bytes(10, 11, 5, 0) == 0  # n_eq > n
    cfg = _lib.ServeConfig()
    L.qp_serve_config_default(ctypes.byref(cfg))
    assert cfg.hbm_budget_bytes == 1 << 30 and cfg.max_inflight == 8
    assert cfg.mode == _lib.QP_SERVE_PERSISTENT and cfg.idle_ms == 50
    h = ctypes.c_void_p()
    # bad modes and idle limits are refused before any device call
    for mode, idle in ((2, 50), (-1, 50), (_lib.QP_SERVE_PERSISTENT, 0),
                       (_lib.QP_SERVE_PERSISTENT, 10001)):
        cfg.mode, cfg.idle_ms = mode, idle
        assert L.qp_serve_create(ctypes.byref(cfg), ctypes.byref(h)) == _lib.QP_EINVAL
    cfg.mode, cfg.idle_ms = _lib.QP_SERVE_LAUNCHES, 50
    cfg.max_inflight = 0
    assert L.qp_serve_create(ctypes.byref(cfg), ctypes.byref(h)) == _lib.QP_EINVAL
    assert L.qp_serve_submit(None, None, None) == _lib.QP_EINVAL
    assert L.qp_serve_poll_any(None, None) == _lib.QP_EINVAL
    assert L.qp_handle_query(None, None) == _lib.QP_EINVAL
    # forced widths that cannot run are refused before any device call
    h2 = ctypes.c_void_p()
    for tpq, dims in ((64, (8, 10, 0, 20)), (32, (8, 40, 0, 20)), (128, (8, 100, 0, 20))):
        d = _lib.Dims(*dims)
        assert L.qp_handle_create_threads(ctypes.byref(d), tpq, ctypes.byref(h2)) == _lib.QP_ENOTSUP


def test_no_fallback_when_the_library_is_missing(monkeypatch, tmp_path):
    """Without libqpgpu.so every call raises: there is no CPU path."""
    from paper_2605_17913_gb300 import _lib

    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libqpgpu.so"))
    with pytest.raises(_lib.QPError, match="not built"):
        _lib.lib()


def test_solver_takes_device_tensors_only(L):
    """Host tensors are refused by the device-array API rather than solved on
    the CPU; without a GPU, creating a solver fails with the CUDA error."""
    import torch

    from paper_2605_17913_gb300 import _lib
    from paper_2605_17913_gb300.solver import QPSolver

    s = QPSolver.__new__(QPSolver)
    with pytest.raises(_lib.QPError, match="CUDA tensor"):
        s._check("Q", torch.zeros(2, 3, 3), (2, 3, 3))
    if not torch.cuda.is_available():
        with pytest.raises(_lib.QPError, match="QP_ECUDA"):
            QPSolver(2, 3, 0, 2)
