"""The seeded generators: determinism, shapes and the structure each workload promises."""
import numpy as np

from qpgen import CONFIGS, make_batch, make_instance, serving_sizes


def test_instance_independent_of_batch():
    b = make_batch("small", 5, seed=3, start=2, dtype=np.float64)
    d = make_instance("small", 4, seed=3)
    np.testing.assert_array_equal(b.Q[2], d["Q"])
    np.testing.assert_array_equal(b.G[2], d["G"])


def test_shapes_and_symmetry():
    for name, cfg in CONFIGS.items():
        if name == "precision":
            continue  # large; covered by the cond test below with a small n
        b = make_batch(name, 3)
        assert b.Q.shape == (3, cfg["n"], cfg["n"]) and b.Q.dtype == np.float32
        assert b.G.shape == (3, cfg["m"], cfg["n"]) and b.A.shape == (3, cfg["p"], cfg["n"])
        np.testing.assert_array_equal(b.Q, np.swapaxes(b.Q, 1, 2))
        assert np.all(np.linalg.eigvalsh(b.Q.astype(np.float64)) > 0)


def test_x0_feasible_and_degenerate_activity():
    d = make_instance("small", 0)
    assert np.all(d["G"] @ d["x0"] < d["h"])
    np.testing.assert_allclose(d["A"] @ d["x0"], d["b"], atol=1e-12)
    d = make_instance("degenerate", 0)
    slack = d["h"] - d["G"] @ d["x0"]
    assert np.count_nonzero(np.abs(slack) < 1e-12) == 50
    assert np.all(slack > -1e-12)


def test_precision_condition_number():
    d = make_instance("precision", 0, n=32, m=64, p=4)
    ev = np.linalg.eigvalsh(d["Q"])
    np.testing.assert_allclose(ev.max() / ev.min(), 1e4, rtol=1e-8)


def test_serving_sizes_range():
    sz = serving_sizes(2000, seed=1)
    ns = np.array([s[0] for s in sz])
    assert ns.min() >= 8 and ns.max() <= 256
    assert all(m == 2 * n and p == n // 10 for n, m, p, _ in sz)
    frac = np.mean([s[3] for s in sz])
    assert 0.25 < frac < 0.35
    assert np.median(ns) < 64  # log-uniform mix is weighted to small n


def test_empty_batch():
    b = make_batch("small", 0)
    assert b.Q.shape == (0, 10, 10)


def test_safety_filter_structure():
    from qpgen.workloads import safety_size

    for k in (1, 2, 7, 9):
        n, m, p = safety_size(k)
        assert (n, m, p) == (2 * k, 4 * k + 3 * k + k * (k - 1) // 2, 0)
        d = make_instance("safety", 3, seed=1, agents=k)
        G, h = d["G"], d["h"]
        np.testing.assert_array_equal(d["Q"], np.eye(n))
        assert G.shape == (m, n) and d["A"].shape == (0, n)
        assert np.all(h > 0)  # u = 0 strictly feasible (safe state, positive gains)
        # box rows: +e_c and -e_c with bound u_max = 2
        for c in range(n):
            np.testing.assert_array_equal(G[2 * c], np.eye(n)[c])
            np.testing.assert_array_equal(G[2 * c + 1], -np.eye(n)[c])
        np.testing.assert_array_equal(h[:4 * k], 2.0)
        # obstacle rows touch one agent's two controls
        obs = G[4 * k:7 * k]
        for r, row in enumerate(obs):
            nz = np.flatnonzero(row)
            assert len(nz) == 2 and nz[0] == 2 * (r // 3) and nz[1] == nz[0] + 1
        # pair rows: opposite gradients on the two agents' blocks
        pair = G[7 * k:]
        rr = 0
        for i in range(k):
            for j in range(i + 1, k):
                row = pair[rr]
                np.testing.assert_array_equal(row[2 * i:2 * i + 2], -row[2 * j:2 * j + 2])
                assert np.count_nonzero(row) == 4
                rr += 1
    # the nominal control has length 3 (goal-seeking gain) unless within 0.1 of the goal
    d = make_instance("safety", 0, seed=0)
    speeds = np.linalg.norm(-d["q"].reshape(-1, 2), axis=1)
    assert np.all(speeds <= 3.0 + 1e-12) and np.median(speeds) > 2.0
