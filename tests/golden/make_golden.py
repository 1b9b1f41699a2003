"""Write the closed-form fixtures of tests/golden/ (FP64, plain numpy).

Nothing here runs the oracle or the CUDA path: every value is a closed form
derived by hand from the problem statement (eq. 1), the relaxed
complementarity z_i s_i = kappa of Alg. 2 (the central path, eq. 10) and the
retraction of App. C, b_k(w) = (w + sqrt(w^2 + 4 kappa)) / 2.  The tests
compare both the FP64 oracle and the GPU path with these numbers.

central_path_separable.json -- n independent 1-D problems stacked:
    minimise 1/2 |x|^2 + q'x  subject to  x <= u     (Q = I, G = I, h = u, no A)
  Relaxed point: with w = u + q, stationarity x + q + z = 0 and z s = kappa
  give s = b_k(w), z = b_k(-w), x = u - s (then x + q + z = w - (s - z) = 0).
  Sensitivities, from differentiating those three equations (l = g'x,
  beta_i = b_k'(w_i) = s_i / (s_i + z_i)):
    dl/dq_i  = -g_i beta_i                      dl/du_i = g_i (1 - beta_i)
    dl/dG_ij = -g_j z_i beta_j - g_i z_i x_j / (s_i + z_i)   (perturbing G_ij
               adds z_i to stationarity row j and x_j to slack row i)
    dl/dQ    : along the symmetric direction e_i e_j' + e_j e_i' the change of
               l is -g_i beta_i x_j - g_j beta_j x_i; the gradient with respect
               to a symmetric Q stores half of it in each of (i, j), (j, i)
               (the diagonal: -g_i beta_i x_i).
equality_projection.json -- minimise 1/2 |x|^2 + q'x subject to a'x = beta:
    y = -(beta + a'q) / |a|^2,  x = -q - a y,
    dl/dq = -(g - a (a'g) / |a|^2),  dl/dbeta = a'g / |a|^2,
    dl/da_k = -y g_k + (a'g / |a|^2) q_k + 2 y (a'g / |a|^2) a_k
  (the last by differentiating x(a) = -q + a (beta + a'q) / |a|^2 directly).

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _b(w, kappa):
    # both signs accurately: b(w) b(-w) = kappa, b(w) - b(-w) = w
    r = np.sqrt(w * w + 4.0 * kappa)
    return np.where(w >= 0, (w + r) / 2.0, 2.0 * kappa / (r - w))


def central_path_separable(kappa: float, seed: int) -> dict:
    rng = np.random.default_rng(seed)
    w = np.array([-3.0, -1.0, -0.3, -0.01, 0.01, 0.3, 1.0, 3.0])
    n = w.size
    q = rng.standard_normal(n)
    u = w - q
    g = rng.standard_normal(n)
    s, z = _b(w, kappa), _b(-w, kappa)
    x = u - s
    beta = s / (s + z)
    dq = -g * beta
    dh = g * (1.0 - beta)
    dG = -np.outer(z, g * beta) - np.outer(g * z / (s + z), x)
    dQ = -0.5 * (np.outer(g * beta, x) + np.outer(x, g * beta))
    return {
        "source": "closed form of the relaxed KKT point z*s = kappa (eq. 1, eq. 10, App. C "
                  "retraction) and its sensitivities, derived by hand; see make_golden.py",
        "n": n, "n_eq": 0, "n_ineq": n, "kappa_relax": kappa,
        "Q": np.eye(n).tolist(), "q": q.tolist(), "G": np.eye(n).tolist(), "h": u.tolist(),
        "A": [], "b": [], "g": g.tolist(),
        "x_relaxed": x.tolist(), "s_relaxed": s.tolist(), "z_relaxed": z.tolist(),
        "x_optimum": np.minimum(-q, u).tolist(),
        "dQ": dQ.tolist(), "dq": dq.tolist(), "dG": dG.tolist(), "dh": dh.tolist(),
    }


def equality_projection(seed: int) -> dict:
    rng = np.random.default_rng(seed)
    n = 6
    a = rng.standard_normal(n)
    q = rng.standard_normal(n)
    beta = float(rng.standard_normal())
    g = rng.standard_normal(n)
    aa = a @ a
    y = -(beta + a @ q) / aa
    x = -q - a * y
    ag = (a @ g) / aa
    dq = -(g - a * ag)
    db = ag
    da = -y * g + ag * q + 2.0 * y * ag * a
    return {
        "source": "closed form of min 1/2|x|^2 + q'x s.t. a'x = beta (eq. 1 with one "
                  "equality, no inequality) and its derivatives, derived by hand; see "
                  "make_golden.py",
        "n": n, "n_eq": 1, "n_ineq": 0,
        "Q": np.eye(n).tolist(), "q": q.tolist(), "A": [a.tolist()], "b": [beta],
        "G": [], "h": [], "g": g.tolist(),
        "x": x.tolist(), "y": [y],
        "dq": dq.tolist(), "dA": [da.tolist()], "db": [db],
    }


def fixtures() -> dict:
    return {
        "central_path_separable.json": {
            "cases": [central_path_separable(1e-2, 11), central_path_separable(1e-4, 12)]},
        "equality_projection.json": {"cases": [equality_projection(21), equality_projection(22)]},
    }


def dumps(content: dict) -> str:
    """One line per field: readable text, exact float round trip."""
    cases = []
    for case in content["cases"]:
        rows = [f" {json.dumps(k)}: {json.dumps(v)}" for k, v in case.items()]
        cases.append("{\n" + ",\n".join(rows) + "\n}")
    return '{"cases": [\n' + ",\n".join(cases) + "\n]}\n"


def main() -> None:
    for name, content in fixtures().items():
        with open(os.path.join(HERE, name), "w") as f:
            f.write(dumps(content))


if __name__ == "__main__":
    main()
