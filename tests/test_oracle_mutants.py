"""Mistakes planted in the FP64 oracle must fail its pins.

Each mutant below is a copy of ``oracle/qp_oracle.c`` with one plausible slip
-- a dropped term, a wrong sign, a swapped operand or index, a wrong divisor
-- in the retraction (eq. 11, App. C), the residuals (eq. 4), the Newton
system (eq. 13 / eq. 14), Alg. 1, Alg. 2, Alg. 3 or the standard form
(eq. 6 / eq. 8).  The copy is compiled apart, the pins (tests/test_oracle_pins.py
and the oracle half of tests/test_golden.py) run against it in a child
process, and at least one pin must fail.  The unmodified source, built and
checked the same way, must pass: the harness itself is sound.

Several slips move only the path of the iteration and leave the solution,
the relaxed point and the gradients where they were: in the implicit method
the iterate is re-retracted from v and kappa after every step, so a wrong
right-hand side or a wrong dz / ds costs iterations, not accuracy.  The pin on
a single direction (Newton's step for the linearised eq. 4 and eq. 11)
catches those.  The centring heuristic itself (Mehrotra's exponent, the
standard form's second-order corrector term) decides only how fast the
iteration gets there; no output fixes it, so it is not planted here.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "qp_oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_golden.py"]

# (label, text in qp_oracle.c, replacement, which occurrence; None = must be unique)
MUTANTS = [
    # retraction and its derivatives (eq. 11, eq. 12, App. C)
    ("b_k, v < 0: wrong sign in the cancellation-free form",
     "return 2.0 * kappa / (r - v);", "return 2.0 * kappa / (r + v);", None),
    ("b_k, v >= 0: the 1/2 dropped",
     "if (v >= 0.0) return 0.5 * (v + r);", "if (v >= 0.0) return (v + r);", None),
    ("d/dv b_k, v >= 0: wrong sign",
     "if (v >= 0.0) return 0.5 * (1.0 + v / r);", "if (v >= 0.0) return 0.5 * (1.0 - v / r);",
     None),
    ("d/dv b_k, v < 0: the 4 kappa term dropped",
     "return 2.0 * kappa / (v * v + 4.0 * kappa - v * r);",
     "return 2.0 * kappa / (v * v - v * r);", None),
    ("d/dkappa b_k: a factor 1/2 too many",
     "return 1.0 / sqrt(v * v + 4.0 * kappa); }", "return 0.5 / sqrt(v * v + 4.0 * kappa); }",
     None),
    # residuals (eq. 4)
    ("r_t without A'y", "R->rt[i] = a + P->q[i] + c + d;", "R->rt[i] = a + P->q[i] + c;", None),
    ("r_t with -G'z", "R->rt[i] = a + P->q[i] + c + d;", "R->rt[i] = a + P->q[i] - c + d;",
     None),
    ("r_i with -s", "R->ri[k] = a + s[k] - P->h[k];", "R->ri[k] = a - s[k] - P->h[k];", None),
    ("r_e with +b", "R->re[k] = a - P->b[k];", "R->re[k] = a + P->b[k];", None),
    ("unscaled KKT measure without z.*s",
     "if (!scaled) return fmax(fmax(fmax(et, ee), fmax(ei, ec)), ezs);",
     "if (!scaled) return fmax(fmax(fmax(et, ee), ei), ezs);", None),
    ("scaled KKT measure without z.*s",
     "return fmax(fmax(fmax(et / dt, ee / de), fmax(ei / di, ec)), ezs / dz);",
     "return fmax(fmax(fmax(et / dt, ee / de), ei / di), ezs / dz);", None),
    # the implicit Newton system (eq. 13, eq. 14)
    ("eq. 14 without the -G'G term",
     "M[IX(i, j, N)] = P->Q[IX(i, j, n)] - gg;", "M[IX(i, j, N)] = P->Q[IX(i, j, n)];", None),
    ("eq. 14 with B_k(v) in place of B_k(-v)",
     "M[IX(n + k, n + k, N)] = -W->Bm[k];", "M[IX(n + k, n + k, N)] = -W->Bp[k];", None),
    ("eq. 14 without the A' block",
     "M[IX(j, n + m + k, N)] = P->A[IX(k, j, n)];", "(void)0;", None),
    ("eq. 14 right-hand side: +G'(...)",
     "r[i] = -(rt[i] - g);", "r[i] = -(rt[i] + g);", None),
    ("eq. 14 right-hand side: wrong sign of c r_kappa",
     "r[n + k] = -(ri[k] - rs[k] - W->c[k] * rkappa);",
     "r[n + k] = -(ri[k] - rs[k] + W->c[k] * rkappa);", None),
    ("eq. 13: dz without the c dkappa term",
     "dz[k] = -rz[k] + W->Bp[k] * dv[k] + W->c[k] * (*dkappa);",
     "dz[k] = -rz[k] + W->Bp[k] * dv[k];", None),
    ("eq. 13: ds with +B_k(-v) dv",
     "ds[k] = -rs[k] - W->Bm[k] * dv[k] + W->c[k] * (*dkappa);",
     "ds[k] = -rs[k] + W->Bm[k] * dv[k] + W->c[k] * (*dkappa);", None),
    ("dense solve without the row permutation",
     "if (piv[k] != k) { double t = r[k];", "if (0) { double t = r[k];", None),
    # Alg. 1
    ("eq. 7 step length ignoring dz",
     "    if (dz[k] < 0.0) a = fmin(a, -z[k] / dz[k]);\n", "", None),
    # Alg. 2
    ("Alg. 2: kappa averaged over m + p rows", "kappa /= (double)m;",
     "kappa /= (double)(m + p);", 2),
    ("Alg. 2: Newton toward the wrong kappa", "kappa - kappa_relax, w.dx",
     "kappa_relax - kappa, w.dx", None),
    # Alg. 3
    ("Alg. 3: adjoint right-hand side +g", "for (int i = 0; i < n; ++i) r[i] = -g[i];",
     "for (int i = 0; i < n; ++i) r[i] = g[i];", None),
    ("Alg. 3: factor at v = s - z", "for (int k = 0; k < m; ++k) w.v[k] = z[k] - s[k];",
     "for (int k = 0; k < m; ++k) w.v[k] = s[k] - z[k];", None),
    ("Alg. 3: dz = B_k(-v) dv", "dzv[k] = w.W.Bp[k] * r[n + k];",
     "dzv[k] = w.W.Bm[k] * r[n + k];", None),
    ("Alg. 3: dy read from the dv block", "dy[k] = r[n + m + k];", "dy[k] = r[n + k];", 1),
    ("Alg. 3: dQ not symmetrised",
     "dQ[IX(i, j, n)] = 0.5 * (dx[i] * x[j] + x[i] * dx[j]);",
     "dQ[IX(i, j, n)] = dx[i] * x[j];", None),
    ("Alg. 3: dA without y dx'", "dA[IX(k, j, n)] = dy[k] * x[j] + y[k] * dx[j];",
     "dA[IX(k, j, n)] = dy[k] * x[j];", None),
    ("Alg. 3: db = +dy", "db[k] = -dy[k];", "db[k] = dy[k];", None),
    ("Alg. 3: dG with s for z", "dG[IX(k, j, n)] = dzv[k] * x[j] + z[k] * dx[j];",
     "dG[IX(k, j, n)] = dzv[k] * x[j] + s[k] * dx[j];", None),
    ("Alg. 3: dh = +dz", "dh[k] = -dzv[k];", "dh[k] = dzv[k];", None),
    # standard form (eq. 6 / eq. 8)
    ("eq. 8 with D(z./s) for D(s./z)",
     "M[IX(n + p + k, n + p + k, N)] = -s[k] / z[k];",
     "M[IX(n + p + k, n + p + k, N)] = -z[k] / s[k];", None),
    ("eq. 6: ds with the wrong sign of s dz",
     "dsp[k] = -(rc[k] + s[k] * dzp[k]) / z[k];", "dsp[k] = -(rc[k] - s[k] * dzp[k]) / z[k];",
     None),
    ("eq. 8 right-hand side: +r_c ./ z",
     "r[n + p + k] = -(w.R.ri[k] - rc[k] / z[k]);", "r[n + p + k] = -(w.R.ri[k] + rc[k] / z[k]);",
     None),
    ("standard form: no fraction to the boundary",
     "double alpha = fmin(1.0, 0.99 * step_length(m, s, z, w.ds, w.dz));",
     "double alpha = step_length(m, s, z, w.ds, w.dz);", None),
]


def _mutate(src: str, old: str, new: str, occurrence) -> str:
    count = src.count(old)
    if occurrence is None:
        assert count == 1, f"expected one occurrence of {old!r}, found {count}"
        return src.replace(old, new)
    assert count > occurrence, f"{old!r} occurs {count} times"
    at = -1
    for _ in range(occurrence + 1):
        at = src.index(old, at + 1)
    return src[:at] + new + src[at + len(old):]


def _build(src: str, where: str) -> str:
    c, so = os.path.join(where, "qp_oracle.c"), os.path.join(where, "liboracle.so")
    with open(c, "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", so,
                    c, "-lm", "-lpthread"], check=True, capture_output=True)
    return so


def _run_pins(so: str) -> subprocess.CompletedProcess:
    env = dict(os.environ, QP_ORACLE_LIB=so)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           "-m", "not gpu", *PINS], cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=600)


def _first_failure(out: str) -> str:
    for line in out.splitlines():
        if line.startswith("FAILED") or line.startswith("ERROR"):
            return line
    return out.strip().splitlines()[-1] if out.strip() else ""


def test_mutants_fail_the_pins(tmp_path):
    with open(SRC) as f:
        src = f.read()
    jobs = {"(unmodified)": src}
    for label, old, new, occ in MUTANTS:
        jobs[label] = _mutate(src, old, new, occ)

    def run(item):
        i, (label, text) = item
        where = tmp_path / f"m{i:02d}"
        where.mkdir()
        return label, _run_pins(_build(text, str(where)))

    workers = max(1, min(8, (os.cpu_count() or 2)))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = dict(ex.map(run, enumerate(jobs.items())))
    control = results.pop("(unmodified)")
    assert control.returncode == 0, control.stdout[-2000:] + control.stderr[-2000:]
    survivors = [label for label, r in results.items() if r.returncode == 0]
    assert not survivors, f"mistakes no pin caught: {survivors}"
    for label, r in results.items():
        # a failing pin, not a crash of the child process
        assert r.returncode == 1, (label, r.returncode, r.stderr[-1000:])
