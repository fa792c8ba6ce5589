"""Planted mistakes in the oracle must fail its pins.

Each mutant is a copy of oracle/oracle.c with one plausible slip: a flipped
filter, a wrong anchor, a transposed or dropped index, a lost term, a wrong
sign, a wrong rounding, a wrong sweep order or border rule.  The copy is built
and the oracle's pin tests (the test_oracle_*.py files, which compare it with
library routines, closed forms, invariants, hand-worked fixtures and brute
force) run against it in a child process, with ORACLE_SRC naming the copy.
Every mutant must make at least one pin fail, and the unmutated copy must pass
them all, so the pins are shown to pin the oracle, not only to agree with it.

Every mutation keeps each memory access of the oracle in bounds; mutants that
compute the same result as the original (e.g. dropping the carry when a
binary16 significand rounds up to 2048, which the bit layout performs anyway)
are not listed.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

TESTS = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(TESTS)
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PINS = ["test_oracle_conv2d.py", "test_oracle_f16.py", "test_oracle_jacobi.py", "test_oracle_op2.py"]

# (name, text in oracle.c, replacement); the first occurrence is replaced
MUTANTS = [
    # conv2d
    ("filter flipped (convolution, not correlation)",
     "const double wt = k[a * kw + bb];", "const double wt = k[(kh - 1 - a) * kw + (kw - 1 - bb)];"),
    ("anchor (k-1)/2 instead of k/2 for even sides",
     "const int ah = kh / 2, aw = kw / 2;", "const int ah = (kh - 1) / 2, aw = (kw - 1) / 2;"),
    ("row and column swapped in the pixel index",
     "load_px(in, dtype, base + r * w + c)", "load_px(in, dtype, base + c * h + r)"),
    ("clamp-to-edge replaced by zero padding",
     "default: return clamp64(i, 0, n - 1);", "default: return -1;"),
    ("last filter column dropped",
     "for (int bb = 0; bb < kw; ++bb) {", "for (int bb = 0; bb + 1 < kw; ++bb) {"),
    ("bound takes the signed weight",
     "b += fabs(wt) * fabs(x);", "b += wt * fabs(x);"),
    ("channel plane offset missing the row count",
     "const int64_t base = ch * h * w;", "const int64_t base = ch * w;"),
    ("reflect period 2n-1",
     "int64_t p = 2 * n, j = ((i % p) + p) % p;", "int64_t p = 2 * n - 1, j = ((i % p) + p) % p;"),
    ("mirror repeats the edge",
     "return j < n ? j : p - j;", "return j < n ? j : p - 1 - j;"),
    ("wrap leaves negative indices negative (read as zero)",
     "case 4: return ((i % n) + n) % n;", "case 4: return i % n;"),
    ("separable outer product transposed",
     "conv_planes(nc, h, w, in, dtype, ky, kx, kd, out, bound, 0);",
     "conv_planes(nc, h, w, in, dtype, kx, ky, kd, out, bound, 0);"),
    ("sampled points read as (ch, j, i)",
     "const int64_t ch = pts[3 * p], i = pts[3 * p + 1], j = pts[3 * p + 2];",
     "const int64_t ch = pts[3 * p], j = pts[3 * p + 1], i = pts[3 * p + 2];"),
    ("separable sampled points with the filter sides swapped",
     "conv_pixel(h, w, in, dtype, ch * h * w, ky, kx, kd,", "conv_pixel(h, w, in, dtype, ch * h * w, kx, ky, kd,"),
    ("interleaved pixels read without the channel stride",
     "load_px(in, dtype, (r * w + c) * nc + ch)", "load_px(in, dtype, (r * w + c) + ch)"),
    ("interleaved rows read with the planar pitch",
     "load_px(in, dtype, (r * w + c) * nc + ch)", "load_px(in, dtype, r * w + c * nc + ch)"),
    ("interleaved result written to the planar position",
     "const int64_t o = (i * w + j) * nc + ch;", "const int64_t o = (ch * h + i) * w + j;"),
    ("binary16 pixels read as raw integers",
     "return oracle_f16_to_f64(((const uint16_t *)in)[idx]);", "return (double)((const uint16_t *)in)[idx];"),
    # binary16 codec
    ("subnormal decode scale 2^-25",
     "v = ldexp((double)f, -24);", "v = ldexp((double)f, -25);"),
    ("exponent bias off by one",
     "v = ldexp((double)(1024 + f), e - 25);", "v = ldexp((double)(1024 + f), e - 24);"),
    ("decode drops the sign",
     "return sign ? -v : v;", "return v;"),
    ("encode truncates",
     "double q = rint(ldexp(a, 10 - e));", "double q = floor(ldexp(a, 10 - e));"),
    ("encode rounds ties away from zero",
     "double q = rint(ldexp(a, 10 - e));", "double q = round(ldexp(a, 10 - e));"),
    ("overflow to infinity one binade late",
     "if (e > 15) return", "if (e > 16) return"),
    ("subnormal encode scale 2^23",
     "double q = rint(ldexp(a, 24));", "double q = rint(ldexp(a, 23));"),
    # Jacobi and residual
    ("left neighbour counted twice",
     "v[p] = (u[p - w] + u[p + w] + u[p - 1] + u[p + 1]) / 4.0;",
     "v[p] = (u[p - w] + u[p + w] + u[p - 1] + u[p - 1]) / 4.0;"),
    ("average divided by 5",
     "v[p] = (u[p - w] + u[p + w] + u[p - 1] + u[p + 1]) / 4.0;",
     "v[p] = (u[p - w] + u[p + w] + u[p - 1] + u[p + 1]) / 5.0;"),
    ("sweep updates in place (Gauss-Seidel order)",
     "jacobi_sweep(h, w, cur, nxt);\n        double *t = cur; cur = nxt; nxt = t;",
     "jacobi_sweep(h, w, cur, cur);"),
    ("right boundary column updated",
     "if (i == 0 || j == 0 || i == h - 1 || j == w - 1)", "if (i == 0 || j == 0 || i == h - 1)"),
    ("residual adds the upper neighbour",
     "const double r = 4.0 * u[i * w + j] - u[(i - 1) * w + j]",
     "const double r = 4.0 * u[i * w + j] + u[(i - 1) * w + j]"),
    ("residual without the square root",
     "return sqrt(acc);", "return acc;"),
    ("FP32 residual centre weight 3",
     "const double r = 4.0 * (double)u[i * w + j]", "const double r = 3.0 * (double)u[i * w + j]"),
    ("residual taken of the previous iterate",
     "res[s / check_every - 1] = oracle_residual2d_f64(h, w, cur);",
     "res[s / check_every - 1] = oracle_residual2d_f64(h, w, nxt);"),
    ("residual sums the last column too",
     "for (int64_t j = 1; j + 1 < w; ++j) {\n            const double r = 4.0 * u[i * w + j]",
     "for (int64_t j = 1; j < w; ++j) {\n            const double r = 4.0 * u[i * w + j]"),
    # red-black SOR
    ("odd points swept first",
     "if (((i + j) & 1) != color) continue;", "if (((i + j) & 1) == color) continue;"),
    ("relaxation weights swapped",
     "u[p] = u[p] + omega * (avg - u[p]);", "u[p] = (1.0 - omega) * avg + omega * u[p];"),
    # edge-to-cell increment
    ("first cell decremented",
     "cell[c0] += edge[i];", "cell[c0] -= edge[i];"),
    ("both increments to one cell",
     "const int32_t c1 = e2c[2 * i + 1], c0 = e2c[2 * i];", "const int32_t c1 = e2c[2 * i], c0 = e2c[2 * i];"),
]


def _mutate(src, old, new):
    assert old in src, f"mutation target not in oracle.c: {old!r}"
    return src.replace(old, new, 1)


def _run_pins(path):
    """Run the pin tests against the oracle built from `path`; (exit code, summary line)."""
    env = dict(os.environ, ORACLE_SRC=path, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    cmd += [os.path.join(TESTS, f) for f in PINS]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    lines = [ln for ln in p.stdout.strip().splitlines() if ln.strip()]
    return p.returncode, (lines[-1] if lines else p.stderr[-400:])


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    with open(SRC) as f:
        src = f.read()
    jobs = [("original", src)] + [(name, _mutate(src, old, new)) for name, old, new in MUTANTS]
    paths = []
    for i, (name, text) in enumerate(jobs):
        d = tmp_path_factory.mktemp(f"mutant{i}")
        path = os.path.join(str(d), "oracle.c")
        with open(path, "w") as f:
            f.write(text)
        # a mutant that does not compile would "fail" its pins for the wrong reason
        subprocess.run(["gcc", "-std=c11", "-fsyntax-only", path], check=True, capture_output=True)
        paths.append(path)
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        results = list(ex.map(_run_pins, paths))
    return {name: r for (name, _), r in zip(jobs, results)}


def test_names_are_unique():
    assert len({m[0] for m in MUTANTS}) == len(MUTANTS)


def test_unmutated_copy_passes_the_pins(outcomes):
    rc, summary = outcomes["original"]
    assert rc == 0, summary


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_mutant_fails_a_pin(outcomes, name):
    rc, summary = outcomes[name]
    assert rc == 1 and "failed" in summary, f"mutant survived or broke the run: {name}: {summary}"
