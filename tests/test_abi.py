"""The C ABI library builds, loads, and exports every function include/pencil.h
declares; argument checks that run before any CUDA call work without a GPU."""
import ctypes
import subprocess

import pytest

import paper_1302_5586_gb300 as pg
from paper_1302_5586_gb300 import build as pg_build


@pytest.fixture(scope="module")
def lib():
    pg_build.build()
    return pg.lib()


def test_every_declared_symbol_is_exported(lib):
    names = pg.declared_symbols()
    assert "pencil_conv2d" in names and "pencil_jacobi2d" in names
    out = subprocess.run(["nm", "-D", "--defined-only", pg.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_header_compiles_as_c99_and_cxx(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "pencil.h"\nint main(void) { return pencil_version() > 0 ? 0 : 1; }\n')
    inc = "-I" + pg.HEADER.rsplit("/", 1)[0]
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-pedantic", inc, "-c", str(src), "-o",
                    str(tmp_path / "a.o")], check=True)
    subprocess.run(["g++", "-x", "c++", "-std=c++17", "-Wall", "-Werror", inc, "-c", str(src), "-o",
                    str(tmp_path / "b.o")], check=True)


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "pencil.h"

int main(int argc, char **argv)
{
    (void)argv;
    const int h0 = argc - 1; /* 0 at run time, unknown to the compiler */
    if (pencil_version() < 100) return 10;
    if (strcmp(pencil_strerror(PENCIL_OK), "ok") != 0) return 11;
    pencil_arena *a = NULL;
    if (pencil_arena_create(4096, 256, &a) != PENCIL_OK || !a) return 12;
    size_t x = 1, y = 1;
    if (pencil_arena_alloc(a, 1, &x) != PENCIL_OK || x != 0) return 13;
    if (pencil_arena_alloc(a, 300, &y) != PENCIL_OK || y != 256) return 14;
    if (pencil_arena_free_bytes(a) != 4096 - 768) return 15;
    if (pencil_arena_alloc(a, 4096, &x) != PENCIL_ERR_NOMEM) return 16;
    if (pencil_arena_free(a, 256) != PENCIL_OK || pencil_arena_free(a, 0) != PENCIL_OK) return 17;
    if (pencil_arena_largest_free(a) != 4096) return 18;
    pencil_arena_destroy(a);
    /* const inputs: C before C2X converts no T[n][m] to const T (*)[m] */
    static const float img[4][4], k[3][3];
    float out[4][4];
    if (pencil_conv2d(4, h0, img, 3, 3, k, out) != PENCIL_ERR_ARG) return 19;
    if (pencil_jacobi2d_workspace_size(100, 100) == 0) return 20;
    printf("c client ok\n");
    return 0;
}
"""


def test_a_c_program_links_and_calls_the_library(lib, tmp_path):
    """The boundary from C itself: a C99 program includes pencil.h, links the
    built library and runs its host-only calls (version, status text, the
    arena, an argument check, a workspace size)."""
    import os
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    libdir = os.path.dirname(pg.LIB_PATH)
    exe = str(tmp_path / "client")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-pedantic", "-I" + os.path.dirname(pg.HEADER),
                    str(src), "-o", exe, "-L" + libdir, "-l:" + os.path.basename(pg.LIB_PATH),
                    "-Wl,-rpath," + libdir], check=True, capture_output=True, text=True)
    p = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert p.returncode == 0 and p.stdout.strip() == "c client ok", (p.returncode, p.stdout, p.stderr)


def test_utility_calls(lib):
    assert pg.pencil_version() >= 100
    assert pg.pencil_strerror(0) == "ok"
    assert "restrict" in pg.pencil_strerror(-3)
    assert pg.pencil_strerror(-99) == "unknown status"


@pytest.mark.parametrize("args,status", [
    ((0, 5, 1, 3, 3, 1, 2), -1),       # h <= 0
    ((5, 5, 1, 0, 3, 1, 2), -1),       # kh <= 0
    ((5, 5, None, 3, 3, 1, 2), -2),    # null input
    ((5, 5, 4096, 3, 3, 1, 4096 + 40), -3),  # out overlaps in
])
def test_conv2d_argument_errors_before_cuda(lib, args, status):
    h, w, i, kh, kw, k, o = args
    assert lib.pencil_conv2d(h, w, i, kh, kw, k, o) == status


def test_ex_argument_errors_before_cuda(lib):
    assert lib.pencil_conv2d_ex(1, 4, 4, 1, 3, 3, 2, 3, 7, 0, None) == -1   # bad dtype
    assert lib.pencil_conv2d_ex(1, 4, 4, 1, 3, 3, 2, 3, 0, 8, None) == -1   # unknown flag
    assert lib.pencil_conv2d_ex(1, 4, 4, 1, 3, 3, 2, 3, 0, 32, None) == -1  # unknown flag
    # interleaved rows of w*c elements must fit an int
    assert lib.pencil_conv2d_ex(3, 1, 1 << 30, 1, 3, 3, 2, 3, 0, pg.PENCIL_LAYOUT_HWC, None) == -8
    assert lib.pencil_conv2d_sep_ex(3, 1, 1 << 30, 1, 3, 2, 3, 3, 5, 0, pg.PENCIL_LAYOUT_HWC, None) == -8
    assert lib.pencil_conv2d_ex(3, 1, 1 << 30, 1, 3, 3, 2, 3, 0, 0, None) != -8  # planar rows are not limited
    assert lib.pencil_conv2d_sep_ex(1, 4, 4, 1, 17, 2, 3, 3, 5, 0, 0, None) == -8  # side > 15
    assert lib.pencil_conv2d_ex(1, 4, 4, 1, 3, 3, 2, 3, 0, 5 << 8, None) == -1   # border mode 5
    assert lib.pencil_conv2d_sep_ex(1, 4, 4, 1, 3, 2, 3, 3, 5, 0, 1, None) == -1  # generic flag not allowed
    assert lib.pencil_conv2d_sep(4, 4, 1, 3, 2, 16, 3, 5) == -8
    assert lib.pencil_jacobi2d_ex(4, 4, 1, -1, 0, None, 256, 1 << 20, 0, None) == -1
    assert lib.pencil_jacobi2d_ex(4, 4, 1, 10, 5, None, 256, 1 << 20, 0, None) == -2  # no res_out
    assert lib.pencil_jacobi2d_ex(64, 64, 1, 10, 0, None, 256, 16, 0, None) == -5     # workspace small
    assert lib.pencil_jacobi2d(3, 3, None, 1) == -2
    ws = pg.pencil_jacobi2d_workspace_size(8192, 8192)
    assert ws >= 8192 * 8192 * 4 and ws % 256 == 0
    assert pg.pencil_jacobi2d_workspace_size(0, 5) == 0
    # CUDA grid limits: rows and channels beyond them are refused up front
    tall = pg.PENCIL_MAX_ROWS + 1
    assert lib.pencil_conv2d_ex(1, tall, 4, 1, 3, 3, 2, 3, 0, 0, None) == -8
    assert lib.pencil_conv2d_ex(pg.PENCIL_MAX_CHANNELS + 1, 4, 4, 1, 3, 3, 2, 3, 0, 0, None) == -8
    assert lib.pencil_conv2d_sep_ex(pg.PENCIL_MAX_CHANNELS + 1, 4, 4, 1, 3, 2, 3, 3, 5, 0, 0, None) == -8
    assert lib.pencil_jacobi2d_ex(tall, 4, 1, 10, 0, None, 256, 1 << 40, 0, None) == -8
    assert lib.pencil_rbsor2d_ex(tall, 4, 1, 10, 1.5, 0, None, 256, 1 << 40, None) == -8
    assert lib.pencil_conv2d(tall, 4, 1, 3, 3, 2, 3) == -8
    # conv -> Jacobi: sweeps < 0, unknown flags, NULL arrays, rows beyond the grid limit
    assert lib.pencil_conv2d_jacobi(1, 8, 8, 1, 3, 3, 2, -1, 3, 0, None) == -1
    assert lib.pencil_conv2d_jacobi(1, 8, 8, 1, 3, 3, 2, 5, 3, 1, None) == -1
    assert lib.pencil_conv2d_jacobi(1, 8, 8, None, 3, 3, 2, 5, 3, 0, None) == -2
    assert lib.pencil_conv2d_jacobi(1, tall, 8, 1, 3, 3, 2, 5, 3, 0, None) == -8


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    import paper_1302_5586_gb300._binding as b
    monkeypatch.setattr(b, "_lib", None)
    monkeypatch.setattr(b, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        b.lib()


def test_batch_argument_errors_before_cuda(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.pencil_batch_create(7, 10, 100, ctypes.byref(h)) == -1      # bad dtype
    assert lib.pencil_batch_create(0, 0, 100, ctypes.byref(h)) == -1      # no images
    assert lib.pencil_batch_create(0, 10, 0, ctypes.byref(h)) == -1       # no tiles
    assert lib.pencil_batch_create(0, 10, 10, None) == -2
    assert lib.pencil_batch_set_variant(None, 3, 0) == -2
    assert lib.pencil_batch_run(None, 1, None, None) == -2
    assert lib.pencil_batch_destroy(None) == 0


def test_binding_constants_match_the_header():
    import re
    text = open(pg.HEADER).read()
    for name in ("PENCIL_MAX_ROWS", "PENCIL_MAX_CHANNELS", "PENCIL_CHAIN_FUSED", "PENCIL_CONV_GENERIC",
                 "PENCIL_LAYOUT_HWC",
                 "PENCIL_OP2_ORDERED", "PENCIL_OP2_ATOMIC", "PENCIL_F32", "PENCIL_F16"):
        m = re.search(r"#define\s+%s\s+(\d+)" % name, text) or re.search(r"\b%s\s*=\s*(\d+)" % name, text)
        assert m, name
        assert getattr(pg, name) == int(m.group(1)), name


def test_status_and_tune_argument_errors_before_cuda(lib):
    done = ctypes.c_int(-1)
    assert lib.pencil_selftest_wait_timeout(0, ctypes.byref(done)) == -1        # limit below 1 us
    assert lib.pencil_selftest_wait_timeout(2000000, ctypes.byref(done)) == -1  # above 1 s
    assert lib.pencil_selftest_wait_timeout(1000, None) == -2
    chosen = (ctypes.c_int * 8)()
    assert lib.pencil_tune(None, 0, None, 1, None, chosen) == -2
    imgs = pg.make_images([(0x1000, 0x2000, 0x3000, 8, 8, 3)])
    assert lib.pencil_tune(None, 1, imgs, 1, None, chosen) == -2


def test_residual_alias_checks_before_cuda(lib):
    """The residual's workspace and result may not overlap the grid or each
    other (checked on the addresses alone, before any CUDA call)."""
    ws = pg.pencil_jacobi2d_workspace_size(4, 4)
    u, res, wsp = 1 << 20, 2 << 20, 3 << 20          # disjoint, 256-byte aligned
    assert lib.pencil_residual2d(4, 4, u, u + 8, wsp, ws, None) == -3       # result inside the grid
    assert lib.pencil_residual2d(4, 4, u, res, u, ws, None) == -3           # workspace over the grid
    assert lib.pencil_residual2d(4, 4, u, wsp + 16, wsp, ws, None) == -3    # result inside the workspace
    assert lib.pencil_residual2d(4, 4, u, res, wsp + 8, ws, None) == -1     # workspace not 256-aligned
    assert lib.pencil_residual2d(4, 4, u, res, wsp, ws - 1, None) == -5     # workspace too small
