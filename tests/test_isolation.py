"""The library and the oracle share no code: no source of either imports,
includes or links the other, importing the library loads no part of the
oracle, and the seeded input generators (the one module both sides use)
import neither."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1302_5586_gb300")
ORACLE = os.path.join(ROOT, "oracle")
SYNTH = os.path.join(ROOT, "synth")
SRC_EXT = (".py", ".cu", ".cuh", ".cpp", ".c", ".h")


def sources(top):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith(SRC_EXT):
                yield os.path.join(d, f)


def code_lines(path):
    """Import / include / load lines of a source file (comments and
    docstrings may name the other side; code may not use it)."""
    pat = re.compile(r"^\s*(import\s|from\s\S+\s+import\s|#\s*include\s)|CDLL\(|dlopen\(|ctypes\.cdll")
    with open(path, encoding="utf-8") as f:
        return [ln for ln in f if pat.search(ln)]


def test_library_sources_do_not_use_the_oracle():
    bad = [(p, ln.strip()) for p in sources(PKG) for ln in code_lines(p) if "oracle" in ln]
    assert not bad, bad


def test_oracle_sources_do_not_use_the_library():
    names = ("paper_1302_5586_gb300", "pencil", "csrc", "libpencilgpu", "synth")
    bad = [(p, ln.strip()) for p in sources(ORACLE) for ln in code_lines(p) if any(n in ln for n in names)]
    assert not bad, bad


def test_input_generators_import_neither_side():
    bad = [(p, ln.strip()) for p in sources(SYNTH) for ln in code_lines(p)
           if "oracle" in ln or "paper_1302_5586_gb300" in ln or "pencil" in ln]
    assert not bad, bad


def test_importing_the_library_loads_no_oracle():
    code = ("import sys, paper_1302_5586_gb300 as pg; "
            "assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules), 'oracle imported'; "
            "maps = open('/proc/self/maps').read() if sys.platform.startswith('linux') else ''; "
            "assert 'liboracle' not in maps, 'oracle library mapped'; print('ok')")
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0 and p.stdout.strip() == "ok", p.stderr[-800:]
