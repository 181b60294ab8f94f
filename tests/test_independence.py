"""The oracle and the CUDA path share no code, and the product path never
reaches the oracle.

No file of the package (Python binding, CUDA sources) or of the C-ABI
headers names the oracle; no oracle file names the package, its CUDA
sources, its library or its header; the seeded input generators (`synth/`),
which both sides use, import neither.  Only the tests, the smoke check and
the benchmark's CPU legs import the oracle.  Without its compiled library
the binding raises instead of computing anything another way."""

import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PACKAGE = "paper_1103_5904_gb300"
SOURCES = (".py", ".c", ".cc", ".cpp", ".cu", ".cuh", ".h")


def _files(*dirs):
    for d in dirs:
        for base, subdirs, names in os.walk(os.path.join(ROOT, d)):
            subdirs[:] = [s for s in subdirs
                          if s not in ("_build", "__pycache__")]
            for n in names:
                if n.endswith(SOURCES):
                    yield os.path.join(base, n)


def _text(path):
    with open(path, encoding="utf-8", errors="replace") as f:
        return f.read()


def test_product_code_never_names_the_oracle():
    pat = re.compile(r"\boracle\b")
    hits = [os.path.relpath(p, ROOT) for p in _files(PACKAGE, "include")
            if pat.search(_text(p))]
    assert not hits, hits


def test_oracle_never_names_the_product():
    pat = re.compile(r"%s|csrc|libtomo|tomo\.h|tomo_internal" % PACKAGE)
    hits = [os.path.relpath(p, ROOT) for p in _files("oracle")
            if pat.search(_text(p))]
    assert not hits, hits


def test_input_generators_import_neither_side():
    pat = re.compile(r"^\s*(from|import)\s+(oracle|%s)\b" % PACKAGE, re.M)
    hits = [os.path.relpath(p, ROOT) for p in _files("synth")
            if pat.search(_text(p))]
    assert not hits, hits


def test_binding_fails_loudly_without_its_library():
    code = ("import %s.tomo as t; "
            "t.load_library('/nonexistent/libtomo.so')" % PACKAGE)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "libtomo.so not found" in r.stderr
