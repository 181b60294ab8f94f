"""Planted mistakes in the FP64 projector oracle (`oracle/siddon_oracle.c`).

Each mutant is a copy of the oracle's C source with one plausible error (a
wrong sign, a swapped operand, a wrong index, a dropped bound or term),
compiled on the CPU into a library of its own.  The oracle's pins
(`test_oracle_pins.py`) then run against it in a child process, and at
least one must fail.  An unmodified copy run the same way passes every pin,
so the failures come from the planted mistakes and not from the harness.
Mutants that cannot change a result (scaling lengths by |u| when u is a
unit vector, say) are not planted."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "siddon_oracle.c")

# (what the mistake is, text in the source, text it is replaced by); each
# text occurs exactly once
MUTANTS = [
    ("roll turns the other way",
     "f1[a] = cr * e1[a] + sr * e2[a];", "f1[a] = cr * e1[a] - sr * e2[a];"),
    ("image axes swapped in the direction",
     "dir[a] = w[a] + tu * f1[a] + tv * f2[a];",
     "dir[a] = w[a] + tu * f2[a] + tv * f1[a];"),
    ("column angle measured from the row reference pixel",
     "tan((iu - p[C_CRPIX_U])", "tan((iu - p[C_CRPIX_V])"),
    ("observer mirrored through the equator",
     "o[2] = d * sin(lat);", "o[2] = -d * sin(lat);"),
    ("ray integrated behind the observer too",
     "double lo = 0.0, hi = INFINITY;", "double lo = -INFINITY, hi = INFINITY;"),
    ("voxel taken at the segment start, not its midpoint",
     "double mid = 0.5 * (merged[q] + merged[q + 1]);",
     "double mid = merged[q];"),
    ("half-open voxels closed on the other side",
     "i[a] = (int32_t)floor(x);", "i[a] = (int32_t)ceil(x) - 1;"),
    ("crossings merged in descending order",
     "(best < 0 || lists[a][h[a]] < lists[best][h[best]]))",
     "(best < 0 || lists[a][h[a]] > lists[best][h[best]]))"),
    ("rays lying in a lower face dropped",
     "if (o[a] < p0 || o[a] >= p1) return 0;",
     "if (o[a] <= p0 || o[a] >= p1) return 0;"),
    ("interpolation weights swapped in P",
     "v = (1.0 - w) * cube[(int64_t)k * nvox + idx[q]] +\n"
     "                        w * cube[(int64_t)(k + 1) * nvox + idx[q]];",
     "v = w * cube[(int64_t)k * nvox + idx[q]] +\n"
     "                        (1.0 - w) * cube[(int64_t)(k + 1) * nvox + idx[q]];"),
    ("gain dropped in the transpose",
     "double yk = p[C_GAIN] * images[id];", "double yk = images[id];"),
    ("mask ignored in the transpose",
     "if (mask && mask[id]) continue;\n            double yk",
     "double yk"),
    ("interpolation weights swapped in the transpose",
     "double a0 = (1.0 - w) * len[q] * yk, a1 = w * len[q] * yk;",
     "double a0 = w * len[q] * yk, a1 = (1.0 - w) * len[q] * yk;"),
    ("last segment dropped (the exit not merged)",
     "merged[m++] = amax;\n", "\n"),
    ("entry and exit not ordered by the direction's sign",
     "lo = fmax(lo, fmin(a0, a1));\n        hi = fmin(hi, fmax(a0, a1));",
     "lo = fmax(lo, a0);\n        hi = fmin(hi, a1);"),
    ("pixel angles without the gnomonic tangent",
     "double tu = tan((iu - p[C_CRPIX_U]) * p[C_CDELT_U] + p[C_CRVAL_U]);",
     "double tu = (iu - p[C_CRPIX_U]) * p[C_CDELT_U] + p[C_CRVAL_U];"),
    ("sphere entered at its far root",
     "double first = -ou - sqrt(disc);", "double first = -ou + sqrt(disc);"),
    ("observer inside the sphere not blocked",
     "if (oo <= r2) return 0; /* observer inside the sphere */", ""),
    ("crossing weights keep the lengths",
     "if (crossing_weights) len[q] = 1.0;", ""),
    ("crossing weights of signed values",
     "if (crossing_weights) yk = fabs(yk);", ""),
    ("impact parameter taken as the observer distance",
     "cross3(o, u, c);", "c[0] = o[0]; c[1] = o[1]; c[2] = o[2];"),
    ("segment count includes masked rays",
     "if (mask && mask[id]) continue;\n            double o[3], u[3];\n"
     "            if (orc_ray(",
     "double o[3], u[3];\n            if (orc_ray("),
]

# Run in a child process: point the oracle at the given library, then call
# every pin with each of its parameter sets until one raises.  Prints
# "READY" once the pins are imported, then "FAIL <pin>" or "PASS".
RUNNER = r"""
import inspect, itertools, os, sys
sys.path.insert(0, sys.argv[2])
import oracle.siddon as siddon
siddon._build.build = lambda force=False: sys.argv[1]
siddon._lib = None
import tests.test_oracle_pins as pins
golden = os.path.join(sys.argv[2], "tests", "golden")
skip = ("test_thomson_voxel_factors_pin_catches_planted_mistakes",)
calls = []
for name, fn in inspect.getmembers(pins, inspect.isfunction):
    if not name.startswith("test_") or name in skip:
        continue
    sets = [{}]
    for m in getattr(fn, "pytestmark", []):
        if m.name != "parametrize":
            continue
        names, values = m.args[0], m.args[1]
        names = [s.strip() for s in names.split(",")] if isinstance(names, str) else list(names)
        new = []
        for kw in sets:
            for v in values:
                v = v if len(names) > 1 else (v,)
                new.append(dict(kw, **dict(zip(names, v))))
        sets = new
    for kw in sets:
        if "golden_dir" in inspect.signature(fn).parameters:
            kw = dict(kw, golden_dir=golden)
        calls.append((name, fn, kw))
print("READY", len(calls), flush=True)
for name, fn, kw in calls:
    try:
        fn(**kw)
    except Exception as e:
        print("FAIL", name, type(e).__name__, flush=True)
        sys.exit(0)
print("PASS", flush=True)
"""


def _compile(source, out_dir):
    c_path = os.path.join(out_dir, "oracle_variant.c")
    so_path = os.path.join(out_dir, "liboracle_variant.so")
    with open(c_path, "w") as f:
        f.write(source)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
                           "-o", so_path, c_path, "-lm"])
    return so_path


def _run_pins(so_path):
    env = dict(os.environ, OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-c", RUNNER, so_path, ROOT],
                       cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    lines = r.stdout.split()
    assert r.returncode == 0 and "READY" in lines, r.stdout + r.stderr
    return r.stdout.strip().splitlines()[-1]


def _source():
    with open(SRC) as f:
        return f.read()


def test_unmodified_copy_passes_every_pin(tmp_path):
    assert _run_pins(_compile(_source(), str(tmp_path))) == "PASS"


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(what, old, new, tmp_path):
    src = _source()
    assert src.count(old) == 1, what
    result = _run_pins(_compile(src.replace(old, new), str(tmp_path)))
    assert result.startswith("FAIL"), "%s: no pin fails" % what
