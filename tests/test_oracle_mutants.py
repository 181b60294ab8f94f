"""Planted mistakes in the FP64 oracle: the C projector
(`oracle/siddon_oracle.c`), the prior and CG (`oracle/solver.py`) and the
Thomson operators (`oracle/thomson.py`).

Each mutant is a copy of one source with one plausible error (a wrong sign,
a swapped operand, a wrong index, a dropped bound, factor or term): a C copy
is compiled on the CPU into a library of its own, a Python copy is loaded
in place of the oracle's module.  The oracle's pins (`test_oracle_pins.py`)
then run against it in a child process, and at least one must fail.  An
unmodified copy run the same way passes every pin, so the failures come
from the planted mistakes and not from the harness.  Mutants that cannot
change a result (scaling lengths by |u| when u is a unit vector, say) are
not planted."""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "siddon_oracle.c")
SOLVER = os.path.join(ROOT, "oracle", "solver.py")
THOMSON = os.path.join(ROOT, "oracle", "thomson.py")

# (what the mistake is, text in the source, text it is replaced by); each
# text occurs exactly once, and no mutant can index outside its arrays
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
    ("longitude measured from the y axis",
     "o[0] = d * cos(lat) * cos(lon);\n    o[1] = d * cos(lat) * sin(lon);",
     "o[0] = d * cos(lat) * sin(lon);\n    o[1] = d * cos(lat) * cos(lon);"),
    ("first image axis reversed", "cross3(w, zhat, e1);", "cross3(zhat, w, e1);"),
    ("second image axis reversed", "cross3(e1, w, e2);", "cross3(w, e1, e2);"),
    ("first image axis not normalised", "for (int a = 0; a < 3; ++a) e1[a] /= n1;",
     ""),
    ("direction not normalised", "u[a] = dir[a] / nd;", "u[a] = dir[a];"),
    ("interpolation weight measured from the next frame",
     "*w = tau - kk;", "*w = kk + 1 - tau;"),
    ("gain dropped in P", "out[r] = p[C_GAIN] * acc;", "out[r] = acc;"),
    ("impact parameter without its z term",
     "c[0] * c[0] + c[1] * c[1] + c[2] * c[2];", "c[0] * c[0] + c[1] * c[1];"),
    ("voxel index with x mirrored",
     "idx[s] = ((int64_t)i[2] * c->n[1] + i[1]) * c->n[0] + i[0];",
     "idx[s] = ((int64_t)i[2] * c->n[1] + i[1]) * c->n[0] + "
     "(c->n[0] - 1 - i[0]);"),
    ("voxel coordinate divided by dx on every axis",
     "double x = (o[a] + mid * u[a] - c->lo[a]) / c->d[a];",
     "double x = (o[a] + mid * u[a] - c->lo[a]) / c->d[0];"),
    ("plane crossings with the observer's sign flipped",
     "double al = (c->lo[a] + k * c->d[a] - o[a]) / u[a];",
     "double al = (c->lo[a] + k * c->d[a] + o[a]) / u[a];"),
    ("segment count includes masked rays",
     "if (mask && mask[id]) continue;\n            double o[3], u[3];\n"
     "            if (orc_ray(",
     "double o[3], u[3];\n            if (orc_ray("),
]

# The same for the solver module (Python): (what, text, replacement).
SOLVER_MUTANTS = [
    ("difference transpose with the wrong sign",
     "out[tuple(sl_lo)] -= g", "out[tuple(sl_lo)] += g"),
    ("temporal difference transpose with the wrong sign",
     "out[:-1] -= g", "out[:-1] += g"),
    ("outer map mask dropped from the prior term",
     "self.lam * self.K(\n            self.R(DtD_frames",
     "self.lam * (\n            self.R(DtD_frames"),
    ("prior weight applied on one side only",
     "self.R(DtD_frames(self.R(self.K(v))))", "DtD_frames(self.R(self.K(v)))"),
    ("temporal prior dropped from the normal operator",
     "out = out + self.lam_t * self.K(DtD_time(self.K(v)))", "out = out"),
    ("map mask not applied to the transpose",
     "return self.K(siddon.backproject(", "return (siddon.backproject("),
    ("map mask not applied to P",
     "return siddon.project(self.geom, self.K(x), self.pointing",
     "return siddon.project(self.geom, x, self.pointing"),
    ("pixel mask inverted", "np.where(self.mask == 0, y, 0.0)",
     "np.where(self.mask != 0, y, 0.0)"),
    ("lambda missing from J",
     "j = float(np.sum(r * r)) + self.lam * spatial",
     "j = float(np.sum(r * r)) + spatial"),
    ("temporal prior missing from J",
     "j += self.lam_t * float(np.sum(Dt_time(kx) ** 2))",
     "j += 0.0 * float(np.sum(Dt_time(kx) ** 2))"),
    ("CG step length from q.q", "alpha = rr / float(np.sum(p * q))",
     "alpha = rr / float(np.sum(q * q))"),
    ("CG residual updated with the wrong sign", "r = r - alpha * q",
     "r = r + alpha * q"),
    ("CG beta inverted", "beta = rr_new / rr", "beta = rr / rr_new"),
    ("CG warm start ignored",
     "r = b - problem.normal(x) if x0 is not None else b.copy()",
     "r = b.copy()"),
]

# The same for the Thomson module (Python): (what, text, replacement).
THOMSON_MUTANTS = [
    ("pB without the impact-parameter factor", "return o * pm", "return pm"),
    ("B with the sign of its pB part flipped",
     "map_mask=map_mask) - o * pm", "map_mask=map_mask) + o * pm"),
    ("pB transpose without the impact-parameter factor",
     "pto = siddon.backproject(geom, o * y,", "pto = siddon.backproject(geom, y,"),
    ("B transpose with m in place of m'",
     "return mp * siddon.backproject(", "return m * siddon.backproject("),
    ("C1 with sin for sin^2", "C1 = c * s * s", "C1 = c * s"),
    ("C3 with the cube term's sign flipped",
     "C3 = 4.0 / 3.0 - c - c ** 3 / 3.0", "C3 = 4.0 / 3.0 - c + c ** 3 / 3.0"),
    ("limb-darkening weights swapped in m",
     "((1.0 - u) * C1 + u * C2)", "(u * C1 + (1.0 - u) * C2)"),
    ("voxel factors at the voxels' lower corners",
     '(np.arange(geom["n" + a]) + 0.5) * geom["d" + a]',
     'np.arange(geom["n" + a]) * geom["d" + a]'),
    ("scattering kept inside the Sun", "out = r > 1.0", "out = r > 0.0"),
]

# Run in a child process: point the oracle at the given C library ("c") or
# load the given file in place of the named oracle module ("py"), then call
# every pin with each of its parameter sets until one raises.  Prints
# "READY" once the pins are imported, then "FAIL <pin>" or "PASS".
RUNNER = r"""
import importlib.util, inspect, os, sys
mode, path, root, name = sys.argv[1:5]
sys.path.insert(0, root)
import oracle
import oracle.siddon as siddon
if mode == "c":
    siddon._build.build = lambda force=False: path
    siddon._lib = None
else:
    spec = importlib.util.spec_from_file_location("oracle." + name, path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules["oracle." + name] = mod
    spec.loader.exec_module(mod)
    setattr(oracle, name, mod)
    if name == "thomson":  # the solver's operators use it too
        oracle.solver.thomson = mod
import tests.test_oracle_pins as pins
if mode == "py":
    assert getattr(oracle, name).__file__ == path
    assert name != "solver" or pins.solver.__file__ == path
golden = os.path.join(root, "tests", "golden")
skip = ("test_thomson_voxel_factors_pin_catches_planted_mistakes",)
calls = []
fns = sorted(inspect.getmembers(pins, inspect.isfunction),
             key=lambda nf: nf[1].__code__.co_firstlineno)  # the file's order
for name, fn in fns:
    if not name.startswith("test_") or name in skip or fn.__module__ != pins.__name__:
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


def _module_copy(source, out_dir):
    path = os.path.join(out_dir, "module_variant.py")
    with open(path, "w") as f:
        f.write(source)
    return path


def _run_pins(path, mode, name):
    """The last line the child prints ("PASS" or "FAIL <pin> <error>"), or
    "ERROR ..." when the harness itself failed."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", RUNNER, mode, path, ROOT,
                            name],
                           cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=900)
    except subprocess.TimeoutExpired:
        return "ERROR timeout"
    if r.returncode != 0 or "READY" not in r.stdout.split():
        return "ERROR exit %d: %s" % (r.returncode, (r.stdout + r.stderr)[-2000:])
    return r.stdout.strip().splitlines()[-1]


def _source(path=SRC):
    with open(path) as f:
        return f.read()


# (key prefix, mode, module name, source file, mutants)
FAMILIES = [("c", "c", "siddon", SRC, MUTANTS),
            ("solver", "py", "solver", SOLVER, SOLVER_MUTANTS),
            ("thomson", "py", "thomson", THOMSON, THOMSON_MUTANTS)]


def _variants():
    """(key, mode, module name, source) of each family's unmodified copy
    (key = the prefix) and of every mutant (key = prefix:what)."""
    out = []
    for prefix, mode, name, src_path, mutants in FAMILIES:
        src = _source(src_path)
        out.append((prefix, mode, name, src))
        for what, old, new in mutants:
            out.append((prefix + ":" + what, mode, name, src.replace(old, new)))
    return out


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    """Every variant built and run against the pins, the children in
    parallel (they are independent processes)."""
    jobs = []
    for i, (key, mode, name, src) in enumerate(_variants()):
        d = str(tmp_path_factory.mktemp("variant%02d" % i))
        path = _compile(src, d) if mode == "c" else _module_copy(src, d)
        jobs.append((key, path, mode, name))
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {key: ex.submit(_run_pins, path, mode, name)
                for key, path, mode, name in jobs}
        return {key: f.result() for key, f in futs.items()}


def test_each_mistake_is_planted_once():
    for prefix, _, _, src_path, mutants in FAMILIES:
        src = _source(src_path)
        for what, old, _ in mutants:
            assert src.count(old) == 1, (prefix, what)


@pytest.mark.parametrize("prefix", [f[0] for f in FAMILIES])
def test_unmodified_copy_passes_every_pin(results, prefix):
    assert results[prefix] == "PASS", results[prefix]


@pytest.mark.parametrize("key", [f[0] + ":" + m[0] for f in FAMILIES
                                 for m in f[4]])
def test_planted_mistake_fails_a_pin(results, key):
    got = results[key]
    assert got.startswith("FAIL"), "%s: %s" % (key, got)
