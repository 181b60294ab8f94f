"""How far CG with float32 vectors drifts from FP64 CG (a CPU emulation).

The GPU solver keeps the CG vectors x, r, p, q and b in float32 and its
scalars (p.q, r.r, alpha, beta and the criterion) in FP64 (Section 2.2,
Eq. criterion; CG as in Sections 3.1 and 5.1).  Rounding every vector
operation to float32 perturbs the Krylov sequence, and the perturbation grows
with the iteration count; the CG tolerances of the GPU tests
(``tests/test_gpu_solver.py``: 1e-3 in x and J after 20 iterations;
``tests/test_gpu_coronagraph.py``: 1e-2 in x and 3e-3 in J after 50) are
derived from the drift this script measures.

The emulation runs the oracle's FP64 normal operator (``oracle/solver.py``)
and rounds its output and every vector update to float32, with FP64 scalar
reductions, then compares x and J with the oracle's FP64 CG on the same data.
It calls only the oracle and the seeded input generators.

    python tests/cg_drift_emulation.py            # both cases
    python tests/cg_drift_emulation.py single     # one of them
"""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import siddon, solver  # noqa: E402

f32 = np.float32


def cg_float32(problem, n_iter):
    """CG with float32 vectors and FP64 scalars, the device's arithmetic
    around the exact projector.  Returns x (float32) and J per iterate from
    the device's identity J_k = y^T M y - x_k^T (r_k + b)."""
    b = problem.rhs().astype(f32)
    x = np.zeros(problem.shape, f32)
    r = b.copy()
    p = r.copy()
    ymy = float(np.sum(problem.masked(problem.y) ** 2))
    rr = float(np.sum(r.astype(np.float64) ** 2))
    Js = [ymy]
    for _ in range(n_iter):
        q = problem.normal(p.astype(np.float64)).astype(f32)
        alpha = rr / float(np.sum(p.astype(np.float64) * q))
        x = (x + f32(alpha) * p).astype(f32)
        r = (r - f32(alpha) * q).astype(f32)
        rr_new = float(np.sum(r.astype(np.float64) ** 2))
        beta = rr_new / rr
        p = (r + f32(beta) * p).astype(f32)
        rr = rr_new
        Js.append(ymy - float(np.sum(x.astype(np.float64) *
                                     (r.astype(np.float64) + b))))
    return x, np.array(Js)


def data(c):
    """The GPU tests' data: the oracle projection of the seeded cube plus
    the seeded noise at the case's SNR (pixels under the mask are 0)."""
    y = siddon.project(c["geom"], c["cube"], c["pointing"], c["nu"], c["nv"],
                       c["mask"])
    if c["snr"]:
        y = synth.add_noise(y, synth.noise_draw(c["noise_seed"], y.shape),
                            c["mask"], c["snr"])
    return y.astype(f32)


CASES = {
    # name: (config, scale, iterations)
    "single": ("single", 2, 20),
    "coronagraph": ("coronagraph", 8, 50),
}


def run(name):
    cfg, scale, n_iter = CASES[name]
    c = synth.make_config(cfg, scale=scale)
    y = data(c)
    pb = solver.Problem(c["geom"], c["pointing"], c["nu"], c["nv"], y,
                        c["mask"], lam=c["lam"])
    x64, rep = solver.cg(pb, n_iter)
    x32, J32 = cg_float32(pb, n_iter)
    dx = np.linalg.norm(x32 - x64) / np.linalg.norm(x64)
    dJ = np.abs(J32 - rep["J"]) / rep["J"]
    return {"case": "%s/%d" % (cfg, scale), "iterations": n_iter,
            "x_rel_drift": float(dx), "J_rel_drift_last": float(dJ[-1]),
            "J_rel_drift_max": float(dJ.max())}


if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    for n in names:
        print(run(n), flush=True)
