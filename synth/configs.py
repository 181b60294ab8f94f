"""The seeded workloads the projector is tested and measured on.

Each recipe returns a plain dict::

    {"name", "geom", "n_frames", "cube" (float32, [T][nz][ny][nx] when T > 1
     else [nz][ny][nx]), "pointing" ((n_img, 12) float64), "nu", "nv",
     "mask" (uint8 [n_img][nv][nu] or None), "lam", "n_iter", "snr",
     "noise_seed"}

The noisy data ``y = P x + n`` are not built here, because they need the
projector: the caller projects with its own projector and then calls
:func:`add_noise` with the seeded draw from :func:`noise_draw`.

Workloads (the paper's STEREO data are not available; these seeded scenes
stand in for them):

``small``        64^3 over [-1.5, 1.5], 8 images 64^2, observers at 215 R_sun
                 every 45 degrees on the ecliptic, FOV 3.2 R_sun; radial
                 density with 10 % uniform noise (seed 0).
``single``       128^3, 60 images 256^2 at longitudes 3 k degrees, latitude
                 jitter U[-7, 7] degrees (seed 1); radial density plus 6
                 streamers; occulter r < 1.0; SNR 50; 20 CG iterations,
                 lambda 1e-2.
``batched``      32 problems, seeds 100..131 (see :func:`batched_problem`).
``temporal``     T = 8 frames of 256^3; 240 images 512^2 in two groups 40
                 degrees apart, 1.5 degree steps; time stamps U[0, 7] (seed 4).
``coronagraph``  512^3 over [-4, 4]; 360 images 1024^2 in two groups 86 degrees
                 apart, 1 degree steps, FOV 8 R_sun; mask r < 1.5 or r > 4;
                 power-law density, 20 streamers, 12 plumes; SNR 30; 50 CG
                 iterations, lambda 1e-2.
``paper128`` / ``paper256``  the paper's performance workload (Section 4): 64
                 images 256^2 and a 128^3 / 256^3 cube, observers every 5.625
                 degrees on the ecliptic.
``cg256``        the CG timing workload at 256^3: the ``temporal`` observers
                 and image size on one static cube (radial + 6 streamers),
                 occulter r < 1.0, SNR 50, 20 iterations, lambda 1e-2.

Every recipe takes a ``scale`` divisor (cube side, image side) so that a
reduced copy of the same scene can be built for the oracle.
"""

import numpy as np

from .geometry import cube_geom, pointing_table
from .corona import corona_cube, corona_frames, random_axes
from .masks import occulter_mask

D_OBS = 215.0  # observer distance [R_sun] (about 1 AU)


def noise_draw(seed, shape):
    """Standard-normal draws for the Gaussian image noise."""
    return np.random.default_rng(seed).standard_normal(shape)


def add_noise(y, z, mask, snr):
    """``y + sigma z`` with ``sigma = rms(y over unmasked pixels) / snr``.
    Masked pixels stay 0."""
    y = np.asarray(y, dtype=np.float64)
    keep = np.ones(y.shape, dtype=bool) if mask is None else (mask == 0)
    rms = np.sqrt(np.mean(y[keep] ** 2)) if keep.any() else 0.0
    out = y + (rms / snr) * z
    out[~keep] = 0.0
    return out


def _scene(name, n, half_width, nu, nv, lons, lats, fov, *, n_frames=1,
           times=None, density=None, mask_radii=(None, None), lam=1e-2,
           n_iter=0, snr=None, noise_seed=None):
    geom = cube_geom(n, half_width)
    pointing = pointing_table(lons, lats, D_OBS, nu, nv, fov, time=times)
    mask = None
    if mask_radii != (None, None):
        mask = occulter_mask(pointing, nu, nv, *mask_radii)
    return {"name": name, "geom": geom, "n_frames": n_frames,
            "cube": density(geom), "pointing": pointing, "nu": nu, "nv": nv,
            "mask": mask, "lam": lam, "n_iter": n_iter, "snr": snr,
            "noise_seed": noise_seed}


def _radial_noisy(seed):
    def f(geom):
        return corona_cube(geom, "exp", noise_frac=0.1,
                           noise_rng=np.random.default_rng(seed))
    return f


def _radial_streamers(seed, n_streamers=6):
    def f(geom):
        axes = random_axes(np.random.default_rng(seed), n_streamers)
        return corona_cube(geom, "exp", structures=[(axes, 0.05, 3.0)])
    return f


def small(scale=1):
    n, npx = 64 // scale, 64 // scale
    lons = 45.0 * np.arange(8)
    return _scene("small", n, 1.5, npx, npx, lons, 0.0, 3.2,
                  density=_radial_noisy(0))


def single(scale=1):
    n, npx = 128 // scale, 256 // scale
    k = np.arange(60)
    lats = np.random.default_rng(1).uniform(-7.0, 7.0, 60)
    return _scene("single", n, 1.5, npx, npx, 3.0 * k, lats, 3.2,
                  density=_radial_streamers(1), mask_radii=(1.0, None),
                  lam=1e-2, n_iter=20, snr=50.0, noise_seed=1001)


def _temporal_frames(seed, n_frames):
    def f(geom):
        rng = np.random.default_rng(seed)
        axes = random_axes(rng, 6)
        phase = rng.uniform(0.0, 2.0 * np.pi, 6)
        t = np.arange(n_frames)[:, None]
        amps = 3.0 * (1.0 + 0.5 * np.sin(2.0 * np.pi * t / n_frames + phase))
        return corona_frames(geom, axes, 0.05, amps)
    return f


def _two_groups(n_per_group, step_deg, separation_deg):
    k = np.arange(n_per_group)
    return np.concatenate([step_deg * k, separation_deg + step_deg * k])


def temporal(scale=1, n_frames=8):
    n, npx = 256 // scale, 512 // scale
    lons = _two_groups(120, 1.5, 40.0)
    times = np.random.default_rng(4).uniform(0.0, n_frames - 1, 240)
    return _scene("temporal", n, 1.5, npx, npx, lons, 0.0, 3.2,
                  n_frames=n_frames, times=times,
                  density=_temporal_frames(4, n_frames))


def _power_structures(seed):
    def f(geom):
        rng = np.random.default_rng(seed)
        streamers = random_axes(rng, 20)
        plumes = random_axes(rng, 12, polar_within_deg=20.0)
        return corona_cube(geom, "power", structures=[
            (streamers, 0.05, 3.0), (plumes, 0.1, 3.0)])
    return f


def coronagraph(scale=1):
    n, npx = 512 // scale, 1024 // scale
    lons = _two_groups(180, 1.0, 86.0)
    return _scene("coronagraph", n, 4.0, npx, npx, lons, 0.0, 8.0,
                  density=_power_structures(5), mask_radii=(1.5, 4.0),
                  lam=1e-2, n_iter=50, snr=30.0, noise_seed=1005)


def paper(n_cube=128, scale=1):
    n, npx = n_cube // scale, 256 // scale
    lons = 5.625 * np.arange(64)
    return _scene("paper%d" % n_cube, n, 1.5, npx, npx, lons, 0.0, 3.2,
                  density=_radial_noisy(0))


def cg256(scale=1):
    n, npx = 256 // scale, 512 // scale
    lons = _two_groups(120, 1.5, 40.0)
    return _scene("cg256", n, 1.5, npx, npx, lons, 0.0, 3.2,
                  density=_radial_streamers(256), mask_radii=(1.0, None),
                  lam=1e-2, n_iter=20, snr=50.0, noise_seed=1256)


def problem_seeds_batched():
    return list(range(100, 132))


def batched_problem(seed, max_side=None):
    """One problem of the batched workload: cube side from {32, 48, 64, 96,
    128}, image count from 16..120, image side from {64, 128, 256, 512},
    observers evenly spaced in longitude on the ecliptic at 215 R_sun with FOV
    3.2 R_sun, radial density with 10 % noise; 10 CG iterations, lambda 1e-2.
    ``max_side`` caps the image side (for reduced oracle runs)."""
    rng = np.random.default_rng(seed)
    n = int(rng.choice([32, 48, 64, 96, 128]))
    n_img = int(rng.integers(16, 121))
    npx = int(rng.choice([64, 128, 256, 512]))
    if max_side is not None:
        npx = min(npx, max_side)
    lons = 360.0 / n_img * np.arange(n_img)
    sc = _scene("batched-%d" % seed, n, 1.5, npx, npx, lons, 0.0, 3.2,
                density=_radial_noisy(seed), lam=1e-2, n_iter=10)
    return sc


def batched(max_side=None):
    return [batched_problem(s, max_side) for s in problem_seeds_batched()]


CONFIGS = {
    "small": small, "single": single, "temporal": temporal,
    "coronagraph": coronagraph, "cg256": cg256,
    "paper128": lambda scale=1: paper(128, scale),
    "paper256": lambda scale=1: paper(256, scale),
}


def make_config(name, scale=1):
    return CONFIGS[name](scale=scale)
