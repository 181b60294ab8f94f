"""Walk rules and the autotuner: the per-image choice of walk (per ray or
plane by plane, counted or every-slab plane walk, plane or per-ray forward)
follows the rules of the problem's size bucket, changing them changes the
schedule and nothing else (P bit for bit, P^T within the oracle's bound),
and tomo_autotune picks rules among its candidates that later single and
batched calls use."""

import numpy as np
import pytest
import torch

import synth
from oracle import siddon
from tests.gpu_util import (assert_transpose_close, mask_dev, require_gpu,
                            to_dev)

pytestmark = pytest.mark.gpu

NEVER = 1e30


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _scene():
    """Views in and out of the ecliptic (counted and every-slab plane walks),
    a rolled view (layout 2), pixels 0.8 voxel apart."""
    rng = np.random.default_rng(77)
    g = synth.cube_geom(48, 1.5, ny=50, nz=47)
    lon = np.array([20.0, 70.0, 110.0, 160.0, 200.0, 250.0])
    lat = np.array([0.0, 0.5, 6.0, -12.0, 20.0, 1.0])
    ptg = synth.pointing_table(lon, lat, 215.0, 64, 60, 3.2)
    ptg[5, 3] = np.pi / 2
    cube = rng.random((47, 50, 48)).astype(np.float32)
    y = rng.random((lat.size, 60, 64)).astype(np.float32)
    mask = (rng.random((lat.size, 60, 64)) < 0.05).astype(np.uint8)
    return g, ptg, cube, y, mask


def _run(T, g, ptg, cube, y, mask, ctx):
    md = mask_dev(mask)
    P = T.tomo_project(to_dev(cube), g, ptg, 64, 60, mask=md, ctx=ctx)
    codes = T.tomo_walk_plan(ptg.shape[0], ctx=ctx)
    Pt = T.tomo_backproject(to_dev(y), g, ptg, mask=md, ctx=ctx)
    return P, Pt, codes


def test_rules_change_the_schedule_not_the_result(T):
    g, ptg, cube, y, mask = _scene()
    want_t = siddon.backproject(g, y, ptg, 64, 60, mask)
    cw = siddon.crossing_weights(g, y, ptg, 64, 60, mask)
    ctx = T.Context()
    P0, Pt0, c0 = _run(T, g, ptg, cube, y, mask, ctx)
    # defaults: plane walks everywhere (pitch ~0.5 voxel), counted walk for
    # the views near the ecliptic, every-slab for the others
    assert np.all(c0 & 1)
    assert not (c0[0] & 4) and (c0[3] & 4) and (c0[4] & 4)
    cases = {
        "per ray": ({"min_pitch": NEVER}, lambda c: np.all((c & 3) == 0)),
        "every slab": ({"general_ratio": 0.0}, lambda c: np.all(c & 4)),
        "counted": ({"general_ratio": NEVER}, lambda c: not np.any(c & 4)),
        "plane forward": ({"fwd_max_ratio": NEVER},
                          lambda c: np.all((c & 3) == 3)),
        "per-ray forward": ({"fwd_max_ratio": 0.0, "fwd_min_pitch": NEVER},
                            lambda c: np.all((c & 3) == 1)),
        # CTA order: groups of 4 images (the last one padded) and one group
        # of every image change no walk
        "groups": ({"fwd_group": 4.0, "adj_group": 65535.0},
                   lambda c: np.array_equal(c, c0)),
    }
    for name, (rules, check) in cases.items():
        T.tomo_set_plane_rules(rules, g, 64, 60, ctx=ctx)
        P, Pt, codes = _run(T, g, ptg, cube, y, mask, ctx)
        assert check(codes), (name, codes)
        assert torch.equal(P, P0), name
        assert_transpose_close(Pt.cpu().numpy(), want_t, cw, g,
                               "P^T rules %s" % name)
        # axes are the view's, whatever the rules
        assert np.array_equal(codes >> 3, c0 >> 3), name
    # the context default applies to buckets without their own rules
    T.tomo_set_plane_rules(None, g, 64, 60, ctx=ctx)
    T.tomo_set_plane_rules({"min_pitch": NEVER}, ctx=ctx)
    g2 = dict(g, nx=g["nx"] + 1)
    T.tomo_project(torch.ones((47, 50, 49), device="cuda"), g2, ptg, 64, 60,
                   ctx=ctx)
    assert np.all((T.tomo_walk_plan(ptg.shape[0], ctx=ctx) & 3) == 0)
    with pytest.raises(T.TomoError):
        T.tomo_set_plane_rules({"min_pitch": -1.0}, ctx=ctx)
    with pytest.raises(T.TomoError):
        T.tomo_walk_plan(ptg.shape[0] + 1, ctx=ctx)
    ctx.close()


def test_autotune_tunes_rules_used_by_single_and_batched_calls(T):
    g, ptg, cube, y, mask = _scene()
    ctx = T.Context()
    P0 = T.tomo_project(to_dev(cube), g, ptg, 64, 60, mask=mask_dev(mask),
                        ctx=ctx)
    best = T.tomo_autotune(to_dev(cube), to_dev(y), g, ptg,
                           mask=mask_dev(mask), ctx=ctx)
    r = best["rules"]
    assert r["min_pitch"] in (NEVER, 0.10, 0.16, 0.25, 0.40)
    assert r["general_ratio"] in (0.0, 0.02, 0.035, 0.06, NEVER)
    assert r["fwd_max_ratio"] in (0.0, 0.01, 0.02, 0.04, NEVER)
    assert r["fwd_min_pitch"] in (0.5, 0.75, 1.0, NEVER)
    assert r["fwd_group"] in (0.0, 1.0, 8.0, 32.0, 65535.0)
    assert r["adj_group"] in (0.0, 1.0, 8.0, 32.0, 65535.0)
    assert best["fwd_ms"] > 0 and best["adj_ms"] > 0
    # the tuned schedule: same images bit for bit, transpose within bound
    P, Pt, codes = _run(T, g, ptg, cube, y, mask, ctx)
    assert torch.equal(P, P0)
    if r["min_pitch"] >= NEVER:
        assert np.all((codes & 3) == 0)
    want_t = siddon.backproject(g, y, ptg, 64, 60, mask)
    cw = siddon.crossing_weights(g, y, ptg, 64, 60, mask)
    assert_transpose_close(Pt.cpu().numpy(), want_t, cw, g, "P^T tuned")
    # the batched path takes the bucket's rules too: forward equal to the
    # single-problem forward, transpose within the oracle bound, for the
    # tuned rules and for forced per-ray and every-slab rules
    prob = {"geom": g, "pointing": ptg, "nu": 64, "nv": 60,
            "cube": to_dev(cube), "mask": mask_dev(mask), "lam": 0.0}
    for rules in (None, {"min_pitch": NEVER}, {"general_ratio": 0.0}):
        if rules is not None:
            T.tomo_set_plane_rules(rules, g, 64, 60, ctx=ctx)
        d = dict(prob, images=torch.zeros((ptg.shape[0], 60, 64),
                                          device="cuda"))
        T.tomo_project_batched([d], ctx=ctx)
        assert torch.equal(d["images"], P0), rules
        d = dict(prob, images=to_dev(y), cube=torch.zeros_like(prob["cube"]))
        T.tomo_backproject_batched([d], ctx=ctx)
        assert_transpose_close(d["cube"].cpu().numpy(), want_t, cw, g,
                               "batched P^T rules %s" % rules)
    ctx.close()
