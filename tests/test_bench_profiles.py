"""The benchmark line's ncu-derived roofline fields on CPU.  The stored DRAM
traffic is the bytes of one full launch of the workload it was captured
for, and the reduction sectors per segment hold for that workload's
geometry: bench.py reports them only for that workload (and, for the
traffic, that image count), and null otherwise."""

import json
import os

import pytest

import bench
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _record(name):
    with open(os.path.join(ROOT, "profiles", name)) as f:
        return json.load(f)


def test_traffic_only_for_its_workload_and_image_count():
    rec = _record("traffic.json")
    workload, n_img = rec["workload"], rec["images"]
    # the capture's image count is the workload's own
    assert synth.make_config(workload)["pointing"].shape[0] == n_img
    for kernel, nbytes in rec["bytes_per_launch"].items():
        assert bench.ncu_traffic(kernel, workload, n_img) == nbytes
        assert bench.ncu_traffic(kernel, workload, n_img // 10) is None
        assert bench.ncu_traffic(kernel, "coronagraph", n_img) is None
    assert bench.ncu_traffic("no_such_kernel", workload, n_img) is None


@pytest.mark.parametrize("kernel", ["k_adjoint_plane<false>"])
def test_reduction_sectors_only_for_its_workload(kernel):
    rec = _record("reduction_sectors.json")[kernel]
    ratio = rec["l1_to_crossbar_reduction_sectors_per_segment"]
    assert 0.0 < ratio < 1.0
    assert bench.ncu_reduction_sectors(kernel, rec["workload"]) == ratio
    assert bench.ncu_reduction_sectors(kernel, "temporal") is None
    assert bench.ncu_reduction_sectors("no_such_kernel", rec["workload"]) is None
