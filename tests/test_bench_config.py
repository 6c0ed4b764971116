"""The benchmark's choice of problem for each curved-element workload (host logic only)."""
import math

import pytest

import bench
from paper_2008_04356_gb300 import synth


@pytest.mark.parametrize("prec", [synth.FP32, synth.FP64])
def test_cylinder_is_navier_stokes_weak_form(prec):
    p = bench.shape_problem("cylinder", "weak", None, prec)
    assert p.geom == synth.GEOM_CYLINDER and p.physics == synth.NAVIER_STOKES
    assert p.volume == synth.VOLUME_WEAK and p.precision == prec and p.N == 7
    assert p.mu > 0.0


@pytest.mark.parametrize("workload,geom", [("annular", synth.GEOM_ANNULAR), ("cone", synth.GEOM_CONE)])
def test_euler_shapes_weak_form(workload, geom):
    p = bench.shape_problem(workload, "weak", None, synth.FP32)
    assert p.geom == geom and p.physics == synth.EULER
    assert p.volume == synth.VOLUME_WEAK and p.riemann == synth.RUSANOV
    assert p.nelem == 2 * 24 * 48 * 16 and p.N == 7
    if workload == "cone":
        assert p.cone_angle == pytest.approx(math.pi / 6)


@pytest.mark.parametrize("workload,geom", [("annular", synth.GEOM_ANNULAR), ("cone", synth.GEOM_CONE)])
@pytest.mark.parametrize("riemann,expect", [(None, synth.ROE_HH), ("roe", synth.ROE_HH), ("rusanov", synth.RUSANOV)])
def test_euler_shapes_split_form(workload, geom, riemann, expect):
    p = bench.shape_problem(workload, "split", riemann, synth.FP32)
    assert p.geom == geom and p.physics == synth.EULER
    assert p.volume == synth.VOLUME_SPLIT and p.riemann == expect


def test_split_cylinder_is_navier_stokes_split_form():
    p = bench.shape_problem("cylinder", "split", None, synth.FP32)
    assert p.geom == synth.GEOM_CYLINDER and p.physics == synth.NAVIER_STOKES
    assert p.volume == synth.VOLUME_SPLIT and p.riemann == synth.ROE_HH and p.mu > 0.0


def test_unknown_workload_rejected():
    with pytest.raises(ValueError):
        bench.shape_problem("sphere", "weak", None, synth.FP32)


def test_traffic_scales_with_the_launch_element_count(monkeypatch):
    import json
    import os
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "dg_element_traffic.json")))
    monkeypatch.setattr(bench, "source_sha", lambda paths: rec["source_sha"])
    assert bench.ncu_traffic() == rec["dram_bytes_per_launch_full_workload"]
    # the captured case (2 x 4x256x64) reads back its own measured bytes
    assert bench.ncu_traffic(2 * 4 * 256 * 64) == pytest.approx(rec["dram_bytes_per_launch_captured"], rel=1e-12)


def test_traffic_is_dropped_when_the_kernel_source_changed(monkeypatch):
    monkeypatch.setattr(bench, "source_sha", lambda paths: "0000000000000000")
    assert bench.ncu_traffic() is None


def test_algorithmic_flop_count_of_the_fp64_path():
    """The method's FP64 operations per DOF-update: the per-node terms at N = 5 add up to
    12 + 27 + 180 + 25 + 39 + 10 + 5 + 25 = 323, and the interface adds its per-face-pair
    work (80 (N+1)^3 + 156 (N+1)^2 flop) spread over the DOF of the two blocks."""
    faces, dof = 65536, 2 * 4 * 256 * 256 * 216
    per_face = 80 * 216 + 156 * 36
    assert bench.algorithmic_flop_per_dof(5, faces, dof) == pytest.approx(323 + per_face * faces / dof, rel=1e-12)
    assert bench.algorithmic_flop_per_dof(5, 0, dof) == pytest.approx(323, rel=1e-12)
    # the contractions grow with N + 1, the face terms shrink with it
    assert bench.algorithmic_flop_per_dof(7, 0, 1) > bench.algorithmic_flop_per_dof(3, 0, 1)
