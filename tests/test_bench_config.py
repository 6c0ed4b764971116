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


def test_split_cylinder_rejected():
    with pytest.raises(ValueError):
        bench.shape_problem("cylinder", "split", None, synth.FP32)


def test_unknown_workload_rejected():
    with pytest.raises(ValueError):
        bench.shape_problem("sphere", "weak", None, synth.FP32)
