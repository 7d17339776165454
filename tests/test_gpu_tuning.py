"""Tile shapes and the autotuner (lbm_set_tuning, lbm_autotune).

Every shape computes the same values node for node: windows per warp only group the fused kernel's
32-node windows, Jacobi segments per warp only group the sweep's segments, and the link block only
groups links.  So the fields after any number of steps are bit-identical across shapes, and the
autotuner, which times candidates from a saved state and restores it, leaves the simulation where
it was.  Shell (Neumann links, projection steps), FP32 and BF16 storage.
"""
import numpy as np
import pytest

from paper_2606_20646_b300 import inputs as I

pytestmark = pytest.mark.gpu

STEPS = 25  # projection steps at 0 and 20


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_20646_b300 import build
    build.build()


def _fields(p, precision, shape=None, autotune=False):
    from paper_2606_20646_b300 import lbm
    sim = lbm.Simulation(p, precision=precision)
    sim.set_initial()
    tune = None
    if shape:
        sim.set_tuning(*shape)
    if autotune:
        sim.step(3)
        before = sim.info()["step"]
        tune = sim.autotune(steps=20)
        assert sim.info()["step"] == before
        sim.step(STEPS - 3)
    else:
        sim.step(STEPS)
    out = [t.cpu().numpy() for t in sim.fields()]
    assert sim.sync(raise_on_status=False) == 0
    got = sim.get_tuning()
    sim.close()
    return out, got, tune


@pytest.fixture(scope="module")
def shell():
    return I.shell_3d(64)


@pytest.mark.parametrize("precision", ["fp32", "bf16s"])
def test_every_shape_gives_the_same_fields(shell, precision):
    ref, got, _ = _fields(shell, precision)
    assert got["windows_per_warp"] == (2 if precision == "bf16s" else 1)
    for shape in [(1, 1, 64), (2, 4, 256), (4, 2, 128), (4, 1, 64)]:
        out, got, _ = _fields(shell, precision, shape)
        assert (got["windows_per_warp"], got["jacobi_segments"], got["link_block"]) == shape
        for a, b in zip(out, ref):
            assert np.array_equal(a, b), (precision, shape)


@pytest.mark.parametrize("precision", ["fp32", "bf16s"])
def test_autotune_restores_the_state(shell, precision):
    ref, _, _ = _fields(shell, precision)
    out, got, tune = _fields(shell, precision, autotune=True)
    print(f"{precision} autotune: {tune}")
    assert tune["candidates"] >= 5
    assert tune["ms_per_step"] <= tune["default_ms_per_step"]
    assert (got["windows_per_warp"], got["jacobi_segments"], got["link_block"]) == \
        (tune["windows_per_warp"], tune["jacobi_segments"], tune["link_block"])
    for a, b in zip(out, ref):
        assert np.array_equal(a, b)


def test_invalid_shapes_are_refused(shell):
    from paper_2606_20646_b300 import lbm
    sim = lbm.Simulation(shell, precision="fp32")
    for bad in [(3, 0, 0), (0, 8, 0), (0, 0, 96)]:
        with pytest.raises(lbm.LbmError):
            sim.set_tuning(*bad)
    sim.close()
