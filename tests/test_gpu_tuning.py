"""Tile shapes, the link schedule and the autotuner (lbm_set_tuning, lbm_autotune).

Every shape computes the same values node for node: windows per warp only group the fused kernel's
32-node windows, Jacobi segments per warp only group the sweep's segments, the link block only
groups links, and the overlapped link schedule only runs the link kernels alongside windows that
share no data with them.  So the fields after any number of steps are bit-identical across shapes
and schedules, and the autotuner, which times candidates from a saved state and restores it, leaves
the simulation where it was.  Shell (Neumann links, projection steps), FP32, BF16 storage and FP64;
an affine annulus (Dirichlet links only) and a periodic box.
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
    assert got["link_schedule"] == 1
    for shape in [(1, 1, 64, 2), (2, 4, 256, 1), (4, 2, 128, 2), (4, 1, 64, 1)]:
        out, got, _ = _fields(shell, precision, shape)
        assert (got["windows_per_warp"], got["jacobi_segments"], got["link_block"], got["link_schedule"]) == shape
        for a, b in zip(out, ref):
            assert np.array_equal(a, b), (precision, shape)


@pytest.mark.parametrize("precision", ["fp32", "bf16s"])
def test_autotune_restores_the_state(shell, precision):
    ref, _, _ = _fields(shell, precision)
    out, got, tune = _fields(shell, precision, autotune=True)
    print(f"{precision} autotune: {tune}")
    assert tune["candidates"] >= 5
    assert tune["ms_per_step"] <= tune["default_ms_per_step"]
    keys = ("windows_per_warp", "jacobi_segments", "link_block", "link_schedule")
    assert tuple(got[k] for k in keys) == tuple(tune[k] for k in keys)
    for a, b in zip(out, ref):
        assert np.array_equal(a, b)


def test_invalid_shapes_are_refused(shell):
    from paper_2606_20646_b300 import lbm
    sim = lbm.Simulation(shell, precision="fp32")
    for bad in [(3, 0, 0), (0, 8, 0), (0, 0, 96), (0, 0, 0, 3)]:
        with pytest.raises(lbm.LbmError):
            sim.set_tuning(*bad)
    sim.close()


def _periodic_hole():
    """A periodic box with a spherical traction-loaded hole: links and neighbours that wrap."""
    import dataclasses
    p = I.random_periodic(3, 24, seed=5)
    opts = dataclasses.replace(p.options, proj_every=5, proj_iters=20)
    return p.with_(name="periodic_hole_3d_24", options=opts,
                   shapes=[I.Shape("sphere", (0.05, 0.5, 0.5), (0.2,), complement=True, boundary_id=0)],
                   bcs=[I.BC(0, "neumann", "const", ramp="sin2", t_ramp=0.05, vec=(0.02, 0.0, 0.01))])


@pytest.mark.parametrize("make,precision,steps", [
    (lambda: I.shell_3d(48), "fp64", 23),
    (lambda: I.affine_annulus_2d(96), "fp32", 30),
    (_periodic_hole, "fp32", 21),
    (lambda: I.random_box(2, 60, 3), "bf16s", 27),
])
def test_link_schedules_give_the_same_fields(make, precision, steps):
    """Overlapped and serial link schedules, and lbm_step_graph with either, give identical fields;
    the boundary windows are a proper, non-empty part of the window list where there are links."""
    from paper_2606_20646_b300 import lbm
    p = make()
    outs = []
    for sched, graph in (("serial", False), ("overlap", False), ("overlap", True)):
        sim = lbm.Simulation(p, precision=precision)
        sim.set_tuning(link_schedule=sched)
        sim.set_initial()
        if graph:
            sim.step(1).step_graph(steps - 1)
        else:
            sim.step(steps)
        outs.append([t.cpu().numpy() for t in sim.fields()])
        assert sim.sync(raise_on_status=False) == 0
        inf = sim.info()
        sim.close()
    if inf["n_cut"] > 0:
        assert 0 < inf["n_boundary_segments"] <= inf["n_segments"]
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b), (p.name, precision)
