"""Tile shapes and the autotuner (lbm_set_tuning, lbm_autotune).

Every shape computes the same values node for node: windows per warp only group the fused kernel's
32-node windows, Jacobi segments per warp only group the sweep's segments, the link block only
groups links, and two Jacobi sweeps per launch repeat the one-sweep kernel's arithmetic node for
node.  So the fields after any number of steps are bit-identical across shapes, and the autotuner,
which times candidates from a saved state and restores it, leaves the simulation where it was.
Shell (Neumann links, projection steps), FP32 and BF16 storage; ragged, face-touching and 2D bodies
and an odd sweep count for the two-sweep kernel.
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
    assert got["jacobi_sweeps"] == 1  # the 3D default
    for shape in [(1, 1, 64, 1), (2, 4, 256, 2), (4, 2, 128, 1), (4, 1, 64, 2)]:
        out, got, _ = _fields(shell, precision, shape)
        assert (got["windows_per_warp"], got["jacobi_segments"], got["link_block"], got["jacobi_sweeps"]) == shape
        for a, b in zip(out, ref):
            assert np.array_equal(a, b), (precision, shape)


@pytest.mark.parametrize("precision", ["fp32", "bf16s"])
def test_autotune_restores_the_state(shell, precision):
    ref, _, _ = _fields(shell, precision)
    out, got, tune = _fields(shell, precision, autotune=True)
    print(f"{precision} autotune: {tune}")
    assert tune["candidates"] >= 5
    assert tune["ms_per_step"] <= tune["default_ms_per_step"]
    keys = ("windows_per_warp", "jacobi_segments", "link_block", "jacobi_sweeps")
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


def _odd_sweeps():
    import dataclasses
    p = I.random_box(3, 20, 4)
    return p.with_(options=dataclasses.replace(p.options, proj_iters=7))


@pytest.mark.parametrize("make,precision,steps", [
    (lambda: I.shell_3d(40), "fp32", 23),
    (lambda: I.random_box(3, 29, 2), "fp32", 12),
    (lambda: I.face_touching_box(3, 26, 3), "bf16s", 12),
    (_odd_sweeps, "fp32", 11),
    (lambda: I.superellipse_shell_2d(230), "fp32", 23),
    (lambda: I.random_box(2, 250, 1), "fp32", 12),
    (lambda: I.face_touching_box(2, 60, 5), "fp32", 12),
])
def test_two_sweeps_per_launch_equal_single_sweeps(make, precision, steps):
    """Two Jacobi sweeps per launch (tiles staged by bulk copies, the first sweep's values kept in
    shared memory) give the same fields, bit for bit, as one sweep per launch; 2D takes two by
    default, 3D one."""
    from paper_2606_20646_b300 import lbm
    p = make()
    sim = lbm.Simulation(p, precision=precision)
    assert sim.get_tuning()["jacobi_sweeps"] == (2 if p.dim == 2 else 1)
    sim.close()
    outs = []
    for sweeps in (1, 2):
        sim = lbm.Simulation(p, precision=precision)
        sim.set_tuning(jacobi_sweeps=sweeps)
        assert sim.get_tuning()["jacobi_sweeps"] == sweeps
        sim.set_initial().step(steps)
        outs.append([t.cpu().numpy() for t in sim.fields()])
        assert sim.sync(raise_on_status=False) == 0
        sim.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b), p.name


def _periodic_hole():
    """A periodic box with a spherical traction-loaded hole (projection steps, wrapping neighbours)."""
    import dataclasses
    p = I.random_periodic(3, 24, seed=5)
    return p.with_(name="periodic_hole_3d_24", options=dataclasses.replace(p.options, proj_every=5, proj_iters=20),
                   shapes=[I.Shape("sphere", (0.05, 0.5, 0.5), (0.2,), complement=True, boundary_id=0)],
                   bcs=[I.BC(0, "neumann", "const", ramp="sin2", t_ramp=0.05, vec=(0.02, 0.0, 0.01))])


@pytest.mark.parametrize("make,precision", [(lambda: I.shell_3d(32), "fp64"), (_periodic_hole, "fp32")])
def test_two_sweeps_per_launch_only_where_available(make, precision):
    """The FP64 form and periodic boxes keep one sweep per launch, even when asked for two."""
    from paper_2606_20646_b300 import lbm
    sim = lbm.Simulation(make(), precision=precision)
    assert sim.get_tuning()["jacobi_sweeps"] == 1
    sim.set_tuning(jacobi_sweeps=2)
    assert sim.get_tuning()["jacobi_sweeps"] == 1
    sim.set_initial().step(11)  # projection steps run with one sweep per launch
    assert sim.sync(raise_on_status=False) == 0
    sim.close()
