"""Failure detection without faulting the GPU: inadmissible states and impossible boundary
data are injected from the host; kernels latch bits in the device status word, which
lbm_sync reports (and clears) as LBM_ERR_DEVICE."""
import numpy as np
import pytest

from paper_2606_20646_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_20646_b300 import build
    build.build()


def test_inverted_element_sets_jacobian_bit():
    from paper_2606_20646_b300 import lbm
    p = I.random_periodic(2, 16, seed=3)
    p.F0[0, 5, 5] = -1.0                       # det F < 0 at one node (Eq. positive-jacobian)
    sim = lbm.Simulation(p, precision="fp32")
    sim.set_initial().step(1)
    st = sim.sync(raise_on_status=False)
    assert st & 2
    assert sim.sync(raise_on_status=False) == 0   # cleared after reporting


def test_nonfinite_state_sets_bit():
    from paper_2606_20646_b300 import lbm
    p = I.random_periodic(3, 8, seed=3)
    p.v0[1, 2, 3, 4] = np.nan
    sim = lbm.Simulation(p, precision="fp64")
    sim.set_initial().step(1)
    with pytest.raises(lbm.LbmError):
        sim.sync()


def test_unsolvable_traction_sets_newton_bit():
    """A traction the local inversion cannot meet (not a number) makes every Newton solve on
    that surface fail; the failure is latched and reported, nothing traps."""
    from paper_2606_20646_b300 import lbm
    p = I.shell_3d(24)
    p.bcs[0] = I.BC(0, "neumann", "radial", ramp="one", center=(0, 0, 0), amp=float("nan"))
    sim = lbm.Simulation(p, precision="fp32")
    sim.set_initial().step(2)
    st = sim.sync(raise_on_status=False)
    assert st & 4


def test_missing_boundary_condition_is_rejected():
    from paper_2606_20646_b300 import lbm
    p = I.shell_3d(24)
    p.bcs = p.bcs[:1]                          # boundary id 1 has no BC
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(p, precision="fp32")
    assert e.value.code == -1


def test_body_reaching_box_face_is_rejected():
    from paper_2606_20646_b300 import lbm
    p = I.shell_3d(24)
    p.shapes[0].axes = (1.5, 1.5, 1.5)         # outer sphere larger than the box
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(p, precision="fp32")
    assert e.value.code == -2


def test_step_before_initial_state_is_rejected():
    from paper_2606_20646_b300 import lbm
    sim = lbm.Simulation(I.shell_3d(16), precision="fp32")
    with pytest.raises(lbm.LbmError) as e:
        sim.step(1)
    assert e.value.code == -5


def test_bulk_copy_wait_that_runs_out_is_reported():
    """The fused kernel's bounded wait for its bulk copies: with its first limit set to 0 polls
    every first wait runs out at once; the kernel latches LBM_DEV_TIMEOUT (128), waits (with the
    full limit) for the copies it issued and returns without writing, and lbm_sync reports the
    bit.  No fault: the context stays usable, and a fresh simulation afterwards runs cleanly."""
    from paper_2606_20646_b300 import lbm
    p = I.shell_3d(32)                          # rows of 32 nodes: the bulk-copy kernel runs
    sim = lbm.Simulation(p, precision="fp32")
    sim.set_initial().step(2)                   # first step (plain kernel, projection), then one fused step
    assert sim.sync(raise_on_status=False) == 0
    sim.set_wait_limit(0)
    sim.step(1)                                 # step 2: a fused step, every first wait runs out
    st = sim.sync(raise_on_status=False)
    assert st & 128
    sim.close()
    sim = lbm.Simulation(p, precision="fp32")
    sim.set_initial().step(3)
    assert sim.sync(raise_on_status=False) == 0
    sim.close()


def test_two_sweep_jacobi_wait_that_runs_out_is_reported():
    """The two-sweep Jacobi kernel's bounded waits: on a 2D body whose rows (230 nodes) are not a
    multiple of 16 the fused kernel uses plain loads, so the projection's two-sweep launches are the
    only kernels that wait for bulk copies.  With the first limit at 0 polls every block gives up at
    once, votes to stop, waits (with the full limit) for the planes it issued and stores nothing;
    LBM_DEV_TIMEOUT is reported and the context stays usable."""
    from paper_2606_20646_b300 import lbm
    p = I.superellipse_shell_2d(230)
    sim = lbm.Simulation(p, precision="fp32")
    assert sim.get_tuning()["jacobi_sweeps"] == 2
    sim.set_initial()
    sim.set_wait_limit(0)
    sim.step(1)                                 # step 0 is a projection step
    st = sim.sync(raise_on_status=False)
    assert st & 128
    sim.close()
    sim = lbm.Simulation(p, precision="fp32")
    sim.set_initial().step(3)
    assert sim.sync(raise_on_status=False) == 0
    sim.close()
