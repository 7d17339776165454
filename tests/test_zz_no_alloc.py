"""lbm_census_static: the geometry census for callers that may not allocate device memory (an
embedding runtime whose device memory is one arena handed out by its own allocator, or a process
at its memory limit that must size a body before it can plan the storage).  Its counts must equal
the ones lbm_create computes with caller-allocated storage, on two calls in a row; it must refuse
the bodies lbm_create refuses; and repeated calls must leave the device's free memory and torch's
allocation unchanged.  Collected last so a failure here does not hide the other tests."""
import dataclasses

import pytest

from paper_2606_20646_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_20646_b300 import build
    build.build()


def _reference_counts(p):
    from paper_2606_20646_b300 import lbm
    sim = lbm.Simulation(p, precision="fp32")
    inf = sim.info()
    sim.close()
    return {"n_active": inf["n_active"], "n_cut": inf["n_cut"], "n_segments": inf["n_segments"]}


def test_census_static_matches_create_two_calls():
    from paper_2606_20646_b300 import lbm
    cases = [I.shell_3d(96), I.random_box(3, 30, 2), I.superellipse_shell_2d(200), I.random_periodic(2, 40, 1),
             I.face_touching_box(3, 32, 3)]
    for p in cases:
        ref = _reference_counts(p)
        first = lbm.census_static(p)
        second = lbm.census_static(p)          # the shared scratch keeps the last call's contents
        assert first == ref, (p.name, first, ref)
        assert second == ref, (p.name, second, ref)


def test_census_static_rejects_oversized_box():
    from paper_2606_20646_b300 import lbm
    p = I.shell_3d(257)                        # 257^3 nodes > LBM_CENSUS_MAX_NODES
    with pytest.raises(lbm.LbmError) as e:
        lbm.census_static(p)
    assert e.value.code == -7


def _empty_body():
    p = I.shell_3d(32)
    # a sphere smaller than half a spacing centred on a cell corner holds no node
    return p.with_(shapes=[I.Shape("sphere", (0.0, 0.0, 0.0), (0.01,), boundary_id=1)])


def _past_the_face():
    p = I.shell_3d(32)
    # the outer sphere reaches beyond the box [-1, 1]^3: links leaving the box do not cross the surface
    sh = [dataclasses.replace(p.shapes[0], axes=(1.5, 1.5, 1.5)), p.shapes[1]]
    return p.with_(shapes=sh)


@pytest.mark.parametrize("make", [_empty_body, _past_the_face])
def test_census_static_applies_the_domain_rules(make):
    """The bodies lbm_create refuses with LBM_ERR_DOMAIN are refused by the census too."""
    from paper_2606_20646_b300 import lbm
    p = make()
    with pytest.raises(lbm.LbmError) as e:
        lbm.Simulation(p, precision="fp32")
    assert e.value.code == -2
    with pytest.raises(lbm.LbmError) as e:
        lbm.census_static(p)
    assert e.value.code == -2


def test_census_static_allocates_nothing():
    """After a first call (which looks up the scratch array's address and loads the kernels), more
    calls change neither the device's free memory nor torch's allocated bytes."""
    import torch
    from paper_2606_20646_b300 import lbm
    p = I.shell_3d(128)
    ref = lbm.census_static(p)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert lbm.census_static(p) == ref
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
