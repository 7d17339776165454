"""lbm_census_static: the geometry census for callers that cannot allocate device memory
(for example while a CUDA graph is being captured).  Its counts must equal the ones
lbm_create computes with caller-allocated storage, on two calls in a row; collected last
so a failure here does not hide the other tests."""
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
    cases = [I.shell_3d(96), I.random_box(3, 30, 2), I.superellipse_shell_2d(200), I.random_periodic(2, 40, 1)]
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
