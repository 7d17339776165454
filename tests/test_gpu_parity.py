"""Parity of the sm_103a CUDA path (called through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 form 1e-12 relative L2 on v, F, u; FP32 form 1e-5 relative L2 on v
and F.  Sizes span several 32-node segments and ragged tails (boxes not multiples of 32).
"""
import numpy as np
import pytest

from paper_2606_20646_b300 import inputs as I
from parity import compare, rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_20646_b300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def _check64(errs, st_gpu, st_orc):
    assert st_gpu == 0 and st_orc == 0
    for k in ("v", "F", "u"):
        assert errs[k] < TOL64, errs


def test_shear_wave_fp64_64x64_2000_steps():
    """2D D2Q4x6 FP64 periodic 64x64 shear wave, 2000 steps (t = 3.125)."""
    p = I.shear_wave_2d(64)
    errs, sg, so, *_ = compare(p, p.steps, "fp64")
    _check64(errs, sg, so)


@pytest.mark.parametrize("dim,n", [(2, 40), (3, 13)])
def test_random_periodic_fp64_forced_damped(dim, n):
    """Periodic box, smooth random v0 and F0, body force, damping, characteristic init with
    finite-difference gradients (dU0 not supplied)."""
    p = I.random_periodic(dim, n, seed=7, gamma=3.0, body_force=(0.4, -0.2, 0.1), init_mode="characteristic")
    errs, sg, so, *_ = compare(p, 60, "fp64")
    _check64(errs, sg, so)


def test_affine_annulus_fp64():
    """Curved velocity-Dirichlet closure, both BFL branches (Sec. 4.2 geometry, N=72)."""
    p = I.affine_annulus_2d(72)
    errs, sg, so, *_ = compare(p, p.steps, "fp64")
    _check64(errs, sg, so)


def test_ellipsoid_fp64():
    """3D rotated ellipsoid, affine Dirichlet (Sec. 5.1 geometry, N=28)."""
    p = I.ellipsoid_3d(28)
    errs, sg, so, *_ = compare(p, 60, "fp64")
    _check64(errs, sg, so)


def test_radial_traction_annulus_fp64():
    """Mixed Dirichlet / nominal-traction Neumann, LSQ + Newton, projection every 20 steps."""
    p = I.radial_traction_annulus_2d(56)
    errs, sg, so, *_ = compare(p, 250, "fp64")
    _check64(errs, sg, so)


@pytest.mark.parametrize("dim,n,seed", [(2, 45, 1), (3, 22, 2)])
def test_random_body_ragged_box_fp64(dim, n, seed):
    """Seeded random body in a ragged box (n, n+3, n+5): Dirichlet hole with an affine ramp,
    Neumann outer surface with a constant traction ramp, projection every 5 steps."""
    p = I.random_box(dim, n, seed)
    errs, sg, so, *_ = compare(p, 40, "fp64")
    _check64(errs, sg, so)


@pytest.mark.parametrize("dim,n,seed", [(2, 48, 1), (3, 32, 2)])
def test_face_touching_body_fp64(dim, n, seed):
    """Body whose surface passes between the outermost nodes and every box face: active nodes on
    the faces with cut links leaving the box (neighbour indices outside the box are never used)."""
    p = I.face_touching_box(dim, n, seed)
    errs, sg, so, *_ = compare(p, 40, "fp64")
    _check64(errs, sg, so)


def test_face_touching_body_fp32():
    """FP32 form of the box-face case, rows a multiple of 16 (the bulk-copy kernel)."""
    p = I.face_touching_box(3, 32, 3)
    errs, sg, so, *_ = compare(p, 40, "fp32")
    assert sg == 0 and so == 0
    assert errs["v"] < TOL32 and errs["F"] < TOL32, errs


def test_shell_fp64_32():
    """3D thick spherical shell, both surfaces Neumann (mean gauge), 32^3."""
    p = I.shell_3d(32)
    errs, sg, so, *_ = compare(p, 120, "fp64")
    _check64(errs, sg, so)


def test_annulus_fp32_128():
    """2D FP32 annulus (inner radial displacement ramp, outer traction-free), 128^2 copy,
    400 steps (mid-ramp)."""
    p = I.annulus_radial_2d(128)
    errs, sg, so, *_ = compare(p, 400, "fp32")
    assert sg == 0 and so == 0
    assert errs["v"] < TOL32 and errs["F"] < TOL32, errs


def test_shell_fp32_64():
    """3D FP32 shell, 64^3 copy of the 256^3 workload, 320 steps (t = 1.0, mid-ramp)."""
    p = I.shell_3d(64)
    errs, sg, so, *_ = compare(p, 320, "fp32")
    assert sg == 0 and so == 0
    assert errs["v"] < TOL32 and errs["F"] < TOL32, errs


@pytest.mark.parametrize("builder,N", [(I.affine_annulus_2d, 384), (I.superellipse_shell_2d, 384),
                                       (I.ellipsoid_3d, 64), (I.shell_3d, 64)])
def test_geometry_matches_oracle(builder, N):
    """Active mask and cut-link list bit-exact; eta and N_b to FP64 rounding; LSQ stencil sizes."""
    import oracle
    from paper_2606_20646_b300 import lbm
    p = builder(N)
    sim = lbm.Simulation(p, precision="fp64")
    o = oracle.Oracle(p)
    assert (sim.active_mask() == o.active_mask()).all()
    g, r = sim.links(), o.links()
    assert len(g["node"]) == len(r["node"])
    assert (g["node"] == r["node"]).all() and (g["q"] == r["q"]).all() and (g["bid"] == r["bid"]).all()
    assert np.abs(g["eta"] - r["eta"]).max() < 1e-12
    assert np.abs(g["Nb"] - r["Nb"]).max() < 1e-12
    assert (g["ns"] == r["ns"]).all()


@pytest.mark.parametrize("builder,N,steps,prec", [(I.affine_annulus_2d, 72, 60, "fp64"),
                                                  (I.shell_3d, 32, 45, "fp64"),
                                                  (I.shell_3d, 48, 45, "fp32")])
def test_sampled_level_set_matches_oracle(builder, N, steps, prec):
    """A body given by node samples of its level set (Sec. 3.1): mask and cut links bit-exact, eta
    and N_b to FP64 rounding, and the run at the form's tolerance."""
    import oracle
    from paper_2606_20646_b300 import lbm
    p = I.sampled_copy(builder(N))
    sim = lbm.Simulation(p, precision=prec)
    o = oracle.Oracle(p)
    assert (sim.active_mask() == o.active_mask()).all()
    g, r = sim.links(), o.links()
    assert (g["node"] == r["node"]).all() and (g["q"] == r["q"]).all() and (g["bid"] == r["bid"]).all()
    assert np.abs(g["eta"] - r["eta"]).max() < 1e-12 and np.abs(g["Nb"] - r["Nb"]).max() < 1e-12
    sim.close()
    errs, sg, so, *_ = compare(p, steps, prec)
    assert sg == 0 and so == 0
    if prec == "fp64":
        _check64(errs, sg, so)
    else:
        assert errs["v"] < TOL32 and errs["F"] < TOL32, errs
