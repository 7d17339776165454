"""A rigid translation through projection steps, on the CUDA path, against its exact solution.

A traction-free disc or ball (and, anchored, an annulus or shell whose hole translates as a Dirichlet
surface) moving at a uniform velocity with F = I: u = vt t, v = vt, F = I is exact (P(I) = 0, zero
tractions, Dirichlet data equal to the translation), and the closure, both projection solves (Sec.
3.5) with their displacement resets and the accumulator bookkeeping (Eq. u-recovery-general) must
keep it.  The FP64 form keeps it to round-off; the FP32 form to its storage precision (populations
shifted by f^eq(0, I), u* as FP32 pairs).
"""
import numpy as np
import pytest

from paper_2606_20646_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_20646_b300 import build
    build.build()


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("anchored", [False, True])
@pytest.mark.parametrize("precision,tol_v,tol_u", [("fp64", 1e-12, 1e-12), ("fp32", 1e-6, 1e-8)])
def test_rigid_translation_kept_through_projection_steps(D, anchored, precision, tol_v, tol_u):
    from paper_2606_20646_b300 import lbm
    p = I.rigid_translation(D, anchored)
    sim = lbm.Simulation(p, precision=precision)
    sim.set_initial().step(p.steps)
    v, F, u = [t.cpu().numpy().astype(np.float64).reshape(t.shape[0], -1) for t in sim.fields()]
    act = sim.active_mask().reshape(-1)
    assert sim.sync(raise_on_status=False) == 0
    sim.close()
    vt, t = p.meta["vt"], p.steps * p.dt
    ev = np.abs(v[:, act] - vt[:, None]).max()
    eF = np.abs(F[:, act] - np.eye(D).reshape(-1, 1)).max()
    eu = np.abs(u[:, act] - vt[:, None] * t).max()
    print(f"{p.name} {precision}: |v - vt| {ev:.2e}, |F - I| {eF:.2e}, |u - vt t| {eu:.2e}")
    assert act.sum() > 100
    assert ev < tol_v and eF < tol_v and eu < tol_u
