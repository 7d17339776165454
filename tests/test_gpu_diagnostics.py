"""Cauchy stress and J output (Eq. cauchy-recovery-general), the node-major field layout, whole-body
diagnostics and the wave-speed audit, through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

from paper_2606_20646_b300 import inputs as I
from parity import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_20646_b300 import build
    build.build()


def _run(p, steps, precision, **kw):
    from paper_2606_20646_b300 import lbm
    sim = lbm.Simulation(p, precision=precision, **kw)
    sim.set_initial().step(steps)
    return sim


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_cauchy_stress_and_J_match_the_oracle(precision, tol):
    import oracle
    p = I.random_box(3, 22, 2)
    steps = 30
    sim = _run(p, steps, precision)
    v, F, u, sig, J = [t.cpu().numpy() for t in sim.fields_ex()]
    assert sim.sync(raise_on_status=False) == 0
    o = oracle.Oracle(p).set_initial()
    o.step(steps)
    rs, rJ = o.stress()
    act = o.active_mask()
    assert rel_l2(sig, rs, act) < tol
    assert rel_l2(J[0], rJ, act) < tol
    # the fields of lbm_fields_ex are those of lbm_fields
    v2, F2, u2 = [t.cpu().numpy() for t in sim.fields()]
    assert np.array_equal(v, v2) and np.array_equal(F, F2) and np.array_equal(u, u2)
    assert (sig[:, ~act] == 0).all() and (J[0][~act] == 0).all()


def test_node_major_layout_is_the_transpose_of_planes():
    p = I.shell_3d(32)
    sim = _run(p, 25, "fp32")
    planes = [t.cpu().numpy() for t in sim.fields_ex(layout="planes")]
    nodes = [t.cpu().numpy() for t in sim.fields_ex(layout="nodes")]
    for a, b in zip(planes, nodes):
        assert np.array_equal(a, np.moveaxis(b, -1, 0))


def test_host_staging_field_output():
    """With host staging, lbm_fields_ex writes pinned host memory; equal to the device call."""
    import ctypes as C
    import torch
    from paper_2606_20646_b300 import lbm
    p = I.shell_3d(24)
    sim = _run(p, 21, "fp32", host_staging=True)
    dev = [t.cpu().numpy() for t in sim.fields_ex()]
    D = 3
    host = [torch.empty((n,) + p.box_shape, dtype=torch.float64).pin_memory() for n in (D, D * D, D, D * D, 1)]
    rc = lbm.load_library().lbm_fields_ex(sim.h, *[C.c_void_p(t.data_ptr()) for t in host], 0)
    assert rc == 0
    sim.stream.synchronize()
    for a, b in zip(dev, host):
        assert np.array_equal(a, b.numpy())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_diagnostics_match_the_oracle(precision):
    """J range, RMS and largest |v|, largest tangent speed and the compatibility residual of a
    Neumann shell with projection (45 steps: projection steps 0, 20, 40) and of a ragged box."""
    import oracle
    for p, steps in ((I.shell_3d(32), 45), (I.random_box(2, 45, 1), 23)):
        sim = _run(p, steps, precision)
        d = sim.diagnostics()
        assert sim.sync(raise_on_status=False) == 0
        o = oracle.Oracle(p).set_initial()
        o.step(steps)
        r = o.diagnostics()
        assert d["n_edges"] == r["n_edges"] and d["n_active"] == o.counts()["n_active"]
        assert d["step"] == steps
        tol = 1e-12 if precision == "fp64" else 1e-5
        for k in ("J_min", "J_max", "v_rms", "v_max", "c_tangent"):
            assert abs(d[k] - r[k]) <= tol * abs(r[k]), (p.name, k, d[k], r[k])
        # the residual is a difference of nearby displacements: FP32 keeps it to 1e-3 of itself
        assert abs(d["incompat_rms"] - r["incompat_rms"]) <= (tol if precision == "fp64" else 1e-3) * r["incompat_rms"]
        sim.close()


def test_wave_speed_audit_of_the_initial_state():
    """lbm_set_initial audits c against the largest tangent speed of F0 over the active nodes: a
    compressed initial state whose speed exceeds c / 2.5 is refused with LBM_ERR_UNSTABLE_C while
    the reference state passes; a negative c_audit turns the audit off."""
    import oracle
    from paper_2606_20646_b300 import lbm
    p = I.random_periodic(3, 12, seed=3, lam=5.0)
    cT0 = np.sqrt(p.lam + 2 * p.mu)
    p.options.c = 2.5 * cT0 * 1.02                  # the reference state passes
    p.F0[:] = 0.0
    for i in range(3):
        p.F0[4 * i] = 0.7                          # F0 = 0.7 I: a faster tangent speed
    cT = np.sqrt(oracle.tangent_speed2(3, p.mu, p.lam, 0.7 * np.eye(3)))
    assert 2.5 * cT > p.options.c
    sim = lbm.Simulation(p, precision="fp32")
    with pytest.raises(lbm.LbmError) as e:
        sim.set_initial()
    assert e.value.code == -8
    sim.close()
    p.options.c_audit = -1.0
    sim = lbm.Simulation(p, precision="fp32")
    sim.set_initial()
    assert sim.info()["step"] == 0
    sim.close()
