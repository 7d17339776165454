"""Full-size checks of the 3D shell workload (256^3 box, 5.84 M active nodes, 299 448 Neumann
links) in the launch configuration the benchmark times (TMA-staged fused kernel, per-link
sources, projection every 20 steps).

1. FP32 form against the FP64 oracle on the whole box for the first steps (a projection step
   and a regular step) from a smooth, non-trivial initial state.
2. A property that holds at any size and any step count: the shell problem is invariant under
   the reflections X_A -> -X_A of the centred box, so v_A is odd and the other velocity
   components even in X_A.  The FP64 form keeps it to round-off at t = 1.0 (1280 steps).
3. The FP32 form against the FP64 form at t = 1.0, and its own mirror asymmetry.
"""
import numpy as np
import pytest

from paper_2606_20646_b300 import inputs as I
from parity import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_20646_b300 import build
    build.build()


def _smooth_initial(p, amp=0.02):
    """Radially symmetric-free smooth perturbation: v0 and F0 - I from low Fourier modes."""
    X = p.coords()
    rng = np.random.default_rng(2606)
    for i in range(3):
        k = rng.integers(1, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi, size=3)
        p.v0[i] = amp * np.sin(np.pi * k[0] * X[0] + ph[0]) * np.cos(np.pi * k[1] * X[1] + ph[1]) * \
            np.cos(np.pi * k[2] * X[2] + ph[2])
    for m in range(9):
        k = rng.integers(1, 3, size=3)
        p.F0[m] += 0.5 * amp * np.cos(np.pi * k[0] * X[0]) * np.sin(np.pi * k[1] * X[1] + 0.3 * m) * \
            np.cos(np.pi * k[2] * X[2])
    return p


def test_shell_256_matches_oracle_first_steps():
    import oracle
    from paper_2606_20646_b300 import lbm
    p = _smooth_initial(I.shell_3d(256))
    steps = 2
    sim = lbm.Simulation(p, precision="fp32")
    assert sim.info()["n_active"] == 5841344
    sim.set_initial().step(steps)
    g = [t.cpu().numpy() for t in sim.fields()]
    assert sim.sync(raise_on_status=False) == 0
    sim.close()
    o = oracle.Oracle(p).set_initial()
    o.step(steps)
    r = o.fields()
    mask = o.active_mask()
    del o
    assert rel_l2(g[0], r[0], mask) < 1e-5
    assert rel_l2(g[1], r[1], mask) < 1e-5


def _mirror_asymmetry(v):
    """Largest relative-L2 and pointwise deviation of v from the reflection symmetry of the
    centred shell (v_A odd, the other components even, in X_A)."""
    rel, mx = 0.0, 0.0
    scale = np.abs(v).max()
    assert scale > 0
    for A in range(3):
        axis = 2 - A                             # arrays are (z, y, x)
        for i in range(3):
            sign = -1.0 if i == A else 1.0
            diff = v[i] - sign * np.flip(v[i], axis=axis)
            rel = max(rel, np.linalg.norm(diff) / np.linalg.norm(v[i]))
            mx = max(mx, np.abs(diff).max() / scale)
    return rel, mx


# 1280 steps reach t = 1.0, half-way up the sin^2 pressure ramp (s = 0.5): the same physical time as
# the 64^3 oracle comparison of the FP32 form, with 64 projection steps
STEPS = 1280


@pytest.fixture(scope="module")
def shell_t1():
    """v and F of the 256^3 shell at t = 1.0, both forms."""
    from paper_2606_20646_b300 import lbm
    out = {}
    for prec in ("fp64", "fp32"):
        sim = lbm.Simulation(I.shell_3d(256), precision=prec)
        sim.set_initial().step(STEPS)
        v, F, _ = [t.cpu().numpy().astype(np.float64) for t in sim.fields()]
        assert sim.sync(raise_on_status=False) == 0
        out[prec] = (v, F, sim.active_mask())
        sim.close()
    return out


def test_shell_256_reflection_symmetry_fp64(shell_t1):
    rel, mx = _mirror_asymmetry(shell_t1["fp64"][0])
    print(f"FP64 mirror asymmetry of v at t = 1: rel-L2 {rel:.3e}, max {mx:.3e}")
    assert rel < 1e-10 and mx < 1e-9


def test_shell_256_fp32_tracks_fp64(shell_t1):
    """The FP32 form against the FP64 form (itself held to the oracle at 1e-12 on smaller boxes)
    on the full box, at the FP32 form's tolerance of 1e-5 relative L2 on v and F."""
    v64, F64, act = shell_t1["fp64"]
    v32, F32, _ = shell_t1["fp32"]
    ev = rel_l2(v32, v64, act)
    eF = rel_l2(F32, F64, act)
    I9 = np.eye(3).reshape(-1)[:, None]
    eG = rel_l2(F32[:, act] - I9, F64[:, act] - I9)
    rel, mx = _mirror_asymmetry(v32)
    print(f"FP32 vs FP64 at 256^3, t = 1: v {ev:.3e}, F {eF:.3e}, F-I {eG:.3e}; "
          f"FP32 mirror asymmetry rel-L2 {rel:.3e}, max {mx:.3e}")
    assert ev < 1e-5 and eF < 1e-5


def test_shell_256_fp32_full_length_run():
    """The workload's full length: 4000 steps (t = 3.125, past the sin^2 ramp that ends at t = 2),
    FP32 in the launch configuration the benchmark times: no device status, finite fields, J
    within the range of a mildly compressed and stretched shell (radial BVP: 0.93 to 1.02), the
    velocity relaxing.  At omega = 1.5, below the paper's 1.8: with 1.8 this stiff shell (lambda = 5)
    blows up 500-1000 steps after the ramp, in the FP32 and FP64 forms alike, starting at the inner
    surface; the extra BGK dissipation of omega = 1.5 holds it (v_rms 2.0e-2 at step 2000, 6e-4 at
    4000)."""
    from paper_2606_20646_b300 import lbm
    p = I.shell_3d(256, omega=1.5)
    sim = lbm.Simulation(p, precision="fp32")
    sim.set_initial()
    act = sim.active_mask()
    vr = []
    for _ in range(4):
        sim.step(1000)
        v, F, u = [t.cpu().numpy() for t in sim.fields()]
        assert sim.sync(raise_on_status=False) == 0
        vr.append(float(np.sqrt((v[:, act] ** 2).mean())))
    assert sim.info()["step"] == 4000
    sim.close()
    Fa = F[:, act].T.reshape(-1, 3, 3).astype(np.float64)
    J = np.linalg.det(Fa)
    print(f"shell 256^3 FP32, 4000 steps: v_rms per 1000 steps {vr}, J in [{J.min():.4f}, {J.max():.4f}]")
    assert np.isfinite(F[:, act]).all() and np.isfinite(u[:, act]).all()
    assert vr[3] < vr[1]          # after the ramp the damping takes the velocity down
    # relaxed to the nonlinear radial BVP (inner nominal traction, outer traction-free): its J
    # spans [1.0014, 1.0191]; the lattice's J (measured [1.0007, 1.0190]) has the same range
    import radial_bvp as rb
    r = rb.solve(3, 1.0, 5.0, 0.4, 0.9, ("P", -1.0), ("P", 0.0))
    assert abs(J.max() - r["J"].max()) < 1e-3 and abs(J.min() - r["J"].min()) < 2e-3
