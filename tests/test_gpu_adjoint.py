"""Reverse mode: dL/dmu (per node) and dL/db of a displacement-misfit loss,
L = 1/2 sum over active nodes |u(t_N) - u_target|^2, through DisplacementRun (saved states every
few steps, recomputation, lbm_adjoint_step), against central finite differences of the forward:
the CUDA FP64 form and the FP64 oracle.  Clamped cube (velocity-Dirichlet faces), constant body
force, smooth non-uniform mu.  Then the whole gradient field against the oracle's own discrete
adjoint (itself pinned to central differences of the oracle's forward on CPU), on the cube and on a
rotated ellipsoid whose cut links take every branch of the interpolated bounce-back.
"""
import dataclasses

import numpy as np
import pytest

from paper_2606_20646_b300 import inputs as I

pytestmark = pytest.mark.gpu

N, STEPS, EVERY = 16, 60, 16       # EVERY does not divide STEPS; rows of 16: the staged kernels
B0 = (0.2, -0.3, -1.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_20646_b300 import build
    build.build()


def _problem(b=B0):
    p = I.inclusion_cube(N, STEPS)
    return p.with_(options=dataclasses.replace(p.options, body_force=tuple(b)))


def _mu0(p):
    X = p.coords()
    return 1.0 + 0.2 * np.sin(2 * np.pi * X[0]) * np.cos(np.pi * X[1]) + 0.1 * X[2]


def _gpu_u(p, mu, precision="fp64"):
    from paper_2606_20646_b300 import lbm
    sim = lbm.Simulation(p, precision=precision, adjoint=True)
    sim.set_mu_field(mu).set_initial().step(STEPS)
    u = sim.fields()[2].cpu().numpy()
    assert sim.sync(raise_on_status=False) == 0
    act = sim.active_mask()
    sim.close()
    return u, act


def _oracle_u(p, mu):
    import oracle
    o = oracle.Oracle(p).set_mu_field(mu).set_initial()
    o.step(STEPS)
    return o.fields()[2], o.active_mask()


def _loss(u, ut, act):
    return 0.5 * float((((u - ut) ** 2) * act).sum())


@pytest.fixture(scope="module")
def setup():
    p = _problem()
    ut, act = _gpu_u(p, p.meta["mu_target"])       # the displacement of the target modulus
    rng = np.random.default_rng(5)
    nodes = [tuple(rng.integers(2, N - 2, size=3)) for _ in range(5)]
    return p, ut, act, _mu0(p), nodes


def _adjoint(p, ut, act, mu0, precision):
    import torch
    from paper_2606_20646_b300 import adjoint, lbm
    sim = lbm.Simulation(p, precision=precision, adjoint=True)
    mu = torch.tensor(mu0, dtype=torch.float64, device="cuda", requires_grad=True)
    b = torch.tensor(B0, dtype=torch.float64, requires_grad=True)
    u = adjoint.displacement(mu, b, sim, STEPS, EVERY)
    utt = torch.as_tensor(ut, device="cuda")
    actt = torch.as_tensor(act, device="cuda")
    L = 0.5 * (((u - utt) ** 2) * actt).sum()
    L.backward()
    assert sim.sync(raise_on_status=False) == 0
    sim.close()
    return float(L.detach()), mu.grad.cpu().numpy(), b.grad.numpy()


def _fd_mu(forward, p, ut, mu0, node, act, rel=1e-4):
    e = rel * mu0[node]
    mp, mm = mu0.copy(), mu0.copy()
    mp[node] += e
    mm[node] -= e
    return (_loss(forward(p, mp)[0], ut, act) - _loss(forward(p, mm)[0], ut, act)) / (2 * e)


def _fd_b(forward, mu0, ut, act, i, h=1e-4):
    bp, bm = list(B0), list(B0)
    bp[i] += h
    bm[i] -= h
    return (_loss(forward(_problem(bp), mu0)[0], ut, act) - _loss(forward(_problem(bm), mu0)[0], ut, act)) / (2 * h)


def test_fp64_adjoint_matches_central_differences(setup):
    p, ut, act, mu0, nodes = setup
    L, gmu, gb = _adjoint(p, ut, act, mu0, "fp64")
    assert L > 0
    for n in nodes:
        fd = _fd_mu(_gpu_u, p, ut, mu0, n, act)
        print(f"dL/dmu{n}: adjoint {gmu[n]:.9e} fd {fd:.9e}")
        assert abs(gmu[n] - fd) <= 1e-4 * abs(fd), (n, gmu[n], fd)
    for i in range(3):
        fd = _fd_b(_gpu_u, mu0, ut, act, i)
        print(f"dL/db{i}: adjoint {gb[i]:.9e} fd {fd:.9e}")
        assert abs(gb[i] - fd) <= 1e-4 * abs(fd), (i, gb[i], fd)
    # inactive-free box: every node carries a gradient; it vanishes nowhere in the interior
    assert np.isfinite(gmu).all()


def test_fp64_adjoint_matches_oracle_differences(setup):
    """The same gradient against central differences of the FP64 oracle's forward."""
    p, ut, act, mu0, nodes = setup
    _, gmu, gb = _adjoint(p, ut, act, mu0, "fp64")
    for n in nodes[:2]:
        fd = _fd_mu(_oracle_u, p, ut, mu0, n, act)
        assert abs(gmu[n] - fd) <= 1e-4 * abs(fd), (n, gmu[n], fd)
    fd = _fd_b(_oracle_u, mu0, ut, act, 2)
    assert abs(gb[2] - fd) <= 1e-4 * abs(fd), (gb[2], fd)


def test_fp32_adjoint_against_fp64(setup):
    """FP32 form: the whole gradient field against the FP64 adjoint, and the sampled entries
    against FP64 central differences."""
    p, ut, act, mu0, nodes = setup
    _, g64, gb64 = _adjoint(p, ut, act, mu0, "fp64")
    _, g32, gb32 = _adjoint(p, ut, act, mu0, "fp32")
    rel = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    print(f"FP32 vs FP64 adjoint: dL/dmu rel-L2 {rel:.3e}, dL/db {gb32} vs {gb64}")
    assert rel < 1e-4
    assert np.abs(gb32 - gb64).max() <= 1e-4 * np.abs(gb64).max()
    for n in nodes:
        fd = _fd_mu(_gpu_u, p, ut, mu0, n, act)
        assert abs(g32[n] - fd) <= 1e-4 * abs(fd) + 1e-4 * np.abs(g64).max(), (n, g32[n], fd)


# ---- against the oracle's discrete adjoint (the whole gradient field) ---------------------------

def _gpu_grad(p, mu0, ut, act, precision, steps, every):
    import torch
    from paper_2606_20646_b300 import adjoint, lbm
    sim = lbm.Simulation(p, precision=precision, adjoint=True)
    mu = torch.tensor(mu0, dtype=torch.float64, device="cuda", requires_grad=True)
    b = torch.tensor(p.options.body_force, dtype=torch.float64, requires_grad=True)
    u = adjoint.displacement(mu, b, sim, steps, every)
    L = 0.5 * (((u - torch.as_tensor(ut, device="cuda")) ** 2) * torch.as_tensor(act, device="cuda")).sum()
    L.backward()
    assert sim.sync(raise_on_status=False) == 0
    sim.close()
    return mu.grad.cpu().numpy(), b.grad.numpy()


def _oracle_grad(p, mu0, ut, act, steps):
    import oracle
    o = oracle.Oracle(p).set_mu_field(mu0).set_initial()
    o.step(steps)
    u = o.fields()[2]
    o = oracle.Oracle(p).set_mu_field(mu0).set_initial()
    return o.adjoint(steps, (u - ut) * act)


def _ellipsoid_from_rest(N):
    """The rotated ellipsoid started from rest with F = I (initial populations independent of mu
    and b), driven by its prescribed surface velocity, with a body force: its links take both
    eta branches and the upstream fallback."""
    p = I.ellipsoid_3d(N)
    D = p.dim
    return p.with_(init_mode="equilibrium", dU0=None, v0=np.zeros((D,) + p.box_shape),
                   u0=np.zeros((D,) + p.box_shape),
                   F0=np.broadcast_to(np.eye(D).reshape(-1, 1, 1, 1), (D * D,) + p.box_shape).copy(),
                   options=dataclasses.replace(p.options, body_force=(0.3, 0.1, -0.5)))


@pytest.fixture(scope="module")
def ellipsoid_case():
    import oracle
    p = _ellipsoid_from_rest(16)
    mu0 = _mu0(p)
    steps = 40
    o = oracle.Oracle(p).set_mu_field(1.3 * mu0).set_initial()
    o.step(steps)
    ut = o.fields()[2]
    act = o.active_mask().reshape(p.box_shape)
    return p, mu0, ut, act, steps


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_fp64_adjoint_equals_oracle_adjoint_cube(setup):
    p, ut, act, mu0, _ = setup
    g, gb = _gpu_grad(p, mu0, ut, act, "fp64", STEPS, EVERY)
    go, gbo = _oracle_grad(p, mu0, ut, act, STEPS)
    print(f"cube: dL/dmu rel-L2 {_rel(g, go):.3e}, dL/db {gb} vs {gbo}")
    assert _rel(g, go) < 1e-12
    assert np.abs(gb - gbo).max() <= 1e-12 * np.abs(gbo).max()


def test_fp64_adjoint_equals_oracle_adjoint_ellipsoid(ellipsoid_case):
    p, mu0, ut, act, steps = ellipsoid_case
    g, gb = _gpu_grad(p, mu0, ut, act, "fp64", steps, 16)
    go, gbo = _oracle_grad(p, mu0, ut, act, steps)
    print(f"ellipsoid: dL/dmu rel-L2 {_rel(g, go):.3e}, dL/db {gb} vs {gbo}")
    assert _rel(g, go) < 1e-12
    assert np.abs(gb - gbo).max() <= 1e-12 * np.abs(gbo).max()
    assert not g[~act.astype(bool)].any()


def test_fp32_adjoint_ellipsoid_against_oracle(ellipsoid_case):
    """FP32 form (staged reverse kernel: rows of 16) on the body with every closure branch."""
    p, mu0, ut, act, steps = ellipsoid_case
    g, gb = _gpu_grad(p, mu0, ut, act, "fp32", steps, 16)
    go, gbo = _oracle_grad(p, mu0, ut, act, steps)
    print(f"ellipsoid FP32: dL/dmu rel-L2 {_rel(g, go):.3e}, dL/db {gb} vs {gbo}")
    assert _rel(g, go) < 1e-4
    assert np.abs(gb - gbo).max() <= 1e-4 * np.abs(gbo).max()


def test_fp64_adjoint_equals_oracle_adjoint_cube_32():
    """The clamped cube at 32^3 (20 steps, checkpoints every 8): the whole gradient field against
    the oracle's discrete adjoint."""
    import oracle
    p = I.inclusion_cube(32, 20)
    p = p.with_(options=dataclasses.replace(p.options, body_force=B0))
    mu0 = _mu0(p)
    o = oracle.Oracle(p).set_mu_field(p.meta["mu_target"]).set_initial()
    o.step(20)
    ut = o.fields()[2]
    act = o.active_mask().reshape(p.box_shape)
    del o
    g, gb = _gpu_grad(p, mu0, ut, act, "fp64", 20, 8)
    go, gbo = _oracle_grad(p, mu0, ut, act, 20)
    print(f"cube 32: dL/dmu rel-L2 {_rel(g, go):.3e}, dL/db {gb} vs {gbo}")
    assert _rel(g, go) < 1e-12
    assert np.abs(gb - gbo).max() <= 1e-12 * np.abs(gbo).max()


def test_inclusion_cube_128_full_length_against_central_differences():
    """The reverse-mode workload at its stated size: the 128^3 clamped cube with the spherical
    inclusion, 3000 steps, saved states every 100.  dL/dmu at five random interior nodes and dL/db
    (all three components) by the FP64 adjoint agree with central differences of the FP64 forward
    to 1e-4.  The FP32 adjoint's error is stated against the FP64 adjoint: after 3000 FP32 forward
    and reverse steps the whole dL/dmu field differs by 3.7e-2 (relative L2), the sampled nodes by
    up to 4.3e-2 and the dominant dL/db_z by 2.9e-2 (bounds: about 1.5 times those)."""
    import torch
    from paper_2606_20646_b300 import adjoint, lbm
    n, steps, every = 128, 3000, 100
    p = I.inclusion_cube(n, steps)
    b0 = tuple(p.options.body_force)
    mu0 = np.ones(p.box_shape)
    sim = lbm.Simulation(p, precision="fp64", adjoint=True)

    def forward(mu, b):
        sim.set_mu_field(mu).set_body_force(b).set_initial().step(steps)
        u = sim.fields()[2].cpu().numpy()
        assert sim.sync(raise_on_status=False) == 0
        return u

    ut = forward(p.meta["mu_target"], b0)
    act = sim.active_mask()
    rng = np.random.default_rng(128)
    nodes = [tuple(int(x) for x in rng.integers(8, n - 8, size=3)) for _ in range(5)]

    def grads(s):
        mu = torch.tensor(mu0, dtype=torch.float64, device="cuda", requires_grad=True)
        b = torch.tensor(b0, dtype=torch.float64, requires_grad=True)
        u = adjoint.displacement(mu, b, s, steps, every)
        L = 0.5 * (((u - torch.as_tensor(ut, device="cuda")) ** 2) * torch.as_tensor(act, device="cuda")).sum()
        L.backward()
        assert s.sync(raise_on_status=False) == 0
        return mu.grad.cpu().numpy(), b.grad.numpy()

    gmu, gb = grads(sim)
    for node in nodes:
        e = 1e-4
        mp, mm = mu0.copy(), mu0.copy()
        mp[node] += e
        mm[node] -= e
        fd = (_loss(forward(mp, b0), ut, act) - _loss(forward(mm, b0), ut, act)) / (2 * e)
        print(f"128^3 dL/dmu{node}: adjoint {gmu[node]:.9e} fd {fd:.9e}")
        assert abs(gmu[node] - fd) <= 1e-4 * abs(fd), (node, gmu[node], fd)
    for i in range(3):
        h = 1e-4
        bp, bm = list(b0), list(b0)
        bp[i] += h
        bm[i] -= h
        fd = (_loss(forward(mu0, bp), ut, act) - _loss(forward(mu0, bm), ut, act)) / (2 * h)
        print(f"128^3 dL/db{i}: adjoint {gb[i]:.9e} fd {fd:.9e}")
        assert abs(gb[i] - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(gb).max()), (i, gb[i], fd)
    sim.close()
    sim32 = lbm.Simulation(p, precision="fp32", adjoint=True)
    gmu32, gb32 = grads(sim32)
    sim32.close()
    ef = float(np.linalg.norm(gmu32 - gmu) / np.linalg.norm(gmu))
    eb = float(abs(gb32[2] - gb[2]) / abs(gb[2]))
    en = max(abs(gmu32[nd] - gmu[nd]) / abs(gmu[nd]) for nd in nodes)
    print(f"FP32 adjoint against the FP64 adjoint: dL/dmu field {ef:.3e}, at the nodes {en:.3e}, dL/db_z {eb:.3e}")
    assert ef < 6e-2 and en < 8e-2 and eb < 5e-2
