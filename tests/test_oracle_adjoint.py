"""Pins of the oracle's discrete adjoint (reverse mode of the FP64 step for velocity-Dirichlet
bodies) against the oracle's own forward: central differences of a displacement-misfit loss
L = 1/2 sum over active nodes |u(t_N) - u_target|^2 with respect to the shear modulus at single
nodes and to the body force, and the directional derivative along a random field of moduli (one
number that every node's gradient enters).  Two bodies: the clamped cube (all face links eta = 0.2,
the upstream branch of the interpolated bounce-back) and a small rotated ellipsoid whose links take
both eta branches and the upstream fallback.  Both start from rest with F = I: the reverse mode
holds the initial populations fixed, and from that state they do not depend on mu or b.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2606_20646_b300 import inputs as I

STEPS = 30


def _cube():
    p = I.inclusion_cube(8, STEPS)
    return p.with_(options=dataclasses.replace(p.options, body_force=(0.2, -0.3, -1.0)))


def _ellipsoid():
    """The ellipsoid from rest (v0 = 0, F0 = I, equilibrium start), so that the initial populations,
    an input of the reverse mode, do not depend on mu (P(I) = 0) or b; the surface's prescribed
    affine velocity sets it in motion."""
    p = I.ellipsoid_3d(12)
    D = p.dim
    return p.with_(init_mode="equilibrium", dU0=None, v0=np.zeros((D,) + p.box_shape),
                   u0=np.zeros((D,) + p.box_shape),
                   F0=np.broadcast_to(np.eye(D).reshape(-1, 1, 1, 1), (D * D,) + p.box_shape).copy(),
                   options=dataclasses.replace(p.options, body_force=(0.3, 0.1, -0.5)))


def _mu(p):
    X = p.coords()
    return 1.0 + 0.2 * np.sin(2 * np.pi * X[0]) * np.cos(np.pi * X[1]) + 0.1 * X[2]


def _u(p, mu):
    o = oracle.Oracle(p).set_mu_field(mu).set_initial()
    o.step(STEPS)
    return o.fields()[2], o.active_mask().reshape(p.box_shape)


def _loss(p, mu, ut, act):
    u, _ = _u(p, mu)
    return 0.5 * float((((u - ut) ** 2) * act).sum())


def _setup(p):
    mu0 = _mu(p)
    ut, act = _u(p, 1.3 * mu0)           # target: a stiffer body
    u0, _ = _u(p, mu0)
    o = oracle.Oracle(p).set_mu_field(mu0).set_initial()
    gmu, gb = o.adjoint(STEPS, (u0 - ut) * act)
    return mu0, ut, act, gmu, gb


@pytest.fixture(scope="module", params=["cube", "ellipsoid"])
def case(request):
    p = _cube() if request.param == "cube" else _ellipsoid()
    return (p,) + _setup(p)


def test_adjoint_mu_matches_central_differences(case):
    p, mu0, ut, act, gmu, _ = case
    nodes = np.argwhere(act)
    rng = np.random.default_rng(3)
    for n in [tuple(nodes[i]) for i in rng.choice(len(nodes), 4, replace=False)] + [tuple(nodes[0])]:
        e = 1e-4 * mu0[n]
        mp, mm = mu0.copy(), mu0.copy()
        mp[n] += e
        mm[n] -= e
        fd = (_loss(p, mp, ut, act) - _loss(p, mm, ut, act)) / (2 * e)
        assert abs(gmu[n] - fd) <= 1e-6 * abs(fd) + 1e-14, (n, gmu[n], fd)


def test_adjoint_b_matches_central_differences(case):
    p, mu0, ut, act, _, gb = case
    for i in range(3):
        h = 1e-4
        bp, bm = list(p.options.body_force), list(p.options.body_force)
        bp[i] += h
        bm[i] -= h
        Lp = _loss(p.with_(options=dataclasses.replace(p.options, body_force=tuple(bp))), mu0, ut, act)
        Lm = _loss(p.with_(options=dataclasses.replace(p.options, body_force=tuple(bm))), mu0, ut, act)
        fd = (Lp - Lm) / (2 * h)
        assert abs(gb[i] - fd) <= 1e-6 * abs(fd) + 1e-14, (i, gb[i], fd)


def test_adjoint_directional_derivative(case):
    """<dL/dmu, delta> against the central difference along a random field delta."""
    p, mu0, ut, act, gmu, _ = case
    delta = np.random.default_rng(11).uniform(-1, 1, size=mu0.shape) * act
    h = 1e-4
    fd = (_loss(p, mu0 + h * delta, ut, act) - _loss(p, mu0 - h * delta, ut, act)) / (2 * h)
    ad = float((gmu * delta).sum())
    assert abs(ad - fd) <= 1e-7 * abs(fd), (ad, fd)


def test_adjoint_vanishes_off_the_body_and_at_the_target():
    """dL/dmu is zero at inactive nodes; at the target modulus the misfit and its gradient are 0."""
    p = _ellipsoid()
    mu0 = _mu(p)
    ut, act = _u(p, mu0)
    o = oracle.Oracle(p).set_mu_field(mu0).set_initial()
    gmu, gb = o.adjoint(STEPS, np.zeros((3,) + p.box_shape))
    assert not gmu.any() and not gb.any()
    u0, _ = _u(p, 1.3 * mu0)
    o = oracle.Oracle(p).set_mu_field(1.3 * mu0).set_initial()
    gmu, _ = o.adjoint(STEPS, (u0 - ut) * act)
    assert not gmu[~act.astype(bool)].any()


def test_adjoint_refuses_neumann_bodies():
    p = I.random_box(2, 20, 1)
    o = oracle.Oracle(p).set_initial()
    with pytest.raises(ValueError):
        o.adjoint(2, np.zeros((p.dim,) + p.box_shape))
