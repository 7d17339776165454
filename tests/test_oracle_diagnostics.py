"""Pins of the oracle's Cauchy stress, tangent wave speed and whole-body diagnostics against
closed forms, printed values and brute force (no GPU)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2606_20646_b300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("D,mu,lam", [(2, 1.0, 2.0), (3, 1.0, 5.0), (3, 0.7, 13.0)])
def test_tangent_speed_at_rest_is_the_p_wave_modulus(D, mu, lam):
    """At F = I the largest tangent speed is the longitudinal one, c_L^2 = lambda + 2 mu."""
    assert abs(oracle.tangent_speed2(D, mu, lam, np.eye(D)) - (lam + 2.0 * mu)) < 1e-13


def _acoustic_tensor_fd(D, mu, lam, F, n, h=1e-6):
    """Q_ik(n) = n_A dP_iA/dF_kB n_B by central differences of the oracle's P along e_k (x) n."""
    Q = np.zeros((D, D))
    for k in range(D):
        E = np.zeros((D, D))
        E[k, :] = n
        Pp, _ = oracle.piola(D, mu, lam, F + h * E)
        Pm, _ = oracle.piola(D, mu, lam, F - h * E)
        Q[:, k] = ((Pp - Pm) / (2 * h)) @ n
    return Q


@pytest.mark.parametrize("D", [2, 3])
def test_tangent_speed_is_the_largest_acoustic_eigenvalue(D):
    """Brute force: the largest eigenvalue of the acoustic tensor (Eq. acoustic-tensor-general-d),
    built by differencing P, maximised over unit directions, equals the oracle's value."""
    from scipy.optimize import minimize
    rng = np.random.default_rng(11 + D)
    mu, lam = 1.2, 4.0
    for _ in range(3):
        while True:
            F = np.eye(D) + 0.3 * rng.standard_normal((D, D))
            if np.linalg.det(F) > 0.3:
                break
        def neg(x):
            n = x / np.linalg.norm(x)
            return -np.linalg.eigvalsh(0.5 * (lambda Q: Q + Q.T)(_acoustic_tensor_fd(D, mu, lam, F, n)))[-1]
        starts = rng.standard_normal((24, D))
        best = min((minimize(neg, x0, method="Nelder-Mead", options=dict(xatol=1e-10, fatol=1e-12, maxiter=4000))
                    for x0 in starts), key=lambda r: r.fun)
        assert abs(-best.fun - oracle.tangent_speed2(D, mu, lam, F)) < 1e-6 * (-best.fun)


def _homogeneous(D, n, F, v=None):
    """Periodic box, uniform F0 and v0, u0 = 0, no damping or force: recovery returns them."""
    p = I.random_periodic(D, n, seed=1)
    p.options.gamma = 0.0
    p.options.body_force = (0.0, 0.0, 0.0)
    p.init_mode = "equilibrium"
    p.F0 = np.broadcast_to(np.asarray(F).reshape(D * D, *([1] * D)), (D * D,) + p.box_shape).copy()
    p.v0 = np.zeros((D,) + p.box_shape)
    if v is not None:
        p.v0 += np.asarray(v).reshape(D, *([1] * D))
    p.u0 = np.zeros((D,) + p.box_shape)
    return p


def test_cauchy_stress_reproduces_the_printed_affine_annulus_stress():
    """sigma = J^-1 P F^T at the homogeneous state F* = I + A of Sec. 4.2 equals the printed
    sigma_ex (Eq. affine-annulus-stress), J the printed J*."""
    g = GOLD["affine_annulus"]
    F = np.eye(2) + np.array(g["A"])
    p = _homogeneous(2, 8, F)
    p.mu, p.lam = g["mu"], g["lambda"]
    o = oracle.Oracle(p).set_initial()
    sig, J = o.stress()
    assert np.allclose(J, g["J_star"], atol=1e-12)
    sig = g["stress_scale_MPa"] * sig.reshape(2, 2, -1)
    assert np.allclose(sig, np.array(g["sigma_MPa"])[:, :, None], atol=5e-5)


def test_diagnostics_of_an_incompatible_homogeneous_state():
    """Periodic box, u = 0 and a uniform F = I + G with G not symmetric: every axis edge exists and
    its residual is G e_A dx, so the RMS is dx sqrt(sum_A |G e_A|^2 / D) over D N edges; J, |v| and
    the tangent speed are the uniform values."""
    D, n = 3, 6
    G = np.array([[0.02, 0.05, -0.01], [0.0, -0.03, 0.04], [0.07, 0.0, 0.01]])
    v = np.array([0.003, -0.004, 0.012])
    p = _homogeneous(D, n, np.eye(D) + G, v)
    o = oracle.Oracle(p).set_initial()
    d = o.diagnostics()
    N = n ** D
    assert d["n_edges"] == D * N
    expect = p.dx * math.sqrt(sum(np.sum(G[:, A] ** 2) for A in range(D)) / D)
    assert abs(d["incompat_rms"] - expect) < 1e-13
    J = np.linalg.det(np.eye(D) + G)
    assert abs(d["J_min"] - J) < 1e-14 and abs(d["J_max"] - J) < 1e-14
    assert abs(d["v_rms"] - np.linalg.norm(v)) < 1e-15 and abs(d["v_max"] - np.linalg.norm(v)) < 1e-15
    c2 = oracle.tangent_speed2(D, p.mu, p.lam, np.eye(D) + G)
    assert abs(d["c_tangent"] - math.sqrt(c2)) < 1e-14


def test_compatible_linear_state_has_no_residual():
    """A body with u = G (X - c) and F = I + G everywhere: the edge relation holds exactly."""
    D = 2
    p = I.affine_annulus_2d(40)
    G = np.array([[0.04, -0.02], [0.03, 0.01]])
    X = p.coords()
    p.init_mode = "equilibrium"
    p.v0 = np.zeros((D,) + p.box_shape)
    p.F0 = np.stack([np.full(p.box_shape, (np.eye(D) + G)[i, j]) for i in range(D) for j in range(D)])
    p.u0 = np.stack([sum(G[i, j] * (X[j] - 0.5) for j in range(D)) for i in range(D)])
    p.options.gamma = 0.0
    o = oracle.Oracle(p).set_initial()
    d = o.diagnostics()
    assert d["n_edges"] > 0 and d["incompat_rms"] < 1e-15


def test_diagnostics_match_a_direct_sum_over_the_fields():
    """On an evolved random state, the oracle's diagnostics equal the definitions summed by numpy
    over its own output fields (edge residuals over active forward neighbours)."""
    p = I.random_box(3, 14, 2)
    o = oracle.Oracle(p).set_initial()
    o.step(12)
    v, F, u = o.fields()
    act = o.active_mask()
    d = o.diagnostics()
    D = 3
    Fm = np.moveaxis(F.reshape(D, D, *act.shape), (0, 1), (-2, -1))
    J = np.linalg.det(Fm)[act]
    assert abs(d["J_min"] - J.min()) < 1e-13 and abs(d["J_max"] - J.max()) < 1e-13
    speed = np.sqrt((v[:, act] ** 2).sum(0))
    assert abs(d["v_rms"] - math.sqrt((speed ** 2).mean())) < 1e-14
    e2, ne = 0.0, 0
    for A in range(D):
        ax = D - 1 - A                                # arrays are (z, y, x)
        sl_m = [slice(None)] * D
        sl_l = [slice(None)] * D
        sl_m[ax] = slice(0, -1)
        sl_l[ax] = slice(1, None)
        both = act[tuple(sl_m)] & act[tuple(sl_l)]
        for i in range(D):
            Gm = F[i * D + A][tuple(sl_m)] - (i == A)
            Gl = F[i * D + A][tuple(sl_l)] - (i == A)
            e = u[i][tuple(sl_m)] - u[i][tuple(sl_l)] + 0.5 * (Gm + Gl) * p.dx
            e2 += float((e[both] ** 2).sum())
        ne += int(both.sum())
    assert d["n_edges"] == ne
    assert abs(d["incompat_rms"] - math.sqrt(e2 / ne)) < 1e-12 * max(1.0, d["incompat_rms"])
