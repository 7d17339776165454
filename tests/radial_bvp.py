"""Static radial boundary-value problem of the neo-Hookean annulus / spherical shell.

Independent reference for the traction benchmarks (Sec. 4.3, Eqs. radial-map ..
radial-equilibrium-2d; Sec. 5.2, Eqs. spherical-stretches-3d,
spherical-equilibrium-3d).  With x = X_c + r(R) e_R:

    lambda_r = r',  lambda_t = r / R,  J = lambda_r lambda_t^(D-1)
    P_r = mu (lambda_r - 1/lambda_r) + lam/2 (J^2 - 1) / lambda_r
    P_t = mu (lambda_t - 1/lambda_t) + lam/2 (J^2 - 1) / lambda_t
    dP_r/dR + (D-1) (P_r - P_t) / R = 0

integrated as a first-order system in (r, P_r) (lambda_r recovered from P_r by a
scalar Newton solve), with the missing boundary value found by shooting.
Pinned by the values the paper prints for its spherical shell.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import solve_ivp
from scipy.optimize import brentq


def principal(D, mu, lam, lr, lt):
    J = lr * lt ** (D - 1)
    Pr = mu * (lr - 1.0 / lr) + 0.5 * lam * (J * J - 1.0) / lr
    Pt = mu * (lt - 1.0 / lt) + 0.5 * lam * (J * J - 1.0) / lt
    return Pr, Pt, J


def _lambda_r(D, mu, lam, Pr, lt):
    # P_r is strictly increasing in lambda_r > 0: bracket and solve
    f = lambda lr: principal(D, mu, lam, lr, lt)[0] - Pr
    lo, hi = 1e-3, 1.0
    while f(hi) < 0:
        hi *= 2.0
    while f(lo) > 0:
        lo *= 0.5
    return brentq(f, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=200)


def _rhs(D, mu, lam):
    def rhs(R, y):
        r, Pr = y
        lt = r / R
        lr = _lambda_r(D, mu, lam, Pr, lt)
        _, Pt, _ = principal(D, mu, lam, lr, lt)
        return [lr, -(D - 1) * (Pr - Pt) / R]
    return rhs


def integrate(D, mu, lam, Ri, Ro, r_i, Pr_i, R_eval=None):
    sol = solve_ivp(_rhs(D, mu, lam), (Ri, Ro), [r_i, Pr_i], rtol=1e-12, atol=1e-13,
                    method="DOP853", dense_output=True, t_eval=R_eval)
    return sol


def solve(D, mu, lam, Ri, Ro, inner, outer):
    """inner = ('r', r(R_i)) or ('P', P_r(R_i)); outer = ('P', P_r(R_o)).
    Returns dict with the dense solution and derived quantities."""
    kind_i, val_i = inner
    kind_o, val_o = outer
    assert kind_o == "P"
    if kind_i == "r":
        g = lambda Pr_i: integrate(D, mu, lam, Ri, Ro, val_i, Pr_i).y[1, -1] - val_o
        a, b = -0.5, 0.5
        while g(a) * g(b) > 0:
            a, b = a * 2.0, b * 2.0
        Pr_i = brentq(g, a, b, xtol=1e-14, rtol=1e-14)
        r_i = val_i
    else:
        g = lambda r_i: integrate(D, mu, lam, Ri, Ro, r_i, val_i).y[1, -1] - val_o
        a, b = 0.6 * Ri, 1.6 * Ri
        r_i = brentq(g, a, b, xtol=1e-14, rtol=1e-14)
        Pr_i = val_i
    sol = integrate(D, mu, lam, Ri, Ro, r_i, Pr_i)
    Rs = np.linspace(Ri, Ro, 401)
    r, Pr = sol.sol(Rs)
    lt = r / Rs
    lr = np.array([_lambda_r(D, mu, lam, P, l) for P, l in zip(Pr, lt)])
    J = lr * lt ** (D - 1)
    return dict(sol=sol, R=Rs, r=r, Pr=Pr, lr=lr, lt=lt, J=J, r_i=r_i, Pr_i=Pr_i, r_o=r[-1])


def displacement_field(res, coords, center):
    """Radial displacement u = (r(R) - R) e_R evaluated at node coordinates (R clipped to
    [R_i, R_o]); returns an array shaped like the coordinate list."""
    D = len(coords)
    d = [coords[a] - center[a] for a in range(D)]
    R = np.sqrt(sum(x * x for x in d))
    Rc = np.clip(R, res["R"][0], res["R"][-1])
    r = res["sol"].sol(Rc.reshape(-1))[0].reshape(R.shape)
    Rs = np.where(R > 0, R, 1.0)
    return np.stack([(r - Rc) * d[a] / Rs for a in range(D)])


def reference_fields(res, coords, center, mu, lam):
    """Displacement, deformation gradient and Cauchy stress of the radial solution at node
    coordinates: u = (r - R) e_R, F = lambda_r e_R (x) e_R + lambda_t (I - e_R (x) e_R)
    (Eq. spherical-stretches-3d and its 2D reduction), sigma = J^-1 P F^T
    (Eq. cauchy-recovery-general) with the neo-Hookean P.  Arrays are (comp, *box) with F and sigma
    row-major; lambda_r is interpolated from the solution's dense table."""
    D = len(coords)
    d = [coords[a] - center[a] for a in range(D)]
    R = np.sqrt(sum(x * x for x in d))
    Rc = np.clip(R, res["R"][0], res["R"][-1])
    Rs = np.where(R > 0, R, 1.0)
    e = [x / Rs for x in d]
    r = res["sol"].sol(Rc.reshape(-1))[0].reshape(R.shape)
    Rt = np.linspace(res["R"][0], res["R"][-1], 4001)
    rt, Pt = res["sol"].sol(Rt)
    lr_t = np.array([_lambda_r(D, mu, lam, P, l) for P, l in zip(Pt, rt / Rt)])
    lr = np.interp(Rc, Rt, lr_t)
    lt = r / Rc
    u = np.stack([(r - Rc) * e[a] for a in range(D)])
    F = np.stack([lr * e[i] * e[j] + lt * ((1.0 if i == j else 0.0) - e[i] * e[j])
                  for i in range(D) for j in range(D)])
    return u, F, cauchy(F, mu, lam)


def cauchy(F, mu, lam):
    """sigma = J^-1 P F^T for the neo-Hookean law, P = mu F + (lam/2 (J^2 - 1) - mu) F^-T, i.e.
    sigma = J^-1 (mu F F^T + (lam/2 (J^2 - 1) - mu) I); F given as (D*D, ...) row-major."""
    D = int(round(np.sqrt(F.shape[0])))
    Fm = np.moveaxis(F.reshape((D, D) + F.shape[1:]), (0, 1), (-2, -1))
    J = np.linalg.det(Fm)
    B = Fm @ np.swapaxes(Fm, -1, -2)
    s = (0.5 * lam * (J * J - 1.0) - mu)[..., None, None] * np.eye(D)
    sig = (mu * B + s) / J[..., None, None]
    return np.moveaxis(sig, (-2, -1), (0, 1)).reshape(F.shape)
