"""ctypes wrapper of the plain FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is what the CUDA path is checked against.
Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import it.  It takes a problem *description* (see
``paper_2606_20646_b300.inputs``) and converts it into its own C structs; it
imports nothing from the CUDA side.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")

_SHAPE = {"sphere": 0, "ellipsoid": 1, "superellipse": 2, "cylinder": 3, "halfspace": 4, "sampled": 5}
_BCKIND = {"dirichlet": 0, "neumann": 1}
_PROFILE = {"zero": 0, "affine": 1, "radial": 2, "twist_stretch": 3, "const": 4}
_RAMP = {"one": 0, "linear": 1, "sin2": 2, "cos": 3, "time": 4}

MAXS = 16
MAXB = 16


class _Shape(C.Structure):
    _fields_ = [("kind", C.c_int), ("complement", C.c_int), ("bid", C.c_int), ("pad", C.c_int),
                ("c", C.c_double * 3), ("a", C.c_double * 3), ("Q", C.c_double * 9), ("p", C.c_double),
                ("phi", C.c_void_p)]


class _BC(C.Structure):
    _fields_ = [("bid", C.c_int), ("kind", C.c_int), ("profile", C.c_int), ("ramp", C.c_int),
                ("t_ramp", C.c_double), ("center", C.c_double * 3), ("A", C.c_double * 9),
                ("vec", C.c_double * 3), ("amp", C.c_double)]


class _Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("periodic", C.c_int * 3), ("nshapes", C.c_int),
                ("nbc", C.c_int), ("proj_every", C.c_int), ("proj_iters", C.c_int), ("pad", C.c_int),
                ("dx", C.c_double), ("origin", C.c_double * 3), ("mu", C.c_double), ("lam", C.c_double),
                ("c", C.c_double), ("omega", C.c_double), ("gamma", C.c_double), ("theta_F", C.c_double),
                ("beta", C.c_double), ("b", C.c_double * 3),
                ("shapes", _Shape * MAXS), ("bcs", _BC * MAXB)]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64, no FMA contraction) into liblbm_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i, l, vp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_long), C.c_void_p
        _lib.orc_create.restype = vp
        _lib.orc_create.argtypes = [C.POINTER(_Problem), i]
        _lib.orc_destroy.argtypes = [vp]
        _lib.orc_set_initial.argtypes = [vp, C.c_int, d, d, d, d]
        _lib.orc_set_mu_field.argtypes = [vp, d]
        _lib.orc_step.argtypes = [vp, C.c_int]
        _lib.orc_fields.argtypes = [vp, d, d, d]
        _lib.orc_populations.argtypes = [vp, d]
        _lib.orc_counts.argtypes = [vp, l]
        _lib.orc_active_mask.argtypes = [vp, C.POINTER(C.c_ubyte)]
        _lib.orc_links.argtypes = [vp, l, i, d, d, d, i, i, d]
        _lib.orc_link_stencil.argtypes = [vp, C.c_long, l, d]
        _lib.orc_piola.restype = C.c_double
        _lib.orc_piola.argtypes = [C.c_int, C.c_double, C.c_double, d, d]
        _lib.orc_dpiola.argtypes = [C.c_int, C.c_double, C.c_double, d, d, d]
        _lib.orc_feq.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, d, d]
        _lib.orc_collide_node.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, d,
                                          C.c_double, C.c_double, d, d, d]
        _lib.orc_lsq_weights.restype = C.c_int
        _lib.orc_lsq_weights.argtypes = [C.c_int, C.c_int, d, C.c_int, d, C.c_double, d]
        _lib.orc_newton.restype = C.c_int
        _lib.orc_newton.argtypes = [C.c_int, C.c_double, C.c_double, d, d, d, d, d]
        _lib.orc_project.argtypes = [vp, d, d, C.c_double, d]
        _lib.orc_adjoint.argtypes = [vp, C.c_int, d, d, d]
        _lib.orc_stress.argtypes = [vp, d, d]
        _lib.orc_diagnostics.argtypes = [vp, d]
        _lib.orc_tangent_speed2.restype = C.c_double
        _lib.orc_tangent_speed2.argtypes = [C.c_int, C.c_double, C.c_double, d]
        _lib.orc_set_threads.restype = C.c_int
        _lib.orc_set_threads.argtypes = [C.c_int]
        _lib.orc_levelset.restype = C.c_double
        _lib.orc_levelset.argtypes = [C.POINTER(_Problem), d, i]
    return _lib


def set_threads(n: int = 0) -> int:
    """Host threads for the oracle's per-node and per-link loops (0 keeps the current count);
    returns the count in use.  The results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))


def tangent_speed2(D, mu, lam, F):
    """Largest squared tangent wave speed max_n eig Q(n; F) of the neo-Hookean law (rho0 = 1)."""
    F = _f64(np.asarray(F).reshape(-1))
    return float(lib().orc_tangent_speed2(int(D), float(mu), float(lam), _dp(F)))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def problem_struct(p) -> _Problem:
    if getattr(p, "groups", None):
        raise ValueError("the oracle takes one body per problem; run each specimen as its own problem")
    s = _Problem()
    s.dim = p.dim
    for a in range(3):
        s.n[a] = int(p.n[a])
        s.periodic[a] = int(bool(p.periodic[a]))
        s.origin[a] = float(p.origin[a])
    s.nshapes = len(p.shapes)
    s.nbc = len(p.bcs)
    o = p.options
    s.proj_every, s.proj_iters = int(o.proj_every), int(o.proj_iters)
    s.dx, s.mu, s.lam = p.dx, p.mu, p.lam
    s.c, s.omega, s.gamma, s.theta_F, s.beta = o.c, o.omega, o.gamma, o.theta_F, o.proj_beta
    for a in range(3):
        s.b[a] = float(o.body_force[a])
    for j, sh in enumerate(p.shapes):
        t = s.shapes[j]
        t.kind, t.complement, t.bid = _SHAPE[sh.kind], int(sh.complement), int(sh.boundary_id)
        for a in range(3):
            t.c[a], t.a[a] = sh.center[a], sh.axes[a]
        for a in range(9):
            t.Q[a] = float(sh.rot.reshape(-1)[a])
        t.p = sh.p
        if sh.kind == "sampled":
            arr = _f64(sh.phi).reshape(-1)
            assert arr.size == p.n_box
            s._keep = getattr(s, "_keep", []) + [arr]   # the samples live as long as the struct
            t.phi = arr.ctypes.data
    for j, bc in enumerate(p.bcs):
        t = s.bcs[j]
        t.bid, t.kind, t.profile, t.ramp = bc.boundary_id, _BCKIND[bc.kind], _PROFILE[bc.profile], _RAMP[bc.ramp]
        t.t_ramp, t.amp = bc.t_ramp, bc.amp
        for a in range(3):
            t.center[a], t.vec[a] = bc.center[a], bc.vec[a]
        for a in range(9):
            t.A[a] = float(bc.A.reshape(-1)[a])
    return s


class Oracle:
    """One oracle simulation of a problem description."""

    def __init__(self, p):
        self.p = p
        self._s = problem_struct(p)
        err = C.c_int(0)
        self.h = lib().orc_create(C.byref(self._s), C.byref(err))
        if not self.h:
            raise ValueError(f"oracle setup failed (code {err.value})")
        self.D, self.K, self.N = p.dim, p.K, p.n_box

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def set_initial(self):
        p = self.p
        v0, F0, u0 = _f64(p.v0), _f64(p.F0), _f64(p.u0)
        dU = _f64(p.dU0) if p.dU0 is not None else None
        lib().orc_set_initial(self.h, 1 if p.init_mode == "characteristic" else 0, _dp(v0), _dp(F0), _dp(u0),
                              _dp(dU) if dU is not None else None)
        return self

    def step(self, n: int) -> int:
        return lib().orc_step(self.h, int(n))

    def set_mu_field(self, mu):
        """Per-node shear modulus (box-shaped array, box order), replacing p.mu; call before
        set_initial.  None restores p.mu."""
        if mu is None:
            lib().orc_set_mu_field(self.h, None)
        else:
            a = _f64(np.asarray(mu).reshape(-1))
            assert a.size == self.N
            lib().orc_set_mu_field(self.h, _dp(a))
        return self

    def adjoint(self, nsteps: int, grad_u):
        """Runs nsteps steps from the current state and returns the discrete adjoint of a loss
        on u after them: (dL/dmu, box-shaped; dL/db, 3 values), given grad_u = dL/du (D x box).
        Velocity-Dirichlet bodies only."""
        g = _f64(np.asarray(grad_u).reshape(self.D, -1))
        assert g.shape[1] == self.N
        mubar = np.zeros(self.N)
        bbar = np.zeros(3)
        rc = lib().orc_adjoint(self.h, int(nsteps), _dp(g), _dp(mubar), _dp(bbar))
        if rc < 0:
            raise ValueError(f"oracle adjoint refused (code {rc})")
        return mubar.reshape(self.p.box_shape), bbar

    def fields(self):
        D, N = self.D, self.N
        v = np.zeros((D, N))
        F = np.zeros((D * D, N))
        u = np.zeros((D, N))
        lib().orc_fields(self.h, _dp(v), _dp(F), _dp(u))
        bs = self.p.box_shape
        return v.reshape((D,) + bs), F.reshape((D * D,) + bs), u.reshape((D,) + bs)

    def stress(self):
        """Cauchy stress sigma = J^-1 P F^T (D*D, *box) and J = det F (*box) at the current time."""
        D, N = self.D, self.N
        sig = np.zeros((D * D, N))
        J = np.zeros(N)
        lib().orc_stress(self.h, _dp(sig), _dp(J))
        bs = self.p.box_shape
        return sig.reshape((D * D,) + bs), J.reshape(bs)

    def diagnostics(self):
        """J range, RMS and largest |v|, largest tangent wave speed, compatibility residual RMS and
        the number of active axis edges, over the active nodes."""
        out = np.zeros(7)
        lib().orc_diagnostics(self.h, _dp(out))
        return dict(J_min=out[0], J_max=out[1], v_rms=out[2], v_max=out[3], c_tangent=out[4],
                    incompat_rms=out[5], n_edges=int(out[6]))

    def populations(self):
        Q = 2 * self.D
        f = np.zeros((Q * self.K, self.N))
        lib().orc_populations(self.h, _dp(f))
        return f

    def counts(self):
        out = (C.c_long * 6)()
        lib().orc_counts(self.h, out)
        return dict(n_active=out[0], n_cut=out[1], n_neumann=out[2], n_dirichlet=out[3],
                    step=out[4], status=out[5])

    def active_mask(self):
        m = np.zeros(self.N, dtype=np.uint8)
        lib().orc_active_mask(self.h, m.ctypes.data_as(C.POINTER(C.c_ubyte)))
        return m.reshape(self.p.box_shape).astype(bool)

    def project(self, F, u, t=0.0):
        """One compatibility-projection solve on box fields F (D*D, *box) and warm start
        u (D, *box); returns (u^c, F^c)."""
        F = _f64(F).reshape(self.D * self.D, -1)
        uc = _f64(u).reshape(self.D, -1).copy()
        Fc = np.zeros_like(F)
        lib().orc_project(self.h, _dp(F), _dp(uc), float(t), _dp(Fc))
        bs = self.p.box_shape
        return uc.reshape((self.D,) + bs), Fc.reshape((self.D * self.D,) + bs)

    def links(self):
        n = self.counts()["n_cut"]
        m = np.zeros(n, dtype=np.int64)
        q = np.zeros(n, dtype=np.int32)
        eta = np.zeros(n)
        Xb = np.zeros((n, 3))
        Nb = np.zeros((n, 3))
        h = np.zeros((n, 3))
        bid = np.zeros(n, dtype=np.int32)
        ns = np.zeros(n, dtype=np.int32)
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
        lib().orc_links(self.h, m.ctypes.data_as(C.POINTER(C.c_long)), ip(q), _dp(eta), _dp(Xb), _dp(Nb),
                        ip(bid), ip(ns), _dp(h))
        return dict(node=m, q=q, eta=eta, Xb=Xb, Nb=Nb, bid=bid, ns=ns, h=h)

    def link_stencil(self, l: int):
        ns = int(self.links()["ns"][l])
        nodes = np.zeros(max(ns, 1), dtype=np.int64)
        w = np.zeros(max((self.D - 1) * ns, 1))
        lib().orc_link_stencil(self.h, int(l), nodes.ctypes.data_as(C.POINTER(C.c_long)), _dp(w))
        return nodes[:ns], w[: (self.D - 1) * ns].reshape(self.D - 1, ns)


# ----------------------------------------------------------------------------
# point functions (for the pins)
# ----------------------------------------------------------------------------

def piola(D, mu, lam, F):
    F = _f64(F).reshape(-1)
    P = np.zeros(D * D)
    J = lib().orc_piola(D, mu, lam, _dp(F), _dp(P))
    return P.reshape(D, D), J


def dpiola(D, mu, lam, F, Z):
    F, Z = _f64(F).reshape(-1), _f64(Z).reshape(-1)
    dP = np.zeros(D * D)
    lib().orc_dpiola(D, mu, lam, _dp(F), _dp(Z), _dp(dP))
    return dP.reshape(D, D)


def feq(D, c, mu, lam, U):
    U = _f64(U)
    K = D + D * D
    out = np.zeros(2 * D * K)
    lib().orc_feq(D, c, mu, lam, _dp(U), _dp(out))
    return out.reshape(2 * D, K)


def collide_node(D, c, omega, dt, gamma, b, mu, lam, f):
    K = D + D * D
    f = _f64(f).reshape(-1)
    b = _f64(b)
    out = np.zeros_like(f)
    U = np.zeros(K)
    lib().orc_collide_node(D, c, omega, dt, gamma, _dp(b), mu, lam, _dp(f), _dp(out), _dp(U))
    return out.reshape(2 * D, K), U


def lsq_weights(D, xi, tangents, dx):
    xi = _f64(xi)
    ns = xi.shape[0]
    t = np.zeros((len(tangents), 3))
    for a, tv in enumerate(tangents):
        t[a, : len(tv)] = tv
    w = np.zeros(len(tangents) * ns)
    r = lib().orc_lsq_weights(D, ns, _dp(xi.reshape(-1)), len(tangents), _dp(t.reshape(-1)), dx, _dp(w))
    return w.reshape(len(tangents), ns), r


def newton(D, mu, lam, N, g, t, T, h0):
    N3 = np.zeros(3)
    N3[:D] = N
    g3 = np.zeros((2, 3))
    t3 = np.zeros((2, 3))
    for a in range(D - 1):
        g3[a, :D] = g[a]
        t3[a, :D] = t[a]
    T3 = np.zeros(3)
    T3[:D] = T
    h = np.zeros(3)
    h[:D] = h0
    it = lib().orc_newton(D, mu, lam, _dp(N3), _dp(g3.reshape(-1)), _dp(t3.reshape(-1)), _dp(T3), _dp(h))
    return h[:D], it


def levelset(p, X):
    s = problem_struct(p)
    X3 = np.zeros(3)
    X3[: len(X)] = X
    w = C.c_int(0)
    v = lib().orc_levelset(C.byref(s), _dp(X3), C.byref(w))
    return v, w.value
