"""Seeded, synthetic problem descriptions for the total-Lagrangian vectorial LBM.

This module only *describes* problems: lattice box, level-set primitives,
material constants, boundary data, solver options and initial fields.  It
holds none of the method's arithmetic (no equilibrium, collision, closure or
projection), so both the CUDA path and the CPU oracle can be fed the same
inputs without sharing any code.  Each side translates the description into
its own structures.

Conventions
-----------
* Nodes are cell centred: ``X_i = origin + (i + 1/2) dx`` (the reading that
  reproduces the active/cut-link counts printed in Tables 1-2 of the paper).
* Box fields are numpy arrays of shape ``(comp, nz, ny, nx)`` in 3D and
  ``(comp, ny, nx)`` in 2D, x fastest.  Node linear index ``x + nx*(y + ny*z)``.
* State ordering follows Eq. (state-general-d): ``U = (v_1..v_D, F_11, F_12,
  .., F_DD)`` with F row-major.
* The body is the intersection (max) of the level sets of its shapes,
  Eq. (level-set-domain); a shape with ``complement=True`` contributes ``-phi``.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

SHAPE_KINDS = ("sphere", "ellipsoid", "superellipse", "cylinder", "halfspace", "sampled")
BC_KINDS = ("dirichlet", "neumann")
BC_PROFILES = ("zero", "affine", "radial", "twist_stretch", "const")
RAMPS = ("one", "linear", "sin2", "cos", "time")


def rot_z(deg: float) -> np.ndarray:
    a = math.radians(deg)
    return np.array([[math.cos(a), -math.sin(a), 0.0],
                     [math.sin(a), math.cos(a), 0.0],
                     [0.0, 0.0, 1.0]])


def rot_y(deg: float) -> np.ndarray:
    a = math.radians(deg)
    return np.array([[math.cos(a), 0.0, math.sin(a)],
                     [0.0, 1.0, 0.0],
                     [-math.sin(a), 0.0, math.cos(a)]])


@dataclass
class Shape:
    """One level-set primitive; local coordinates are ``xi = rot^T (X - center)``.

    sphere:       phi = |X - c| - axes[0]                      (circle in 2D)
    ellipsoid:    phi = sum_a (xi_a / axes[a])^2 - 1           (ellipse in 2D)
    superellipse: phi = |xi_1/axes[0]|^p + |xi_2/axes[1]|^p - 1 (2D only)
    cylinder:     phi = |(X_1, X_2) - (c_1, c_2)| - axes[0]     (axis along X_3)
    halfspace:    phi = axes . (X - c)   (axes = unit outward normal)
    sampled:      phi given at the lattice nodes (``phi``, box-shaped); between nodes the
                  multilinear interpolant (linear along every link)
    """
    kind: str
    center: Sequence[float] = (0.0, 0.0, 0.0)
    axes: Sequence[float] = (1.0, 1.0, 1.0)
    rot: np.ndarray = field(default_factory=lambda: np.eye(3))
    p: float = 2.0
    complement: bool = False
    boundary_id: int = 0
    phi: Optional[np.ndarray] = None   # sampled: node values, box-shaped

    def __post_init__(self):
        assert self.kind in SHAPE_KINDS, self.kind
        assert (self.kind == "sampled") == (self.phi is not None), "node samples go with the sampled kind"
        self.center = tuple(float(x) for x in self.center) + (0.0,) * (3 - len(self.center))
        self.axes = tuple(float(x) for x in self.axes) + (1.0,) * (3 - len(self.axes))
        self.rot = np.asarray(self.rot, dtype=np.float64).reshape(3, 3)


@dataclass
class BC:
    """Boundary data for the cut links whose boundary point carries ``boundary_id``.

    dirichlet profiles (prescribed displacement u_D; the lattice sees v_D = du_D/dt):
      zero:          u_D = 0
      affine:        u_D = s(t) A (X - center)
      radial:        u_D = amp s(t) e_R,  e_R = (X - center)/|X - center|
      twist_stretch: u_D = ((R_{s(t) amp} - I) X_perp, s(t) vec[2])  (3D, axis X_3)
      const:         u_D = s(t) vec  (translation)
    neumann profiles (nominal traction T = P N):
      const:         T = s(t) vec
      radial:        T = amp s(t) e_R
    ramps s(t): one (1), linear (t/T_r, then 1), sin2 (sin^2(pi t / 2T_r), then 1),
      cos ((1 - cos(pi t/T_r))/2, then 1), time (t).
    """
    boundary_id: int
    kind: str
    profile: str
    ramp: str = "one"
    t_ramp: float = 1.0
    center: Sequence[float] = (0.0, 0.0, 0.0)
    A: np.ndarray = field(default_factory=lambda: np.zeros((3, 3)))
    vec: Sequence[float] = (0.0, 0.0, 0.0)
    amp: float = 0.0

    def __post_init__(self):
        assert self.kind in BC_KINDS and self.profile in BC_PROFILES and self.ramp in RAMPS
        self.center = tuple(float(x) for x in self.center) + (0.0,) * (3 - len(self.center))
        self.vec = tuple(float(x) for x in self.vec) + (0.0,) * (3 - len(self.vec))
        A = np.zeros((3, 3))
        a = np.asarray(self.A, dtype=np.float64)
        A[: a.shape[0], : a.shape[1]] = a
        self.A = A


@dataclass
class Group:
    """One specimen of a multi-specimen body: shapes[first_shape : first_shape + nshapes] (their
    max is the specimen's level set), a box [lo, hi] containing it, and its material."""
    first_shape: int
    nshapes: int
    lo: Sequence[float]
    hi: Sequence[float]
    mu: float
    lam: float

    def __post_init__(self):
        self.lo = tuple(float(x) for x in self.lo) + (0.0,) * (3 - len(self.lo))
        self.hi = tuple(float(x) for x in self.hi) + (0.0,) * (3 - len(self.hi))


@dataclass
class Options:
    c: float = 10.0            # lattice speed dx/dt
    omega: float = 1.8         # BGK relaxation, 0 < omega < 2
    gamma: float = 0.0         # velocity-proportional damping B = (-gamma v, 0)
    theta_F: float = 1.0       # deformation-gradient repair weight
    proj_every: int = 20       # compatibility projection cadence (steps) when Neumann links exist
    proj_iters: int = 50       # damped-Jacobi sweeps per projection solve
    proj_beta: float = 2.0 / 3.0  # Jacobi damping
    body_force: Sequence[float] = (0.0, 0.0, 0.0)
    c_audit: float = 0.0       # wave-speed audit factor: c >= c_audit * largest tangent speed (0: 2.5, < 0: off)


@dataclass
class Problem:
    name: str
    dim: int
    n: Sequence[int]
    dx: float
    origin: Sequence[float]
    periodic: Sequence[bool]
    mu: float
    lam: float
    options: Options
    shapes: List[Shape] = field(default_factory=list)
    bcs: List[BC] = field(default_factory=list)
    groups: List[Group] = field(default_factory=list)   # several disjoint specimens (empty: one body)
    init_mode: str = "equilibrium"          # or "characteristic"
    v0: Optional[np.ndarray] = None         # (D, *box)
    F0: Optional[np.ndarray] = None         # (D*D, *box)
    u0: Optional[np.ndarray] = None         # (D, *box)
    dU0: Optional[np.ndarray] = None        # (D*K, *box): d U0_k / d X_A at [A*K + k]
    steps: int = 0                          # nominal run length of the workload
    meta: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return self.dim + self.dim * self.dim

    @property
    def Q(self) -> int:
        return 2 * self.dim

    @property
    def dt(self) -> float:
        return self.dx / self.options.c

    @property
    def box_shape(self):
        nx, ny, nz = self.n
        return (ny, nx) if self.dim == 2 else (nz, ny, nx)

    @property
    def n_box(self) -> int:
        return int(np.prod(self.box_shape))

    def coords(self):
        """Node coordinates as a list of D arrays of box shape (cell-centred)."""
        axes = [self.origin[a] + (np.arange(self.n[a]) + 0.5) * self.dx for a in range(self.dim)]
        grids = np.meshgrid(*axes[::-1], indexing="ij")  # (z,y,x) or (y,x)
        return [grids[::-1][a] for a in range(self.dim)]

    def with_(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def _identity_F(dim, box_shape):
    F = np.zeros((dim * dim,) + tuple(box_shape))
    for i in range(dim):
        F[i * dim + i] = 1.0
    return F


def _rest_fields(p: Problem) -> Problem:
    D = p.dim
    p.v0 = np.zeros((D,) + p.box_shape)
    p.u0 = np.zeros((D,) + p.box_shape)
    p.F0 = _identity_F(D, p.box_shape)
    return p


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def shear_wave_2d(n: int = 64, amp: float = 0.01, mu: float = 1.0, lam: float = 2.0,
                  c: float = 10.0, omega: float = 2.0, t_end: float = 3.125) -> Problem:
    """Periodic square L=1, v_2 = amp sin(2 pi X_1), F = I (2D FP64 workload, 64x64 nominal).

    For this neo-Hookean law F = I + g e_2 (x) e_1 has J = 1 and P linear in g, so
    v_2 = amp sin(kX) cos(k t sqrt(mu)), F_21 = amp/sqrt(mu) cos(kX) sin(k t sqrt(mu))
    is an exact finite-amplitude solution (Sec. 2.1-2.2, Eq. validation-nh-energy).
    Characteristic initialisation (Eq. init-general-d) with the analytic gradient.
    """
    dx = 1.0 / n
    p = Problem(name=f"shear_wave_2d_{n}", dim=2, n=(n, n, 1), dx=dx, origin=(0.0, 0.0, 0.0),
                periodic=(True, True, True), mu=mu, lam=lam,
                options=Options(c=c, omega=omega, gamma=0.0, proj_every=0),
                init_mode="characteristic")
    _rest_fields(p)
    X, _Y = p.coords()
    k = 2.0 * math.pi
    p.v0[1] = amp * np.sin(k * X)
    K = p.K
    p.dU0 = np.zeros((2 * K,) + p.box_shape)
    p.dU0[0 * K + 1] = amp * k * np.cos(k * X)       # d v_2 / d X_1
    p.steps = int(round(t_end / p.dt))
    p.meta = dict(amp=amp, k=k, t_end=t_end)
    return p


def shear_wave_exact(p: Problem, t: float):
    """Exact (v_2, F_21) of :func:`shear_wave_2d` at time t."""
    X, _ = p.coords()
    k, amp = p.meta["k"], p.meta["amp"]
    cs = math.sqrt(p.mu)
    v2 = amp * np.sin(k * X) * np.cos(k * cs * t)
    F21 = amp / cs * np.cos(k * X) * np.sin(k * cs * t)
    return v2, F21


def annulus_radial_2d(n: int = 512, steps: Optional[int] = None, ramp_steps: int = 5000,
                      omega: float = 1.5) -> Problem:
    """2D FP32 workload: annulus R_i=0.3, R_o=1.0 in a 2.2-wide box, inner radial
    displacement 0.2 (sin^2 ramp over ``ramp_steps`` steps of the 512^2 lattice),
    outer surface traction-free, mu=1, lambda=10, c=10, gamma=10, projection every 20 steps.
    omega = 1.5: with the traction benchmarks' 1.8 this stiff body (lambda = 10) blows up at the
    inner Dirichlet surface soon after the ramp from 256^2 on (the oracle and both GPU forms
    alike); 1.5 adds the BGK dissipation that keeps it stable."""
    L = 2.2
    dx = L / n
    p = Problem(name=f"annulus_radial_2d_{n}", dim=2, n=(n, n, 1), dx=dx,
                origin=(-L / 2, -L / 2, 0.0), periodic=(False, False, False), mu=1.0, lam=10.0,
                options=Options(c=10.0, omega=omega, gamma=10.0))
    t_ramp = ramp_steps * (L / 512) / 10.0
    p.shapes = [Shape("sphere", (0, 0), (1.0,), boundary_id=1),
                Shape("sphere", (0, 0), (0.3,), complement=True, boundary_id=0)]
    p.bcs = [BC(0, "dirichlet", "radial", ramp="sin2", t_ramp=t_ramp, center=(0, 0), amp=0.2),
             BC(1, "neumann", "const", vec=(0, 0))]
    _rest_fields(p)
    p.steps = steps if steps is not None else int(round(5.0 * t_ramp / p.dt))
    p.meta = dict(R_i=0.3, R_o=1.0, u_inner=0.2, t_ramp=t_ramp)
    return p


def shell_3d(n: int = 256, steps: Optional[int] = None, p_in: float = 1.0, omega: float = 1.8) -> Problem:
    """3D FP32 workload: thick spherical shell R_i=0.4, R_o=0.9 in [-1,1]^3, mu=1, lambda=5,
    inner nominal traction p s(t) e_R (sin^2 ramp, T_r=2), outer traction-free,
    c=10, omega=1.8 (the paper's setting for traction benchmarks), gamma=10, projection every 20
    steps.  4000 steps at 256^3 reach t = 3.125.  At omega = 1.8 the 256^3 shell blows up soon
    after the ramp (steps 2500-3000, both forms); omega = 1.5 runs the whole length."""
    dx = 2.0 / n
    p = Problem(name=f"shell_3d_{n}", dim=3, n=(n, n, n), dx=dx, origin=(-1.0, -1.0, -1.0),
                periodic=(False, False, False), mu=1.0, lam=5.0,
                options=Options(c=10.0, omega=omega, gamma=10.0))
    p.shapes = [Shape("sphere", (0, 0, 0), (0.9,), boundary_id=1),
                Shape("sphere", (0, 0, 0), (0.4,), complement=True, boundary_id=0)]
    p.bcs = [BC(0, "neumann", "radial", ramp="sin2", t_ramp=2.0, center=(0, 0, 0), amp=p_in),
             BC(1, "neumann", "const", vec=(0, 0, 0))]
    _rest_fields(p)
    # 4000 steps at 256^3 reach t = 3.125; smaller copies run to the same time.
    p.steps = steps if steps is not None else int(round(3.125 / p.dt))
    p.meta = dict(R_i=0.4, R_o=0.9, p_in=p_in)
    return p


def affine_annulus_2d(N: int) -> Problem:
    """Affine Dirichlet annulus (Sec. 4.2): unit square, centre (0.5,0.5), R_i=0.18, R_o=0.42,
    u = (t/T) A (X - X_c), T=0.2, A=[[0.35,0.18],[-0.10,0.24]], omega=2.0, both surfaces Dirichlet."""
    A = np.array([[0.35, 0.18], [-0.10, 0.24]])
    T = 0.2
    dx = 1.0 / N
    p = Problem(name=f"affine_annulus_{N}", dim=2, n=(N, N, 1), dx=dx, origin=(0, 0, 0),
                periodic=(False, False, False), mu=1.0, lam=2.0 / 3.0,
                options=Options(c=10.0, omega=2.0, gamma=0.0), init_mode="characteristic")
    xc = (0.5, 0.5)
    p.shapes = [Shape("sphere", xc, (0.42,), boundary_id=0),
                Shape("sphere", xc, (0.18,), complement=True, boundary_id=0)]
    p.bcs = [BC(0, "dirichlet", "affine", ramp="linear", t_ramp=T, center=xc, A=A)]
    _rest_fields(p)
    X, Y = p.coords()
    p.v0[0] = (A[0, 0] * (X - 0.5) + A[0, 1] * (Y - 0.5)) / T
    p.v0[1] = (A[1, 0] * (X - 0.5) + A[1, 1] * (Y - 0.5)) / T
    K = p.K
    p.dU0 = np.zeros((2 * K,) + p.box_shape)
    for Aax in range(2):
        for i in range(2):
            p.dU0[Aax * K + i] = A[i, Aax] / T
    p.steps = int(round(T / p.dt))
    p.meta = dict(A=A, T=T, xc=xc)
    return p


def radial_traction_annulus_2d(N: int, t_end: float = 5.0) -> Problem:
    """Radial traction annulus geometry (Sec. 4.3): inner circle clamped, outer nominal
    traction p0 s(t) e_R with p0=1, sin^2 ramp T_r=2, mu=1, lambda=2/3, omega=1.8, gamma=10."""
    dx = 1.0 / N
    p = Problem(name=f"radial_annulus_{N}", dim=2, n=(N, N, 1), dx=dx, origin=(0, 0, 0),
                periodic=(False, False, False), mu=1.0, lam=2.0 / 3.0,
                options=Options(c=10.0, omega=1.8, gamma=10.0))
    xc = (0.5, 0.5)
    p.shapes = [Shape("sphere", xc, (0.42,), boundary_id=1),
                Shape("sphere", xc, (0.18,), complement=True, boundary_id=0)]
    p.bcs = [BC(0, "dirichlet", "zero"),
             BC(1, "neumann", "radial", ramp="sin2", t_ramp=2.0, center=xc, amp=1.0)]
    _rest_fields(p)
    p.steps = int(round(t_end / p.dt))
    p.meta = dict(R_i=0.18, R_o=0.42, p0=1.0, xc=xc)
    return p


def superellipse_shell_2d(N: int) -> Problem:
    """Rotated superellipse shell (Sec. 4.4): outer a=0.42,b=0.30,theta=20deg, inner a=0.16,
    b=0.10, theta=-15deg, p=4, centre (0.5,0.5); inner clamped, outer T = s(t)(0, 0.125)."""
    dx = 1.0 / N
    p = Problem(name=f"superellipse_{N}", dim=2, n=(N, N, 1), dx=dx, origin=(0, 0, 0),
                periodic=(False, False, False), mu=1.0, lam=2.0 / 3.0,
                options=Options(c=10.0, omega=1.8, gamma=10.0))
    xc = (0.5, 0.5)
    p.shapes = [Shape("superellipse", xc, (0.42, 0.30), rot=rot_z(20.0), p=4.0, boundary_id=1),
                Shape("superellipse", xc, (0.16, 0.10), rot=rot_z(-15.0), p=4.0,
                      complement=True, boundary_id=0)]
    p.bcs = [BC(0, "dirichlet", "zero"),
             BC(1, "neumann", "const", ramp="sin2", t_ramp=2.0, vec=(0.0, 0.125))]
    _rest_fields(p)
    p.steps = int(round(20.0 / p.dt))
    return p


def ellipsoid_3d(N: int) -> Problem:
    """Rotated ellipsoid with affine Dirichlet data (Sec. 5.1): centre 0.5, semi-axes
    (0.34,0.25,0.18), Q = R_z(25) R_y(18), u = t A (X - X_c), T=0.4599, omega=1.8."""
    A = np.array([[0.0, 0.80, 0.0], [0.0, 0.0, -0.60], [0.45, 0.0, 0.08]])
    T = 0.4599
    dx = 1.0 / N
    p = Problem(name=f"ellipsoid_{N}", dim=3, n=(N, N, N), dx=dx, origin=(0, 0, 0),
                periodic=(False, False, False), mu=1.0, lam=2.0 / 3.0,
                options=Options(c=10.0, omega=1.8, gamma=0.0), init_mode="characteristic")
    xc = (0.5, 0.5, 0.5)
    p.shapes = [Shape("ellipsoid", xc, (0.34, 0.25, 0.18), rot=rot_z(25.0) @ rot_y(18.0), boundary_id=0)]
    p.bcs = [BC(0, "dirichlet", "affine", ramp="time", center=xc, A=A)]
    _rest_fields(p)
    X = p.coords()
    K = p.K
    p.dU0 = np.zeros((3 * K,) + p.box_shape)
    for i in range(3):
        p.v0[i] = sum(A[i, j] * (X[j] - 0.5) for j in range(3))
        for Aax in range(3):
            p.dU0[Aax * K + i] = A[i, Aax]
    p.steps = int(round(T / p.dt))
    p.meta = dict(A=A, T=T, xc=xc)
    return p


def sphere_shell_paper_3d(N: int, t_end: float = 5.0) -> Problem:
    """Spherical shell of Sec. 5.2: centre 0.5, R_i=0.20, R_o=0.38, mu=1, lambda=2/3, both
    surfaces Neumann; inner traction 1.15242 s(t) e_R (the level matching r(R_i)=0.28)."""
    dx = 1.0 / N
    p = Problem(name=f"sphere_shell_{N}", dim=3, n=(N, N, N), dx=dx, origin=(0, 0, 0),
                periodic=(False, False, False), mu=1.0, lam=2.0 / 3.0,
                options=Options(c=10.0, omega=1.8, gamma=10.0))
    xc = (0.5, 0.5, 0.5)
    p.shapes = [Shape("sphere", xc, (0.38,), boundary_id=1),
                Shape("sphere", xc, (0.20,), complement=True, boundary_id=0)]
    p.bcs = [BC(0, "neumann", "radial", ramp="sin2", t_ramp=2.0, center=xc, amp=1.1524206),
             BC(1, "neumann", "const")]
    _rest_fields(p)
    p.steps = int(round(t_end / p.dt))
    return p


def sampled_copy(p: Problem) -> Problem:
    """The same body with each sphere/circle primitive replaced by its node samples: the signed
    distance |X - c| - R (negated for a complement) at the lattice nodes, given as a sampled level
    set with the primitive's boundary id."""
    X = p.coords()
    shapes = []
    for sh in p.shapes:
        assert sh.kind == "sphere", "sampled copies are made of sphere/circle bodies"
        r = np.sqrt(sum((X[a] - sh.center[a]) ** 2 for a in range(p.dim)))
        shapes.append(Shape("sampled", complement=sh.complement, boundary_id=sh.boundary_id,
                            phi=np.ascontiguousarray(r - sh.axes[0])))
    q = dataclasses.replace(p, name=p.name + "_sampled", shapes=shapes)
    return q


def tube_3d(nxy: int = 76, nz: int = 300, dx: float = 0.01) -> Problem:
    """Finite tube (Sec. 5.3): R_i=0.15, R_o=0.30 about (0.38,0.38), 0<=Z<=L=3; walls
    traction-free, Z=0 clamped, Z=L stretch 50% + twist 45deg with the cosine ramp T_r=10."""
    L = nz * dx
    p = Problem(name=f"tube_{nxy}x{nxy}x{nz}", dim=3, n=(nxy, nxy, nz), dx=dx, origin=(0, 0, 0),
                periodic=(False, False, False), mu=1.0, lam=2.0 / 3.0,
                options=Options(c=10.0, omega=1.8, gamma=10.0))
    xc = (0.38, 0.38, 0.0)
    p.shapes = [Shape("cylinder", xc, (0.30,), boundary_id=1),
                Shape("cylinder", xc, (0.15,), complement=True, boundary_id=1),
                Shape("halfspace", (0, 0, 0), (0, 0, -1), boundary_id=2),
                Shape("halfspace", (0, 0, L), (0, 0, 1), boundary_id=3)]
    p.bcs = [BC(1, "neumann", "const"),
             BC(2, "dirichlet", "zero"),
             BC(3, "dirichlet", "twist_stretch", ramp="cos", t_ramp=10.0, center=xc,
                amp=math.radians(45.0), vec=(0.0, 0.0, 0.5 * L))]
    _rest_fields(p)
    p.steps = int(round(100.0 / p.dt))
    return p


def rigid_translation(dim: int, anchored: bool, n: Optional[int] = None, proj_every: int = 5,
                      steps: int = 23) -> Problem:
    """A disc (2D) or ball (3D) of radius 0.37 in the unit box moving at the uniform velocity
    vt = (0.01, -0.02, 0.015) with F = I, its surface traction-free; with `anchored`, a hole of
    radius 0.15 whose surface carries the Dirichlet translation u_D = t vt.  u = vt t, v = vt, F = I
    is the exact solution (P(I) = 0, zero tractions), kept through projection steps every
    `proj_every` steps."""
    n = n if n is not None else (40 if dim == 2 else 20)
    p = Problem(name=f"rigid_translation_{dim}d{'_anchored' if anchored else ''}", dim=dim,
                n=(n, n, n if dim == 3 else 1), dx=1.0 / n, origin=(0.0, 0.0, 0.0),
                periodic=(False, False, False), mu=1.0, lam=2.0,
                options=Options(c=10.0, omega=1.8, gamma=0.0, proj_every=proj_every))
    c = (0.5, 0.5, 0.5)
    vt = np.array([0.01, -0.02, 0.015])[:dim]
    p.shapes = [Shape("sphere", c, (0.37,), boundary_id=1)]
    p.bcs = [BC(1, "neumann", "const", vec=(0.0, 0.0, 0.0))]
    if anchored:
        p.shapes.append(Shape("sphere", c, (0.15,), complement=True, boundary_id=0))
        p.bcs.append(BC(0, "dirichlet", "const", ramp="time", vec=tuple(vt)))
    _rest_fields(p)
    for i in range(dim):
        p.v0[i] = vt[i]
    p.steps = steps
    p.meta = dict(vt=vt)
    return p


def random_periodic(dim: int, n: int, seed: int, amp: float = 0.02, mu: float = 1.0,
                    lam: float = 3.0, omega: float = 1.7, gamma: float = 0.0,
                    body_force=(0.0, 0.0, 0.0), init_mode: str = "equilibrium") -> Problem:
    """Periodic box with seeded smooth random v0 and F0 = I + small random smooth field
    (low Fourier modes), for parity runs with no embedded boundary."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / n
    p = Problem(name=f"random_periodic_{dim}d_{n}_{seed}", dim=dim,
                n=(n, n, n if dim == 3 else 1), dx=dx, origin=(0, 0, 0),
                periodic=(True, True, True), mu=mu, lam=lam,
                options=Options(c=10.0, omega=omega, gamma=gamma, proj_every=0,
                                body_force=tuple(body_force)), init_mode=init_mode)
    _rest_fields(p)
    X = p.coords()

    def smooth():
        out = np.zeros(p.box_shape)
        for _ in range(3):
            kvec = rng.integers(-2, 3, size=dim)
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.normal()
            out += a * np.sin(2 * math.pi * sum(int(kvec[j]) * X[j] for j in range(dim)) + ph)
        return out

    for i in range(dim):
        p.v0[i] = amp * smooth()
    for k in range(dim * dim):
        p.F0[k] += 0.5 * amp * smooth()
    return p


def random_box(dim: int, n: int, seed: int, precision_note: str = "") -> Problem:
    """Seeded random embedded body (ellipse/ellipsoid with one complemented ellipse hole),
    mixed Dirichlet (hole, affine ramp) and Neumann (outer, constant traction) boundaries,
    a ragged box (n, n+3, n+5), for parity runs that exercise every closure branch."""
    rng = np.random.default_rng(seed)
    dims = (n, n + 3, n + 5) if dim == 3 else (n, n + 3, 1)
    dx = 1.0 / n
    ext = [dims[a] * dx for a in range(dim)]
    ctr = tuple(0.5 * e for e in ext)
    R = rot_z(rng.uniform(0, 90)) @ (rot_y(rng.uniform(0, 90)) if dim == 3 else np.eye(3))
    outer_axes = tuple(0.5 * min(ext) * rng.uniform(0.75, 0.9) for _ in range(dim))
    inner_axes = tuple(a * rng.uniform(0.3, 0.4) for a in outer_axes)
    p = Problem(name=f"random_box_{dim}d_{n}_{seed}", dim=dim, n=dims, dx=dx, origin=(0, 0, 0),
                periodic=(False, False, False), mu=1.0, lam=float(rng.uniform(1.0, 5.0)),
                options=Options(c=10.0, omega=1.8, gamma=10.0, proj_every=5, proj_iters=20))
    p.shapes = [Shape("ellipsoid", ctr, outer_axes, rot=R, boundary_id=1),
                Shape("ellipsoid", ctr, inner_axes, rot=R.T, complement=True, boundary_id=0)]
    A = rng.uniform(-0.2, 0.2, size=(3, 3))
    if dim == 2:
        A[2, :] = 0
        A[:, 2] = 0
    tr = rng.uniform(-0.05, 0.05, size=3)
    if dim == 2:
        tr[2] = 0
    p.bcs = [BC(0, "dirichlet", "affine", ramp="sin2", t_ramp=0.05, center=ctr, A=A),
             BC(1, "neumann", "const", ramp="sin2", t_ramp=0.05, vec=tuple(tr))]
    _rest_fields(p)
    return p


def face_touching_box(dim: int, n: int, seed: int) -> Problem:
    """Seeded axis-aligned ellipsoidal body whose surface passes between the outermost node centres
    and every box face (semi-axes = half box extent - 0.2 dx), so active nodes lie on all the box
    faces and their links across the faces are cut links to the outside of the box.  A seeded
    elliptic hole carries affine Dirichlet data, the outer surface a constant Neumann traction;
    ragged box (n, n+3, n+5).  For parity runs of box-face cut links."""
    rng = np.random.default_rng(seed)
    dims = (n, n + 3, n + 5) if dim == 3 else (n, n + 3, 1)
    dx = 1.0 / n
    ext = [dims[a] * dx for a in range(dim)]
    ctr = tuple(0.5 * e for e in ext)
    outer_axes = tuple(0.5 * e - 0.2 * dx for e in ext)
    inner_axes = tuple(0.5 * min(ext) * rng.uniform(0.25, 0.35) for _ in range(dim))
    R = rot_z(rng.uniform(0, 90)) @ (rot_y(rng.uniform(0, 90)) if dim == 3 else np.eye(3))
    p = Problem(name=f"face_touching_{dim}d_{n}_{seed}", dim=dim, n=dims, dx=dx, origin=(0, 0, 0),
                periodic=(False, False, False), mu=1.0, lam=float(rng.uniform(1.0, 5.0)),
                options=Options(c=10.0, omega=1.8, gamma=10.0, proj_every=5, proj_iters=20))
    p.shapes = [Shape("ellipsoid", ctr, outer_axes, boundary_id=1),
                Shape("ellipsoid", ctr, inner_axes, rot=R, complement=True, boundary_id=0)]
    A = rng.uniform(-0.2, 0.2, size=(3, 3))
    if dim == 2:
        A[2, :] = 0
        A[:, 2] = 0
    tr = rng.uniform(-0.05, 0.05, size=3)
    if dim == 2:
        tr[2] = 0
    p.bcs = [BC(0, "dirichlet", "affine", ramp="sin2", t_ramp=0.05, center=ctr, A=A),
             BC(1, "neumann", "const", ramp="sin2", t_ramp=0.05, vec=tuple(tr))]
    _rest_fields(p)
    return p


def batch_2d(n_spec: int = 96, seed: int = 20260646, side: Sequence[int] = (64, 768), dx: float = 1.0 / 256,
             width: int = 4992, gap: int = 12, steps: int = 1000, margin: int = 8, t_ramp: float = 0.3,
             stretch: float = 0.02):
    """Many 2D specimens of uneven size packed into one box and advanced as one body (a level set
    with one group per specimen, each with its own material).

    Specimen k: a square of s_k ~ U{side} nodes per edge, with 1-5 elliptic holes (semi-axes
    U[0.05, 0.2] L, random centres and angles, kept apart from each other and from the edges by
    rejection), mu ~ U[0.5, 2], lambda/mu ~ U[1, 20].  Left edge clamped (Dirichlet zero), right
    edge translated by (stretch, 0) with a sin^2 ramp over t_ramp (Dirichlet translation), top, bottom and holes
    traction-free (Neumann zero); omega = 1.8, gamma = 10, projection every 20 steps; lattice speed
    c = max(10, 2.5 max_k sqrt(lambda_k + 2 mu_k)), shared by all specimens.  Specimens
    are shelf-packed left to right, `gap` nodes apart (beyond the 3 dx reach of the LSQ stencils),
    in a box `width` nodes wide.

    Returns (packed problem, [(specimen problem, (i0, j0)) ...]): each specimen problem is the same
    specimen alone in its own box, whose node (0, 0) is node (i0, j0) of the packed box, so the two
    runs see identical node coordinates."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side[0], side[1] + 1, size=n_spec)
    order = np.argsort(-sides, kind="stable")
    # shelf packing (largest first)
    place = {}
    x = y = gap
    shelf = 0
    for k in order:
        s_ = int(sides[k])
        if x + s_ + gap > width:
            x, y = gap, y + shelf + gap
            shelf = 0
        place[k] = (x, y)
        x += s_ + gap
        shelf = max(shelf, s_)
    height = y + shelf + gap
    opts = Options(c=10.0, omega=1.8, gamma=10.0, proj_every=20, proj_iters=50)
    bcs = [BC(0, "dirichlet", "zero"),
           BC(1, "dirichlet", "const", ramp="sin2", t_ramp=t_ramp, vec=(stretch, 0.0)),
           BC(2, "neumann", "zero")]
    shapes, groups, specs = [], [], []
    for k in range(n_spec):
        s_ = int(sides[k])
        i0, j0 = place[k]
        L = s_ * dx
        ox, oy = i0 * dx, j0 * dx                      # lower-left corner of the specimen's nodes
        xl, xr = ox + 0.2 * dx, ox + (s_ - 0.4) * dx   # edges between node centres
        yb, yt = oy + 0.3 * dx, oy + (s_ - 0.3) * dx
        mine = [Shape("halfspace", (xl, 0), (-1.0, 0.0), boundary_id=0),
                Shape("halfspace", (xr, 0), (1.0, 0.0), boundary_id=1),
                Shape("halfspace", (0, yb), (0.0, -1.0), boundary_id=2),
                Shape("halfspace", (0, yt), (0.0, 1.0), boundary_id=2)]
        holes = []
        for _ in range(int(rng.integers(1, 6))):
            for _try in range(200):
                a, b = rng.uniform(0.05, 0.2, size=2) * L
                th = rng.uniform(0, 180)
                c = (ox + rng.uniform(0.25, 0.75) * L, oy + rng.uniform(0.25, 0.75) * L)
                r = max(a, b)
                if min(c[0] - xl, xr - c[0], c[1] - yb, yt - c[1]) < r + 6 * dx:
                    continue
                if any(np.hypot(c[0] - h[0][0], c[1] - h[0][1]) < r + h[1] + 6 * dx for h in holes):
                    continue
                holes.append((c, r))
                mine.append(Shape("ellipsoid", c, (a, b), rot=rot_z(th), complement=True, boundary_id=2))
                break
        mu = float(rng.uniform(0.5, 2.0))
        lam = float(mu * rng.uniform(1.0, 20.0))
        groups.append(Group(len(shapes), len(mine), (ox - 2 * dx, oy - 2 * dx), (ox + (s_ + 2) * dx, oy + (s_ + 2) * dx),
                            mu, lam))
        shapes.extend(mine)
        nb = s_ + 2 * margin
        sp = Problem(name=f"batch_specimen_{k}", dim=2, n=(nb, nb, 1), dx=dx,
                     origin=((i0 - margin) * dx, (j0 - margin) * dx, 0.0), periodic=(False, False, False),
                     mu=mu, lam=lam, options=opts, shapes=list(mine), bcs=list(bcs))
        _rest_fields(sp)
        sp.steps = steps
        specs.append((sp, (i0 - margin, j0 - margin)))
    # one lattice speed for the packed run: the smallest the library's wave-speed audit accepts
    # (2.5 times the largest tangent speed of the reference state, sqrt(lambda + 2 mu) with rho0 = 1;
    # lbm_create refuses less with LBM_ERR_UNSTABLE_C), and at least 10.  The stiffest draws
    # (lambda + 2 mu ~ 42) blow up at c = 10 and, under this loading, still at c = 2 c_L; 2.16 c_L ran.
    opts.c = max(10.0, 2.5 * max(np.sqrt(g.lam + 2.0 * g.mu) for g in groups))
    packed = Problem(name=f"batch_2d_{n_spec}", dim=2, n=(width, int(-(-height // 16) * 16), 1), dx=dx,
                     origin=(0.0, 0.0, 0.0), periodic=(False, False, False), mu=1.0, lam=1.0, options=opts,
                     shapes=shapes, bcs=list(bcs), groups=groups)
    _rest_fields(packed)
    packed.steps = steps
    packed.meta = dict(sides=sides.tolist(), place=[place[k] for k in range(n_spec)])
    return packed, specs


def inclusion_cube(n: int = 128, steps: int = 3000, lam: float = 2.0, b: Sequence[float] = (0.0, 0.0, -0.1)):
    """Unit cube whose six faces are clamped (velocity-Dirichlet zero), the body a box inset by
    0.3 dx so that every box node is active and the links leaving the box are cut links; constant
    body force b; c = 10, omega = 1.8, gamma = 10.  meta["mu_target"]: shear modulus 2 inside the
    sphere of radius 0.25 at the centre and 1 outside, blended over one cell (the field a
    displacement-misfit loss would recover); lambda fixed.  For the reverse-mode runs: the
    parameter is a per-node mu field (start: 1), the loss a misfit of u(t_N)."""
    dx = 1.0 / n
    p = Problem(name=f"inclusion_cube_{n}", dim=3, n=(n, n, n), dx=dx, origin=(0, 0, 0),
                periodic=(False, False, False), mu=1.0, lam=lam,
                options=Options(c=10.0, omega=1.8, gamma=10.0, body_force=tuple(b)))
    e = 0.3 * dx
    p.shapes = [Shape("halfspace", (e, 0, 0), (-1, 0, 0), boundary_id=0),
                Shape("halfspace", (1 - e, 0, 0), (1, 0, 0), boundary_id=0),
                Shape("halfspace", (0, e, 0), (0, -1, 0), boundary_id=0),
                Shape("halfspace", (0, 1 - e, 0), (0, 1, 0), boundary_id=0),
                Shape("halfspace", (0, 0, e), (0, 0, -1), boundary_id=0),
                Shape("halfspace", (0, 0, 1 - e), (0, 0, 1), boundary_id=0)]
    p.bcs = [BC(0, "dirichlet", "zero")]
    _rest_fields(p)
    X = p.coords()
    r = np.sqrt(sum((X[a] - 0.5) ** 2 for a in range(3)))
    w = np.clip((0.25 + 0.5 * dx - r) / dx, 0.0, 1.0)
    p.meta = dict(mu_target=1.0 + w)
    p.steps = steps
    return p

