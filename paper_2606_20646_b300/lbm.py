"""Thin Python binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

PyTorch provides device memory and the CUDA stream; every step of the method runs
in the sm_103a kernels of ``liblbm_b300.so``.  Importing this module loads the
library and raises if it is missing: there is no CPU or PyTorch fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

# LBM_B300_CHECK=1 selects the bounds-checked build (kernels check their data-dependent indices and
# latch LBM_DEV_BOUNDS); the arithmetic is the same
_LIB_PATH = _build.LIB_CHECK if os.environ.get("LBM_B300_CHECK") == "1" else _build.LIB

_SHAPE = {"sphere": 0, "ellipsoid": 1, "superellipse": 2, "cylinder": 3, "halfspace": 4, "sampled": 5}
_BCKIND = {"dirichlet": 0, "neumann": 1}
_PROFILE = {"zero": 0, "affine": 1, "radial": 2, "twist_stretch": 3, "const": 4}
_RAMP = {"one": 0, "linear": 1, "sin2": 2, "cos": 3, "time": 4}
PREC = {"fp64": 0, "fp32": 1, "bf16s": 2}
DEV_STATUS = {1: "nonfinite", 2: "jacobian", 4: "newton", 8: "lsq", 16: "capacity", 128: "timeout", 256: "bounds"}
MAX_SHAPES = 16
MAX_BCS = 16


class lbm_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("periodic", C.c_int * 3), ("reserved", C.c_int),
                ("dx", C.c_double), ("origin", C.c_double * 3)]


class lbm_shape(C.Structure):
    _fields_ = [("kind", C.c_int), ("complement", C.c_int), ("boundary_id", C.c_int), ("reserved", C.c_int),
                ("center", C.c_double * 3), ("axes", C.c_double * 3), ("rot", C.c_double * 9), ("p", C.c_double),
                ("phi", C.c_void_p)]


class lbm_material(C.Structure):
    _fields_ = [("mu", C.c_double), ("lambda_", C.c_double)]


class lbm_group(C.Structure):
    _fields_ = [("first_shape", C.c_int), ("nshapes", C.c_int), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("material", lbm_material)]


class lbm_levelset(C.Structure):
    _fields_ = [("nshapes", C.c_int), ("shapes", C.POINTER(lbm_shape)), ("ngroups", C.c_int),
                ("groups", C.POINTER(lbm_group))]


class lbm_bc(C.Structure):
    _fields_ = [("boundary_id", C.c_int), ("kind", C.c_int), ("profile", C.c_int), ("ramp", C.c_int),
                ("t_ramp", C.c_double), ("center", C.c_double * 3), ("A", C.c_double * 9),
                ("vec", C.c_double * 3), ("amp", C.c_double)]


class lbm_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("proj_every", C.c_int), ("proj_iters", C.c_int), ("host_staging", C.c_int),
                ("c", C.c_double), ("omega", C.c_double), ("gamma", C.c_double), ("theta_F", C.c_double),
                ("proj_beta", C.c_double), ("body_force", C.c_double * 3), ("adjoint", C.c_int),
                ("reserved", C.c_int), ("c_audit", C.c_double)]


class lbm_info(C.Structure):
    _fields_ = [("n_box", C.c_longlong), ("n_active", C.c_longlong), ("n_cut", C.c_longlong),
                ("n_neumann", C.c_longlong), ("n_dirichlet", C.c_longlong), ("n_segments", C.c_longlong),
                ("step", C.c_longlong), ("t", C.c_double), ("dt", C.c_double), ("geometry_bytes", C.c_size_t),
                ("storage_bytes", C.c_size_t), ("launches", C.c_longlong), ("lsq_entries", C.c_longlong)]


class lbm_kernel_time(C.Structure):
    _fields_ = [("stream_collide_ms", C.c_double), ("cutlink_ms", C.c_double), ("projection_ms", C.c_double),
                ("stream_collide_launches", C.c_longlong), ("cutlink_launches", C.c_longlong),
                ("projection_launches", C.c_longlong), ("jacobi_ms", C.c_double), ("jacobi_launches", C.c_longlong)]


class lbm_diag(C.Structure):
    _fields_ = [("J_min", C.c_double), ("J_max", C.c_double), ("v_rms", C.c_double), ("v_max", C.c_double),
                ("c_tangent", C.c_double), ("incompat_rms", C.c_double), ("n_active", C.c_longlong),
                ("n_edges", C.c_longlong), ("step", C.c_longlong), ("t", C.c_double)]


LAYOUT = {"planes": 0, "nodes": 1}


class lbm_tuning(C.Structure):
    _fields_ = [("windows_per_warp", C.c_int), ("jacobi_segments", C.c_int), ("link_block", C.c_int),
                ("jacobi_sweeps", C.c_int), ("candidates", C.c_int), ("ms_per_step", C.c_double),
                ("default_ms_per_step", C.c_double)]


# symbol -> (restype, argtypes); every entry point declared in include/lbm.h
_vp, _d, _i, _sz = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_size_t)
SIGNATURES = {
    "lbm_geometry_bytes": (C.c_int, [C.POINTER(lbm_grid), _sz]),
    "lbm_create": (C.c_int, [C.POINTER(lbm_grid), C.POINTER(lbm_levelset), C.POINTER(lbm_material),
                             C.POINTER(lbm_bc), C.c_int, C.POINTER(lbm_options), _vp, C.c_size_t, _vp,
                             C.POINTER(_vp)]),
    "lbm_storage_bytes": (C.c_int, [_vp, _sz]),
    "lbm_bind_storage": (C.c_int, [_vp, _vp, C.c_size_t]),
    "lbm_set_initial": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp]),
    "lbm_step": (C.c_int, [_vp, C.c_int]),
    "lbm_fields": (C.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_fields_ex": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_int]),
    "lbm_diagnostics": (C.c_int, [_vp, C.POINTER(lbm_diag)]),
    "lbm_sync": (C.c_int, [_vp, _i]),
    "lbm_get_info": (C.c_int, [_vp, C.POINTER(lbm_info)]),
    "lbm_enable_timing": (C.c_int, [_vp, C.c_int]),
    "lbm_step_graph": (C.c_int, [_vp, C.c_int]),
    "lbm_set_tuning": (C.c_int, [_vp, C.POINTER(lbm_tuning)]),
    "lbm_get_tuning": (C.c_int, [_vp, C.POINTER(lbm_tuning)]),
    "lbm_autotune": (C.c_int, [_vp, C.c_int, _vp, C.POINTER(lbm_tuning)]),
    "lbm_set_mu_field": (C.c_int, [_vp, _vp]),
    "lbm_set_wait_limit": (C.c_int, [_vp, C.c_int]),
    "lbm_set_body_force": (C.c_int, [_vp, _d]),
    "lbm_state_bytes": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "lbm_save_state": (C.c_int, [_vp, _vp]),
    "lbm_load_state": (C.c_int, [_vp, _vp]),
    "lbm_moments_bytes": (C.c_int, [_vp, C.POINTER(C.c_size_t)]),
    "lbm_step_moments": (C.c_int, [_vp, _vp]),
    "lbm_adjoint_begin": (C.c_int, [_vp, _vp]),
    "lbm_adjoint_step": (C.c_int, [_vp, _vp]),
    "lbm_adjoint_gradients": (C.c_int, [_vp, _vp, _d]),
    "lbm_kernel_times": (C.c_int, [_vp, C.POINTER(lbm_kernel_time)]),
    "lbm_copy_links": (C.c_int, [_vp, C.POINTER(C.c_longlong), _i, _d, _d, _d, _i, _i]),
    "lbm_copy_active": (C.c_int, [_vp, C.POINTER(C.c_ubyte)]),
    "lbm_destroy": (None, [_vp]),
    "lbm_error_string": (C.c_char_p, [C.c_int]),
    "lbm_census_static": (C.c_int, [C.POINTER(lbm_grid), C.POINTER(lbm_levelset), _vp, C.POINTER(C.c_longlong),
                                    C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
}

_lib = None


def load_library(path: str = _LIB_PATH):
    """Load liblbm_b300.so and declare every entry point; raises if the library is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2606_20646_b300.build` "
                               "(there is no fallback implementation)")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        _lib = lib
    return _lib


class LbmError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load_library().lbm_error_string(code).decode()
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


def _check(code: int, where: str):
    if code != 0:
        raise LbmError(code, where)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def descriptors(p, precision="fp32", host_staging=False, adjoint=False, keep=None):
    """Translate a problem description into the ABI structs.  Sampled level sets are copied to the
    device; the tensors are appended to `keep`, which must outlive the simulation."""
    g = lbm_grid()
    g.dim = p.dim
    for a in range(3):
        g.n[a] = int(p.n[a])
        g.periodic[a] = int(bool(p.periodic[a]))
        g.origin[a] = float(p.origin[a])
    g.dx = p.dx
    shapes = (lbm_shape * max(1, len(p.shapes)))()
    for j, sh in enumerate(p.shapes):
        s = shapes[j]
        s.kind, s.complement, s.boundary_id = _SHAPE[sh.kind], int(sh.complement), int(sh.boundary_id)
        for a in range(3):
            s.center[a], s.axes[a] = sh.center[a], sh.axes[a]
        for a in range(9):
            s.rot[a] = float(sh.rot.reshape(-1)[a])
        s.p = sh.p
        if sh.kind == "sampled":
            t = torch.as_tensor(np.ascontiguousarray(sh.phi, dtype=np.float64).reshape(-1), device="cuda")
            assert t.numel() == p.n_box
            if keep is not None:
                keep.append(t)
            s.phi = t.data_ptr()
    groups = getattr(p, "groups", None) or []
    gs = (lbm_group * max(1, len(groups)))()
    for j, gr in enumerate(groups):
        G = gs[j]
        G.first_shape, G.nshapes = int(gr.first_shape), int(gr.nshapes)
        for a in range(3):
            G.lo[a], G.hi[a] = float(gr.lo[a]), float(gr.hi[a])
        G.material = lbm_material(gr.mu, gr.lam)
    ls = lbm_levelset(len(p.shapes), shapes, len(groups), gs)
    mat = lbm_material(p.mu, p.lam)
    bcs = (lbm_bc * max(1, len(p.bcs)))()
    for j, bc in enumerate(p.bcs):
        b = bcs[j]
        b.boundary_id, b.kind, b.profile, b.ramp = bc.boundary_id, _BCKIND[bc.kind], _PROFILE[bc.profile], _RAMP[bc.ramp]
        b.t_ramp, b.amp = bc.t_ramp, bc.amp
        for a in range(3):
            b.center[a], b.vec[a] = bc.center[a], bc.vec[a]
        for a in range(9):
            b.A[a] = float(bc.A.reshape(-1)[a])
    o = p.options
    opt = lbm_options()
    opt.precision = PREC[precision]
    opt.proj_every, opt.proj_iters, opt.host_staging = int(o.proj_every), int(o.proj_iters), int(bool(host_staging))
    opt.c, opt.omega, opt.gamma, opt.theta_F, opt.proj_beta = o.c, o.omega, o.gamma, o.theta_F, o.proj_beta
    for a in range(3):
        opt.body_force[a] = float(o.body_force[a])
    opt.adjoint = int(bool(adjoint))
    opt.c_audit = float(getattr(o, "c_audit", 0.0))
    return g, (shapes, gs), ls, mat, bcs, opt


class Simulation:
    """One TL vectorial LBM simulation on the current CUDA device, via the C ABI."""

    def __init__(self, p, precision: str = "fp32", stream: torch.cuda.Stream | None = None,
                 host_staging: bool = False, device: str | torch.device = "cuda", adjoint: bool = False):
        lib = load_library()
        self.p, self.precision, self.device = p, precision, torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._keep = []  # device copies of sampled level sets, alive as long as the simulation
        self._desc = descriptors(p, precision, host_staging, adjoint, keep=self._keep)
        g, shapes, ls, mat, bcs, opt = self._desc
        nbytes = C.c_size_t(0)
        _check(lib.lbm_geometry_bytes(C.byref(g), C.byref(nbytes)), "lbm_geometry_bytes")
        self.geometry = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        _check(lib.lbm_create(C.byref(g), C.byref(ls), C.byref(mat), bcs, len(p.bcs), C.byref(opt),
                              _ptr(self.geometry), nbytes.value, C.c_void_p(self.stream.cuda_stream), C.byref(h)),
               "lbm_create")
        self.h = h
        _check(lib.lbm_storage_bytes(self.h, C.byref(nbytes)), "lbm_storage_bytes")
        self.storage = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        _check(lib.lbm_bind_storage(self.h, _ptr(self.storage), nbytes.value), "lbm_bind_storage")
        self.D, self.K = p.dim, p.K

    def close(self):
        if getattr(self, "h", None):
            load_library().lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters, saved states, reverse mode ------------------------------------------------
    def set_mu_field(self, mu):
        """Per-node shear modulus (box-shaped array or tensor); needs adjoint=True."""
        t = torch.as_tensor(mu, dtype=torch.float64, device=self.device).contiguous()
        assert t.numel() == self.p.n_box
        _check(load_library().lbm_set_mu_field(self.h, C.c_void_p(t.data_ptr())), "lbm_set_mu_field")
        self.stream.synchronize()
        return self

    def set_wait_limit(self, polls: int):
        """First-wait poll limit of the bulk-copy kernels (lbm_set_wait_limit; < 0: the default)."""
        _check(load_library().lbm_set_wait_limit(self.h, int(polls)), "lbm_set_wait_limit")
        return self

    def set_body_force(self, b):
        arr = (C.c_double * 3)(*[float(x) for x in list(b) + [0.0] * (3 - len(b))])
        _check(load_library().lbm_set_body_force(self.h, arr), "lbm_set_body_force")
        return self

    def state_bytes(self) -> int:
        n = C.c_size_t(0)
        _check(load_library().lbm_state_bytes(self.h, C.byref(n)), "lbm_state_bytes")
        return n.value

    def save_state(self, out: torch.Tensor | None = None) -> torch.Tensor:
        buf = out if out is not None else torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        _check(load_library().lbm_save_state(self.h, _ptr(buf)), "lbm_save_state")
        return buf

    def load_state(self, buf: torch.Tensor):
        _check(load_library().lbm_load_state(self.h, _ptr(buf)), "lbm_load_state")
        return self

    def adjoint_begin(self, grad_u: torch.Tensor):
        g = grad_u.to(device=self.device, dtype=torch.float64).contiguous()
        assert g.numel() == self.D * self.p.n_box
        self._grad_u = g
        _check(load_library().lbm_adjoint_begin(self.h, C.c_void_p(g.data_ptr())), "lbm_adjoint_begin")
        return self

    def moments_bytes(self) -> int:
        n = C.c_size_t(0)
        _check(load_library().lbm_moments_bytes(self.h, C.byref(n)), "lbm_moments_bytes")
        return n.value

    def step_moments(self, buf: torch.Tensor):
        """One step recording its recovered F into `buf` (moments_bytes() bytes, device)."""
        _check(load_library().lbm_step_moments(self.h, _ptr(buf)), "lbm_step_moments")
        return self

    def adjoint_step(self, moments: torch.Tensor):
        """Reverse the next step of the sweep, given its recorded moments."""
        _check(load_library().lbm_adjoint_step(self.h, _ptr(moments)), "lbm_adjoint_step")
        return self

    def adjoint_gradients(self):
        """(dL/dmu as a box-shaped float64 tensor on the device, dL/db as 3 floats)."""
        gm = torch.empty(self.p.box_shape, dtype=torch.float64, device=self.device)
        gb = (C.c_double * 3)()
        _check(load_library().lbm_adjoint_gradients(self.h, C.c_void_p(gm.data_ptr()), gb), "lbm_adjoint_gradients")
        return gm, np.array(list(gb))

    # -- state --------------------------------------------------------------------------------
    def set_initial(self, v0=None, F0=None, u0=None, dU0=None, mode=None):
        """Initial fields (defaults: the problem's arrays), device tensors or pinned host tensors."""
        p = self.p

        def dev(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                return a.to(torch.float64).contiguous()
            return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=self.device)

        self._init = [dev(x) for x in (v0 if v0 is not None else p.v0, F0 if F0 is not None else p.F0,
                                       u0 if u0 is not None else p.u0, dU0 if dU0 is not None else p.dU0)]
        m = mode if mode is not None else p.init_mode
        _check(load_library().lbm_set_initial(self.h, 1 if m == "characteristic" else 0,
                                              *[_ptr(t) for t in self._init]), "lbm_set_initial")
        return self

    def step(self, n: int = 1):
        _check(load_library().lbm_step(self.h, int(n)), "lbm_step")
        return self

    def step_graph(self, n: int):
        """n steps captured as one CUDA graph and launched once (lbm_step_graph)."""
        _check(load_library().lbm_step_graph(self.h, int(n)), "lbm_step_graph")
        return self

    # -- tile shapes -----------------------------------------------------------------------------
    _TUNE_KEYS = ("windows_per_warp", "jacobi_segments", "link_block", "jacobi_sweeps", "candidates",
                  "ms_per_step", "default_ms_per_step")

    def get_tuning(self) -> dict:
        t = lbm_tuning()
        _check(load_library().lbm_get_tuning(self.h, C.byref(t)), "lbm_get_tuning")
        return {k: getattr(t, k) for k in self._TUNE_KEYS[:4]}

    def set_tuning(self, windows_per_warp: int = 0, jacobi_segments: int = 0, link_block: int = 0,
                   jacobi_sweeps: int = 0):
        """Tile shapes (0: the default); jacobi_sweeps: sweeps per Jacobi launch, 2 or 1."""
        t = lbm_tuning(windows_per_warp, jacobi_segments, link_block, jacobi_sweeps, 0, 0.0, 0.0)
        _check(load_library().lbm_set_tuning(self.h, C.byref(t)), "lbm_set_tuning")
        return self

    def autotune(self, steps: int = 20) -> dict:
        """Times the candidate tile shapes on this simulation from its current state (restored
        afterwards) and keeps the fastest (lbm_autotune)."""
        scratch = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        t = lbm_tuning()
        _check(load_library().lbm_autotune(self.h, int(steps), _ptr(scratch), C.byref(t)), "lbm_autotune")
        del scratch
        return {k: getattr(t, k) for k in self._TUNE_KEYS}

    def fields(self, out=None):
        """v (D,*box), F (D*D,*box), u (D,*box) as float64 tensors (device unless `out` given)."""
        D, bs = self.D, self.p.box_shape
        if out is None:
            out = (torch.empty((D,) + bs, dtype=torch.float64, device=self.device),
                   torch.empty((D * D,) + bs, dtype=torch.float64, device=self.device),
                   torch.empty((D,) + bs, dtype=torch.float64, device=self.device))
        _check(load_library().lbm_fields(self.h, *[_ptr(t) for t in out]), "lbm_fields")
        return out

    def fields_ex(self, sigma: bool = True, J: bool = True, layout: str = "planes"):
        """(v, F, u, sigma, J) as float64 device tensors (lbm_fields_ex); sigma = J^-1 P F^T.  Layout
        "planes": (ncomp, *box); "nodes": (*box, ncomp) with a node's components contiguous."""
        D, bs = self.D, self.p.box_shape
        shp = (lambda n: (n,) + bs) if layout == "planes" else (lambda n: bs + (n,))
        out = [torch.empty(shp(D), dtype=torch.float64, device=self.device),
               torch.empty(shp(D * D), dtype=torch.float64, device=self.device),
               torch.empty(shp(D), dtype=torch.float64, device=self.device),
               torch.empty(shp(D * D), dtype=torch.float64, device=self.device) if sigma else None,
               torch.empty(shp(1), dtype=torch.float64, device=self.device) if J else None]
        _check(load_library().lbm_fields_ex(self.h, *[_ptr(t) for t in out], LAYOUT[layout]), "lbm_fields_ex")
        return out

    def diagnostics(self) -> dict:
        """J range, RMS and largest |v|, largest tangent wave speed, compatibility residual (lbm_diagnostics)."""
        d = lbm_diag()
        _check(load_library().lbm_diagnostics(self.h, C.byref(d)), "lbm_diagnostics")
        return {k: getattr(d, k) for k, _ in lbm_diag._fields_}

    def sync(self, raise_on_status: bool = True) -> int:
        st = C.c_int(0)
        rc = load_library().lbm_sync(self.h, C.byref(st))
        if rc not in (0, -6):
            _check(rc, "lbm_sync")
        if rc == -6 and raise_on_status:
            names = [n for b, n in DEV_STATUS.items() if st.value & b]
            raise LbmError(rc, f"lbm_sync device status {st.value} ({', '.join(names)})")
        return st.value

    # -- diagnostics --------------------------------------------------------------------------
    def info(self) -> dict:
        inf = lbm_info()
        _check(load_library().lbm_get_info(self.h, C.byref(inf)), "lbm_get_info")
        return {k: getattr(inf, k) for k, _ in lbm_info._fields_}

    def enable_timing(self, on: bool = True):
        _check(load_library().lbm_enable_timing(self.h, int(on)), "lbm_enable_timing")

    def kernel_times(self) -> dict:
        kt = lbm_kernel_time()
        _check(load_library().lbm_kernel_times(self.h, C.byref(kt)), "lbm_kernel_times")
        return {k: getattr(kt, k) for k, _ in lbm_kernel_time._fields_}

    def links(self) -> dict:
        n = self.info()["n_cut"]
        node = np.zeros(n, dtype=np.int64)
        q = np.zeros(n, dtype=np.int32)
        eta = np.zeros(n)
        Xb = np.zeros((n, 3))
        Nb = np.zeros((n, 3))
        bid = np.zeros(n, dtype=np.int32)
        ns = np.zeros(n, dtype=np.int32)
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        _check(load_library().lbm_copy_links(self.h, node.ctypes.data_as(C.POINTER(C.c_longlong)), ip(q), dp(eta),
                                             dp(Xb), dp(Nb), ip(bid), ip(ns)), "lbm_copy_links")
        return dict(node=node, q=q, eta=eta, Xb=Xb, Nb=Nb, bid=bid, ns=ns)

    def active_mask(self) -> np.ndarray:
        m = np.zeros(self.p.n_box, dtype=np.uint8)
        _check(load_library().lbm_copy_active(self.h, m.ctypes.data_as(C.POINTER(C.c_ubyte))), "lbm_copy_active")
        return m.reshape(self.p.box_shape).astype(bool)


def census_static(p, stream: torch.cuda.Stream | None = None) -> dict:
    """Active nodes, cut links and active segments of a problem's grid and level set, computed
    by lbm_census_static (no device allocation; scratch in the library's fixed device array)."""
    lib = load_library()
    keep = []
    g, shapes, ls, mat, bcs, opt = descriptors(p, keep=keep)
    st = stream if stream is not None else torch.cuda.current_stream()
    a, c, s = C.c_longlong(0), C.c_longlong(0), C.c_longlong(0)
    _check(lib.lbm_census_static(C.byref(g), C.byref(ls), C.c_void_p(st.cuda_stream), C.byref(a), C.byref(c),
                                 C.byref(s)), "lbm_census_static")
    return {"n_active": a.value, "n_cut": c.value, "n_segments": s.value}
