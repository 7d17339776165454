"""The C-ABI library loads and exports every entry point include/lbm.h declares, and its
host-side validation answers without touching a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2606_20646_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    from paper_2606_20646_b300 import lbm
    return lbm.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    from paper_2606_20646_b300 import lbm
    assert set(names) == set(lbm.SIGNATURES)


def test_error_strings(lib):
    for code in range(0, -9, -1):
        assert lib.lbm_error_string(code)
    assert lib.lbm_error_string(-9).decode() == "unknown error"
    assert lib.lbm_error_string(-3).decode() == "CUDA runtime error"


def test_geometry_bytes_and_validation_without_gpu(lib):
    from paper_2606_20646_b300 import inputs as I, lbm
    p = I.shell_3d(64)
    g, shapes, ls, mat, bcs, opt = lbm.descriptors(p)
    n = C.c_size_t(0)
    assert lib.lbm_geometry_bytes(C.byref(g), C.byref(n)) == 0
    assert n.value >= p.n_box * 9
    bad = lbm.lbm_grid.from_buffer_copy(g)
    bad.dim = 4
    assert lib.lbm_geometry_bytes(C.byref(bad), C.byref(n)) == -1
    h = C.c_void_p()
    # descriptor errors are reported before any device work
    opt.omega = 2.5
    assert lib.lbm_create(C.byref(g), C.byref(ls), C.byref(mat), bcs, len(p.bcs), C.byref(opt), None, 0, None,
                          C.byref(h)) == -1
    opt.omega = 1.8
    # missing geometry storage
    assert lib.lbm_create(C.byref(g), C.byref(ls), C.byref(mat), bcs, len(p.bcs), C.byref(opt), None, 0, None,
                          C.byref(h)) == -4
    # an unknown boundary profile for a Neumann condition
    bcs[0].profile = 1
    assert lib.lbm_create(C.byref(g), C.byref(ls), C.byref(mat), bcs, len(p.bcs), C.byref(opt), None, 0, None,
                          C.byref(h)) == -1


def test_group_descriptors_validated_without_gpu(lib):
    """Multi-specimen level sets: group ranges, boxes and materials are checked before any device
    work; the allocation-free census takes single bodies only."""
    from paper_2606_20646_b300 import inputs as I, lbm
    packed, _ = I.batch_2d(n_spec=3, side=(40, 48), width=192, seed=3)
    g, shapes, ls, mat, bcs, opt = lbm.descriptors(packed)
    h = C.c_void_p()
    args = lambda: (C.byref(g), C.byref(ls), C.byref(mat), bcs, len(packed.bcs), C.byref(opt), None, 0, None,
                    C.byref(h))
    assert ls.ngroups == 3
    assert lib.lbm_create(*args()) == -4           # valid descriptors, no storage given
    gs = shapes[1]
    gs[1].first_shape = len(packed.shapes)          # group past the shape list
    assert lib.lbm_create(*args()) == -1
    gs[1].first_shape = 0
    gs[2].material.mu = -1.0                        # invalid group material
    assert lib.lbm_create(*args()) == -1
    gs[2].material.mu = 1.0
    gs[0].lo[0], gs[0].hi[0] = 1.0, 0.0             # empty box
    assert lib.lbm_create(*args()) == -1
    n = [C.c_longlong(0) for _ in range(3)]
    assert lib.lbm_census_static(C.byref(g), C.byref(ls), None, *[C.byref(x) for x in n]) == -1


def test_bf16_storage_descriptors_without_gpu(lib):
    """The BF16-storage form is a valid precision; it does not take the reverse mode; unknown
    precisions are refused.  All checked before any device work."""
    from paper_2606_20646_b300 import inputs as I, lbm
    p = I.shell_3d(32)
    g, shapes, ls, mat, bcs, opt = lbm.descriptors(p, precision="bf16s")
    h = C.c_void_p()
    args = lambda: (C.byref(g), C.byref(ls), C.byref(mat), bcs, len(p.bcs), C.byref(opt), None, 0, None, C.byref(h))
    assert opt.precision == 2
    assert lib.lbm_create(*args()) == -4           # valid descriptors, no storage given
    opt.adjoint = 1
    assert lib.lbm_create(*args()) == -1
    opt.adjoint = 0
    opt.precision = 3
    assert lib.lbm_create(*args()) == -1


def test_new_entry_points_refuse_bad_arguments_without_gpu(lib):
    """Tuning, autotuner, saved states and reverse mode check their arguments before any device
    work: a null handle or buffer is LBM_ERR_ARG."""
    from paper_2606_20646_b300 import lbm
    t = lbm.lbm_tuning(0, 0, 0, 0, 0, 0.0, 0.0)
    assert lib.lbm_set_tuning(None, C.byref(t)) == -1
    assert lib.lbm_get_tuning(None, C.byref(t)) == -1
    assert lib.lbm_autotune(None, 20, None, None) == -1
    n = C.c_size_t(0)
    assert lib.lbm_state_bytes(None, C.byref(n)) == -1
    assert lib.lbm_save_state(None, None) == -1
    assert lib.lbm_load_state(None, None) == -1
    assert lib.lbm_moments_bytes(None, C.byref(n)) == -1
    assert lib.lbm_step_moments(None, None) == -1
    assert lib.lbm_adjoint_begin(None, None) == -1
    assert lib.lbm_adjoint_step(None, None) == -1
    assert lib.lbm_adjoint_gradients(None, None, None) == -1


def test_wave_speed_audit_at_create_without_gpu(lib):
    """lbm_create audits the lattice speed against the largest tangent wave speed of the reference
    state, sqrt(lambda + 2 mu) (rho0 = 1), before any device work: c below c_audit times it is
    LBM_ERR_UNSTABLE_C; the default factor is 2.5; a negative factor turns the audit off."""
    from paper_2606_20646_b300 import inputs as I, lbm
    p = I.shell_3d(32)                              # mu = 1, lambda = 5: c_T = sqrt(7)
    g, shapes, ls, mat, bcs, opt = lbm.descriptors(p)
    h = C.c_void_p()
    args = lambda: (C.byref(g), C.byref(ls), C.byref(mat), bcs, len(p.bcs), C.byref(opt), None, 0, None, C.byref(h))
    cT = 7.0 ** 0.5
    opt.c = 2.5 * cT * 1.001
    assert lib.lbm_create(*args()) == -4           # passes the audit; no storage given
    opt.c = 2.5 * cT * 0.999
    assert lib.lbm_create(*args()) == -8
    opt.c_audit = 2.0                               # a smaller factor accepts it
    assert lib.lbm_create(*args()) == -4
    opt.c_audit = -1.0                              # audit off
    opt.c = 1.0
    assert lib.lbm_create(*args()) == -4
    opt.c_audit = 0.0
    assert lib.lbm_create(*args()) == -8
    opt.c_audit = float("nan")
    assert lib.lbm_create(*args()) == -1


def test_field_and_diagnostic_calls_refuse_bad_arguments_without_gpu(lib):
    from paper_2606_20646_b300 import lbm
    d = lbm.lbm_diag()
    assert lib.lbm_fields_ex(None, None, None, None, None, None, 0) == -1
    assert lib.lbm_diagnostics(None, C.byref(d)) == -1
