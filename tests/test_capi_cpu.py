"""The C-ABI library builds, loads and exports every entry point that include/aim.h declares.

These tests make no compute calls (no GPU here): only host-only entry points run.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim
    return aim.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "aim.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(aim_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("aim_setup", "aim_matvec", "aim_solve", "aim_destroy", "aim_grid_product", "aim_rhs_planewave",
                 "aim_query_bytes", "aim_reserve", "aim_get_info", "aim_status_str", "aim_last_error"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(8):
        assert lib.aim_status_str(code)
    assert lib.aim_status_str(99) == b"unknown status"


def test_query_bytes_is_host_only_and_scales(lib):
    from paper_2606_10784_gb300 import aim
    nodes = synth.circle_polygon(1.0, 256)
    b1 = aim.query_bytes(nodes, aim.TE, 64, nrhs=1)
    b8 = aim.query_bytes(nodes, aim.TE, 64, nrhs=8)
    big = aim.query_bytes(synth.circle_polygon(100.0, 4000), aim.TE, 1024, nrhs=1)
    assert 0 < b1 < b8 < big


def test_query_bytes_counts_the_near_field_of_the_given_radius(lib):
    # the count runs the host setup, so a near radius that takes in more pairs costs more bytes
    # (the old bound assumed at most 64 entries per row whatever the radius)
    from paper_2606_10784_gb300 import aim
    nodes = synth.StarContour.from_seed(2).polygon(100.0, 1000)
    base = aim.query_bytes(nodes, aim.TE, 256, nrhs=1)
    wide = aim.query_bytes(nodes, aim.TE, 256, nrhs=1, near_radius=3.0)
    # 3 wavelengths at 10 segments per wavelength: ~60 segments each side, ~120+ hats per row,
    # two complex128 and two complex64 values plus a column per entry
    assert wide - base > 1000 * 100 * (2 * 16 + 2 * 8 + 4) * 0.5


def test_query_solve_bytes_adds_the_krylov_basis_of_the_restart(lib):
    from paper_2606_10784_gb300 import aim
    nodes = synth.circle_polygon(50.0, 3000)
    b100 = aim.query_solve_bytes(nodes, aim.TE, 512, nrhs=4, restart=100)
    b600 = aim.query_solve_bytes(nodes, aim.TE, 512, nrhs=4, restart=600)
    basis = 500 * 4 * 3000 * 16          # 500 more basis vectors of n x nrhs complex128
    hess = lambda r: (r + r * (r + 1) // 2) * 16 * 4   # packed Hessenberg matrix per rhs
    basis += hess(600) - hess(100)
    assert basis <= b600 - b100 <= basis + (8 << 20)
    assert b100 > aim.query_bytes(nodes, aim.TE, 512, nrhs=4)
    mixed = aim.query_solve_bytes(nodes, aim.TE, 512, nrhs=4, restart=100, precision=aim.MIXED)
    assert mixed >= b100


def test_query_calls_reject_bad_arguments(lib):
    from paper_2606_10784_gb300 import aim
    nodes = synth.circle_polygon(1.0, 64)
    with pytest.raises(aim.AimError) as exc:
        aim.query_bytes(nodes, aim.TE, 4)
    assert exc.value.status == aim.EINVAL
    with pytest.raises(aim.AimError) as exc:
        aim.query_solve_bytes(nodes, aim.TE, 32, restart=0)
    assert exc.value.status == aim.EINVAL


def test_setup_rejects_bad_arguments_before_touching_the_gpu(lib):
    from paper_2606_10784_gb300 import aim
    nodes = synth.circle_polygon(1.0, 64)
    for kw, status in ((dict(m=4), aim.EINVAL), (dict(m=32, fft_P=48), aim.EINVAL), (dict(m=16, fft_P=32), aim.EINVAL),
                       (dict(m=32, s=1), aim.EINVAL),
                       (dict(m=32, alpha=1.0), aim.EINVAL)):
        with pytest.raises(aim.AimError) as exc:
            aim.Context(nodes, 2 * np.pi, aim.TE, **kw)
        assert exc.value.status == status
    with pytest.raises(aim.AimError):
        aim.Context(nodes[:2], 2 * np.pi, aim.TE, 32)


def test_schedule_calls_reject_null_arguments(lib):
    from paper_2606_10784_gb300 import aim
    sc = aim.Schedule(1, 128, 0)
    assert lib.aim_set_schedule(None, 0, ctypes.byref(sc)) == aim.EINVAL
    assert lib.aim_get_schedule(None, 0, ctypes.byref(sc)) == aim.EINVAL
    assert lib.aim_autotune(None, 1, 0, None, None) == aim.EINVAL


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    from paper_2606_10784_gb300 import aim
    monkeypatch.setattr(aim, "_lib", None)
    monkeypatch.setattr(aim, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        aim.lib()


def test_new_entry_points_reject_bad_arguments_before_the_gpu(lib):
    from paper_2606_10784_gb300 import aim
    i = ctypes.c_int
    assert lib.aim_batcher_create(-1, ctypes.byref(ctypes.c_void_p())) == aim.EINVAL
    assert lib.aim_batcher_create(200, None) == aim.EINVAL
    assert lib.aim_batcher_stats(None, None, None, None) == aim.EINVAL
    assert lib.aim_solve_batched(None, None, 0, 1, None, None, 0, None, None, None) == aim.EINVAL
    assert lib.aim_kernel_table(None, 0, None, None) == aim.EINVAL
    a = (ctypes.c_double * 4)()
    assert lib.aim_lanczos_bidiag(None, 0, 4, 0, None, a, a, None, None, None) == aim.EINVAL
    assert lib.aim_matvec_multi(0, None, None, None, None, None, 0, None) == aim.EINVAL
    assert lib.aim_matvec_multi(33, None, None, None, None, None, 0, None) == aim.EINVAL
    assert lib.aim_dft_stage(4, 1, 1, None, None, None) == aim.EINVAL
    assert lib.aim_dft_stage(0, 0, 1, None, None, None) == aim.EINVAL
    assert lib.aim_dft_stage(0, 1, -1, None, None, None) == aim.EINVAL
    assert lib.aim_dft_stage(2, 1, 1, None, None, None) == aim.EINVAL
    lib.aim_batcher_destroy(None)        # NULL is allowed


def test_setup_rejects_unknown_filter_kind(lib):
    from paper_2606_10784_gb300 import aim
    nodes = synth.circle_polygon(1.0, 64)
    for kind in (-1, 3):
        with pytest.raises(aim.AimError) as exc:
            aim.Context(nodes, 2 * np.pi, aim.TE, 32, alpha=4.0 * np.pi, filter_kind=kind)
        assert exc.value.status == aim.EINVAL
