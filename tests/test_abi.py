"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects bad arguments on the host before any launch.

Every call here fails validation (bad nx, negative size, NULL, misaligned or
overlapping pointers), so no kernel is ever enqueued, with or without a GPU.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import ref
from paper_2011_04981_gb300 import build as nbuild
from paper_2011_04981_gb300 import nekax

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    return nekax.load()


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "nekax.h")).read()
    return sorted(set(re.findall(r"^(?:const\s+)?\w+\s*\*?\s*(nek_\w+)\s*\(", txt, re.M)))


def test_every_declared_symbol_is_exported(lib):
    syms = _declared_symbols()
    assert len(syms) >= 18
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(nekax.exported_symbols())


def test_status_strings(lib):
    for st, name in [(0, "NEK_OK"), (1, "NEK_ERR_INVALID_ARG"), (2, "NEK_ERR_UNSUPPORTED_NX"), (3, "NEK_ERR_CUDA"),
                     (4, "NEK_ERR_NOT_CONVERGED"), (5, "NEK_ERR_BREAKDOWN"), (6, "NEK_ERR_TIMEOUT"),
                     (7, "NEK_ERR_NOMEM"), (8, "NEK_ERR_TOO_LARGE"), (99, "NEK_ERR_UNKNOWN")]:
        assert nekax.status_string(st) == name
    assert nekax.version() >= 100


@pytest.mark.parametrize("nx", range(2, 17))
def test_host_gll_matches_oracle(lib, nx):
    xi, rho, D = nekax.gll(nx)
    xo, ro, Do = ref.gll(nx)
    assert np.max(np.abs(xi - xo)) <= 4e-16
    assert np.max(np.abs(rho - ro)) <= 4e-16 * nx
    assert np.max(np.abs(D - Do)) <= 2e-15 * nx * np.abs(Do).max()


def test_ax_rejects_bad_arguments_before_launch(lib):
    A16 = 0x10000  # 16-byte aligned fake addresses, never dereferenced
    L = lib
    assert L.nek_ax(4, 1, A16, A16, A16, A16 * 2, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_ax(4, 17, A16, A16, A16, A16 * 2, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_ax(-1, 8, A16, A16, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax(0, 8, None, None, None, None, None) == nekax.OK  # empty input is a no-op
    assert L.nek_ax(4, 8, None, A16, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax(4, 8, A16, None, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax(4, 8, A16, A16 + 8, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG  # G misaligned
    assert L.nek_ax(4, 8, A16, A16, A16 + 4, A16 * 2, None) == nekax.ERR_INVALID_ARG  # u misaligned
    assert L.nek_ax(4, 8, A16 + 4, A16, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG  # D misaligned
    # u and w overlap (4 elements of 512 doubles = 16 KiB each)
    assert L.nek_ax(4, 8, A16, A16, A16, A16 + 4096, None) == nekax.ERR_INVALID_ARG


def test_ax_oz_rejects_bad_arguments_before_launch(lib):
    A16 = 0x10000  # 16-byte aligned fake addresses, never dereferenced
    L = lib
    for nx in (1, 3, 9, 11, 12, 16, 17):  # even nx up to 10 only
        assert L.nek_ax_oz(4, nx, A16, A16, A16, A16 * 2, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_ax_oz(-1, 8, A16, A16, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_oz(0, 8, None, None, None, None, None) == nekax.OK  # empty input is a no-op
    assert L.nek_ax_oz(4, 8, None, A16, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_oz(4, 8, A16, None, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_oz(4, 8, A16, A16 + 8, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG  # Gff misaligned
    assert L.nek_ax_oz(4, 8, A16, A16, A16 + 8, A16 * 2, None) == nekax.ERR_INVALID_ARG  # u not 16-byte aligned
    assert L.nek_ax_oz(4, 8, A16, A16, A16, A16 * 2 + 8, None) == nekax.ERR_INVALID_ARG  # w not 16-byte aligned
    assert L.nek_geom_oz(4, 7, A16, A16 * 2, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_geom_oz(-1, 8, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_geom_oz(0, 8, None, None, None) == nekax.OK
    assert L.nek_geom_oz(4, 8, A16, A16 * 2 + 8, None) == nekax.ERR_INVALID_ARG  # Goz misaligned
    assert L.nek_geom_oz(4, 8, A16, A16 + 64, None) == nekax.ERR_INVALID_ARG  # overlap
    assert L.nek_ax_oz(4, 8, A16, A16, A16, A16 + 4096, None) == nekax.ERR_INVALID_ARG  # u and w overlap
    t = ctypes.c_int(0)
    assert L.nek_ax_oz_selftest(1, 0, ctypes.byref(t)) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_oz_selftest(1, 2000001, ctypes.byref(t)) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_oz_selftest(1, 100, None) == nekax.ERR_INVALID_ARG


def test_ax_lowp_tc5_rejects_bad_arguments_before_launch(lib):
    A16 = 0x10000
    L = lib
    for nx in (1, 12, 16):
        assert L.nek_ax_lowp_tc5(4, nx, 1, A16, A16, A16, A16, A16 * 2, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_ax_lowp_tc5(4, 8, 0, A16, A16, A16, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG  # FP32: no MMA form
    assert L.nek_ax_lowp_tc5(4, 8, 3, A16, A16, A16, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_lowp_tc5(-1, 8, 1, A16, A16, A16, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_lowp_tc5(0, 8, 1, None, None, None, None, None, None) == nekax.OK
    assert L.nek_ax_lowp_tc5(4, 8, 1, None, A16, A16, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_lowp_tc5(4, 8, 1, A16, A16 + 2, A16, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG  # Glp
    assert L.nek_ax_lowp_tc5(4, 8, 1, A16, A16, A16, A16, A16 + 256, None) == nekax.ERR_INVALID_ARG  # overlap


def test_other_entry_points_reject_bad_arguments(lib):
    L = lib
    A16 = 0x10000
    assert L.nek_geom(4, 1, A16, A16, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_geom(-2, 4, A16, A16, None) == nekax.ERR_INVALID_ARG
    assert L.nek_geom(4, 4, None, A16, None) == nekax.ERR_INVALID_ARG
    assert L.nek_geom(4, 4, A16, A16 + 8, None) == nekax.ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert L.nek_gs_create(1, 1, None, ctypes.byref(h)) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_gs_create(-1, 3, None, ctypes.byref(h)) == nekax.ERR_INVALID_ARG
    assert L.nek_gs_create(1, 3, None, ctypes.byref(h)) == nekax.ERR_INVALID_ARG
    assert L.nek_gs_create(1, 3, None, None) == nekax.ERR_INVALID_ARG
    bad = np.full(27, -1, dtype=np.int64)
    assert L.nek_gs_create(1, 3, bad.ctypes.data, ctypes.byref(h)) == nekax.ERR_INVALID_ARG
    assert L.nek_gs_create(1 << 22, 16, None, ctypes.byref(h)) == nekax.ERR_TOO_LARGE
    assert L.nek_dssum(None, A16, None) == nekax.ERR_INVALID_ARG
    assert L.nek_gs_destroy(None) == nekax.OK
    assert L.nek_gs_info(None, None, None, None) == nekax.ERR_INVALID_ARG
    assert L.nek_mask(-1, A16, A16, None) == nekax.ERR_INVALID_ARG
    assert L.nek_mask(0, None, None, None) == nekax.OK
    assert L.nek_mask(8, None, A16, None) == nekax.ERR_INVALID_ARG
    assert L.nek_dot_c(None, A16, A16, A16, None) == nekax.ERR_INVALID_ARG
    assert L.nek_jacobi_minv(None, 1, 3, A16, A16, A16, A16, None) == nekax.ERR_INVALID_ARG
    assert L.nek_jacobi_minv(None, 1, 1, A16, A16, A16, A16, None) == nekax.ERR_UNSUPPORTED_NX
    it, rr = ctypes.c_int(5), ctypes.c_double(5.0)
    assert L.nek_cg_solve(None, 1, 3, A16, A16, A16, None, A16, A16, 1e-8, 10, None, ctypes.byref(it),
                          ctypes.byref(rr), None) == nekax.ERR_INVALID_ARG
    assert it.value == 0 and rr.value == 0.0
    assert L.nek_cg_solve(None, 1, 20, A16, A16, A16, None, A16, A16, 1e-8, 10, None, None, None,
                          None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_gll(1, None, None, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_cg_workspace_bytes(-1, 8, 1) == 0
    n = 10 * 8 ** 3
    assert L.nek_cg_workspace_bytes(10, 8, 1) >= 4 * 8 * n  # r, p, w, minv
    assert L.nek_cg_workspace_bytes(10, 8, 0) >= 3 * 8 * n


def test_ff_entry_points_reject_bad_arguments(lib):
    L = lib
    A16 = 0x10000
    assert L.nek_ax_ff(4, 1, A16, A16, A16, A16 * 2, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_ax_ff(-1, 8, A16, A16, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_ff(0, 8, None, None, None, None, None) == nekax.OK
    assert L.nek_ax_ff(4, 8, A16, None, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_ff(4, 8, A16, A16 + 8, A16, A16 * 2, None) == nekax.ERR_INVALID_ARG  # Gff misaligned
    assert L.nek_ax_ff(4, 8, A16, A16, A16 + 4, A16 * 2, None) == nekax.ERR_INVALID_ARG  # u misaligned
    assert L.nek_ax_ff(4, 8, A16, A16, A16, A16 + 4096, None) == nekax.ERR_INVALID_ARG  # overlap
    assert L.nek_ax_ff_energy(4, 1, A16, A16, A16, A16 * 2, A16 * 4, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_ax_ff_energy(0, 8, None, None, None, None, None, None) == nekax.OK
    assert L.nek_ax_ff_energy(4, 8, A16, A16, A16, A16 * 2, None, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_ff_energy(4, 8, A16, A16, A16, A16 * 2, A16 * 4 + 4, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_ff_energy(4, 8, A16, A16, A16, A16 * 2, A16 * 2 + 64, None) == nekax.ERR_INVALID_ARG  # on w
    assert L.nek_geom_ff(4, 1, A16, A16, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_geom_ff(4, 4, A16, A16 + 8, None) == nekax.ERR_INVALID_ARG
    assert L.nek_geom_ff(4, 4, A16, A16 + 64, None) == nekax.ERR_INVALID_ARG  # overlap
    # CG with the float-float operator but no split G
    opts = nekax.NekCgOpts(1, 0, 0.0, 0, 0, nekax.AX_FF, None)
    assert L.nek_cg_solve_ex(None, 1, 3, A16, A16, A16, None, A16, A16, 1e-8, 10, None, None, None,
                             ctypes.byref(opts), None) == nekax.ERR_INVALID_ARG


def test_tuning_and_lowp_entry_points_reject_bad_arguments(lib):
    L = lib
    A16 = 0x10000
    assert L.nek_set_ax_epb(7, 8, 1) == nekax.ERR_INVALID_ARG
    assert L.nek_set_ax_epb(0, 1, 1) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_set_ax_epb(0, 8, 3) == nekax.ERR_INVALID_ARG
    assert L.nek_set_ax_epb(1, 16, 4) == nekax.ERR_INVALID_ARG  # 4 x 1024 threads does not fit
    assert L.nek_set_ax_epb(1, 8, 2) == nekax.OK and L.nek_get_ax_epb(1, 8) == 2
    assert L.nek_set_ax_epb(1, 8, 0) == nekax.OK and L.nek_get_ax_epb(1, 8) == 0
    # NEK_AX_FF sets both float-float forms; NEK_AX_FF_ENERGY the energy form alone
    assert L.nek_set_ax_epb(1, 8, 4) == nekax.OK and L.nek_get_ax_epb(2, 8) == 4
    assert L.nek_set_ax_epb(2, 8, 1) == nekax.OK and L.nek_get_ax_epb(2, 8) == 1 and L.nek_get_ax_epb(1, 8) == 4
    assert L.nek_set_ax_epb(1, 8, 0) == nekax.OK and L.nek_get_ax_epb(2, 8) == 0
    assert L.nek_get_ax_epb(7, 8) == 0
    # nx = 12's item-mapped kernel at four elements per CTA (576 threads) just fits 227 KB of shared memory
    assert L.nek_set_ax_epb(1, 12, 4) == nekax.OK and L.nek_set_ax_epb(1, 12, 0) == nekax.OK
    assert L.nek_set_ax_epb(1, 10, 4) == nekax.OK and L.nek_set_ax_epb(1, 10, 0) == nekax.OK
    assert L.nek_tune_ax(0, 0, 8, A16, A16, A16, A16 * 2, None, None, None) == nekax.ERR_INVALID_ARG
    assert L.nek_tune_ax(0, 4, 8, A16, A16 + 8, A16, A16 * 2, None, None, None) == nekax.ERR_INVALID_ARG
    assert L.nek_tune_ax(0, 4, 8, A16, A16, A16, A16 + 64, None, None, None) == nekax.ERR_INVALID_ARG
    assert L.nek_lowp_bytes_per_value(0) == 4 and L.nek_lowp_bytes_per_value(1) == 2
    assert L.nek_lowp_bytes_per_value(2) == 2 and L.nek_lowp_bytes_per_value(3) == 0
    assert L.nek_geom_lowp(4, 8, 3, A16, A16, A16, None) == nekax.ERR_INVALID_ARG
    assert L.nek_geom_lowp(4, 1, 0, A16, A16, A16, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_ax_lowp(4, 8, 1, A16, A16, A16, A16, A16 + 64, None) == nekax.ERR_INVALID_ARG  # overlap
    assert L.nek_ax_lowp(4, 8, 5, A16, A16, A16, A16, A16 * 4, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_lowp(0, 8, 1, None, None, None, None, None, None) == nekax.OK
    info = nekax.NekMixedInfo()
    # inner_tol must be in (0, 1); tol must be > 0
    assert L.nek_cg_solve_mixed(None, 1, 3, A16, A16, None, 0, A16, A16, A16, None, A16, A16, 1e-8, 1.5, 5, 10,
                                None, ctypes.byref(info), None) == nekax.ERR_INVALID_ARG
    assert L.nek_cg_mixed_workspace_bytes(10, 8, 1) > 10 * 512 * (3 * 8 + 7 * 4)


def test_batch_entry_points_reject_bad_arguments(lib):
    L = lib
    h = ctypes.c_void_p()
    ne = np.array([2, 2], dtype=np.int64)
    nx_bad_order = np.array([8, 6], dtype=np.int32)
    nx_bad = np.array([6, 20], dtype=np.int32)
    glo = np.zeros(2 * 512, dtype=np.int64)
    assert L.nek_batch_create(0, ne.ctypes.data, nx_bad.ctypes.data, glo.ctypes.data, ctypes.byref(h)) == \
        nekax.ERR_INVALID_ARG
    assert L.nek_batch_create(2, ne.ctypes.data, nx_bad.ctypes.data, glo.ctypes.data, ctypes.byref(h)) == \
        nekax.ERR_UNSUPPORTED_NX
    assert L.nek_batch_create(2, ne.ctypes.data, nx_bad_order.ctypes.data, glo.ctypes.data, ctypes.byref(h)) == \
        nekax.ERR_INVALID_ARG
    assert L.nek_batch_destroy(None) == nekax.OK
    assert L.nek_batch_info(None, None, None, None) == nekax.ERR_INVALID_ARG
    assert L.nek_batch_workspace_bytes(None, 1) == 0
    stats = nekax.NekBatchStats()
    assert L.nek_batch_cg_solve(None, 0x100, None, 0x100, None, 0x100, 0x100, 1e-8, 10, 5, None, None, None, None,
                                ctypes.byref(stats), None) == nekax.ERR_INVALID_ARG


def test_lvec_entry_points_reject_bad_arguments(lib):
    L = lib
    h = ctypes.c_void_p()
    glo = np.array([0, 1, 1, 2], dtype=np.int64)
    good = np.array([1, 1, 1, 0], dtype=np.uint8)
    disagree = np.array([1, 1, 0, 0], dtype=np.uint8)  # the two copies of node 1 differ
    neg = np.array([0, -1, 1, 2], dtype=np.int64)
    assert L.nek_lvec_create(4, glo.ctypes.data, good.ctypes.data, None) == nekax.ERR_INVALID_ARG
    assert L.nek_lvec_create(-1, glo.ctypes.data, good.ctypes.data, ctypes.byref(h)) == nekax.ERR_INVALID_ARG
    assert L.nek_lvec_create(4, None, good.ctypes.data, ctypes.byref(h)) == nekax.ERR_INVALID_ARG
    assert L.nek_lvec_create(4, glo.ctypes.data, disagree.ctypes.data, ctypes.byref(h)) == nekax.ERR_INVALID_ARG
    assert L.nek_lvec_create(4, neg.ctypes.data, good.ctypes.data, ctypes.byref(h)) == nekax.ERR_INVALID_ARG
    assert L.nek_lvec_create(1 << 31, glo.ctypes.data, good.ctypes.data, ctypes.byref(h)) == nekax.ERR_TOO_LARGE
    assert h.value is None
    assert L.nek_lvec_destroy(None) == nekax.OK
    assert L.nek_lvec_size(None) == -1
    assert L.nek_lvec_cg_workspace_bytes(None) == 0
    for f in (L.nek_lvec_scatter, L.nek_lvec_restrict, L.nek_lvec_assemble):
        assert f(None, 0x100, 0x100, None) == nekax.ERR_INVALID_ARG
    assert L.nek_lvec_ax_ff(None, 1, 8, 0x100, 0x100, 0x100, 0x200, 0x300, None) == nekax.ERR_INVALID_ARG
    assert L.nek_lvec_ax_ff(None, 1, 17, 0x100, 0x100, 0x100, 0x200, 0x300, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_lvec_jacobi_minv(None, 1, 8, 0x100, 0x100, 0x100, 0x200, None) == nekax.ERR_INVALID_ARG
    it, rr = ctypes.c_int(7), ctypes.c_double(7.0)
    assert L.nek_lvec_cg_solve(None, 1, 8, 0x100, 0x100, 0x100, 0x100, 0x200, 1e-8, 10, None, ctypes.byref(it),
                               ctypes.byref(rr), None, None) == nekax.ERR_INVALID_ARG
    assert it.value == 0 and rr.value == 0.0


def test_net_apply_bf16_rejects_bad_arguments(lib):
    L = lib
    assert L.nek_net_apply_bf16(4, 10, 0x100, 0x100, 0x100, 0x100, 0x100, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_net_apply_bf16(-1, 8, 0x100, 0x100, 0x100, 0x100, 0x100, None) == nekax.ERR_INVALID_ARG
    assert L.nek_net_apply_bf16(4, 8, None, 0x100, 0x100, 0x100, 0x100, None) == nekax.ERR_INVALID_ARG
    assert L.nek_net_apply_bf16(0, 8, None, None, None, None, None, None) == nekax.OK


def test_ax_lowp_tc_rejects_bad_arguments(lib):
    L = lib
    A = 0x1000
    assert L.nek_ax_lowp_tc(4, 8, nekax.PREC_F32, A, A, A, A, A + 0x100000, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_lowp_tc(4, 17, nekax.PREC_BF16, A, A, A, A, A + 0x100000, None) == nekax.ERR_UNSUPPORTED_NX
    assert L.nek_ax_lowp_tc(-1, 8, nekax.PREC_BF16, A, A, A, A, A + 0x100000, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_lowp_tc(4, 8, nekax.PREC_F16, A, A, A, A, A, None) == nekax.ERR_INVALID_ARG  # u and w overlap
    assert L.nek_ax_lowp_tc(4, 8, nekax.PREC_F16, A + 2, A, A, A, A + 0x100000, None) == nekax.ERR_INVALID_ARG
    assert L.nek_ax_lowp_tc(0, 8, nekax.PREC_BF16, None, None, None, None, None, None) == nekax.OK


def test_cg_solve_host_rejects_bad_arguments_before_launch(lib):
    A = 0x10000
    L = lib
    assert L.nek_cg_host_staging_bytes(-1, 10) == 0 and L.nek_cg_host_staging_bytes(2, 1) == 0
    assert L.nek_cg_host_staging_bytes(2, 4) == 2 * 1024  # two vectors of 128 doubles, each 256-byte aligned
    # bad nx, no plan, negative size, bad tolerance, misaligned staging
    assert L.nek_cg_solve_host(None, 1, 1, A, A, A, A, A, A, 0.0, 1, None, None, None, None, None, None) == \
        nekax.ERR_UNSUPPORTED_NX
    assert L.nek_cg_solve_host(None, 1, 4, A, A, A, A, A, A, 0.0, 1, None, None, None, None, None, None) == \
        nekax.ERR_INVALID_ARG
    # the remaining checks need a plan (device memory): see the GPU test of nek_cg_solve_host
