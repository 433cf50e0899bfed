"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every function include/lqcd.h declares, and rejects bad arguments on the host
before touching the device."""
import ctypes

import pytest

from paper_1212_0785_gb300 import lqcd


@pytest.fixture(scope="module")
def L():
    return lqcd.lib()


def test_exports_every_declared_symbol(L):
    names = lqcd.header_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding marshals every declared function
    assert set(names) <= set(lqcd._SIGS), set(names) - set(lqcd._SIGS)


def test_version_and_error_string(L):
    assert "sm_103a" in lqcd.version()
    assert isinstance(L.lqcd_last_error(), bytes)
    assert lqcd.launch_count() >= 0


@pytest.mark.parametrize("dims", [(4, 4, 4, 3), (0, 4, 4, 4), (4, -2, 4, 4), (5, 4, 4, 4)])
def test_field_alloc_rejects_bad_lattice(L, dims):
    h = ctypes.c_void_p()
    rc = L.lqcd_field_alloc(ctypes.byref(lqcd.lattice(dims)), lqcd.GAUGE, lqcd.F64, 18, ctypes.byref(h))
    assert rc == lqcd.EINVAL
    assert b"even" in L.lqcd_last_error() or b"positive" in L.lqcd_last_error()
    assert not h.value


@pytest.mark.parametrize("kind,prec,recon", [(lqcd.GAUGE, lqcd.F64, 12), (lqcd.GAUGE, lqcd.F16N, 18),
                                             (lqcd.MOMENTUM, lqcd.F32, 0), (lqcd.SPINOR_FULL, lqcd.BF16, 0),
                                             (lqcd.SPINOR_EVEN, lqcd.F64, 12), (7, lqcd.F64, 0)])
def test_field_alloc_rejects_bad_combination(L, kind, prec, recon):
    h = ctypes.c_void_p()
    rc = L.lqcd_field_alloc(ctypes.byref(lqcd.lattice((4, 4, 4, 4))), kind, prec, recon, ctypes.byref(h))
    assert rc == lqcd.EINVAL and not h.value


def test_bad_boundary_and_huge_volume(L):
    h = ctypes.c_void_p()
    rc = L.lqcd_field_alloc(ctypes.byref(lqcd.lattice((4, 4, 4, 4), t_bc=0)), lqcd.GAUGE, lqcd.F64, 18,
                            ctypes.byref(h))
    assert rc == lqcd.EINVAL
    rc = L.lqcd_field_alloc(ctypes.byref(lqcd.lattice((2048, 2048, 2048, 2))), lqcd.GAUGE, lqcd.F64, 18,
                            ctypes.byref(h))
    assert rc == lqcd.EINVAL and b"2^31" in L.lqcd_last_error()


def test_null_arguments_are_rejected(L):
    p = lqcd.cg_params()
    info = lqcd.CgInfo()
    assert L.lqcd_cg_solve(None, None, None, None, 0.1, ctypes.byref(p), ctypes.byref(info), None) == lqcd.EINVAL
    assert L.lqcd_dslash(None, None, None, 0, None) == lqcd.EINVAL
    assert L.lqcd_plaquette(None, None, None) == lqcd.EINVAL
    assert L.lqcd_hmc_trajectory(None, None, None, None) == lqcd.EINVAL
    assert L.lqcd_df_split(None, 4, None, None, None) == lqcd.EINVAL
    assert L.lqcd_df_split(None, 0, None, None, None) == lqcd.OK  # nothing to do
    assert L.lqcd_field_free(None) == lqcd.OK


def test_timer_class_lists_are_checked_on_the_host(L):
    """every name of a timer-class list is checked before the device is touched"""
    for bad in (b"bogus", b"dslash_f16n,bogus", b"dslash_f16n,", b",dslash_f16n"):
        assert L.lqcd_kernel_timers_only(bad) == lqcd.EINVAL, bad
    assert b"unknown class" in L.lqcd_last_error()
    assert L.lqcd_kernel_timers_only(None) == lqcd.EINVAL
    assert L.lqcd_kernel_timer_read(b"bogus", None, None, None) == lqcd.EINVAL
    assert "dslash_f16n_plain" in lqcd.KERNEL_CLASSES


def test_allocator_hook_validation(L):
    a = lqcd.ALLOC_FN(lambda n, s, c: None)
    assert L.lqcd_set_allocator(a, lqcd.FREE_FN(), None) == lqcd.EINVAL
    assert L.lqcd_set_allocator(lqcd.ALLOC_FN(), lqcd.FREE_FN(), None) == lqcd.OK


def test_dslash_form_switch_is_host_state(L):
    """the FP16+norm hopping-term form is a process-wide host setting: set,
    query and restore need no device; an unknown form is refused and changes
    nothing"""
    prev = lqcd.dslash_form()
    try:
        assert prev in (lqcd.DSLASH_GATHER, lqcd.DSLASH_PREFETCH, lqcd.DSLASH_PACKED)
        lqcd.dslash_form(lqcd.DSLASH_GATHER)
        assert lqcd.dslash_form(lqcd.DSLASH_PREFETCH) == lqcd.DSLASH_GATHER
        assert lqcd.dslash_form() == lqcd.DSLASH_PREFETCH
        assert L.lqcd_dslash_form(7) == -1 and lqcd.dslash_form() == lqcd.DSLASH_PREFETCH
        assert b"unknown form" in L.lqcd_last_error()
        with pytest.raises(ValueError):
            lqcd.dslash_form(3)
    finally:
        lqcd.dslash_form(prev)


def test_info_structs_carry_the_solver_counters():
    """lqcd_cg_info and lqcd_traj_info end with the accurate-residual and
    failed-check counters (appended, so the earlier fields keep their offsets)"""
    names = [f for f, _ in lqcd.CgInfo._fields_]
    assert names[:4] == ["iters", "restarts", "true_rel_res", "seconds"]
    assert names[4:] == ["accurate_residuals", "failed_checks", "guess_refined"]
    tnames = [f for f, _ in lqcd.TrajInfo._fields_]
    assert tnames[-4:] == ["traj", "cg_accurate_residuals", "cg_failed_checks", "cg_guesses_refined"]


def test_autotune_table_is_host_state(tmp_path):
    """the threads-per-block table: a saved file loads into the process-wide
    table (one best row per class and lattice; block sizes this build cannot
    launch are ignored), lookups return it, clear empties it -- no device"""
    f = tmp_path / "tune.txt"
    f.write_text("# kernel Lx Ly Lz Lt block ms_per_launch best\n"
                 "gauge_force_f32 8 8 8 8 64 0.10 0\n"
                 "gauge_force_f32 8 8 8 8 96 0.08 1\n"
                 "dslash_f16n 8 8 8 8 256 0.02 1\n"
                 "link_update_f32 8 8 8 8 100 0.01 1\n"
                 "no_such_kernel 8 8 8 8 64 0.01 1\n")
    lqcd.autotune_clear()
    try:
        lqcd.autotune_load(f)
        assert lqcd.autotune_block("gauge_force_f32", (8, 8, 8, 8)) == 96
        assert lqcd.autotune_block("dslash_f16n", (8, 8, 8, 8)) == 256
        assert lqcd.autotune_block("link_update_f32", (8, 8, 8, 8)) == 0  # 100 is not a candidate
        assert lqcd.autotune_block("gauge_force_f32", (4, 4, 4, 4)) == 0
        rows = lqcd.read_tune_table(f)
        assert len(rows) == 5 and rows[1]["best"] and rows[1]["block"] == 96
        with pytest.raises(lqcd.LqcdError):
            lqcd.autotune_block("no_such_kernel", (8, 8, 8, 8))
    finally:
        lqcd.autotune_clear()
    assert lqcd.autotune_block("gauge_force_f32", (8, 8, 8, 8)) == 0
