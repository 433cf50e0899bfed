"""Thin ctypes binding of liblqcd.so (declared in include/lqcd.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch supplies the device allocator (its caching allocator,
installed as the library's allocator hook) and the CUDA stream.  There is no
CPU fallback: if the library cannot be built or loaded, every call raises.

Host arrays use the canonical layouts of include/lqcd.h as numpy arrays:
  gauge    complex128 (V, 4, 3, 3)      momentum float64 (V, 4, 8)
  half spinor (EVEN/ODD) complex128 (V/2, 4, 3) in checkerboard order
  full spinor complex128 (V, 4, 3)
"""
from __future__ import annotations

import ctypes
import json
import os
import re
import time
import threading

import numpy as np

from . import build as _build

# ---------------------------------------------------------------- constants

OK, EINVAL, ENOMEM, ENOCONV, ENUMERIC, ECUDA, EAGAIN, ETIMEOUT = range(8)
STATUS_NAMES = {0: "LQCD_OK", 1: "LQCD_EINVAL", 2: "LQCD_ENOMEM", 3: "LQCD_ENOCONV", 4: "LQCD_ENUMERIC",
                5: "LQCD_ECUDA", 6: "LQCD_EAGAIN", 7: "LQCD_ETIMEOUT"}
GAUGE, MOMENTUM, SPINOR_EVEN, SPINOR_ODD, SPINOR_FULL = range(5)
F64, F32, F16N, BF16 = range(4)
PREC_NAMES = {"f64": F64, "f32": F32, "f16n": F16N, "bf16": BF16}
LEAPFROG, OMELYAN = 0, 1


class LqcdError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# ---------------------------------------------------------------- structs

class Lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("t_bc", ctypes.c_int), ("xi0", ctypes.c_double), ("nu", ctypes.c_double)]


class CgParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("sloppy", ctypes.c_int),
                ("delta", ctypes.c_double), ("max_restarts", ctypes.c_int), ("guess", ctypes.c_int)]


class CgInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("true_rel_res", ctypes.c_double),
                ("seconds", ctypes.c_double), ("accurate_residuals", ctypes.c_int), ("failed_checks", ctypes.c_int),
                ("guess_refined", ctypes.c_int)]


class HmcParams(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("kappa", ctypes.c_double), ("tau", ctypes.c_double),
                ("nsteps", ctypes.c_int), ("integrator", ctypes.c_int), ("n_flavors", ctypes.c_int),
                ("cg", CgParams), ("reunitarize", ctypes.c_int), ("metropolis", ctypes.c_int),
                ("chrono", ctypes.c_int), ("force_prec", ctypes.c_int), ("hasenbusch_kappa", ctypes.c_double),
                ("gauge_substeps", ctypes.c_int), ("heavy_inner", ctypes.c_int), ("chrono_mre", ctypes.c_int)]


class ServiceParams(ctypes.Structure):
    _fields_ = [("cg", CgParams), ("hbm_budget", ctypes.c_size_t), ("max_active_rhs", ctypes.c_int)]


class SolveReq(ctypes.Structure):
    _fields_ = [("gauge", ctypes.c_int), ("kappa", ctypes.c_double), ("site", ctypes.c_int * 4),
                ("nrhs", ctypes.c_int)]


class SolveResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("nrhs", ctypes.c_int), ("iters", ctypes.c_int),
                ("refinements", ctypes.c_int), ("true_rel_res_max", ctypes.c_double), ("queue_s", ctypes.c_double),
                ("latency_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TrajInfo(ctypes.Structure):
    _fields_ = [("dH", ctypes.c_double), ("H0", ctypes.c_double), ("H1", ctypes.c_double),
                ("plaq", ctypes.c_double), ("u", ctypes.c_double), ("max_unitarity_dev", ctypes.c_double),
                ("seconds", ctypes.c_double), ("cg_true_rel_res_max", ctypes.c_double),
                ("accepted", ctypes.c_int), ("cg_iters", ctypes.c_int), ("n_solves", ctypes.c_int),
                ("cg_failures", ctypes.c_int), ("traj", ctypes.c_uint32), ("cg_accurate_residuals", ctypes.c_int),
                ("cg_failed_checks", ctypes.c_int), ("cg_guesses_refined", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# ---------------------------------------------------------------- loading

_vp, _sz, _u32, _i, _d = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)
_pp = ctypes.POINTER(ctypes.c_void_p)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_SIGS = {
    "lqcd_last_error": (ctypes.c_char_p, []),
    "lqcd_version": (ctypes.c_char_p, []),
    "lqcd_launch_count": (ctypes.c_uint64, []),
    "lqcd_set_allocator": (_i, [ALLOC_FN, FREE_FN, _vp]),
    "lqcd_kernel_timers": (_i, [_i]),
    "lqcd_kernel_timers_only": (_i, [ctypes.c_char_p]),
    "lqcd_kernel_timer_read": (_i, [ctypes.c_char_p, _dp, ctypes.POINTER(ctypes.c_uint64), _dp]),
    "lqcd_field_alloc": (_i, [ctypes.POINTER(Lattice), _i, _i, _i, _pp]),
    "lqcd_field_free": (_i, [_vp]),
    "lqcd_field_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "lqcd_field_data": (_i, [_vp, _pp, _pp]),
    "lqcd_field_upload": (_i, [_vp, _dp, _vp]),
    "lqcd_field_download": (_i, [_vp, _dp, _vp]),
    "lqcd_field_copy": (_i, [_vp, _vp, _vp]),
    "lqcd_philox_blocks": (_i, [_vp, _sz, _u32, _u32, _u32, _u32, _u32, _u32, _vp]),
    "lqcd_df_split": (_i, [_vp, _sz, _vp, _vp, _vp]),
    "lqcd_gauge_start": (_i, [_vp, _u32, _u32, _d, _vp]),
    "lqcd_momentum_refresh": (_i, [_vp, _u32, _u32, _u32, _vp]),
    "lqcd_eta_refresh": (_i, [_vp, _u32, _u32, _u32, _vp]),
    "lqcd_dslash": (_i, [_vp, _vp, _vp, _i, _vp]),
    "lqcd_dslash_form": (_i, [_i]),
    "lqcd_autotune": (_i, [ctypes.POINTER(Lattice), ctypes.c_char_p, _vp]),
    "lqcd_autotune_load": (_i, [ctypes.c_char_p]),
    "lqcd_autotune_block": (_i, [ctypes.c_char_p, ctypes.POINTER(Lattice), ctypes.POINTER(ctypes.c_int)]),
    "lqcd_autotune_clear": (_i, []),
    "lqcd_mhat": (_i, [_vp, _vp, _vp, _d, _i, _vp]),
    "lqcd_cg_solve": (_i, [_vp, _vp, _vp, _vp, _d, ctypes.POINTER(CgParams), ctypes.POINTER(CgInfo), _vp]),
    "lqcd_gauge_force": (_i, [_vp, _vp, _d, _d, _vp]),
    "lqcd_gauge_force_ex": (_i, [_vp, _vp, _d, _d, _i, _vp]),
    "lqcd_fermion_force": (_i, [_vp, _vp, _vp, _d, _d, _vp]),
    "lqcd_fermion_force_ex": (_i, [_vp, _vp, _vp, _d, _d, _i, _vp]),
    "lqcd_link_update": (_i, [_vp, _vp, _d, _vp, _vp]),
    "lqcd_link_update_ex": (_i, [_vp, _vp, _d, _vp, _i, _vp]),
    "lqcd_reunitarize": (_i, [_vp, _dp, _vp]),
    "lqcd_plaquette": (_i, [_vp, _dp, _vp]),
    "lqcd_plaquette_noalloc": (_i, [_vp, _vp, _vp]),
    "lqcd_kinetic_energy": (_i, [_vp, _dp, _vp]),
    "lqcd_spinor_dot": (_i, [_vp, _vp, _dp, _vp]),
    "lqcd_hmc_state_create": (_i, [_vp, _u32, _u32, _u32, _pp]),
    "lqcd_hmc_state_destroy": (_i, [_vp]),
    "lqcd_hmc_state_fields": (_i, [_vp, _pp, _pp, _pp]),
    "lqcd_hmc_state_traj": (_i, [_vp, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]),
    "lqcd_hmc_refresh": (_i, [_vp, ctypes.POINTER(HmcParams), _dp, _vp]),
    "lqcd_hmc_hamiltonian": (_i, [_vp, ctypes.POINTER(HmcParams), _dp, _vp]),
    "lqcd_md_step": (_i, [_vp, ctypes.POINTER(HmcParams), _vp]),
    "lqcd_hmc_trajectory": (_i, [_vp, ctypes.POINTER(HmcParams), ctypes.POINTER(TrajInfo), _vp]),
    "lqcd_cg_solve_batch": (_i, [_i, _pp, _pp, _pp, _pp, _dp, ctypes.POINTER(CgParams), ctypes.POINTER(CgInfo), _vp]),
    "lqcd_batch_create": (_i, [_pp, _i, _pp]),
    "lqcd_batch_destroy": (_i, [_vp]),
    "lqcd_batch_trajectory": (_i, [_vp, ctypes.POINTER(HmcParams), ctypes.POINTER(TrajInfo), _vp]),
    "lqcd_service_create": (_i, [ctypes.POINTER(ServiceParams), _pp]),
    "lqcd_service_add_gauge": (_i, [_vp, _vp, ctypes.POINTER(ctypes.c_int)]),
    "lqcd_solve_submit": (_i, [_vp, ctypes.POINTER(SolveReq), ctypes.POINTER(ctypes.c_uint64)]),
    "lqcd_solve_poll": (_i, [_vp, ctypes.c_uint64, ctypes.POINTER(SolveResult)]),
    "lqcd_solve_solution": (_i, [_vp, ctypes.c_uint64, _i, _pp, _pp]),
    "lqcd_solve_release": (_i, [_vp, ctypes.c_uint64]),
    "lqcd_service_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "lqcd_service_destroy": (_i, [_vp]),
    "lqcd_kernel_timers_every": (_i, [_i]),
}

_lock = threading.Lock()
_lib = None
_allocator_installed = False
_alloc_keep = []


def header_functions() -> list[str]:
    """Names of every function declared in include/lqcd.h."""
    txt = open(os.path.join(_build.INCLUDE, "lqcd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lqcd_[a-z0-9_]+)\s*\(", txt)))


def lib(build_if_needed: bool = True):
    """The loaded library (built first if missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_needed:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"{_build.LIB} is missing: run paper_1212_0785_gb300.build.build()")
            L = ctypes.CDLL(_build.LIB)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc, where):
    if rc != OK:
        raise LqcdError(rc, where, lib().lqcd_last_error().decode())
    return rc


def version() -> str:
    return lib().lqcd_version().decode()


def launch_count() -> int:
    return int(lib().lqcd_launch_count())


KERNEL_CLASSES = ("dslash_f64", "dslash_f32", "dslash_f16n", "dslash_bf16", "dslash_df64", "gauge_force",
                  "fermion_force", "link_update", "dslash_f16n_plain")


def kernel_timers(enable: bool, only: str | None = None, every: int = 1):
    """Enable (clearing the totals) or disable the library's per-class event
    timers; only: time those classes alone (comma-separated names); every:
    time one launch in every `every` of each class"""
    _check(lib().lqcd_kernel_timers_every(int(every)), "kernel_timers_every")
    if enable and only:
        _check(lib().lqcd_kernel_timers_only(only.encode()), "kernel_timers_only")
    else:
        _check(lib().lqcd_kernel_timers(int(enable)), "kernel_timers")


def kernel_timer_read(kernel_class: str):
    """(total milliseconds, launches, algorithmic bytes) of one kernel class
    since the timers were enabled"""
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    nb = ctypes.c_double()
    _check(lib().lqcd_kernel_timer_read(kernel_class.encode(), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(nb)),
           "kernel_timer_read")
    return ms.value, n.value, nb.value


# ---------------------------------------------------------------- torch plumbing

def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("liblqcd needs a CUDA device; none is visible")
    return torch


def install_torch_allocator():
    """Point the library's allocator hook at PyTorch's caching allocator."""
    global _allocator_installed
    if _allocator_installed:
        return
    torch = _torch()

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0) or None)
        except Exception:  # out of memory: the library reports LQCD_ENOMEM
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _alloc_keep.extend([a, f])
    _check(lib().lqcd_set_allocator(a, f, None), "set_allocator")
    _allocator_installed = True


def set_allocator(alloc, free):
    """Point the library's allocator hook at Python callables alloc(nbytes,
    stream) -> device pointer or None, and free(ptr, stream); None, None
    restores PyTorch's caching allocator.  Fields remember the hook that made
    them and are released through it."""
    global _allocator_installed
    if alloc is None:
        _allocator_installed = False
        install_torch_allocator()
        return

    def _alloc(nbytes, stream, ctx):
        try:
            return alloc(int(nbytes), stream)
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        free(int(ptr), stream)

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _alloc_keep.extend([a, f])
    _check(lib().lqcd_set_allocator(a, f, None), "set_allocator")
    _allocator_installed = True


def current_stream() -> int:
    return _torch().cuda.current_stream().cuda_stream


def _s(stream):
    return ctypes.c_void_p(current_stream() if stream is None else int(stream))


# ---------------------------------------------------------------- fields

def lattice(dims, t_bc=-1, xi0=1.0, nu=1.0) -> Lattice:
    """the lattice of a field: extents, fermion boundary factor in t, and the
    anisotropy of the actions (xi0: the gauge action's plaquettes with t weigh
    beta xi0, the spatial ones beta / xi0; the Wilson operator's spatial hops
    weigh nu / xi0)"""
    return Lattice((ctypes.c_int * 4)(*[int(d) for d in dims]), int(t_bc), float(xi0), float(nu))


class Field:
    """A device field owned by the library (lqcd_field*)."""

    def __init__(self, dims, kind, prec=F64, recon=None, t_bc=-1, aniso=(1.0, 1.0)):
        install_torch_allocator()
        self.dims = tuple(int(d) for d in dims)
        self.kind, self.prec, self.t_bc, self.aniso = kind, prec, t_bc, tuple(float(v) for v in aniso)
        if recon is None:
            recon = (18 if prec == F64 else 12) if kind == GAUGE else 0
        self.recon = recon
        h = ctypes.c_void_p()
        _check(lib().lqcd_field_alloc(ctypes.byref(lattice(dims, t_bc, *self.aniso)), kind, prec, recon,
                                      ctypes.byref(h)), "field_alloc")
        self.h = h
        self._owned = True

    @classmethod
    def borrowed(cls, handle, dims, kind, prec=F64, t_bc=-1, aniso=(1.0, 1.0)):
        f = cls.__new__(cls)
        f.dims, f.kind, f.prec, f.t_bc, f.aniso = tuple(dims), kind, prec, t_bc, tuple(aniso)
        f.recon = (18 if prec == F64 else 12) if kind == GAUGE else 0
        f.h = ctypes.c_void_p(handle)
        f._owned = False
        return f

    @property
    def V(self):
        return int(np.prod(self.dims))

    def host_shape(self):
        V = self.V
        return {GAUGE: (V, 4, 3, 3), MOMENTUM: (V, 4, 8), SPINOR_EVEN: (V // 2, 4, 3),
                SPINOR_ODD: (V // 2, 4, 3), SPINOR_FULL: (V, 4, 3)}[self.kind]

    def host_dtype(self):
        return np.float64 if self.kind == MOMENTUM else np.complex128

    def upload(self, arr, stream=None):
        a = np.ascontiguousarray(arr, dtype=self.host_dtype())
        assert a.shape == self.host_shape(), (a.shape, self.host_shape())
        buf = a.view(np.float64) if a.dtype == np.complex128 else a
        _check(lib().lqcd_field_upload(self.h, buf.ctypes.data_as(_dp), _s(stream)), "field_upload")
        return self

    def download(self, stream=None, out=None):
        a = out if out is not None else np.empty(self.host_shape(), self.host_dtype())
        buf = a.view(np.float64) if a.dtype == np.complex128 else a
        _check(lib().lqcd_field_download(self.h, buf.ctypes.data_as(_dp), _s(stream)), "field_download")
        return a

    def copy_from(self, src: "Field", stream=None):
        _check(lib().lqcd_field_copy(self.h, src.h, _s(stream)), "field_copy")
        return self

    def nbytes(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().lqcd_field_bytes(self.h, ctypes.byref(n)), "field_bytes")
        return n.value

    def data_ptr(self) -> int:
        p = ctypes.c_void_p()
        _check(lib().lqcd_field_data(self.h, ctypes.byref(p), None), "field_data")
        return p.value

    def free(self):
        if getattr(self, "_owned", False) and self.h:
            lib().lqcd_field_free(self.h)
            self.h = None
            self._owned = False

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def gauge_field(dims, prec=F64, t_bc=-1, aniso=(1.0, 1.0)):
    """aniso = (xi0, nu): the anisotropic actions (see lattice); every field of
    one computation carries the same"""
    return Field(dims, GAUGE, prec, t_bc=t_bc, aniso=aniso)


def spinor_field(dims, parity, prec=F64, t_bc=-1, aniso=(1.0, 1.0)):
    return Field(dims, SPINOR_EVEN if parity == 0 else SPINOR_ODD, prec, t_bc=t_bc, aniso=aniso)


def momentum_field(dims, t_bc=-1, aniso=(1.0, 1.0)):
    return Field(dims, MOMENTUM, F64, t_bc=t_bc, aniso=aniso)


# ---------------------------------------------------------------- operations

def df_split(in_ptr: int, n: int, pairs_ptr: int, back_ptr: int, stream=None):
    """the float-float codec on n device doubles (lqcd_df_split)"""
    _check(lib().lqcd_df_split(ctypes.c_void_p(in_ptr), n, ctypes.c_void_p(pairs_ptr), ctypes.c_void_p(back_ptr),
                               _s(stream)), "df_split")


def philox_blocks(out_ptr: int, n_blocks: int, ctr, key, stream=None):
    _check(lib().lqcd_philox_blocks(ctypes.c_void_p(out_ptr), n_blocks, *[int(c) for c in ctr],
                                    int(key[0]), int(key[1]), _s(stream)), "philox_blocks")


def gauge_start(U: Field, seed, eps, chain=0, stream=None):
    _check(lib().lqcd_gauge_start(U.h, seed, chain, eps, _s(stream)), "gauge_start")


def momentum_refresh(P: Field, seed, traj, chain=0, stream=None):
    _check(lib().lqcd_momentum_refresh(P.h, seed, chain, traj, _s(stream)), "momentum_refresh")


def eta_refresh(eta: Field, seed, traj, chain=0, stream=None):
    _check(lib().lqcd_eta_refresh(eta.h, seed, chain, traj, _s(stream)), "eta_refresh")


def dslash(out: Field, U: Field, inp: Field, dagger=False, stream=None):
    _check(lib().lqcd_dslash(out.h, U.h, inp.h, int(dagger), _s(stream)), "dslash")


def mhat(out: Field, U: Field, inp: Field, kappa, dagger=False, stream=None):
    _check(lib().lqcd_mhat(out.h, U.h, inp.h, kappa, int(dagger), _s(stream)), "mhat")


def cg_params(tol=1e-10, maxiter=10000, sloppy=F64, delta=0.1, max_restarts=3, guess=False) -> CgParams:
    return CgParams(tol, maxiter, sloppy, delta, max_restarts, int(guess))


def cg_solve(x: Field, U: Field, b: Field, kappa, params: CgParams | None = None, U_sloppy: Field | None = None,
             stream=None, check=True):
    """returns (status, CgInfo)"""
    params = params or cg_params()
    info = CgInfo()
    rc = lib().lqcd_cg_solve(x.h, U.h, U_sloppy.h if U_sloppy is not None else None, b.h, kappa,
                             ctypes.byref(params), ctypes.byref(info), _s(stream))
    if check and rc not in (OK, ENOCONV):
        _check(rc, "cg_solve")
    return rc, info


def gauge_force(P: Field, U: Field, beta, coeff, arith=None, stream=None):
    if arith is None:
        _check(lib().lqcd_gauge_force(P.h, U.h, beta, coeff, _s(stream)), "gauge_force")
    else:
        _check(lib().lqcd_gauge_force_ex(P.h, U.h, beta, coeff, arith, _s(stream)), "gauge_force_ex")


def fermion_force(P: Field, U: Field, X: Field, kappa, coeff, arith=None, stream=None):
    if arith is None:
        _check(lib().lqcd_fermion_force(P.h, U.h, X.h, kappa, coeff, _s(stream)), "fermion_force")
    else:
        _check(lib().lqcd_fermion_force_ex(P.h, U.h, X.h, kappa, coeff, arith, _s(stream)), "fermion_force_ex")


def link_update(U: Field, P: Field, c, U_sloppy: Field | None = None, stream=None, arith=None):
    """U <- exp(i c P) U (arith F32: the FP32 exponential with a float-float product)"""
    us = U_sloppy.h if U_sloppy is not None else None
    if arith is None:
        _check(lib().lqcd_link_update(U.h, P.h, c, us, _s(stream)), "link_update")
    else:
        _check(lib().lqcd_link_update_ex(U.h, P.h, c, us, int(arith), _s(stream)), "link_update_ex")


def reunitarize(U: Field, stream=None) -> float:
    d = ctypes.c_double()
    _check(lib().lqcd_reunitarize(U.h, ctypes.byref(d), _s(stream)), "reunitarize")
    return d.value


def plaquette(U: Field, stream=None) -> float:
    d = ctypes.c_double()
    _check(lib().lqcd_plaquette(U.h, ctypes.byref(d), _s(stream)), "plaquette")
    return d.value


def kinetic_energy(P: Field, stream=None) -> float:
    d = ctypes.c_double()
    _check(lib().lqcd_kinetic_energy(P.h, ctypes.byref(d), _s(stream)), "kinetic_energy")
    return d.value


def spinor_dot(a: Field, b: Field, stream=None) -> float:
    d = ctypes.c_double()
    _check(lib().lqcd_spinor_dot(a.h, b.h, ctypes.byref(d), _s(stream)), "spinor_dot")
    return d.value


# ---------------------------------------------------------------- HMC

def hmc_params(beta, kappa, tau=1.0, nsteps=10, integrator=LEAPFROG, n_flavors=2, cg=None, reunitarize=True,
               metropolis=True, force_prec=F64, chrono=False, hasenbusch_kappa=0.0, gauge_substeps=0,
               heavy_inner=False, chrono_mre=False) -> HmcParams:
    return HmcParams(beta, kappa, tau, nsteps, integrator, n_flavors, cg or cg_params(), int(reunitarize),
                     int(metropolis), int(chrono), int(force_prec), float(hasenbusch_kappa), int(gauge_substeps),
                     int(heavy_inner), int(chrono_mre))


class HmcState:
    """One Markov chain on the device; borrows the FP64 gauge field U."""

    def __init__(self, U: Field, seed, chain=0, traj0=0):
        h = ctypes.c_void_p()
        _check(lib().lqcd_hmc_state_create(U.h, seed, chain, traj0, ctypes.byref(h)), "hmc_state_create")
        self.h, self.U, self.seed, self.chain = h, U, int(seed), int(chain)

    def fields(self):
        u, p, phi = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().lqcd_hmc_state_fields(self.h, ctypes.byref(u), ctypes.byref(p), ctypes.byref(phi)),
               "hmc_state_fields")
        d, t, a = self.U.dims, self.U.t_bc, self.U.aniso
        return (self.U, Field.borrowed(p.value, d, MOMENTUM, t_bc=t, aniso=a),
                Field.borrowed(phi.value, d, SPINOR_EVEN, t_bc=t, aniso=a))

    @property
    def traj(self) -> int:
        v = ctypes.c_uint32()
        _check(lib().lqcd_hmc_state_traj(self.h, ctypes.byref(v), None), "hmc_state_traj")
        return v.value

    @traj.setter
    def traj(self, value):
        v = ctypes.c_uint32(value)
        _check(lib().lqcd_hmc_state_traj(self.h, None, ctypes.byref(v)), "hmc_state_traj")

    def refresh(self, params: HmcParams, stream=None) -> float:
        H = ctypes.c_double()
        _check(lib().lqcd_hmc_refresh(self.h, ctypes.byref(params), ctypes.byref(H), _s(stream)), "hmc_refresh")
        return H.value

    def hamiltonian(self, params: HmcParams, stream=None) -> float:
        H = ctypes.c_double()
        _check(lib().lqcd_hmc_hamiltonian(self.h, ctypes.byref(params), ctypes.byref(H), _s(stream)),
               "hmc_hamiltonian")
        return H.value

    def md_step(self, params: HmcParams, stream=None):
        _check(lib().lqcd_md_step(self.h, ctypes.byref(params), _s(stream)), "md_step")

    def trajectory(self, params: HmcParams, stream=None, log=None) -> dict:
        """One trajectory; its info as a dict.  log: a path or a text file to
        which one JSON line with the trajectory's metrics is appended."""
        info = TrajInfo()
        rc = lib().lqcd_hmc_trajectory(self.h, ctypes.byref(params), ctypes.byref(info), _s(stream))
        d = info.as_dict()
        if log is not None:
            write_log_line(log, dict(d, status=int(rc), seed=self.seed, chain=self.chain, dims=list(self.U.dims),
                                     time=time.time()))
        _check(rc, "hmc_trajectory")
        return d

    def checkpoint(self, path):
        """Saves what resuming this chain needs -- the FP64 links in the
        canonical host layout, the Philox key (seed, chain) and the trajectory
        counter -- to an .npz file.  The random numbers of every trajectory
        follow from (seed, chain, traj) alone, so a resumed chain repeats the
        unbroken one bit for bit."""
        np.savez(path, U=self.U.download(), dims=np.array(self.U.dims), t_bc=self.U.t_bc,
                 aniso=np.array(self.U.aniso), seed=self.seed,
                 chain=self.chain, traj=self.traj)

    @classmethod
    def resume(cls, path) -> "HmcState":
        """A new chain state (and its FP64 gauge field, state.U) from a checkpoint file."""
        z = np.load(path)
        U = gauge_field(tuple(int(v) for v in z["dims"]), t_bc=int(z["t_bc"]),
                        aniso=tuple(float(v) for v in z["aniso"])).upload(z["U"])
        return cls(U, int(z["seed"]), int(z["chain"]), int(z["traj"]))

    def close(self):
        if self.h:
            lib().lqcd_hmc_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batches

TUNED_CLASSES = ("dslash_f16n", "gauge_force_f32", "gauge_force_f64", "fermion_force_f32", "link_update_f32")


def autotune(dims, path=None, t_bc=-1, stream=None) -> dict:
    """Times every candidate block size of the tunable kernel classes on a
    lattice (paper Sec. 4), keeps the fastest for later launches on it, writes
    the timings to path (if given); returns {class: block}."""
    lat = lattice(dims, t_bc)
    _check(lib().lqcd_autotune(ctypes.byref(lat), None if path is None else str(path).encode(), _s(stream)),
           "autotune")
    return {k: autotune_block(k, dims, t_bc) for k in TUNED_CLASSES}


def autotune_load(path):
    _check(lib().lqcd_autotune_load(str(path).encode()), "autotune_load")


def autotune_block(kernel_class, dims, t_bc=-1) -> int:
    """the tuned block size of a class on a lattice (0: not tuned)"""
    lat = lattice(dims, t_bc)
    b = ctypes.c_int()
    _check(lib().lqcd_autotune_block(kernel_class.encode(), ctypes.byref(lat), ctypes.byref(b)), "autotune_block")
    return b.value


def autotune_clear():
    _check(lib().lqcd_autotune_clear(), "autotune_clear")


def read_tune_table(path) -> list[dict]:
    """the rows of an autotune file"""
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, lx, ly, lz, lt, block, ms, best = line.split()
        rows.append({"class": k, "dims": (int(lx), int(ly), int(lz), int(lt)), "block": int(block),
                     "ms": float(ms), "best": best == "1"})
    return rows


def write_log_line(log, record: dict):
    """Appends record as one JSON line to log (a path or a text file)."""
    line = json.dumps(record, sort_keys=True) + "\n"
    if hasattr(log, "write"):
        log.write(line)
        log.flush()
    else:
        with open(log, "a") as fh:
            fh.write(line)


def _ptrs(fields):
    arr = (ctypes.c_void_p * max(1, len(fields)))()
    for i, f in enumerate(fields):
        arr[i] = f.h.value if isinstance(f.h, ctypes.c_void_p) else f.h
    return arr


def cg_solve_batch(xs, Us, U_sloppys, bs, kappas, params: CgParams, stream=None, check=True):
    """n independent mixed solves with shared launches; returns (status, [CgInfo])"""
    n = len(xs)
    infos = (CgInfo * max(1, n))()
    k = (ctypes.c_double * max(1, n))(*kappas)
    rc = lib().lqcd_cg_solve_batch(n, _ptrs(xs), _ptrs(Us), _ptrs(U_sloppys), _ptrs(bs), k, ctypes.byref(params),
                                   infos, _s(stream))
    if check and rc not in (OK, ENOCONV):
        _check(rc, "cg_solve_batch")
    return rc, [infos[i] for i in range(n)]


class Batch:
    """Chains (HmcState) advanced together, their solves in shared launches."""

    def __init__(self, states):
        self.states = list(states)
        arr = (ctypes.c_void_p * len(self.states))(*[s.h.value for s in self.states])
        h = ctypes.c_void_p()
        _check(lib().lqcd_batch_create(arr, len(self.states), ctypes.byref(h)), "batch_create")
        self.h = h

    def trajectory(self, params, stream=None):
        n = len(self.states)
        if isinstance(params, HmcParams):
            params = [params] * n
        parr = (HmcParams * n)(*params)
        infos = (TrajInfo * n)()
        _check(lib().lqcd_batch_trajectory(self.h, parr, infos, _s(stream)), "batch_trajectory")
        return [infos[i].as_dict() for i in range(n)]

    def close(self):
        if self.h:
            lib().lqcd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- solve service

def service_params(tol=1e-10, maxiter=20000, sloppy=F16N, delta=0.003, hbm_budget=64 << 30,
                   max_active_rhs=0) -> ServiceParams:
    return ServiceParams(cg_params(tol=tol, maxiter=maxiter, sloppy=sloppy, delta=delta), int(hbm_budget),
                         int(max_active_rhs))


class Service:
    """Point-source Wilson-Dirac solves on resident gauge fields, continuously
    batched by the library's worker thread."""

    def __init__(self, params: ServiceParams):
        install_torch_allocator()
        h = ctypes.c_void_p()
        _check(lib().lqcd_service_create(ctypes.byref(params), ctypes.byref(h)), "service_create")
        self.h = h
        self.gauges = {}

    def add_gauge(self, U: Field) -> int:
        gid = ctypes.c_int()
        _check(lib().lqcd_service_add_gauge(self.h, U.h, ctypes.byref(gid)), "service_add_gauge")
        self.gauges[gid.value] = U
        return gid.value

    def submit(self, gauge, kappa, site, nrhs=12) -> int:
        req = SolveReq(int(gauge), float(kappa), (ctypes.c_int * 4)(*[int(c) for c in site]), int(nrhs))
        t = ctypes.c_uint64()
        _check(lib().lqcd_solve_submit(self.h, ctypes.byref(req), ctypes.byref(t)), "solve_submit")
        return t.value

    def poll(self, ticket):
        """None while pending, else the result as a dict"""
        r = SolveResult()
        rc = lib().lqcd_solve_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(r))
        if rc == EAGAIN:
            return None
        _check(rc, "solve_poll")
        return r.as_dict()

    def wait(self, ticket, timeout=600.0):
        import time
        t0 = time.perf_counter()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError(f"solve {ticket} not done after {timeout} s")
            time.sleep(2e-4)

    def solution(self, ticket, k):
        """(x_e, x_o) of right-hand side k as borrowed F64 fields"""
        e, o = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().lqcd_solve_solution(self.h, ctypes.c_uint64(ticket), int(k), ctypes.byref(e), ctypes.byref(o)),
               "solve_solution")
        return e.value, o.value

    def release(self, ticket):
        _check(lib().lqcd_solve_release(self.h, ctypes.c_uint64(ticket)), "solve_release")

    def bytes(self):
        """(counted, fixed): the device bytes hbm_budget covers, and the gauge
        fields' link copies and shared temporaries outside it"""
        c, f = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib().lqcd_service_bytes(self.h, ctypes.byref(c), ctypes.byref(f)), "service_bytes")
        return c.value, f.value

    def close(self):
        if self.h:
            rc = lib().lqcd_service_destroy(self.h)
            self.h = None
            _check(rc, "service_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


DSLASH_GATHER, DSLASH_PREFETCH, DSLASH_PACKED = 0, 1, 2


def dslash_form(form=None) -> int:
    """query (None) or select the form of the FP16+norm hopping term: 0
    gathered, 1 prefetched links, 2 prefetched links with packed FP32x2
    arithmetic (the default); returns the previous form"""
    if form is not None and int(form) not in (0, 1, 2):
        raise ValueError("dslash form must be 0, 1 or 2")
    return int(lib().lqcd_dslash_form(-1 if form is None else int(form)))
