"""ctypes binding of the FP64 CPU oracle (lqcd_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline / reference legs of ``bench.py``.  The product library
never loads it.

Array conventions (numpy, C order, lexicographic site i = x + Lx(y + Ly(z + Lz t))):
  U    complex128 (V, 4, 3, 3)   link U_mu(x)[row][col]
  psi  complex128 (V, 4, 3)      spinor [spin][color]; even/odd fields are
                                 full-lattice arrays with the other parity zero
  P    float64    (V, 4, 8)      momentum Gell-Mann coefficients p_a
dims = (Lx, Ly, Lz, Lt), t_bc = -1 (antiperiodic fermions in t) or +1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lqcd_oracle.c")
_LIBS = {"serial": os.path.join(_HERE, "liblqcd_oracle.so"),
         "openmp": os.path.join(_HERE, "liblqcd_oracle_omp.so")}
_lock = threading.Lock()
_loaded = {}
_variant = "serial"

CFLAGS = ["-O2", "-fPIC", "-shared", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False, variant: str = "serial") -> str:
    """Compile lqcd_oracle.c into liblqcd_oracle.so (serial) or
    liblqcd_oracle_omp.so (the same source with -fopenmp) next to it (gcc)."""
    out = _LIBS[variant]
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    extra = ["-fopenmp"] if variant == "openmp" else []
    subprocess.check_call(["gcc", *CFLAGS, *extra, _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


def use_openmp(on: bool) -> str:
    """Select the build every call below goes to (the OpenMP build spreads the
    site loops over OMP_NUM_THREADS threads, bitwise the same results);
    returns the previous selection."""
    global _variant
    prev = _variant
    _variant = "openmp" if on else "serial"
    return prev


def lib():
    with _lock:
        L = _loaded.get(_variant)
        if L is None:
            build(variant=_variant)
            L = ctypes.CDLL(_LIBS[_variant])
            _declare(L)
            _loaded[_variant] = L
    return L


class anisotropy:
    """Context in which every oracle call uses the anisotropic Wilson actions:
    the gauge plaquettes of the planes with t weighted by xi0 and the spatial
    ones by 1/xi0 (beta xi0 and beta / xi0), the spatial hops of the Wilson
    operator by nu / xi0 (the t hops by 1).  (1, 1) is the isotropic action."""

    def __init__(self, xi0, nu):
        self.xi0, self.nu = float(xi0), float(nu)

    def __enter__(self):
        lib().or_set_anisotropy(self.xi0, self.nu)
        return self

    def __exit__(self, *exc):
        lib().or_set_anisotropy(1.0, 1.0)


def num_threads() -> int:
    """threads the selected build's site loops use"""
    return int(lib().or_num_threads())


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)
_up = ctypes.POINTER(ctypes.c_uint32)
_i, _d, _u32, _l = ctypes.c_int, ctypes.c_double, ctypes.c_uint32, ctypes.c_long


def _declare(L):
    sig = {
        "or_num_threads": (_i, []),
        "or_set_anisotropy": (None, [_d, _d]),
        "or_gamma": (None, [_i, _dp]),
        "or_philox4x32_10": (None, [_up, _up, _up]),
        "or_uniform2": (None, [_u32] * 6 + [_dp]),
        "or_gauss2": (None, [_u32] * 6 + [_dp]),
        "or_plaquette": (_i, [_ip, _dp, _dp]),
        "or_gauge_action": (_i, [_ip, _dp, _d, _dp]),
        "or_dslash": (_i, [_ip, _i, _dp, _dp, _dp, _i, _i]),
        "or_dslash_at": (_i, [_ip, _i, _dp, _dp, _i, _l, _lp, _dp]),
        "or_mhat": (_i, [_ip, _i, _dp, _d, _dp, _dp, _i]),
        "or_mdagm": (_i, [_ip, _i, _dp, _d, _dp, _dp]),
        "or_cg": (_i, [_ip, _i, _dp, _d, _dp, _dp, _d, _i, _ip, _dp]),
        "or_gauge_force": (_i, [_ip, _dp, _d, _dp]),
        "or_gauge_force_at": (_i, [_ip, _dp, _d, _l, _lp, _dp]),
        "or_fermion_force": (_i, [_ip, _i, _dp, _d, _dp, _l, _lp, _dp]),
        "or_fermion_action": (_i, [_ip, _i, _dp, _d, _dp, _d, _i, _dp, _ip]),
        "or_su3_expi": (None, [_dp, _d, _dp]),
        "or_algebra_to_mat": (None, [_dp, _dp]),
        "or_reunit_mat": (None, [_dp, _dp]),
        "or_gauge_start": (_i, [_ip, _u32, _u32, _d, _dp]),
        "or_momentum_refresh": (_i, [_ip, _u32, _u32, _u32, _dp]),
        "or_eta_refresh": (_i, [_ip, _u32, _u32, _u32, _dp]),
        "or_link_update": (_i, [_ip, _dp, _dp, _d]),
        "or_reunitarize": (_i, [_ip, _dp, _dp]),
        "or_kinetic": (_d, [_ip, _dp]),
        "or_md_integrate": (_i, [_ip, _i, _dp, _dp, _dp, _d, _d, _d, _i, _i, _i, _d, _i, _dp]),
        "or_hamiltonian": (_i, [_ip, _i, _dp, _dp, _dp, _d, _d, _i, _d, _i, _dp]),
        "or_hmc_trajectory": (_i, [_ip, _i, _dp, _d, _d, _d, _i, _i, _i, _d, _i,
                                   _u32, _u32, _u32, _i, _i, _dp]),
        "or_eta_refresh_h": (_i, [_ip, _u32, _u32, _u32, _dp]),
        "or_hasenbusch_ratio": (_i, [_ip, _i, _dp, _d, _d, _dp, _d, _i, _dp, _dp]),
        "or_hasenbusch_refresh": (_i, [_ip, _i, _dp, _d, _d, _dp, _dp, _d, _i, _dp, _dp]),
        "or_hmc_trajectory_hb": (_i, [_ip, _i, _dp, _d, _d, _d, _d, _i, _i, _i, _i, _i, _d, _i,
                                      _u32, _u32, _u32, _i, _i, _dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


# ----------------------------------------------------------------- helpers

def _dims(dims):
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    return d


def _vol(dims):
    return int(np.prod(dims))


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.complex128:
        return a.view(np.float64).ctypes.data_as(_dp)
    assert a.dtype == np.float64, a.dtype
    return a.ctypes.data_as(_dp)


def _check(rc):
    if rc < 0:
        raise ValueError("oracle: invalid lattice geometry (dims must be positive and even)")
    return rc


def new_gauge(dims):
    return np.zeros((_vol(dims), 4, 3, 3), np.complex128)


def new_spinor(dims):
    return np.zeros((_vol(dims), 4, 3), np.complex128)


def new_momentum(dims):
    return np.zeros((_vol(dims), 4, 8), np.float64)


def parity(dims) -> np.ndarray:
    """parity (x+y+z+t) % 2 of every lexicographic site"""
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return ((x + y + z + t) % 2).reshape(-1)


# ----------------------------------------------------------------- API

def gamma(which: int) -> np.ndarray:
    out = np.zeros((4, 4), np.complex128)
    lib().or_gamma(which, _ptr(out))
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return np.array(list(o), np.uint32)


def uniform2(seed, chain, site, j, purpose, traj):
    o = np.zeros(2)
    lib().or_uniform2(seed, chain, site, j, purpose, traj, _ptr(o))
    return o


def gauss2(seed, chain, site, j, purpose, traj):
    o = np.zeros(2)
    lib().or_gauss2(seed, chain, site, j, purpose, traj, _ptr(o))
    return o


def plaquette(dims, U) -> float:
    o = ctypes.c_double()
    _check(lib().or_plaquette(_dims(dims), _ptr(U), ctypes.byref(o)))
    return o.value


def gauge_action(dims, U, beta) -> float:
    o = ctypes.c_double()
    _check(lib().or_gauge_action(_dims(dims), _ptr(U), beta, ctypes.byref(o)))
    return o.value


def dslash(dims, U, psi, dagger=False, out_parity=-1, t_bc=-1) -> np.ndarray:
    out = new_spinor(dims)
    _check(lib().or_dslash(_dims(dims), t_bc, _ptr(U), _ptr(psi), _ptr(out), int(dagger), out_parity))
    return out


def dslash_at(dims, U, psi, sites, dagger=False, t_bc=-1) -> np.ndarray:
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.zeros((len(sites), 4, 3), np.complex128)
    _check(lib().or_dslash_at(_dims(dims), t_bc, _ptr(U), _ptr(psi), int(dagger), len(sites),
                              sites.ctypes.data_as(_lp), _ptr(out)))
    return out


def mhat(dims, U, kappa, psi, dagger=False, t_bc=-1) -> np.ndarray:
    out = new_spinor(dims)
    _check(lib().or_mhat(_dims(dims), t_bc, _ptr(U), kappa, _ptr(psi), _ptr(out), int(dagger)))
    return out


def mdagm(dims, U, kappa, psi, t_bc=-1) -> np.ndarray:
    out = new_spinor(dims)
    _check(lib().or_mdagm(_dims(dims), t_bc, _ptr(U), kappa, _ptr(psi), _ptr(out)))
    return out


def cg(dims, U, kappa, b, tol=1e-10, maxiter=10000, t_bc=-1):
    """returns (x, converged, iters, true_rel_res)"""
    x = new_spinor(dims)
    it = ctypes.c_int()
    rel = ctypes.c_double()
    rc = _check(lib().or_cg(_dims(dims), t_bc, _ptr(U), kappa, _ptr(b), _ptr(x), tol, maxiter,
                            ctypes.byref(it), ctypes.byref(rel)))
    return x, rc == 0, it.value, rel.value


def gauge_force(dims, U, beta, links=None) -> np.ndarray:
    if links is None:
        F = new_momentum(dims)
        _check(lib().or_gauge_force(_dims(dims), _ptr(U), beta, _ptr(F)))
        return F
    links = np.ascontiguousarray(links, dtype=np.int64)
    F = np.zeros((len(links), 8))
    _check(lib().or_gauge_force_at(_dims(dims), _ptr(U), beta, len(links), links.ctypes.data_as(_lp), _ptr(F)))
    return F


def fermion_force(dims, U, kappa, X, links=None, t_bc=-1) -> np.ndarray:
    if links is None:
        F = new_momentum(dims)
        _check(lib().or_fermion_force(_dims(dims), t_bc, _ptr(U), kappa, _ptr(X), -1, None, _ptr(F)))
        return F
    links = np.ascontiguousarray(links, dtype=np.int64)
    F = np.zeros((len(links), 8))
    _check(lib().or_fermion_force(_dims(dims), t_bc, _ptr(U), kappa, _ptr(X), len(links),
                                  links.ctypes.data_as(_lp), _ptr(F)))
    return F


def fermion_action(dims, U, kappa, phi, tol=1e-12, maxiter=10000, t_bc=-1):
    S = ctypes.c_double()
    it = ctypes.c_int()
    _check(lib().or_fermion_action(_dims(dims), t_bc, _ptr(U), kappa, _ptr(phi), tol, maxiter,
                                   ctypes.byref(S), ctypes.byref(it)))
    return S.value


def su3_expi(H: np.ndarray, c: float) -> np.ndarray:
    H = np.ascontiguousarray(H, np.complex128)
    out = np.zeros((3, 3), np.complex128)
    lib().or_su3_expi(_ptr(H), c, _ptr(out))
    return out


def algebra_to_mat(c8) -> np.ndarray:
    c8 = np.ascontiguousarray(c8, np.float64)
    out = np.zeros((3, 3), np.complex128)
    lib().or_algebra_to_mat(_ptr(c8), _ptr(out))
    return out


def reunit_mat(m) -> np.ndarray:
    m = np.ascontiguousarray(m, np.complex128)
    out = np.zeros((3, 3), np.complex128)
    lib().or_reunit_mat(_ptr(m), _ptr(out))
    return out


def gauge_start(dims, seed, eps, chain=0) -> np.ndarray:
    U = new_gauge(dims)
    _check(lib().or_gauge_start(_dims(dims), seed, chain, eps, _ptr(U)))
    return U


def momentum_refresh(dims, seed, traj, chain=0) -> np.ndarray:
    P = new_momentum(dims)
    _check(lib().or_momentum_refresh(_dims(dims), seed, chain, traj, _ptr(P)))
    return P


def eta_refresh(dims, seed, traj, chain=0) -> np.ndarray:
    e = new_spinor(dims)
    _check(lib().or_eta_refresh(_dims(dims), seed, chain, traj, _ptr(e)))
    return e


def link_update(dims, U, P, c) -> np.ndarray:
    U = U.copy()
    _check(lib().or_link_update(_dims(dims), _ptr(U), _ptr(P), c))
    return U


def reunitarize(dims, U):
    U = U.copy()
    m = ctypes.c_double()
    _check(lib().or_reunitarize(_dims(dims), _ptr(U), ctypes.byref(m)))
    return U, m.value


def kinetic(dims, P) -> float:
    return lib().or_kinetic(_dims(dims), _ptr(P))


LEAPFROG, OMELYAN = 0, 1


def md_integrate(dims, U, P, phi, beta, kappa, tau, nsteps, integrator=LEAPFROG, n_flavors=2,
                 cg_tol=1e-10, cg_maxiter=10000, t_bc=-1):
    """returns (U, P, stats) with stats = [cg_iters, n_solves, cg_failures]"""
    U = U.copy()
    P = P.copy()
    if phi is None:
        phi = new_spinor(dims)
    st = np.zeros(3)
    _check(lib().or_md_integrate(_dims(dims), t_bc, _ptr(U), _ptr(P), _ptr(phi), beta, kappa, tau, nsteps,
                                 integrator, n_flavors, cg_tol, cg_maxiter, _ptr(st)))
    return U, P, st


def hamiltonian(dims, U, P, phi, beta, kappa, n_flavors=2, cg_tol=1e-12, cg_maxiter=10000, t_bc=-1):
    if phi is None:
        phi = new_spinor(dims)
    H = ctypes.c_double()
    _check(lib().or_hamiltonian(_dims(dims), t_bc, _ptr(U), _ptr(P), _ptr(phi), beta, kappa, n_flavors,
                                cg_tol, cg_maxiter, ctypes.byref(H)))
    return H.value


TRAJ_KEYS = ("dH", "accepted", "plaq", "cg_iters", "H0", "H1", "u", "max_unitarity_dev", "n_solves",
             "cg_failures")


def hmc_trajectory(dims, U, beta, kappa, tau, nsteps, integrator=LEAPFROG, n_flavors=2, cg_tol=1e-10,
                   cg_maxiter=10000, seed=1, chain=0, traj=0, reunit=True, metropolis=True, t_bc=-1):
    """one full trajectory; returns (U_new, info dict)"""
    U = U.copy()
    info = np.zeros(10)
    _check(lib().or_hmc_trajectory(_dims(dims), t_bc, _ptr(U), beta, kappa, tau, nsteps, integrator,
                                   n_flavors, cg_tol, cg_maxiter, seed, chain, traj, int(reunit),
                                   int(metropolis), _ptr(info)))
    return U, dict(zip(TRAJ_KEYS, info.tolist()))


def eta_refresh_h(dims, seed, traj, chain=0) -> np.ndarray:
    """the Hasenbusch action's second eta (Philox purpose 4)"""
    eta = new_spinor(dims)
    _check(lib().or_eta_refresh_h(_dims(dims), seed, chain, traj, _ptr(eta)))
    return eta


def hasenbusch_ratio(dims, U, kappa, kappa_h, phi_r, tol=1e-12, maxiter=10000, force=True, t_bc=-1):
    """S_r = chi^dag (Mhat^dag Mhat)^-1 chi, chi = W^dag phi_r with W = Mhat(kappa_h),
    and its force coefficients (V, 4, 8) (Sec. 6.2: mass preconditioning)"""
    S = ctypes.c_double()
    F = new_momentum(dims) if force else None
    rc = lib().or_hasenbusch_ratio(_dims(dims), t_bc, _ptr(U), kappa, kappa_h, _ptr(phi_r), tol, maxiter,
                                   ctypes.byref(S), _ptr(F) if force else None)
    if rc < 0:
        raise ValueError("bad geometry")
    return S.value, F


def hasenbusch_refresh(dims, U, kappa, kappa_h, eta, eta_h, tol=1e-12, maxiter=10000, t_bc=-1):
    """(phi_r, phi_h) = (W (W^dag W)^-1 Mhat^dag eta, W^dag eta_h)"""
    phi_r, phi_h = new_spinor(dims), new_spinor(dims)
    rc = lib().or_hasenbusch_refresh(_dims(dims), t_bc, _ptr(U), kappa, kappa_h, _ptr(eta), _ptr(eta_h), tol,
                                     maxiter, _ptr(phi_r), _ptr(phi_h))
    if rc < 0:
        raise ValueError("bad geometry")
    return phi_r, phi_h


def hmc_trajectory_hb(dims, U, beta, kappa, kappa_h, tau, nsteps, integrator=LEAPFROG, n_flavors=2,
                      gauge_substeps=0, heavy_inner=False, cg_tol=1e-10, cg_maxiter=10000, seed=1, chain=0, traj=0,
                      reunit=True, metropolis=True, t_bc=-1):
    """one trajectory with the Hasenbusch action (kappa_h > 0) and the nested
    integrator (gauge_substeps >= 2); returns (U_new, info dict)"""
    U = U.copy()
    info = np.zeros(10)
    _check(lib().or_hmc_trajectory_hb(_dims(dims), t_bc, _ptr(U), beta, kappa, kappa_h, tau, nsteps, integrator,
                                      n_flavors, gauge_substeps, int(heavy_inner), cg_tol, cg_maxiter, seed, chain,
                                      traj, int(reunit), int(metropolis), _ptr(info)))
    return U, dict(zip(TRAJ_KEYS, info.tolist()))


def wilson(dims, U, kappa, psi, t_bc=-1) -> np.ndarray:
    """The full Wilson operator M psi = psi - kappa D psi (Sec. 6.2: the Wilson
    fermions the trajectories run)."""
    return psi - kappa * dslash(dims, U, psi, t_bc=t_bc)


def wilson_solve(dims, U, kappa, b, tol=1e-12, maxiter=10000, t_bc=-1):
    """M x = b for a full-lattice source b through the even-odd reduction the
    Krylov solver of Sec. 6 runs on: b'_e = b_e + kappa D_eo b_o, the normal
    equations Mhat^dag Mhat x_e = Mhat^dag b'_e by CG, then x_o = b_o + kappa
    D_oe x_e.  Returns (x, converged, cg iterations)."""
    par = parity(dims)
    even = (par == 0)[:, None, None]
    b_e, b_o = np.where(even, b, 0), np.where(even, 0, b)
    bp = b_e + kappa * dslash(dims, U, b_o, out_parity=0, t_bc=t_bc)
    src = mhat(dims, U, kappa, bp, dagger=True, t_bc=t_bc)
    x_e, conv, iters, _ = cg(dims, U, kappa, src, tol=tol, maxiter=maxiter, t_bc=t_bc)
    x_o = b_o + kappa * dslash(dims, U, x_e, out_parity=1, t_bc=t_bc)
    return np.where(even, x_e, x_o), conv, iters
