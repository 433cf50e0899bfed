"""Oracle pins for mass preconditioning and the nested integrator.

- the ratio action's force against central finite differences of the action;
- kappa_h = kappa: W = Mhat, the ratio action is |phi_r|^2 whatever the links,
  so its force vanishes;
- the refresh reproduces S_r = |eta|^2 and S_h = |eta_h|^2;
- kappa_h -> 0 (W = 1) and one level reproduce the plain trajectory;
- the nested integrators conserve H to O(h^2): |dH| falls by ~4 when every
  level's step halves.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs
from tests import lattice_np as ln


def _T(a):
    c = np.zeros(8)
    c[a] = 1
    return orc.algebra_to_mat(c)


def _perturbed(U, site, mu, a, eps):
    Up = U.copy()
    Up[site, mu] = scipy.linalg.expm(1j * eps * _T(a)) @ U[site, mu]
    return Up


def test_ratio_force_finite_difference():
    dims = (4, 2, 2, 4)
    kappa, kappa_h = 0.13, 0.09
    U = inputs.random_gauge(dims, 18, spread=0.6)
    V = int(np.prod(dims))
    phi = inputs.random_spinor(dims, 19, parity=0)
    S, F = orc.hasenbusch_ratio(dims, U, kappa, kappa_h, phi, tol=1e-14)
    scale = np.abs(F).max()
    assert scale > 1e-3
    h = 1e-4
    tsite = [s for s in range(V) if ln.coords(dims)[3][s] == dims[3] - 1]
    par = orc.parity(dims)
    for site, mu, a in [(0, 0, 3), (1, 1, 0), (5, 2, 7), (tsite[0], 3, 1), (int(np.where(par == 1)[0][2]), 3, 6)]:
        sp, _ = orc.hasenbusch_ratio(dims, _perturbed(U, site, mu, a, h), kappa, kappa_h, phi, tol=1e-14, force=False)
        sm, _ = orc.hasenbusch_ratio(dims, _perturbed(U, site, mu, a, -h), kappa, kappa_h, phi, tol=1e-14,
                                     force=False)
        fd = (sp - sm) / (2 * h)
        assert abs(fd - F[site, mu, a]) < 1e-6 * scale, (site, mu, a, fd, F[site, mu, a])


def test_ratio_with_equal_masses_is_constant():
    dims = (4, 4, 2, 2)
    kappa = 0.12
    U = inputs.random_gauge(dims, 21, spread=0.5)
    phi = inputs.random_spinor(dims, 22, parity=0)
    S, F = orc.hasenbusch_ratio(dims, U, kappa, kappa, phi, tol=1e-14)
    assert abs(S - np.vdot(phi, phi).real) < 1e-10 * S
    assert np.abs(F).max() < 1e-9


def test_refresh_gives_gaussian_actions():
    dims = (4, 4, 2, 4)
    kappa, kappa_h = 0.135, 0.1
    U = orc.gauge_start(dims, seed=7, eps=0.4)
    eta = orc.eta_refresh(dims, seed=7, traj=3)
    eta_h = orc.eta_refresh_h(dims, seed=7, traj=3)
    assert np.abs(eta_h).max() > 0 and not np.array_equal(eta, eta_h)
    assert np.all(eta_h[orc.parity(dims) == 1] == 0)
    phi_r, phi_h = orc.hasenbusch_refresh(dims, U, kappa, kappa_h, eta, eta_h, tol=1e-14)
    S_r, _ = orc.hasenbusch_ratio(dims, U, kappa, kappa_h, phi_r, tol=1e-14, force=False)
    assert abs(S_r - np.vdot(eta, eta).real) < 1e-9 * S_r
    S_h = orc.fermion_action(dims, U, kappa_h, phi_h, tol=1e-14)
    assert abs(S_h - np.vdot(eta_h, eta_h).real) < 1e-9 * S_h


@pytest.mark.parametrize("integrator", [orc.LEAPFROG, orc.OMELYAN])
def test_trivial_preconditioning_reproduces_plain_trajectory(integrator):
    dims = (4, 4, 4, 4)
    U = orc.gauge_start(dims, seed=1, eps=0.3)
    Up, ip = orc.hmc_trajectory(dims, U, 5.6, 0.156, 0.25, 3, integrator=integrator, seed=1, traj=0)
    for kh in (0.0, 1e-200):  # kappa_h^2 underflows: W = 1
        Uh, ih = orc.hmc_trajectory_hb(dims, U, 5.6, 0.156, kh, 0.25, 3, integrator=integrator, seed=1, traj=0)
        assert abs(ih["dH"] - ip["dH"]) < 1e-9, (kh, ih["dH"], ip["dH"])
        assert np.max(np.abs(Uh - Up)) < 1e-11
        if kh:
            eta_h = orc.eta_refresh_h(dims, 1, 0)
            assert abs((ih["H0"] - ip["H0"]) - np.vdot(eta_h, eta_h).real) < 1e-8


@pytest.mark.parametrize("integrator,kappa_h,m,inner", [(orc.LEAPFROG, 0.0, 3, False), (orc.OMELYAN, 0.12, 2, False),
                                                         (orc.LEAPFROG, 0.12, 2, True)])
def test_nested_integrator_second_order(integrator, kappa_h, m, inner):
    dims = (4, 4, 4, 4)
    U = orc.gauge_start(dims, seed=3, eps=0.3)
    dh = []
    for n in (2, 4):
        _, info = orc.hmc_trajectory_hb(dims, U, 5.6, 0.15, kappa_h, 0.5, n, integrator=integrator,
                                        gauge_substeps=m, heavy_inner=inner, seed=3, traj=1, cg_tol=1e-12,
                                        metropolis=False)
        dh.append(abs(info["dH"]))
    ratio = dh[0] / dh[1]
    assert 2.5 < ratio < 6.5, (dh, ratio)
