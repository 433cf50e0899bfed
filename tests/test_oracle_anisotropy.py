"""Oracle pins for the anisotropic Wilson actions (the paper's runs, Fig. 3):
gauge plaquettes of the planes with t weighted by xi0 and spatial ones by
1/xi0, the spatial hops of the Wilson operator weighted by nu / xi0.

- free field: plane waves are eigenvectors of the weighted hopping term with
  the closed form sum_mu c_mu (2 cos p_mu - 2 i gamma_mu sin p_mu);
- the dagger stays the adjoint, D^dag = gamma5 D gamma5, gauge covariance;
- configurations whose temporal (spatial) plaquettes are all 1 scale their
  action by exactly 1/xi0 (xi0) against the isotropic one;
- both forces are the finite differences of the anisotropic actions;
- the anisotropic molecular dynamics is reversible and |dH| ~ dt^2;
- (1, 1) is bitwise the isotropic oracle.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs
from tests import lattice_np as ln

XI0, NU = 1.7, 0.9


def _unit_gauge(dims):
    U = np.zeros((int(np.prod(dims)), 4, 3, 3), np.complex128)
    U[:] = np.eye(3)
    return U


def _T(a):
    c = np.zeros(8)
    c[a] = 1
    return orc.algebra_to_mat(c)


def _perturbed(U, site, mu, a, eps):
    Up = U.copy()
    Up[site, mu] = scipy.linalg.expm(1j * eps * _T(a)) @ U[site, mu]
    return Up


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (3, 1, 1, 2)])
def test_free_field_plane_wave_anisotropic(n):
    dims = (4, 4, 6, 8)
    x = ln.coords(dims)
    p = [2 * np.pi * n[mu] / dims[mu] for mu in range(3)] + [(2 * n[3] + 1) * np.pi / dims[3]]
    rng = np.random.default_rng(2)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    phase = np.exp(1j * sum(p[mu] * x[mu] for mu in range(4)))
    psi = phase[:, None, None] * u[None]
    with orc.anisotropy(XI0, NU):
        out = orc.dslash(dims, _unit_gauge(dims), psi)
    G = [orc.gamma(mu) for mu in range(4)]
    c = [NU / XI0] * 3 + [1.0]
    K = sum(c[mu] * (2 * np.cos(p[mu]) * np.eye(4) - 2j * np.sin(p[mu]) * G[mu]) for mu in range(4))
    expect = phase[:, None, None] * (K @ u)[None]
    assert np.max(np.abs(out - expect)) < 1e-13


def test_adjoint_hermiticity_covariance_anisotropic():
    dims = (4, 4, 4, 6)
    U = inputs.random_gauge(dims, 5)
    a = inputs.random_spinor(dims, 6)
    b = inputs.random_spinor(dims, 7)
    g5 = orc.gamma(4)
    Om = inputs.random_gauge_transform(dims, 8)
    with orc.anisotropy(XI0, NU):
        lhs = np.vdot(a, orc.dslash(dims, U, b))
        rhs = np.vdot(orc.dslash(dims, U, a, dagger=True), b)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)
        d1 = orc.dslash(dims, U, b, dagger=True)
        d2 = np.einsum("ab,xbc->xac", g5, orc.dslash(dims, U, np.einsum("ab,xbc->xac", g5, b)))
        assert np.max(np.abs(d1 - d2)) < 1e-13
        Up = ln.gauge_transform(U, Om, dims)
        lhs = orc.dslash(dims, Up, np.einsum("xab,xsb->xsa", Om, b))
        rhs = np.einsum("xab,xsb->xsa", Om, orc.dslash(dims, U, b))
        assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_gauge_action_plane_weights():
    """links independent of t with U_t = 1: every temporal plaquette is 1, so
    S(xi0) = S(1) / xi0; spatial links 1 and U_t independent of t: every
    spatial plaquette is 1, so S(xi0) = xi0 S(1)"""
    dims = (4, 4, 4, 6)
    V = int(np.prod(dims))
    x = ln.coords(dims)
    base = inputs.random_gauge((4, 4, 4, 1), 11, spread=0.6)  # one time slice
    U = np.zeros((V, 4, 3, 3), complex)
    idx3 = x[0] + 4 * (x[1] + 4 * x[2])
    U[:, :3] = base[idx3, :3]
    U[:, 3] = np.eye(3)
    S1 = orc.gauge_action(dims, U, 5.6)
    with orc.anisotropy(XI0, NU):
        Sx = orc.gauge_action(dims, U, 5.6)
    assert S1 > 1 and abs(Sx - S1 / XI0) < 1e-12 * S1
    U2 = np.zeros_like(U)
    U2[:] = np.eye(3)
    U2[:, 3] = base[idx3, 0]
    S1 = orc.gauge_action(dims, U2, 5.6)
    with orc.anisotropy(XI0, NU):
        Sx = orc.gauge_action(dims, U2, 5.6)
    assert S1 > 1 and abs(Sx - XI0 * S1) < 1e-12 * S1
    # the plaquette observable itself is the unweighted mean
    p_iso = orc.plaquette(dims, U2)
    with orc.anisotropy(XI0, NU):
        assert orc.plaquette(dims, U2) == p_iso


def test_forces_finite_difference_anisotropic():
    dims = (4, 2, 2, 4)
    kappa = 0.13
    U = inputs.random_gauge(dims, 8, spread=0.6)
    phi = inputs.random_spinor(dims, 9, parity=0)
    h = 1e-4
    cases = [(0, 0, 3), (1, 1, 0), (5, 2, 7), (13, 3, 1), (14, 3, 5), (6, 0, 2)]
    with orc.anisotropy(XI0, NU):
        Fg = orc.gauge_force(dims, U, 5.6)
        X, conv, _, _ = orc.cg(dims, U, kappa, phi, tol=1e-14)
        assert conv
        Ff = orc.fermion_force(dims, U, kappa, X)
        for site, mu, a in cases:
            fd = (orc.gauge_action(dims, _perturbed(U, site, mu, a, h), 5.6)
                  - orc.gauge_action(dims, _perturbed(U, site, mu, a, -h), 5.6)) / (2 * h)
            assert abs(fd - Fg[site, mu, a]) < 1e-6 * max(1, abs(Fg[site, mu, a])), (site, mu, a)
            fd = (orc.fermion_action(dims, _perturbed(U, site, mu, a, h), kappa, phi, tol=1e-14)
                  - orc.fermion_action(dims, _perturbed(U, site, mu, a, -h), kappa, phi, tol=1e-14)) / (2 * h)
            assert abs(fd - Ff[site, mu, a]) < 1e-6 * np.abs(Ff).max(), (site, mu, a, fd, Ff[site, mu, a])
    # the anisotropy changes both forces
    assert np.abs(Fg - orc.gauge_force(dims, U, 5.6)).max() > 1e-3
    assert np.abs(Ff - orc.fermion_force(dims, U, kappa, X)).max() > 1e-3


def test_anisotropic_dynamics_reversible_and_dt_squared():
    dims = (4, 4, 4, 4)
    U0 = orc.gauge_start(dims, seed=1, eps=0.3)
    P0 = orc.momentum_refresh(dims, seed=1, traj=0)
    with orc.anisotropy(XI0, NU):
        eta = orc.eta_refresh(dims, seed=1, traj=0)
        phi = orc.mhat(dims, U0, 0.14, eta, dagger=True)
        kw = dict(beta=5.6, kappa=0.14, tau=0.3, nsteps=3, integrator=orc.OMELYAN, cg_tol=1e-13)
        U1, P1, _ = orc.md_integrate(dims, U0, P0, phi, **kw)
        U2, P2, _ = orc.md_integrate(dims, U1, -P1, phi, **kw)
        assert np.abs(U1 - U0).max() > 1e-2 and np.abs(U2 - U0).max() < 1e-10 and np.abs(P2 + P0).max() < 1e-10
        dH = [orc.hmc_trajectory(dims, U0, 5.6, 0.14, 0.25, n, seed=1, traj=0, metropolis=False,
                                 cg_tol=1e-12)[1]["dH"] for n in (5, 10)]
    assert 3.5 < dH[0] / dH[1] < 4.5, dH


def test_unit_anisotropy_is_the_isotropic_oracle():
    dims = (4, 4, 4, 4)
    U = orc.gauge_start(dims, seed=2, eps=0.3)
    ref = orc.hmc_trajectory(dims, U, 5.6, 0.15, 0.3, 3, seed=2, traj=0)
    with orc.anisotropy(1.0, 1.0):
        got = orc.hmc_trajectory(dims, U, 5.6, 0.15, 0.3, 3, seed=2, traj=0)
    assert np.array_equal(ref[0], got[0]) and ref[1] == got[1]
