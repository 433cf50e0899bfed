"""Oracle pins for the plaquette, the gauge action and the two forces.

- unit gauge -> plaquette 1; gauge invariance; an abelian constant-field
  configuration with a closed-form plaquette;
- forces f_a = d/de S(exp(i e T_a) U_mu(x)) at e = 0 against central finite
  differences of the actions (scipy expm builds the perturbation);
- force covariance under gauge transformations.
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


def test_plaquette_unit_gauge_and_invariance():
    dims = (4, 4, 4, 6)
    V = int(np.prod(dims))
    U1 = np.zeros((V, 4, 3, 3), complex)
    U1[:] = np.eye(3)
    assert orc.plaquette(dims, U1) == 1.0
    assert orc.gauge_action(dims, U1, 5.6) == 0.0
    U = inputs.random_gauge(dims, 3, spread=0.4)
    Om = inputs.random_gauge_transform(dims, 4)
    p = orc.plaquette(dims, U)
    assert abs(orc.plaquette(dims, ln.gauge_transform(U, Om, dims)) - p) < 1e-14
    S = orc.gauge_action(dims, U, 5.6)
    assert abs(S - 5.6 * 6 * V * (1 - p)) < 1e-9 * S


def test_plaquette_abelian_closed_form():
    """U_y(x) = diag(e^{i th x}, e^{-i th x}, 1), all other links 1, with
    th = 2 pi k / Lx: every xy plaquette is diag(e^{i th}, e^{-i th}, 1) (up to
    orientation), the other five planes are 1, so
    <P> = (5 + (2 cos th + 1) / 3) / 6."""
    dims = (6, 4, 4, 4)
    V = int(np.prod(dims))
    x = ln.coords(dims)[0]
    for k in (1, 2):
        th = 2 * np.pi * k / dims[0]
        U = np.zeros((V, 4, 3, 3), complex)
        U[:] = np.eye(3)
        U[:, 1, 0, 0] = np.exp(1j * th * x)
        U[:, 1, 1, 1] = np.exp(-1j * th * x)
        expect = (5 + (2 * np.cos(th) + 1) / 3) / 6
        assert abs(orc.plaquette(dims, U) - expect) < 1e-13


def _perturbed(U, site, mu, a, eps):
    Up = U.copy()
    Up[site, mu] = scipy.linalg.expm(1j * eps * _T(a)) @ U[site, mu]
    return Up


def test_gauge_force_finite_difference():
    dims = (4, 4, 4, 4)
    beta = 5.6
    U = orc.gauge_start(dims, seed=1, eps=0.3)
    F = orc.gauge_force(dims, U, beta)
    rng = np.random.default_rng(0)
    h = 1e-4
    for _ in range(12):
        site, mu, a = int(rng.integers(256)), int(rng.integers(4)), int(rng.integers(8))
        sp = orc.gauge_action(dims, _perturbed(U, site, mu, a, h), beta)
        sm = orc.gauge_action(dims, _perturbed(U, site, mu, a, -h), beta)
        fd = (sp - sm) / (2 * h)
        assert abs(fd - F[site, mu, a]) < 1e-6 * max(1, abs(F[site, mu, a])), (site, mu, a)
    links = np.array([0, 7, 100, 1023])
    assert np.array_equal(orc.gauge_force(dims, U, beta, links), F.reshape(-1, 8)[links])


def test_fermion_force_finite_difference():
    dims = (4, 2, 2, 4)  # small enough for tight CG solves at every perturbation
    kappa = 0.13
    U = inputs.random_gauge(dims, 8, spread=0.6)
    V = int(np.prod(dims))
    phi = inputs.random_spinor(dims, 9, parity=0)
    X, conv, _, _ = orc.cg(dims, U, kappa, phi, tol=1e-14)
    assert conv
    F = orc.fermion_force(dims, U, kappa, X)
    scale = np.abs(F).max()
    h = 1e-4
    par = orc.parity(dims)
    # every direction, both parities, and the links crossing the t boundary
    tsite = [s for s in range(V) if ln.coords(dims)[3][s] == dims[3] - 1]
    cases = [(0, 0, 3), (1, 1, 0), (5, 2, 7), (tsite[0], 3, 1), (tsite[1], 3, 5), (int(np.where(par == 1)[0][3]), 0, 2)]
    for site, mu, a in cases:
        sp = orc.fermion_action(dims, _perturbed(U, site, mu, a, h), kappa, phi, tol=1e-14)
        sm = orc.fermion_action(dims, _perturbed(U, site, mu, a, -h), kappa, phi, tol=1e-14)
        fd = (sp - sm) / (2 * h)
        assert abs(fd - F[site, mu, a]) < 1e-6 * scale, (site, mu, a, fd, F[site, mu, a])
    links = np.array([3, 17, 60, 255])
    assert np.allclose(orc.fermion_force(dims, U, kappa, X, links), F.reshape(-1, 8)[links], atol=1e-15)


@pytest.mark.parametrize("which", ["gauge", "fermion"])
def test_force_covariance(which):
    """F[U^Om]_mu(x) = Om(x) F[U]_mu(x) Om(x)^dag (as matrices sum_a f_a T_a)."""
    dims = (4, 4, 2, 4)
    U = inputs.random_gauge(dims, 40, spread=0.5)
    Om = inputs.random_gauge_transform(dims, 41)
    Up = ln.gauge_transform(U, Om, dims)
    if which == "gauge":
        F, Fp = orc.gauge_force(dims, U, 5.6), orc.gauge_force(dims, Up, 5.6)
    else:
        X = inputs.random_spinor(dims, 42, parity=0)
        Xp = np.einsum("xab,xsb->xsa", Om, X)
        F, Fp = orc.fermion_force(dims, U, 0.14, X), orc.fermion_force(dims, Up, 0.14, Xp)
    T = np.array([_T(a) for a in range(8)])
    M = np.einsum("xma,aij->xmij", F, T)
    Mp = np.einsum("xma,aij->xmij", Fp, T)
    rot = np.einsum("xab,xmbc,xdc->xmad", Om, M, Om.conj())
    assert np.max(np.abs(Mp - rot)) < 1e-12 * np.abs(M).max()
