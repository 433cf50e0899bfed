"""Oracle pins for the Wilson hopping term D, the even-odd operator Mhat and the CG.

- free field: plane waves are eigenvectors with the momentum-space closed form
  sum_mu (2 cos p_mu - 2 i gamma_mu sin p_mu), p_t = (2n+1) pi / L_t for
  antiperiodic fermions;
- <chi, D psi> = <D^dag chi, psi> (the oracle's dagger is the adjoint);
- gauge covariance D[U^Om] (Om psi) = Om D[U] psi;
- Mhat is the Schur complement of M = 1 - kappa D on the even sites and
  det M = det Mhat (dense linear algebra on a small lattice);
- CG solutions agree with numpy.linalg.solve and meet the true-residual bound;
- phi = Mhat^dag eta gives phi^dag (Mhat^dag Mhat)^-1 phi = eta^dag eta.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs
from tests import lattice_np as ln


def _unit_gauge(dims):
    V = int(np.prod(dims))
    U = np.zeros((V, 4, 3, 3), np.complex128)
    U[:] = np.eye(3)
    return U


@pytest.mark.parametrize("t_bc", [-1, 1])
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (3, 1, 1, 2)])
def test_free_field_plane_wave(t_bc, n):
    dims = (4, 4, 6, 8)
    x = ln.coords(dims)
    p = [2 * np.pi * n[mu] / dims[mu] for mu in range(3)]
    p.append(((2 * n[3] + 1) if t_bc == -1 else 2 * n[3]) * np.pi / dims[3])
    rng = np.random.default_rng(1)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    phase = np.exp(1j * sum(p[mu] * x[mu] for mu in range(4)))
    psi = phase[:, None, None] * u[None]
    out = orc.dslash(dims, _unit_gauge(dims), psi, t_bc=t_bc)
    G = [orc.gamma(mu) for mu in range(4)]
    K = sum(2 * np.cos(p[mu]) * np.eye(4) - 2j * np.sin(p[mu]) * G[mu] for mu in range(4))
    expect = phase[:, None, None] * (K @ u)[None]
    assert np.max(np.abs(out - expect)) < 1e-13


def test_dagger_is_adjoint():
    dims = (4, 4, 4, 6)
    U = inputs.random_gauge(dims, 5)
    a = inputs.random_spinor(dims, 6)
    b = inputs.random_spinor(dims, 7)
    lhs = np.vdot(a, orc.dslash(dims, U, b))
    rhs = np.vdot(orc.dslash(dims, U, a, dagger=True), b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # and D^dag = gamma5 D gamma5 (gamma5 hermiticity)
    g5 = orc.gamma(4)
    lhs = orc.dslash(dims, U, b, dagger=True)
    rhs = np.einsum("ab,xbc->xac", g5, orc.dslash(dims, U, np.einsum("ab,xbc->xac", g5, b)))
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_gauge_covariance():
    dims = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, 11)
    Om = inputs.random_gauge_transform(dims, 12)
    psi = inputs.random_spinor(dims, 13)
    Up = ln.gauge_transform(U, Om, dims)
    lhs = orc.dslash(dims, Up, np.einsum("xab,xsb->xsa", Om, psi))
    rhs = np.einsum("xab,xsb->xsa", Om, orc.dslash(dims, U, psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_parity_structure_and_site_evaluation():
    dims = (4, 2, 4, 6)
    U = inputs.random_gauge(dims, 1)
    par = orc.parity(dims)
    psi_e = inputs.random_spinor(dims, 2, parity=0)
    out = orc.dslash(dims, U, psi_e)
    assert np.all(out[par == 0] == 0)  # D only couples even <-> odd
    out_o = orc.dslash(dims, U, psi_e, out_parity=1)
    assert np.array_equal(out_o, out)
    sites = np.array([0, 5, 17, 40, 191])
    at = orc.dslash_at(dims, U, psi_e, sites)
    assert np.array_equal(at, out[sites])
    atd = orc.dslash_at(dims, U, psi_e, sites, dagger=True)
    assert np.max(np.abs(atd - orc.dslash(dims, U, psi_e, dagger=True)[sites])) < 1e-14


def _dense_D(dims, U, dagger=False):
    V = int(np.prod(dims))
    return ln.dense_operator(lambda v: orc.dslash(dims, U, v, dagger=dagger), V * 12, (V, 4, 3))


def test_mhat_is_schur_complement_and_det():
    dims = (2, 2, 2, 4)
    kappa = 0.13
    U = inputs.random_gauge(dims, 21)
    V = int(np.prod(dims))
    D = _dense_D(dims, U)
    Dd = _dense_D(dims, U, dagger=True)
    assert np.allclose(Dd, D.conj().T, atol=1e-14)
    par = np.repeat(orc.parity(dims), 12)
    e, o = np.where(par == 0)[0], np.where(par == 1)[0]
    M = np.eye(V * 12) - kappa * D
    schur = M[np.ix_(e, e)] - M[np.ix_(e, o)] @ np.linalg.solve(M[np.ix_(o, o)], M[np.ix_(o, e)])
    Mh = ln.dense_operator(lambda v: orc.mhat(dims, U, kappa, v), V * 12, (V, 4, 3))[np.ix_(e, e)]
    assert np.max(np.abs(Mh - schur)) < 1e-14
    Mhd = ln.dense_operator(lambda v: orc.mhat(dims, U, kappa, v, dagger=True), V * 12, (V, 4, 3))[np.ix_(e, e)]
    assert np.max(np.abs(Mhd - Mh.conj().T)) < 1e-14
    s1, l1 = np.linalg.slogdet(M)
    s2, l2 = np.linalg.slogdet(Mh)
    assert abs(l1 - l2) < 1e-11 and abs(s1 - s2) < 1e-11


def test_cg_matches_dense_solve():
    dims = (2, 2, 2, 4)
    kappa = 0.156
    U = ln_gauge = inputs.random_gauge(dims, 31, spread=0.5)
    V = int(np.prod(dims))
    par = np.repeat(orc.parity(dims), 12)
    e = np.where(par == 0)[0]
    b = inputs.random_spinor(dims, 32, parity=0)
    x, conv, iters, rel = orc.cg(dims, U, kappa, b, tol=1e-12)
    assert conv and rel <= 1e-12 and iters > 0
    A = ln.dense_operator(lambda v: orc.mdagm(dims, ln_gauge, kappa, v), V * 12, (V, 4, 3))[np.ix_(e, e)]
    xd = np.linalg.solve(A, b.reshape(-1)[e])
    assert np.linalg.norm(x.reshape(-1)[e] - xd) < 1e-9 * np.linalg.norm(xd)
    # not converged within maxiter -> reported
    _, conv2, it2, rel2 = orc.cg(dims, U, kappa, b, tol=1e-12, maxiter=2)
    assert not conv2 and it2 == 2 and rel2 > 1e-12


def test_cg_true_residual_and_eta_identity():
    dims = (4, 4, 4, 4)
    kappa = 0.156
    U = orc.gauge_start(dims, seed=1, eps=0.3)
    eta = orc.eta_refresh(dims, seed=1, traj=0)
    phi = orc.mhat(dims, U, kappa, eta, dagger=True)
    x, conv, iters, rel = orc.cg(dims, U, kappa, phi, tol=1e-10)
    assert conv and rel <= 1e-10
    r = phi - orc.mdagm(dims, U, kappa, x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(phi)
    S = orc.fermion_action(dims, U, kappa, phi, tol=1e-13)
    assert abs(S - np.vdot(eta, eta).real) < 1e-9 * S
    # zero source
    x0, conv0, it0, rel0 = orc.cg(dims, U, kappa, np.zeros_like(phi))
    assert conv0 and it0 == 0 and np.all(x0 == 0)
