"""Oracle pins for the molecular dynamics and the full trajectory.

- reversibility: forward, flip P, forward returns (U0, -P0);
- |dH| ~ dt^2 for leapfrog and Omelyan 2MN, Omelyan far smaller;
- link update preserves SU(3); H0's pseudofermion part is eta^dag eta;
- Metropolis decision follows u < exp(-dH) and reject restores U;
- Creutz equality <exp(-dH)> = 1 in equilibrium on a 2^4 lattice.
"""
import numpy as np
import pytest

from oracle import oracle as orc

DIMS = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def start():
    return orc.gauge_start(DIMS, seed=1, eps=0.3)


@pytest.mark.parametrize("integrator", [orc.LEAPFROG, orc.OMELYAN])
def test_reversibility(start, integrator):
    U0 = start
    P0 = orc.momentum_refresh(DIMS, seed=1, traj=0)
    eta = orc.eta_refresh(DIMS, seed=1, traj=0)
    phi = orc.mhat(DIMS, U0, 0.156, eta, dagger=True)
    kw = dict(beta=5.6, kappa=0.156, tau=0.3, nsteps=3, integrator=integrator, cg_tol=1e-13)
    U1, P1, st = orc.md_integrate(DIMS, U0, P0, phi, **kw)
    assert st[2] == 0 and np.abs(U1 - U0).max() > 1e-2
    U2, P2, _ = orc.md_integrate(DIMS, U1, -P1, phi, **kw)
    assert np.abs(U2 - U0).max() < 1e-10
    assert np.abs(P2 + P0).max() < 1e-10


@pytest.mark.parametrize("integrator,n_flavors", [(orc.LEAPFROG, 2), (orc.OMELYAN, 2), (orc.LEAPFROG, 0)])
def test_dH_scales_as_dt_squared(start, integrator, n_flavors):
    dH = []
    for n in (5, 10):
        _, info = orc.hmc_trajectory(DIMS, start, 5.6, 0.156, 0.25, n, integrator=integrator, n_flavors=n_flavors,
                                     seed=1, traj=0, metropolis=False, cg_tol=1e-12)
        dH.append(info["dH"])
    ratio = dH[0] / dH[1]
    assert 3.5 < ratio < 4.5, dH


def test_omelyan_beats_leapfrog(start):
    kw = dict(seed=1, traj=0, metropolis=False, cg_tol=1e-12)
    _, lf = orc.hmc_trajectory(DIMS, start, 5.6, 0.156, 0.25, 5, integrator=orc.LEAPFROG, **kw)
    _, om = orc.hmc_trajectory(DIMS, start, 5.6, 0.156, 0.25, 5, integrator=orc.OMELYAN, **kw)
    assert abs(om["dH"]) < abs(lf["dH"]) / 5


def test_link_update_keeps_su3(start):
    P = orc.momentum_refresh(DIMS, seed=1, traj=3)
    U = orc.link_update(DIMS, start, P, 0.1)
    dev = np.abs(np.einsum("xmab,xmcb->xmac", U, U.conj()) - np.eye(3)).max()
    assert dev < 1e-14 and np.abs(np.linalg.det(U) - 1).max() < 1e-14
    U2, d = orc.reunitarize(DIMS, U)
    assert d == pytest.approx(dev, abs=1e-16) and np.abs(U2 - U).max() < 1e-14


def test_trajectory_h0_and_metropolis(start):
    U1, info = orc.hmc_trajectory(DIMS, start, 5.6, 0.156, 1.0, 10, seed=1, traj=0)
    P = orc.momentum_refresh(DIMS, seed=1, traj=0)
    eta = orc.eta_refresh(DIMS, seed=1, traj=0)
    H0 = orc.kinetic(DIMS, P) + orc.gauge_action(DIMS, start, 5.6) + np.vdot(eta, eta).real
    assert abs(info["H0"] - H0) < 1e-9 * H0
    assert info["u"] == orc.uniform2(1, 0, 0, 0, 3, 0)[0]
    assert bool(info["accepted"]) == (info["u"] < np.exp(-info["dH"]))
    assert info["n_solves"] == 12 and info["cg_failures"] == 0
    if not info["accepted"]:
        U_r, _ = orc.reunitarize(DIMS, start)
        assert np.array_equal(U1, U_r)
    # an accepted trajectory: small step size at the same start
    U2, info2 = orc.hmc_trajectory(DIMS, start, 5.6, 0.156, 0.2, 10, integrator=orc.OMELYAN, seed=1, traj=0)
    assert info2["accepted"] == 1.0 and not np.allclose(U2, start)


def test_creutz_equality_small_lattice():
    """<exp(-dH)> = 1 over an equilibrium ensemble (area preservation +
    reversibility).  2^4 lattice, beta 5.6, kappa 0.156, 300 thermalisation and
    600 measured trajectories."""
    dims = (2, 2, 2, 2)
    U = orc.gauge_start(dims, seed=5, eps=0.3)
    vals = []
    for traj in range(900):
        U, info = orc.hmc_trajectory(dims, U, 5.6, 0.156, 0.5, 5, integrator=orc.OMELYAN, seed=5, traj=traj,
                                     cg_tol=1e-10)
        if traj >= 300:
            vals.append(np.exp(-info["dH"]))
    vals = np.array(vals)
    mean, err = vals.mean(), vals.std() / np.sqrt(len(vals))
    assert abs(mean - 1) < 3 * err + 1e-3, (mean, err)
