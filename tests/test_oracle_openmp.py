"""The OpenMP build of the oracle (the same source with -fopenmp: the loops
over sites with disjoint outputs split across threads, every sum kept serial
in site order) gives bitwise the results of the serial build: hopping term,
forces, link update, reunitarization, refresh and whole trajectories."""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs


@pytest.fixture
def both():
    os.environ.setdefault("OMP_NUM_THREADS", str(max(2, os.cpu_count() or 2)))
    prev = orc.use_openmp(False)
    yield
    orc.use_openmp(prev == "openmp")


def _run(fn, omp):
    orc.use_openmp(omp)
    return fn()


def test_openmp_build_uses_threads(both):
    orc.use_openmp(True)
    assert orc.num_threads() >= 2
    orc.use_openmp(False)
    assert orc.num_threads() == 1


def test_openmp_operators_bitwise(both):
    dims = (6, 4, 2, 10)
    U = inputs.random_gauge(dims, 80)
    psi = inputs.random_spinor(dims, 81, parity=0)
    P = inputs.random_momentum(dims, 82)
    for fn in (lambda: orc.dslash(dims, U, psi, dagger=True, out_parity=1),
               lambda: orc.mdagm(dims, U, 0.15, psi),
               lambda: orc.gauge_force(dims, U, 5.7),
               lambda: orc.fermion_force(dims, U, 0.15, psi),
               lambda: orc.link_update(dims, U, P, 0.07),
               lambda: orc.reunitarize(dims, U * 1.001)[0],
               lambda: orc.gauge_start(dims, 5, 0.3),
               lambda: orc.momentum_refresh(dims, 5, 2),
               lambda: orc.eta_refresh(dims, 5, 2),
               lambda: orc.cg(dims, U, 0.15, psi, tol=1e-10)[0]):
        a, b = _run(fn, False), _run(fn, True)
        assert np.array_equal(a, b)


def test_openmp_trajectories_bitwise(both):
    dims = (4, 4, 4, 4)
    U = orc.gauge_start(dims, seed=1, eps=0.3)
    for integ in (orc.LEAPFROG, orc.OMELYAN):
        fn = lambda: orc.hmc_trajectory(dims, U, 5.6, 0.156, 0.5, 6, integrator=integ, seed=1, traj=0)
        (Ua, ia), (Ub, ib) = _run(fn, False), _run(fn, True)
        assert np.array_equal(Ua, Ub) and ia == ib
    fn = lambda: orc.hmc_trajectory_hb(dims, U, 5.6, 0.156, 0.12, 0.5, 4, integrator=orc.OMELYAN,
                                       gauge_substeps=2, seed=1, traj=0)
    (Ua, ia), (Ub, ib) = _run(fn, False), _run(fn, True)
    assert np.array_equal(Ua, Ub) and ia == ib
