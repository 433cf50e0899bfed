"""GPU parity at the benchmark's full size (32^3x64, V/2 = 1,048,576, the
launch configuration bench.py times), on sampled outputs the oracle computes
one by one, and through properties that hold at any size."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import lqcd
from tests.gpu_util import full_from_half, half, rel_err

pytestmark = pytest.mark.gpu

DIMS = (32, 32, 32, 64)
SEED, EPS, BETA, KAPPA = 3, 0.15, 5.8, 0.1570
V = int(np.prod(DIMS))
RNG = np.random.default_rng(2026)
SITES = np.sort(RNG.choice(V, 48, replace=False))


@pytest.fixture(scope="module")
def fields():
    U = lqcd.gauge_field(DIMS)
    lqcd.gauge_start(U, SEED, EPS)
    Uh = U.download()
    eta = lqcd.spinor_field(DIMS, 0)
    lqcd.eta_refresh(eta, SEED, traj=0)
    return U, Uh, eta, eta.download()


def _gen(a):
    c = np.zeros(8)
    c[a] = 1
    return orc.algebra_to_mat(c)


def test_start_configuration_sampled(fields):
    """links at sampled sites = exp(i eps sum_a h_a T_a) with the oracle's
    Philox Gaussians and power-series exponential"""
    _, Uh, _, _ = fields
    T = [_gen(a) for a in range(8)]
    for x in SITES[:16]:
        h = np.concatenate([orc.gauss2(SEED, 0, int(x), j, 0, 0) for j in range(16)])
        for mu in range(4):
            H = sum(h[mu * 8 + a] * T[a] for a in range(8))
            assert np.max(np.abs(Uh[x, mu] - orc.su3_expi(H, EPS))) < 1e-14


def test_refresh_sampled(fields):
    P = lqcd.momentum_field(DIMS)
    lqcd.momentum_refresh(P, SEED, traj=7)
    Ph = P.download()
    _, _, _, etah = fields
    par = orc.parity(DIMS)
    even_sites = np.where(par == 0)[0]
    for x in SITES[:16]:
        ref = np.concatenate([orc.gauss2(SEED, 0, int(x), j, 1, 7) for j in range(16)]).reshape(4, 8)
        assert np.max(np.abs(Ph[x] - ref)) < 1e-13
    for cb in RNG.choice(V // 2, 16, replace=False):
        x = int(even_sites[cb])
        g = np.concatenate([orc.gauss2(SEED, 0, x, j, 2, 0) for j in range(12)]) * np.sqrt(0.5)
        ref = (g[0::2] + 1j * g[1::2]).reshape(4, 3)
        assert np.max(np.abs(etah[cb] - ref)) < 1e-13


@pytest.mark.parametrize("prec,tol", [(lqcd.F64, 1e-13), (lqcd.F32, 2e-6), (lqcd.F16N, 3e-3)])
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_sampled(fields, prec, tol, dagger):
    U, Uh, eta, etah = fields
    if prec == lqcd.F64:
        Ul, inp = U, eta
    else:
        Ul = lqcd.gauge_field(DIMS, prec).copy_from(U)
        inp = lqcd.spinor_field(DIMS, 0, prec).copy_from(eta)
    out = lqcd.spinor_field(DIMS, 1, prec)
    lqcd.dslash(out, Ul, inp, dagger)
    got = out.download()
    par = orc.parity(DIMS)
    odd_sites = np.where(par == 1)[0]
    cbs = np.sort(RNG.choice(V // 2, 48, replace=False))
    # t = 0 and t = Lt - 1 slices: the antiperiodic hops
    cbs = np.concatenate([cbs, [0, 1, V // 2 - 1, V // 2 - 2]])
    ref = orc.dslash_at(DIMS, Uh, full_from_half(etah, DIMS, 0), odd_sites[cbs], dagger=dagger)
    assert rel_err(got[cbs], ref) < tol


def test_forces_sampled(fields):
    U, Uh, eta, etah = fields
    links = np.sort(RNG.choice(4 * V, 64, replace=False))
    P = lqcd.momentum_field(DIMS)
    P.upload(np.zeros((V, 4, 8)))
    lqcd.gauge_force(P, U, BETA, 1.0)
    got = -P.download().reshape(-1, 8)[links]
    ref = orc.gauge_force(DIMS, Uh, BETA, links)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.abs(ref).max()
    P.upload(np.zeros((V, 4, 8)))
    lqcd.fermion_force(P, U, eta, KAPPA, 1.0)
    got = -P.download().reshape(-1, 8)[links]
    ref = orc.fermion_force(DIMS, Uh, KAPPA, full_from_half(etah, DIMS, 0), links)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.abs(ref).max()


def test_mixed_solve_true_residual_full_size(fields):
    """the benchmark's solver configuration; the residual recomputed by the
    oracle's FP64 operator over the whole lattice"""
    U, Uh, eta, etah = fields
    Us = lqcd.gauge_field(DIMS, lqcd.F16N).copy_from(U)
    x = lqcd.spinor_field(DIMS, 0)
    rc, info = lqcd.cg_solve(x, U, eta, KAPPA, lqcd.cg_params(tol=1e-10, sloppy=lqcd.F16N, delta=0.003), U_sloppy=Us)
    assert rc == lqcd.OK and info.true_rel_res <= 1e-10
    b = full_from_half(etah, DIMS, 0)
    r = b - orc.mdagm(DIMS, Uh, KAPPA, full_from_half(x.download(), DIMS, 0))
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)


def test_reversibility_full_size():
    """one Omelyan step forward, momenta flipped, one step forward: back to the
    start (FP64 path, tight solves)"""
    U = lqcd.gauge_field(DIMS)
    lqcd.gauge_start(U, SEED, EPS)
    U0 = U.download()
    st = lqcd.HmcState(U, seed=SEED)
    params = lqcd.hmc_params(BETA, KAPPA, 1.0 / 16, 1, lqcd.OMELYAN, cg=lqcd.cg_params(tol=1e-12))
    st.refresh(params)
    _, P, _ = st.fields()
    P0 = P.download()
    st.md_step(params)
    assert np.abs(U.download() - U0).max() > 1e-3
    P.upload(-P.download())
    st.md_step(params)
    assert np.abs(U.download() - U0).max() < 1e-10
    assert np.abs(P.download() + P0).max() < 1e-9
    st.close()
