"""GPU parity of the anisotropic Wilson actions (gauge plaquettes of the planes
with t weighted by xi0, spatial ones by 1/xi0; spatial hops of the Wilson
operator by nu / xi0) against the oracle: the hopping term in every precision
and form, both forces, whole trajectories on the FP64 and the mixed path, and
the batched chains against the same chains alone."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs, lqcd
from tests.gpu_util import full_from_half, half, rel_err

pytestmark = pytest.mark.gpu

XI0, NU = 1.7, 0.9
A = (XI0, NU)
F16N_TOL = 3e-3  # ~6 FP16 unit roundoffs: storage, projection and output rounding (test_gpu_operators)


@pytest.fixture
def form():
    prev = lqcd.dslash_form()
    yield
    lqcd.dslash_form(prev)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 10)])
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_anisotropic(dims, dagger, form):
    Uh = inputs.random_gauge(dims, 11, spread=0.5)
    U = lqcd.gauge_field(dims, aniso=A).upload(Uh)
    Us = lqcd.gauge_field(dims, lqcd.F16N, aniso=A).copy_from(U)
    for par in (0, 1):
        s = inputs.random_spinor(dims, 12 + par, parity=par)
        with orc.anisotropy(*A):
            ref = half(orc.dslash(dims, Uh, s, dagger=dagger, out_parity=1 - par), dims, 1 - par)
        inp = lqcd.spinor_field(dims, par, aniso=A).upload(half(s, dims, par))
        out = lqcd.spinor_field(dims, 1 - par, aniso=A)
        lqcd.dslash(out, U, inp, dagger)
        assert rel_err(out.download(), ref) < 1e-13
        inp16 = lqcd.spinor_field(dims, par, lqcd.F16N, aniso=A).copy_from(inp)
        for f in (lqcd.DSLASH_GATHER, lqcd.DSLASH_PREFETCH, lqcd.DSLASH_PACKED):
            lqcd.dslash_form(f)
            o16 = lqcd.spinor_field(dims, 1 - par, lqcd.F16N, aniso=A)
            lqcd.dslash(o16, Us, inp16, dagger)
            assert rel_err(o16.download(), ref) < F16N_TOL, f
    iso = orc.dslash(dims, Uh, s, dagger=dagger, out_parity=1 - par)  # outside the context: isotropic
    assert rel_err(half(iso, dims, 1 - par), ref) > 1e-3  # the anisotropy matters


def test_forces_and_solve_anisotropic():
    dims = (4, 4, 2, 6)
    Uh = orc.gauge_start(dims, seed=5, eps=0.4)
    Ph = inputs.random_momentum(dims, 18)
    X = inputs.random_spinor(dims, 19, parity=0)
    kappa = 0.14
    with orc.anisotropy(*A):
        Fg = orc.gauge_force(dims, Uh, 5.6)
        Ff = orc.fermion_force(dims, Uh, kappa, X)
        xo, conv, _, _ = orc.cg(dims, Uh, kappa, X, tol=1e-12)
    for arith, tol in ((lqcd.F64, 1e-12), (lqcd.F32, 5e-6)):
        U = lqcd.gauge_field(dims, aniso=A).upload(Uh)
        P = lqcd.momentum_field(dims, aniso=A).upload(Ph)
        lqcd.gauge_force(P, U, 5.6, 1.0, arith=arith)
        assert rel_err(Ph - P.download(), Fg) < tol, arith
        P.upload(Ph)
        lqcd.fermion_force(P, U, lqcd.spinor_field(dims, 0, aniso=A).upload(half(X, dims, 0)), kappa, 1.0,
                           arith=arith)
        assert rel_err(Ph - P.download(), Ff) < tol, arith
    U = lqcd.gauge_field(dims, aniso=A).upload(Uh)
    b = lqcd.spinor_field(dims, 0, aniso=A).upload(half(X, dims, 0))
    for sl in (lqcd.F64, lqcd.F16N):
        x = lqcd.spinor_field(dims, 0, aniso=A)
        Us = None if sl == lqcd.F64 else lqcd.gauge_field(dims, sl, aniso=A).copy_from(U)
        rc, info = lqcd.cg_solve(x, U, b, kappa, lqcd.cg_params(tol=1e-12, sloppy=sl, delta=0.01), U_sloppy=Us)
        assert rc == lqcd.OK and rel_err(x.download(), half(xo, dims, 0)) < 1e-9


@pytest.mark.parametrize("mixed", [False, True])
def test_trajectory_anisotropic(mixed):
    """FP64 path: dH to 1e-8 and links to 1e-9 of the oracle; the mixed path
    (FP16+norm solver, FP32 forces) within the bounds of the mixed parity
    tests (1e-6 sqrt(32 V) in dH, 1e-5 in the links)"""
    dims = (4, 4, 4, 4)
    Uh = orc.gauge_start(dims, seed=1, eps=0.3)
    kw = dict(beta=5.6, kappa=0.14, tau=0.5, nsteps=5, integrator=lqcd.OMELYAN, metropolis=False)
    if mixed:
        p = lqcd.hmc_params(cg=lqcd.cg_params(tol=1e-10, sloppy=lqcd.F16N, delta=0.003), force_prec=lqcd.F32,
                            chrono=3, **kw)
        tol_dh, tol_u = 1e-6 * np.sqrt(32 * 256), 1e-5
    else:
        p = lqcd.hmc_params(cg=lqcd.cg_params(tol=1e-10), **kw)
        tol_dh, tol_u = 1e-8, 1e-9
    U = lqcd.gauge_field(dims, aniso=A).upload(Uh)
    st = lqcd.HmcState(U, seed=1)
    g = st.trajectory(p)
    st.close()
    with orc.anisotropy(*A):
        Uo, o = orc.hmc_trajectory(dims, Uh, 5.6, 0.14, 0.5, 5, integrator=orc.OMELYAN, seed=1, traj=0,
                                   cg_tol=1e-10, metropolis=False)
    assert abs(g["H0"] - o["H0"]) < 1e-10 * abs(o["H0"])
    assert abs(g["dH"] - o["dH"]) < tol_dh, (g["dH"], o["dH"])
    assert np.max(np.abs(U.download() - Uo)) < tol_u
    assert abs(g["plaq"] - o["plaq"]) < 1e-8  # the plaquette observable is the unweighted mean


def test_batched_chains_anisotropic_equal_solo():
    specs = [((4, 4, 4, 4), 1), ((6, 4, 2, 10), 2)]
    cg = lqcd.cg_params(tol=1e-10, sloppy=lqcd.F16N, delta=0.01)
    p = lqcd.hmc_params(5.7, 0.14, 0.3, 3, lqcd.OMELYAN, cg=cg, force_prec=lqcd.F32, chrono=3)
    solo = []
    for dims, seed in specs:
        U = lqcd.gauge_field(dims, aniso=A)
        lqcd.gauge_start(U, seed, 0.3)
        st = lqcd.HmcState(U, seed=seed, chain=seed)
        solo.append((st.trajectory(p), U.download()))
        st.close()
    fields, states = [], []
    for dims, seed in specs:
        U = lqcd.gauge_field(dims, aniso=A)
        lqcd.gauge_start(U, seed, 0.3)
        fields.append(U)
        states.append(lqcd.HmcState(U, seed=seed, chain=seed))
    batch = lqcd.Batch(states)
    got = batch.trajectory(p)
    for i in range(len(specs)):
        assert got[i]["dH"] == solo[i][0]["dH"] and np.array_equal(fields[i].download(), solo[i][1])
    batch.close()
    for st in states:
        st.close()
