"""The forms of the FP16+norm hopping term: every operand gathered by its
thread (0) and each thread's links prefetched into shared memory by cp.async
(1) give bitwise the same results on full and ragged last blocks, across the
z and t boundaries, for both boundary conditions, both parities, D and D^dag,
the axpy/CG epilogues and a whole mixed solve.  The packed form (2, the
default) rounds its spin projection to FP16 and its FP32 products in another
order, and agrees with them within those roundings; all match the oracle to
FP16 accuracy."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs, lqcd
from tests.gpu_util import full_from_half, half, rel_err

pytestmark = pytest.mark.gpu

# Vh = 512, 576 (whole blocks of 128), 432 and 1728 (a ragged last block)
DIMS = [(16, 16, 4, 4), (32, 8, 4, 6), (6, 6, 4, 6), (8, 6, 6, 12)]
FORMS = (lqcd.DSLASH_GATHER, lqcd.DSLASH_PREFETCH)
F16N_TOL = 3e-3  # ~6 FP16 unit roundoffs: storage, projection and output rounding (test_gpu_operators)


@pytest.fixture
def form():
    prev = lqcd.dslash_form()
    yield
    lqcd.dslash_form(prev)


def _fields(dims, t_bc, seed):
    Uh = inputs.random_gauge(dims, seed, spread=0.5)
    U = lqcd.gauge_field(dims, t_bc=t_bc).upload(Uh)
    Us = lqcd.gauge_field(dims, lqcd.F16N, t_bc=t_bc).copy_from(U)
    return Uh, U, Us


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_forms_dslash_bitwise(dims, t_bc, form):
    forms = FORMS
    Uh, U, Us = _fields(dims, t_bc, 50)
    for par in (0, 1):
        psi = inputs.random_spinor(dims, 51 + par, parity=par)
        inp = lqcd.spinor_field(dims, par, lqcd.F16N, t_bc=t_bc).copy_from(
            lqcd.spinor_field(dims, par, t_bc=t_bc).upload(half(psi, dims, par)))
        for dag in (False, True):
            outs = []
            for f in forms:
                lqcd.dslash_form(f)
                out = lqcd.spinor_field(dims, 1 - par, lqcd.F16N, t_bc=t_bc)
                lqcd.dslash(out, Us, inp, dag)
                outs.append(out.download())
            assert np.array_equal(outs[0], outs[1]), (par, dag)
            ref = orc.dslash(dims, Uh, full_from_half(inp.download(), dims, par), dagger=dag, t_bc=t_bc)
            assert rel_err(outs[1], half(ref, dims, 1 - par)) < F16N_TOL


@pytest.mark.parametrize("dims", DIMS[1:2] + DIMS[3:])
def test_forms_mhat_and_mixed_solve_bitwise(dims, form):
    forms = FORMS
    Uh, U, Us = _fields(dims, -1, 60)
    eta = inputs.random_spinor(dims, 61, parity=0)
    b = lqcd.spinor_field(dims, 0).upload(half(eta, dims, 0))
    b16 = lqcd.spinor_field(dims, 0, lqcd.F16N).copy_from(b)
    res = []
    for f in forms:
        lqcd.dslash_form(f)
        m = lqcd.spinor_field(dims, 0, lqcd.F16N)
        lqcd.mhat(m, Us, b16, 0.155, True)
        x = lqcd.spinor_field(dims, 0)
        rc, info = lqcd.cg_solve(x, U, b, 0.155, lqcd.cg_params(tol=1e-11, sloppy=lqcd.F16N, delta=0.01),
                                 U_sloppy=Us)
        assert rc == lqcd.OK
        res.append((m.download(), x.download(), info.iters, info.restarts))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1]) and res[0][2:] == res[1][2:]
    r = half(eta, dims, 0) - half(orc.mdagm(dims, Uh, 0.155, full_from_half(res[1][1], dims, 0)), dims, 0)
    assert np.linalg.norm(r) <= 1.01e-11 * np.linalg.norm(half(eta, dims, 0))


@pytest.mark.parametrize("dims", [DIMS[0], DIMS[3]])
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_packed_form_matches_prefetched(dims, t_bc, form):
    """form 2 rounds each projected component to FP16 (|error| <= 2^-11 of a
    sum of two stored values, so <= 2^-10 N_nb per real part with N_nb the
    neighbour's norm) and orders its FP32 products differently.  Through a
    link row (sum_j |u_aj| <= sqrt 3) a hop's output component moves by at
    most sqrt 3 * sqrt 2 * 2^-10 N_nb, eight hops by 8 sqrt 6 2^-10 max N_nb;
    the two stored outputs add one FP16 rounding each (2^-11 N_out).  That
    worst case holds site by site; the errors are independent roundings, so
    their rms is far smaller (about 0.5 2^-10 of the output's rms): the test
    asserts 2^-10.  Both forms match the oracle to the FP16+norm bound."""
    Uh, U, Us = _fields(dims, t_bc, 90)
    for par in (0, 1):
        psi = inputs.random_spinor(dims, 91 + par, parity=par)
        inp = lqcd.spinor_field(dims, par, lqcd.F16N, t_bc=t_bc).copy_from(
            lqcd.spinor_field(dims, par, t_bc=t_bc).upload(half(psi, dims, par)))
        ref = orc.dslash(dims, Uh, full_from_half(inp.download(), dims, par), t_bc=t_bc)
        for dag in (False, True):
            outs = []
            for f in (lqcd.DSLASH_PREFETCH, lqcd.DSLASH_PACKED):
                lqcd.dslash_form(f)
                out = lqcd.spinor_field(dims, 1 - par, lqcd.F16N, t_bc=t_bc)
                lqcd.dslash(out, Us, inp, dag)
                outs.append(out.download())
            site_norm = np.max(np.abs(outs[0]).reshape(len(outs[0]), -1), axis=1)
            in_norm = float(np.max(np.abs(inp.download())))
            diff = np.max(np.abs(outs[1] - outs[0]).reshape(len(outs[0]), -1), axis=1)
            bound = 2.0 ** -10 * site_norm + 8 * np.sqrt(6) * 2.0 ** -10 * in_norm + 1e-6 * in_norm
            assert np.all(diff <= bound), (par, dag, float(np.max(diff / bound)))
            rms = np.sqrt(np.mean(np.abs(outs[1] - outs[0]) ** 2) / np.mean(np.abs(outs[0]) ** 2))
            assert rms <= 2.0 ** -10, (par, dag, rms)
            if not dag:
                assert rel_err(outs[1], half(ref, dims, 1 - par)) < F16N_TOL


def test_packed_form_mixed_solve_and_batch(form):
    """a whole mixed solve in form 2 reaches the FP64 tolerance, and the
    batched engine (which follows the form) equals the single solve bitwise"""
    dims = DIMS[3]
    Uh, U, Us = _fields(dims, -1, 95)
    eta = inputs.random_spinor(dims, 96, parity=0)
    b = lqcd.spinor_field(dims, 0).upload(half(eta, dims, 0))
    lqcd.dslash_form(lqcd.DSLASH_PACKED)
    prm = lqcd.cg_params(tol=1e-11, sloppy=lqcd.F16N, delta=0.01)
    x = lqcd.spinor_field(dims, 0)
    rc, info = lqcd.cg_solve(x, U, b, 0.155, prm, U_sloppy=Us)
    assert rc == lqcd.OK
    r = half(eta, dims, 0) - half(orc.mdagm(dims, Uh, 0.155, full_from_half(x.download(), dims, 0)), dims, 0)
    assert np.linalg.norm(r) <= 1.01e-11 * np.linalg.norm(half(eta, dims, 0))
    xb = lqcd.spinor_field(dims, 0)
    rc, infos = lqcd.cg_solve_batch([xb], [U], [Us], [b], [0.155], prm)
    assert rc == lqcd.OK and infos[0].iters == info.iters
    assert np.array_equal(xb.download(), x.download())
