"""The forms of the FP16+norm hopping term: every operand gathered by its
thread (0) and each thread's links prefetched into shared memory by cp.async
(1) give bitwise the same results on full and ragged last blocks, across the
z and t boundaries, for both boundary conditions, both parities, D and D^dag,
the axpy/CG epilogues and a whole mixed solve.  The packed FP32x2 form (2,
the default) rounds in another order and agrees with them to one FP16 step;
all match the oracle to FP16 accuracy."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs, lqcd
from tests.gpu_util import full_from_half, half, rel_err

pytestmark = pytest.mark.gpu

# Vh = 512, 576 (whole blocks of 128), 432 and 1728 (a ragged last block)
DIMS = [(16, 16, 4, 4), (32, 8, 4, 6), (6, 6, 4, 6), (8, 6, 6, 12)]
FORMS = (lqcd.DSLASH_GATHER, lqcd.DSLASH_PREFETCH)
F16N_TOL = 3e-3  # FP16+norm storage rounding, derived in the design doc section 7a


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
    """form 2 (packed FP32x2 arithmetic) rounds its products in another order:
    its FP32 results agree with form 1's to FP32 rounding, so the stored FP16
    values differ by at most one FP16 step of the site norm (2^-10 relative);
    both match the oracle to the FP16+norm bound"""
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
            diff = np.max(np.abs(outs[1] - outs[0]).reshape(len(outs[0]), -1), axis=1)
            assert np.all(diff <= 2.0 ** -10 * site_norm + 1e-30), (par, dag, float(np.max(diff / site_norm)))
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
