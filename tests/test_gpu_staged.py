"""The three forms of the FP16+norm hopping term -- gathered operands (0),
the +-t operands staged in shared memory by bulk asynchronous copies (1), and
each thread's links prefetched into shared memory by cp.async (2, the
default) -- give bitwise the same results, on lattices whose z-t slabs hold
whole blocks and on lattices with a ragged last block, across the z and t
boundaries, for both boundary conditions, both parities, D and D^dag, the
axpy/CG epilogues and a whole mixed solve; and they match the oracle to FP16
accuracy."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs, lqcd
from tests.gpu_util import full_from_half, half, rel_err

pytestmark = pytest.mark.gpu

STAGED_DIMS = [(16, 16, 4, 4), (32, 8, 4, 6), (16, 16, 2, 6)]
# Vh = 432 and 1728: the last block of 128 sites is ragged (form 1 falls back to 0)
RAGGED_DIMS = [(6, 6, 4, 6), (8, 6, 6, 12)]
FORMS = (lqcd.DSLASH_GATHER, lqcd.DSLASH_STAGED, lqcd.DSLASH_PREFETCH)


@pytest.fixture
def staging():
    prev = lqcd.dslash_staging()
    yield
    lqcd.dslash_staging(prev)


def _fields(dims, t_bc, seed):
    Uh = inputs.random_gauge(dims, seed, spread=0.5)
    U = lqcd.gauge_field(dims, t_bc=t_bc).upload(Uh)
    Us = lqcd.gauge_field(dims, lqcd.F16N, t_bc=t_bc).copy_from(U)
    return Uh, U, Us


@pytest.mark.parametrize("dims", STAGED_DIMS + RAGGED_DIMS)
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_staged_dslash_bitwise(dims, t_bc, staging):
    Uh, U, Us = _fields(dims, t_bc, 50)
    for par in (0, 1):
        psi = inputs.random_spinor(dims, 51 + par, parity=par)
        inp = lqcd.spinor_field(dims, par, lqcd.F16N, t_bc=t_bc).copy_from(
            lqcd.spinor_field(dims, par, t_bc=t_bc).upload(half(psi, dims, par)))
        for dag in (False, True):
            outs = []
            for form in FORMS:
                lqcd.dslash_staging(form)
                out = lqcd.spinor_field(dims, 1 - par, lqcd.F16N, t_bc=t_bc)
                lqcd.dslash(out, Us, inp, dag)
                outs.append(out.download())
            assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2]), (par, dag)
            ref = orc.dslash(dims, Uh, full_from_half(inp.download(), dims, par), dagger=dag, t_bc=t_bc)
            assert rel_err(outs[1], half(ref, dims, 1 - par)) < 3e-3
    lqcd.dslash_check()


@pytest.mark.parametrize("dims", STAGED_DIMS[:2] + RAGGED_DIMS[1:])
def test_staged_mhat_and_mixed_solve_bitwise(dims, staging):
    Uh, U, Us = _fields(dims, -1, 60)
    eta = inputs.random_spinor(dims, 61, parity=0)
    b = lqcd.spinor_field(dims, 0).upload(half(eta, dims, 0))
    b16 = lqcd.spinor_field(dims, 0, lqcd.F16N).copy_from(b)
    res = []
    for form in FORMS:
        lqcd.dslash_staging(form)
        m = lqcd.spinor_field(dims, 0, lqcd.F16N)
        lqcd.mhat(m, Us, b16, 0.155, True)
        x = lqcd.spinor_field(dims, 0)
        rc, info = lqcd.cg_solve(x, U, b, 0.155, lqcd.cg_params(tol=1e-11, sloppy=lqcd.F16N, delta=0.01),
                                 U_sloppy=Us)
        assert rc == lqcd.OK
        res.append((m.download(), x.download(), info.iters, info.restarts))
    for k in (1, 2):
        assert np.array_equal(res[0][0], res[k][0])
        assert np.array_equal(res[0][1], res[k][1]) and res[0][2:] == res[k][2:]
    r = half(eta, dims, 0) - half(orc.mdagm(dims, Uh, 0.155, full_from_half(res[1][1], dims, 0)), dims, 0)
    assert np.linalg.norm(r) <= 1.01e-11 * np.linalg.norm(half(eta, dims, 0))


def test_staging_switch_and_unfit_lattices(staging):
    assert lqcd.dslash_staging() == lqcd.DSLASH_PREFETCH  # the default
    assert lqcd.dslash_staging(lqcd.DSLASH_STAGED) == lqcd.DSLASH_PREFETCH
    assert lqcd.dslash_staging() == lqcd.DSLASH_STAGED
    assert lqcd.dslash_staging(False) == lqcd.DSLASH_STAGED and lqcd.dslash_staging() == lqcd.DSLASH_GATHER
    with pytest.raises(ValueError):
        lqcd.dslash_staging(3)
    # Lx/2 * Ly = 32: form 1 falls back to the gathered kernels
    lqcd.dslash_staging(lqcd.DSLASH_STAGED)
    dims = (8, 8, 4, 4)
    Uh, U, Us = _fields(dims, -1, 70)
    psi = inputs.random_spinor(dims, 71, parity=0)
    inp = lqcd.spinor_field(dims, 0, lqcd.F16N).copy_from(lqcd.spinor_field(dims, 0).upload(half(psi, dims, 0)))
    out = lqcd.spinor_field(dims, 1, lqcd.F16N)
    lqcd.dslash(out, Us, inp)
    ref = orc.dslash(dims, Uh, full_from_half(inp.download(), dims, 0))
    assert rel_err(out.download(), half(ref, dims, 1)) < 3e-3
    lqcd.dslash_check()
