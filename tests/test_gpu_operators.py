"""GPU parity: even-odd dslash (every storage precision), Mhat, CG (FP64 and
reliable-update mixed), gauge and fermion forces, against the oracle."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs, lqcd
from tests.gpu_util import PARITY_DIMS, full_from_half, half, rel_err, upload_gauge, upload_half

pytestmark = pytest.mark.gpu

# max|a - b| / max|b| of the low-precision hop against FP64.  Each output
# real is a sum of 96 link x spinor products; each factor carries a storage
# rounding of relative size u (FP16 2^-11, BF16 2^-8, FP32 2^-24; row 2 of a
# 12-real link, rebuilt from rows 0 and 1, up to ~3u), the packed FP16 form
# rounds each projected component once more (u), and the output is rounded
# to storage (u of its site norm).  As a random walk of independent
# roundings the expected maximum over a test lattice is ~3u of max|out|; the
# bounds sit at ~6u (FP16 3e-3, BF16 2.5e-2).  FP32 adds its 96-term
# arithmetic (~sqrt(96) 2^-24 typical): 2e-6.  A wrong sign, a transposed
# operand or a dropped hop moves the output by O(max|out|).
LOWPREC_TOL = {lqcd.F32: 2e-6, lqcd.F16N: 3e-3, lqcd.BF16: 2.5e-2}


@pytest.mark.parametrize("dims", PARITY_DIMS)
@pytest.mark.parametrize("in_par", [0, 1])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_dslash_fp64_matches_oracle(dims, in_par, dagger, t_bc):
    Uh = inputs.random_gauge(dims, 11)
    s = inputs.random_spinor(dims, 12, parity=in_par)
    ref = orc.dslash(dims, Uh, s, dagger=dagger, out_parity=1 - in_par, t_bc=t_bc)
    U = lqcd.gauge_field(dims, t_bc=t_bc).upload(Uh)
    inp = lqcd.spinor_field(dims, in_par, t_bc=t_bc).upload(half(s, dims, in_par))
    out = lqcd.spinor_field(dims, 1 - in_par, t_bc=t_bc)
    lqcd.dslash(out, U, inp, dagger)
    assert rel_err(out.download(), half(ref, dims, 1 - in_par)) < 1e-13


@pytest.mark.parametrize("prec", [lqcd.F32, lqcd.F16N, lqcd.BF16])
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_low_precision(prec, dagger):
    dims = (8, 6, 6, 12)
    Uh = orc.gauge_start(dims, seed=3, eps=0.5)
    s = inputs.random_spinor(dims, 13, parity=0)
    ref = half(orc.dslash(dims, Uh, s, dagger=dagger, out_parity=1), dims, 1)
    U, Us = upload_gauge(Uh, dims, prec)
    inp = upload_half(s, dims, 0, prec)
    out = lqcd.spinor_field(dims, 1, prec)
    lqcd.dslash(out, Us, inp, dagger)
    assert rel_err(out.download(), ref) < LOWPREC_TOL[prec]


@pytest.mark.parametrize("dagger", [False, True])
def test_mhat_matches_oracle(dagger):
    dims = (6, 6, 10, 12)
    kappa = 0.1575
    Uh = orc.gauge_start(dims, seed=2, eps=0.2)
    s = inputs.random_spinor(dims, 14, parity=0)
    ref = half(orc.mhat(dims, Uh, kappa, s, dagger=dagger), dims, 0)
    U = lqcd.gauge_field(dims).upload(Uh)
    inp = upload_half(s, dims, 0)
    out = lqcd.spinor_field(dims, 0)
    lqcd.mhat(out, U, inp, kappa, dagger)
    assert rel_err(out.download(), ref) < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 6, 10, 12)])
def test_cg_fp64_matches_oracle(dims):
    kappa = 0.156
    Uh = orc.gauge_start(dims, seed=1, eps=0.3)
    b = inputs.random_spinor(dims, 15, parity=0)
    xr, conv, it_r, rel_r = orc.cg(dims, Uh, kappa, b, tol=1e-12)
    assert conv
    U = lqcd.gauge_field(dims).upload(Uh)
    bf = upload_half(b, dims, 0)
    x = lqcd.spinor_field(dims, 0)
    rc, info = lqcd.cg_solve(x, U, bf, kappa, lqcd.cg_params(tol=1e-12))
    assert rc == lqcd.OK and info.true_rel_res <= 1e-12
    assert abs(info.iters - it_r) <= 2, (info.iters, it_r)
    assert rel_err(x.download(), half(xr, dims, 0)) < 1e-9
    # independent residual check with the oracle's operator
    xf = full_from_half(x.download(), dims, 0)
    r = b - orc.mdagm(dims, Uh, kappa, xf)
    assert np.linalg.norm(r) <= 1.01e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("sloppy", [lqcd.F32, lqcd.F16N, lqcd.BF16])
def test_cg_mixed_reaches_fp64_tolerance(sloppy):
    dims = (6, 6, 10, 12)
    kappa = 0.156
    Uh = orc.gauge_start(dims, seed=1, eps=0.3)
    b = inputs.random_spinor(dims, 16, parity=0)
    xr, conv, _, _ = orc.cg(dims, Uh, kappa, b, tol=1e-12)
    U, Us = upload_gauge(Uh, dims, sloppy)
    bf = upload_half(b, dims, 0)
    x = lqcd.spinor_field(dims, 0)
    rc, info = lqcd.cg_solve(x, U, bf, kappa, lqcd.cg_params(tol=1e-10, sloppy=sloppy, delta=0.1), U_sloppy=Us)
    assert rc == lqcd.OK and info.true_rel_res <= 1e-10 and info.restarts >= 1
    xf = full_from_half(x.download(), dims, 0)
    r = b - orc.mdagm(dims, Uh, kappa, xf)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
    assert rel_err(x.download(), half(xr, dims, 0)) < 1e-8


def test_cg_edge_cases():
    dims = (4, 4, 4, 4)
    Uh = orc.gauge_start(dims, seed=1, eps=0.3)
    U = lqcd.gauge_field(dims).upload(Uh)
    x = lqcd.spinor_field(dims, 0)
    zero = lqcd.spinor_field(dims, 0).upload(np.zeros((128, 4, 3), complex))
    rc, info = lqcd.cg_solve(x, U, zero, 0.156)
    assert rc == lqcd.OK and info.iters == 0 and np.all(x.download() == 0)
    b = upload_half(inputs.random_spinor(dims, 17, parity=0), dims, 0)
    rc, info = lqcd.cg_solve(x, U, b, 0.156, lqcd.cg_params(tol=1e-12, maxiter=3), check=False)
    assert rc == lqcd.ENOCONV and info.iters == 3 and info.true_rel_res > 1e-12
    with pytest.raises(lqcd.LqcdError):
        lqcd.cg_solve(x, U, x, 0.156)


@pytest.mark.parametrize("dims", PARITY_DIMS[:3])
def test_gauge_force_matches_oracle(dims):
    beta, coeff = 5.6, 0.037
    Uh = orc.gauge_start(dims, seed=5, eps=0.4)
    Ph = inputs.random_momentum(dims, 18)
    U = lqcd.gauge_field(dims).upload(Uh)
    P = lqcd.momentum_field(dims).upload(Ph)
    lqcd.gauge_force(P, U, beta, coeff)
    F = orc.gauge_force(dims, Uh, beta)
    assert np.max(np.abs(P.download() - (Ph - coeff * F))) < 1e-13 * max(1, np.abs(F).max())


@pytest.mark.parametrize("dims", PARITY_DIMS[:3])
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_fermion_force_matches_oracle(dims, t_bc):
    kappa, coeff = 0.156, 0.05
    Uh = orc.gauge_start(dims, seed=6, eps=0.4)
    X = inputs.random_spinor(dims, 19, parity=0)
    Ph = inputs.random_momentum(dims, 20)
    U = lqcd.gauge_field(dims, t_bc=t_bc).upload(Uh)
    P = lqcd.momentum_field(dims, t_bc=t_bc).upload(Ph)
    Xf = lqcd.spinor_field(dims, 0, t_bc=t_bc).upload(half(X, dims, 0))
    lqcd.fermion_force(P, U, Xf, kappa, coeff)
    F = orc.fermion_force(dims, Uh, kappa, X, t_bc=t_bc)
    assert np.max(np.abs(P.download() - (Ph - coeff * F))) < 1e-12 * max(1, np.abs(F).max())


@pytest.mark.parametrize("which", ["gauge", "fermion"])
def test_fp32_forces_close_to_oracle(which):
    """FP32-arithmetic forces (the mixed trajectory's) against the FP64 oracle:
    FP32 rounding of links, spinors and staple products bounds the error at a
    few 1e-6 of the largest force component."""
    dims = (8, 6, 6, 12)
    kappa, beta, coeff = 0.156, 5.6, 0.05
    Uh = orc.gauge_start(dims, seed=6, eps=0.4)
    Ph = inputs.random_momentum(dims, 21)
    U = lqcd.gauge_field(dims).upload(Uh)
    P = lqcd.momentum_field(dims).upload(Ph)
    if which == "gauge":
        lqcd.gauge_force(P, U, beta, coeff, arith=lqcd.F32)
        F = orc.gauge_force(dims, Uh, beta)
    else:
        X = inputs.random_spinor(dims, 22, parity=0)
        Xf = lqcd.spinor_field(dims, 0).upload(half(X, dims, 0))
        lqcd.fermion_force(P, U, Xf, kappa, coeff, arith=lqcd.F32)
        F = orc.fermion_force(dims, Uh, kappa, X)
    err = np.max(np.abs((Ph - P.download()) / coeff - F))
    assert err < 5e-6 * np.abs(F).max(), err
    assert err > 0  # it really ran in FP32


@pytest.mark.parametrize("sloppy", [lqcd.F32, lqcd.F16N])
def test_cg_mixed_tight_tolerance(sloppy):
    """Solving to 1e-12 needs the float-float residual of the reliable updates
    to be accurate to ~1e-13 of |b|; the oracle's FP64 operator checks it."""
    dims = (8, 6, 6, 12)
    kappa = 0.156
    Uh = orc.gauge_start(dims, seed=2, eps=0.3)
    b = inputs.random_spinor(dims, 23, parity=0)
    U, Us = upload_gauge(Uh, dims, sloppy)
    bf = upload_half(b, dims, 0)
    x = lqcd.spinor_field(dims, 0)
    rc, info = lqcd.cg_solve(x, U, bf, kappa, lqcd.cg_params(tol=1e-12, sloppy=sloppy, delta=0.05), U_sloppy=Us)
    assert rc == lqcd.OK and info.true_rel_res <= 1e-12
    r = b - orc.mdagm(dims, Uh, kappa, full_from_half(x.download(), dims, 0))
    assert np.linalg.norm(r) <= 1.05e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("sloppy", [lqcd.F64, lqcd.F16N])
def test_cg_warm_start(sloppy):
    """x on entry as the initial guess: the exact solution needs no iteration,
    a perturbed one converges in fewer iterations than x0 = 0 to the same true
    residual"""
    dims = (8, 6, 6, 12)
    kappa = 0.156
    Uh = orc.gauge_start(dims, seed=2, eps=0.3)
    bh = inputs.random_spinor(dims, 24, parity=0)
    xr, _, _, _ = orc.cg(dims, Uh, kappa, bh, tol=1e-13)
    if sloppy == lqcd.F64:
        U, Us = lqcd.gauge_field(dims).upload(Uh), None
    else:
        U, Us = upload_gauge(Uh, dims, sloppy)
    b = upload_half(bh, dims, 0)
    prm = dict(tol=1e-10, sloppy=sloppy, delta=0.01)
    x = lqcd.spinor_field(dims, 0)
    rc, cold = lqcd.cg_solve(x, U, b, kappa, lqcd.cg_params(**prm), U_sloppy=Us)
    assert rc == lqcd.OK
    x.upload(half(xr, dims, 0))
    rc, exact = lqcd.cg_solve(x, U, b, kappa, lqcd.cg_params(**prm, guess=True), U_sloppy=Us)
    assert rc == lqcd.OK and exact.iters == 0 and exact.true_rel_res <= 1e-10
    noise = 1e-4 * inputs.random_spinor(dims, 25, parity=0)
    x.upload(half(xr + noise, dims, 0))
    rc, warm = lqcd.cg_solve(x, U, b, kappa, lqcd.cg_params(**prm, guess=True), U_sloppy=Us)
    assert rc == lqcd.OK and warm.true_rel_res <= 1e-10 and 0 < warm.iters < cold.iters
    r = bh - orc.mdagm(dims, Uh, kappa, full_from_half(x.download(), dims, 0))
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bh)
    # accurate residuals: one per restart (reliable update or failed check) and
    # one at the end, plus one of the guess; a guess that solves takes just that
    assert cold.accurate_residuals == cold.restarts + 1 and warm.accurate_residuals == warm.restarts + 2
    assert exact.accurate_residuals == 1 and exact.restarts == 0
    for info in (cold, exact, warm):
        assert 0 <= info.failed_checks <= info.restarts
