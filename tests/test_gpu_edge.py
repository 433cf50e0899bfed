"""GPU degenerate and edge cases against the oracle or closed forms: extents of
2 (forward and backward neighbours coincide), the free field, kappa = 0,
zero momenta, mismatched arguments."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs, lqcd
from tests.gpu_util import full_from_half, half, rel_err, upload_half

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 6), (4, 2, 2, 2)])
def test_dslash_extent_two(dims):
    Uh = inputs.random_gauge(dims, 1)
    s = inputs.random_spinor(dims, 2, parity=0)
    U = lqcd.gauge_field(dims).upload(Uh)
    out = lqcd.spinor_field(dims, 1)
    lqcd.dslash(out, U, upload_half(s, dims, 0))
    ref = half(orc.dslash(dims, Uh, s, out_parity=1), dims, 1)
    assert rel_err(out.download(), ref) < 1e-13


def test_free_field_closed_form():
    """unit links: a plane wave with antiperiodic p_t is an eigenvector of D with
    eigenvalue matrix sum_mu (2 cos p_mu - 2 i gamma_mu sin p_mu) (restricted to
    the odd output sites)"""
    dims = (4, 6, 4, 8)
    V = int(np.prod(dims))
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    coords = [c.reshape(-1) for c in (x, y, z, t)]
    p = [2 * np.pi / Lx, 2 * np.pi * 2 / Ly, 0.0, 3 * np.pi / Lt]
    u = inputs.random_spinor((1, 1, 1, 1), 3)[0]
    phase = np.exp(1j * sum(p[m] * coords[m] for m in range(4)))
    psi = phase[:, None, None] * u[None]
    Ug = np.zeros((V, 4, 3, 3), complex)
    Ug[:] = np.eye(3)
    U = lqcd.gauge_field(dims).upload(Ug)
    out = lqcd.spinor_field(dims, 1)
    lqcd.dslash(out, U, upload_half(psi, dims, 0))
    G = [orc.gamma(m) for m in range(4)]
    K = sum(2 * np.cos(p[m]) * np.eye(4) - 2j * np.sin(p[m]) * G[m] for m in range(4))
    expect = half(phase[:, None, None] * (K @ u)[None], dims, 1)
    assert np.max(np.abs(out.download() - expect)) < 1e-13


def test_kappa_zero_solve_is_identity():
    dims = (4, 4, 4, 4)
    U = lqcd.gauge_field(dims).upload(inputs.random_gauge(dims, 4))
    b = upload_half(inputs.random_spinor(dims, 5, parity=0), dims, 0)
    x = lqcd.spinor_field(dims, 0)
    rc, info = lqcd.cg_solve(x, U, b, 0.0, lqcd.cg_params(tol=1e-12))
    assert rc == lqcd.OK and info.iters == 1
    assert np.max(np.abs(x.download() - b.download())) < 1e-15


def test_zero_momenta_keep_links():
    dims = (4, 4, 4, 4)
    Uh = orc.gauge_start(dims, 1, 0.3)
    U = lqcd.gauge_field(dims).upload(Uh)
    P = lqcd.momentum_field(dims).upload(np.zeros((256, 4, 8)))
    lqcd.link_update(U, P, 0.7)
    assert np.max(np.abs(U.download() - Uh)) < 1e-15


def test_mismatched_arguments_are_rejected():
    a, b = (4, 4, 4, 4), (4, 4, 4, 6)
    U = lqcd.gauge_field(a)
    out = lqcd.spinor_field(b, 1)
    with pytest.raises(lqcd.LqcdError) as e:
        lqcd.dslash(out, U, lqcd.spinor_field(a, 0))
    assert e.value.status == lqcd.EINVAL
    with pytest.raises(lqcd.LqcdError):  # same parity in and out
        lqcd.dslash(lqcd.spinor_field(a, 0), U, lqcd.spinor_field(a, 0))
    with pytest.raises(lqcd.LqcdError):  # FP16 spinors with FP64 links
        lqcd.dslash(lqcd.spinor_field(a, 1, lqcd.F16N), U, lqcd.spinor_field(a, 0, lqcd.F16N))
    with pytest.raises(lqcd.LqcdError):
        lqcd.gauge_force(lqcd.momentum_field(b), U, 5.6, 0.1)
    with pytest.raises(lqcd.LqcdError):  # mixed solve without matching sloppy links
        lqcd.cg_solve(lqcd.spinor_field(a, 0), U, lqcd.spinor_field(a, 0), 0.1,
                      lqcd.cg_params(sloppy=lqcd.F16N), U_sloppy=lqcd.gauge_field(a, lqcd.BF16))
    st = lqcd.HmcState(U, seed=1)
    with pytest.raises(lqcd.LqcdError):
        st.trajectory(lqcd.hmc_params(5.6, 0.1, tau=1.0, nsteps=0))
    st.close()
