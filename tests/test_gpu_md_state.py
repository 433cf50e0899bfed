"""State the mixed molecular dynamics keeps between calls: the FP64 links,
written only after the molecular dynamics from the float-float copy, and the
float-float copy of phi, made once per refresh and reused by later solves.
Both must follow what the caller does between calls."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs, lqcd
from tests.gpu_util import full_from_half, half

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 6)


def _params(chrono=0):
    cg = lqcd.cg_params(tol=1e-10, sloppy=lqcd.F16N, delta=0.01)
    return lqcd.hmc_params(5.6, 0.15, 0.4, 4, lqcd.OMELYAN, cg=cg, force_prec=lqcd.F32, chrono=chrono)


def test_md_step_leaves_current_fp64_links():
    """after each md_step the FP64 links are the evolved ones: equal to the
    oracle's molecular dynamics from the same start within the FP32 bounds,
    and unitary (the lag never leaves stale links behind)"""
    U0 = orc.gauge_start(DIMS, seed=2, eps=0.3)
    U = lqcd.gauge_field(DIMS).upload(U0)
    st = lqcd.HmcState(U, seed=2)
    p = _params()
    st.refresh(p)
    _, P, phi = st.fields()
    P0, phi0 = P.download(), phi.download()
    for _ in range(2):
        before = U.download()
        st.md_step(p)
        after = U.download()
        assert np.max(np.abs(after - before)) > 1e-4  # the links moved
        uu = np.einsum("xmab,xmcb->xmac", after, after.conj())
        assert np.max(np.abs(uu - np.eye(3))) < 1e-12
    Uo, Po, _ = orc.md_integrate(DIMS, U0, P0, full_from_half(phi0, DIMS, 0), beta=5.6, kappa=0.15, tau=0.2,
                                 nsteps=2, integrator=orc.OMELYAN, cg_tol=1e-12)
    assert np.max(np.abs(U.download() - Uo)) < 1e-5
    st.close()


def test_phi_written_between_md_steps_is_used():
    """a solve reuses the float-float copy of phi only while phi is unchanged:
    after the caller writes phi between two md_steps, the second step is
    bitwise the step of a fresh state given the same links, momenta and phi"""
    U0 = orc.gauge_start(DIMS, seed=3, eps=0.3)
    p = _params()
    new_phi = half(inputs.random_spinor(DIMS, 7, parity=0), DIMS, 0)
    # a: one step with the refreshed phi (its copy is cached), then the new phi
    Ua = lqcd.gauge_field(DIMS).upload(U0)
    a = lqcd.HmcState(Ua, seed=3)
    a.refresh(p)
    _, Pa, phia = a.fields()
    P0 = Pa.download()
    a.md_step(p)
    Ua.upload(U0)
    Pa.upload(P0)
    phia.upload(new_phi)
    a.md_step(p)
    # b: a fresh state, the same links, momenta and phi
    Ub = lqcd.gauge_field(DIMS).upload(U0)
    b = lqcd.HmcState(Ub, seed=3)
    b.refresh(p)
    _, Pb, phib = b.fields()
    Pb.upload(P0)
    phib.upload(new_phi)
    b.md_step(p)
    assert np.array_equal(Pa.download(), Pb.download())
    assert np.array_equal(Ua.download(), Ub.download())
    a.close()
    b.close()
