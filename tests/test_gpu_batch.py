"""Batched solves and batched chains: systems on lattices of different sizes
solved with shared launches give, system by system, exactly the iterates of
their solves alone; chains advanced together give their solo trajectories."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs, lqcd
from tests.gpu_util import full_from_half, half, upload_half

pytestmark = pytest.mark.gpu

LATTICES = [(4, 4, 4, 4), (6, 4, 2, 10), (8, 6, 6, 12), (4, 4, 4, 4), (2, 2, 2, 2)]


def _systems():
    out = []
    for k, dims in enumerate(LATTICES):
        Uh = orc.gauge_start(dims, seed=10 + k, eps=0.3)
        U = lqcd.gauge_field(dims).upload(Uh)
        Us = lqcd.gauge_field(dims, lqcd.F16N).copy_from(U)
        bh = inputs.random_spinor(dims, 30 + k, parity=0)
        b = upload_half(bh, dims, 0)
        out.append((dims, Uh, U, Us, bh, b, 0.150 + 0.0015 * k))
    return out


def test_batched_solve_equals_single_solves():
    systems = _systems()
    prm = lqcd.cg_params(tol=1e-10, sloppy=lqcd.F16N, delta=0.01)
    singles = []
    for dims, Uh, U, Us, bh, b, kappa in systems:
        x = lqcd.spinor_field(dims, 0)
        rc, info = lqcd.cg_solve(x, U, b, kappa, prm, U_sloppy=Us)
        assert rc == lqcd.OK
        singles.append((x.download(), info.iters, info.restarts))
    xs = [lqcd.spinor_field(s[0], 0) for s in systems]
    rc, infos = lqcd.cg_solve_batch(xs, [s[2] for s in systems], [s[3] for s in systems], [s[5] for s in systems],
                                    [s[6] for s in systems], prm)
    assert rc == lqcd.OK
    for (dims, Uh, U, Us, bh, b, kappa), x, info, (xr, it, rs) in zip(systems, xs, infos, singles):
        assert info.iters == it and info.restarts == rs
        assert np.array_equal(x.download(), xr)  # bitwise: same kernels, same reduction order
        r = bh - orc.mdagm(dims, Uh, kappa, full_from_half(x.download(), dims, 0))
        assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bh)


def test_batched_solve_edge_cases():
    systems = _systems()[:2]
    prm = lqcd.cg_params(tol=1e-10, sloppy=lqcd.F16N, delta=0.01)
    assert lqcd.cg_solve_batch([], [], [], [], [], prm)[0] == lqcd.OK
    # a zero source finishes at start; the other system still runs
    zero = lqcd.spinor_field(systems[0][0], 0).upload(np.zeros((128, 4, 3), complex))
    xs = [lqcd.spinor_field(s[0], 0) for s in systems]
    rc, infos = lqcd.cg_solve_batch(xs, [s[2] for s in systems], [s[3] for s in systems], [zero, systems[1][5]],
                                    [0.15, 0.15], prm)
    assert rc == lqcd.OK and infos[0].iters == 0 and infos[1].iters > 0
    assert np.all(xs[0].download() == 0)
    # maxiter reached in one system
    rc, infos = lqcd.cg_solve_batch(xs, [s[2] for s in systems], [s[3] for s in systems], [s[5] for s in systems],
                                    [0.15, 0.15], lqcd.cg_params(tol=1e-12, maxiter=3, sloppy=lqcd.F16N, delta=0.01),
                                    check=False)
    assert rc == lqcd.ENOCONV and all(i.iters <= 4 for i in infos)
    with pytest.raises(lqcd.LqcdError):  # the batched engine is mixed precision only
        lqcd.cg_solve_batch(xs, [s[2] for s in systems], [s[3] for s in systems], [s[5] for s in systems],
                            [0.15, 0.15], lqcd.cg_params())


@pytest.mark.parametrize("chrono", [0, 1, 3])
def test_batched_chains_equal_solo_chains(chrono):
    specs = [((4, 4, 4, 4), 5.6, 0.150, 1), ((6, 4, 2, 10), 5.7, 0.153, 2), ((8, 6, 6, 12), 5.9, 0.157, 3)]
    cg = lqcd.cg_params(tol=1e-10, sloppy=lqcd.F16N, delta=0.01)

    def params(beta, kappa):
        return lqcd.hmc_params(beta, kappa, 0.3, 4, lqcd.OMELYAN, cg=cg, force_prec=lqcd.F32, chrono=chrono)

    solo = []
    for dims, beta, kappa, seed in specs:
        U = lqcd.gauge_field(dims)
        lqcd.gauge_start(U, seed, 0.3)
        st = lqcd.HmcState(U, seed=seed, chain=seed)
        infos = [st.trajectory(params(beta, kappa)) for _ in range(2)]
        solo.append((U.download(), infos))
        st.close()
    fields, states = [], []
    for dims, beta, kappa, seed in specs:
        U = lqcd.gauge_field(dims)
        lqcd.gauge_start(U, seed, 0.3)
        fields.append(U)
        states.append(lqcd.HmcState(U, seed=seed, chain=seed))
    batch = lqcd.Batch(states)
    plist = [params(beta, kappa) for _, beta, kappa, _ in specs]
    got = [batch.trajectory(plist) for _ in range(2)]
    for i in range(len(specs)):
        Us, infos = solo[i]
        for t in range(2):
            g, o = got[t][i], infos[t]
            assert g["dH"] == o["dH"] and g["accepted"] == o["accepted"] and g["cg_iters"] == o["cg_iters"]
        assert np.array_equal(fields[i].download(), Us)
    batch.close()
    for st in states:
        st.close()
