"""Failure detection and recovery, made on the host without faulting the GPU:
an allocator hook that returns NULL at every allocation in turn during a whole
trajectory (LQCD_ENOMEM, nothing leaked, the state usable afterwards and then
bitwise the unbroken result), a NaN planted in the host links (LQCD_ENUMERIC,
the trajectory rejected, no hang), a solver capped at one iteration (the
trajectory goes on and reports the failure), checkpoint and resume bit for bit
against an unbroken chain, and the per-trajectory JSONL log."""
import json

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1212_0785_gb300 import lqcd

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)


def mixed_params(**kw):
    cg = lqcd.cg_params(tol=1e-10, maxiter=kw.pop("maxiter", 20000), sloppy=lqcd.F16N, delta=0.003)
    base = dict(tau=0.5, nsteps=4, integrator=lqcd.OMELYAN, cg=cg, force_prec=lqcd.F32, chrono=3, chrono_mre=True)
    base.update(kw)
    return lqcd.hmc_params(5.8, 0.157, **base)


class CountingAllocator:
    """device memory from PyTorch's caching allocator; counts the calls, keeps
    the live blocks, and returns NULL at call number fail_at"""

    def __init__(self, fail_at=None):
        self.fail_at, self.calls, self.live = fail_at, 0, {}

    def alloc(self, nbytes, stream):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(nbytes)
        self.live[p] = nbytes
        return p

    def free(self, ptr, stream):
        assert ptr in self.live, "freed a block this hook did not give out"
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(ptr)


@pytest.fixture
def hook():
    yield
    lqcd.set_allocator(None, None)


def _reference(p):
    U = lqcd.gauge_field(DIMS)
    lqcd.gauge_start(U, 3, 0.3)
    st = lqcd.HmcState(U, seed=3)
    g = st.trajectory(p)
    out = U.download()
    st.close()
    return g, out


def test_allocation_failure_at_every_allocation(hook):
    p = mixed_params()
    ref, Uref = _reference(p)
    counter = CountingAllocator()
    lqcd.set_allocator(counter.alloc, counter.free)
    U = lqcd.gauge_field(DIMS)
    lqcd.gauge_start(U, 3, 0.3)
    st = lqcd.HmcState(U, seed=3)
    st.trajectory(p)
    st.close()
    U.free()
    total = counter.calls
    assert total > 10 and not counter.live
    failures = 0
    for fail_at in range(1, total + 1):
        a = CountingAllocator(fail_at)
        lqcd.set_allocator(a.alloc, a.free)
        U = st = None
        try:
            U = lqcd.gauge_field(DIMS)
            lqcd.gauge_start(U, 3, 0.3)
            st = lqcd.HmcState(U, seed=3)
            st.trajectory(p)
        except lqcd.LqcdError as e:
            assert e.status == lqcd.ENOMEM, (fail_at, e)
            failures += 1
            if st is not None:
                # the failed trajectory left the state usable: the same
                # trajectory again (allocations succeed now) is bitwise the
                # unbroken one
                a.fail_at = None
                lqcd.gauge_start(U, 3, 0.3)
                st.traj = 0
                g = st.trajectory(p)
                assert g["dH"] == ref["dH"] and g["cg_iters"] == ref["cg_iters"], fail_at
                assert np.array_equal(U.download(), Uref), fail_at
        finally:
            if st is not None:
                st.close()
            if U is not None:
                U.free()
        assert not a.live, (fail_at, len(a.live))  # every block came back
    assert failures == total


@pytest.mark.parametrize("mixed", [False, True])
def test_nan_link_is_rejected(mixed):
    Uh = orc.gauge_start(DIMS, seed=1, eps=0.3)
    Uh[17, 2, 1, 0] = np.nan
    U = lqcd.gauge_field(DIMS).upload(Uh)
    st = lqcd.HmcState(U, seed=1)
    # no reunitarization after the reject, so the restored links are the uploaded bits
    p = (mixed_params(reunitarize=False) if mixed else
         lqcd.hmc_params(5.6, 0.156, 0.5, 4, cg=lqcd.cg_params(tol=1e-10), reunitarize=False))
    with pytest.raises(lqcd.LqcdError) as ei:
        st.trajectory(p)
    assert ei.value.status == lqcd.ENUMERIC
    back = U.download()  # rejected: the links are the uploaded ones
    assert np.isnan(back[17, 2, 1, 0]) and np.array_equal(np.nan_to_num(back), np.nan_to_num(Uh))
    st.close()
    # pure gauge: the non-finite dH rejects
    U2 = lqcd.gauge_field(DIMS).upload(Uh)
    st2 = lqcd.HmcState(U2, seed=1)
    with pytest.raises(lqcd.LqcdError) as ei:
        st2.trajectory(lqcd.hmc_params(5.6, 0.0, 0.5, 4, n_flavors=0, reunitarize=False))
    assert ei.value.status == lqcd.ENUMERIC
    st2.close()
    # the library stays usable
    g, _ = _reference(mixed_params())
    assert np.isfinite(g["dH"])


def test_solver_capped_at_one_iteration():
    """maxiter 1: every solve stops unconverged; the trajectory finishes and
    reports the failed solves instead of raising"""
    U = lqcd.gauge_field(DIMS)
    lqcd.gauge_start(U, 3, 0.3)
    st = lqcd.HmcState(U, seed=3)
    g = st.trajectory(mixed_params(maxiter=1, chrono=0, chrono_mre=False))
    assert g["cg_failures"] == g["n_solves"] > 0 and g["cg_iters"] <= g["n_solves"] + 1
    st.close()


def test_checkpoint_resume_is_bitwise(tmp_path):
    p = mixed_params(metropolis=False)
    U = lqcd.gauge_field(DIMS)
    lqcd.gauge_start(U, 3, 0.3)
    st = lqcd.HmcState(U, seed=3, chain=5)
    unbroken = [st.trajectory(p) for _ in range(3)]
    U_unbroken = U.download()
    st.close()
    U = lqcd.gauge_field(DIMS)
    lqcd.gauge_start(U, 3, 0.3)
    st = lqcd.HmcState(U, seed=3, chain=5)
    first = st.trajectory(p)
    ck = tmp_path / "chain.npz"
    st.checkpoint(ck)
    st.close()
    U.free()
    st2 = lqcd.HmcState.resume(ck)
    assert st2.traj == 1 and st2.seed == 3 and st2.chain == 5
    rest = [st2.trajectory(p) for _ in range(2)]
    for a, b in zip([first] + rest, unbroken):
        assert a == {**b, "seconds": a["seconds"]}, (a, b)
    assert np.array_equal(st2.U.download(), U_unbroken)
    st2.close()


def test_trajectory_jsonl_log(tmp_path):
    log = tmp_path / "traj.jsonl"
    U = lqcd.gauge_field(DIMS)
    lqcd.gauge_start(U, 3, 0.3)
    st = lqcd.HmcState(U, seed=3)
    infos = [st.trajectory(mixed_params(), log=str(log)) for _ in range(2)]
    st.close()
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert len(lines) == 2
    for rec, info in zip(lines, infos):
        for k in ("dH", "accepted", "plaq", "cg_iters", "cg_true_rel_res_max", "seconds", "traj"):
            assert rec[k] == info[k]
        assert rec["status"] == lqcd.OK and rec["dims"] == list(DIMS) and rec["seed"] == 3
