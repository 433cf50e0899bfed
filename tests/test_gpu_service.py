"""The solve service: point-source solves of the full Wilson operator on
resident gauge fields, continuously batched.  Each right-hand side meets the
full-operator tolerance, agrees with the oracle's solve, and gives bitwise the
same solution alone and in a mix of concurrent requests."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import lqcd
from tests.gpu_util import full_from_half

pytestmark = pytest.mark.gpu

LATS = [(4, 4, 4, 4), (6, 4, 4, 8), (8, 8, 8, 8)]
TOL = 1e-10


def _gauges():
    out = []
    for k, dims in enumerate(LATS):
        Uh = orc.gauge_start(dims, seed=20 + k, eps=0.25)
        out.append((dims, Uh, lqcd.gauge_field(dims).upload(Uh)))
    return out


def _solution(svc, ticket, k, dims):
    e, o = svc.solution(ticket, k)
    xe = lqcd.Field.borrowed(e, dims, lqcd.SPINOR_EVEN).download()
    xo = lqcd.Field.borrowed(o, dims, lqcd.SPINOR_ODD).download()
    return full_from_half(xe, dims, 0) + full_from_half(xo, dims, 1)


def _point(dims, site, comp):
    V = int(np.prod(dims))
    b = np.zeros((V, 4, 3), complex)
    x, y, z, t = site
    i = x + dims[0] * (y + dims[1] * (z + dims[2] * t))
    b[i, comp // 3, comp % 3] = 1.0
    return b


REQS = [(0, 0.150, (1, 2, 3, 0), 12), (1, 0.1575, (5, 0, 2, 7), 3), (2, 0.156, (0, 0, 0, 0), 2),
        (0, 0.158, (3, 3, 3, 3), 4), (2, 0.152, (7, 1, 4, 5), 1)]


def test_service_solves_against_oracle():
    gauges = _gauges()
    svc = lqcd.Service(lqcd.service_params(tol=TOL))
    ids = [svc.add_gauge(U) for _, _, U in gauges]
    tickets = [svc.submit(ids[g], kappa, site, nrhs) for g, kappa, site, nrhs in REQS]
    for t, (g, kappa, site, nrhs) in zip(tickets, REQS):
        r = svc.wait(t)
        assert r["status"] == lqcd.OK and r["nrhs"] == nrhs and r["iters"] > 0
        assert r["true_rel_res_max"] <= TOL and r["latency_s"] >= r["queue_s"] >= 0
        dims, Uh, _ = gauges[g]
        for k in range(nrhs):
            x = _solution(svc, t, k, dims)
            b = _point(dims, site, k)
            res = np.linalg.norm(b - orc.wilson(dims, Uh, kappa, x))
            assert res <= 1.05 * TOL  # the oracle's FP64 operator agrees with the reported residual
            if g == 0 or k == 0:
                xo, conv, _ = orc.wilson_solve(dims, Uh, kappa, b, tol=1e-13)
                assert conv
                assert np.max(np.abs(x - xo)) <= 1e-8 * np.max(np.abs(xo))
        svc.release(t)
    svc.close()


def _run(reqs, gauges, **kw):
    svc = lqcd.Service(lqcd.service_params(tol=TOL, **kw))
    ids = [svc.add_gauge(U) for _, _, U in gauges]
    tickets = [svc.submit(ids[g], kappa, site, nrhs) for g, kappa, site, nrhs in reqs]
    out = []
    for t, (g, _, _, nrhs) in zip(tickets, reqs):
        r = svc.wait(t)
        assert r["status"] == lqcd.OK, r
        out.append((r, [_solution(svc, t, k, gauges[g][0]) for k in range(nrhs)]))
    svc.close()
    return out


def test_same_result_alone_and_in_the_mix():
    gauges = _gauges()
    mixed = _run(REQS * 2, gauges)
    for i, req in enumerate(REQS):
        (ra, xa), = _run([req], gauges)
        for rm, xm in (mixed[i], mixed[i + len(REQS)]):
            assert rm["iters"] == ra["iters"] and rm["refinements"] == ra["refinements"]
            assert rm["true_rel_res_max"] == ra["true_rel_res_max"]
            for a, m in zip(xa, xm):
                assert np.array_equal(a, m)


def test_admission_by_footprint():
    """a budget below two requests runs them one at a time; the results do not change"""
    gauges = _gauges()[:2]
    reqs = [(1, 0.155, (1, 1, 1, 1), 6), (0, 0.152, (0, 1, 2, 3), 6), (1, 0.157, (2, 0, 0, 6), 6)]
    free = _run(reqs, gauges)
    tight = _run(reqs, gauges, hbm_budget=1)  # every request alone
    cap = _run(reqs, gauges, max_active_rhs=6)
    for (rf, xf), (rt, xt), (rc, xc) in zip(free, tight, cap):
        assert rf["iters"] == rt["iters"] == rc["iters"]
        for a, b, c in zip(xf, xt, xc):
            assert np.array_equal(a, b) and np.array_equal(a, c)
    # alone, a later request waits for the earlier ones
    assert tight[2][0]["queue_s"] >= tight[0][0]["latency_s"] * 0.5


class LiveBytes:
    """an allocator hook over PyTorch's caching allocator that tracks the live
    device bytes the library holds and their peak"""

    def __init__(self):
        import torch
        self.torch, self.live, self.sizes, self.peak = torch, 0, {}, 0

    def alloc(self, nbytes, stream):
        p = self.torch.cuda.caching_allocator_alloc(nbytes)
        self.sizes[p] = nbytes
        self.live += nbytes
        self.peak = max(self.peak, self.live)
        return p

    def free(self, ptr, stream):
        self.live -= self.sizes.pop(ptr)
        self.torch.cuda.caching_allocator_delete(ptr)


def test_device_bytes_stay_within_budget():
    """the idle solver work spaces pooled for reuse count against hbm_budget:
    with a budget of one 12-source request, requests on two 8^4 gauge fields
    in turn keep the service's device bytes (everything the library
    allocates, less the gauge fields' fixed link copies and temporaries)
    within the budget plus the batch engine's small tables; the first field's
    idle work spaces are freed to admit the second's request"""
    dims = (8, 8, 8, 8)
    Us = [lqcd.gauge_field(dims).upload(orc.gauge_start(dims, seed=30 + k, eps=0.25)) for k in range(2)]
    Vh = int(np.prod(dims)) // 2
    # one right-hand side: float-float solution and source, FP32 increment,
    # four FP16+norm vectors, the FP64 solution halves, scalars and partials
    one = Vh * (2 * 192 + 96 + 4 * 52 + 2 * 192) + 2048 * 8 + 4096
    budget = 12 * one + one // 2
    tables = 1 << 20
    live = LiveBytes()
    lqcd.set_allocator(live.alloc, live.free)
    try:
        svc = lqcd.Service(lqcd.service_params(tol=TOL, hbm_budget=budget))
        ids = [svc.add_gauge(U) for U in Us]
        for rnd in range(2):
            for g in ids:
                t = svc.submit(g, 0.152 + 0.002 * g, (1, 2, 3, rnd), 12)
                r = svc.wait(t)
                assert r["status"] == lqcd.OK and r["true_rel_res_max"] <= TOL
                counted, fixed = svc.bytes()
                assert 0 < counted <= budget
                svc.release(t)
        counted, fixed = svc.bytes()
        assert 0 < counted <= budget  # the idle pool of the last field
        assert fixed > 0 and live.peak - fixed <= budget + tables, (live.peak, fixed, budget)
        svc.close()
        assert live.live == 0
    finally:
        lqcd.set_allocator(None, None)


def test_service_rejects_bad_requests():
    gauges = _gauges()[:1]
    with pytest.raises(lqcd.LqcdError):
        lqcd.Service(lqcd.service_params(sloppy=lqcd.F64))
    with pytest.raises(lqcd.LqcdError):
        lqcd.Service(lqcd.service_params(hbm_budget=0))
    svc = lqcd.Service(lqcd.service_params())
    gid = svc.add_gauge(gauges[0][2])
    with pytest.raises(lqcd.LqcdError):
        svc.add_gauge(lqcd.gauge_field((4, 4, 4, 4), lqcd.F16N))
    for bad in [dict(gauge=gid + 1), dict(nrhs=0), dict(nrhs=13), dict(site=(4, 0, 0, 0)), dict(site=(0, 0, -1, 0))]:
        a = dict(gauge=gid, kappa=0.15, site=(0, 0, 0, 0), nrhs=1)
        a.update(bad)
        with pytest.raises(lqcd.LqcdError):
            svc.submit(**a)
    with pytest.raises(lqcd.LqcdError):
        svc.poll(12345)
    t = svc.submit(gid, 0.15, (0, 0, 0, 0), 1)
    assert svc.wait(t)["status"] == lqcd.OK
    with pytest.raises(lqcd.LqcdError):
        svc.solution(t, 1)
    svc.release(t)
    with pytest.raises(lqcd.LqcdError):
        svc.poll(t)
    svc.close()
    svc.close()  # idempotent
