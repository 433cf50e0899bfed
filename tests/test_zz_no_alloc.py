"""The allocation-free plaquette (lqcd_plaquette_noalloc) against the
allocating one (lqcd_plaquette), called through the C ABI.

It serves callers that must not let the library allocate device memory, for
instance code on a thread that cannot call back into an allocator hook that
enters the Python interpreter.  Its partial sums live in one fixed device
array shared by all calls, so two calls in a row must both give the right
answer.  This file is collected last so that a run stopping at its first
failure has run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs, lqcd

pytestmark = pytest.mark.gpu


def _noalloc(U: lqcd.Field) -> float:
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    rc = lqcd.lib().lqcd_plaquette_noalloc(U.h, ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(lqcd.current_stream()))
    assert rc == lqcd.OK, lqcd.lib().lqcd_last_error().decode()
    torch.cuda.synchronize()
    return float(out.item())


def test_noalloc_plaquette_matches_allocating_call_twice():
    fields = []
    for dims, seed, eps in (((8, 6, 6, 12), 4, 0.4), ((6, 6, 10, 12), 5, 0.2)):
        U = lqcd.gauge_field(dims).upload(orc.gauge_start(dims, seed=seed, eps=eps))
        fields.append(U)
    # two calls in a row on different fields, then the first field again
    for U in fields + fields[:1]:
        ref = lqcd.plaquette(U)
        got = _noalloc(U)
        assert abs(got - ref) <= 1e-14 * abs(ref), (got, ref)


def test_noalloc_plaquette_full_size_and_random_links():
    dims = (32, 32, 32, 64)
    U = lqcd.gauge_field(dims)
    lqcd.gauge_start(U, seed=3, eps=0.15)
    ref = lqcd.plaquette(U)
    assert abs(_noalloc(U) - ref) <= 1e-14 * ref
    small = (4, 4, 4, 4)
    V = lqcd.gauge_field(small).upload(inputs.random_gauge(small, 9))
    assert abs(_noalloc(V) - lqcd.plaquette(V)) <= 1e-14


def test_noalloc_plaquette_rejects_lattices_above_its_limit():
    # 2 x 2 x 2 x 2097154 = 16,777,232 sites, just above LQCD_NOALLOC_MAX_SITES
    U = lqcd.gauge_field((2, 2, 2, 2097154))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lqcd.lib().lqcd_plaquette_noalloc(U.h, ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(lqcd.current_stream()))
    assert rc == lqcd.EINVAL
    assert b"fixed maximum" in lqcd.lib().lqcd_last_error()
    U.free()
    assert np.isfinite(out.cpu().numpy()).all()
