"""Oracle pins: Philox4x32-10 against cuRAND's host generator, and the
distributions of uniforms, Gaussians, momenta and pseudofermion sources."""
import ctypes
import os

import numpy as np
import pytest
import scipy.stats

from oracle import oracle as orc

_CURAND_PATHS = ["/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"]
CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for p in _CURAND_PATHS:
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1, (5 << 32) | 7, 0xDEADBEEFCAFEBABE])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host-side PHILOX4_32_10 generator with a 64-bit seed s emits, as
    its n-th 128-bit block (n < 1024), Philox4x32-10 of counter (0, 0, n, 0)
    under key (s mod 2^32, s >> 32): a library implementation of the SC'11
    algorithm that shares nothing with the oracle."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    g = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        for n0 in (0, 2, 999):
            assert cr.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
            assert cr.curandSetGeneratorOffset(g, ctypes.c_ulonglong(4 * n0)) == 0
            buf = (ctypes.c_uint32 * 64)()
            assert cr.curandGenerate(g, buf, ctypes.c_size_t(64)) == 0
            got = np.array(list(buf), np.uint32).reshape(16, 4)
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for k in range(16):
                assert np.array_equal(orc.philox4x32_10([0, 0, n0 + k, 0], key), got[k])
    finally:
        cr.curandDestroyGenerator(g)


def test_philox_counter_words_all_matter():
    base = orc.philox4x32_10([1, 2, 3, 4], [5, 6])
    for w in range(4):
        c = [1, 2, 3, 4]
        c[w] ^= 1
        assert not np.array_equal(orc.philox4x32_10(c, [5, 6]), base)
    for w in range(2):
        k = [5, 6]
        k[w] ^= 1
        assert not np.array_equal(orc.philox4x32_10([1, 2, 3, 4], k), base)


def test_uniforms_open_interval_and_moments():
    u = np.array([orc.uniform2(9, 0, s, j, 1, 0) for s in range(2000) for j in range(4)]).ravel()
    assert np.all(u > 0) and np.all(u < 1)
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / u.size)
    assert scipy.stats.kstest(u, "uniform").pvalue > 1e-4


def test_gaussians_standard_normal():
    g = np.array([orc.gauss2(11, 3, s, j, 2, 5) for s in range(3000) for j in range(4)]).ravel()
    assert abs(g.mean()) < 4 / np.sqrt(g.size)
    assert abs(g.var() - 1) < 4 * np.sqrt(2 / g.size)
    assert scipy.stats.kstest(g, "norm").pvalue > 1e-4


def test_momentum_and_eta_refresh_distributions():
    dims = (4, 4, 4, 8)
    V = int(np.prod(dims))
    P = orc.momentum_refresh(dims, seed=2, traj=7)
    assert P.shape == (V, 4, 8)
    assert abs(P.var() - 1) < 4 * np.sqrt(2 / P.size)
    assert scipy.stats.kstest(P.ravel(), "norm").pvalue > 1e-4
    P2 = orc.momentum_refresh(dims, seed=2, traj=8)
    assert not np.allclose(P, P2)
    eta = orc.eta_refresh(dims, seed=2, traj=7)
    par = orc.parity(dims)
    assert np.all(eta[par == 1] == 0)
    re = np.concatenate([eta[par == 0].real.ravel(), eta[par == 0].imag.ravel()])
    assert abs(re.var() - 0.5) < 4 * 0.5 * np.sqrt(2 / re.size)
    assert scipy.stats.kstest(re / np.sqrt(0.5), "norm").pvalue > 1e-4


def test_gauge_start_is_special_unitary_and_seeded():
    dims = (4, 4, 4, 4)
    U = orc.gauge_start(dims, seed=1, eps=0.3)
    dev = np.abs(np.einsum("xmab,xmcb->xmac", U, U.conj()) - np.eye(3)).max()
    assert dev < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    assert np.array_equal(U, orc.gauge_start(dims, seed=1, eps=0.3))
    assert not np.allclose(U, orc.gauge_start(dims, seed=2, eps=0.3))
    # eps -> 0 gives the unit gauge; mean plaquette decreases with eps
    assert abs(orc.plaquette(dims, orc.gauge_start(dims, 1, 0.0)) - 1) < 1e-15
    p = [orc.plaquette(dims, orc.gauge_start(dims, 1, e)) for e in (0.1, 0.2, 0.3)]
    assert 1 > p[0] > p[1] > p[2] > 0.5
