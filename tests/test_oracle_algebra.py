"""Oracle pins: gamma matrices, su(3) generators, exp, reunitarization.

Each test checks the oracle against mathematics fixed independently of it
(the Clifford algebra, the su(3) Lie algebra, scipy's expm, numpy's QR)."""
import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs


def test_gamma_clifford_algebra():
    g = [orc.gamma(k) for k in range(4)]
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0), "gamma_mu Hermitian"
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2 * np.eye(4) * (mu == nu), atol=0)


def test_gamma5_chiral_diagonal():
    g5 = orc.gamma(4)
    prod = orc.gamma(0) @ orc.gamma(1) @ orc.gamma(2) @ orc.gamma(3)
    assert np.array_equal(g5, prod)
    assert np.array_equal(g5, np.diag([1, 1, -1, -1]).astype(complex))
    for mu in range(4):
        assert np.allclose(g5 @ orc.gamma(mu) + orc.gamma(mu) @ g5, 0, atol=0)


def _gen(a):
    c = np.zeros(8)
    c[a] = 1.0
    return orc.algebra_to_mat(c)


def test_generators_normalised_hermitian_traceless():
    T = [_gen(a) for a in range(8)]
    for a in range(8):
        assert np.allclose(T[a], T[a].conj().T, atol=1e-16)
        assert abs(np.trace(T[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) - 0.5 * (a == b)) < 1e-15


def test_generators_close_su3_algebra():
    """[T_a, T_b] = i f_abc T_c with f real, totally antisymmetric, f_123 = 1,
    and Casimir sum_a T_a^2 = 4/3 (the fundamental of su(3))."""
    T = [_gen(a) for a in range(8)]
    f = np.zeros((8, 8, 8))
    for a in range(8):
        for b in range(8):
            comm = T[a] @ T[b] - T[b] @ T[a]
            for c in range(8):
                f[a, b, c] = (2 * np.trace(comm @ T[c]) / 1j).real
                assert abs((2 * np.trace(comm @ T[c]) / 1j).imag) < 1e-15
            recon = sum(1j * f[a, b, c] * T[c] for c in range(8))
            assert np.allclose(recon, comm, atol=1e-15)
    assert np.allclose(f, -np.transpose(f, (1, 0, 2)), atol=1e-15)
    assert np.allclose(f, np.transpose(f, (1, 2, 0)), atol=1e-15)
    assert abs(f[0, 1, 2] - 1) < 1e-15
    cas = sum(t @ t for t in T)
    assert np.allclose(cas, 4 / 3 * np.eye(3), atol=1e-15)


@pytest.mark.parametrize("scale", [1e-3, 0.3, 2.0, 7.0])
def test_expi_matches_scipy_expm(scale):
    rng = np.random.default_rng(7)
    for _ in range(20):
        c8 = rng.standard_normal(8)
        H = orc.algebra_to_mat(c8)
        E = orc.su3_expi(H, scale)
        ref = scipy.linalg.expm(1j * scale * H)
        assert np.max(np.abs(E - ref)) < 2e-14 * max(1.0, scale)
        assert np.max(np.abs(E @ E.conj().T - np.eye(3))) < 1e-14 * max(1.0, scale)
        assert abs(np.linalg.det(E) - 1) < 1e-14 * max(1.0, scale)


def test_reunit_matches_qr_and_fixes_det():
    rng = np.random.default_rng(3)
    U = inputs.random_unitary3(rng, 50, 1.0)
    for u in U:
        noisy = u + 1e-3 * (rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)))
        r = orc.reunit_mat(noisy)
        assert np.max(np.abs(r @ r.conj().T - np.eye(3))) < 1e-15
        assert abs(np.linalg.det(r) - 1) < 1e-15
        # rows 0, 1 are Gram-Schmidt of the input rows = Q of a QR of the transpose
        q, R = np.linalg.qr(noisy.T)
        q = q * (np.diag(R) / np.abs(np.diag(R)))[None, :]
        assert np.allclose(r[0], q[:, 0], atol=1e-15)
        assert np.allclose(r[1], q[:, 1], atol=1e-15)
        # an exact SU(3) matrix is a fixed point
        assert np.allclose(orc.reunit_mat(u), u, atol=2e-15)
