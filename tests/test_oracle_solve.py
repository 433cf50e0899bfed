"""The oracle's full-operator solve (even-odd reduction, CG on the normal
equations, odd reconstruction) against a dense solve of M x = b built column
by column on lattices small enough for it."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs


def _dense_wilson(dims, U, kappa):
    V = int(np.prod(dims))
    n = 12 * V
    M = np.zeros((n, n), complex)
    for j in range(n):
        e = np.zeros(n, complex)
        e[j] = 1.0
        M[:, j] = orc.wilson(dims, U, kappa, e.reshape(V, 4, 3)).reshape(-1)
    return M


@pytest.mark.parametrize("dims,kappa", [((2, 2, 2, 4), 0.124), ((2, 2, 4, 2), 0.158)])
def test_wilson_solve_matches_dense(dims, kappa):
    U = inputs.random_gauge(dims, seed=5)
    V = int(np.prod(dims))
    M = _dense_wilson(dims, U, kappa)
    # the dense matrix is 1 - kappa D: its diagonal is exactly one
    assert np.allclose(np.diag(M), 1.0, atol=0, rtol=0)
    for site, comp in [(0, 0), (V - 1, 11), (3, 7)]:
        b = np.zeros((V, 4, 3), complex)
        b[site, comp // 3, comp % 3] = 1.0
        x, conv, iters = orc.wilson_solve(dims, U, kappa, b, tol=1e-13)
        assert conv and iters > 0
        xd = np.linalg.solve(M, b.reshape(-1)).reshape(V, 4, 3)
        assert np.max(np.abs(x - xd)) <= 1e-10 * np.max(np.abs(xd))
        assert np.linalg.norm(orc.wilson(dims, U, kappa, x) - b) <= 1e-11


def test_wilson_solve_free_field_momentum_space():
    """U = 1, periodic t: M is diagonal in momentum space with eigenvalues
    1 - kappa sum_mu (2 cos p_mu - 2 i gamma_mu sin p_mu) on each spin block."""
    dims = (4, 2, 2, 2)
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(3, dtype=complex), (V, 4, 3, 3)).copy()
    kappa = 0.11
    rng = np.random.default_rng(1)
    b = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    x, conv, _ = orc.wilson_solve(dims, U, kappa, b, tol=1e-13, t_bc=1)
    assert conv
    Lx, Ly, Lz, Lt = dims
    xs = x.reshape(Lt, Lz, Ly, Lx, 4, 3)
    bs = b.reshape(Lt, Lz, Ly, Lx, 4, 3)
    xf = np.fft.fftn(xs, axes=(0, 1, 2, 3))
    bf = np.fft.fftn(bs, axes=(0, 1, 2, 3))
    g = [orc.gamma(m) for m in range(4)]
    for it in range(Lt):
        for iz in range(Lz):
            for iy in range(Ly):
                for ix in range(Lx):
                    p = [2 * np.pi * ix / Lx, 2 * np.pi * iy / Ly, 2 * np.pi * iz / Lz, 2 * np.pi * it / Lt]
                    # psi(x + mu) -> e^{i p_mu} in the forward hop (1 - gamma), e^{-i p_mu} backward (1 + gamma)
                    D = sum((np.eye(4) - g[m]) * np.exp(1j * p[m]) + (np.eye(4) + g[m]) * np.exp(-1j * p[m])
                            for m in range(4))
                    Mp = np.eye(4) - kappa * D
                    lhs = Mp @ xf[it, iz, iy, ix]
                    assert np.allclose(lhs, bf[it, iz, iy, ix], atol=1e-9 * np.abs(bf).max())
