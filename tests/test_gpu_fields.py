"""GPU parity: Philox streams, start configuration, refreshes, host transfer
and precision codecs, plaquette, kinetic energy, link update, reunitarize,
against the oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_1212_0785_gb300 import inputs, lqcd
from tests.gpu_util import PARITY_DIMS, half, rel_err, upload_gauge

pytestmark = pytest.mark.gpu


def test_philox_blocks_bit_exact():
    n = 5000
    out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    ctr, key = (7, 3, 1, 9), (12345, 6)
    lqcd.philox_blocks(out.data_ptr(), n, ctr, key)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    for i in list(range(64)) + list(range(n - 64, n)) + [1000, 2500]:
        assert np.array_equal(got[i], orc.philox4x32_10([ctr[0] + i, ctr[1], ctr[2], ctr[3]], key)), i
    # counter words wrap at 2^32 like the oracle's
    lqcd.philox_blocks(out.data_ptr(), 4, (0xFFFFFFFE, 0, 2, 0), (1, 2))
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    for i in range(4):
        assert np.array_equal(got[i], orc.philox4x32_10([(0xFFFFFFFE + i) & 0xFFFFFFFF, 0, 2, 0], (1, 2)))


def _df_codec_inputs():
    """doubles over the whole exponent range, with the cases the bit-level
    split must get right: exact floats, rounding ties both ways, carries out
    of the fraction, the edges of the range it handles itself, zeros,
    subnormals, Inf and NaN"""
    rng = np.random.default_rng(11)
    n = 200_000
    sign = rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63)
    expo = rng.integers(0, 2047, n, dtype=np.uint64) << np.uint64(52)
    frac = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    words = [sign | expo | frac]
    # exponents near the split's own range [-74, 126] and typical field values
    e = rng.integers(-80, 131, n).astype(np.uint64) + np.uint64(1023)
    words.append(sign | (e << np.uint64(52)) | frac)
    words.append(np.frombuffer(rng.standard_normal(n).astype(np.float64).tobytes(), dtype=np.uint64))
    # the 29 dropped bits: exactly half (ties to even both ways), zero, all ones
    kept = frac & ~np.uint64((1 << 29) - 1)
    for t in (1 << 28, 0, (1 << 29) - 1, (1 << 28) - 1, (1 << 28) + 1):
        words.append(sign | (e << np.uint64(52)) | kept | np.uint64(t))
    # all-ones fractions: rounding carries into the exponent
    words.append(sign | (e << np.uint64(52)) | np.uint64((1 << 52) - 1))
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1e-300, 1.7976931348623157e308,
                        np.inf, -np.inf, np.nan, 2.0 ** -74, 2.0 ** -75, -(2.0 ** 126), 2.0 ** 127, 2.0 ** 128,
                        1.0, -1.0, 1.0 + 2.0 ** -52, 3.4028235677973366e38, 1.401298464324817e-45])
    words.append(special.view(np.uint64))
    return np.concatenate(words).view(np.float64)


def test_float_float_codec_matches_ieee_rounding():
    d = _df_codec_inputs()
    with np.errstate(over="ignore", invalid="ignore"):
        hi = d.astype(np.float32)
        lo = (d - hi.astype(np.float64)).astype(np.float32)
        back = hi.astype(np.float64) + lo.astype(np.float64)
    din = torch.from_numpy(d.copy()).cuda()
    pairs = torch.empty(2 * d.size, dtype=torch.float32, device="cuda")
    got_back = torch.empty(d.size, dtype=torch.float64, device="cuda")
    lqcd.df_split(din.data_ptr(), d.size, pairs.data_ptr(), got_back.data_ptr())
    torch.cuda.synchronize()
    p = pairs.cpu().numpy().reshape(-1, 2)
    gb = got_back.cpu().numpy()
    for name, want, got in (("hi", hi, p[:, 0]), ("lo", lo, p[:, 1]), ("back", back, gb)):
        nan = np.isnan(want)
        assert np.array_equal(np.isnan(got), nan), name
        iw = want.view(np.uint32 if want.dtype == np.float32 else np.uint64)
        ig = got.view(iw.dtype)
        bad = np.flatnonzero((iw != ig) & ~nan)
        assert bad.size == 0, (name, d[bad[:5]], want[bad[:5]], got[bad[:5]])


@pytest.mark.parametrize("dims", PARITY_DIMS[:3])
def test_gauge_start_matches_oracle(dims):
    U = lqcd.gauge_field(dims)
    lqcd.gauge_start(U, seed=2, eps=0.2, chain=1)
    ref = orc.gauge_start(dims, seed=2, eps=0.2, chain=1)
    assert rel_err(U.download(), ref) < 1e-13


@pytest.mark.parametrize("dims", PARITY_DIMS[:3])
def test_refresh_matches_oracle(dims):
    P = lqcd.momentum_field(dims)
    lqcd.momentum_refresh(P, seed=3, traj=5, chain=2)
    assert np.max(np.abs(P.download() - orc.momentum_refresh(dims, 3, 5, chain=2))) < 1e-13
    eta = lqcd.spinor_field(dims, 0)
    lqcd.eta_refresh(eta, seed=3, traj=5, chain=2)
    ref = half(orc.eta_refresh(dims, 3, 5, chain=2), dims, 0)
    assert np.max(np.abs(eta.download() - ref)) < 1e-13


def test_transfer_roundtrip_and_codecs():
    dims = (6, 4, 2, 10)
    Uh = inputs.random_gauge(dims, 1)
    U = lqcd.gauge_field(dims).upload(Uh)
    assert np.array_equal(U.download(), Uh)
    for prec, tol in ((lqcd.F32, 1e-6), (lqcd.F16N, 2e-3), (lqcd.BF16, 1.6e-2)):
        Us = lqcd.gauge_field(dims, prec).copy_from(U)
        assert rel_err(Us.download(), Uh) < tol, prec  # row 2 reconstructed from rows 0, 1
    P = inputs.random_momentum(dims, 2)
    assert np.array_equal(lqcd.momentum_field(dims).upload(P).download(), P)
    s = inputs.random_spinor(dims, 3)
    for par in (0, 1):
        h = half(s, dims, par)
        f = lqcd.spinor_field(dims, par).upload(h)
        assert np.array_equal(f.download(), h)
        for prec, tol in ((lqcd.F32, 1e-6), (lqcd.F16N, 1e-3), (lqcd.BF16, 8e-3)):
            g = lqcd.spinor_field(dims, par, prec).copy_from(f)
            assert rel_err(g.download(), h) < tol
    full = lqcd.Field(dims, lqcd.SPINOR_FULL).upload(s)
    assert np.array_equal(full.download(), s)


def _pinned_like(a):
    """a page-locked host array with a's contents"""
    t = torch.empty(a.size * a.itemsize // 8, dtype=torch.float64, pin_memory=True)
    out = t.numpy().view(a.dtype).reshape(a.shape)
    out[...] = a
    return out, t


@pytest.mark.parametrize("dims", [(6, 6, 2, 2), (4, 4, 4, 4), (2, 2, 2, 2)])
def test_pinned_and_pageable_transfers_agree(dims):
    """pinned host arrays are converted in place by the kernel, pageable ones
    through a device buffer: both give bitwise the same fields and arrays
    (4V = 576 links: a ragged last block of 128; 1024: whole blocks; 64: one
    partial block)"""
    Uh = inputs.random_gauge(dims, 31)
    pin, keep = _pinned_like(Uh)
    assert keep.is_pinned()
    for prec in (lqcd.F64, lqcd.F32, lqcd.F16N, lqcd.BF16):
        a = lqcd.gauge_field(dims, prec).upload(Uh)
        b = lqcd.gauge_field(dims, prec).upload(pin)
        down_a = a.download()
        out, keep2 = _pinned_like(np.zeros_like(Uh))
        b.download(out=out)
        assert np.array_equal(down_a, out), prec
        if prec == lqcd.F64:
            assert np.array_equal(down_a, Uh)
    P = inputs.random_momentum(dims, 32)
    ppin, keep3 = _pinned_like(P)
    m = lqcd.momentum_field(dims).upload(ppin)
    assert np.array_equal(m.download(), P)
    s = half(inputs.random_spinor(dims, 33, parity=1), dims, 1)
    spin, keep4 = _pinned_like(s)
    f = lqcd.spinor_field(dims, 1).upload(spin)
    back, keep5 = _pinned_like(np.zeros_like(s))
    f.download(out=back)
    assert np.array_equal(back, s)


@pytest.mark.parametrize("dims", PARITY_DIMS)
def test_plaquette_and_kinetic(dims):
    Uh = orc.gauge_start(dims, seed=4, eps=0.4)
    U = lqcd.gauge_field(dims).upload(Uh)
    assert abs(lqcd.plaquette(U) - orc.plaquette(dims, Uh)) < 1e-14
    Ph = inputs.random_momentum(dims, 5)
    P = lqcd.momentum_field(dims).upload(Ph)
    assert abs(lqcd.kinetic_energy(P) - orc.kinetic(dims, Ph)) < 1e-12 * orc.kinetic(dims, Ph)


@pytest.mark.parametrize("dims", PARITY_DIMS[:3])
def test_link_update_matches_oracle(dims):
    Uh = orc.gauge_start(dims, seed=6, eps=0.3)
    Ph = orc.momentum_refresh(dims, 6, 0)
    U = lqcd.gauge_field(dims).upload(Uh)
    P = lqcd.momentum_field(dims).upload(Ph)
    Us = lqcd.gauge_field(dims, lqcd.F16N)
    lqcd.link_update(U, P, 0.07, U_sloppy=Us)
    ref = orc.link_update(dims, Uh, Ph, 0.07)
    assert rel_err(U.download(), ref) < 1e-13
    assert rel_err(Us.download(), ref) < 2e-3
    # large steps take the Cayley-Hamilton exp through all its branches
    for c in (1.5, -2.0, 1e-9):
        U = lqcd.gauge_field(dims).upload(Uh)
        lqcd.link_update(U, P, c)
        assert rel_err(U.download(), orc.link_update(dims, Uh, Ph, c)) < 1e-12, c


@pytest.mark.parametrize("c", [0.07, 1.5, -0.3])
def test_fp32_link_update_close_and_unitary(c):
    """the FP32 molecular dynamics' update: within the FP32 exponential's
    error of the oracle, special unitary to float-float precision"""
    dims = (6, 4, 2, 10)
    Uh = orc.gauge_start(dims, seed=16, eps=0.3)
    Ph = orc.momentum_refresh(dims, 16, 0)
    U = lqcd.gauge_field(dims).upload(Uh)
    P = lqcd.momentum_field(dims).upload(Ph)
    Us = lqcd.gauge_field(dims, lqcd.F16N)
    lqcd.link_update(U, P, c, U_sloppy=Us, arith=lqcd.F32)
    got = U.download()
    assert rel_err(got, orc.link_update(dims, Uh, Ph, c)) < 2e-6
    dev = np.abs(np.einsum("xmab,xmcb->xmac", got, got.conj()) - np.eye(3)).max()
    assert dev < 1e-13 and np.abs(np.linalg.det(got) - 1).max() < 1e-13
    assert rel_err(Us.download(), got) < 2e-3
    with pytest.raises(lqcd.LqcdError):
        lqcd.link_update(U, P, c, arith=lqcd.F16N)


def test_link_update_degenerate_momenta():
    """momenta with degenerate eigenvalues (single diagonal generators) and zero"""
    dims = (4, 4, 4, 4)
    V = 256
    Uh = orc.gauge_start(dims, seed=7, eps=0.3)
    Ph = np.zeros((V, 4, 8))
    Ph[:, 0, 7] = 1.3   # lambda_8: eigenvalues (a, a, -2a)
    Ph[:, 1, 2] = -0.8  # lambda_3: (a, -a, 0)
    Ph[:, 2, 0] = 2.0   # lambda_1
    U = lqcd.gauge_field(dims).upload(Uh)
    P = lqcd.momentum_field(dims).upload(Ph)
    lqcd.link_update(U, P, 0.5)
    assert rel_err(U.download(), orc.link_update(dims, Uh, Ph, 0.5)) < 1e-13


def test_reunitarize_matches_oracle():
    dims = (6, 4, 2, 10)
    Uh = orc.gauge_start(dims, seed=8, eps=0.3)
    rng = np.random.default_rng(0)
    noisy = Uh + 1e-4 * (rng.standard_normal(Uh.shape) + 1j * rng.standard_normal(Uh.shape))
    U = lqcd.gauge_field(dims).upload(noisy)
    dev = lqcd.reunitarize(U)
    ref, ref_dev = orc.reunitarize(dims, noisy)
    assert abs(dev - ref_dev) < 1e-12
    assert rel_err(U.download(), ref) < 1e-14
