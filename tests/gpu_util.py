"""Helpers for the GPU parity tests: layout conversion between the oracle's
full-lattice arrays and the library's checkerboard half fields, and error
measures."""
import numpy as np

from oracle import oracle as orc
from paper_1212_0785_gb300 import lqcd


def half(full, dims, parity):
    """full-lattice (V,4,3) -> the sites of one parity in checkerboard order"""
    return np.ascontiguousarray(full[orc.parity(dims) == parity])


def full_from_half(h, dims, parity):
    out = np.zeros((int(np.prod(dims)), 4, 3), np.complex128)
    out[orc.parity(dims) == parity] = h
    return out


def rel_err(a, b):
    """max |a - b| / max |b|"""
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def upload_gauge(U_host, dims, prec=lqcd.F64):
    U = lqcd.gauge_field(dims, lqcd.F64)
    U.upload(U_host)
    if prec == lqcd.F64:
        return U
    Us = lqcd.gauge_field(dims, prec)
    Us.copy_from(U)
    return U, Us


def upload_half(full, dims, parity, prec=lqcd.F64):
    f = lqcd.spinor_field(dims, parity, prec)
    f.upload(half(full, dims, parity))
    return f


# lattices for parity tests: several thread blocks and a ragged tail
# (V/2 = 128, 240, 1728, 2160 against 128-thread blocks)
PARITY_DIMS = [(4, 4, 4, 4), (6, 4, 2, 10), (8, 6, 6, 12), (6, 6, 10, 12)]
