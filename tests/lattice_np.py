"""Plain numpy lattice helpers for the tests (shifts, plane waves, dense
operators).  Test-side geometry only: neither the oracle nor the library use it."""
import numpy as np


def shape4(dims):
    Lx, Ly, Lz, Lt = dims
    return (Lt, Lz, Ly, Lx)


_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}  # mu -> numpy axis of the (t, z, y, x) shaped array


def shift(field, dims, mu, sign):
    """field(x + sign*mu) as a lexicographic array (periodic; no boundary phase)"""
    f = field.reshape(shape4(dims) + field.shape[1:])
    return np.roll(f, -sign, axis=_AXIS[mu]).reshape(field.shape)


def coords(dims):
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return [c.reshape(-1) for c in (x, y, z, t)]


def gauge_transform(U, Om, dims):
    """U_mu(x) -> Om(x) U_mu(x) Om(x+mu)^dag"""
    Up = np.empty_like(U)
    for mu in range(4):
        Omf = shift(Om, dims, mu, +1)
        Up[:, mu] = Om @ U[:, mu] @ np.conj(np.swapaxes(Omf, -1, -2))
    return Up


def dense_operator(apply, n_in, in_shape, out_index=None):
    """Dense matrix of a linear map given as a python callable on complex arrays."""
    cols = []
    for k in range(n_in):
        e = np.zeros(n_in, np.complex128)
        e[k] = 1
        cols.append(apply(e.reshape(in_shape)).reshape(-1))
    M = np.array(cols).T
    if out_index is not None:
        M = M[out_index]
    return M
