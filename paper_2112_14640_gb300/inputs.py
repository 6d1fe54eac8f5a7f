"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the method's arithmetic: it only draws random
numbers and shapes them into gauge fields and source vectors.

* Links: U_mu(n) = exp(i * eps * sum_k a_k lambda_k), a_k ~ N(0,1), with the
  generalized Gell-Mann matrices (Tr lambda_a lambda_b = 2 delta_ab), i.e. a
  random SU(Nc) element per link whose roughness grows with eps.  The
  exponential goes through a Hermitian eigendecomposition, so U is unitary
  with det 1 to rounding.  Layout (Nt, Nz, Ny, Nx, 4, Nc, Nc), complex128.
* Sources: Re and Im independently N(0,1).
  Wilson-type (Nt, Nz, Ny, Nx, Nc, 4, Nv), staggered (Nt, Nz, Ny, Nx, Nc, Nv).

All generators use numpy's PCG64 with an explicit seed, so the same call
gives the same numbers on any machine.
"""
import numpy as np


def gell_mann(nc):
    """Generalized Gell-Mann basis of su(nc): (nc^2-1, nc, nc), Tr(l_a l_b) = 2 delta_ab."""
    mats = []
    for j in range(nc):
        for k in range(j + 1, nc):
            s = np.zeros((nc, nc), np.complex128)
            s[j, k] = s[k, j] = 1.0
            mats.append(s)
            a = np.zeros((nc, nc), np.complex128)
            a[j, k] = -1j
            a[k, j] = 1j
            mats.append(a)
    for l in range(1, nc):
        dg = np.zeros((nc, nc), np.complex128)
        for j in range(l):
            dg[j, j] = 1.0
        dg[l, l] = -l
        mats.append(dg * np.sqrt(2.0 / (l * (l + 1))))
    return np.array(mats)


def _expi_hermitian(H, eps):
    w, v = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ij,...j,...kj->...ik", v, ph, v.conj())


def random_su_n(shape, nc, eps, rng):
    """Array of random SU(nc) matrices of the given leading shape.  For nc = 1
    (no su(1) generators) the links are U(1) phases exp(i eps a), a ~ N(0,1)."""
    if nc == 1:
        a = rng.standard_normal(tuple(shape))
        return np.exp(1j * eps * a)[..., None, None]
    gm = gell_mann(nc)
    out = np.empty(tuple(shape) + (nc, nc), np.complex128)
    flat = out.reshape(-1, nc, nc)
    n = flat.shape[0]
    chunk = 1 << 18
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        a = rng.standard_normal((e - s, gm.shape[0]))
        H = np.tensordot(a, gm, axes=(1, 0))
        flat[s:e] = _expi_hermitian(H, eps)
    return out


def gauge_field(dims, nc=3, eps=0.4, seed=1234):
    """Random SU(nc) links for a lattice dims = (Nx, Ny, Nz, Nt)."""
    nx, ny, nz, nt = dims
    rng = np.random.Generator(np.random.PCG64(seed))
    return random_su_n((nt, nz, ny, nx, 4), nc, eps, rng)


def unit_gauge_field(dims, nc=3):
    """Free field U = 1."""
    nx, ny, nz, nt = dims
    U = np.zeros((nt, nz, ny, nx, 4, nc, nc), np.complex128)
    U[..., :, :] = np.eye(nc)
    return U


def gauge_transform(dims, nc=3, seed=99):
    """Random site-local SU(nc) matrices Omega(n), shape (Nt, Nz, Ny, Nx, Nc, Nc)."""
    nx, ny, nz, nt = dims
    rng = np.random.Generator(np.random.PCG64(seed))
    return random_su_n((nt, nz, ny, nx), nc, 1.0, rng)


def source(dims, nc=3, nv=12, seed=4321, staggered=False):
    """Gaussian complex multi-RHS source vector."""
    nx, ny, nz, nt = dims
    shape = (nt, nz, ny, nx, nc, nv) if staggered else (nt, nz, ny, nx, nc, 4, nv)
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im


def su_n_direction(dims, nc=3, seed=7):
    """Random su(nc) field X_mu(n) = i sum_k a_k lambda_k (traceless anti-Hermitian),
    shape (Nt, Nz, Ny, Nx, 4, Nc, Nc); used as finite-difference directions."""
    nx, ny, nz, nt = dims
    rng = np.random.Generator(np.random.PCG64(seed))
    gm = gell_mann(nc)
    a = rng.standard_normal((nt, nz, ny, nx, 4, gm.shape[0]))
    return 1j * np.tensordot(a, gm, axes=(-1, 0))
