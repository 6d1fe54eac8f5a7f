"""Host logic of the slab CG (paper_2112_14640_gb300.domain.cg_normal) on CPU.

The slabs here are stand-ins with the interface of domain.SlabOperator whose
arithmetic is a few lines of torch on the host: a complex nearest-neighbour
operator along t, D = (m + 2) - a T+ - b T- (T+- shift by one time slice,
periodic), with ghost slices exchanged exactly as the GPU slabs exchange
theirs.  This checks, without a GPU, the parts of cg_normal that are host
code: the halo exchange order of apply_in_process for D and D^dag, the
owned-site reductions summed over the slabs, the per-RHS step lengths and the
convergence test.  The reference is numpy's dense solve of the whole-lattice
normal equations."""
import numpy as np
import pytest
import torch

from paper_2112_14640_gb300 import domain

A_HOP, B_HOP = 0.45 + 0.2j, 0.3 - 0.35j


class FakeOp:
    """The vector interface cg_normal uses: [t][site in slice][v] complex128."""

    def __init__(self, nt_local, slice_sites, nv):
        self.shape = (nt_local + 2, slice_sites, nv)
        self.nv = nv
        self.device = torch.device("cpu")
        self.slice_sites = slice_sites

    def new_vector(self):
        return torch.zeros(self.shape, dtype=torch.complex128)

    def axpby(self, a, x, b, y, z=None):
        r = a * x + b * y            # coefficients broadcast over the last (RHS) axis
        if z is None:
            return r
        z.copy_(r)
        return z

    def _rows(self, v, site0, nsites):
        flat = v.reshape(-1, self.nv)
        return flat[site0:site0 + nsites]

    def norm2_range(self, v, site0, nsites):
        return (self._rows(v, site0, nsites).abs() ** 2).sum(0)

    def dot_range(self, u, v, site0, nsites):
        return (self._rows(u, site0, nsites).conj() * self._rows(v, site0, nsites)).sum(0)


class FakeSlab:
    def __init__(self, world, rank, nt, slice_sites, nv):
        self.world, self.rank = world, rank
        self.t0, self.t1 = domain.slab_bounds(nt, world, rank)
        self.nt_local = self.t1 - self.t0
        self.slice_sites = slice_sites
        self.op = FakeOp(self.nt_local, slice_sites, nv)

    def pack(self, x, dagger=False):
        return x[1].clone(), x[self.nt_local].clone()

    def unpack(self, x, recv_lo, recv_hi, dagger=False):
        x[0] = recv_lo
        x[self.nt_local + 1] = recv_hi

    def apply_owned(self, x, out, m0, dagger=False):
        a, b = (np.conj(B_HOP), np.conj(A_HOP)) if dagger else (A_HOP, B_HOP)
        out[1:-1] = (m0 + 2.0) * x[1:-1] - a * x[2:] - b * x[:-2]
        return out


def dense_D(nt, slice_sites, m0):
    n = nt * slice_sites
    D = np.zeros((n, n), dtype=complex)
    for t in range(nt):
        for s in range(slice_sites):
            i = t * slice_sites + s
            D[i, i] = m0 + 2.0
            D[i, ((t + 1) % nt) * slice_sites + s] -= A_HOP
            D[i, ((t - 1) % nt) * slice_sites + s] -= B_HOP
    return D


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_slab_cg_host_logic_solves_the_whole_lattice(world):
    nt, slice_sites, nv, m0 = 12, 5, 3, 0.05
    rng = np.random.default_rng(7)
    b = rng.normal(size=(nt, slice_sites, nv)) + 1j * rng.normal(size=(nt, slice_sites, nv))
    slabs, bs = [], []
    for r in range(world):
        s = FakeSlab(world, r, nt, slice_sites, nv)
        v = s.op.new_vector()
        v[1:-1] = torch.from_numpy(b[s.t0:s.t1])
        v[0] = 7.0               # ghosts hold garbage: the exchange must overwrite them
        v[-1] = -3.0
        slabs.append(s)
        bs.append(v)
    xs, iters, relres = domain.cg_normal(slabs, bs, m0, tol=1e-12, maxit=500)
    assert np.all(relres < 1e-12) and 1 < iters < 500, (iters, relres)
    x = np.concatenate([xv[1:-1].numpy() for xv in xs], axis=0)
    D = dense_D(nt, slice_sites, m0)
    want = np.linalg.solve(D, b.reshape(nt * slice_sites, nv)).reshape(nt, slice_sites, nv)
    assert np.abs(x - want).max() <= 1e-9 * np.abs(want).max()
    # b is left as it was (its halos are exchanged in a copy)
    assert torch.equal(bs[0][0], torch.full_like(bs[0][0], 7.0))


def test_slab_cg_refuses_a_partial_set_of_slabs():
    slabs = [FakeSlab(3, r, 6, 2, 1) for r in range(2)]
    with pytest.raises(ValueError):
        domain.cg_normal(slabs, [s.op.new_vector() for s in slabs], 0.1)


def test_slab_cg_zero_rhs_returns_zero():
    slabs = [FakeSlab(2, r, 4, 3, 2) for r in range(2)]
    xs, iters, relres = domain.cg_normal(slabs, [s.op.new_vector() for s in slabs], 0.1)
    assert iters == 0 and np.all(relres == 0)
    assert all(torch.count_nonzero(x) == 0 for x in xs)
