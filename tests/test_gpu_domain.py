"""Slab decomposition along t on one GPU (paper_2112_14640_gb300.domain): the
lattice is cut into 1, 2 or 4 slabs, each held by its own slab operator with
one ghost slice per side; the ghost slices start zeroed, are filled by
packing, exchanging (device copies between the slabs) and unpacking the edge
slices -- half spinors for D_W -- and each slab applies D on its owned
slices.  The owned slices put together must equal the oracle's D on the
whole lattice, for D_W, D_B, D_S, their daggers, FP64 and FP32."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import check, to_numpy
from paper_2112_14640_gb300 import dirac as D
from paper_2112_14640_gb300 import domain
from paper_2112_14640_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("prec", [D.F64, D.F32])
@pytest.mark.parametrize("world", [1, 2, 4])
@pytest.mark.parametrize("kind", [D.WILSON, D.BRILLOUIN, D.STAGGERED])
def test_slabs_match_the_whole_lattice(kind, world, prec, dagger):
    dims, nc, nv, bc = (4, 2, 4, 8), 3, 3, (1, -1, 1, -1)
    m0 = 0.05 if kind == D.STAGGERED else 0.1
    U = I.gauge_field(dims, nc, 0.4, 61)
    src = I.source(dims, nc, nv, 62, staggered=(kind == D.STAGGERED))
    ref = O.Operator(kind, U, bc)
    want = ref.apply_dagger(src, m0) if dagger else ref.apply(src, m0)
    slabs, xs, outs = [], [], []
    for r in range(world):
        s = domain.SlabOperator(kind, U, nv, bc, prec, world, r)
        v = domain.slab_vector(src, world, r)
        v[0] = 0
        v[-1] = 0                                   # ghosts must come from the exchange
        xs.append(s.op.to_prec(s.op.from_site_outer(torch.from_numpy(v).cuda())))
        outs.append(s.op.new_vector())
        slabs.append(s)
    domain.apply_in_process(slabs, xs, outs, m0, dagger)
    got = np.concatenate([to_numpy(s.op, o)[1:-1] for s, o in zip(slabs, outs)], axis=0)
    check(got, want, prec, kind, world, dagger)
    for s in slabs:
        s.close()


def test_wilson_halo_is_half_a_slice():
    """The D_W halo travels as half spinors: half the bytes of a full slice;
    the other kinds send full slices."""
    dims, nc, nv = (4, 4, 2, 4), 3, 5
    U = I.gauge_field(dims, nc, 0.4, 63)
    s = domain.SlabOperator(D.WILSON, U, nv, (1, 1, 1, -1), D.F32, 2, 0)
    full = D.lib().dirac_halo_bytes(s.op._h, 0)
    assert full == (4 * 4 * 2) * 3 * 4 * nv * 8     # slice sites x colours x spins x RHS x complex FP32
    assert D.lib().dirac_halo_bytes(s.op._h, 1) == full // 2 == D.lib().dirac_halo_bytes(s.op._h, -1)
    lo, hi = s.pack(s.op.new_vector())
    assert lo.numel() == full // 2 and hi.numel() == full // 2
    s.close()
    st = domain.SlabOperator(D.STAGGERED, U, nv, (1, 1, 1, -1), D.F32, 2, 0)
    assert D.lib().dirac_halo_bytes(st.op._h, 1) == 0          # half spinors: Wilson-type vectors only
    lo, hi = st.pack(st.op.new_vector())
    assert lo.numel() == (4 * 4 * 2) * 3 * nv * 8
    st.close()


def test_apply_range_leaves_other_sites_untouched():
    dims, nc, nv = (4, 4, 4, 4), 3, 2
    U = torch.from_numpy(I.gauge_field(dims, nc, 0.4, 64)).cuda()
    op = D.DiracOp(D.WILSON, U, nv, (1, 1, 1, -1), D.F32, layout=D.SITE_INNER)
    x = op.new_vector()
    x.real.normal_()
    full = op.apply(x, m0=0.1)
    out = torch.full_like(full, 7.0)
    slice_sites = 4 * 4 * 4
    op.apply_range(x, out, slice_sites, 2 * slice_sites, m0=0.1)
    o, f = to_numpy(op, out), to_numpy(op, full)
    assert np.array_equal(o[1:3], f[1:3])
    assert np.all(o[0] == 7.0) and np.all(o[3] == 7.0)
    op.close()


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("kind", [D.WILSON, D.BRILLOUIN, D.STAGGERED])
def test_cg_over_slabs_matches_the_whole_lattice(kind, world):
    """CG on D^dag D over slabs (halo exchange per apply, dot products over
    the owned sites summed over the slabs): the solution assembled from the
    owned slices solves the whole-lattice normal equations (oracle residual)
    and agrees with the library's single-operator CG."""
    dims, nc, nv, bc = (4, 2, 4, 8), 3, 2, (1, -1, 1, -1)
    m0 = 0.2
    U = I.gauge_field(dims, nc, 0.4, 71)
    src = I.source(dims, nc, nv, 72, staggered=(kind == D.STAGGERED))
    slabs, bs = [], []
    for r in range(world):
        s = domain.SlabOperator(kind, U, nv, bc, D.F64, world, r)
        bs.append(s.op.from_site_outer(torch.from_numpy(domain.slab_vector(src, world, r)).cuda()))
        slabs.append(s)
    xs, iters, relres = domain.cg_normal(slabs, bs, m0, tol=1e-10, maxit=5000)
    assert np.all(relres < 1e-10) and iters > 5, (iters, relres)
    x = np.concatenate([to_numpy(s.op, xv)[1:-1] for s, xv in zip(slabs, xs)], axis=0)
    ref = O.Operator(kind, U, bc)
    bN = ref.apply_dagger(src, m0)
    res = np.sqrt(O.norm2(bN - ref.apply_normal(x, m0)) / O.norm2(bN))
    assert np.all(res < 2e-10), res
    # the same system solved by the library on the whole lattice
    op = D.DiracOp(kind, torch.from_numpy(U).cuda(), nv, bc, D.F64)
    xw, st = op.solve(op.from_site_outer(torch.from_numpy(src).cuda()), m0=m0, tol=1e-12, maxit=5000)
    want = to_numpy(op, xw)
    assert np.linalg.norm(x - want) <= 1e-8 * np.linalg.norm(want)
    op.close()
    for s in slabs:
        s.close()


def test_range_reductions_cover_exactly_the_owned_sites():
    """dirac_vec_norm2_range / dot_range over a site range equal the full
    reductions of vectors that are zero outside the range, for both layouts;
    invalid ranges are refused."""
    dims, nc, nv = (4, 4, 2, 6), 3, 3
    U = torch.from_numpy(I.gauge_field(dims, nc, 0.4, 73)).cuda()
    for layout in (D.SITE_OUTER, D.SITE_INNER):
        op = D.DiracOp(D.WILSON, U, nv, (1, 1, 1, 1), D.F64, layout=layout)
        x, y = op.new_vector(), op.new_vector()
        x.real.normal_()
        x.imag.normal_()
        y.real.normal_()
        slice_sites = 4 * 4 * 2
        s0, n = slice_sites, 3 * slice_sites
        mask = np.zeros(dims[::-1], dtype=bool)
        mask[1:4] = True
        xm, ym = to_numpy(op, x), to_numpy(op, y)
        keep = mask.reshape(mask.shape + (1,) * (xm.ndim - mask.ndim))
        want_n = np.sum(np.abs(np.where(keep, xm, 0)) ** 2, axis=tuple(range(xm.ndim - 1)))
        want_d = np.sum(np.conj(np.where(keep, xm, 0)) * ym, axis=tuple(range(xm.ndim - 1)))
        assert np.allclose(op.norm2_range(x, s0, n).cpu().numpy(), want_n, rtol=1e-12)
        assert np.allclose(op.dot_range(x, y, s0, n).cpu().numpy(), want_d, rtol=1e-12)
        full = op.norm2_range(x, 0, int(np.prod(dims)))
        assert torch.allclose(full, op.norm2(x), rtol=1e-13)
        for bad in ((-1, 4), (0, 0), (int(np.prod(dims)) - 3, 4)):
            with pytest.raises(D.DiracError):
                op.norm2_range(x, *bad)
        op.close()
