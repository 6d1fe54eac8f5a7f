"""Bounds of every write: each output buffer sits between guard regions
filled with a sentinel, and after the call the guards must be untouched
(stencils with odd N_v and both layouts, daggers, D^dag D, the site-range
apply, the halo pack and unpack, a solve's solution, the force).  Also a
host-side fault the solvers must survive without a GPU fault: a NaN in one
right-hand side ends the solve with DIRAC_NONFINITE and leaves the operator
usable (maxit = 1 and zero right-hand sides are in test_gpu_solvers)."""
import numpy as np
import pytest
import torch

from helpers import to_device
from paper_2112_14640_gb300 import dirac as D
from paper_2112_14640_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GUARD = 256          # elements before and after each output
SENTINEL = 12345.0 - 6789.0j


def make(kind, dims, nc, nv, bc, prec, layout=D.SITE_OUTER, seed=11):
    U = torch.from_numpy(I.gauge_field(dims, nc, 0.4, seed)).cuda()
    op = D.DiracOp(kind, U, nv, bc, prec, layout=layout)
    return op, I.source(dims, nc, nv, seed + 1, staggered=(kind == D.STAGGERED))


def guarded(shape, dtype):
    n = int(np.prod(shape))
    big = torch.full((n + 2 * GUARD,), SENTINEL, dtype=dtype, device="cuda")
    return big, big[GUARD:GUARD + n].view(shape)


def guards_intact(big):
    torch.cuda.synchronize()
    want = torch.full((GUARD,), SENTINEL, dtype=big.dtype, device=big.device)
    return torch.equal(big[:GUARD], want) and torch.equal(big[-GUARD:], want)


@pytest.mark.parametrize("layout", [D.SITE_OUTER, D.SITE_INNER])
@pytest.mark.parametrize("prec", [D.F64, D.F32])
@pytest.mark.parametrize("kind", [D.WILSON, D.BRILLOUIN, D.STAGGERED])
def test_outputs_stay_inside_their_buffers(kind, prec, layout):
    dims, nc, nv = (4, 2, 4, 6), 3, 5
    m0 = 0.05 if kind == D.STAGGERED else 0.1
    op, src = make(kind, dims, nc, nv, (1, -1, 1, -1), prec, layout=layout)
    x = to_device(op, src)
    shape, dtype = tuple(op.vector_shape()), x.dtype
    for call in ("apply", "dagger", "normal", "range"):
        big, out = guarded(shape, dtype)
        if call == "apply":
            op.apply(x, out, m0=m0)
        elif call == "dagger":
            op.apply(x, out, m0=m0, dagger=True)
        elif call == "normal":
            op.apply_normal(x, out, m0=m0)
        else:
            op.apply_range(x, out, 4 * 2 * 4, 3 * 4 * 2 * 4, m0=m0)
        assert guards_intact(big), call
    # halo slices of the first and the last time slice, packed and unpacked
    for proj in ((0, 1, -1) if kind != D.STAGGERED else (0,)):
        nb = int(D.lib().dirac_halo_bytes(op._h, proj))
        for t in (0, dims[3] - 1):
            bigb = torch.full((nb + 2 * GUARD,), 0xA5, dtype=torch.uint8, device="cuda")
            buf = bigb[GUARD:GUARD + nb]
            op.halo_pack(x, t, buf, proj)
            torch.cuda.synchronize()
            assert torch.all(bigb[:GUARD] == 0xA5) and torch.all(bigb[-GUARD:] == 0xA5), (proj, t)
            big, v = guarded(shape, dtype)
            v.zero_()
            op.halo_unpack(buf, t, v, proj)
            assert guards_intact(big), (proj, t)
    # a solve's solution vector
    big, xs = guarded(shape, dtype)
    xs.zero_()
    solver = D.BICGSTAB if kind == D.BRILLOUIN else D.CG_NORMAL
    op.solve(x, x=xs, m0=0.3, tol=1e-4, maxit=200, solver=solver)
    assert guards_intact(big), "solve"
    # the force of the pseudofermion action
    fshape = (dims[3], dims[2], dims[1], dims[0], 4, nc, nc)
    big, f = guarded(fshape, dtype)
    rc = D.lib().dirac_force(op._h, x.data_ptr(), x.data_ptr(), f.data_ptr(), 0, None)
    assert rc == 0 and guards_intact(big), "force"
    op.close()


@pytest.mark.parametrize("kind", [D.WILSON, D.STAGGERED])
def test_nan_in_one_rhs_ends_the_solve_nonfinite(kind):
    op, src = make(kind, (4, 4, 4, 4), 3, 3, (1, 1, 1, 1), D.F64)
    b = to_device(op, src)
    b[..., 1] = float("nan")
    x, st = op.solve(b, m0=0.1, tol=1e-10, maxit=500)
    assert st["status"] == 4 and st["iters"] <= 2, st        # DIRAC_NONFINITE
    # the operator stays usable afterwards
    x, st = op.solve(to_device(op, src), m0=0.1, tol=1e-10, maxit=5000)
    assert st["status"] == 0
    op.close()
