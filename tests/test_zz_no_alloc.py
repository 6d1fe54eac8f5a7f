"""The allocation-free norm entry point, dirac_vec_norm2_noalloc.

It exists for callers that must not allocate device memory (all device
memory owned by a pooling allocator they must not bypass, loops that cannot
afford the device synchronisation an allocation may cause, programs at the
memory limit); its partial sums live in a fixed device array in the library.
Its results are checked against the allocating entry point and against the
oracle's norms of the same (rounded) inputs.  This
file is collected last so that a failure here never hides the other tests,
and it passes both alone in a fresh process and after the whole suite.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from helpers import rounded
from paper_2112_14640_gb300 import dirac as D
from paper_2112_14640_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _noalloc(v, prec, rows, nv, out):
    lib = D.lib()
    return lib.dirac_vec_norm2_noalloc(ctypes.c_void_p(v.data_ptr()), prec, rows, nv,
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _case(dims, nv, prec, seed):
    U = torch.from_numpy(I.gauge_field(dims, 3, 0.4, seed)).cuda()
    op = D.DiracOp(D.WILSON, U, nv, (1, 1, 1, -1), prec)
    src = I.source(dims, 3, nv, seed + 1)
    x = op.to_prec(torch.from_numpy(src).cuda())
    rows = int(np.prod(dims)) * 3 * 4
    return op, x, rows, O.norm2(rounded(src, prec))


def test_noalloc_norm_matches_the_allocating_entry_point_twice():
    # call 1: a large vector (the grid fills every slot of the static array)
    op1, x1, rows1, oracle1 = _case((16, 16, 16, 32), 12, D.F32, 3)
    out1 = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(x1, D.F32, rows1, 12, out1) == 0
    want1 = op1.norm2(x1)
    # call 2, straight after: a small vector in another precision, few blocks,
    # so stale partial sums of call 1 would show up if they were read
    op2, x2, rows2, oracle2 = _case((4, 4, 4, 4), 5, D.F64, 8)
    out2 = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(x2, D.F64, rows2, 5, out2) == 0
    want2 = op2.norm2(x2)
    torch.cuda.synchronize()
    assert torch.allclose(out1, want1, rtol=1e-12, atol=0)
    assert torch.allclose(out2, want2, rtol=1e-12, atol=0)
    assert np.allclose(out1.cpu().numpy(), oracle1, rtol=1e-12, atol=0)
    assert np.allclose(out2.cpu().numpy(), oracle2, rtol=1e-12, atol=0)
    op1.close()
    op2.close()


def test_noalloc_norm_rejects_sizes_beyond_its_capacity():
    op, x, rows, _ = _case((4, 4, 4, 4), 4, D.F32, 5)
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    assert _noalloc(x, D.F32, rows, 65, out) == -8        # nv above the static capacity of 64
    assert _noalloc(x, D.F32, rows, 0, out) == -1         # no right-hand side
    assert _noalloc(x, D.F32, 0, 4, out) == -1            # empty vector
    assert "static capacity" in D.error_string(-8)
    op.close()
