"""Batched, graph-captured solves (dirac_solve_batched) against the oracle:
every solution of a mixed batch (kinds, lattices, N_v) is checked by the FP64
oracle applying D^dag D to it, and a solve that starts converged finishes at
set-up."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import to_device, to_numpy
from paper_2112_14640_gb300 import dirac as D
from paper_2112_14640_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SPECS = [  # kind, dims, nv, m0
    (D.WILSON, (4, 4, 4, 4), 1, 0.2),
    (D.STAGGERED, (4, 4, 4, 8), 3, 0.1),
    (D.WILSON, (6, 4, 2, 8), 5, 0.3),
    (D.STAGGERED, (8, 8, 4, 4), 12, 0.2),
    (D.BRILLOUIN, (4, 4, 2, 4), 2, 0.2),
    (D.WILSON, (8, 4, 4, 4), 12, 0.15),
]


@pytest.mark.parametrize("prec,tol", [(D.F64, 1e-10), (D.F32, 1e-5)])
def test_batched_solves_match_oracle(prec, tol):
    ops, refs, bs, bn = [], [], [], []
    for i, (kind, dims, nv, m0) in enumerate(SPECS):
        U = I.gauge_field(dims, 3, 0.4, 300 + i)
        ops.append(D.DiracOp(kind, torch.from_numpy(U).cuda(), nv, (1, 1, 1, -1), prec, layout=i % 2))
        refs.append(O.Operator(kind, U, (1, 1, 1, -1)))
        b = I.source(dims, 3, nv, 400 + i, staggered=(kind == D.STAGGERED))
        bn.append(b)
        bs.append(to_device(ops[-1], b))
    m0s = [s[3] for s in SPECS]
    xs, stats, rc = D.solve_batched(ops, bs, m0s=m0s, solver=D.CG_NORMAL, tol=tol, maxit=20000)
    assert rc == 0
    for i, (op, ref, b, st) in enumerate(zip(ops, refs, bn, stats)):
        assert st["status"] == 0 and st["iters"] > 0 and st["seconds"] > 0, (i, st)
        # the whole convergence loop ran as one graph launch (device-side while node)
        assert st["host_launches"] == 1, st
        xsn = to_numpy(op, xs[i])
        bN = ref.apply_dagger(b, m0s[i])
        res = np.sqrt(O.norm2(bN - ref.apply_normal(xsn, m0s[i])) / O.norm2(bN))
        assert np.all(res < 1.05 * tol if prec == D.F64 else 5 * tol), (i, res)
        op.close()


def test_batched_solve_already_converged_and_hpd():
    kind, dims, nv, m0 = D.STAGGERED, (4, 4, 4, 4), 2, 0.2
    U = I.gauge_field(dims, 3, 0.4, 7)
    opA = D.DiracOp(kind, torch.from_numpy(U).cuda(), nv, (1, 1, 1, 1), D.F64)
    opB = D.DiracOp(kind, torch.from_numpy(U).cuda(), nv, (1, 1, 1, 1), D.F64)
    b = to_device(opA, I.source(dims, 3, nv, 8, staggered=True))
    x0, st0 = opA.solve(b, m0=m0, solver=D.CG_HPD, tol=1e-12, maxit=5000)
    xs, stats, rc = D.solve_batched([opA, opB], [b, b.clone()], xs=[x0.clone(), opB.new_vector()], m0s=[m0, m0],
                                    solver=D.CG_HPD, tol=1e-10, maxit=5000)
    assert rc == 0
    assert stats[0]["iters"] == 0          # converged at set-up
    assert stats[0]["host_launches"] == 1
    assert stats[1]["iters"] > 0
    assert torch.allclose(xs[1], x0, rtol=0, atol=1e-8 * x0.abs().max().item())
