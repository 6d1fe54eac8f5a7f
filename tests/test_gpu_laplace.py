"""GPU parity of the Laplace operators A = -1/2 Lap + m^2/2 (Eqs. app_wlap,
app_blap; the paper's wlap, blap, wsuv, bsuv) through the C ABI against the
FP64 oracle: A element by element for all four kinds, both layouts, F64 and
F32, ragged shapes; every launch variant; the 16^3 x 32, N_v = 12 workload on
sampled sites; the host apply; CG on A x = b (plain, mixed F64/F32,
batched) and BiCGstab, every solution checked by the oracle's A; and the
argument rules (no CG on the normal equations, no 16-bit storage, no
clover term).

Tolerances as in test_gpu_parity: relative L2 1e-12 FP64, 1e-5 FP32.
"""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import TOL, check, rel_l2, to_device, to_numpy
from paper_2112_14640_gb300 import dirac as D
from paper_2112_14640_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LAYOUTS = [D.SITE_OUTER, D.SITE_INNER]
KINDS = [D.WLAP, D.BLAP, D.WSUV, D.BSUV]


def colour_only(kind):
    return kind in (D.WSUV, D.BSUV)


def make(kind, dims, nc, nv, bc, prec, seed=5, layout=D.SITE_OUTER):
    U = I.gauge_field(dims, nc, 0.4, seed)
    op = D.DiracOp(kind, torch.from_numpy(U).cuda(), nv, bc, prec, layout=layout)
    ref = O.Operator(kind, U, bc)
    src = I.source(dims, nc, nv, seed + 1, staggered=colour_only(kind))
    return op, ref, src


CASES = [
    # dims, nc, nv, bc
    ((4, 4, 4, 4), 3, 1, (1, 1, 1, -1)),
    ((8, 8, 8, 8), 3, 12, (1, 1, 1, -1)),
    ((6, 4, 2, 8), 3, 3, (1, -1, 1, -1)),
    ((4, 6, 4, 2), 2, 4, (1, 1, 1, 1)),
    ((2, 4, 4, 6), 4, 5, (-1, 1, 1, -1)),
    ((5, 3, 2, 4), 1, 8, (1, 1, 1, -1)),
]


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", [D.F64, D.F32])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_laplace_apply(kind, prec, case, layout):
    dims, nc, nv, bc = CASES[case]
    m = 0.3
    op, ref, src = make(kind, dims, nc, nv, bc, prec, layout=layout)
    x = to_device(op, src)
    want = ref.apply(src, m)
    for dag in (False, True):   # hermitian: the dagger is A itself
        got = to_numpy(op, op.apply(x, m0=m, dagger=dag))
        check(got, want, prec, kind, dims, nc, nv, dag)
    assert rel_l2(to_numpy(op, op.apply_normal(x, m0=m)), ref.apply(want, m)) <= TOL[prec]
    op.close()


@pytest.mark.parametrize("kind", KINDS)
def test_laplace_every_launch_variant(kind):
    dims, nc, nv, bc = (4, 4, 2, 6), 3, 12, (1, -1, 1, -1)
    for layout in LAYOUTS:
        op, ref, src = make(kind, dims, nc, nv, bc, D.F32, layout=layout)
        x = to_device(op, src)
        want = ref.apply(src, 0.2)
        tried = 0
        for vr in (1, 2, 4):
            for minb in (1, 3, 4, 5, 6):
                try:
                    op.set_launch(vr, minb, 128)
                except D.DiracError:
                    continue
                tried += 1
                got = to_numpy(op, op.apply(x, m0=0.2))
                check(got, want, D.F32, kind, layout, vr, minb)
        assert tried == 15, (kind, tried)
        op.close()


@pytest.mark.parametrize("kind", KINDS)
def test_laplace_full_size_sampled_sites(kind):
    """16^3 x 32, N_c = 3, N_v = 12, FP32, site-inner layout, autotuned launch
    variant (as the benchmark's Laplace lines), 64 sampled output sites."""
    dims, nc, nv, bc = (16, 16, 16, 32), 3, 12, (1, 1, 1, -1)
    op, ref, src = make(kind, dims, nc, nv, bc, D.F32, seed=2024, layout=D.SITE_INNER)
    op.autotune(0.1)
    x = to_device(op, src)
    rng = np.random.default_rng(2)
    V = int(np.prod(dims))
    sites = np.concatenate([[0, V - 1, dims[0] - 1, V - dims[0]], rng.choice(V, 60, replace=False)])
    got = to_numpy(op, op.apply(x, m0=0.1)).reshape((V,) + src.shape[4:])[sites]
    assert rel_l2(got, ref.apply_sites(src, sites, 0.1)) <= TOL[D.F32], kind
    op.close()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_laplace_host_apply_matches_device_apply(layout):
    for kind in KINDS:
        op, ref, src = make(kind, (4, 4, 4, 12), 3, 12, (1, 1, 1, -1), D.F32, layout=layout)
        x = to_device(op, src)
        dev = op.apply(x, m0=0.1).cpu()
        hin = x.cpu().pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        op.apply_host(hin, hout, m0=0.1)
        assert torch.equal(hout, dev)
        op.close()


def _relres(ref, x, b, m):
    return np.sqrt(O.norm2(b - ref.apply(x, m)) / O.norm2(b))


@pytest.mark.parametrize("kind", KINDS)
def test_laplace_solvers(kind):
    """CG on A x = b (the paper's cg_wlap / cg_blap, dp and mp) and BiCGstab,
    m = 0.05 (a light boson mass), solutions checked by the oracle's A."""
    dims, nc, nv, bc, m = (4, 4, 4, 6), 3, 3, (1, 1, 1, -1), 0.05
    op, ref, b = make(kind, dims, nc, nv, bc, D.F64)
    bd = to_device(op, b)
    x, st = op.solve(bd, m0=m, solver=D.CG_HPD, tol=1e-10, maxit=10000)
    assert st["status"] == 0, st
    assert np.all(_relres(ref, to_numpy(op, x), b, m) < 1.01e-10)
    assert np.allclose(st["true_relres"], _relres(ref, to_numpy(op, x), b, m), rtol=1e-3, atol=1e-13)
    x, st = op.solve(bd, m0=m, solver=D.CG_HPD, tol=1e-10, maxit=20000, inner_prec=D.F32)
    assert st["status"] == 0, st
    assert np.all(_relres(ref, to_numpy(op, x), b, m) < 1.01e-10)
    x, st = op.solve(bd, m0=m, solver=D.BICGSTAB, tol=1e-10, maxit=10000)
    assert st["status"] == 0, st
    assert np.all(_relres(ref, to_numpy(op, x), b, m) < 1.01e-10)
    # the Lanczos extremes of the CG coefficients bracket A's spectrum: >= m^2/2
    x, st = op.solve(bd, m0=m, solver=D.CG_HPD, tol=1e-10, maxit=10000)
    assert min(st["lambda_min"][:nv]) >= 0.5 * m * m * (1 - 1e-6)
    with pytest.raises(D.DiracError):
        op.solve(bd, m0=m, solver=D.CG_NORMAL)
    with pytest.raises(D.DiracError):
        op.solve(bd, m0=m, solver=D.CG_HPD, inner_prec=D.F16)
    op.close()


def test_laplace_batched_solves():
    specs = [(D.WLAP, (4, 4, 4, 4), 2), (D.BSUV, (4, 4, 2, 4), 3), (D.WSUV, (6, 4, 2, 8), 5),
             (D.BLAP, (4, 2, 4, 4), 1)]
    ops, refs, bs, bn = [], [], [], []
    for i, (kind, dims, nv) in enumerate(specs):
        op, ref, b = make(kind, dims, 3, nv, (1, 1, 1, -1), D.F64, seed=600 + i, layout=i % 2)
        ops.append(op)
        refs.append(ref)
        bn.append(b)
        bs.append(to_device(op, b))
    m0s = [0.1, 0.2, 0.05, 0.3]
    xs, stats, rc = D.solve_batched(ops, bs, m0s=m0s, solver=D.CG_HPD, tol=1e-10, maxit=20000)
    assert rc == 0
    for i, (op, ref, b) in enumerate(zip(ops, refs, bn)):
        assert stats[i]["status"] == 0, (i, stats[i])
        assert np.all(_relres(ref, to_numpy(op, xs[i]), b, m0s[i]) < 1.05e-10), i
    with pytest.raises(D.DiracError):
        D.solve_batched(ops, bs, m0s=m0s, solver=D.CG_NORMAL, tol=1e-10)
    for op in ops:
        op.close()


def test_laplace_argument_rules():
    dims = (4, 4, 4, 4)
    U = torch.from_numpy(I.gauge_field(dims, 3, 0.4, 9)).cuda()
    for kind in KINDS:
        for prec in (D.BF16, D.F16):
            with pytest.raises(D.DiracError):
                D.DiracOp(kind, U, 2, (1, 1, 1, 1), prec)
        op = D.DiracOp(kind, U, 2, (1, 1, 1, 1), D.F32)
        with pytest.raises(D.DiracError):
            op.set_clover(1.0, U)
        with pytest.raises(D.DiracError):
            op.force(op.new_vector(), op.new_vector())
        op.close()
    # W links of the Brillouin Laplacian equal those of D_B on the same field
    a = D.DiracOp(D.BLAP, U, 2, (1, 1, 1, -1), D.F64)
    b = D.DiracOp(D.BRILLOUIN, U, 2, (1, 1, 1, -1), D.F64)
    assert torch.equal(a.copy_w(), b.copy_w())
    a.close()
    b.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", [D.F64, D.F32])
def test_laplace_extreme_shapes(kind, prec):
    """N_v = 64 on the 2^4 lattice and one RHS with N_c = 4 on a lattice long
    in t, both layouts."""
    for layout in LAYOUTS:
        for dims, nc, nv, bc in (((2, 2, 2, 2), 3, 64, (1, 1, 1, -1)), ((2, 2, 2, 34), 4, 1, (-1, 1, 1, -1))):
            op, ref, src = make(kind, dims, nc, nv, bc, prec, layout=layout)
            x = to_device(op, src)
            assert rel_l2(to_numpy(op, op.apply(x, m0=0.2)), ref.apply(src, 0.2)) <= TOL[prec], (kind, dims, layout)
            op.close()
