"""GPU parity of the clover term (Eq. def_clov) fused into D_W and D_B,
through the C ABI, against the FP64 oracle: D + C, its dagger and the normal
operator element by element; every launch variant; the 16^3 x 32, N_v = 12
workload on sampled sites; the host apply; the solvers and the batched solves
with a clover operator (solutions checked by the oracle's D + C); and the
lifetime rules (c_SW = 0 and a new gauge field remove the term).

Tolerances as in test_gpu_parity: relative L2 1e-12 FP64, 1e-5 FP32, 1e-2
for 16-bit storage.  c_SW = 1 is the tree-level value the paper's solver
tests use; F is built from a second field V (the paper builds it from a
smeared field) except where noted.
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
KINDS = [D.WILSON, D.BRILLOUIN]


def make(kind, dims, nc, nv, bc, prec, csw=1.0, seed=5, own_v=True, layout=D.SITE_OUTER,
         link_storage=D.LINKS_NATIVE, v_f32=False):
    U = I.gauge_field(dims, nc, 0.4, seed)
    V = I.gauge_field(dims, nc, 0.3, seed + 100) if own_v else U
    op = D.DiracOp(kind, torch.from_numpy(U).cuda(), nv, bc, prec, layout=layout, link_storage=link_storage)
    Vt = torch.from_numpy(V).cuda()
    if v_f32:
        Vt = Vt.to(torch.complex64)
        V = V.astype(np.complex64).astype(np.complex128)
    op.set_clover(csw, Vt)
    ref = O.Operator(kind, U, bc, csw=csw, V=V)
    src = I.source(dims, nc, nv, seed + 1)
    return op, ref, src


CASES = [
    # dims, nc, nv, bc
    ((4, 4, 4, 4), 3, 1, (1, 1, 1, -1)),
    ((8, 8, 8, 8), 3, 12, (1, 1, 1, -1)),
    ((6, 4, 2, 8), 3, 3, (1, -1, 1, -1)),
    ((4, 6, 4, 2), 2, 4, (1, 1, 1, 1)),
    ((2, 4, 4, 6), 4, 5, (-1, 1, 1, -1)),
    ((4, 4, 2, 4), 1, 8, (1, 1, 1, -1)),
]


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", [D.F64, D.F32])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_clover_apply_dagger_normal(kind, prec, case, layout):
    dims, nc, nv, bc = CASES[case]
    m0 = -0.2
    op, ref, src = make(kind, dims, nc, nv, bc, prec, csw=1.0 + 0.25 * case, own_v=case % 2 == 0,
                        layout=layout)
    x = to_device(op, src)
    for dag in (False, True):
        got = to_numpy(op, op.apply(x, m0=m0, dagger=dag))
        want = ref.apply_dagger(src, m0) if dag else ref.apply(src, m0)
        check(got, want, prec, kind, dims, nc, nv, dag)
    check(to_numpy(op, op.apply_normal(x, m0=m0)), ref.apply_normal(src, m0), prec, kind, "normal")
    op.close()


def test_clover_term_alone_matches_oracle():
    """(D + C) psi - D psi on the GPU against the oracle's C psi, F64: isolates
    the field strength and the block form from the stencil."""
    dims, nc, nv, bc = (4, 6, 4, 6), 3, 4, (1, 1, 1, -1)
    for kind in KINDS:
        for layout in LAYOUTS:
            op, ref, src = make(kind, dims, nc, nv, bc, D.F64, csw=1.0, layout=layout)
            x = to_device(op, src)
            with_c = to_numpy(op, op.apply(x, m0=0.1))
            op.set_clover(0.0)
            plain = to_numpy(op, op.apply(x, m0=0.1))
            want = O.clover(ref.F, 1.0, src)
            assert rel_l2(with_c - plain, want) <= 1e-12, (kind, layout)
            op.close()


@pytest.mark.parametrize("links", [D.LINKS_NATIVE, D.LINKS_F32])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", [D.BF16, D.F16])
def test_clover_low_precision_storage(kind, prec, links):
    dims, nc, nv, bc = (8, 4, 4, 8), 3, 12, (1, 1, 1, -1)
    op, ref, src = make(kind, dims, nc, nv, bc, prec, layout=D.SITE_INNER, link_storage=links, v_f32=True)
    x = to_device(op, src)
    for dag in (False, True):
        got = to_numpy(op, op.apply(x, m0=0.1, dagger=dag))
        want = ref.apply_dagger(src, 0.1) if dag else ref.apply(src, 0.1)
        check(got, want, prec, kind, links, dag)
    op.close()


@pytest.mark.parametrize("kind", KINDS)
def test_clover_every_launch_variant(kind):
    dims, nc, nv, bc = (4, 4, 2, 6), 3, 12, (1, -1, 1, -1)
    for layout in LAYOUTS:
        op, ref, src = make(kind, dims, nc, nv, bc, D.F32, layout=layout)
        x = to_device(op, src)
        want = ref.apply(src, 0.1)
        tried = 0
        for vr in (1, 2, 4):
            for minb in (1, 3, 4, 5, 6):
                try:
                    op.set_launch(vr, minb, 128)
                except D.DiracError:
                    continue
                tried += 1
                got = to_numpy(op, op.apply(x, m0=0.1))
                check(got, want, D.F32, kind, layout, vr, minb)
        assert tried >= 8
        op.close()


@pytest.mark.parametrize("kind", KINDS)
def test_clover_full_size_sampled_sites(kind):
    """16^3 x 32, N_c = 3, N_v = 12, FP32, c_SW = 1, site-inner layout and the
    autotuned launch variant (as the benchmark's clover line), 64 sampled sites."""
    dims, nc, nv, bc = (16, 16, 16, 32), 3, 12, (1, 1, 1, -1)
    op, ref, src = make(kind, dims, nc, nv, bc, D.F32, seed=2024, own_v=False, layout=D.SITE_INNER)
    op.autotune(0.1)
    x = to_device(op, src)
    rng = np.random.default_rng(1)
    V = int(np.prod(dims))
    sites = np.concatenate([[0, V - 1, dims[0] - 1, V - dims[0]], rng.choice(V, 60, replace=False)])
    for dag in (False, True):
        got = to_numpy(op, op.apply(x, m0=0.1, dagger=dag)).reshape((V,) + src.shape[4:])[sites]
        want = ref.apply_sites(src, sites, 0.1, dagger=dag)
        check(got, want, D.F32, kind, dag, site_axes=1)
    op.close()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_clover_host_apply_matches_device_apply(layout):
    for kind in KINDS:
        op, ref, src = make(kind, (4, 4, 4, 12), 3, 12, (1, 1, 1, -1), D.F32, layout=layout)
        x = to_device(op, src)
        dev = op.apply(x, m0=0.1).cpu()
        hin = x.cpu().pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        op.apply_host(hin, hout, m0=0.1)
        assert torch.equal(hout, dev)
        op.close()


def _true_relres(ref, x, b, m0):
    return np.sqrt(O.norm2(b - ref.apply(x, m0)) / O.norm2(b))


@pytest.mark.parametrize("kind", KINDS)
def test_clover_solvers(kind):
    """CG on the normal equations (FP64, and FP64 outer with FP32 / FP16
    inner) and BiCGstab, on D + C; solutions checked by the oracle's D + C."""
    dims, nc, nv, bc, m0 = (4, 4, 4, 6), 3, 3, (1, 1, 1, -1), 0.1
    op, ref, b = make(kind, dims, nc, nv, bc, D.F64, csw=1.0)
    bd = to_device(op, b)
    x, st = op.solve(bd, m0=m0, tol=1e-10, maxit=10000)
    assert st["status"] == 0, st
    xs = to_numpy(op, x)
    bN = ref.apply_dagger(b, m0)
    assert np.all(np.sqrt(O.norm2(bN - ref.apply_normal(xs, m0)) / O.norm2(bN)) < 1.01e-10)
    for inner in (D.F32, D.F16):
        x, st = op.solve(bd, m0=m0, tol=1e-10, maxit=20000, inner_prec=inner)
        assert st["status"] == 0, (inner, st)
        xs = to_numpy(op, x)
        assert np.all(np.sqrt(O.norm2(bN - ref.apply_normal(xs, m0)) / O.norm2(bN)) < 1.01e-10)
    x, st = op.solve(bd, m0=m0, solver=D.BICGSTAB, tol=1e-10, maxit=10000)
    assert st["status"] == 0, st
    assert np.all(_true_relres(ref, to_numpy(op, x), b, m0) < 1.01e-10)
    op.close()


def test_clover_batched_solves():
    specs = [(D.WILSON, (4, 4, 4, 4), 2, 0.2), (D.BRILLOUIN, (4, 4, 2, 4), 3, 0.2),
             (D.WILSON, (6, 4, 2, 8), 5, 0.3)]
    ops, refs, bs, bn = [], [], [], []
    for i, (kind, dims, nv, m0) in enumerate(specs):
        op, ref, b = make(kind, dims, 3, nv, (1, 1, 1, -1), D.F64, csw=1.0, seed=500 + i, layout=i % 2)
        ops.append(op)
        refs.append(ref)
        bn.append(b)
        bs.append(to_device(op, b))
    m0s = [s[3] for s in specs]
    xs, stats, rc = D.solve_batched(ops, bs, m0s=m0s, solver=D.CG_NORMAL, tol=1e-10, maxit=20000)
    assert rc == 0
    for i, (op, ref, b) in enumerate(zip(ops, refs, bn)):
        xsn = to_numpy(op, xs[i])
        bN = ref.apply_dagger(b, m0s[i])
        res = np.sqrt(O.norm2(bN - ref.apply_normal(xsn, m0s[i])) / O.norm2(bN))
        assert np.all(res < 1.05e-10), (i, res)
        op.close()


def test_clover_lifetime_and_refusals():
    dims, nc, nv, bc = (4, 4, 4, 4), 3, 2, (1, 1, 1, -1)
    U = I.gauge_field(dims, nc, 0.4, 9)
    Ut = torch.from_numpy(U).cuda()
    src = I.source(dims, nc, nv, 10)
    plain = O.Operator(D.WILSON, U, bc).apply(src, 0.1)
    op = D.DiracOp(D.WILSON, Ut, nv, bc, D.F64)
    x = to_device(op, src)
    op.set_clover(1.0, Ut)
    assert rel_l2(to_numpy(op, op.apply(x, m0=0.1)), O.Operator(D.WILSON, U, bc, csw=1.0).apply(src, 0.1)) < 1e-12
    with pytest.raises(D.DiracError):          # the force is derived without the clover term
        op.force(x, x)
    op.set_clover(0.0)
    assert rel_l2(to_numpy(op, op.apply(x, m0=0.1)), plain) < 1e-12
    op.set_clover(1.0, Ut)
    op.update_links(Ut)                         # a new field drops the term
    assert rel_l2(to_numpy(op, op.apply(x, m0=0.1)), plain) < 1e-12
    with pytest.raises(ValueError):
        op.set_clover(1.0)                      # no field given
    op.close()
    st = D.DiracOp(D.STAGGERED, Ut, nv, bc, D.F64)
    with pytest.raises(D.DiracError):
        st.set_clover(1.0, Ut)
    st.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", [D.F64, D.F32])
def test_clover_extreme_shapes(kind, prec):
    """N_v = 64 on the 2^4 lattice (every plaquette leaf wraps onto the same
    links; forward and backward neighbours coincide), and one RHS with N_c = 4
    on a lattice long in t, both layouts."""
    for layout in LAYOUTS:
        for dims, nc, nv, bc in (((2, 2, 2, 2), 3, 64, (1, 1, 1, -1)), ((2, 2, 2, 34), 4, 1, (-1, 1, 1, -1))):
            op, ref, src = make(kind, dims, nc, nv, bc, prec, csw=1.5, layout=layout)
            x = to_device(op, src)
            for dag in (False, True):
                got = to_numpy(op, op.apply(x, m0=0.1, dagger=dag))
                want = ref.apply_dagger(src, 0.1) if dag else ref.apply(src, 0.1)
                check(got, want, prec, kind, dims, nv, dag, layout)
            op.close()
