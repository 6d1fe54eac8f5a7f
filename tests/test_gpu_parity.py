"""GPU parity: every stencil, its dagger and D^dag D, the W-link builder and
the BLAS-1 reductions, through the C ABI, element by element against the FP64
oracle on the same seeded inputs.

Tolerances (relative L2 over the whole output): 1e-12 FP64, 1e-5 FP32,
1e-2 BF16/FP16 storage (FP32 arithmetic).  Small lattices span many thread
blocks and ragged tails (odd extents, odd N_v); the full 16^3x32, N_v = 12
workload is checked on sampled output sites.
"""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import TOL, check, rel_l2, to_device, to_numpy
from paper_2112_14640_gb300 import dirac as D
from paper_2112_14640_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KINDS = [D.WILSON, D.BRILLOUIN, D.STAGGERED]


LAYOUTS = [D.SITE_OUTER, D.SITE_INNER]


def make(kind, dims, nc, nv, bc, prec, eps=0.4, seed=5, u_f32=False, layout=D.SITE_OUTER,
         link_storage=D.LINKS_NATIVE):
    U = I.gauge_field(dims, nc, eps, seed)
    Ut = torch.from_numpy(U).cuda()
    if u_f32:
        Ut = Ut.to(torch.complex64)
    op = D.DiracOp(kind, Ut, nv, bc, prec, layout=layout, link_storage=link_storage)
    ref = O.Operator(kind, U.astype(np.complex64).astype(np.complex128) if u_f32 else U, bc)
    src = I.source(dims, nc, nv, seed + 1, staggered=(kind == D.STAGGERED))
    return op, ref, src


CASES = [
    # dims, nc, nv, bc
    ((4, 4, 4, 4), 3, 1, (1, 1, 1, -1)),
    ((8, 8, 8, 8), 3, 12, (1, 1, 1, -1)),
    ((6, 4, 2, 8), 3, 3, (1, -1, 1, -1)),
    ((4, 6, 4, 2), 2, 4, (1, 1, 1, 1)),
    ((2, 4, 4, 6), 4, 5, (-1, 1, 1, -1)),
    ((4, 4, 2, 4), 1, 8, (1, 1, 1, -1)),
    # N_c beyond 4 (FP64/FP32 storage; the paper's N_c sweep reaches 8 and beyond)
    ((4, 2, 4, 2), 5, 4, (-1, 1, 1, 1)),
    ((4, 4, 2, 4), 6, 3, (1, 1, 1, -1)),
    ((2, 4, 2, 4), 7, 2, (1, 1, -1, 1)),
    ((2, 4, 4, 2), 8, 2, (1, -1, 1, -1)),
]


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", [D.F64, D.F32])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_apply_and_dagger(kind, prec, case, layout):
    dims, nc, nv, bc = CASES[case]
    m0 = 0.1 if kind != D.STAGGERED else 0.05
    op, ref, src = make(kind, dims, nc, nv, bc, prec, layout=layout)
    x = to_device(op, src)
    for dag in (False, True):
        got = to_numpy(op, op.apply(x, m0=m0, dagger=dag))
        want = ref.apply_dagger(src, m0) if dag else ref.apply(src, m0)
        check(got, want, prec, kind, dims, nc, nv, dag)
    got = to_numpy(op, op.apply_normal(x, m0=m0))
    check(got, ref.apply_normal(src, m0), prec, kind, "normal")
    op.close()


@pytest.mark.parametrize("links", [D.LINKS_NATIVE, D.LINKS_F32])
@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", [D.BF16, D.F16])
def test_apply_low_precision_storage(kind, prec, layout, links):
    dims, nc, nv, bc = (8, 4, 4, 8), 3, 12, (1, 1, 1, -1)
    m0 = 0.1
    op, ref, src = make(kind, dims, nc, nv, bc, prec, layout=layout, link_storage=links)
    x = to_device(op, src)
    for dag in (False, True):
        got = to_numpy(op, op.apply(x, m0=m0, dagger=dag))
        want = ref.apply_dagger(src, m0) if dag else ref.apply(src, m0)
        check(got, want, prec, kind, layout, links, dag)
    op.close()


def test_f32_links_from_f32_gauge_field():
    """U handed over in FP32 (the paper keeps links in sp, Sec. 2)."""
    dims = (4, 4, 4, 8)
    for kind in KINDS:
        op, ref, src = make(kind, dims, 3, 4, (1, 1, 1, -1), D.F64, u_f32=True)
        got = to_numpy(op, op.apply(to_device(op, src), m0=0.2))
        assert rel_l2(got, ref.apply(src, 0.2)) <= 1e-12
        op.close()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("prec", [D.F64, D.F32])
def test_w_links_match_path_enumeration(prec, layout):
    dims, nc, bc = (4, 6, 2, 4), 3, (1, -1, 1, -1)
    op, ref, _ = make(D.BRILLOUIN, dims, nc, 2, bc, prec, layout=layout)
    w = op.copy_w()
    w = torch.view_as_complex(w.contiguous()) if w.dtype in (torch.bfloat16, torch.float16) else w
    got = w.to(torch.complex128).cpu().numpy()
    if layout == D.SITE_INNER:
        got = np.ascontiguousarray(np.transpose(got, (3, 4, 5, 6, 0, 1, 2)))
    want = np.delete(ref.W, 40, axis=4)
    assert rel_l2(got, want) <= (1e-13 if prec == D.F64 else 1e-6)
    op.close()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("kind", KINDS)
def test_full_size_sampled_sites(kind, layout):
    """16^3 x 32, N_c = 3, N_v = 12, FP32: the benchmark configuration, in the
    launch configuration the benchmark times (autotuned variant), checked on
    64 sampled sites."""
    dims, nc, nv, bc = (16, 16, 16, 32), 3, 12, (1, 1, 1, -1)
    m0 = 0.05 if kind == D.STAGGERED else 0.1
    op, ref, src = make(kind, dims, nc, nv, bc, D.F32, seed=2024, layout=layout)
    op.autotune(m0)
    x = to_device(op, src)
    rng = np.random.default_rng(0)
    V = int(np.prod(dims))
    sites = np.concatenate([[0, V - 1, dims[0] - 1, V - dims[0]], rng.choice(V, 60, replace=False)])
    for dag in (False, True):
        got = to_numpy(op, op.apply(x, m0=m0, dagger=dag)).reshape((V,) + src.shape[4:])[sites]
        want = ref.apply_sites(src, sites, m0, dagger=dag)
        check(got, want, D.F32, kind, dag, site_axes=1)
    op.close()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("prec", [D.F64, D.F32, D.BF16])
@pytest.mark.parametrize("kind", [D.WILSON, D.STAGGERED])
def test_blas_reductions(kind, prec, layout):
    dims, nc, nv = (6, 4, 4, 4), 3, 7 if prec != D.BF16 else 6
    op, ref, src = make(kind, dims, nc, nv, (1, 1, 1, 1), prec, layout=layout)
    src2 = I.source(dims, nc, nv, 77, staggered=(kind == D.STAGGERED))
    from helpers import rounded
    a, b = rounded(src, prec), rounded(src2, prec)
    x, y = to_device(op, src), to_device(op, src2)
    n2 = op.norm2(x).cpu().numpy()
    assert np.allclose(n2, O.norm2(a), rtol=1e-12)
    dt = op.dot(x, y).cpu().numpy()
    assert np.allclose(dt, O.dot(a, b), rtol=1e-12, atol=1e-9 * np.abs(O.dot(a, b)).max())
    # deterministic: bitwise identical on repeat
    assert np.array_equal(op.norm2(x).cpu().numpy(), n2)
    alpha = (np.arange(nv) + 1j * (0.5 - np.arange(nv))) / nv
    op.axpy(torch.from_numpy(alpha), x, y)
    got = to_numpy(op, y)
    assert rel_l2(got, b + alpha * a) <= TOL[prec]
    op.gamma5_(x)
    want = O.epsilon(a) if kind == D.STAGGERED else O.gamma5(a)
    assert rel_l2(to_numpy(op, x), want) <= (1e-15 if prec != D.BF16 else 1e-2)
    op.close()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("dims", [(8, 8, 4, 8), (4, 4, 4, 6), (4, 4, 4, 20), (4, 4, 2, 2)])
def test_host_apply_matches_device_apply(dims, layout):
    """The host apply (copies and stencil pipelined over slabs of time slices
    for N_t >= 3, one copy each way otherwise) equals the device apply bit for
    bit."""
    for kind in KINDS:
        op, ref, src = make(kind, dims, 3, 12, (1, 1, 1, -1), D.F32, layout=layout)
        x = to_device(op, src)
        dev = op.apply(x, m0=0.1).cpu()
        hin = x.cpu().pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        op.apply_host(hin, hout, m0=0.1)
        assert torch.equal(hout, dev)
        op.close()


@pytest.mark.parametrize("dims", [(8, 8, 4, 8), (4, 4, 4, 2)])
def test_async_host_applies_overlap_and_match(dims):
    """dirac_apply_host_async on three operators enqueued back to back, twice
    in a row (the second round reuses the staging buffers), one wait: every
    output equals the device apply bit for bit."""
    ops, hins, houts, devs = [], [], [], []
    for kind in KINDS:
        op, ref, src = make(kind, dims, 3, 12, (1, 1, 1, -1), D.F32, layout=D.SITE_INNER)
        x = to_device(op, src)
        devs.append(op.apply(x, m0=0.1).cpu())
        hins.append(x.cpu().pin_memory())
        houts.append(torch.zeros_like(hins[-1]).pin_memory())
        ops.append(op)
    torch.cuda.synchronize()
    for _ in range(2):
        for op, hi, ho in zip(ops, hins, houts):
            op.apply_host_async(hi, ho, m0=0.1)
    torch.cuda.current_stream().synchronize()
    for op, ho, dv in zip(ops, houts, devs):
        assert torch.equal(ho, dv)
    # the synchronous and the asynchronous form in turn on one operator (their
    # stencils run on different streams): each sees the other's staging buffers free
    op, hi = ops[0], hins[0]
    h2 = (2 * hi).pin_memory()
    want2 = op.apply(h2.cuda(), m0=0.1).cpu()
    o1, o2, o3 = (torch.zeros_like(hi).pin_memory() for _ in range(3))
    op.apply_host_async(h2, o1, m0=0.1)
    op.apply_host(hi, o2, m0=0.1)
    op.apply_host_async(h2, o3, m0=0.1)
    torch.cuda.current_stream().synchronize()
    assert torch.equal(o1, want2) and torch.equal(o2, devs[0]) and torch.equal(o3, want2)
    for op in ops:
        op.close()


def test_precision_convert_roundtrip():
    op, ref, src = make(D.WILSON, (4, 4, 4, 4), 3, 4, (1, 1, 1, 1), D.F64)
    x = to_device(op, src)
    for p in (D.F32, D.BF16, D.F16):
        lo = op.convert(x, D.F64, p)
        back = op.convert(lo, p, D.F64)
        from helpers import rounded
        assert np.array_equal(to_numpy(op, back), rounded(src, p))
    op.close()


def test_error_codes_from_the_abi():
    U = torch.from_numpy(I.gauge_field((4, 4, 4, 4), 3, 0.4, 1)).cuda()
    with pytest.raises(D.DiracError) as e:
        D.DiracOp(D.STAGGERED, U[:, :, :, :3].contiguous(), 2)       # odd Nx
    assert e.value.code == -1
    with pytest.raises(D.DiracError) as e:
        D.DiracOp(D.WILSON, U, 65)                                  # N_v > 64
    assert e.value.code == -1
    op = D.DiracOp(D.WILSON, U, 2, prec=D.F32)
    x = op.new_vector()
    buf = torch.zeros(x.numel() * 2 + 8, dtype=torch.float32, device="cuda")
    lib = D.lib()
    import ctypes
    # a pointer 4 bytes into an allocation: rejected before any launch
    rc = lib.dirac_apply(op._h, ctypes.c_void_p(buf.data_ptr() + 4), ctypes.c_void_p(x.data_ptr()), 0.1,
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -4
    rc = lib.dirac_apply(op._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 0.1,
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1   # in place is rejected
    op.close()


def test_f32_links_reduce_the_error_of_16bit_operators():
    """With FP32 links only the rounding of the stored output remains: the
    error of an F16 apply with F32 links equals that rounding alone, and the
    all-F16 operator adds the link rounding on top."""
    from helpers import rounded
    dims, nc, nv, bc = (8, 4, 4, 8), 3, 4, (1, 1, 1, -1)
    errs = {}
    for links in (D.LINKS_NATIVE, D.LINKS_F32):
        op, ref, src = make(D.WILSON, dims, nc, nv, bc, D.F16, link_storage=links)
        srcr = rounded(src, D.F16)
        want = ref.apply(srcr, 0.1)
        got = to_numpy(op, op.apply(to_device(op, src), m0=0.1))
        errs[links] = rel_l2(got, want)
        errs["round"] = rel_l2(rounded(want, D.F16), want)
        op.close()
    assert errs[D.LINKS_F32] < 1.05 * errs["round"], errs
    assert errs[D.LINKS_NATIVE] > errs[D.LINKS_F32], errs


@pytest.mark.parametrize("kind", KINDS)
def test_every_launch_variant_matches_the_oracle(kind):
    """Every compiled (VR, register class, block size) variant gives the same
    operator (the autotuner may pick any of them)."""
    dims, nc, nv, bc = (4, 4, 2, 6), 3, 12, (1, -1, 1, -1)
    m0 = 0.05 if kind == D.STAGGERED else 0.1
    for layout in LAYOUTS:
        op, ref, src = make(kind, dims, nc, nv, bc, D.F32, layout=layout)
        x = to_device(op, src)
        want = ref.apply(src, m0)
        tried = 0
        for vr in (1, 2, 4):
            for minb in (1, 3, 4, 5, 6):
                for block in (64, 128, 384):
                    try:
                        op.set_launch(vr, minb, block)
                    except D.DiracError:
                        continue
                    tried += 1
                    got = to_numpy(op, op.apply(x, m0=m0))
                    check(got, want, D.F32, kind, layout, vr, minb, block)
        assert tried >= 20
        op.close()


def test_set_launch_rejects_invalid_variants():
    op, _, _ = make(D.WILSON, (4, 4, 4, 4), 3, 12, (1, 1, 1, 1), D.F32)
    for args in ((3, 1, 128), (2, 2, 128), (2, 1, 100), (2, 1, 256), (8, 1, 128)):
        with pytest.raises(D.DiracError):
            op.set_launch(*args)
    op.set_launch(2, 4, 256)
    assert op.get_launch() == (2, 4, 256)
    op.set_launch(0)
    vr, minb, block = op.get_launch()
    assert 12 % vr == 0 and block % 32 == 0
    op.close()
    op, _, _ = make(D.WILSON, (4, 4, 4, 4), 3, 6, (1, 1, 1, 1), D.F32)
    with pytest.raises(D.DiracError):
        op.set_launch(4, 1, 128)        # 4 does not divide N_v = 6
    op.close()


@pytest.mark.parametrize("prec", [D.F32, D.BF16])
def test_blas_reductions_full_size(prec):
    """Norms and dot products over 16^3x32 x Nv = 4 (6.3 M complex numbers per
    column group) keep FP64-level accuracy: compensated FP32 accumulation in
    the thread loops, FP64 across threads."""
    dims, nc, nv = (16, 16, 16, 32), 3, 4
    op = D.DiracOp(D.WILSON, torch.from_numpy(I.unit_gauge_field(dims, nc)).cuda(), nv, (1, 1, 1, 1), prec)
    g = torch.Generator(device="cpu").manual_seed(7)
    rows = op.vec_bytes() // (nv * (8 if prec == D.F32 else 4))
    a = torch.randn(rows, nv, dtype=torch.complex128, generator=g) * 3 + 1
    b = torch.randn(rows, nv, dtype=torch.complex128, generator=g)
    if prec == D.F32:
        xa, xb = a.to(torch.complex64), b.to(torch.complex64)
        ha, hb = xa.to(torch.complex128), xb.to(torch.complex128)
    else:
        xa = torch.view_as_real(a).to(torch.bfloat16)
        xb = torch.view_as_real(b).to(torch.bfloat16)
        ha = torch.view_as_complex(xa.to(torch.float64).contiguous())
        hb = torch.view_as_complex(xb.to(torch.float64).contiguous())
    n2 = op.norm2(xa.cuda().reshape(op.new_vector().shape)).cpu().numpy()
    want = (ha.abs() ** 2).sum(0).numpy()
    assert np.allclose(n2, want, rtol=1e-12, atol=0)
    dt = op.dot(xa.cuda().reshape(op.new_vector().shape), xb.cuda().reshape(op.new_vector().shape)).cpu().numpy()
    wdot = (ha.conj() * hb).sum(0).numpy()
    scale = (ha.abs() ** 2).sum(0).sqrt().numpy() * (hb.abs() ** 2).sum(0).sqrt().numpy()
    assert np.all(np.abs(dt - wdot) <= 1e-12 * scale), (np.abs(dt - wdot) / scale)
    op.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", [D.F64, D.F32])
def test_extreme_shapes(kind, prec):
    """The largest N_v (64) on the smallest lattice (extent 2 in every
    direction: the forward and backward neighbour are the same site), and a
    single RHS with N_c = 4 on a lattice long in t."""
    for dims, nc, nv, bc in (((2, 2, 2, 2), 3, 64, (1, 1, 1, -1)), ((2, 2, 2, 34), 4, 1, (-1, 1, 1, -1))):
        m0 = 0.05 if kind == D.STAGGERED else 0.1
        op, ref, src = make(kind, dims, nc, nv, bc, prec)
        x = to_device(op, src)
        for dag in (False, True):
            got = to_numpy(op, op.apply(x, m0=m0, dagger=dag))
            want = ref.apply_dagger(src, m0) if dag else ref.apply(src, m0)
            check(got, want, prec, kind, dims, nv, dag)
        n2 = op.norm2(x).cpu().numpy()
        assert np.allclose(n2, O.norm2(src if prec == D.F64 else src.astype(np.complex64).astype(np.complex128)),
                           rtol=1e-12)
        op.close()


@pytest.mark.parametrize("nc", [5, 6, 8])
def test_large_nc_rejected_for_16bit_storage_and_variants(nc):
    """N_c above 4 is compiled for FP64/FP32 storage with one RHS per thread:
    16-bit storage and wider launch variants are refused by the C ABI."""
    U = torch.from_numpy(I.gauge_field((2, 2, 2, 2), nc, 0.4, 3)).cuda()
    for prec in (D.BF16, D.F16):
        with pytest.raises(D.DiracError) as e:
            D.DiracOp(D.WILSON, U, 2, (1, 1, 1, 1), prec)
        assert e.value.code == -2
    op = D.DiracOp(D.WILSON, U, 4, (1, 1, 1, 1), D.F32)
    with pytest.raises(D.DiracError):
        op.set_launch(2, 1, 128)
    op.set_launch(1, 1, 64)
    assert op.get_launch() == (1, 1, 64)
    op.close()
    with pytest.raises(D.DiracError) as e:
        D.DiracOp(D.WILSON, torch.from_numpy(I.gauge_field((2, 2, 2, 2), 9, 0.4, 3)).cuda(), 2)
    assert e.value.code == -2


@pytest.mark.parametrize("kind", KINDS)
def test_large_nc_full_lattice_sampled(kind):
    """N_c = 6 and 8 at N_v = 12 on 8^3x4 (many thread blocks), FP32,
    site-inner, autotuned: sampled sites against the oracle."""
    for nc in (6, 8):
        dims, nv, bc = (8, 8, 8, 4), 12, (1, 1, 1, -1)
        m0 = 0.05 if kind == D.STAGGERED else 0.1
        op, ref, src = make(kind, dims, nc, nv, bc, D.F32, seed=77, layout=D.SITE_INNER)
        op.autotune(m0)
        x = to_device(op, src)
        V = int(np.prod(dims))
        sites = np.concatenate([[0, V - 1], np.random.default_rng(nc).choice(V, 40, replace=False)])
        got = to_numpy(op, op.apply(x, m0=m0)).reshape((V,) + src.shape[4:])[sites]
        check(got, ref.apply_sites(src, sites, m0), D.F32, kind, nc, site_axes=1)
        op.close()
