"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/dirac.h declares, and its argument
validation and pure host helpers behave as documented."""
import ctypes
import os
import re

import pytest

from paper_2112_14640_gb300 import build as B
from paper_2112_14640_gb300 import dirac as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dirac.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(dirac_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_functions():
    names = declared_functions()
    assert "dirac_apply" in names and "dirac_solve" in names and len(names) >= 15


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in D.SIGNATURES, "binding lacks a signature for %s" % name


def test_flop_counts_match_app_e(lib):
    """dirac_flops_per_site against the values and N_c polynomials App. E
    prints (tests/golden/app_e_flops_per_site.txt)."""
    from helpers import golden_flops
    kinds = {"wilson": D.WILSON, "brillouin": D.BRILLOUIN, "staggered": D.STAGGERED}
    for name, (nc, flops, flops12, poly) in golden_flops().items():
        assert D.flops_per_site(kinds[name], nc) == flops
        for n in (1, 2, 3, 4):
            assert D.flops_per_site(kinds[name], n) == eval(poly.replace("^", "**"), {"nc": n})
    assert D.flops_per_site(9, 3) == -1


def test_error_strings(lib):
    assert D.error_string(0) == "success"
    assert "aligned" in D.error_string(-4)
    assert "1%" in D.error_string(2)
    assert D.error_string(12345) == "unknown code"


def test_create_validates_before_touching_the_device(lib):
    """Invalid geometry is rejected before any CUDA call, so this runs without a GPU."""
    out = ctypes.c_void_p()

    def create(kind, dims, nc, nv, bc=(1, 1, 1, 1), prec=D.F32, U=1 << 20, u_prec=D.F64):
        g = D.Geom()
        g.dims[:] = dims
        g.nc, g.nv, g.prec = nc, nv, prec
        g.bc[:] = bc
        return lib.dirac_op_create(kind, ctypes.byref(g), ctypes.c_void_p(U), u_prec, None, ctypes.byref(out))

    assert create(D.WILSON, (4, 4, 4, 1), 3, 4) == -1          # extent < 2
    assert create(D.STAGGERED, (4, 4, 3, 4), 3, 4) == -1       # odd extent for staggered
    assert create(D.WILSON, (4, 4, 4, 4), 9, 4) == -2          # N_c above 8 not compiled
    assert create(D.WILSON, (4, 4, 4, 4), 0, 4) == -2          # no colours
    assert create(D.WILSON, (4, 4, 4, 4), 5, 4, prec=D.BF16) == -2   # N_c 5..8 only in FP64/FP32
    assert create(D.WILSON, (4, 4, 4, 4), 8, 4, prec=D.F16) == -2
    assert create(D.WILSON, (4, 4, 4, 4), 3, 0) == -1          # N_v = 0
    assert create(D.WILSON, (4, 4, 4, 4), 3, 65) == -1         # N_v > 64
    assert create(D.WILSON, (4, 4, 4, 4), 3, 4, bc=(1, 1, 1, 2)) == -1
    assert create(D.WILSON, (4, 4, 4, 4), 3, 4, prec=9) == -3
    assert create(D.WILSON, (4, 4, 4, 4), 3, 4, U=0) == -1     # null gauge field
    assert create(D.WILSON, (4, 4, 4, 4), 3, 4, u_prec=D.BF16) == -3
    assert create(9, (4, 4, 4, 4), 3, 4) == -1
    assert lib.dirac_op_create(0, None, None, 0, None, ctypes.byref(out)) == -1
    assert out.value is None


def test_null_handles_are_rejected(lib):
    p = ctypes.c_void_p(1 << 20)
    assert lib.dirac_apply(None, p, p, 0.0, None) == -1
    assert lib.dirac_apply_normal(None, p, p, 0.0, None) == -1
    assert lib.dirac_vec_norm2(None, p, p, None) == -1
    assert lib.dirac_solve(None, p, p, 0.0, None, None, None) == -1
    assert lib.dirac_vec_bytes(None) == 0
    lib.dirac_op_destroy(None)


def test_set_clover_validates_without_device(lib):
    """A null operator is refused before any CUDA call."""
    assert lib.dirac_op_set_clover(None, 1.0, None, D.F64, None) == -1
    assert lib.dirac_op_set_clover(None, 0.0, None, D.F64, None) == -1


def test_clover_flop_count_matches_app_e(lib):
    """dirac_clover_flops_per_site against the two-multiplication count App. E
    prints (tests/golden/app_e_clover_flops.txt)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "app_e_clover_flops.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    (form, nc, flops, poly, mults), = [r for r in rows if r[0] == "two_products"]
    assert D.clover_flops_per_site(int(nc)) == int(flops)
    for n in (1, 2, 3, 4):
        assert D.clover_flops_per_site(n) == eval(poly.replace("^", "**"), {"nc": n})


def test_laplace_kinds_flops_and_validation(lib):
    """dirac_flops_per_site for the Laplace kinds against App. E
    (tests/golden/app_e_laplace_flops.txt); 16-bit Laplace operators are
    refused before any CUDA call."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "app_e_laplace_flops.txt")
    kinds = {"wlap": D.WLAP, "wsuv": D.WSUV, "blap": D.BLAP, "bsuv": D.BSUV}
    for name, nc, flops, f12, poly in (ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")):
        assert D.flops_per_site(kinds[name], int(nc)) == int(flops)
        for n in (1, 2, 3, 4):
            assert D.flops_per_site(kinds[name], n) == eval(poly.replace("^", "**"), {"nc": n})
    out = ctypes.c_void_p()
    g = D.Geom()
    g.dims[:] = (4, 4, 4, 4)
    g.nc, g.nv = 3, 4
    g.bc[:] = (1, 1, 1, 1)
    for kind in (D.WLAP, D.BLAP, D.WSUV, D.BSUV):
        for prec in (D.BF16, D.F16):
            g.prec = prec
            assert lib.dirac_op_create(kind, ctypes.byref(g), ctypes.c_void_p(1 << 20), D.F64, None,
                                       ctypes.byref(out)) == -3
    g.prec = D.F32
    assert lib.dirac_op_create(7, ctypes.byref(g), ctypes.c_void_p(1 << 20), D.F64, None, ctypes.byref(out)) == -1


def test_stout_smear_validates_without_device(lib):
    dims = (ctypes.c_int * 4)(4, 4, 4, 4)
    bad = (ctypes.c_int * 4)(4, 1, 4, 4)
    p = ctypes.c_void_p(1 << 20)
    assert lib.dirac_stout_smear(None, p, dims, 3, D.F64, 0.12, 3, None) == -1
    assert lib.dirac_stout_smear(p, p, bad, 3, D.F64, 0.12, 3, None) == -1
    assert lib.dirac_stout_smear(p, p, dims, 3, D.F64, 0.12, -1, None) == -1
    assert lib.dirac_stout_smear(p, p, dims, 9, D.F64, 0.12, 3, None) == -2
    assert lib.dirac_stout_smear(p, p, dims, 3, D.BF16, 0.12, 3, None) == -3
