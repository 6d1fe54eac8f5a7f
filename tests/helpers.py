"""Shared helpers for the GPU parity tests: move seeded numpy inputs to the
device in the library's formats and compare with the oracle."""
import numpy as np
import torch

from paper_2112_14640_gb300 import dirac as D

TOL = {D.F64: 1e-12, D.F32: 1e-5, D.BF16: 1e-2, D.F16: 1e-2}


def rel_l2(got, want):
    got = np.asarray(got)
    want = np.asarray(want)
    return float(np.linalg.norm((got - want).ravel()) / max(np.linalg.norm(want.ravel()), 1e-300))


def site_err(got, want, site_axes=4):
    """Largest per-site error: max over sites of |got_n - want_n| divided by the
    root-mean-square over sites of |want_n| (a site = the first `site_axes`
    axes; the rest, colour, spin and RHS, form the site's vector).  A single
    wrong site shows here even when the global relative L2 error hides it."""
    got = np.asarray(got)
    want = np.asarray(want)
    nsite = int(np.prod(want.shape[:site_axes]))
    d = np.linalg.norm((got - want).reshape(nsite, -1), axis=1)
    w = np.linalg.norm(want.reshape(nsite, -1), axis=1)
    return float(d.max() / max(np.sqrt(np.mean(w ** 2)), 1e-300))


def check(got, want, prec, *ctx, site_axes=4, tol=None):
    """Parity bar: global relative L2 <= tol (TOL[prec] by default) and
    per-site error (site_err) <= 2 tol."""
    tol = TOL[prec] if tol is None else tol
    e, es = rel_l2(got, want), site_err(got, want, site_axes)
    assert e <= tol and es <= 2 * tol, (ctx, e, es)
    return e


def to_device(op, v_np, prec=None):
    """numpy complex128 vector in the paper's site-outer order -> device tensor
    in the op's layout and (or the given) precision."""
    t = torch.from_numpy(np.ascontiguousarray(v_np)).to(op.device)
    return op.to_prec(op.from_site_outer(t), op.prec if prec is None else prec)


def to_numpy(op, v):
    """device vector in the op's layout -> numpy complex128 in site-outer order."""
    return op.to_site_outer(op.to_complex(v).to(torch.complex128)).cpu().numpy()


def rounded(v_np, prec):
    """The storage rounding of a complex128 array in precision prec (so the
    oracle sees exactly the input the kernel reads)."""
    t = torch.from_numpy(np.ascontiguousarray(v_np))
    if prec == D.F64:
        return v_np
    if prec == D.F32:
        return t.to(torch.complex64).to(torch.complex128).numpy()
    dt = torch.bfloat16 if prec == D.BF16 else torch.float16
    r = torch.view_as_real(t).to(dt).to(torch.float64)
    return torch.view_as_complex(r.contiguous()).numpy()


def golden_flops():
    """tests/golden/app_e_flops_per_site.txt as {operator: (nc, flops, flops_nv12 or None, polynomial)}."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "app_e_flops_per_site.txt")
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, nc, f, f12, poly = line.split()
        out[name] = (int(nc), int(f), None if f12 == "-" else int(f12), poly)
    return out
