"""Thin ctypes binding of ``include/dirac.h`` (libdirac.so).

Argument marshalling only: torch tensors supply device memory and the CUDA
stream; every step of every operation runs in the library's CUDA kernels.
There is no fallback: if libdirac.so is missing or no GPU is present the
calls raise.

Vector tensors (device, C-contiguous), layout SITE_OUTER (the paper's order):
  F64  complex128  Wilson-type (Nt, Nz, Ny, Nx, Nc, 4, Nv), colour-only (Nt, Nz, Ny, Nx, Nc, Nv)
  F32  complex64   same shapes
layout SITE_INNER: Wilson-type (Nc, 4, Nt, Nz, Ny, Nx, Nv), colour-only (Nc, Nt, Nz, Ny, Nx, Nv).
Wilson-type: WILSON, BRILLOUIN, WLAP, BLAP; colour-only: STAGGERED, WSUV, BSUV.
  BF16 bfloat16    same shapes + trailing (re, im) axis of length 2
  F16  float16     same shapes + trailing (re, im) axis of length 2
Gauge field U: complex128 or complex64, (Nt, Nz, Ny, Nx, 4, Nc, Nc), no boundary phases.
"""
import ctypes
import os

import torch

from . import build as _build

WILSON, BRILLOUIN, STAGGERED = 0, 1, 2
# Laplace operators A = -1/2 Lap + m^2/2 (standard / Brillouin Laplacian) on
# Wilson-type vectors (WLAP, BLAP) or colour-only vectors (WSUV, BSUV)
WLAP, BLAP, WSUV, BSUV = 3, 4, 5, 6
LAPLACE = (WLAP, BLAP, WSUV, BSUV)
F64, F32, BF16, F16 = 0, 1, 2, 3
CG_NORMAL, BICGSTAB, CG_HPD = 0, 1, 2
MIXED_RELIABLE, MIXED_RESTART, MIXED_ADAPTIVE = 0, 1, 2
FORCE_TA, FORCE_GRAD = 0, 1
PREC_NAMES = {F64: "f64", F32: "f32", BF16: "bf16", F16: "f16"}
KIND_NAMES = {WILSON: "wilson", BRILLOUIN: "brillouin", STAGGERED: "staggered",
              WLAP: "wlap", BLAP: "blap", WSUV: "wsuv", BSUV: "bsuv"}
_TORCH_DTYPE = {F64: torch.complex128, F32: torch.complex64, BF16: torch.bfloat16, F16: torch.float16}


SITE_OUTER, SITE_INNER = 0, 1   # vector layouts (include/dirac.h)
LINKS_NATIVE, LINKS_F32 = 0, 1  # link storage of 16-bit operators


class Geom(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("nc", ctypes.c_int), ("nv", ctypes.c_int),
                ("bc", ctypes.c_int * 4), ("prec", ctypes.c_int), ("layout", ctypes.c_int),
                ("link_storage", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("inner_prec", ctypes.c_int), ("inner_tol", ctypes.c_double), ("recompute_every", ctypes.c_int),
                ("mixed_mode", ctypes.c_int), ("sloppy_links", ctypes.c_int), ("delta", ctypes.c_double)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("recomputes", ctypes.c_int),
                ("status", ctypes.c_int), ("status_per_rhs", ctypes.c_int * 64), ("relres", ctypes.c_double * 64),
                ("true_relres", ctypes.c_double * 64), ("seconds", ctypes.c_double),
                ("lambda_min", ctypes.c_double * 64), ("lambda_max", ctypes.c_double * 64),
                ("host_launches", ctypes.c_int), ("iters_16bit", ctypes.c_int), ("seconds_16bit", ctypes.c_double)]


class DiracError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (code %d)" % (what, error_string(code), code))
        self.code = code


_lib = None

# every symbol include/dirac.h declares, with its ctypes signature
_P, _I, _D, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
SIGNATURES = {
    "dirac_op_create": (_I, [_I, ctypes.POINTER(Geom), _P, _I, _P, ctypes.POINTER(_P)]),
    "dirac_op_update_links": (_I, [_P, _P, _I, _P]),
    "dirac_op_copy_w": (_I, [_P, _P, _P]),
    "dirac_op_set_clover": (_I, [_P, _D, _P, _I, _P]),
    "dirac_stout_smear": (_I, [_P, _P, ctypes.POINTER(_I), _I, _I, _D, _I, _P]),
    "dirac_stout_backward": (_I, [_P, _P, _P, ctypes.POINTER(_I), _I, _I, _D, _I, _P]),
    "dirac_op_destroy": (None, [_P]),
    "dirac_apply": (_I, [_P, _P, _P, _D, _P]),
    "dirac_apply_dagger": (_I, [_P, _P, _P, _D, _P]),
    "dirac_apply_normal": (_I, [_P, _P, _P, _D, _P]),
    "dirac_apply_host": (_I, [_P, _P, _P, _D, _I, _P]),
    "dirac_apply_host_async": (_I, [_P, _P, _P, _D, _I, _P]),
    "dirac_op_set_launch": (_I, [_P, _I, _I, _I]),
    "dirac_op_get_launch": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "dirac_op_autotune": (_I, [_P, _D, _P, ctypes.POINTER(_D)]),
    "dirac_vec_bytes": (_SZ, [_P]),
    "dirac_vec_norm2": (_I, [_P, _P, _P, _P]),
    "dirac_vec_dot": (_I, [_P, _P, _P, _P, _P]),
    "dirac_vec_axpy": (_I, [_P, _P, _P, _P, _P]),
    "dirac_vec_axpby": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "dirac_vec_norm2_range": (_I, [_P, _P, ctypes.c_longlong, ctypes.c_longlong, _P, _P]),
    "dirac_vec_dot_range": (_I, [_P, _P, _P, ctypes.c_longlong, ctypes.c_longlong, _P, _P]),
    "dirac_vec_gamma5": (_I, [_P, _P, _P]),
    "dirac_vec_convert": (_I, [_P, _P, _I, _P, _I, _P]),
    "dirac_vec_norm2_noalloc": (_I, [_P, _I, ctypes.c_longlong, _I, _P, _P]),
    "dirac_solve": (_I, [_P, _P, _P, _D, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), _P]),
    "dirac_force_wilson": (_I, [_P, _P, _P, _P, _I, _P]),
    "dirac_force": (_I, [_P, _P, _P, _P, _I, _P]),
    "dirac_solve_batched": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                 ctypes.POINTER(_D), ctypes.POINTER(SolveParams), ctypes.POINTER(SolveStats), _P]),
    "dirac_error_string": (ctypes.c_char_p, [_I]),
    "dirac_flops_per_site": (ctypes.c_long, [_I, _I]),
    "dirac_clover_flops_per_site": (ctypes.c_long, [_I]),
    "dirac_version": (_I, []),
    "dirac_measure_fp32_peak": (_I, [_I, ctypes.POINTER(_D), ctypes.POINTER(_I), _P]),
    "dirac_apply_range": (_I, [_P, _P, _P, _D, _I, ctypes.c_longlong, ctypes.c_longlong, _P]),
    "dirac_halo_bytes": (_SZ, [_P, _I]),
    "dirac_halo_pack": (_I, [_P, _P, _I, _I, _P, _P]),
    "dirac_halo_unpack": (_I, [_P, _P, _I, _I, _P, _P]),
}


def lib_path():
    return _build.LIB


def lib():
    """Load libdirac.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("libdirac.so not found at %s: build it with __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def error_string(code):
    return lib().dirac_error_string(int(code)).decode()


def flops_per_site(kind, nc):
    return int(lib().dirac_flops_per_site(int(kind), int(nc)))


def measure_fp32_peak(iters=20000, stream=None):
    """(TFLOP/s, SM count) of the FMA-only probe kernel on the current device."""
    t, n = ctypes.c_double(), ctypes.c_int()
    st = torch.cuda.current_stream() if stream is None else stream
    rc = lib().dirac_measure_fp32_peak(int(iters), ctypes.byref(t), ctypes.byref(n), _P(st.cuda_stream))
    if rc:
        raise DiracError(rc, "dirac_measure_fp32_peak")
    return t.value, n.value


def stout_smear(U, rho=0.12, nsteps=3, out=None, stream=None):
    """nsteps steps of stout smearing of the gauge field U (CUDA tensor,
    complex128 or complex64, (Nt, Nz, Ny, Nx, 4, Nc, Nc), no boundary
    phases); returns V (a new tensor, or ``out``, which may be U itself)."""
    if not U.is_cuda or U.dtype not in (torch.complex128, torch.complex64) or not U.is_contiguous():
        raise ValueError("U must be a contiguous complex128 or complex64 CUDA tensor")
    nt, nz, ny, nx = U.shape[:4]
    out = torch.empty_like(U) if out is None else out
    if out.shape != U.shape or out.dtype != U.dtype or not out.is_contiguous():
        raise ValueError("out must match U")
    dims = (ctypes.c_int * 4)(nx, ny, nz, nt)
    prec = F64 if U.dtype == torch.complex128 else F32
    _check(lib().dirac_stout_smear(_ptr(U), _ptr(out), dims, int(U.shape[-1]), prec, float(rho), int(nsteps),
                                   _stream(stream)), "dirac_stout_smear")
    return out


def stout_backward(U, G_V, rho=0.12, nsteps=3, stream=None):
    """Chain rule through stout smearing (dirac_stout_backward): for
    V = stout_smear(U, rho, nsteps) and G_V with dS = Re sum conj(G_V) dV,
    returns G_U with dS = Re sum conj(G_U) dU (same shape and dtype as U)."""
    if not U.is_cuda or U.dtype not in (torch.complex128, torch.complex64) or not U.is_contiguous():
        raise ValueError("U must be a contiguous complex128 or complex64 CUDA tensor")
    if G_V.shape != U.shape or G_V.dtype != U.dtype or not G_V.is_contiguous():
        raise ValueError("G_V must match U")
    nt, nz, ny, nx = U.shape[:4]
    out = torch.empty_like(U)
    dims = (ctypes.c_int * 4)(nx, ny, nz, nt)
    prec = F64 if U.dtype == torch.complex128 else F32
    _check(lib().dirac_stout_backward(_ptr(U), _ptr(G_V), _ptr(out), dims, int(U.shape[-1]), prec, float(rho),
                                      int(nsteps), _stream(stream)), "dirac_stout_backward")
    return out


def clover_flops_per_site(nc):
    return int(lib().dirac_clover_flops_per_site(int(nc)))


def _check(rc, what):
    if rc < 0:
        raise DiracError(rc, what)
    return rc


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class DiracOp:
    """One of D_W, D_B, D_S on a fixed gauge field, for N_v right-hand sides."""

    def __init__(self, kind, U, nv, bc=(1, 1, 1, 1), prec=F32, stream=None, layout=SITE_OUTER,
                 link_storage=LINKS_NATIVE):
        if not U.is_cuda:
            raise ValueError("U must be a CUDA tensor")
        if U.dtype not in (torch.complex128, torch.complex64):
            raise ValueError("U must be complex128 or complex64")
        U = U.contiguous()
        nt, nz, ny, nx = U.shape[:4]
        self.kind, self.nv, self.prec, self.layout = int(kind), int(nv), int(prec), int(layout)
        self.dims = (nx, ny, nz, nt)
        self.nc = U.shape[-1]
        self.bc = tuple(int(b) for b in bc)
        self.device = U.device
        g = Geom()
        g.dims[:] = self.dims
        g.nc, g.nv, g.prec, g.layout, g.link_storage = self.nc, self.nv, self.prec, self.layout, int(link_storage)
        g.bc[:] = self.bc
        self._geom = g
        self.csw = 0.0
        h = ctypes.c_void_p()
        u_prec = F64 if U.dtype == torch.complex128 else F32
        _check(lib().dirac_op_create(self.kind, ctypes.byref(g), _ptr(U), u_prec, _stream(stream),
                                     ctypes.byref(h)), "dirac_op_create")
        self._h = h

    # ------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.dirac_op_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update_links(self, U, stream=None):
        """New gauge field; a clover term set before is removed."""
        u_prec = F64 if U.dtype == torch.complex128 else F32
        _check(lib().dirac_op_update_links(self._h, _ptr(U.contiguous()), u_prec, _stream(stream)),
               "dirac_op_update_links")
        self.csw = 0.0

    def set_clover(self, csw, V=None, stream=None):
        """Add the clover term of Eq. (def_clov) with coefficient csw, its field
        strength built from the gauge field V (a CUDA tensor shaped like U);
        csw = 0 removes it."""
        if V is None:
            if csw != 0.0:
                raise ValueError("V is required for a non-zero c_SW")
            ptr, v_prec = ctypes.c_void_p(), F64
        else:
            if not V.is_cuda or V.dtype not in (torch.complex128, torch.complex64):
                raise ValueError("V must be a complex128 or complex64 CUDA tensor")
            V = V.contiguous()
            ptr, v_prec = _ptr(V), (F64 if V.dtype == torch.complex128 else F32)
        _check(lib().dirac_op_set_clover(self._h, float(csw), ptr, v_prec, _stream(stream)),
               "dirac_op_set_clover")
        self.csw = float(csw)

    # ---------------------------------------------------------------- shapes
    @property
    def staggered(self):
        return self.kind == STAGGERED

    @property
    def colour_only(self):
        """Vectors without spin components (staggered, WSUV, BSUV)."""
        return self.kind in (STAGGERED, WSUV, BSUV)

    def vector_shape(self, prec=None):
        prec = self.prec if prec is None else prec
        nx, ny, nz, nt = self.dims
        internal = (self.nc,) if self.colour_only else (self.nc, 4)
        if self.layout == SITE_OUTER:
            shape = (nt, nz, ny, nx) + internal + (self.nv,)
        else:
            shape = internal + (nt, nz, ny, nx, self.nv)
        return shape + (2,) if prec in (BF16, F16) else shape

    def _perm(self):
        # axes of a site-outer vector in site-inner order
        return (4, 0, 1, 2, 3, 5) if self.colour_only else (4, 5, 0, 1, 2, 3, 6)

    def from_site_outer(self, v):
        """Reorder a complex tensor given in the paper's site-outer order into this operator's layout."""
        if self.layout == SITE_OUTER:
            return v.contiguous()
        return v.permute(*self._perm()).contiguous()

    def to_site_outer(self, v):
        """Reorder a complex tensor in this operator's layout into the site-outer order."""
        if self.layout == SITE_OUTER:
            return v.contiguous()
        p = self._perm()
        inv = [p.index(i) for i in range(len(p))]
        return v.permute(*inv).contiguous()

    def new_vector(self, prec=None, zero=True):
        prec = self.prec if prec is None else prec
        f = torch.zeros if zero else torch.empty
        return f(self.vector_shape(prec), dtype=_TORCH_DTYPE[prec], device=self.device)

    def to_prec(self, v, prec=None):
        """Torch-side representation change of a complex tensor into the vector
        format of ``prec`` (no arithmetic beyond the storage rounding)."""
        prec = self.prec if prec is None else prec
        if prec in (BF16, F16):
            return torch.view_as_real(v.to(torch.complex64)).to(_TORCH_DTYPE[prec]).contiguous()
        return v.to(_TORCH_DTYPE[prec]).contiguous()

    def to_complex(self, v):
        if v.dtype in (torch.bfloat16, torch.float16):
            return torch.view_as_complex(v.float().contiguous())
        return v

    def set_launch(self, vr, minb=1, block=0):
        """Pick the stencil launch variant (vr RHS per thread, register class minb, threads per block)."""
        _check(lib().dirac_op_set_launch(self._h, int(vr), int(minb), int(block)), "dirac_op_set_launch")

    def get_launch(self):
        vr, mb, bl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().dirac_op_get_launch(self._h, ctypes.byref(vr), ctypes.byref(mb), ctypes.byref(bl)),
               "dirac_op_get_launch")
        return vr.value, mb.value, bl.value

    def autotune(self, m0=0.0, stream=None):
        """Time every compiled launch variant and keep the fastest; returns ms per apply."""
        ms = ctypes.c_double()
        _check(lib().dirac_op_autotune(self._h, float(m0), _stream(stream), ctypes.byref(ms)), "dirac_op_autotune")
        return ms.value

    def vec_bytes(self):
        return int(lib().dirac_vec_bytes(self._h))

    def _vec(self, v, what):
        if tuple(v.shape) != self.vector_shape() or v.dtype != _TORCH_DTYPE[self.prec] or not v.is_contiguous():
            raise ValueError("%s: expected contiguous %s %s, got %s %s" % (
                what, tuple(self.vector_shape()), _TORCH_DTYPE[self.prec], tuple(v.shape), v.dtype))
        return _ptr(v)

    # ---------------------------------------------------------------- apply
    def apply(self, psi, out=None, m0=0.0, dagger=False, stream=None):
        out = self.new_vector(zero=False) if out is None else out
        f = lib().dirac_apply_dagger if dagger else lib().dirac_apply
        _check(f(self._h, self._vec(psi, "psi"), self._vec(out, "out"), float(m0), _stream(stream)), "dirac_apply")
        return out

    def apply_normal(self, psi, out=None, m0=0.0, stream=None):
        out = self.new_vector(zero=False) if out is None else out
        _check(lib().dirac_apply_normal(self._h, self._vec(psi, "psi"), self._vec(out, "out"), float(m0),
                                        _stream(stream)), "dirac_apply_normal")
        return out

    def apply_host(self, host_in, host_out, m0=0.0, dagger=False, stream=None):
        """End-to-end apply on host (CPU, ideally pinned) tensors; blocks."""
        if host_in.is_cuda or host_out.is_cuda:
            raise ValueError("apply_host takes host tensors")
        nb = self.vec_bytes()
        if host_in.numel() * host_in.element_size() != nb or host_out.numel() * host_out.element_size() != nb:
            raise ValueError("host buffers must hold exactly one vector")
        _check(lib().dirac_apply_host(self._h, _ptr(host_in), _ptr(host_out), float(m0), int(bool(dagger)),
                                      _stream(stream)), "dirac_apply_host")
        return host_out

    def apply_range(self, x, out, site0, nsites, m0=0.0, dagger=False, stream=None):
        """D (or D^dag) x for the output sites [site0, site0 + nsites) only
        (dirac_apply_range); the rest of ``out`` is left untouched."""
        _check(lib().dirac_apply_range(self._h, self._vec(x, "x"), self._vec(out, "out"), float(m0),
                                       int(bool(dagger)), int(site0), int(nsites), _stream(stream)),
               "dirac_apply_range")
        return out

    def halo_buffer(self, proj=0):
        """A device buffer for one packed time slice (dirac_halo_bytes)."""
        nb = int(lib().dirac_halo_bytes(self._h, int(proj)))
        if nb == 0:
            raise DiracError(-1, "dirac_halo_bytes")
        return torch.empty(nb, dtype=torch.uint8, device=self.device)

    def halo_pack(self, x, t, buf, proj=0, stream=None):
        _check(lib().dirac_halo_pack(self._h, self._vec(x, "x"), int(t), int(proj), _ptr(buf), _stream(stream)),
               "dirac_halo_pack")
        return buf

    def halo_unpack(self, buf, t, x, proj=0, stream=None):
        _check(lib().dirac_halo_unpack(self._h, _ptr(buf), int(t), int(proj), self._vec(x, "x"), _stream(stream)),
               "dirac_halo_unpack")
        return x

    def apply_host_async(self, host_in, host_out, m0=0.0, dagger=False, stream=None):
        """apply_host without the final synchronisation (dirac_apply_host_async):
        host_out is ready once ``stream`` (torch's current stream by default)
        has reached this point; host applies of different operators overlap."""
        if host_in.is_cuda or host_out.is_cuda:
            raise ValueError("apply_host_async takes host tensors")
        nb = self.vec_bytes()
        if host_in.numel() * host_in.element_size() != nb or host_out.numel() * host_out.element_size() != nb:
            raise ValueError("host buffers must hold exactly one vector")
        _check(lib().dirac_apply_host_async(self._h, _ptr(host_in), _ptr(host_out), float(m0), int(bool(dagger)),
                                            _stream(stream)), "dirac_apply_host_async")
        return host_out

    def copy_w(self, stream=None):
        """The 80 stored W links (Brillouin): (Nt, Nz, Ny, Nx, 80, Nc, Nc[, 2])."""
        nx, ny, nz, nt = self.dims
        if self.layout == SITE_OUTER:
            shape = (nt, nz, ny, nx, 80, self.nc, self.nc)
        else:
            shape = (80, self.nc, self.nc, nt, nz, ny, nx)
        if self.prec in (BF16, F16):
            shape = shape + (2,)
        w = torch.empty(shape, dtype=_TORCH_DTYPE[self.prec], device=self.device)
        _check(lib().dirac_op_copy_w(self._h, _ptr(w), _stream(stream)), "dirac_op_copy_w")
        return w

    # ---------------------------------------------------------------- BLAS-1
    def norm2(self, v, stream=None):
        out = torch.empty(self.nv, dtype=torch.float64, device=self.device)
        _check(lib().dirac_vec_norm2(self._h, self._vec(v, "v"), _ptr(out), _stream(stream)), "dirac_vec_norm2")
        return out

    def dot(self, u, v, stream=None):
        out = torch.empty(self.nv, dtype=torch.complex128, device=self.device)
        _check(lib().dirac_vec_dot(self._h, self._vec(u, "u"), self._vec(v, "v"), _ptr(out), _stream(stream)),
               "dirac_vec_dot")
        return out

    def axpy(self, alpha, x, y, stream=None):
        a = alpha.to(device=self.device, dtype=torch.complex128).contiguous()
        _check(lib().dirac_vec_axpy(self._h, _ptr(a), self._vec(x, "x"), self._vec(y, "y"), _stream(stream)),
               "dirac_vec_axpy")
        return y

    def axpby(self, a, x, b, y, z=None, stream=None):
        """z = a x + b y per RHS (a, b: N_v complex coefficients; z may be x or y)."""
        z = self.new_vector(zero=False) if z is None else z
        a = a.to(device=self.device, dtype=torch.complex128).contiguous()
        b = b.to(device=self.device, dtype=torch.complex128).contiguous()
        _check(lib().dirac_vec_axpby(self._h, _ptr(a), self._vec(x, "x"), _ptr(b), self._vec(y, "y"),
                                     self._vec(z, "z"), _stream(stream)), "dirac_vec_axpby")
        return z

    def norm2_range(self, v, site0, nsites, stream=None):
        """Per-RHS |v|^2 over the sites [site0, site0 + nsites) only."""
        out = torch.empty(self.nv, dtype=torch.float64, device=self.device)
        _check(lib().dirac_vec_norm2_range(self._h, self._vec(v, "v"), int(site0), int(nsites), _ptr(out),
                                           _stream(stream)), "dirac_vec_norm2_range")
        return out

    def dot_range(self, u, v, site0, nsites, stream=None):
        """Per-RHS <u, v> over the sites [site0, site0 + nsites) only."""
        out = torch.empty(self.nv, dtype=torch.complex128, device=self.device)
        _check(lib().dirac_vec_dot_range(self._h, self._vec(u, "u"), self._vec(v, "v"), int(site0), int(nsites),
                                         _ptr(out), _stream(stream)), "dirac_vec_dot_range")
        return out

    def gamma5_(self, v, stream=None):
        _check(lib().dirac_vec_gamma5(self._h, self._vec(v, "v"), _stream(stream)), "dirac_vec_gamma5")
        return v

    def convert(self, src, src_prec, dst_prec, stream=None):
        dst = self.new_vector(prec=dst_prec, zero=False)
        _check(lib().dirac_vec_convert(self._h, _ptr(src.contiguous()), int(src_prec), _ptr(dst), int(dst_prec),
                                       _stream(stream)), "dirac_vec_convert")
        return dst

    def force(self, psi, chi, mode=FORCE_TA, stream=None):
        """Link derivative of S = sum Re phi^dag (D^dag D)^-1 phi (Wilson or staggered):
        (Nt, Nz, Ny, Nx, 4, Nc, Nc) complex, from psi = (D^dag D)^-1 phi, chi = D psi."""
        nx, ny, nz, nt = self.dims
        out = torch.empty((nt, nz, ny, nx, 4, self.nc, self.nc), dtype=_TORCH_DTYPE[self.prec], device=self.device)
        _check(lib().dirac_force(self._h, self._vec(psi, "psi"), self._vec(chi, "chi"), _ptr(out), int(mode),
                                 _stream(stream)), "dirac_force")
        return out

    # ---------------------------------------------------------------- solve
    def solve(self, b, x=None, m0=0.0, solver=CG_NORMAL, tol=1e-10, maxit=10000, inner_prec=None,
              inner_tol=0.0, recompute_every=0, mixed_mode=MIXED_RELIABLE, delta=0.0, sloppy_links=LINKS_NATIVE,
              stream=None):
        """Solve D x = b (BiCGstab), D^dag D x = D^dag b (CG_NORMAL) or D^dag D x = b
        (CG_HPD) for all RHS.  Returns (x, stats dict); non-convergence is
        reported in the stats."""
        x = self.new_vector() if x is None else x
        p = SolveParams(int(solver), float(tol), int(maxit), int(self.prec if inner_prec is None else inner_prec),
                        float(inner_tol), int(recompute_every), int(mixed_mode), int(sloppy_links), float(delta))
        st = SolveStats()
        rc = _check(lib().dirac_solve(self._h, self._vec(b, "b"), self._vec(x, "x"), float(m0), ctypes.byref(p),
                                      ctypes.byref(st), _stream(stream)), "dirac_solve")
        nv = self.nv
        stats = dict(code=rc, status=st.status, iters=st.iters, outer_iters=st.outer_iters,
                     recomputes=st.recomputes, status_per_rhs=list(st.status_per_rhs[:nv]),
                     relres=list(st.relres[:nv]), true_relres=list(st.true_relres[:nv]), seconds=st.seconds,
                     lambda_min=list(st.lambda_min[:nv]), lambda_max=list(st.lambda_max[:nv]),
                     iters_16bit=st.iters_16bit, seconds_16bit=st.seconds_16bit)
        return x, stats


def solve_batched(ops, bs, xs=None, m0s=None, solver=CG_NORMAL, tol=1e-6, maxit=20000, recompute_every=0,
                  stream=None):
    """Run independent CG solves (one per operator) as one graph-captured batch.
    Returns (xs, list of per-solve stats dicts, return code)."""
    n = len(ops)
    xs = [op.new_vector() for op in ops] if xs is None else xs
    m0s = [0.0] * n if m0s is None else m0s
    P = ctypes.c_void_p
    h = (P * n)(*[op._h for op in ops])
    pb = (P * n)(*[op._vec(b, "b") for op, b in zip(ops, bs)])
    px = (P * n)(*[op._vec(x, "x") for op, x in zip(ops, xs)])
    pm = (ctypes.c_double * n)(*[float(m) for m in m0s])
    prm = SolveParams(int(solver), float(tol), int(maxit), int(ops[0].prec), 0.0, int(recompute_every), 0, 0, 0.0)
    st = (SolveStats * n)()
    rc = _check(lib().dirac_solve_batched(n, h, pb, px, pm, ctypes.byref(prm), st, _stream(stream)),
                "dirac_solve_batched")
    out = []
    for op, s in zip(ops, st):
        nv = op.nv
        out.append(dict(status=s.status, iters=s.iters, relres=list(s.relres[:nv]),
                        status_per_rhs=list(s.status_per_rhs[:nv]), seconds=s.seconds,
                        host_launches=s.host_launches))
    return xs, out, rc
