"""FP64 CPU oracle for the multi-RHS Dirac operators and solvers of
Duerr, arXiv:2112.14640.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.  It shares no
code with the CUDA path.

The stencils live in ``oracle.c`` (plain loops over the paper's equations);
this module adds the composite operators the paper builds from them
(D^dagger = gamma5 D gamma5 or epsilon D epsilon, D^dagger D), textbook CG and
BiCGstab with the paper's recompute/exit rules (Sec. 9), the Lanczos
condition estimate of the ``cond`` module (App. F), the App. E flop counts,
the clover term of Eq. (def_clov), the Laplace operators, stout smearing and
the fermion forces of S = phi^dag (D^dag D)^-1 phi for D_W, D_S and D_B (derived here; the
paper has none).

Array shapes (complex128, C order):
  links  U   (Nt, Nz, Ny, Nx, 4, Nc, Nc)      mu = 0..3 <-> x, y, z, t
  W links    (Nt, Nz, Ny, Nx, 81, Nc, Nc)     see ``oracle.c`` for dir numbering
  field strength F (Nt, Nz, Ny, Nx, 6, Nc, Nc) planes (mu,nu) = PLANES
  Wilson-type vectors (Nt, Nz, Ny, Nx, Nc, 4, Nv)
  staggered vectors   (Nt, Nz, Ny, Nx, Nc, Nv)
``dims`` is always (Nx, Ny, Nz, Nt).
"""
import ctypes
import itertools
import math
import os

import numpy as np

from . import build as _build

_lib = None

WILSON, BRILLOUIN, STAGGERED = 0, 1, 2
# Laplace operators A = -1/2 Lap + m^2/2 (Secs. 6, 7; App. F wlap, blap, wsuv, bsuv):
# standard / Brillouin Laplacian on Wilson-type (4 spins) or colour-only vectors
WLAP, BLAP, WSUV, BSUV = 3, 4, 5, 6
KIND_NAMES = {WILSON: "wilson", BRILLOUIN: "brillouin", STAGGERED: "staggered",
              WLAP: "wlap", BLAP: "blap", WSUV: "wsuv", BSUV: "bsuv"}
LAPLACE = (WLAP, BLAP, WSUV, BSUV)


def spins(kind):
    """Spin components per colour of the kind's vectors."""
    return 1 if kind in (STAGGERED, WSUV, BSUV) else 4


def uses_w(kind):
    return kind in (BRILLOUIN, BLAP, BSUV)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        P = ctypes.c_void_p
        I4 = ctypes.POINTER(ctypes.c_int)
        I = ctypes.c_int
        D = ctypes.c_double
        _lib.orc_phase_links.argtypes = [I4, I, I4, P, P]
        _lib.orc_wilson.argtypes = [I4, I, I, P, D, P, P]
        _lib.orc_staggered.argtypes = [I4, I, I, P, D, P, P]
        _lib.orc_brillouin.argtypes = [I4, I, I, P, D, P, P]
        _lib.orc_build_w.argtypes = [I4, I, P, P]
        _lib.orc_gamma5.argtypes = [I4, I, I, P, P]
        _lib.orc_epsilon.argtypes = [I4, I, I, P, P]
        _lib.orc_gamma.argtypes = [I, P]
        _lib.orc_wilson_sites.argtypes = [I4, I, I, P, D, P, P, ctypes.c_long, P]
        _lib.orc_staggered_sites.argtypes = [I4, I, I, P, D, P, P, ctypes.c_long, P]
        _lib.orc_brillouin_sites.argtypes = [I4, I, I, P, D, P, P, ctypes.c_long, P]
        _lib.orc_build_w_sites.argtypes = [I4, I, P, P, ctypes.c_long, P]
        _lib.orc_field_strength.argtypes = [I4, I, P, P]
        _lib.orc_wlap.argtypes = [I4, I, I, I, P, D, P, P]
        _lib.orc_blap.argtypes = [I4, I, I, I, P, D, P, P]
        _lib.orc_wlap_sites.argtypes = [I4, I, I, I, P, D, P, P, ctypes.c_long, P]
        _lib.orc_blap_sites.argtypes = [I4, I, I, I, P, D, P, P, ctypes.c_long, P]
        for f in (_lib.orc_wlap, _lib.orc_blap, _lib.orc_wlap_sites, _lib.orc_blap_sites,
                  _lib.orc_field_strength, _lib.orc_phase_links, _lib.orc_wilson, _lib.orc_staggered, _lib.orc_brillouin,
                  _lib.orc_build_w, _lib.orc_gamma5, _lib.orc_epsilon, _lib.orc_gamma,
                  _lib.orc_wilson_sites, _lib.orc_staggered_sites, _lib.orc_brillouin_sites,
                  _lib.orc_build_w_sites):
            f.restype = None
    return _lib


def _i4(v):
    return (ctypes.c_int * 4)(*[int(a) for a in v])


def _p(a):
    assert a.dtype == np.complex128 and a.flags.c_contiguous
    return ctypes.c_void_p(a.ctypes.data)


def _dims_of_links(U):
    nt, nz, ny, nx = U.shape[:4]
    return (nx, ny, nz, nt), U.shape[-1]


# ----------------------------------------------------------------- primitives

def gamma(mu):
    """4x4 chiral gamma matrix gamma_{mu+1} (App. A)."""
    g = np.zeros((4, 4), np.complex128)
    lib().orc_gamma(int(mu), _p(g))
    return g


def phase_links(U, bc):
    """Links with the boundary phase bc[mu] folded into U_mu(n) where n_mu = N_mu - 1."""
    dims, nc = _dims_of_links(U)
    U = np.ascontiguousarray(U, np.complex128)
    out = np.empty_like(U)
    lib().orc_phase_links(_i4(dims), nc, _i4(bc), _p(U), _p(out))
    return out


def build_w(Up):
    """All 81 W_s(n) (Tab. off-axis) from phased links, by k!-path enumeration."""
    dims, nc = _dims_of_links(Up)
    Up = np.ascontiguousarray(Up, np.complex128)
    W = np.empty(Up.shape[:4] + (81, nc, nc), np.complex128)
    lib().orc_build_w(_i4(dims), nc, _p(Up), _p(W))
    return W


def _stencil(fn, dims, nc, nv, field, m0, v):
    v = np.ascontiguousarray(v, np.complex128)
    out = np.empty_like(v)
    fn(_i4(dims), nc, nv, _p(np.ascontiguousarray(field)), float(m0), _p(v), _p(out))
    return out


def wilson(Up, m0, psi):
    """Eq. (app_wils) with already-phased links."""
    dims, nc = _dims_of_links(Up)
    return _stencil(lib().orc_wilson, dims, nc, psi.shape[-1], Up, m0, psi)


def staggered(Up, m0, phi):
    """Eq. (def_stag) with already-phased links."""
    dims, nc = _dims_of_links(Up)
    return _stencil(lib().orc_staggered, dims, nc, phi.shape[-1], Up, m0, phi)


def brillouin(W, m0, psi):
    """Eq. (app_bril) with W from ``build_w``."""
    nt, nz, ny, nx = W.shape[:4]
    nc = W.shape[-1]
    return _stencil(lib().orc_brillouin, (nx, ny, nz, nt), nc, psi.shape[-1], W, m0, psi)


def laplace(kind, field, m, v):
    """A v for the Laplace kinds, Eq. (app_wlap) (field = phased links) or
    Eq. (app_blap) (field = W from ``build_w``)."""
    nt, nz, ny, nx = v.shape[:4]
    nc, nv = v.shape[4], v.shape[-1]
    v = np.ascontiguousarray(v, np.complex128)
    out = np.empty_like(v)
    fn = lib().orc_blap if uses_w(kind) else lib().orc_wlap
    fn(_i4((nx, ny, nz, nt)), nc, spins(kind), nv, _p(np.ascontiguousarray(field)), float(m), _p(v), _p(out))
    return out


def _sites_arr(sites):
    a = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    return a, ctypes.c_void_p(a.ctypes.data), len(a)


def build_w_sites(Up, sites):
    """The 81 W_s(n) at the listed sites only: shape (len(sites), 81, Nc, Nc)."""
    dims, nc = _dims_of_links(Up)
    Up = np.ascontiguousarray(Up, np.complex128)
    a, pa, ns = _sites_arr(sites)
    W = np.empty((ns, 81, nc, nc), np.complex128)
    lib().orc_build_w_sites(_i4(dims), nc, _p(Up), pa, ns, _p(W))
    return W


def stencil_sites(kind, field, m0, v, sites):
    """(D v)(n) for n in sites; field = phased links (Wilson, staggered, WLAP,
    WSUV) or build_w_sites(...) of the same sites (Brillouin, BLAP, BSUV); for
    the Laplace kinds m0 is the mass m of A.  Returns (len(sites),) + v.shape[4:]."""
    nt, nz, ny, nx = v.shape[:4]
    nc, nv = v.shape[4], v.shape[-1]
    v = np.ascontiguousarray(v, np.complex128)
    a, pa, ns = _sites_arr(sites)
    out = np.empty((ns,) + v.shape[4:], np.complex128)
    if kind in LAPLACE:
        fn = lib().orc_blap_sites if uses_w(kind) else lib().orc_wlap_sites
        fn(_i4((nx, ny, nz, nt)), nc, spins(kind), nv, _p(np.ascontiguousarray(field)), float(m0), _p(v), pa, ns,
           _p(out))
        return out
    fn = {WILSON: lib().orc_wilson_sites, STAGGERED: lib().orc_staggered_sites,
          BRILLOUIN: lib().orc_brillouin_sites}[kind]
    fn(_i4((nx, ny, nz, nt)), nc, nv, _p(np.ascontiguousarray(field)), float(m0), _p(v), pa, ns, _p(out))
    return out


# planes of the clover term, in the paper's order (1,2),(1,3),(1,4),(2,3),(2,4),(3,4)
PLANES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def field_strength(U):
    """Clover-leaf F_mu,nu(n) = (Q - Q^dag) / (8i) for the six PLANES (Sec. 5;
    the leaf sum Q is the reading stated in ``oracle.c``)."""
    dims, nc = _dims_of_links(U)
    U = np.ascontiguousarray(U, np.complex128)
    F = np.empty(U.shape[:4] + (6, nc, nc), np.complex128)
    lib().orc_field_strength(_i4(dims), nc, _p(U), _p(F))
    return F


def sigma(mu, nu):
    """sigma_mu,nu = (i/2) [gamma_mu, gamma_nu] (Sec. 5), from the 4x4 gammas."""
    a, b = gamma(mu), gamma(nu)
    return 0.5j * (a @ b - b @ a)


def clover(F, csw, psi):
    """C psi of Eq. (def_clov): -(c_SW / 2) sum_{mu<nu} (sigma_mu,nu (x) F_mu,nu(n)) psi(n),
    site by site.  F has shape (..., 6, Nc, Nc) and psi (..., Nc, 4, Nv) over
    the same leading (site) axes."""
    out = np.zeros(np.broadcast_shapes(psi.shape), np.complex128)
    for k, (mu, nu) in enumerate(PLANES):
        out += np.einsum("st,...ab,...btv->...asv", sigma(mu, nu), F[..., k, :, :], psi)
    return -0.5 * csw * out


def _shift_links(U, mu, k):
    """U(n + k mu-hat) for a field shaped (Nt, Nz, Ny, Nx, ...)."""
    return np.roll(U, -k, axis=3 - mu)


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def _expi_herm(Q):
    """exp(i Q) of hermitian matrices by eigendecomposition (numpy eigh)."""
    w, v = np.linalg.eigh(Q)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), v.conj())


def stout_smear(U, rho=0.12, nsteps=3):
    """nsteps steps of stout smearing (Morningstar and Peardon, the smearing the
    paper's V comes from, Sec. 2 and App. F), all links updated at once:
      C_mu(n) = rho sum_{nu != mu} [ U_nu(n) U_mu(n+nu) U_nu(n+mu)^dag
                                   + U_nu(n-nu)^dag U_mu(n-nu) U_nu(n-nu+mu) ],
      Omega = C_mu(n) U_mu(n)^dag,
      Q = (i/2)(Omega^dag - Omega) - (i/2N) Tr(Omega^dag - Omega),
      U_mu(n) <- exp(i Q) U_mu(n).
    Periodic field without boundary phases (closed loops make the step commute
    with them)."""
    V = np.array(U, np.complex128)
    nc = V.shape[-1]
    for _ in range(nsteps):
        new = np.empty_like(V)
        for mu in range(4):
            Umu = V[..., mu, :, :]
            C = np.zeros_like(Umu)
            for nu in range(4):
                if nu == mu:
                    continue
                Unu = V[..., nu, :, :]
                C += Unu @ _shift_links(Umu, nu, 1) @ _dag(_shift_links(Unu, mu, 1))
                Unu_b = _shift_links(Unu, nu, -1)
                C += _dag(Unu_b) @ _shift_links(Umu, nu, -1) @ _shift_links(_shift_links(Unu, nu, -1), mu, 1)
            Om = rho * C @ _dag(Umu)
            D = _dag(Om) - Om
            Q = 0.5j * D - (0.5j / nc) * np.trace(D, axis1=-2, axis2=-1)[..., None, None] * np.eye(nc)
            new[..., mu, :, :] = _expi_herm(Q) @ Umu
        V = new
    return V


def _expi_frechet(Q, G):
    """L(iQ, G), the Frechet derivative of the matrix exponential at iQ (Q
    hermitian) in the direction G, by the Daleckii-Krein formula in the
    eigenbasis Q = V diag(w) V^dag: L = V [F o (V^dag G V)] V^dag with the
    divided differences F_jk = (e^{i w_j} - e^{i w_k}) / (i w_j - i w_k)
    = e^{i (w_j + w_k)/2} sinc((w_j - w_k)/2) (e^{i w_j} on the diagonal).
    It also gives the adjoint: tr[L(iQ, E) G] = tr[E L(iQ, G)]."""
    w, v = np.linalg.eigh(Q)
    h = 0.5 * (w[..., :, None] - w[..., None, :])
    F = np.exp(0.5j * (w[..., :, None] + w[..., None, :])) * np.sinc(h / np.pi)
    Gt = _dag(v) @ G @ v
    return v @ (F * Gt) @ _dag(v)


def _stout_parts(U, mu, rho):
    """Staple sum C (times rho), Q and exp(iQ) of one stout step for links mu."""
    nc = U.shape[-1]
    Umu = U[..., mu, :, :]
    C = np.zeros_like(Umu)
    for nu in range(4):
        if nu == mu:
            continue
        Unu = U[..., nu, :, :]
        C += Unu @ _shift_links(Umu, nu, 1) @ _dag(_shift_links(Unu, mu, 1))
        C += _dag(_shift_links(Unu, nu, -1)) @ _shift_links(Umu, nu, -1) @ _shift_links(_shift_links(Unu, nu, -1), mu, 1)
    C = rho * C
    Om = C @ _dag(Umu)
    D = _dag(Om) - Om
    Q = 0.5j * D - (0.5j / nc) * np.trace(D, axis1=-2, axis2=-1)[..., None, None] * np.eye(nc)
    return C, Q, _expi_herm(Q)


def stout_backward(U, G_V, rho=0.12, nsteps=3):
    """Chain rule of the link derivative through nsteps stout steps (derived
    here; the paper only cites the smearing): given G_V with
    dS = Re sum conj(G_V) dV for V = stout_smear(U), returns G_U with
    dS = Re sum conj(G_U) dU.  In the form dS = Re sum tr[dV Sigma'] (Sigma'
    = G_V^dag) one step V = exp(iQ) U, Q from Omega = C U^dag, gives
      Sigma = Sigma' e^{iQ} - C^dag Xi  plus the staple terms of Y = U^dag Xi,
      Xi = the anti-hermitian part of Lambda - tr(Lambda)/N,
      Lambda = L(iQ, U Sigma')            (tr[d e^{iQ} U Sigma'] = tr[i dQ Lambda]),
    and every link in the staples of C_mu(x) receives the derivative of
    rho tr[d(staple) Y_mu(x)], one term per factor (the dagger of the
    transported product for a factor that enters daggered).  The
    intermediate fields are recomputed from U."""
    fields = [np.array(U, np.complex128)]
    for _ in range(nsteps):
        fields.append(stout_smear(fields[-1], rho, 1))
    Sig = _dag(np.asarray(G_V, np.complex128))
    sh = lambda A, mu, k: _shift_links(A, mu, k)
    for i in reversed(range(nsteps)):
        Uin = fields[i]
        new = np.zeros_like(Sig)
        Y = np.zeros_like(Sig)
        for mu in range(4):
            C, Q, E = _stout_parts(Uin, mu, rho)
            Umu = Uin[..., mu, :, :]
            Lam = _expi_frechet(Q, Umu @ Sig[..., mu, :, :])
            nc = Lam.shape[-1]
            Lp = Lam - (np.trace(Lam, axis1=-2, axis2=-1) / nc)[..., None, None] * np.eye(nc)
            Xi = 0.5 * (Lp - _dag(Lp))
            new[..., mu, :, :] += Sig[..., mu, :, :] @ E - _dag(C) @ Xi
            Y[..., mu, :, :] = _dag(Umu) @ Xi
        for mu in range(4):
            Ym = Y[..., mu, :, :]
            Umu = Uin[..., mu, :, :]
            for nu in range(4):
                if nu == mu:
                    continue
                Unu = Uin[..., nu, :, :]
                # up staple U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag of link (x, mu)
                new[..., nu, :, :] += rho * sh(Umu, nu, 1) @ _dag(sh(Unu, mu, 1)) @ Ym
                new[..., mu, :, :] += rho * sh(_dag(sh(Unu, mu, 1)) @ Ym @ Unu, nu, -1)
                new[..., nu, :, :] += rho * sh(_dag(Ym @ Unu @ sh(Umu, nu, 1)), mu, -1)
                # down staple U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) of link (x, mu)
                Unb, Umb = sh(Unu, nu, -1), sh(Umu, nu, -1)
                Unbm = sh(Unb, mu, 1)
                new[..., nu, :, :] += rho * sh(_dag(Umb @ Unbm @ Ym), nu, 1)
                new[..., mu, :, :] += rho * sh(Unbm @ Ym @ _dag(Unb), nu, 1)
                new[..., nu, :, :] += rho * sh(sh(Ym @ _dag(Unb) @ Umb, nu, 1), mu, -1)
        Sig = new
    return _dag(Sig)


def gamma5(psi):
    nt, nz, ny, nx, nc, _, nv = psi.shape
    psi = np.ascontiguousarray(psi, np.complex128)
    out = np.empty_like(psi)
    lib().orc_gamma5(_i4((nx, ny, nz, nt)), nc, nv, _p(psi), _p(out))
    return out


def epsilon(phi):
    nt, nz, ny, nx, nc, nv = phi.shape
    phi = np.ascontiguousarray(phi, np.complex128)
    out = np.empty_like(phi)
    lib().orc_epsilon(_i4((nx, ny, nz, nt)), nc, nv, _p(phi), _p(out))
    return out


# ------------------------------------------------------------ operator object

class Operator:
    """D in {D_W, D_B, D_S} on a fixed gauge field, with its dagger and D^dag D.

    D_W^dag = gamma5 D_W gamma5, D_B^dag = gamma5 D_B gamma5 and
    D_S^dag = epsilon D_S epsilon, the forms the paper's solvers use (App. F).
    With csw != 0 (Wilson and Brillouin) the clover term C of Eq. (def_clov),
    built from the field strength of the gauge field V (default: U), is added:
    v = (D + C) u, as in Eqs. (def_wils) and (def_bril).
    The Laplace kinds (WLAP, BLAP, WSUV, BSUV) apply A = -1/2 Lap + m^2/2 with
    m = m0; A is hermitian, so its dagger is A itself.
    """

    def __init__(self, kind, U, bc=(1, 1, 1, 1), m0=0.0, csw=0.0, V=None):
        self.kind = kind
        self.m0 = float(m0)
        self.bc = tuple(int(b) for b in bc)
        self.Up = phase_links(U, self.bc)
        self._W = None
        self.csw = float(csw)
        self.F = None
        if self.csw != 0.0:
            if kind not in (WILSON, BRILLOUIN):
                raise ValueError("the clover term acts on Wilson-type vectors only")
            self.F = field_strength(U if V is None else V)

    @property
    def W(self):
        """All 81 W links (Brillouin-type kinds), built on first use."""
        if self._W is None and uses_w(self.kind):
            self._W = build_w(self.Up)
        return self._W

    def apply(self, v, m0=None):
        m = self.m0 if m0 is None else m0
        if self.kind in LAPLACE:
            return laplace(self.kind, self.W if uses_w(self.kind) else self.Up, m, v)
        if self.kind == WILSON:
            out = wilson(self.Up, m, v)
        elif self.kind == BRILLOUIN:
            out = brillouin(self.W, m, v)
        else:
            return staggered(self.Up, m, v)
        if self.F is not None:
            out = out + clover(self.F, self.csw, v)
        return out

    def apply_sites(self, v, sites, m0=None, dagger=False):
        """(D v)(n) or (D^dag v)(n) at the listed site indices only."""
        m = self.m0 if m0 is None else m0
        if uses_w(self.kind):
            field = build_w_sites(self.Up, sites)
        else:
            field = self.Up
        if self.kind in LAPLACE:
            return stencil_sites(self.kind, field, m, v, sites)
        if not dagger:
            return stencil_sites(self.kind, field, m, v, sites) + self._clover_sites(v, sites)
        out = stencil_sites(self.kind, field, m, self._sandwich(v), sites) + \
            self._clover_sites(self._sandwich(v), sites)
        if self.kind == STAGGERED:
            nt, nz, ny, nx = v.shape[:4]
            s = np.asarray(sites)
            x, y, z, t = s % nx, (s // nx) % ny, (s // (nx * ny)) % nz, s // (nx * ny * nz)
            eps = np.where((x + y + z + t) % 2 == 1, -1.0, 1.0)
            return out * eps[:, None, None]
        out = out.copy()
        out[:, :, 2:, :] *= -1
        return out

    def _clover_sites(self, v, sites):
        if self.F is None:
            return 0.0
        s = np.asarray(sites)
        return clover(self.F.reshape((-1,) + self.F.shape[4:])[s], self.csw,
                      v.reshape((-1,) + v.shape[4:])[s])

    def _sandwich(self, v):
        return epsilon(v) if self.kind == STAGGERED else gamma5(v)

    def apply_dagger(self, v, m0=None):
        if self.kind in LAPLACE:
            return self.apply(v, m0)
        return self._sandwich(self.apply(self._sandwich(v), m0))

    def apply_normal(self, v, m0=None):
        return self.apply_dagger(self.apply(v, m0), m0)


# ------------------------------------------------------------- BLAS-1 helpers

def norm2(v):
    """Per-RHS squared 2-norms (last axis = RHS), accumulated in FP64."""
    a = v.reshape(-1, v.shape[-1])
    return np.sum(a.real ** 2 + a.imag ** 2, axis=0)


def dot(u, v):
    """Per-RHS <u, v>, linear in the second argument (Sec. 3 convention)."""
    a = u.reshape(-1, u.shape[-1])
    b = v.reshape(-1, v.shape[-1])
    return np.sum(np.conj(a) * b, axis=0)


# --------------------------------------------------------------------- solvers

CONVERGED, MAXIT, STAGNATED, BREAKDOWN = 0, 1, 2, 3


def cg(apply_A, b, x0=None, tol=1e-10, maxit=10000, recompute_every=50):
    """CG on an HPD operator, one independent recursion per RHS (Sec. 9).

    Recompute r = b - A x when the iteration count is a multiple of
    ``recompute_every``, when every active RHS's updated residual passes tol,
    or at maxit.  Exit when every RHS's recomputed residual passes, when the
    updated and recomputed norms of an unconverged RHS differ by more than
    1%, or at maxit.  Reading for the paper's silent point: an RHS whose
    recomputed residual passes is frozen (alpha = beta = 0).
    Returns (x, info) with info holding iterations, recomputes, status, the
    per-RHS CG coefficients (for the Lanczos estimate) and final residuals.
    """
    nv = b.shape[-1]
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.complex128)
    nb = np.sqrt(norm2(b))
    r = b - apply_A(x)
    p = r.copy()
    rr = norm2(r)
    active = np.sqrt(rr) >= tol * nb
    alphas, betas = [], []
    it = recomputes = 0
    status = CONVERGED
    while active.any():
        it += 1
        q = apply_A(p)
        pq = dot(p, q).real
        alpha = np.where(active, rr / np.where(active, pq, 1.0), 0.0)
        x += alpha * p
        r -= alpha * q
        rr_new = norm2(r)
        alphas.append(alpha.copy())
        if (it % recompute_every == 0 or np.all(np.sqrt(rr_new[active]) < tol * nb[active])
                or it >= maxit):
            recomputes += 1
            rt = b - apply_A(x)
            rr_true = norm2(rt)
            disc = np.abs(np.sqrt(rr_new) - np.sqrt(rr_true)) / np.maximum(np.sqrt(rr_true), 1e-300)
            r = rt
            rr_new = rr_true
            active &= ~(np.sqrt(rr_true) < tol * nb)
            if not active.any():
                break
            if np.any(disc[active] > 0.01):
                status = STAGNATED
                break
            if it >= maxit:
                status = MAXIT
                break
        beta = np.where(active, rr_new / np.where(active, rr, 1.0), 0.0)
        betas.append(beta.copy())
        p = r + beta * p
        rr = rr_new
    res = np.sqrt(norm2(b - apply_A(x))) / nb
    return x, dict(iters=it, recomputes=recomputes, status=status, relres=res,
                   alphas=np.array(alphas).reshape(-1, nv), betas=np.array(betas).reshape(-1, nv))


def cg_normal(op, b, x0=None, tol=1e-10, maxit=10000, recompute_every=50, m0=None):
    """Solve D^dag D x = D^dag b by CG; stopping on ||r_N|| / ||D^dag b|| < tol.

    Reading (the paper's residual is defined for the system being solved):
    the normal-equation residual decides convergence; the true ||b - D x|| / ||b||
    is reported beside it as ``true_relres``.
    """
    bN = op.apply_dagger(b, m0)
    x, info = cg(lambda v: op.apply_normal(v, m0), bN, x0, tol, maxit, recompute_every)
    info["true_relres"] = np.sqrt(norm2(b - op.apply(x, m0))) / np.sqrt(norm2(b))
    return x, info


def bicgstab(op, b, x0=None, tol=1e-10, maxit=10000, recompute_every=50, m0=None):
    """BiCGstab (van der Vorst) on D x = b per RHS, shadow residual r_hat = r_0.

    Same recompute/exit rules as ``cg``; breakdown (|rho| or |omega| below
    1e-30 of its scale) marks that RHS as BREAKDOWN and freezes it.
    """
    nv = b.shape[-1]
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.complex128)
    nb = np.sqrt(norm2(b))
    r = b - op.apply(x, m0)
    rhat = r.copy()
    rho = np.ones(nv, np.complex128)
    alpha = np.ones(nv, np.complex128)
    omega = np.ones(nv, np.complex128)
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    active = np.sqrt(norm2(r)) >= tol * nb
    broken = np.zeros(nv, bool)
    it = recomputes = 0
    status = CONVERGED
    while active.any():
        it += 1
        rho_new = dot(rhat, r)
        bad = active & (np.abs(rho_new) < 1e-30 * np.sqrt(norm2(rhat) * norm2(r)))
        broken |= bad
        active &= ~bad
        a_ = active
        beta = np.where(a_, (rho_new / np.where(a_, rho, 1)) * (alpha / np.where(a_, omega, 1)), 0)
        p = np.where(a_, r + beta * (p - omega * v), p)
        v = op.apply(p, m0)
        rv = dot(rhat, v)
        alpha = np.where(a_, rho_new / np.where(a_, rv, 1), 0)
        s = r - alpha * v
        t = op.apply(s, m0)
        tt = norm2(t)
        omega = np.where(a_, dot(t, s) / np.where(a_ & (tt > 0), tt, 1), 0)
        bad = a_ & (np.abs(omega) < 1e-30)
        broken |= bad
        x = x + np.where(a_, alpha * p + omega * s, 0)
        r = np.where(a_, s - omega * t, r)
        rho = np.where(a_, rho_new, rho)
        active &= ~bad
        rr = norm2(r)
        if (it % recompute_every == 0 or np.all(np.sqrt(rr[active]) < tol * nb[active])
                or it >= maxit):
            recomputes += 1
            rt = b - op.apply(x, m0)
            rr_true = norm2(rt)
            disc = np.abs(np.sqrt(rr) - np.sqrt(rr_true)) / np.maximum(np.sqrt(rr_true), 1e-300)
            r = rt
            active &= ~(np.sqrt(rr_true) < tol * nb)
            if not active.any():
                break
            if np.any(disc[active] > 0.01):
                status = STAGNATED
                break
            if it >= maxit:
                status = MAXIT
                break
    if broken.any() and status == CONVERGED:
        status = BREAKDOWN
    res = np.sqrt(norm2(b - op.apply(x, m0))) / nb
    return x, dict(iters=it, recomputes=recomputes, status=status, relres=res, broken=broken)


def lanczos_tridiagonal(alphas, betas):
    """Lanczos matrix of CG (the ``cond`` module, App. F), one per RHS.

    With CG coefficients alpha_j, beta_j: diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1},
    off-diagonal sqrt(beta_j)/alpha_j.  Returns a list of (diag, offdiag).
    """
    out = []
    alphas = np.asarray(alphas)
    betas = np.asarray(betas)
    for i in range(alphas.shape[1]):
        a = alphas[:, i]
        k = int(np.count_nonzero(a))
        a = a[:k]
        b = betas[:max(k - 1, 0), i]
        diag = 1.0 / a
        diag[1:] += b / a[:-1]
        off = np.sqrt(b) / a[:-1]
        out.append((diag, off))
    return out


def lanczos_cond(alphas, betas):
    """(lambda_min, lambda_max) per RHS from the CG Lanczos matrix."""
    res = []
    for diag, off in lanczos_tridiagonal(alphas, betas):
        T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
        ev = np.linalg.eigvalsh(T)
        res.append((ev[0], ev[-1]))
    return np.array(res)


# --------------------------------------------------------------- force
# The paper has no force; this is derived for S = sum_v phi_v^dag (D_W^dag D_W)^-1 phi_v.
# With psi = (D^dag D)^-1 phi and chi = D psi, dS = -2 Re <chi, dD psi>.  Only
# the two hops through U_mu(n) depend on it:
#   forward  at n:     -1/2 (1 - gamma_mu) U_mu(n) psi(n+mu)
#   backward at n+mu:  -1/2 (1 + gamma_mu) U_mu(n)^dag psi(n)
# so with the colour matrices (spin and RHS summed)
#   B_mu(n) = sum psi(n+mu) [(1 - gamma_mu) chi(n)]^dag,
#   C_mu(n) = sum psi(n) [(1 + gamma_mu) chi(n+mu)]^dag
# one finds dS = Re sum tr[dU_mu(n) (B_mu(n) + C_mu(n)^dag)].  For U -> exp(eps X) U,
# X in su(N): dS/deps = Re sum tr[X M] with M = U B - C U^dag, and only the
# traceless anti-hermitian part F = P_TA(M) contributes.

def _proj(chi, mu, sign):
    """(1 + sign*gamma_mu) applied in spinor space to a Wilson-type vector."""
    g = gamma(mu)
    return chi + sign * np.einsum("st,...ctv->...csv", g, chi)


def _shift(v, mu, step):
    """v(n + step*mu), periodic (axes of the vector: t, z, y, x first)."""
    ax = {0: 3, 1: 2, 2: 1, 3: 0}[mu]
    return np.roll(v, -step, axis=ax)


def wilson_force_terms(op, psi, chi):
    """(B, C) per link, each of shape (Nt, Nz, Ny, Nx, 4, Nc, Nc)."""
    if op.F is not None:
        raise ValueError("the force is derived for D_W without the clover term")
    sh = psi.shape[:4] + (4, psi.shape[4], psi.shape[4])
    B = np.empty(sh, np.complex128)
    C = np.empty(sh, np.complex128)
    for mu in range(4):
        B[..., mu, :, :] = np.einsum("...asv,...bsv->...ab", _shift(psi, mu, 1), np.conj(_proj(chi, mu, -1)))
        C[..., mu, :, :] = np.einsum("...asv,...bsv->...ab", psi, np.conj(_proj(_shift(chi, mu, 1), mu, +1)))
    return B, C


def staggered_force_terms(op, phi, chi):
    """(B, C) per link for S = sum_v Re phi_v^dag (D_S^dag D_S)^-1 phi_v, from
    psi = (D^dag D)^-1 phi (here ``phi``) and chi = D psi, derived from
    Eq. (def_stag): dS = -2 Re <chi, dD psi> and the two hops through U_mu(n)
    give dS = Re sum tr[dU (B + C^dag)] with
      B_mu(n) = -eta_mu(n) sum_v psi(n+mu) chi(n)^dag,
      C_mu(n) =  eta_mu(n) sum_v psi(n) chi(n+mu)^dag
    (eta_mu depends only on the coordinates before mu, so eta_mu(n+mu) =
    eta_mu(n)).  Colour-vector fields (Nt, Nz, Ny, Nx, Nc, Nv)."""
    nt, nz, ny, nx = phi.shape[:4]
    t, z, y, x = np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    co = [x, y, z, t]
    sh = phi.shape[:4] + (4, phi.shape[4], phi.shape[4])
    B = np.empty(sh, np.complex128)
    C = np.empty(sh, np.complex128)
    for mu in range(4):
        e = sum(co[nu] + 1 for nu in range(mu))
        eta = np.where(np.asarray(e) % 2 == 1, -1.0, 1.0)[..., None, None]
        fwd = lambda v: np.roll(v, -1, axis=3 - mu)
        B[..., mu, :, :] = -eta * np.einsum("...av,...bv->...ab", fwd(phi), np.conj(chi))
        C[..., mu, :, :] = eta * np.einsum("...av,...bv->...ab", phi, np.conj(fwd(chi)))
    return B, C


def staggered_force(op, psi, chi):
    """F_mu(n) = P_TA(U B - C U^dag) with the staggered B, C and phased links."""
    B, C = staggered_force_terms(op, psi, chi)
    U = op.Up
    return project_ta(U @ B - C @ np.conj(np.swapaxes(U, -1, -2)))


def staggered_action_gradient(op, psi, chi):
    """G with dS = Re sum conj(G) dU for the unphased links: bc-phase * (B^dag + C)."""
    B, C = staggered_force_terms(op, psi, chi)
    ph = phase_links(np.ones(op.Up.shape, np.complex128), op.bc)
    return (np.conj(np.swapaxes(B, -1, -2)) + C) * ph


def _roll_sites(A, o):
    """A(n + o) for a field with leading axes (t, z, y, x) and an offset o = (ox, oy, oz, ot)."""
    return np.roll(A, shift=(-o[3], -o[2], -o[1], -o[0]), axis=(0, 1, 2, 3))


def brillouin_force_terms(op, psi, chi):
    """K_mu(n) with dS = Re sum tr[dU_mu(n) K_mu(n)] for S = sum_v Re phi_v^dag
    (D_B^dag D_B)^-1 phi_v, psi = (D^dag D)^-1 phi, chi = D_B psi (derived here;
    the paper has no force).  From Eq. (app_bril), dS = -2 Re <chi, dD psi> and
    dD psi(n) = sum_s S_s (x) dW_s(n) psi(n+s) with the spin factor
    S_s = rho_k sum_mu s_mu gamma_mu - lambda_k/2, so
      dS = -2 Re sum_{n,s} tr[dW_s(n) M_s(n)],  M_s(n) = sum_v (S_s psi(n+s)) chi(n)^dag
    (spin contracted).  W_s(n) is the average of the k! hop orderings of
    Tab. off-axis; the derivative of one ordering's product P_1 ... P_k is
    sum_j P_<j dV_j P_>j, so link j of the path receives (-2/k!) P_>j M_s P_<j
    for a forward hop (V = U_mu(m)) and its dagger for a backward hop
    (V = U_mu(m - mu)^dag).  Uses the operator's phased links."""
    Up = op.Up
    nc = Up.shape[-1]
    g = [gamma(mu) for mu in range(4)]
    K = np.zeros_like(Up)
    dag = lambda A: np.conj(np.swapaxes(A, -1, -2))
    eye = np.broadcast_to(np.eye(nc, dtype=np.complex128), Up.shape[:4] + (nc, nc))
    for s in itertools.product((-1, 0, 1), repeat=4):
        s = s[::-1]   # (sx, sy, sz, st) with st slowest, any order will do
        axes = [mu for mu in range(4) if s[mu] != 0]
        k = len(axes)
        if k == 0:
            continue
        S = sum(RHO_B[k] * s[mu] * g[mu] for mu in axes) - 0.5 * LAM_B[k] * np.eye(4)
        Spsi = np.einsum("ab,...cbv->...cav", S, _roll_sites(psi, s))
        M = np.einsum("...bav,...cav->...bc", Spsi, np.conj(chi))      # colour (b, c)
        for order in itertools.permutations(axes):
            hops, o = [], [0, 0, 0, 0]
            for mu in order:
                sg = s[mu]
                if sg > 0:
                    V = _roll_sites(Up[..., mu, :, :], o)
                else:
                    om = list(o)
                    om[mu] -= 1
                    V = dag(_roll_sites(Up[..., mu, :, :], om))
                hops.append((mu, sg, list(o), V))
                o[mu] += sg
            pre = [eye]
            for (_, _, _, V) in hops:
                pre.append(pre[-1] @ V)
            post = [eye]
            for (_, _, _, V) in reversed(hops):
                post.append(V @ post[-1])
            post = post[::-1]   # post[j] = product of hops j .. k-1
            c = -2.0 / math.factorial(k)
            for j, (mu, sg, oj, V) in enumerate(hops):
                X = post[j + 1] @ M @ pre[j]
                if sg > 0:   # link U_mu at n + o_j: value at site m is X(m - o_j)
                    K[..., mu, :, :] += c * _roll_sites(X, [-a for a in oj])
                else:        # link U_mu at n + o_j - mu, entering as its dagger
                    om = [-a for a in oj]
                    om[mu] += 1
                    K[..., mu, :, :] += c * dag(_roll_sites(X, om))
    return K


def brillouin_force(op, psi, chi):
    """F_mu(n) = P_TA(U K): dS/deps = Re sum tr[X F] for U -> exp(eps X) U."""
    return project_ta(op.Up @ brillouin_force_terms(op, psi, chi))


def brillouin_action_gradient(op, psi, chi):
    """G with dS = Re sum conj(G) dU for the unphased links: bc-phase * K^dag."""
    K = brillouin_force_terms(op, psi, chi)
    ph = phase_links(np.ones(op.Up.shape, np.complex128), op.bc)
    return np.conj(np.swapaxes(K, -1, -2)) * ph


RHO_B = {1: 64.0 / 432.0, 2: 16.0 / 432.0, 3: 4.0 / 432.0, 4: 1.0 / 432.0}
LAM_B = {1: 8.0 / 64.0, 2: 4.0 / 64.0, 3: 2.0 / 64.0, 4: 1.0 / 64.0}


def project_ta(M):
    """Traceless anti-hermitian part of each colour matrix."""
    A = 0.5 * (M - np.conj(np.swapaxes(M, -1, -2)))
    n = M.shape[-1]
    tr = np.trace(A, axis1=-2, axis2=-1) / n
    return A - tr[..., None, None] * np.eye(n)


def wilson_force(op, psi, chi):
    """F_mu(n) = P_TA(U B - C U^dag) with the operator's phased links."""
    B, C = wilson_force_terms(op, psi, chi)
    U = op.Up
    M = U @ B - C @ np.conj(np.swapaxes(U, -1, -2))
    return project_ta(M)


def wilson_action_gradient(op, psi, chi):
    """dS/dU in the convention dS = Re sum conj(G) dU for the unphased links:
    G = bc-phase * (B^dag + C)."""
    B, C = wilson_force_terms(op, psi, chi)
    G = np.conj(np.swapaxes(B, -1, -2)) + C
    ph = phase_links(np.ones(op.Up.shape, np.complex128), op.bc)
    return G * ph


def pseudofermion_action(op, phi, m0=None, tol=1e-13, maxit=20000):
    """S = sum_v Re phi_v^dag (D^dag D)^-1 phi_v and the solution psi."""
    psi, info = cg(lambda v: op.apply_normal(v, m0), phi, None, tol, maxit, 50)
    return float(np.sum(np.real(np.conj(phi) * psi))), psi


# ------------------------------------------------------------ App. E counts

def clover_flops_per_site(nc, multiplications=2):
    """Flops per site per RHS of the clover term (App. E): 192Nc^2 with one
    colour multiplication per plane, 64Nc^2 with the sigma_mu,nu structure
    used (two multiplications per chiral half), the count the paper's code
    adds to D_W and D_B when c_SW > 0."""
    if multiplications == 6:
        return ((8 * nc * nc - 2 * nc) + 2 * nc) * 4 * 6
    return ((8 * nc * nc - 2 * nc) + 2 * nc) * 4 * 2


def flops_per_site(kind, nc):
    """Flops per site per RHS (App. E): Wilson 128Nc^2+72Nc, Brillouin
    2560Nc^2+2376Nc, staggered 64Nc^2+2Nc; Laplace operators on Wilson-type
    vectors 256Nc^2+8Nc (standard) and 2560Nc^2+648Nc (Brillouin), a quarter
    of that on colour-only vectors."""
    if kind == WLAP:
        return 256 * nc * nc + 8 * nc
    if kind == WSUV:
        return 64 * nc * nc + 2 * nc
    if kind == BLAP:
        return 2560 * nc * nc + 648 * nc
    if kind == BSUV:
        return 640 * nc * nc + 162 * nc
    if kind == WILSON:
        return 128 * nc * nc + 72 * nc
    if kind == BRILLOUIN:
        return 2560 * nc * nc + 2376 * nc
    return 64 * nc * nc + 2 * nc
