"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expectation is a closed
form (free-field momentum-space symbols), an identity the operators must obey
(gamma5-hermiticity, anti-hermiticity of the staggered hop, gauge covariance,
W_{-s}(n) = W_s(n-s)^dag), a value the paper prints (the App. D eta phases,
the App. E flop counts, the free-field spectral edges of Sec. 9), or a
library routine on a dense brute-force matrix.
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O
from paper_2112_14640_gb300 import inputs as I

# Pauli matrices and the tensor-product form of the chiral gammas (App. A),
# built here independently of the oracle's own tables.
S0 = np.eye(2, dtype=complex)
S1 = np.array([[0, 1], [1, 0]], complex)
S2 = np.array([[0, -1j], [1j, 0]], complex)
S3 = np.array([[1, 0], [0, -1]], complex)
GAMMA = [np.kron(S2, S1), np.kron(S2, S2), np.kron(S2, S3), np.kron(S1, S0)]
G5 = np.diag([1, 1, -1, -1]).astype(complex)


def plane_wave(dims, p, chi):
    """psi(n) = exp(i p.n) chi, chi of shape (Nc, 4, Nv) or (Nc, Nv)."""
    nx, ny, nz, nt = dims
    t, z, y, x = np.meshgrid(np.arange(nt), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[(...,) + (None,) * chi.ndim] * chi


def momenta(dims, bc, rng, count):
    out = []
    for _ in range(count):
        p = []
        for mu in range(4):
            k = rng.integers(0, dims[mu])
            p.append(np.pi * (2 * k + 1) / dims[mu] if bc[mu] < 0 else 2 * np.pi * k / dims[mu])
        out.append(np.array(p))
    return out


def wilson_symbol(p, m0):
    return (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))


def brillouin_symbol(p, m0):
    lap = m0 + 2.0 * (1.0 - np.prod(np.cos(p / 2) ** 2))
    der = sum(GAMMA[m] * np.sin(p[m]) * np.prod([2 + np.cos(p[n]) for n in range(4) if n != m]) / 27.0
              for m in range(4))
    return lap * np.eye(4) + 1j * der


# ------------------------------------------------------------- gamma matrices

def test_gammas_match_app_a_tensor_form_and_clifford():
    for mu in range(4):
        assert np.allclose(O.gamma(mu), GAMMA[mu], atol=0, rtol=0)
    for a in range(4):
        for b in range(4):
            anti = GAMMA[a] @ GAMMA[b] + GAMMA[b] @ GAMMA[a]
            assert np.allclose(anti, 2 * np.eye(4) * (a == b))
    g5 = O.gamma(0) @ O.gamma(1) @ O.gamma(2) @ O.gamma(3)
    assert np.allclose(g5, G5)


# ---------------------------------------------------------------- free fields

@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 1, 1, -1)])
@pytest.mark.parametrize("nc", [1, 3])
def test_wilson_free_field_symbol(bc, nc):
    dims = (4, 4, 2, 6)
    rng = np.random.default_rng(3)
    m0 = 0.1
    op = O.Operator(O.WILSON, I.unit_gauge_field(dims, nc), bc, m0)
    for p in momenta(dims, bc, rng, 6):
        chi = rng.standard_normal((nc, 4, 2)) + 1j * rng.standard_normal((nc, 4, 2))
        out = op.apply(plane_wave(dims, p, chi))
        want = plane_wave(dims, p, np.einsum("st,ctv->csv", wilson_symbol(p, m0), chi))
        assert np.abs(out - want).max() < 1e-13


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 1, 1, -1)])
def test_brillouin_free_field_symbol(bc):
    dims = (4, 2, 4, 6)
    rng = np.random.default_rng(4)
    m0 = -0.3
    op = O.Operator(O.BRILLOUIN, I.unit_gauge_field(dims, 3), bc, m0)
    for p in momenta(dims, bc, rng, 6):
        chi = rng.standard_normal((3, 4, 3)) + 1j * rng.standard_normal((3, 4, 3))
        out = op.apply(plane_wave(dims, p, chi))
        want = plane_wave(dims, p, np.einsum("st,ctv->csv", brillouin_symbol(p, m0), chi))
        assert np.abs(out - want).max() < 1e-13


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 1, 1, -1), (-1, 1, -1, -1)])
def test_staggered_normal_free_field(bc):
    """D_S^dag D_S = m^2 + sum_mu sin^2 p_mu on every plane wave."""
    dims = (4, 4, 6, 4)
    rng = np.random.default_rng(5)
    m0 = 0.05
    op = O.Operator(O.STAGGERED, I.unit_gauge_field(dims, 3), bc, m0)
    for p in momenta(dims, bc, rng, 6):
        chi = rng.standard_normal((3, 2)) + 1j * rng.standard_normal((3, 2))
        psi = plane_wave(dims, p, chi)
        out = op.apply_normal(psi)
        assert np.abs(out - (m0 ** 2 + np.sum(np.sin(p) ** 2)) * psi).max() < 1e-13


def test_free_spectral_edges_sec9():
    """Sec. 9: free D_B reaches Re z = 2 + m0, free D_W reaches 8 + m0 (at p = pi)."""
    m0 = 0.01
    p = np.full(4, np.pi)
    assert np.allclose(np.linalg.eigvals(brillouin_symbol(p, m0)).real, 2 + m0)
    assert np.allclose(np.linalg.eigvals(wilson_symbol(p, m0)).real, 8 + m0)
    # and through the oracle on a 2^4 lattice, where p = pi is a lattice momentum
    dims = (2, 2, 2, 2)
    chi = np.zeros((3, 4, 1), complex)
    chi[1, 2, 0] = 1
    for kind, edge in ((O.WILSON, 8 + m0), (O.BRILLOUIN, 2 + m0)):
        op = O.Operator(kind, I.unit_gauge_field(dims, 3), (1, 1, 1, 1), m0)
        psi = plane_wave(dims, p, chi)
        assert np.allclose(op.apply(psi), edge * psi, atol=1e-13)


def test_staggered_eta_phases_app_d():
    """App. D: eta_2 = -1 at (1-based) x = 1, eta_4 = -1 at x = y = z = 1, eta_3 = +1 there."""
    dims = (4, 4, 4, 4)
    op = O.Operator(O.STAGGERED, I.unit_gauge_field(dims, 1), (1, 1, 1, 1), 0.0)
    phi = np.zeros((4, 4, 4, 4, 1, 1), complex)
    phi[0, 0, 0, 0] = 1.0
    out = op.apply(phi)[..., 0, 0]
    # out[t, z, y, x]; neighbours of the origin reached by the forward hop
    assert np.isclose(out[0, 0, 0, 3], +0.5)   # n = -x, eta_1 = 1
    assert np.isclose(out[0, 0, 3, 0], -0.5)   # n = -y, eta_2 = (-1)^1
    assert np.isclose(out[0, 3, 0, 0], +0.5)   # n = -z, eta_3 = (-1)^(1+1)
    assert np.isclose(out[3, 0, 0, 0], -0.5)   # n = -t, eta_4 = (-1)^(1+1+1)
    assert np.isclose(out[0, 0, 1, 0], +0.5)   # n = +y, backward hop: -eta_2/2
    assert np.isclose(np.abs(out).sum(), 4.0)


# ------------------------------------------------------ identities on random U

def _dotc(a, b):
    return np.vdot(a.ravel(), b.ravel())


@pytest.mark.parametrize("kind", [O.WILSON, O.BRILLOUIN])
@pytest.mark.parametrize("nc", [2, 3])
def test_gamma5_hermiticity(kind, nc):
    dims = (4, 2, 2, 4)
    U = I.gauge_field(dims, nc, 0.4, seed=11)
    op = O.Operator(kind, U, (1, 1, 1, -1), 0.1)
    phi = I.source(dims, nc, 2, seed=1)
    psi = I.source(dims, nc, 2, seed=2)
    lhs = _dotc(phi, O.gamma5(op.apply(psi)))
    rhs = np.conj(_dotc(psi, O.gamma5(op.apply(phi))))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    # the dagger used by the solvers is the adjoint
    assert abs(_dotc(phi, op.apply(psi)) - _dotc(op.apply_dagger(phi), psi)) < 1e-11 * abs(lhs)


def test_staggered_hop_antihermitian_and_dagger():
    dims = (4, 4, 2, 2)
    U = I.gauge_field(dims, 3, 0.4, seed=12)
    op0 = O.Operator(O.STAGGERED, U, (1, 1, 1, -1), 0.0)
    phi = I.source(dims, 3, 2, seed=3, staggered=True)
    psi = I.source(dims, 3, 2, seed=4, staggered=True)
    a = _dotc(phi, op0.apply(psi))
    b = _dotc(psi, op0.apply(phi))
    assert abs(a + np.conj(b)) < 1e-12 * abs(a)
    op = O.Operator(O.STAGGERED, U, (1, 1, 1, -1), 0.3)
    assert abs(_dotc(phi, op.apply(psi)) - _dotc(op.apply_dagger(phi), psi)) < 1e-11 * abs(a)


def _transform_links(U, Om):
    """U^Omega_mu(n) = Omega(n) U_mu(n) Omega(n+mu)^dag."""
    out = np.empty_like(U)
    for mu, ax in enumerate((3, 2, 1, 0)):
        Om_f = np.roll(Om, -1, axis=ax)
        out[..., mu, :, :] = Om @ U[..., mu, :, :] @ np.conj(np.swapaxes(Om_f, -1, -2))
    return out


@pytest.mark.parametrize("kind", [O.WILSON, O.BRILLOUIN, O.STAGGERED])
def test_gauge_covariance(kind):
    dims = (4, 2, 4, 2)
    nc = 3
    U = I.gauge_field(dims, nc, 0.5, seed=21)
    Om = I.gauge_transform(dims, nc, seed=22)
    stag = kind == O.STAGGERED
    psi = I.source(dims, nc, 2, seed=23, staggered=stag)
    bc = (1, -1, 1, -1)
    op = O.Operator(kind, U, bc, 0.2)
    opg = O.Operator(kind, _transform_links(U, Om), bc, 0.2)
    rot = (lambda v: np.einsum("...ab,...bv->...av", Om, v)) if stag else \
          (lambda v: np.einsum("...ab,...bsv->...asv", Om, v))
    lhs = opg.apply(rot(psi))
    rhs = rot(op.apply(psi))
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


# ------------------------------------------------------------- W-link facts

def _offset(d):
    return np.array([d % 3 - 1, (d // 3) % 3 - 1, (d // 9) % 3 - 1, (d // 27) % 3 - 1])


def test_w_reflection_and_unitarity():
    dims = (4, 4, 2, 4)
    U = I.gauge_field(dims, 3, 0.4, seed=31)
    W = O.build_w(O.phase_links(U, (1, 1, -1, -1)))
    eye = np.eye(3)
    assert np.allclose(W[..., 40, :, :], eye)
    nonunit = 0
    for d in range(81):
        if d == 40:
            continue
        s = _offset(d)
        k = int(np.abs(s).sum())
        # W_{-s}(n) = W_s(n - s)^dag  (Tab. off-axis caption)
        Ws_shift = np.roll(W[..., d, :, :], shift=(s[3], s[2], s[1], s[0]), axis=(0, 1, 2, 3))
        assert np.abs(W[..., 80 - d, :, :] - np.conj(np.swapaxes(Ws_shift, -1, -2))).max() < 1e-14
        dev = np.abs(W[..., d, :, :] @ np.conj(np.swapaxes(W[..., d, :, :], -1, -2)) - eye).max()
        if k == 1:
            assert dev < 1e-13
        else:
            assert dev > 1e-3
            nonunit += 1
    assert nonunit == 72   # 36 of the 40 stored directions, plus their reflections


def test_w_commuting_constant_links():
    """For constant commuting (diagonal) links every path gives prod_mu U_mu^{s_mu}:
    pins the 1/k! normalisation and the orientation of each hop."""
    dims = (3, 3, 3, 3)
    rng = np.random.default_rng(8)
    th = rng.uniform(-np.pi, np.pi, (4, 3))
    th[:, 2] = -th[:, 0] - th[:, 1]
    U = np.zeros((3, 3, 3, 3, 4, 3, 3), complex)
    for mu in range(4):
        U[..., mu, :, :] = np.diag(np.exp(1j * th[mu]))
    W = O.build_w(O.phase_links(U, (1, 1, 1, 1)))
    for d in range(81):
        s = _offset(d)
        want = np.diag(np.exp(1j * (s @ th)))
        assert np.abs(W[..., d, :, :] - want).max() < 1e-13


def test_w_gauge_covariance():
    dims = (2, 4, 2, 4)
    U = I.gauge_field(dims, 3, 0.5, seed=41)
    Om = I.gauge_transform(dims, 3, seed=42)
    W = O.build_w(U)
    Wg = O.build_w(_transform_links(U, Om))
    for d in (0, 13, 22, 39, 44, 62, 80):
        s = _offset(d)
        Om_s = np.roll(Om, shift=(-s[3], -s[2], -s[1], -s[0]), axis=(0, 1, 2, 3))
        want = Om @ W[..., d, :, :] @ np.conj(np.swapaxes(Om_s, -1, -2))
        assert np.abs(Wg[..., d, :, :] - want).max() < 1e-13


# ------------------------------------------------------- dense brute force

def dense(apply, shape):
    n = int(np.prod(shape))
    cols = []
    for j in range(n):
        e = np.zeros(n, complex)
        e[j] = 1
        cols.append(apply(e.reshape(shape)).ravel())
    return np.array(cols).T


@pytest.mark.parametrize("kind", [O.WILSON, O.BRILLOUIN, O.STAGGERED])
def test_dense_2x4_dagger_is_conjugate_transpose(kind):
    """2^4 lattice: every offset aliases onto another site; the matrix of the
    dagger must still be the conjugate transpose of the matrix of D."""
    dims = (2, 2, 2, 2)
    U = I.gauge_field(dims, 3, 0.4, seed=51)
    op = O.Operator(kind, U, (1, 1, 1, -1), 0.1)
    shape = (2, 2, 2, 2, 3, 1) if kind == O.STAGGERED else (2, 2, 2, 2, 3, 4, 1)
    D = dense(op.apply, shape)
    Dd = dense(op.apply_dagger, shape)
    assert np.abs(Dd - D.conj().T).max() < 1e-13


# ---------------------------------------------------------------- solvers

@pytest.mark.parametrize("kind", [O.WILSON, O.BRILLOUIN, O.STAGGERED])
def test_cg_normal_matches_dense_solve(kind):
    dims = (2, 2, 2, 4)
    U = I.gauge_field(dims, 3, 0.4, seed=61)
    op = O.Operator(kind, U, (1, 1, 1, -1), 0.1)
    stag = kind == O.STAGGERED
    b = I.source(dims, 3, 3, seed=62, staggered=stag)
    x, info = O.cg_normal(op, b, tol=1e-12, maxit=2000)
    assert info["status"] == O.CONVERGED
    shape1 = b.shape[:-1] + (1,)
    D = dense(op.apply, shape1)
    for v in range(3):
        xv = np.linalg.solve(D, b[..., v].ravel())
        assert np.abs(x[..., v].ravel() - xv).max() < 1e-9 * np.abs(xv).max()
    assert np.all(info["true_relres"] < 1e-10)


@pytest.mark.parametrize("kind", [O.WILSON, O.BRILLOUIN])
def test_bicgstab_matches_dense_solve(kind):
    dims = (2, 2, 4, 2)
    U = I.gauge_field(dims, 3, 0.4, seed=71)
    op = O.Operator(kind, U, (1, 1, 1, -1), 0.2)
    b = I.source(dims, 3, 2, seed=72)
    x, info = O.bicgstab(op, b, tol=1e-12, maxit=2000)
    assert info["status"] == O.CONVERGED
    D = dense(op.apply, b.shape[:-1] + (1,))
    for v in range(2):
        xv = np.linalg.solve(D, b[..., v].ravel())
        assert np.abs(x[..., v].ravel() - xv).max() < 1e-9 * np.abs(xv).max()


def test_lanczos_condition_estimate_matches_dense_spectrum():
    dims = (4, 2, 2, 4)
    U = I.gauge_field(dims, 3, 0.4, seed=81)
    op = O.Operator(O.STAGGERED, U, (1, 1, 1, -1), 0.05)
    b = I.source(dims, 3, 2, seed=82, staggered=True)
    bN = op.apply_dagger(b)
    x, info = O.cg(op.apply_normal, bN, tol=1e-13, maxit=5000, recompute_every=10 ** 6)
    est = O.lanczos_cond(info["alphas"], info["betas"])
    A = dense(op.apply_normal, b.shape[:-1] + (1,))
    ev = np.linalg.eigvalsh(0.5 * (A + A.conj().T))
    for lo, hi in est:
        assert abs(hi - ev[-1]) < 1e-6 * ev[-1]
        assert abs(lo - ev[0]) < 1e-3 * ev[0]


def test_cg_stagnation_rule_reports_discrepancy():
    """A CG fed an operator with a deliberate rounding (float32 products) must
    stop on the 1% updated-vs-recomputed rule rather than run to maxit (Sec. 9)."""
    dims = (2, 2, 2, 4)
    U = I.gauge_field(dims, 3, 0.4, seed=91)
    op = O.Operator(O.WILSON, U, (1, 1, 1, -1), 0.01)

    def A32(v):
        r = op.apply_normal(v.astype(np.complex64).astype(np.complex128))
        return r.astype(np.complex64).astype(np.complex128)

    b = I.source(dims, 3, 2, seed=92)
    x, info = O.cg(A32, b, tol=1e-12, maxit=5000, recompute_every=20)
    assert info["status"] == O.STAGNATED
    assert info["iters"] < 5000


# ------------------------------------------------------------ App. E counts

def test_flop_counts_app_e():
    """The oracle's flop counts against the values and N_c polynomials App. E
    prints (tests/golden/app_e_flops_per_site.txt)."""
    from helpers import golden_flops
    kinds = {"wilson": O.WILSON, "brillouin": O.BRILLOUIN, "staggered": O.STAGGERED}
    for name, (nc, flops, flops12, poly) in golden_flops().items():
        assert O.flops_per_site(kinds[name], nc) == flops
        if flops12 is not None:
            assert 12 * O.flops_per_site(kinds[name], nc) == flops12
        for n in (1, 2, 3, 4):
            assert O.flops_per_site(kinds[name], n) == eval(poly.replace("^", "**"), {"nc": n})


# ------------------------------------------------------------- fermion force

def _expm_ah(X):
    """exp of anti-hermitian matrices via eigendecomposition of the Hermitian -iX."""
    w, v = np.linalg.eigh(-1j * X)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), v.conj())


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 1, 1, -1)])
def test_force_matches_finite_differences(bc):
    """dS/deps along U -> exp(eps X) U equals Re sum tr[X F] (central differences,
    eps = 1e-4, FP64 solves to 1e-13) for random su(3) directions X."""
    dims = (4, 2, 2, 4)
    m0 = 0.3
    U = I.gauge_field(dims, 3, 0.4, seed=101)
    phi = I.source(dims, 3, 2, seed=102)
    op = O.Operator(O.WILSON, U, bc, m0)
    S0, psi = O.pseudofermion_action(op, phi)
    F = O.wilson_force(op, psi, op.apply(psi))
    assert np.allclose(F, -np.conj(np.swapaxes(F, -1, -2)), atol=1e-14)
    assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-13
    eps = 1e-4
    for seed in range(4):
        X = I.su_n_direction(dims, 3, seed=200 + seed)
        Sp, _ = O.pseudofermion_action(O.Operator(O.WILSON, _expm_ah(eps * X) @ U, bc, m0), phi)
        Sm, _ = O.pseudofermion_action(O.Operator(O.WILSON, _expm_ah(-eps * X) @ U, bc, m0), phi)
        fd = (Sp - Sm) / (2 * eps)
        an = np.sum(np.real(np.einsum("...ab,...ba->...", X, F)))
        assert abs(fd - an) < 1e-6 * max(abs(an), 1.0), (seed, fd, an)


def test_action_gradient_matches_finite_differences():
    """The complex gradient G (dS = Re sum conj(G) dU) against central differences
    along an arbitrary complex perturbation dU (off the group manifold too)."""
    dims = (2, 2, 2, 4)
    m0, bc = 0.4, (1, 1, 1, -1)
    U = I.gauge_field(dims, 3, 0.4, seed=111)
    phi = I.source(dims, 3, 1, seed=112)
    op = O.Operator(O.WILSON, U, bc, m0)
    S0, psi = O.pseudofermion_action(op, phi)
    G = O.wilson_action_gradient(op, psi, op.apply(psi))
    rng = np.random.default_rng(5)
    dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    eps = 1e-5
    Sp, _ = O.pseudofermion_action(O.Operator(O.WILSON, U + eps * dU, bc, m0), phi)
    Sm, _ = O.pseudofermion_action(O.Operator(O.WILSON, U - eps * dU, bc, m0), phi)
    fd = (Sp - Sm) / (2 * eps)
    an = float(np.sum(np.real(np.conj(G) * dU)))
    assert abs(fd - an) < 1e-6 * abs(an)


def test_brillouin_weights_golden_and_free_field_moments():
    """The printed weights (tests/golden/brillouin_weights.txt) satisfy the
    identities that make Eq. (def_ider) a derivative and Eq. (def_blap) a
    Laplacian on the 3^4 hypercube: sum_s rho_k s_mu^2 = 1, sum_s lambda_k =
    0, sum_s lambda_k s_mu^2 = 2 (k = |s|_1); and the oracle's free D_B acting
    on a plane wave of momentum p along x equals the symbol built from them."""
    import itertools
    import os
    from fractions import Fraction
    path = os.path.join(os.path.dirname(__file__), "golden", "brillouin_weights.txt")
    w = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, rest = line.split(None, 1)
        nums, den = rest.split("/")
        w[name] = [Fraction(int(a), int(den)) for a in nums.split()]
    rho, lam = [None] + w["rho"], w["lambda"]
    offs = [s for s in itertools.product((-1, 0, 1), repeat=4)]
    k = lambda s: sum(1 for a in s if a)
    assert sum(rho[k(s)] * s[0] ** 2 for s in offs if k(s)) == 1
    assert sum(lam[k(s)] for s in offs) == 0
    assert sum(lam[k(s)] * s[0] ** 2 for s in offs) == 2
    # free field: D_B e^{ipx} = [sum_s (rho_k i s.gamma-part) ...]; check the
    # scalar (Laplacian) part on a plane wave through the oracle with m0 = 0:
    # the gamma-free part of the symbol is -1/2 sum_s lambda_k e^{i p s_x}
    dims, p = (8, 4, 4, 4), 2 * np.pi / 8
    U = I.unit_gauge_field(dims, 1)
    op = O.Operator(O.BRILLOUIN, U, (1, 1, 1, 1))
    x = np.arange(dims[0])
    psi = np.zeros((dims[3], dims[2], dims[1], dims[0], 1, 4, 1), complex)
    psi[..., 0, 0, 0] = np.exp(1j * p * x)[None, None, None, :]
    out = op.apply(psi, 0.0)
    scal = float(-0.5 * sum(lam[k(s)] * np.cos(p * s[0]) for s in offs))
    assert np.allclose(out[..., 0, 0, 0], scal * psi[..., 0, 0, 0], atol=1e-12)


# ------------------------------------------------------------- clover term

def _golden(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    return [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]


PAULI = [S0, S1, S2, S3]


def test_sigma_munu_match_app_a_printed_forms():
    """sigma_mu,nu of the oracle against the tensor forms App. A prints
    (tests/golden/sigma_munu_app_a.txt); all six planes, in the oracle's order."""
    rows = _golden("sigma_munu_app_a.txt")
    assert len(rows) == 6
    for k, (mu, nu, sign, a, b) in enumerate(rows):
        mu, nu = int(mu) - 1, int(nu) - 1
        assert O.PLANES[k] == (mu, nu)
        want = float(sign) * np.kron(PAULI[int(a)], PAULI[int(b)])
        assert np.allclose(O.sigma(mu, nu), want, atol=1e-15, rtol=0)


def _abelian_angles(dims, rng):
    """theta[t,z,y,x,mu,c]: one U(1) angle per link and colour."""
    nx, ny, nz, nt = dims
    return rng.uniform(-np.pi, np.pi, (nt, nz, ny, nx, 4, 3))


def test_field_strength_abelian_closed_form():
    """Diagonal links exp(i theta_mu(n)) per colour: each leaf is the phase of
    one plaquette, so F_mu,nu(n) = diag( (1/4) sum over the four plaquettes
    with a corner at n of sin(plaquette angle) ), zero off the diagonal.  The
    plaquette angles are summed here from the link angles with np.roll."""
    dims = (4, 3, 2, 5)
    rng = np.random.Generator(np.random.PCG64(41))
    th = _abelian_angles(dims, rng)
    U = np.zeros(th.shape[:5] + (3, 3), complex)
    for c in range(3):
        U[..., c, c] = np.exp(1j * th[..., c])
    F = O.field_strength(U)
    axis = {0: 3, 1: 2, 2: 1, 3: 0}     # coordinate mu -> array axis (t, z, y, x order)

    def sh(a, mu, k):                   # a(n + k mu-hat)
        return np.roll(a, -k, axis=axis[mu])

    for k, (mu, nu) in enumerate(O.PLANES):
        tm, tn = th[..., mu, :], th[..., nu, :]
        P = tm + sh(tn, mu, 1) - sh(tm, nu, 1) - tn          # plaquette with lower corner m
        want = 0.25 * (np.sin(P) + np.sin(sh(P, mu, -1)) + np.sin(sh(sh(P, mu, -1), nu, -1))
                       + np.sin(sh(P, nu, -1)))
        got = F[..., k, :, :]
        assert np.abs(np.diagonal(got, axis1=-2, axis2=-1) - want).max() < 1e-13
        off = got - np.einsum("...c,cd->...cd", np.diagonal(got, axis1=-2, axis2=-1), np.eye(3))
        assert np.abs(off).max() < 1e-15


def test_field_strength_constant_field_and_clover_eigenvalues():
    """A constant field B in the (1,2) plane only (U_x(n) = exp(-i B y), the
    y extent a multiple of 2 pi / B): F_12 = sin(B), the other planes vanish,
    and C = -(c_SW/2) sigma_12 sin B = (c_SW/2) sin B (pauli_0 (x) pauli_3)
    multiplies spins 1, 3 by +(c_SW/2) sin B and spins 2, 4 by its negative."""
    dims = (2, 6, 2, 2)
    B = 2 * np.pi / 6
    nx, ny, nz, nt = dims
    y = np.arange(ny)[None, None, :, None]
    U = np.zeros((nt, nz, ny, nx, 4, 1, 1), complex)
    U[..., :, 0, 0] = 1.0
    U[..., 0, 0, 0] = np.exp(-1j * B * y) * np.ones((nt, nz, ny, nx))
    F = O.field_strength(U)
    assert np.abs(F[..., 0, 0, 0] - np.sin(B)).max() < 1e-14
    assert np.abs(F[..., 1:, :, :]).max() < 1e-14
    csw = 1.7
    psi = I.source(dims, 1, 3, seed=42)
    Cpsi = O.clover(F, csw, psi)
    lam = 0.5 * csw * np.sin(B)
    sign = np.array([1, -1, 1, -1])[None, None, None, None, None, :, None]
    assert np.abs(Cpsi - lam * sign * psi).max() < 1e-14


def test_field_strength_vanishes_for_pure_gauge():
    """U_mu(n) = g(n) g(n+mu)^dag has every closed loop equal to 1, so F = 0."""
    dims = (4, 2, 3, 4)
    g = I.gauge_transform(dims, 3, seed=43)
    U = _transform_links(I.unit_gauge_field(dims, 3), g)
    assert np.abs(O.field_strength(U)).max() < 1e-13


def test_field_strength_gauge_covariant_hermitian_and_phase_blind():
    dims = (4, 2, 4, 3)
    U = I.gauge_field(dims, 3, 0.6, seed=44)
    g = I.gauge_transform(dims, 3, seed=45)
    F = O.field_strength(U)
    Fg = O.field_strength(_transform_links(U, g))
    want = np.einsum("...ab,...kbc,...dc->...kad", g, F, np.conj(g))
    assert np.abs(Fg - want).max() < 1e-13
    assert np.abs(F - np.conj(np.swapaxes(F, -1, -2))).max() < 1e-15
    assert np.abs(O.field_strength(O.phase_links(U, (-1, 1, -1, -1))) - F).max() < 1e-15
    assert np.abs(F).max() > 0.05          # not trivially zero


@pytest.mark.parametrize("kind", [O.WILSON, O.BRILLOUIN])
def test_clover_operator_dense_hermiticity_and_gamma5(kind):
    """On a 2^4 lattice as dense matrices: C is hermitian and commutes with
    gamma5, so (D + C) stays gamma5-hermitian and its oracle dagger is the
    conjugate transpose; C vanishes on the free field."""
    dims, nc = (2, 2, 2, 2), 2
    U = I.gauge_field(dims, nc, 0.7, seed=46)
    op = O.Operator(kind, U, (1, 1, 1, -1), 0.1, csw=1.3)
    F = op.F
    n = 16 * nc * 4
    basis = np.eye(n, dtype=complex).reshape((n,) + (2, 2, 2, 2, nc, 4))
    basis = np.moveaxis(basis, 0, -1)                     # nv = n unit vectors
    Cm = O.clover(F, 1.3, basis).reshape(n, n)
    assert np.abs(Cm - Cm.conj().T).max() < 1e-14
    g5 = np.kron(np.eye(16 * nc), np.diag([1, 1, -1, -1]))
    assert np.abs(g5 @ Cm - Cm @ g5).max() < 1e-14
    Dm = op.apply(basis).reshape(n, n)
    Dd = op.apply_dagger(basis).reshape(n, n)
    assert np.abs(Dd - Dm.conj().T).max() < 1e-13
    D0 = O.Operator(kind, U, (1, 1, 1, -1), 0.1).apply(basis).reshape(n, n)
    assert np.abs(Dm - D0 - Cm).max() < 1e-13
    assert np.abs(O.field_strength(I.unit_gauge_field(dims, nc))).max() == 0


def test_clover_sites_match_full_apply():
    dims = (4, 2, 2, 4)
    U = I.gauge_field(dims, 3, 0.5, seed=47)
    psi = I.source(dims, 3, 2, seed=48)
    op = O.Operator(O.WILSON, U, (1, 1, 1, -1), -0.3, csw=1.0)
    full = op.apply(psi).reshape((-1, 3, 4, 2))
    fulld = op.apply_dagger(psi).reshape((-1, 3, 4, 2))
    sites = [0, 5, 17, 63]
    assert np.abs(op.apply_sites(psi, sites) - full[sites]).max() < 1e-13
    assert np.abs(op.apply_sites(psi, sites, dagger=True) - fulld[sites]).max() < 1e-13


def test_clover_flop_counts_app_e():
    for form, nc, flops, poly, mults in _golden("app_e_clover_flops.txt"):
        assert O.clover_flops_per_site(int(nc), int(mults)) == int(flops)
        for n in (1, 2, 3, 4):
            assert O.clover_flops_per_site(n, int(mults)) == eval(poly.replace("^", "**"), {"nc": n})


# ------------------------------------------------------- Laplace operators

LAP_KINDS = [O.WLAP, O.BLAP, O.WSUV, O.BSUV]


def laplace_symbol(kind, p, m):
    """Free-field eigenvalue of A = -1/2 Lap + m^2/2 at momentum p: the
    standard Laplacian gives sum_mu (1 - cos p_mu), the Brillouin one
    2 (1 - prod_mu cos^2(p_mu / 2)) (its weights lambda_k sum to
    4 prod cos^2(p/2) - 4 over the hypercube)."""
    if kind in (O.WLAP, O.WSUV):
        return 0.5 * m * m + np.sum(1 - np.cos(p))
    return 0.5 * m * m + 2.0 * (1.0 - np.prod(np.cos(p / 2) ** 2))


@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 1, 1, -1)])
@pytest.mark.parametrize("kind", LAP_KINDS)
def test_laplace_free_field_symbol(kind, bc):
    dims, nc, m = (4, 4, 6, 4), 2, 0.3
    op = O.Operator(kind, I.unit_gauge_field(dims, nc), bc)
    rng = np.random.default_rng(61)
    for p in momenta(dims, bc, rng, 5):
        shape = (nc, 4, 3) if O.spins(kind) == 4 else (nc, 3)
        chi = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        psi = plane_wave(dims, p, chi)
        got = op.apply(psi, m)
        assert np.abs(got - laplace_symbol(kind, p, m) * psi).max() < 1e-12


@pytest.mark.parametrize("kind", [O.WILSON, O.BRILLOUIN])
def test_laplace_is_the_hermitian_part_of_the_dirac_operator(kind):
    """gamma_mu nabla_mu is anti-hermitian, so (D + D^dag)/2 = -1/2 Lap + m0:
    the Laplace operator at m^2/2 = m0 against the (pinned) Dirac operator and
    its adjoint, on a random gauge field with twisted boundary phases."""
    dims, nc, m = (4, 2, 4, 6), 3, 0.7
    U = I.gauge_field(dims, nc, 0.5, seed=62)
    bc = (1, -1, 1, -1)
    psi = I.source(dims, nc, 3, seed=63)
    Dop = O.Operator(kind, U, bc)
    herm = 0.5 * (Dop.apply(psi, 0.5 * m * m) + Dop.apply_dagger(psi, 0.5 * m * m))
    lap = O.Operator(O.WLAP if kind == O.WILSON else O.BLAP, U, bc).apply(psi, m)
    assert np.abs(lap - herm).max() < 1e-12 * np.abs(herm).max()


def test_colour_only_laplace_is_the_spin_diagonal_one():
    dims, nc = (4, 2, 2, 4), 3
    U = I.gauge_field(dims, nc, 0.5, seed=64)
    psi = I.source(dims, nc, 2, seed=65)
    for full, suv in ((O.WLAP, O.WSUV), (O.BLAP, O.BSUV)):
        a = O.Operator(full, U, (1, 1, 1, -1)).apply(psi, 0.4)
        b = O.Operator(suv, U, (1, 1, 1, -1))
        for sp in range(4):
            assert np.abs(a[..., sp, :] - b.apply(np.ascontiguousarray(psi[..., sp, :]), 0.4)).max() < 1e-13


@pytest.mark.parametrize("kind", LAP_KINDS)
def test_laplace_gauge_covariance(kind):
    dims, nc = (4, 2, 4, 2), 3
    U = I.gauge_field(dims, nc, 0.5, seed=66)
    Om = I.gauge_transform(dims, nc, seed=67)
    cols = O.spins(kind) == 1
    psi = I.source(dims, nc, 2, seed=68, staggered=cols)
    rot = (lambda v: np.einsum("...ab,...bv->...av", Om, v)) if cols else \
          (lambda v: np.einsum("...ab,...bsv->...asv", Om, v))
    bc = (1, -1, 1, -1)
    lhs = O.Operator(kind, _transform_links(U, Om), bc).apply(rot(psi), 0.2)
    rhs = rot(O.Operator(kind, U, bc).apply(psi, 0.2))
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


@pytest.mark.parametrize("kind", [O.WSUV, O.BSUV])
def test_laplace_dense_hermitian_positive_and_cg(kind):
    """Dense on 2^4 x N_c = 2: A is hermitian with spectrum >= m^2/2 (the paper
    calls it hpd), and oracle CG on A x = b matches a dense solve."""
    dims, nc, m = (2, 2, 2, 2), 2, 0.3
    U = I.gauge_field(dims, nc, 0.8, seed=69)
    op = O.Operator(kind, U, (1, 1, 1, -1))
    n = 16 * nc
    basis = np.moveaxis(np.eye(n, dtype=complex).reshape((n, 2, 2, 2, 2, nc)), 0, -1)
    A = op.apply(basis, m).reshape(n, n)
    assert np.abs(A - A.conj().T).max() < 1e-14
    assert np.linalg.eigvalsh(A).min() >= 0.5 * m * m - 1e-12
    b = I.source(dims, nc, 2, seed=70, staggered=True)
    x, info = O.cg(lambda v: op.apply(v, m), b, tol=1e-12, maxit=500)
    assert info["status"] == O.CONVERGED
    want = np.linalg.solve(A, b.reshape(n, 2))
    assert np.abs(x.reshape(n, 2) - want).max() < 1e-10 * np.abs(want).max()


def test_laplace_sites_match_full_apply():
    dims = (4, 2, 2, 4)
    U = I.gauge_field(dims, 3, 0.5, seed=71)
    sites = [0, 7, 21, 63]
    for kind in LAP_KINDS:
        cols = O.spins(kind) == 1
        psi = I.source(dims, 3, 2, seed=72, staggered=cols)
        op = O.Operator(kind, U, (1, 1, 1, -1))
        full = op.apply(psi, 0.3).reshape((-1,) + psi.shape[4:])
        assert np.abs(op.apply_sites(psi, sites, 0.3) - full[sites]).max() < 1e-13


def test_laplace_flop_counts_app_e():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "app_e_laplace_flops.txt")
    kinds = {"wlap": O.WLAP, "wsuv": O.WSUV, "blap": O.BLAP, "bsuv": O.BSUV}
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 4
    for name, nc, flops, f12, poly in rows:
        assert O.flops_per_site(kinds[name], int(nc)) == int(flops)
        if f12 != "-":
            assert 12 * O.flops_per_site(kinds[name], int(nc)) == int(f12)
        for n in (1, 2, 3, 4):
            assert O.flops_per_site(kinds[name], n) == eval(poly.replace("^", "**"), {"nc": n})


# ------------------------------------------------------------ stout smearing

def test_stout_identity_cases_and_pure_gauge():
    """rho = 0 or no step leaves U alone; a pure gauge U_mu(n) = g(n) g(n+mu)^dag
    has every staple equal to its link, so Omega is a multiple of 1 and Q = 0."""
    dims = (4, 2, 2, 4)
    U = I.gauge_field(dims, 3, 0.5, seed=81)
    assert np.array_equal(O.stout_smear(U, 0.12, 0), U)
    assert np.abs(O.stout_smear(U, 0.0, 2) - U).max() < 1e-15
    g = I.gauge_transform(dims, 3, seed=82)
    P = _transform_links(I.unit_gauge_field(dims, 3), g)
    assert np.abs(O.stout_smear(P, 0.12, 3) - P).max() < 1e-13


def test_stout_unitary_covariant_and_phase_commuting():
    dims = (4, 2, 4, 2)
    U = I.gauge_field(dims, 3, 0.6, seed=83)
    V = O.stout_smear(U, 0.12, 3)
    eye = np.eye(3)
    assert np.abs(V @ np.conj(np.swapaxes(V, -1, -2)) - eye).max() < 1e-13
    assert np.abs(np.linalg.det(V) - 1).max() < 1e-13
    assert np.abs(V - U).max() > 0.05
    g = I.gauge_transform(dims, 3, seed=84)
    assert np.abs(O.stout_smear(_transform_links(U, g), 0.12, 3) - _transform_links(V, g)).max() < 1e-12
    bc = (1, -1, 1, -1)
    assert np.abs(O.stout_smear(O.phase_links(U, bc), 0.12, 2) -
                  O.phase_links(O.stout_smear(U, 0.12, 2), bc)).max() < 1e-13


def test_stout_abelian_closed_form():
    """Diagonal links exp(i theta_c) (theta_3 = -theta_1 - theta_2): Omega is
    diagonal and one step moves every angle by rho sum_nu [sin(forward staple
    angle - theta) + sin(backward staple angle - theta)], minus the colour
    average of that shift (the traceless projection); summed here from the
    link angles with np.roll."""
    dims = (4, 3, 2, 5)
    rng = np.random.Generator(np.random.PCG64(85))
    th = rng.uniform(-1.0, 1.0, (dims[3], dims[2], dims[1], dims[0], 4, 3))
    th[..., 2] = -th[..., 0] - th[..., 1]
    U = np.zeros(th.shape[:5] + (3, 3), complex)
    for c in range(3):
        U[..., c, c] = np.exp(1j * th[..., c])
    rho = 0.12
    V = O.stout_smear(U, rho, 1)
    axis = {0: 3, 1: 2, 2: 1, 3: 0}

    def sh(a, mu, k):
        return np.roll(a, -k, axis=axis[mu])

    shift = np.zeros_like(th)
    for mu in range(4):
        t = th[..., mu, :]
        acc = np.zeros_like(t)
        for nu in range(4):
            if nu == mu:
                continue
            tn = th[..., nu, :]
            fwd = tn + sh(t, nu, 1) - sh(tn, mu, 1)
            bwd = -sh(tn, nu, -1) + sh(t, nu, -1) + sh(sh(tn, nu, -1), mu, 1)
            acc += np.sin(fwd - t) + np.sin(bwd - t)
        shift[..., mu, :] = rho * acc - rho * acc.mean(axis=-1, keepdims=True)
    want = np.zeros_like(U)
    for c in range(3):
        want[..., c, c] = np.exp(1j * (th[..., c] + shift[..., c]))
    assert np.abs(V - want).max() < 1e-13


def test_stout_smooths_the_plaquette():
    """Stout smearing raises the average plaquette of a rough field (the
    purpose of a fat-link background): a sanity property of the oracle."""
    dims = (4, 4, 4, 4)
    U = I.gauge_field(dims, 3, 0.6, seed=86)

    def fwd(a, mu):                      # a(n + mu-hat), field axes (t, z, y, x)
        return np.roll(a, -1, axis=3 - mu)

    def dag(a):
        return np.conj(np.swapaxes(a, -1, -2))

    def plaq(X):
        F = 0.0
        for mu in range(4):
            for nu in range(mu + 1, 4):
                P = X[..., mu, :, :] @ fwd(X[..., nu, :, :], mu) @ dag(fwd(X[..., mu, :, :], nu)) @ \
                    dag(X[..., nu, :, :])
                F += np.trace(P, axis1=-2, axis2=-1).real.mean() / 3
        return F / 6

    p0, p3 = plaq(U), plaq(O.stout_smear(U, 0.12, 3))
    assert p3 > p0 + 0.05


# ------------------------------------------------------ staggered fermion force

@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, 1, 1, -1)])
def test_staggered_force_matches_finite_differences(bc):
    """S = sum Re phi^dag (D_S^dag D_S)^-1 phi: dS/deps along U -> exp(eps X) U
    equals Re sum tr[X F] (central differences, eps = 1e-4, FP64 solves; the
    mass keeps the O(eps^2) truncation of the difference below 1e-6)."""
    dims = (4, 2, 2, 4)
    m0 = 0.4
    U = I.gauge_field(dims, 3, 0.4, seed=121)
    phi = I.source(dims, 3, 2, seed=122, staggered=True)
    op = O.Operator(O.STAGGERED, U, bc, m0)
    S0, psi = O.pseudofermion_action(op, phi)
    F = O.staggered_force(op, psi, op.apply(psi))
    assert np.allclose(F, -np.conj(np.swapaxes(F, -1, -2)), atol=1e-14)
    assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-13
    eps = 1e-4
    for seed in range(4):
        X = I.su_n_direction(dims, 3, seed=300 + seed)
        Sp, _ = O.pseudofermion_action(O.Operator(O.STAGGERED, _expm_ah(eps * X) @ U, bc, m0), phi)
        Sm, _ = O.pseudofermion_action(O.Operator(O.STAGGERED, _expm_ah(-eps * X) @ U, bc, m0), phi)
        fd = (Sp - Sm) / (2 * eps)
        an = np.sum(np.real(np.einsum("...ab,...ba->...", X, F)))
        assert abs(fd - an) < 1e-6 * max(abs(an), 1.0), (seed, fd, an)


def test_staggered_action_gradient_matches_finite_differences():
    dims = (2, 2, 2, 4)
    m0, bc = 0.3, (1, 1, 1, -1)
    U = I.gauge_field(dims, 3, 0.4, seed=131)
    phi = I.source(dims, 3, 1, seed=132, staggered=True)
    op = O.Operator(O.STAGGERED, U, bc, m0)
    S0, psi = O.pseudofermion_action(op, phi)
    G = O.staggered_action_gradient(op, psi, op.apply(psi))
    rng = np.random.default_rng(6)
    dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    eps = 1e-5
    Sp, _ = O.pseudofermion_action(O.Operator(O.STAGGERED, U + eps * dU, bc, m0), phi)
    Sm, _ = O.pseudofermion_action(O.Operator(O.STAGGERED, U - eps * dU, bc, m0), phi)
    fd = (Sp - Sm) / (2 * eps)
    an = float(np.sum(np.real(np.conj(G) * dU)))
    assert abs(fd - an) < 1e-6 * abs(an)


# ------------------------------------------------------ Brillouin fermion force

@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, -1, 1, -1)])
def test_brillouin_force_matches_finite_differences(bc):
    """S = sum Re phi^dag (D_B^dag D_B)^-1 phi with the force through the W
    path averages: dS/deps along U -> exp(eps X) U against Re sum tr[X F]
    (central differences, eps = 1e-4, FP64 solves)."""
    dims = (4, 2, 2, 4)
    m0 = 0.4
    U = I.gauge_field(dims, 3, 0.4, seed=141)
    phi = I.source(dims, 3, 2, seed=142)
    op = O.Operator(O.BRILLOUIN, U, bc, m0)
    S0, psi = O.pseudofermion_action(op, phi)
    F = O.brillouin_force(op, psi, op.apply(psi))
    assert np.allclose(F, -np.conj(np.swapaxes(F, -1, -2)), atol=1e-14)
    assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-13
    eps = 1e-4
    for seed in range(3):
        X = I.su_n_direction(dims, 3, seed=500 + seed)
        Sp, _ = O.pseudofermion_action(O.Operator(O.BRILLOUIN, _expm_ah(eps * X) @ U, bc, m0), phi)
        Sm, _ = O.pseudofermion_action(O.Operator(O.BRILLOUIN, _expm_ah(-eps * X) @ U, bc, m0), phi)
        fd = (Sp - Sm) / (2 * eps)
        an = np.sum(np.real(np.einsum("...ab,...ba->...", X, F)))
        assert abs(fd - an) < 1e-6 * max(abs(an), 1.0), (seed, fd, an)


def test_brillouin_action_gradient_matches_finite_differences():
    """The complex gradient along an arbitrary complex dU (off the group, so
    every path product's dependence on every link is exercised)."""
    dims = (2, 2, 2, 4)
    m0, bc = 0.4, (1, 1, 1, -1)
    U = I.gauge_field(dims, 3, 0.4, seed=151)
    phi = I.source(dims, 3, 1, seed=152)
    op = O.Operator(O.BRILLOUIN, U, bc, m0)
    S0, psi = O.pseudofermion_action(op, phi)
    G = O.brillouin_action_gradient(op, psi, op.apply(psi))
    rng = np.random.default_rng(7)
    dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    eps = 1e-5
    Sp, _ = O.pseudofermion_action(O.Operator(O.BRILLOUIN, U + eps * dU, bc, m0), phi)
    Sm, _ = O.pseudofermion_action(O.Operator(O.BRILLOUIN, U - eps * dU, bc, m0), phi)
    fd = (Sp - Sm) / (2 * eps)
    an = float(np.sum(np.real(np.conj(G) * dU)))
    assert abs(fd - an) < 1e-6 * abs(an)


# ------------------------------------- W path average for non-commuting links

def _su3_directions(rng):
    """Four random traceless anti-hermitian 3x3 matrices X_mu (su(3))."""
    out = []
    for _ in range(4):
        A = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        H = (A + A.conj().T) / 2
        H -= np.trace(H) / 3 * np.eye(3)
        out.append(1j * H)
    return out


def _constant_links(X, eps, dims=(3, 3, 3, 3)):
    from scipy.linalg import expm
    U = np.zeros(tuple(dims[::-1]) + (4, 3, 3), complex)
    for mu in range(4):
        U[..., mu, :, :] = expm(eps * X[mu])
    return U


def _eps3_ratios(w_of_eps, X, eps=0.04):
    """For constant links U_mu = exp(eps X_mu) every hop ordering of offset s
    is a product of exp(+-eps X_mu); by Baker-Campbell-Hausdorff the average
    over all k! orderings (Tab. off-axis) is exp(eps sum_mu s_mu X_mu) + O(eps^3):
    the O(eps^2) commutator terms cancel pairwise.  Returns, per offset with
    k >= 2 hops, the ratio of the deviations at eps and eps/2 (8 for an
    O(eps^3) deviation, 4 for an O(eps^2) one)."""
    from scipy.linalg import expm
    out = {}
    W1, W2 = w_of_eps(eps), w_of_eps(eps / 2)
    for d in range(81):
        s = _offset(d)
        if int(np.abs(s).sum()) < 2:
            continue
        S = sum(s[mu] * X[mu] for mu in range(4))
        e1 = np.abs(W1[d] - expm(eps * S)).max()
        e2 = np.abs(W2[d] - expm(eps / 2 * S)).max()
        out[d] = e1 / e2
    return out


def _w_const_subset(X, eps, orderings):
    """W_s for constant links averaged over the hop orderings `orderings(hops)`
    returns (a planted mistake when that is not all k! of them)."""
    from scipy.linalg import expm
    Wd = {}
    for d in range(81):
        s = _offset(d)
        hops = [mu for mu in range(4) if s[mu]]
        perms = orderings(hops)
        acc = np.zeros((3, 3), complex)
        for perm in perms:
            M = np.eye(3, dtype=complex)
            for mu in perm:
                M = M @ expm(s[mu] * eps * X[mu])
            acc += M
        Wd[d] = acc / len(perms)
    return Wd


def _cyclic(hops):
    return [hops[i:] + hops[:i] for i in range(len(hops))] if hops else [[]]


def test_w_all_orderings_average_is_exp_sum_to_third_order():
    """Pins the completeness of the k!-ordering average of Tab. off-axis for
    k = 2, 3, 4 with non-commuting links: the deviation from
    exp(eps sum s_mu X_mu) must fall as eps^3.  An average over only the k
    cyclic orderings (a plausible enumeration mistake) falls as eps^2 and is
    rejected by the same check."""
    rng = np.random.default_rng(17)
    X = _su3_directions(rng)

    def oracle_w(eps):
        W = O.build_w(O.phase_links(_constant_links(X, eps), (1, 1, 1, 1)))
        return {d: W[1, 2, 0, 1, d] for d in range(81)}

    ratios = _eps3_ratios(oracle_w, X)
    for k in (2, 3, 4):
        rk = [r for d, r in ratios.items() if int(np.abs(_offset(d)).sum()) == k]
        assert len(rk) == {2: 24, 3: 32, 4: 16}[k]
        assert all(6.5 < r < 9.5 for r in rk), (k, min(rk), max(rk))
    # the full enumeration written here agrees with the oracle (constant links)
    full = _w_const_subset(X, 0.04, lambda h: [list(p) for p in itertools.permutations(h)] or [[]])
    W = oracle_w(0.04)
    assert max(np.abs(full[d] - W[d]).max() for d in range(81)) < 1e-14
    # planted mistake: cyclic orderings only -> O(eps^2) for k = 3, 4
    bad = _eps3_ratios(lambda e: _w_const_subset(X, e, _cyclic), X)
    worst = [r for d, r in bad.items() if int(np.abs(_offset(d)).sum()) >= 3]
    assert not all(6.5 < r < 9.5 for r in worst)
    assert min(worst) < 5.0


# ------------------------------------ element-wise dense matrices (2^4, 3x3x2x2)
# Built here from the equations, entry by entry, without the oracle's code:
# the links are phased here, W is enumerated here, the gammas are the
# tensor-product forms above.

def _site(c, dims):
    x, y, z, t = c
    return ((t * dims[2] + z) * dims[1] + y) * dims[0] + x


def _phased_here(U, bc, dims):
    Up = U.copy()
    for mu, ax in enumerate((3, 2, 1, 0)):
        idx = [slice(None)] * 4
        idx[ax] = dims[mu] - 1
        Up[tuple(idx) + (mu,)] *= bc[mu]
    return Up


def _link(Up, c, mu):
    x, y, z, t = c
    return Up[t, z, y, x, mu]


def _step(c, mu, sgn, dims):
    c = list(c)
    c[mu] = (c[mu] + sgn) % dims[mu]
    return tuple(c)


def _w_here(Up, c, s, dims):
    hops = [mu for mu in range(4) if s[mu]]
    nc = Up.shape[-1]
    if not hops:
        return np.eye(nc, dtype=complex)
    acc = np.zeros((nc, nc), complex)
    perms = list(itertools.permutations(hops))
    for perm in perms:
        pos, M = c, np.eye(nc, dtype=complex)
        for mu in perm:
            if s[mu] > 0:
                M = M @ _link(Up, pos, mu)
                pos = _step(pos, mu, +1, dims)
            else:
                pos = _step(pos, mu, -1, dims)
                M = M @ _link(Up, pos, mu).conj().T
        acc += M
    return acc / len(perms)


def _dense_elementwise(kind, U, bc, m0, dims, rho, lam):
    nc = U.shape[-1]
    ns = 1 if kind == O.STAGGERED else 4
    blk = nc * ns
    V = int(np.prod(dims))
    Up = _phased_here(U, bc, dims)
    Dm = np.zeros((V * blk, V * blk), complex)
    I4 = np.eye(4)
    for c in itertools.product(*[range(d) for d in dims]):
        n = _site(c, dims)
        rows = slice(n * blk, (n + 1) * blk)

        def add(m, M):
            Dm[rows, m * blk:(m + 1) * blk] += M

        if kind == O.WILSON:
            add(n, (4 + m0) * np.eye(blk))
            for mu in range(4):
                fw, bw = _step(c, mu, +1, dims), _step(c, mu, -1, dims)
                add(_site(fw, dims), -0.5 * np.kron(_link(Up, c, mu), I4 - GAMMA[mu]))
                add(_site(bw, dims), -0.5 * np.kron(_link(Up, bw, mu).conj().T, I4 + GAMMA[mu]))
        elif kind == O.STAGGERED:
            add(n, m0 * np.eye(blk))
            for mu in range(4):
                eta = (-1) ** sum(c[nu] + 1 for nu in range(mu))
                fw, bw = _step(c, mu, +1, dims), _step(c, mu, -1, dims)
                add(_site(fw, dims), 0.5 * eta * _link(Up, c, mu))
                add(_site(bw, dims), -0.5 * eta * _link(Up, bw, mu).conj().T)
        else:
            for s in itertools.product((-1, 0, 1), repeat=4):
                k = sum(1 for a in s if a)
                if k == 0:
                    S = (m0 - 0.5 * lam[0]) * I4
                else:
                    S = rho[k] * sum(s[mu] * GAMMA[mu] for mu in range(4)) - 0.5 * lam[k] * I4
                m = c
                for mu in range(4):
                    m = _step(m, mu, s[mu], dims)
                add(_site(m, dims), np.kron(_w_here(Up, c, s, dims), S))
    return Dm


def _printed_weights():
    w = {}
    for name, *rest in _golden("brillouin_weights.txt"):
        nums = rest[:rest.index("/")]
        den = float(rest[-1])
        w[name] = [float(a) / den for a in nums]
    return [None] + w["rho"], w["lambda"]


@pytest.mark.parametrize("kind", [O.WILSON, O.BRILLOUIN, O.STAGGERED])
@pytest.mark.parametrize("dims,nc", [((2, 2, 2, 2), 3), ((3, 3, 2, 2), 2), ((4, 2, 2, 2), 3)])
def test_dense_elementwise_matches_oracle_apply(kind, dims, nc):
    """The whole matrix of D, written entry by entry from Eqs. (app_wils,
    app_bril, def_stag) with the printed Brillouin weights, equals the matrix
    of the oracle's apply; on 2^4 every offset aliases onto another site, so
    the summation over offsets is checked too."""
    if kind == O.STAGGERED and any(d % 2 for d in dims):
        pytest.skip("staggered needs even extents")
    rho, lam = _printed_weights()
    U = I.gauge_field(dims, nc, 0.5, seed=71)
    bc = (1, -1, 1, -1)
    m0 = 0.05 if kind == O.STAGGERED else 0.1
    op = O.Operator(kind, U, bc, m0)
    shape = tuple(dims[::-1]) + ((nc, 1) if kind == O.STAGGERED else (nc, 4, 1))
    want = _dense_elementwise(kind, U, bc, m0, dims, rho, lam)
    got = dense(op.apply, shape)
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


# ------------------------------------------ chain rule through stout smearing

def _smeared_action_and_gradient(U, phi, bc, m0, rho, nsteps, kind=O.WILSON):
    V = O.stout_smear(U, rho, nsteps)
    op = O.Operator(kind, V, bc)
    S, psi = O.pseudofermion_action(op, phi, m0, tol=1e-14)
    chi = op.apply(psi, m0)
    GV = {O.WILSON: O.wilson_action_gradient, O.STAGGERED: O.staggered_action_gradient,
          O.BRILLOUIN: O.brillouin_action_gradient}[kind](op, psi, chi)
    return S, GV


def _fd_check(U, phi, bc, m0, rho, nsteps, GU, kind, rng, count=2):
    worst = 0.0
    for _ in range(count):
        dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
        eps = 1e-5
        Sp = O.pseudofermion_action(O.Operator(kind, O.stout_smear(U + eps * dU, rho, nsteps), bc), phi, m0,
                                    tol=1e-14)[0]
        Sm = O.pseudofermion_action(O.Operator(kind, O.stout_smear(U - eps * dU, rho, nsteps), bc), phi, m0,
                                    tol=1e-14)[0]
        fd = (Sp - Sm) / (2 * eps)
        an = float(np.sum(np.real(np.conj(GU) * dU)))
        worst = max(worst, abs(fd - an) / abs(an))
    return worst


@pytest.mark.parametrize("kind", [O.WILSON, O.STAGGERED])
def test_stout_chain_rule_matches_finite_differences(kind):
    """S(U) = sum Re phi^dag (D[V]^dag D[V])^-1 phi with V = stout^2(U): the
    gradient carried back through the two stout steps (oracle.stout_backward)
    against central differences along random complex directions dU."""
    dims, nc, nv, m0, bc = (4, 4, 2, 4), 3, 2, 0.3, (1, 1, 1, -1)
    U = I.gauge_field(dims, nc, 0.4, 81)
    phi = I.source(dims, nc, nv, 82, staggered=(kind == O.STAGGERED))
    rho, nsteps = 0.12, 2
    _, GV = _smeared_action_and_gradient(U, phi, bc, m0, rho, nsteps, kind)
    GU = O.stout_backward(U, GV, rho, nsteps)
    assert _fd_check(U, phi, bc, m0, rho, nsteps, GU, kind, np.random.default_rng(3)) < 1e-7


def test_stout_chain_rule_identity_cases_and_planted_mistake(monkeypatch):
    """No step (or rho = 0) passes the gradient through unchanged; and a
    Frechet derivative that treats exp(iQ) as commuting with its direction
    (a plausible shortcut), planted in the oracle, fails the difference check."""
    dims, nc, nv, m0, bc = (4, 2, 2, 4), 3, 2, 0.3, (1, 1, 1, -1)
    U = I.gauge_field(dims, nc, 0.5, 83)
    phi = I.source(dims, nc, nv, 84)
    G = np.random.default_rng(5).standard_normal(U.shape) + 0j
    assert np.array_equal(O.stout_backward(U, G, 0.12, 0), G)
    assert np.abs(O.stout_backward(U, G, 0.0, 3) - G).max() < 1e-14
    rho, nsteps = 0.12, 1
    _, GV = _smeared_action_and_gradient(U, phi, bc, m0, rho, nsteps)
    good = O.stout_backward(U, GV, rho, nsteps)
    assert _fd_check(U, phi, bc, m0, rho, nsteps, good, O.WILSON, np.random.default_rng(6), 1) < 1e-7
    monkeypatch.setattr(O.oracle, "_expi_frechet", lambda Q, G: O.oracle._expi_herm(Q) @ G)
    bad = O.stout_backward(U, GV, rho, nsteps)
    assert _fd_check(U, phi, bc, m0, rho, nsteps, bad, O.WILSON, np.random.default_rng(6), 1) > 1e-4
