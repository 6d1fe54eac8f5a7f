"""Fermion force and autograd through the C ABI.

S = sum_v Re phi_v^dag (D^dag D)^-1 phi_v for D = D_W, D_S and D_B.  The force kernel is compared
with the oracle's force on the same solution vector; the autograd gradient
with the oracle's complex gradient; and the whole chain with central finite
differences of S along random su(3) directions at the 16^3 x 32, N_v = 4
configuration (FP64 solves, step 1e-4)."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import rel_l2, to_device, to_numpy
from paper_2112_14640_gb300 import dirac as D
from paper_2112_14640_gb300 import inputs as I
from paper_2112_14640_gb300.autograd import PseudofermionAction

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout", [D.SITE_OUTER, D.SITE_INNER])
@pytest.mark.parametrize("prec,tol", [(D.F64, 1e-10), (D.F32, 1e-5)])
@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, -1, 1, -1)])
def test_force_kernel_matches_oracle(prec, tol, bc, layout):
    dims, nc, nv, m0 = (4, 4, 2, 6), 3, 3, 0.2
    U = I.gauge_field(dims, nc, 0.4, 41)
    op = D.DiracOp(D.WILSON, torch.from_numpy(U).cuda(), nv, bc, prec, layout=layout)
    ref = O.Operator(D.WILSON, U, bc)
    psi = I.source(dims, nc, nv, 42)
    x = to_device(op, psi)
    chi = op.apply(x, m0=m0)
    got_ta = op.force(x, chi, D.FORCE_TA).to(torch.complex128).cpu().numpy()
    got_g = op.force(x, chi, D.FORCE_GRAD).to(torch.complex128).cpu().numpy()
    chi_ref = ref.apply(psi, m0)
    assert rel_l2(got_ta, O.wilson_force(ref, psi, chi_ref)) <= tol
    assert rel_l2(got_g, O.wilson_action_gradient(ref, psi, chi_ref)) <= tol
    op.close()


def test_autograd_matches_oracle_gradient_f64():
    dims, nc, nv, m0, bc = (4, 4, 4, 4), 3, 2, 0.3, (1, 1, 1, -1)
    U_np = I.gauge_field(dims, nc, 0.4, 51)
    phi_np = I.source(dims, nc, nv, 52)
    U = torch.from_numpy(U_np).cuda().requires_grad_(True)
    phi = torch.from_numpy(phi_np).cuda().requires_grad_(True)
    act = PseudofermionAction(m0, bc, prec=D.F64, tol=1e-13)
    S = act(U, phi)
    gU, gphi = torch.autograd.grad(S, (U, phi))
    ref = O.Operator(D.WILSON, U_np, bc)
    S_ref, psi = O.pseudofermion_action(ref, phi_np, m0)
    assert abs(S.item() - S_ref) < 1e-11 * abs(S_ref)
    G_ref = O.wilson_action_gradient(ref, psi, ref.apply(psi, m0))
    assert rel_l2(gU.cpu().numpy(), G_ref) < 1e-10
    assert rel_l2(gphi.cpu().numpy(), 2 * psi) < 1e-10


def test_config5_finite_differences_16x16x16x32():
    """16^3 x 32, N_c = 3, N_v = 4: dS/deps along 16 random su(3) link directions
    (central differences, eps = 1e-4, FP64 solves) against the FP64 force, and
    the FP32-forward force against the oracle force on the FP64 solution."""
    dims, nc, nv, m0, bc = (16, 16, 16, 32), 3, 4, 0.2, (1, 1, 1, -1)
    U_np = I.gauge_field(dims, nc, 0.4, 61)
    phi_np = I.source(dims, nc, nv, 62)
    U = torch.from_numpy(U_np).cuda()
    phi = torch.from_numpy(phi_np).cuda()
    act64 = PseudofermionAction(m0, bc, prec=D.F64, tol=1e-12)
    F64 = act64.force(U, phi)
    act32 = PseudofermionAction(m0, bc, prec=D.F32, tol=1e-6)
    F32 = act32.force(U, phi)
    # oracle force on the FP64 solution
    op = act64.op
    x, st = op.solve(phi, m0=m0, solver=D.CG_HPD, tol=1e-12, maxit=20000)
    ref = O.Operator(D.WILSON, U_np, bc)
    xs = x.cpu().numpy()
    F_ref = O.wilson_force(ref, xs, ref.apply(xs, m0))
    assert rel_l2(F64.cpu().numpy(), F_ref) < 1e-10
    assert rel_l2(F32.to(torch.complex128).cpu().numpy(), F_ref) < 1e-4
    eps = 1e-4
    for k in range(16):
        X = torch.from_numpy(I.su_n_direction(dims, nc, seed=700 + k)).cuda()
        Sp = act64(torch.matrix_exp(eps * X) @ U, phi).item()
        Sm = act64(torch.matrix_exp(-eps * X) @ U, phi).item()
        fd = (Sp - Sm) / (2 * eps)
        an = torch.einsum("...ab,...ba->...", X, F64).real.sum().item()
        assert abs(fd - an) < 1e-5 * abs(an), (k, fd, an)


@pytest.mark.parametrize("layout", [D.SITE_OUTER, D.SITE_INNER])
@pytest.mark.parametrize("prec,tol", [(D.F64, 1e-10), (D.F32, 1e-5)])
@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, -1, 1, -1)])
def test_staggered_force_kernel_matches_oracle(prec, tol, bc, layout):
    """The staggered force (derived from Eq. def_stag) against the oracle's,
    both modes, on the same solution vector."""
    dims, nc, nv, m0 = (4, 4, 2, 6), 3, 3, 0.2
    U = I.gauge_field(dims, nc, 0.4, 43)
    op = D.DiracOp(D.STAGGERED, torch.from_numpy(U).cuda(), nv, bc, prec, layout=layout)
    ref = O.Operator(D.STAGGERED, U, bc)
    psi = I.source(dims, nc, nv, 44, staggered=True)
    x = to_device(op, psi)
    chi = op.apply(x, m0=m0)
    got_ta = op.force(x, chi, D.FORCE_TA).to(torch.complex128).cpu().numpy()
    got_g = op.force(x, chi, D.FORCE_GRAD).to(torch.complex128).cpu().numpy()
    chi_ref = ref.apply(psi, m0)
    assert rel_l2(got_ta, O.staggered_force(ref, psi, chi_ref)) <= tol
    assert rel_l2(got_g, O.staggered_action_gradient(ref, psi, chi_ref)) <= tol
    op.close()


def test_staggered_autograd_and_finite_differences():
    """Autograd of S = sum Re phi^dag (D_S^dag D_S)^-1 phi against the oracle's
    gradient, and the GPU force against central differences of the GPU action
    along random su(3) directions (FP64, 8^4, N_v = 3)."""
    dims, nc, nv, m0, bc = (8, 8, 8, 8), 3, 3, 0.3, (1, 1, 1, -1)
    U_np = I.gauge_field(dims, nc, 0.4, 53)
    phi_np = I.source(dims, nc, nv, 54, staggered=True)
    U = torch.from_numpy(U_np).cuda().requires_grad_(True)
    phi = torch.from_numpy(phi_np).cuda().requires_grad_(True)
    act = PseudofermionAction(m0, bc, prec=D.F64, tol=1e-13, kind=D.STAGGERED)
    S = act(U, phi)
    gU, gphi = torch.autograd.grad(S, (U, phi))
    ref = O.Operator(D.STAGGERED, U_np, bc)
    S_ref, psi = O.pseudofermion_action(ref, phi_np, m0)
    assert abs(S.item() - S_ref) < 1e-11 * abs(S_ref)
    assert rel_l2(gU.cpu().numpy(), O.staggered_action_gradient(ref, psi, ref.apply(psi, m0))) < 1e-10
    assert rel_l2(gphi.cpu().numpy(), 2 * psi) < 1e-10
    F = act.force(U.detach(), phi.detach()).cpu().numpy()
    eps = 1e-4
    for seed in range(4):
        X = I.su_n_direction(dims, nc, seed=400 + seed)
        wv, vv = np.linalg.eigh(-1j * eps * X)
        E = np.einsum("...ij,...j,...kj->...ik", vv, np.exp(1j * wv), vv.conj())
        Sp = act(torch.from_numpy(E @ U_np).cuda(), phi.detach()).item()
        Sm = act(torch.from_numpy(np.conj(np.swapaxes(E, -1, -2)) @ U_np).cuda(), phi.detach()).item()
        fd = (Sp - Sm) / (2 * eps)
        an = float(np.sum(np.real(np.einsum("...ab,...ba->...", X, F))))
        assert abs(fd - an) < 1e-5 * max(abs(an), 1.0), (seed, fd, an)


@pytest.mark.parametrize("layout", [D.SITE_OUTER, D.SITE_INNER])
@pytest.mark.parametrize("prec,tol", [(D.F64, 1e-10), (D.F32, 1e-5)])
@pytest.mark.parametrize("bc", [(1, 1, 1, 1), (1, -1, 1, -1)])
def test_brillouin_force_kernel_matches_oracle(prec, tol, bc, layout):
    """The Brillouin force (back-propagated through the W recursion) against
    the oracle's path-by-path derivative of Tab. off-axis, both modes."""
    dims, nc, nv, m0 = (4, 4, 2, 6), 3, 3, 0.2
    U = I.gauge_field(dims, nc, 0.4, 45)
    op = D.DiracOp(D.BRILLOUIN, torch.from_numpy(U).cuda(), nv, bc, prec, layout=layout)
    ref = O.Operator(D.BRILLOUIN, U, bc)
    psi = I.source(dims, nc, nv, 46)
    x = to_device(op, psi)
    chi = op.apply(x, m0=m0)
    got_ta = op.force(x, chi, D.FORCE_TA).to(torch.complex128).cpu().numpy()
    got_g = op.force(x, chi, D.FORCE_GRAD).to(torch.complex128).cpu().numpy()
    chi_ref = ref.apply(psi, m0)
    assert rel_l2(got_ta, O.brillouin_force(ref, psi, chi_ref)) <= tol
    assert rel_l2(got_g, O.brillouin_action_gradient(ref, psi, chi_ref)) <= tol
    op.close()


@pytest.mark.parametrize("dims,nc", [((2, 2, 2, 2), 3), ((3, 2, 3, 4), 2), ((2, 4, 2, 2), 5)])
def test_brillouin_force_small_lattices_and_nc(dims, nc):
    """Extent 2 (every offset wraps onto a neighbour, so forward and backward
    hops share links), odd extents, and N_c = 2, 5: FP64 against the oracle."""
    nv, m0, bc = 2, 0.1, (1, 1, 1, -1)
    U = I.gauge_field(dims, nc, 0.5, 47)
    op = D.DiracOp(D.BRILLOUIN, torch.from_numpy(U).cuda(), nv, bc, D.F64)
    ref = O.Operator(D.BRILLOUIN, U, bc)
    psi = I.source(dims, nc, nv, 48)
    x = to_device(op, psi)
    got = op.force(x, op.apply(x, m0=m0), D.FORCE_GRAD).cpu().numpy()
    assert rel_l2(got, O.brillouin_action_gradient(ref, psi, ref.apply(psi, m0))) <= 1e-10
    op.close()


def test_brillouin_autograd_and_finite_differences():
    """Autograd of S = sum Re phi^dag (D_B^dag D_B)^-1 phi against the
    oracle's gradient, and the GPU force against central differences of the
    GPU action along random su(3) directions (FP64, 8^4, N_v = 2)."""
    dims, nc, nv, m0, bc = (8, 8, 8, 8), 3, 2, 0.2, (1, 1, 1, -1)
    U_np = I.gauge_field(dims, nc, 0.4, 55)
    phi_np = I.source(dims, nc, nv, 56)
    U = torch.from_numpy(U_np).cuda().requires_grad_(True)
    phi = torch.from_numpy(phi_np).cuda().requires_grad_(True)
    act = PseudofermionAction(m0, bc, prec=D.F64, tol=1e-13, kind=D.BRILLOUIN)
    S = act(U, phi)
    gU, gphi = torch.autograd.grad(S, (U, phi))
    ref = O.Operator(D.BRILLOUIN, U_np, bc)
    S_ref, psi = O.pseudofermion_action(ref, phi_np, m0)
    assert abs(S.item() - S_ref) < 1e-11 * abs(S_ref)
    assert rel_l2(gU.cpu().numpy(), O.brillouin_action_gradient(ref, psi, ref.apply(psi, m0))) < 1e-10
    assert rel_l2(gphi.cpu().numpy(), 2 * psi) < 1e-10
    F = act.force(U.detach(), phi.detach()).cpu().numpy()
    eps = 1e-4
    for seed in range(4):
        X = I.su_n_direction(dims, nc, seed=500 + seed)
        wv, vv = np.linalg.eigh(-1j * eps * X)
        E = np.einsum("...ij,...j,...kj->...ik", vv, np.exp(1j * wv), vv.conj())
        Sp = act(torch.from_numpy(E @ U_np).cuda(), phi.detach()).item()
        Sm = act(torch.from_numpy(np.conj(np.swapaxes(E, -1, -2)) @ U_np).cuda(), phi.detach()).item()
        fd = (Sp - Sm) / (2 * eps)
        an = float(np.sum(np.real(np.einsum("...ab,...ba->...", X, F))))
        assert abs(fd - an) < 1e-5 * max(abs(an), 1.0), (seed, fd, an)
