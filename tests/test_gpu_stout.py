"""GPU stout smearing (dirac_stout_smear) against the FP64 oracle: the
smeared field element by element (FP64 1e-12, FP32 storage 1e-6 relative
L2), in place and out of place, several N_c and step counts; and the
paper's solver setting, where D and the clover term are both built from
the smeared field, checked through the operators against the oracle; and
the chain rule of the force through the smearing (dirac_stout_backward),
against the oracle's and, composed with the pseudofermion action by
autograd, against finite differences."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import TOL, rel_l2, to_device, to_numpy
from paper_2112_14640_gb300 import dirac as D
from paper_2112_14640_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nc,dims,nsteps", [(3, (4, 4, 4, 4), 3), (3, (6, 4, 2, 8), 1), (2, (4, 2, 4, 6), 2),
                                             (4, (2, 4, 4, 2), 3), (1, (4, 4, 2, 2), 2)])
def test_stout_matches_oracle(nc, dims, nsteps):
    U = I.gauge_field(dims, nc, 0.5, seed=90 + nc)
    want = O.stout_smear(U, 0.12, nsteps)
    Ut = torch.from_numpy(U).cuda()
    got = D.stout_smear(Ut, 0.12, nsteps).cpu().numpy()
    assert rel_l2(got, want) < 1e-12
    # in place, FP64
    D.stout_smear(Ut, 0.12, nsteps, out=Ut)
    assert rel_l2(Ut.cpu().numpy(), want) < 1e-12
    # FP32 storage (FP64 arithmetic per step, FP32 rounding between steps)
    U32 = torch.from_numpy(U).to(torch.complex64).cuda()
    got32 = D.stout_smear(U32, 0.12, nsteps).cpu().numpy().astype(np.complex128)
    assert rel_l2(got32, want) < 1e-6
    assert np.array_equal(D.stout_smear(U32, 0.12, 0).cpu().numpy(), U32.cpu().numpy())


def test_stout_full_size_unitarity_and_sampled_links():
    """16^3 x 32 with the paper's rho = 0.12, three steps: every smeared link
    unitary with det 1, and sampled links against the oracle (which smears
    the whole field in FP64)."""
    dims = (16, 16, 16, 32)
    U = I.gauge_field(dims, 3, 0.4, seed=2024)
    V = D.stout_smear(torch.from_numpy(U).cuda(), 0.12, 3).cpu().numpy()
    assert np.abs(V @ np.conj(np.swapaxes(V, -1, -2)) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(V) - 1).max() < 1e-13
    want = O.stout_smear(U, 0.12, 3)
    rng = np.random.default_rng(3)
    idx = tuple(rng.integers(0, e, 64) for e in (32, 16, 16, 16))
    assert rel_l2(V[idx], want[idx]) < 1e-12


@pytest.mark.parametrize("kind", [D.WILSON, D.BRILLOUIN])
def test_operators_on_smeared_field_with_clover(kind):
    """The paper's solver setting: V from three steps of rho = 0.12 stout
    smearing, D and the clover term (c_SW = 1) both from V."""
    dims, nc, nv, bc = (4, 4, 4, 6), 3, 4, (1, 1, 1, -1)
    U = I.gauge_field(dims, nc, 0.6, seed=95)
    V = D.stout_smear(torch.from_numpy(U).cuda(), 0.12, 3)
    op = D.DiracOp(kind, V, nv, bc, D.F64)
    op.set_clover(1.0, V)
    ref = O.Operator(kind, O.stout_smear(U, 0.12, 3), bc, csw=1.0)
    src = I.source(dims, nc, nv, 96)
    x = to_device(op, src)
    for dag in (False, True):
        got = to_numpy(op, op.apply(x, m0=-0.1, dagger=dag))
        want = ref.apply_dagger(src, -0.1) if dag else ref.apply(src, -0.1)
        assert rel_l2(got, want) <= TOL[D.F64]
    op.close()


def test_stout_extent_two():
    """Extent 2 in every direction: a link's forward and backward staples
    share links, and n + mu - nu wraps twice."""
    U = I.gauge_field((2, 2, 2, 2), 3, 0.7, seed=97)
    want = O.stout_smear(U, 0.12, 3)
    got = D.stout_smear(torch.from_numpy(U).cuda(), 0.12, 3).cpu().numpy()
    assert rel_l2(got, want) < 1e-12


@pytest.mark.parametrize("prec,tol", [(torch.complex128, 1e-11), (torch.complex64, 1e-5)])
@pytest.mark.parametrize("dims,nc,nsteps", [((4, 4, 2, 4), 3, 3), ((2, 4, 3, 2), 2, 1), ((4, 2, 2, 2), 4, 2)])
def test_stout_backward_matches_oracle(prec, tol, dims, nc, nsteps):
    """The chain rule through stout smearing on the GPU against the oracle's
    (which is pinned by finite differences on the CPU), for a random complex
    G_V; the block-exponential Frechet derivative against the oracle's
    eigenbasis formula."""
    U_np = I.gauge_field(dims, nc, 0.5, 91)
    rng = np.random.default_rng(92)
    G_np = rng.standard_normal(U_np.shape) + 1j * rng.standard_normal(U_np.shape)
    U = torch.from_numpy(U_np).cuda().to(prec)
    G = torch.from_numpy(G_np).cuda().to(prec)
    got = D.stout_backward(U, G, 0.12, nsteps).to(torch.complex128).cpu().numpy()
    Uw = U_np if prec == torch.complex128 else U_np.astype(np.complex64).astype(np.complex128)
    Gw = G_np if prec == torch.complex128 else G_np.astype(np.complex64).astype(np.complex128)
    want = O.stout_backward(Uw, Gw, 0.12, nsteps)
    assert rel_l2(got, want) <= tol


def test_smeared_action_autograd_and_finite_differences():
    """S(U) = sum Re phi^dag (D_W[V]^dag D_W[V])^-1 phi with V = stout^3(U),
    differentiated by autograd through PseudofermionAction and stout_smear:
    against the oracle's chain rule and against central differences of the
    GPU action along random complex directions (FP64, 4^4, N_v = 2)."""
    from paper_2112_14640_gb300.autograd import PseudofermionAction, stout_smear
    dims, nc, nv, m0, bc, rho, ns = (4, 4, 4, 4), 3, 2, 0.3, (1, 1, 1, -1), 0.12, 3
    U_np = I.gauge_field(dims, nc, 0.4, 93)
    phi_np = I.source(dims, nc, nv, 94)
    U = torch.from_numpy(U_np).cuda().requires_grad_(True)
    phi = torch.from_numpy(phi_np).cuda()
    act = PseudofermionAction(m0, bc, prec=D.F64, tol=1e-13)
    S = act(stout_smear(U, rho, ns), phi)
    gU, = torch.autograd.grad(S, (U,))
    V_np = O.stout_smear(U_np, rho, ns)
    ref = O.Operator(O.WILSON, V_np, bc)
    S_ref, psi = O.pseudofermion_action(ref, phi_np, m0)
    assert abs(S.item() - S_ref) < 1e-10 * abs(S_ref)
    want = O.stout_backward(U_np, O.wilson_action_gradient(ref, psi, ref.apply(psi, m0)), rho, ns)
    assert rel_l2(gU.cpu().numpy(), want) < 1e-9
    rng = np.random.default_rng(95)
    for _ in range(3):
        dU = torch.from_numpy(rng.standard_normal(U_np.shape) + 1j * rng.standard_normal(U_np.shape)).cuda()
        eps = 1e-5
        with torch.no_grad():
            Sp = act(stout_smear(U + eps * dU, rho, ns), phi).item()
            Sm = act(stout_smear(U - eps * dU, rho, ns), phi).item()
        fd = (Sp - Sm) / (2 * eps)
        an = torch.sum(torch.real(torch.conj(gU) * dU)).item()
        assert abs(fd - an) < 1e-6 * abs(an), (fd, an)
