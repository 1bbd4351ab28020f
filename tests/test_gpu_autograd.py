"""Gradients of y = gamma5 D_w(mu; U) x (Sec. 1, Eq. 1.2) through the library's
adjoint kernels, against the oracle's derivatives of A (finite-difference
pinned) and against finite differences of the GPU forward itself."""
import numpy as np
import pytest

from gpu_common import KAPPA, torch_c128
from oracle import frechet as Fr
from oracle import wilson as W
from paper_0810_4228_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    from paper_0810_4228_gb300 import autograd as AG
    from paper_0810_4228_gb300 import ovl as O
    O.load()
    return torch, O, AG


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (4, 4, 2, 4)])
def test_dw_gradients_vs_oracle(mods, dims):
    """L = Re <w, A x>: dL/dmu = Re <w, dA/dmu x>, dL along dU = Re <w, dA/dU[dU] x>
    = Re sum conj(grad_U) dU, grad_x = A^dag w (PyTorch's complex-gradient convention)."""
    torch, O, AG = mods
    mu = 0.3
    U = synth.gauge_field(dims, 1.0, 61)
    x = synth.gaussian_source(dims, 62)
    w = synth.gaussian_source(dims, 63)
    rng = np.random.default_rng(64)
    dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    lat = O.Context(dims)
    Ut = torch_c128(U).requires_grad_(True)
    mut = torch.tensor(mu, dtype=torch.float64, device="cuda", requires_grad=True)
    xt = torch_c128(x).requires_grad_(True)
    wt = torch_c128(w)
    y = AG.apply_A(Ut, mut, xt, lat, KAPPA)
    L = torch.real(torch.vdot(wt, y))
    L.backward()
    A = W.a_operator(U, dims, mu, KAPPA)
    ref_mu = np.real(np.vdot(w, Fr.dA_dmu(U, dims, mu, KAPPA) @ x))
    assert abs(mut.grad.item() - ref_mu) <= 1e-12 * max(1.0, abs(ref_mu))
    ref_dir = np.real(np.vdot(w, Fr.dA_dU_apply(U, dU, dims, mu, KAPPA, x)))
    got_dir = np.real(np.vdot(Ut.grad.cpu().numpy().ravel(), dU.ravel()))
    assert abs(got_dir - ref_dir) <= 1e-11 * max(1.0, abs(ref_dir))
    np.testing.assert_allclose(xt.grad.cpu().numpy(), A.conj().T @ w, atol=1e-13)


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (4, 4, 4, 4)])
def test_dw_gradients_f32_vs_oracle(mods, dims):
    """The FP32 form of the stencil adjoint (OVL_F32: the link force in FP32) against the oracle's
    dA/dU: relative error below 1e-6; d/dmu (FP64 in both forms) as in FP64."""
    torch, O, AG = mods
    mu = 0.3
    U = synth.gauge_field(dims, 1.0, 61)
    x = synth.gaussian_source(dims, 62)
    w = synth.gaussian_source(dims, 63)
    rng = np.random.default_rng(64)
    dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    lat = O.Context(dims)
    lat.set_gauge(torch_c128(U))
    gU = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
    _, gmu = lat.dw_grad(mu, KAPPA, torch_c128(x), torch_c128(w), gU, flags=O.F32)
    ref_dir = np.real(np.vdot(w, Fr.dA_dU_apply(U, dU, dims, mu, KAPPA, x)))
    got_dir = np.real(np.vdot(gU.cpu().numpy().ravel(), dU.ravel()))
    assert abs(got_dir - ref_dir) <= 1e-6 * abs(ref_dir), (got_dir, ref_dir)
    ref_mu = np.real(np.vdot(w, Fr.dA_dmu(U, dims, mu, KAPPA) @ x))
    assert abs(gmu - ref_mu) <= 1e-12 * max(1.0, abs(ref_mu))
    gU64 = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
    lat.dw_grad(mu, KAPPA, torch_c128(x), torch_c128(w), gU64)
    assert (gU - gU64).abs().max().item() <= 1e-6 * gU64.abs().max().item()


def test_dw_gradients_vs_finite_differences(mods):
    torch, O, AG = mods
    dims, mu = (4, 2, 2, 4), 0.25
    U = synth.gauge_field(dims, 1.0, 71)
    x = synth.gaussian_source(dims, 72)
    w = synth.gaussian_source(dims, 73)
    lat = O.Context(dims)
    Ut = torch_c128(U).requires_grad_(True)
    mut = torch.tensor(mu, dtype=torch.float64, device="cuda", requires_grad=True)
    y = AG.apply_A(Ut, mut, torch_c128(x), lat, KAPPA)
    L = torch.real(torch.vdot(torch_c128(w), y))
    L.backward()

    def Lval(Uv, m):
        yy = lat.apply_Dw(m, KAPPA, torch_c128(x)) if Uv is None else None
        if Uv is not None:
            lat.set_gauge(torch_c128(Uv))
            yy = lat.apply_Dw(m, KAPPA, torch_c128(x))
            lat.set_gauge(torch_c128(U))
        return float(torch.real(torch.vdot(torch_c128(w), yy)).item())

    lat.set_gauge(torch_c128(U))
    h = 1e-5
    fd_mu = (Lval(None, mu + h) - Lval(None, mu - h)) / (2 * h)
    assert abs(mut.grad.item() - fd_mu) < 1e-7 * max(1, abs(fd_mu))
    rng = np.random.default_rng(74)
    dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    fd_u = (Lval(U + h * dU, mu) - Lval(U - h * dU, mu)) / (2 * h)
    got = np.real(np.vdot(Ut.grad.cpu().numpy().ravel(), dU.ravel()))
    assert abs(got - fd_u) < 1e-6 * max(1, abs(fd_u))
