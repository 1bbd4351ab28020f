"""Gradients of l = Re <g, sgn(A) b>, A = gamma5 D_w(mu; U), from the library's
resolvent-form derivative (ovl_sign_grad: one two-sided Lanczos process from
(b, g)), against the oracle's Frechet derivative of sgn (oracle.frechet.frechet_sign_dk,
Daleckii-Krein on the dense 4^4 operator, itself pinned to the block-triangular form and to
finite differences) in FP64 and in the mixed-precision form, and against central differences
of the GPU forward at 8^4."""
import numpy as np
import pytest

from gpu_common import KAPPA, config4, rel, torch_c128
from oracle import frechet as Fr
from oracle import sign as S
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


def _link_direction_matrix(U, dU, dims, mu):
    """(dA/dU)[dU] as a sparse matrix: the hopping part of A built from dU (forward hops) and
    dU^dag (backward hops)."""
    import scipy.sparse as sp
    V = int(np.prod(dims))
    I = sp.identity(12 * V, dtype=np.complex128, format="csr")
    return (W.gamma5_operator(V) @ (W.wilson_dirac(dU, dims, mu, KAPPA) - I)).tocsr()


@pytest.fixture(scope="module")
def frechet4():
    """The oracle's Frechet derivatives L(A, E) (Daleckii-Krein, oracle.frechet.frechet_sign_dk) at
    the 4^4 workload for E = dA/dmu and E = dA/dU[dU] with a seeded direction dU, applied to b."""
    c4 = config4()
    Ad = c4["A"].toarray()
    rng = np.random.default_rng(2200)
    dU = rng.standard_normal(c4["U"].shape) + 1j * rng.standard_normal(c4["U"].shape)
    E_mu = Fr.dA_dmu(c4["U"], c4["dims"], c4["mu"], KAPPA).toarray()
    E_U = _link_direction_matrix(c4["U"], dU, c4["dims"], c4["mu"]).toarray()
    return {"dU": dU, "Lmu_b": Fr.frechet_sign_dk(Ad, E_mu) @ c4["b"], "LU_b": Fr.frechet_sign_dk(Ad, E_U) @ c4["b"]}


@pytest.fixture(scope="module")
def grad4(mods):
    """GPU gradients at 4^4, k = 400, for a Gaussian cotangent g."""
    torch, O, AG = mods
    c4 = config4()
    g = synth.gaussian_source(c4["dims"], 2100)
    lat = O.Context(c4["dims"])
    lat.set_gauge(torch_c128(c4["U"]))
    y = torch.empty(lat.n, dtype=torch.complex128, device="cuda")
    gU = torch.empty(c4["U"].shape, dtype=torch.complex128, device="cuda")
    gb = torch.empty(lat.n, dtype=torch.complex128, device="cuda")
    gmu, info = lat.sign_grad(400, c4["mu"], KAPPA, torch_c128(c4["b"]), torch_c128(g), y=y, grad_U=gU,
                              grad_b=gb)
    out = dict(g=g, y=y.cpu().numpy(), gU=gU.cpu().numpy(), gb=gb.cpu().numpy(), gmu=gmu, info=info)
    lat.close()
    return c4, out


def test_sign_grad_forward_matches_dense(grad4):
    c4, o = grad4
    assert o["info"]["k_used"] > 0
    assert rel(o["y"], c4["ref"]) < 1e-10


def test_sign_grad_mu_vs_frechet(grad4, frechet4):
    c4, o = grad4
    ref = float(np.real(np.vdot(o["g"], frechet4["Lmu_b"])))
    assert abs(o["gmu"] - ref) <= 1e-6 * abs(ref), (o["gmu"], ref)


def test_sign_grad_links_vs_frechet(grad4, frechet4):
    c4, o = grad4
    ref = float(np.real(np.vdot(o["g"], frechet4["LU_b"])))
    got = float(np.real(np.vdot(o["gU"].ravel(), frechet4["dU"].ravel())))
    assert abs(got - ref) <= 1e-6 * abs(ref), (got, ref)


def test_sign_grad_mixed_vs_frechet(mods, grad4, frechet4):
    """The mixed-precision gradient (OVL_MIXED: the two-sided Lanczos process in FP32 with 12-real
    links, FP64 coefficients and quadrature, the combination and link force in FP32) against the
    same Frechet derivatives: the link-direction derivative, y and g_b within 1e-4; d/dmu, a sum
    with cancellation (only the temporal hops depend on mu), within 5e-3 (measured 1.3e-3 on GB300;
    at 8^4 and k = 800 the mixed d/dmu is within 4e-6 of the FP64 one)."""
    torch, O, AG = mods
    c4, o = grad4
    lat = O.Context(c4["dims"])
    lat.set_gauge(torch_c128(c4["U"]))
    y = torch.empty(lat.n, dtype=torch.complex128, device="cuda")
    gU = torch.empty(c4["U"].shape, dtype=torch.complex128, device="cuda")
    gb = torch.empty(lat.n, dtype=torch.complex128, device="cuda")
    gmu, info = lat.sign_grad(400, c4["mu"], KAPPA, torch_c128(c4["b"]), torch_c128(o["g"]), y=y, grad_U=gU,
                              grad_b=gb, flags=O.MIXED)
    ref_mu = float(np.real(np.vdot(o["g"], frechet4["Lmu_b"])))
    ref_U = float(np.real(np.vdot(o["g"], frechet4["LU_b"])))
    got_U = float(np.real(np.vdot(gU.cpu().numpy().ravel(), frechet4["dU"].ravel())))
    err_mu, err_U = abs(gmu - ref_mu) / abs(ref_mu), abs(got_U - ref_U) / abs(ref_U)
    print(f"mixed gradient: rel err d/dmu {err_mu:.2e}, dU direction {err_U:.2e}, "
          f"y {rel(y.cpu().numpy(), c4['ref']):.2e}, g_b vs FP64 {rel(gb.cpu().numpy(), o['gb']):.2e}")
    assert err_mu <= 5e-3 and err_U <= 1e-4, (err_mu, err_U, gmu, ref_mu)
    assert rel(y.cpu().numpy(), c4["ref"]) < 1e-4
    assert rel(gb.cpu().numpy(), o["gb"]) < 1e-4
    lat.close()


def test_sign_grad_source_vs_dense(grad4):
    """l is linear in b for the exact sign: g_b = sgn(A)^dag g."""
    c4, o = grad4
    X, Xi, lam = c4["X"], c4["Xi"], c4["lam"]
    ref = Xi.conj().T @ (np.conj(S.csign(lam)) * (X.conj().T @ o["g"]))
    assert rel(o["gb"], ref) < 1e-6


def test_sign_grad_repeat_is_deterministic(mods):
    torch, O, AG = mods
    dims, mu = (4, 4, 2, 4), 0.3
    U = synth.gauge_field(dims, 0.5, 2300)
    b = torch_c128(synth.gaussian_source(dims, 2301))
    g = torch_c128(synth.gaussian_source(dims, 2302))
    lat = O.Context(dims)
    lat.set_gauge(torch_c128(U))
    res = []
    for _ in range(2):
        gU = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
        gb = torch.empty(lat.n, dtype=torch.complex128, device="cuda")
        gmu, _ = lat.sign_grad(120, mu, KAPPA, b, g, grad_U=gU, grad_b=gb)
        res.append((gmu, gU.cpu().numpy(), gb.cpu().numpy()))
    assert res[1][0] == res[0][0]
    assert np.array_equal(res[1][1], res[0][1])
    assert np.array_equal(res[1][2], res[0][2])
    lat.close()


def test_sign_function_autograd(mods):
    """SignFunction routes loss.backward() to ovl_sign_grad."""
    torch, O, AG = mods
    dims, mu, k = (4, 4, 2, 4), 0.25, 150
    U = synth.gauge_field(dims, 0.5, 2400)
    b = synth.gaussian_source(dims, 2401)
    g = synth.gaussian_source(dims, 2402)
    lat = O.Context(dims)
    Ut = torch_c128(U).requires_grad_(True)
    mut = torch.tensor(mu, dtype=torch.float64, device="cuda", requires_grad=True)
    bt = torch_c128(b).requires_grad_(True)
    y = AG.sign_A(Ut, mut, bt, lat, KAPPA, k)
    L = torch.real(torch.vdot(torch_c128(g), y))
    L.backward()
    gU = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
    gb = torch.empty(lat.n, dtype=torch.complex128, device="cuda")
    lat.set_gauge(torch_c128(U))
    gmu, _ = lat.sign_grad(k, mu, KAPPA, torch_c128(b), torch_c128(g), grad_U=gU, grad_b=gb)
    assert mut.grad.item() == gmu
    assert torch.equal(Ut.grad, gU)
    assert torch.equal(bt.grad, gb)
    lat.close()


def test_sign_grad_zero_source(mods):
    torch, O, AG = mods
    dims = (2, 2, 2, 4)
    lat = O.Context(dims)
    lat.set_gauge(torch_c128(synth.gauge_field(dims, 0.5, 2500)))
    b = torch.zeros(lat.n, dtype=torch.complex128, device="cuda")
    g = torch_c128(synth.gaussian_source(dims, 2501))
    gU = torch.full((lat.V, 4, 3, 3), 7.0, dtype=torch.complex128, device="cuda")
    gb = torch.full((lat.n,), 7.0, dtype=torch.complex128, device="cuda")
    gmu, info = lat.sign_grad(20, 0.3, KAPPA, b, g, grad_U=gU, grad_b=gb)
    assert gmu == 0.0 and info["k_used"] == 0
    assert not torch.any(gU) and not torch.any(gb)
    lat.close()


def test_sign_grad_8x4_vs_central_differences(mods):
    """8^4 (eps = 1.0, mu = 0.3): the derivative of the converged k = 800 solve against central
    differences of the GPU forward (step 1e-4: truncation ~1e-8, forward noise ~1e-11 / 1e-4)."""
    torch, O, AG = mods
    dims, mu, k, h = (8, 8, 8, 8), 0.3, 800, 1e-4
    U = synth.gauge_field(dims, 1.0, 1001)
    b = torch_c128(synth.gaussian_source(dims, 2001))
    g = torch_c128(synth.gaussian_source(dims, 2600))
    rng = np.random.default_rng(2601)
    dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    lat = O.Context(dims)
    lat.set_gauge(torch_c128(U))
    gU = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
    gmu, _ = lat.sign_grad(k, mu, KAPPA, b, g, grad_U=gU)

    def loss(Uc, m):
        lat.set_gauge(torch_c128(Uc))
        y, _ = lat.sign_krylov(O.LANCZOS2, k, m, KAPPA, b)
        return float(torch.real(torch.vdot(g, y)).item())

    fd_mu = (loss(U, mu + h) - loss(U, mu - h)) / (2 * h)
    fd_U = (loss(U + h * dU, mu) - loss(U - h * dU, mu)) / (2 * h)
    got_U = float(np.real(np.vdot(gU.cpu().numpy().ravel(), dU.ravel())))
    assert abs(gmu - fd_mu) <= 1e-5 * abs(fd_mu), (gmu, fd_mu)
    assert abs(got_U - fd_U) <= 1e-5 * abs(fd_U), (got_U, fd_U)
    lat.close()
