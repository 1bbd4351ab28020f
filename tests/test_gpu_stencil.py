"""GPU parity of the Wilson stencil kernels (Sec. 1, Eq. 1.2) against the FP64
oracle, through the C ABI: A = gamma5 D_w(mu), A^dag, D_w, the pair form of
the two-sided Lanczos step, FP64 / FP32-12 / FP32-18 links, ragged and
degenerate lattice shapes, host and device pointers."""
import numpy as np
import pytest

from gpu_common import KAPPA, maxrel, torch_c128
from oracle import wilson as W
from paper_0810_4228_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (2, 2, 2, 2), (2, 2, 2, 4), (3, 2, 5, 4), (6, 4, 2, 8), (8, 8, 8, 8)]


@pytest.fixture(scope="module")
def ovl():
    from paper_0810_4228_gb300 import ovl as O
    O.load()
    return O


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("mu", [0.0, 0.3])
@pytest.mark.parametrize("bc_t", [-1, 1])
@pytest.mark.parametrize("layout", ["SITE", "SPLIT"])
def test_A_fp64(ovl, dims, mu, bc_t, layout):
    U = synth.gauge_field(dims, 1.0, 7)
    x = synth.gaussian_source(dims, 8)
    ref = W.a_operator(U, dims, mu, KAPPA, bc_t) @ x
    ctx = ovl.Context(dims, bc_t)
    ctx.set_gauge(torch_c128(U))
    fl = ovl.GAMMA5 | getattr(ovl, "STENCIL_" + layout)
    y = ctx.apply_Dw(mu, KAPPA, torch_c128(x), flags=fl).cpu().numpy()
    assert maxrel(y, ref) < 1e-14


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 4)])
def test_dw_and_dagger_fp64(ovl, dims):
    mu = 0.4
    U = synth.gauge_field(dims, 1.0, 9)
    x = synth.gaussian_source(dims, 10)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    y = ctx.apply_Dw(mu, KAPPA, torch_c128(x), flags=0).cpu().numpy()
    assert maxrel(y, W.wilson_dirac(U, dims, mu, KAPPA) @ x) < 1e-14
    y = ctx.apply_Dw(mu, KAPPA, torch_c128(x), flags=ovl.DAGGER).cpu().numpy()
    A = W.a_operator(U, dims, mu, KAPPA)
    assert maxrel(y, A.conj().T @ x) < 1e-14


@pytest.mark.parametrize("flag,tol", [("F32", 3e-6), ("F32_FULL", 3e-6)])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 2, 5, 4), (8, 8, 8, 8)])
@pytest.mark.parametrize("layout", ["SITE", "SPLIT"])
def test_A_fp32(ovl, dims, flag, tol, layout):
    mu = 0.3
    U = synth.gauge_field(dims, 1.0, 11)
    x = synth.gaussian_source(dims, 12)
    ref = W.a_operator(U, dims, mu, KAPPA) @ x
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    fl = ovl.GAMMA5 | getattr(ovl, flag) | getattr(ovl, "STENCIL_" + layout)
    y = ctx.apply_Dw(mu, KAPPA, torch_c128(x), flags=fl).cpu().numpy()
    assert maxrel(y, ref) < tol


def test_host_pointers(ovl):
    dims, mu = (4, 4, 2, 4), 0.25
    U = synth.gauge_field(dims, 1.0, 13)
    x = synth.gaussian_source(dims, 14)
    ctx = ovl.Context(dims)
    ctx.set_gauge(np.ascontiguousarray(U))
    y = ctx.apply_Dw(mu, KAPPA, np.ascontiguousarray(x), flags=ovl.GAMMA5)
    assert isinstance(y, np.ndarray)
    assert maxrel(y, W.a_operator(U, dims, mu, KAPPA) @ x) < 1e-14


def test_pack_roundtrip_and_native(ovl):
    import torch
    dims, mu = (4, 2, 4, 6), 0.3
    U = synth.gauge_field(dims, 1.0, 15)
    x = synth.gaussian_source(dims, 16)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    xc = torch_c128(x)
    nat = ctx.empty_native(0)
    ctx.pack(xc, nat, 0)
    back = torch.empty_like(xc)
    ctx.unpack(nat, back, 0)
    assert torch.equal(back, xc)
    out = ctx.empty_native(0)
    ctx.apply_Dw(mu, KAPPA, nat, out, flags=ovl.GAMMA5 | ovl.NATIVE)
    ctx.unpack(out, back, 0)
    assert maxrel(back.cpu().numpy(), W.a_operator(U, dims, mu, KAPPA) @ x) < 1e-14


@pytest.mark.parametrize("prec,tol", [(0, 1e-14), (1, 3e-6)])
def test_pair(ovl, prec, tol):
    """t = A v, s = A^dag w and alpha = w^dag t in one pass (Sec. 4, Eq. 4.2)."""
    import torch
    dims, mu = (4, 4, 4, 4), 0.3
    U = synth.gauge_field(dims, 1.0, 17)
    v = synth.gaussian_source(dims, 18)
    w = synth.gaussian_source(dims, 19)
    A = W.a_operator(U, dims, mu, KAPPA)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    nv, nw = ctx.empty_native(0), ctx.empty_native(0)
    ctx.pack(torch_c128(v), nv, 0)
    ctx.pack(torch_c128(w), nw, 0)
    if prec == 1:
        nv32, nw32 = ctx.empty_native(1), ctx.empty_native(1)
        ctx.pack(torch_c128(v), nv32, 1)
        ctx.pack(torch_c128(w), nw32, 1)
        nv, nw = nv32, nw32
    t, s = ctx.empty_native(prec), ctx.empty_native(prec)
    alpha = ctx.apply_pair(mu, KAPPA, nv, nw, t, s, prec)
    tc = torch.empty(ctx.n, dtype=torch.complex128, device="cuda")
    sc = torch.empty_like(tc)
    ctx.unpack(t, tc, prec)
    ctx.unpack(s, sc, prec)
    tr, sr = A @ v, A.conj().T @ w
    assert maxrel(tc.cpu().numpy(), tr) < tol
    assert maxrel(sc.cpu().numpy(), sr) < tol
    ar = np.vdot(w, tr)
    assert abs(alpha - ar) / abs(ar) < (1e-12 if prec == 0 else 1e-5)


@pytest.mark.parametrize("site", [0, 1, 777, 4095])
def test_sampled_sites_8x4(ovl, site):
    """8^4 FP64 against the oracle's single-site evaluator."""
    dims, mu = (8, 8, 8, 8), 0.5
    U = synth.gauge_field(dims, 1.0, 21)
    x = synth.gaussian_source(dims, 22)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    y = ctx.apply_Dw(mu, KAPPA, torch_c128(x), flags=ovl.GAMMA5).cpu().numpy()
    np.testing.assert_allclose(y[12 * site:12 * site + 12], W.wilson_site(U, dims, mu, KAPPA, x, site), atol=1e-13)


def test_invalid_arguments(ovl):
    with pytest.raises(ovl.OvlError):
        ovl.Context((4, 4, 4, 3))  # odd time extent
    with pytest.raises(ovl.OvlError):
        ovl.Context((1, 4, 4, 4))
    ctx = ovl.Context((2, 2, 2, 2))
    import torch
    x = torch.zeros(192, dtype=torch.complex128, device="cuda")
    with pytest.raises(ovl.OvlError) as e:
        ctx.apply_Dw(0.1, KAPPA, x)  # no gauge field
    assert e.value.code == ovl.ESTATE


@pytest.mark.parametrize("layout", ["SITE", "SPLIT"])
def test_large_lattice_sampled(ovl, layout):
    """24^4 (331776 sites, above the split threshold): sampled sites of the FP64
    and FP32-12 stencils against the oracle's single-site evaluator."""
    dims, mu = (24, 24, 24, 24), 0.3
    U = synth.gauge_field(dims, 1.0, 23)
    x = synth.gaussian_source(dims, 24)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    fl = getattr(ovl, "STENCIL_" + layout)
    y = ctx.apply_Dw(mu, KAPPA, torch_c128(x), flags=ovl.GAMMA5 | fl).cpu().numpy()
    y32 = ctx.apply_Dw(mu, KAPPA, torch_c128(x), flags=ovl.GAMMA5 | ovl.F32 | fl).cpu().numpy()
    rng = np.random.default_rng(25)
    for site in list(rng.integers(0, 331776, 6)) + [0, 331775]:
        ref = W.wilson_site(U, dims, mu, KAPPA, x, int(site))
        np.testing.assert_allclose(y[12 * site:12 * site + 12], ref, atol=1e-13)
        np.testing.assert_allclose(y32[12 * site:12 * site + 12], ref, atol=3e-5)


@pytest.mark.parametrize("dims", [(16, 16, 16, 48), (20, 14, 16, 48)])
def test_row_grouped_traversal_sampled(ovl, dims):
    """Lattices whose (x0, x1) rows are whole 64-site blocks take the row-grouped block order of the
    single stencil (groups of x1 rows, x0 inside a group): 16^3 x 48 (groups of 16 rows) and
    20 x 14 x 16 x 48 (one group of 14).  Sampled sites, among them the first and last of rows and
    of the lattice, of the FP64, FP32-12 and FP32-18 stencils against the oracle's single-site
    evaluator; the one-thread-per-site and direction-split layouts agree."""
    mu = 0.3
    V = dims[0] * dims[1] * dims[2] * dims[3]
    U = synth.gauge_field(dims, 1.0, 31)
    x = synth.gaussian_source(dims, 32)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    xs = torch_c128(x)
    y = ctx.apply_Dw(mu, KAPPA, xs, flags=ovl.GAMMA5 | ovl.STENCIL_SITE).cpu().numpy()
    ys = ctx.apply_Dw(mu, KAPPA, xs, flags=ovl.GAMMA5 | ovl.STENCIL_SPLIT).cpu().numpy()
    assert maxrel(y, ys) < 1e-14
    y12 = ctx.apply_Dw(mu, KAPPA, xs, flags=ovl.GAMMA5 | ovl.F32 | ovl.STENCIL_SITE).cpu().numpy()
    y18 = ctx.apply_Dw(mu, KAPPA, xs, flags=ovl.GAMMA5 | ovl.F32_FULL | ovl.STENCIL_SITE).cpu().numpy()
    row = dims[2] * dims[3]
    rng = np.random.default_rng(33)
    sites = [0, 1, row - 1, row, V // 2 - 1, V // 2, V - row, V - 1] + list(rng.integers(0, V, 8))
    for site in sites:
        ref = W.wilson_site(U, dims, mu, KAPPA, x, int(site))
        np.testing.assert_allclose(y[12 * site:12 * site + 12], ref, atol=1e-13)
        np.testing.assert_allclose(y12[12 * site:12 * site + 12], ref, atol=3e-5)
        np.testing.assert_allclose(y18[12 * site:12 * site + 12], ref, atol=3e-5)


@pytest.mark.parametrize("prec,tol", [(0, 1e-14), (1, 3e-6)])
def test_pair_row_grouped_large(ovl, prec, tol):
    """The fused pair on a lattice that takes the row-grouped block order (16^3 x 48): t = A v and
    s = A^dag w against the single stencil (itself checked against the oracle there) and at
    sampled sites against the oracle's single-site evaluator; alpha = w^dag t (reduced over the
    three-dimensional grid in linear block order) against torch's FP64 inner product of the
    results."""
    import torch
    dims, mu = (16, 16, 16, 48), 0.3
    V = dims[0] * dims[1] * dims[2] * dims[3]
    U = synth.gauge_field(dims, 1.0, 41)
    v = synth.gaussian_source(dims, 42)
    w = synth.gaussian_source(dims, 43)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    nv, nw = ctx.empty_native(prec), ctx.empty_native(prec)
    ctx.pack(torch_c128(v), nv, prec)
    ctx.pack(torch_c128(w), nw, prec)
    t, s = ctx.empty_native(prec), ctx.empty_native(prec)
    alpha = ctx.apply_pair(mu, KAPPA, nv, nw, t, s, prec)
    tc = torch.empty(ctx.n, dtype=torch.complex128, device="cuda")
    sc = torch.empty_like(tc)
    ctx.unpack(t, tc, prec)
    ctx.unpack(s, sc, prec)
    tr = ctx.apply_Dw(mu, KAPPA, torch_c128(v), flags=ovl.GAMMA5)
    sr = ctx.apply_Dw(mu, KAPPA, torch_c128(w), flags=ovl.DAGGER)
    assert maxrel(tc.cpu().numpy(), tr.cpu().numpy()) < tol
    assert maxrel(sc.cpu().numpy(), sr.cpu().numpy()) < tol
    ar = torch.vdot(torch_c128(w), tc).item()
    assert abs(alpha - ar) / abs(ar) < (1e-12 if prec == 0 else 1e-5)
    t_np = tc.cpu().numpy()
    for site in (0, V // 2 + 7, V - 1):
        ref = W.wilson_site(U, dims, mu, KAPPA, v, site)
        np.testing.assert_allclose(t_np[12 * site:12 * site + 12], ref, atol=1e-13 if prec == 0 else 3e-5)
