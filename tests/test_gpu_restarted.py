"""Restarted Arnoldi through the C ABI (ovl_sign_arnoldi_restarted: cycles of m delayed-CGS2 steps
on a double-float basis of m + 1 vectors, the accumulated Hessenberg matrix's inner sign by the
resolvent quadrature) against the oracle's restarted Arnoldi (oracle.krylov.sign_arnoldi_restarted,
the same restart with Roberts' iteration for the inner sign), the dense sgn(A) b on 4^4, the
unrestarted solve for one cycle, and the free-field closed form where the Krylov space is
invariant."""
import numpy as np
import pytest

from gpu_common import KAPPA, config4, rel, torch_c128
from oracle import deflation as Dm
from oracle import freefield as F
from oracle import krylov as K
from oracle import wilson as W
from paper_0810_4228_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ovl():
    from paper_0810_4228_gb300 import ovl as O
    O.load()
    return O


def _deflated_ctx(ovl, c4, m=20):
    lam, X, Xi = c4["lam"], c4["X"], c4["Xi"]
    idx = np.argsort(np.abs(lam.real))[:m]
    ctx = ovl.Context(c4["dims"])
    ctx.set_gauge(torch_c128(c4["U"]))
    ctx.set_deflation(c4["mu"], KAPPA, lam[idx], torch_c128(np.ascontiguousarray(X[:, idx].T)),
                      torch_c128(np.ascontiguousarray(Xi[idx, :].conj())))
    defl = Dm.Deflation(lam=lam[idx], R=X[:, idx], L=Xi[idx, :].conj().T)
    return ctx, defl


def test_one_cycle_equals_unrestarted(ovl):
    c4 = config4()
    ctx = ovl.Context(c4["dims"])
    ctx.set_gauge(torch_c128(c4["U"]))
    b = torch_c128(c4["b"])
    for m in (1, 7, 60):
        y1, info = ctx.sign_arnoldi_restarted(m, 1, c4["mu"], KAPPA, b)
        y0, _ = ctx.sign_krylov(ovl.ARNOLDI, m, c4["mu"], KAPPA, b, flags=ovl.MIXED)
        assert info["k_used"] == m
        assert rel(y1.cpu().numpy(), y0.cpu().numpy()) < 1e-12


@pytest.mark.parametrize("m,cycles", [(10, 4), (30, 10)])
def test_matches_oracle_restart_and_dense(ovl, m, cycles):
    """Deflated (20 exact eigenpairs) on 4^4: the oracle's restarted process to 1e-9; at 30 x 10
    the dense sgn(A) b to 1e-10."""
    c4 = config4()
    ctx, defl = _deflated_ctx(ovl, c4)
    y, info = ctx.sign_arnoldi_restarted(m, cycles, c4["mu"], KAPPA, torch_c128(c4["b"]))
    assert info["status"] == 0 and info["k_used"] == m * cycles
    y = y.cpu().numpy()
    yo = K.sign_arnoldi_restarted(c4["A"].dot, c4["b"], m, cycles, defl)
    assert rel(y, yo) < 1e-9
    if cycles == 10:
        assert rel(y, c4["ref"]) < 1e-10
        # D_ov b
        yov, _ = ctx.sign_arnoldi_restarted(m, cycles, c4["mu"], KAPPA, torch_c128(c4["b"]), flags=ovl.OVERLAP)
        g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), 256)
        assert rel(yov.cpu().numpy(), c4["b"] + g5 * c4["ref"]) < 1e-10


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (3, 2, 5, 4)])
def test_small_ragged_lattices(ovl, dims):
    U = synth.gauge_field(dims, 0.4, 41)
    A = W.a_operator(U, dims, 0.3, KAPPA)
    b = synth.gaussian_source(dims, 42)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    for m, cyc in ((8, 5), (20, 6)):
        y, _ = ctx.sign_arnoldi_restarted(m, cyc, 0.3, KAPPA, torch_c128(b))
        assert rel(y.cpu().numpy(), K.sign_arnoldi_restarted(A.dot, b, m, cyc)) < 1e-9


def test_invariant_krylov_space(ovl):
    """A one-momentum free-field source spans a two-dimensional Krylov space: the process stops in
    the first cycle (info k_used <= 2) at the closed form, with the later cycles doing nothing."""
    dims, mu = (4, 4, 4, 4), 0.3
    V = 256
    t = np.arange(V) % 4
    rng = np.random.default_rng(77)
    spin = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    b = (np.exp(1j * np.pi * 3 * t / 4)[:, None] * spin[None, :]).reshape(-1)
    g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), V)
    ref = g5 * (F.overlap_free_apply(dims, mu, KAPPA, b) - b)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(synth.free_gauge_field(dims)))
    y, info = ctx.sign_arnoldi_restarted(10, 5, mu, KAPPA, torch_c128(b))
    assert info["status"] == 0 and info["k_used"] <= 2, info
    assert rel(y.cpu().numpy(), ref) < 1e-10


def test_fully_deflated_and_zero_source(ovl):
    """A source inside the deflated space gives the exact part R sgn(Lambda) L^dag b alone; a zero
    source gives zero (the restarted process does not start)."""
    c4 = config4()
    ctx, defl = _deflated_ctx(ovl, c4)
    b = defl.R @ (np.arange(1, 21) * (1 + 0.5j))
    y, info = ctx.sign_arnoldi_restarted(10, 3, c4["mu"], KAPPA, torch_c128(b))
    assert info["k_used"] == 0
    ref = defl.R @ (np.sign(defl.lam.real) * (defl.L.conj().T @ b))
    assert rel(y.cpu().numpy(), ref) < 1e-10
    z, info = ctx.sign_arnoldi_restarted(10, 3, c4["mu"], KAPPA, torch_c128(np.zeros_like(b)))
    assert info["k_used"] == 0 and np.abs(z.cpu().numpy()).max() == 0.0
