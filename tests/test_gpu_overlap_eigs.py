"""Eigenvalues of the overlap operator nearest 0 (Eq. 1.1; the application Sec. 5 names), through
the C ABI (ovl_overlap_eigs: thick-restart Arnoldi with D_ov applied by the library's sign
solves) against the oracle's dense spectrum of D_ov (oracle.sign.overlap_eigenvalues), and at
mu = 0 against the circle |lambda - 1| = 1 on which the whole spectrum lies there."""
import numpy as np
import pytest

from gpu_common import KAPPA, config4, gamma5_diag, torch_c128
from oracle import sign as S
from oracle import wilson as W
from paper_0810_4228_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ovl():
    from paper_0810_4228_gb300 import ovl as O
    O.load()
    return O


def _match(got, ref_sorted, tol):
    """Every computed eigenvalue lies within tol of an eigenvalue of the oracle, and every oracle
    eigenvalue clearly nearer 0 than the farthest computed one was found (no gap in the set)."""
    got = np.asarray(got)
    for g in got:
        assert np.min(np.abs(ref_sorted - g)) <= tol, (g, ref_sorted[:len(got) + 2])
    rmax = np.abs(got).max()
    for r in ref_sorted[np.abs(ref_sorted) < rmax - 1e-6]:
        assert np.min(np.abs(got - r)) <= tol, (r, got)


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_small_lattice_exhausted_krylov(ovl, mu):
    """2^3 x 4 (N = 384): Arnoldi with k = N applies D_ov exactly (Krylov space exhausted, Sec. 2),
    so the 6 eigenvalues nearest 0 match the dense spectrum to 1e-9, with eigenvectors whose
    residual |D_ov x - lambda x| is below 1e-9."""
    import torch
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 1.0, 501)
    A = W.dense_a(U, dims, mu, KAPPA)
    ref = S.overlap_eigenvalues(A, gamma5_diag(32))
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    vecs = torch.empty((6, 384), dtype=torch.complex128, device="cuda")
    lam, info = ctx.overlap_eigs(ovl.ARNOLDI, 384, mu, KAPPA, 6, nkrylov=40, tol=1e-11, vecs=vecs)
    assert info["nconv"] == 6 and info["max_residual"] < 1e-9, info
    assert np.all(np.diff(np.abs(lam)) >= -1e-12)
    _match(lam, ref, 1e-9)
    # the eigenvectors against the dense operator
    D = S.overlap_dense(A, gamma5_diag(32))
    X = vecs.cpu().numpy()
    for i in range(6):
        assert np.linalg.norm(D @ X[i] - lam[i] * X[i]) < 1e-9
    if mu == 0.0:
        np.testing.assert_allclose(np.abs(lam - 1.0), 1.0, atol=1e-10)


def test_4x4_deflated_lanczos2(ovl):
    """4^4 (N = 3072), mu = 0.3, D_ov applied by deflated two-sided Lanczos (20 exact eigenpairs,
    k = 300; relative error about 1e-11): the 8 eigenvalues nearest 0 match the oracle's dense
    spectrum of D_ov to 1e-8; the same through the mixed-precision two-pass solve to 1e-6."""
    c = config4()
    lam, X, Xi = c["lam"], c["X"], c["Xi"]
    sgn = X @ (S.csign(lam)[:, None] * Xi)
    ref = S.overlap_eigenvalues(c["A"], gamma5_diag(256), sign=sgn)
    idx = np.argsort(np.abs(lam.real))[:20]
    ctx = ovl.Context(c["dims"])
    ctx.set_gauge(torch_c128(c["U"]))
    ctx.set_deflation(c["mu"], KAPPA, lam[idx], torch_c128(np.ascontiguousarray(X[:, idx].T)),
                      torch_c128(np.ascontiguousarray(Xi[idx, :].conj())))
    got, info = ctx.overlap_eigs(ovl.LANCZOS2, 300, c["mu"], KAPPA, 8, tol=1e-10)
    assert info["nconv"] == 8 and info["max_residual"] < 1e-8, info
    _match(got, ref, 1e-8)
    gm, info = ctx.overlap_eigs(ovl.LANCZOS2, 300, c["mu"], KAPPA, 8, flags=ovl.MIXED, tol=1e-8)
    _match(gm, ref, 1e-6)


def test_zero_mu_circle_4x4(ovl):
    """At mu = 0 D_ov = 1 + gamma5 sgn(H), H = gamma5 D_w Hermitian, is 1 plus a unitary matrix: the
    computed eigenvalues nearest 0 lie on |lambda - 1| = 1 (4^4, undeflated Arnoldi, k = 400)."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.5, 1000)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    got, info = ctx.overlap_eigs(ovl.ARNOLDI, 400, 0.0, KAPPA, 6, tol=1e-9)
    assert info["nconv"] == 6
    np.testing.assert_allclose(np.abs(got - 1.0), 1.0, atol=1e-8)
