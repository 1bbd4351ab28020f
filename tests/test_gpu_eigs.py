"""GPU deflation phase (Sec. 3, Eq. 3.1; Sec. 5): the critical left/right
eigenpairs computed by the library against the dense eigendecomposition
(4^4) and against their defining relations (8^4)."""
import numpy as np
import pytest

from gpu_common import KAPPA, config4, rel, torch_c128
from oracle import wilson as W
from paper_0810_4228_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ovl():
    from paper_0810_4228_gb300 import ovl as O
    O.load()
    return O


def _check_pairs(A, lam, R, L, tol):
    R = R.T  # (N, m)
    L = L.T
    nA = 3.0
    assert np.abs(A @ R - R * lam).max() <= tol * nA
    assert np.abs((A.conj().T @ L).conj().T - lam[:, None] * L.conj().T).max() <= tol * nA
    assert np.abs(L.conj().T @ R - np.eye(len(lam))).max() <= 1e-9


def test_eigs_4x4_vs_dense(ovl):
    c4 = config4()
    m, extra = 12, 6
    ctx = ovl.Context(c4["dims"])
    ctx.set_gauge(torch_c128(c4["U"]))
    info = ctx.deflation_eigs(c4["mu"], KAPPA, m, nextra=extra, tol=1e-11)
    lam, R, L = ctx.get_deflation(device=False)
    assert info["m"] == m and len(lam) == m
    # the same selection applied to the dense spectrum: the m of smallest |Re| among the
    # m + extra of smallest |lambda|
    w = c4["lam"]
    near = w[np.argsort(np.abs(w))[:m + extra]]
    ref = np.sort_complex(near[np.argsort(np.abs(near.real))[:m]])
    np.testing.assert_allclose(np.sort_complex(lam), ref, atol=1e-9)
    _check_pairs(c4["A"], lam, R, L, 1e-9)
    # the installed deflation drives a solve to the dense result
    y, _ = ctx.sign_krylov(ovl.LANCZOS2, 300, c4["mu"], KAPPA, torch_c128(c4["b"]))
    assert rel(y.cpu().numpy(), c4["ref"]) < 1e-10


def test_eigs_8x4_relations(ovl):
    """8^4, eps = 1.0, mu = 0.3, m = 20: eigenpair residuals, bi-orthonormality,
    and a deflated mixed solve that agrees with the undeflated FP64 one."""
    dims, mu = (8, 8, 8, 8), 0.3
    U = synth.gauge_field(dims, 1.0, 1001)
    A = W.a_operator(U, dims, mu, KAPPA)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    b = synth.gaussian_source(dims, 2001)
    y0, _ = ctx.sign_krylov(ovl.LANCZOS2, 900, mu, KAPPA, torch_c128(b))
    info = ctx.deflation_eigs(mu, KAPPA, 20, nextra=10, tol=1e-10)
    lam, R, L = ctx.get_deflation(device=False)
    assert len(lam) == 20
    assert np.abs(lam.real).max() < 0.2  # the critical end of the spectrum
    _check_pairs(A, lam, R, L, 1e-9)
    y1, _ = ctx.sign_krylov(ovl.LANCZOS2, 600, mu, KAPPA, torch_c128(b), flags=ovl.MIXED)
    assert rel(y1.cpu().numpy(), y0.cpu().numpy()) < 1e-8
