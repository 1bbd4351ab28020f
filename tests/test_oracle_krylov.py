"""Pins of the oracle's Krylov approximations (Secs. 2-5) against the dense
spectral sign, exactness statements of the paper (interpolation at all
eigenvalues, full deflation), the Krylov relations, closed forms on
(gauge-transformed) free fields, and a brute-force full-dimension run."""
import numpy as np
import pytest

from oracle import deflation as Dm
from oracle import freefield as F
from oracle import krylov as K
from oracle import sign as S
from oracle import wilson as W
from paper_0810_4228_gb300 import synth


def _setup(dims, mu=0.3, eps=0.8, seed=31, kappa=0.2):
    U = synth.gauge_field(dims, eps, seed)
    A = W.a_operator(U, dims, mu, kappa)
    Ad = A.conj().T.tocsr()
    return U, A, Ad


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_arnoldi_relations():
    _, A, _ = _setup((2, 2, 2, 4))
    b = synth.gaussian_source((2, 2, 2, 4), seed=1)
    k = 30
    V, H, nb = K.arnoldi(A.dot, b, k)
    np.testing.assert_allclose(V.conj().T @ V, np.eye(k + 1), atol=1e-12)
    np.testing.assert_allclose(A @ V[:, :k], V @ H, atol=1e-12)
    np.testing.assert_allclose(np.tril(H[:k, :k], -2), 0, atol=0)
    np.testing.assert_allclose(V[:, :k].conj().T @ (A @ V[:, :k]), H[:k, :k], atol=1e-12)
    np.testing.assert_allclose(V[:, 0] * nb, b, atol=1e-12)


def test_arnoldi_full_dimension_is_exact():
    """k = N: the implicit polynomial interpolates sgn at every eigenvalue
    of A, so the approximation is exact (Sec. 2, Eq. 2.1)."""
    dims = (2, 2, 2, 2)
    _, A, _ = _setup(dims)
    b = synth.gaussian_source(dims, seed=2)
    ref = S.sign_spectral(A.toarray()) @ b
    y = K.sign_arnoldi(A.dot, b, 192)
    assert _rel(y, ref) < 1e-10


def test_lanczos2_relations():
    _, A, Ad = _setup((2, 2, 2, 4))
    b = synth.gaussian_source((2, 2, 2, 4), seed=3)
    v1 = b / np.linalg.norm(b)
    k = 25
    V, Wm, a, be, ga = K.lanczos2(A.dot, Ad.dot, v1, v1, k)
    np.testing.assert_allclose(Wm.conj().T @ V, np.eye(k), atol=1e-9)
    G = K.tridiag(a, be, ga)
    np.testing.assert_allclose(Wm.conj().T @ (A @ V), G, atol=1e-9)
    np.testing.assert_allclose(be.imag, 0, atol=0)  # beta_i = |v_hat| is real positive
    assert (be.real > 0).all()


@pytest.mark.parametrize("method", ["arnoldi", "lanczos2"])
def test_converges_to_dense(method):
    dims = (2, 2, 2, 4)
    _, A, Ad = _setup(dims, eps=0.3, seed=5)
    b = synth.gaussian_source(dims, seed=4)
    ref = S.sign_spectral(A.toarray()) @ b
    errs = []
    for k in (20, 60, 200):
        if method == "arnoldi":
            y = K.sign_arnoldi(A.dot, b, k)
        else:
            y = K.sign_lanczos2(A.dot, Ad.dot, b, k)
        errs.append(_rel(y, ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6


def test_full_deflation_is_exact():
    """m = N: b_perp = 0 and R sgn(Lambda) L^dag b is sgn(A) b (Sec. 3, Eq. 3.3)."""
    dims = (2, 2, 2, 2)
    _, A, Ad = _setup(dims)
    Ad_ = A.toarray()
    b = synth.gaussian_source(dims, seed=5)
    defl = Dm.eigenpairs_dense(Ad_, 192)
    ref = S.sign_spectral(Ad_) @ b
    for fn in (lambda: K.sign_arnoldi(A.dot, b, 5, defl),
               lambda: K.sign_lanczos2(A.dot, Ad.dot, b, 5, defl)):
        assert _rel(fn(), ref) < 1e-10


def test_deflated_pieces():
    """b_parallel = R L^dag b lies in span(R); A maps span(R) into itself and
    b_perp^R, b_perp^L are annihilated by L^dag and R^dag."""
    dims = (2, 2, 2, 4)
    _, A, _ = _setup(dims)
    Ad_ = A.toarray()
    defl = Dm.eigenpairs_dense(Ad_, 12)
    np.testing.assert_allclose(Ad_ @ defl.R, defl.R * defl.lam, atol=1e-11)
    np.testing.assert_allclose(defl.L.conj().T @ Ad_, defl.lam[:, None] * defl.L.conj().T, atol=1e-11)
    np.testing.assert_allclose(defl.L.conj().T @ defl.R, np.eye(12), atol=1e-11)
    b = synth.gaussian_source(dims, seed=6)
    exact, bR, bL = K._split(b, defl)
    np.testing.assert_allclose(defl.L.conj().T @ bR, 0, atol=1e-11)
    np.testing.assert_allclose(defl.R.conj().T @ bL, 0, atol=1e-11)


@pytest.mark.parametrize("method", ["arnoldi", "lanczos2"])
def test_deflated_converges_faster(method):
    dims = (2, 2, 2, 4)
    _, A, Ad = _setup(dims, eps=1.0)
    Ad_ = A.toarray()
    b = synth.gaussian_source(dims, seed=7)
    ref = S.sign_spectral(Ad_) @ b
    defl = Dm.eigenpairs_dense(Ad_, 24)
    k = 50
    if method == "arnoldi":
        e0 = _rel(K.sign_arnoldi(A.dot, b, k), ref)
        e1 = _rel(K.sign_arnoldi(A.dot, b, k, defl), ref)
        e2 = _rel(K.sign_arnoldi(A.dot, b, 200, defl), ref)
    else:
        e0 = _rel(K.sign_lanczos2(A.dot, Ad.dot, b, k), ref)
        e1 = _rel(K.sign_lanczos2(A.dot, Ad.dot, b, k, defl), ref)
        e2 = _rel(K.sign_lanczos2(A.dot, Ad.dot, b, 200, defl), ref)
    assert e1 < e0
    assert e2 < 1e-9


def test_twopass_equals_onepass():
    dims = (2, 2, 2, 4)
    _, A, Ad = _setup(dims)
    Ad_ = A.toarray()
    b = synth.gaussian_source(dims, seed=8)
    defl = Dm.eigenpairs_dense(Ad_, 8)
    for d in (None, defl):
        y1 = K.sign_lanczos2(A.dot, Ad.dot, b, 70, d)
        y2 = K.sign_lanczos2_twopass(A.dot, Ad.dot, b, 70, d)
        assert _rel(y2, y1) < 1e-11


def test_newton_inner_equals_spectral_inner():
    dims = (2, 2, 2, 4)
    _, A, Ad = _setup(dims)
    b = synth.gaussian_source(dims, seed=9)
    y1 = K.sign_lanczos2(A.dot, Ad.dot, b, 80, inner="spectral")
    y2 = K.sign_lanczos2(A.dot, Ad.dot, b, 80, inner="newton")
    assert _rel(y2, y1) < 1e-11


@pytest.mark.parametrize("gauge", [False, True])
def test_free_field_4x4_closed_form(gauge):
    """4^4, U = 1 (or a gauge transform of it), mu = 0.3: both Krylov methods
    reproduce the momentum-space closed form of D_ov b.  The free spectrum has
    few distinct eigenvalues (fewer than 120), so k = 120 is exact."""
    dims, mu, kappa = (4, 4, 4, 4), 0.3, 0.2
    V = 256
    b = synth.gaussian_source(dims, seed=10)
    ref = F.overlap_free_apply(dims, mu, kappa, b)
    if gauge:
        g = synth.gauge_transformation(dims, seed=11)
        fwd, _, _, _ = W.neighbours(dims)
        U = np.einsum("vab,vndb->vnad", g, g[fwd].conj())
        Gb = np.einsum("vab,vsb->vsa", g, b.reshape(V, 4, 3)).reshape(-1)
        ref = np.einsum("vab,vsb->vsa", g, ref.reshape(V, 4, 3)).reshape(-1)
        b = Gb
    else:
        U = synth.free_gauge_field(dims)
    A = W.a_operator(U, dims, mu, kappa)
    Ad = A.conj().T.tocsr()
    g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), V)
    ya = K.sign_arnoldi(A.dot, b, 120)
    yl = K.sign_lanczos2(A.dot, Ad.dot, b, 120)
    assert _rel(b + g5 * ya, ref) < 1e-10
    assert _rel(b + g5 * yl, ref) < 1e-10


def test_free_plane_wave_two_steps():
    """On the free field a source of one momentum p (any spin-colour part) spans an
    A-invariant space of dimension two: A(p) = 2 kappa gamma5 (a - i gamma.s) gives
    A(p)^2 = 4 kappa^2 (a^2 + s.s) (gamma5 anticommutes with every gamma_nu), so the Arnoldi
    process stops with a lucky breakdown after two steps and its result is the closed form."""
    dims, mu, kappa = (4, 4, 4, 4), 0.3, 0.2
    V = 256
    t = np.arange(V) % 4  # time fastest
    rng = np.random.default_rng(77)
    spin = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    b = (np.exp(1j * np.pi * 3 * t / 4)[:, None] * spin[None, :]).reshape(-1)  # p_4 = 3 pi / 4
    A = W.a_operator(synth.free_gauge_field(dims), dims, mu, kappa)
    # A^2 b is a multiple of b, with the closed-form factor
    p4 = 3 * np.pi / 4 - 1j * mu
    a = -1.5 + (1 - np.cos(p4))  # m_w = 1/(2 kappa) - 4 = -1.5; spatial momenta zero
    ss = np.sin(p4) ** 2
    np.testing.assert_allclose(A.dot(A.dot(b)), 4 * kappa ** 2 * (a * a + ss) * b, rtol=1e-12, atol=1e-12)
    _, H, _ = K.arnoldi(A.dot, b, 10)
    assert H.shape[1] == 2 and abs(H[2, 1]) < 1e-13
    g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), V)
    ref = F.overlap_free_apply(dims, mu, kappa, b)
    assert _rel(b + g5 * K.sign_arnoldi(A.dot, b, 10), ref) < 1e-12


def test_breakdowns():
    """Lucky breakdown (v_hat = 0: K_1 is invariant, the process stops and the
    result is exact) and serious breakdown (v_hat, w_hat nonzero, w_hat^dag
    v_hat = 0) of the two-sided Lanczos recurrences of Sec. 4."""
    M = np.diag([1.0, 2.0, -1.5, 3.0]).astype(complex)
    v1 = np.array([1, 0, 0, 0], dtype=complex)
    w1 = np.array([1, 1, 0, 0], dtype=complex)
    V, Wm, a, be, ga = K.lanczos2(M.dot, M.conj().T.dot, v1, w1, 3)
    assert len(a) == 1 and a[0] == 1
    y = K.sign_lanczos2(M.dot, M.conj().T.dot, v1, 3)
    np.testing.assert_allclose(y, v1, atol=1e-15)
    # A e1 = (0, 1, -1), A^dag e1 = (0, 1, 1): orthogonal, both nonzero
    M2 = np.array([[0, 1, 1], [1, 0, 0], [-1, 0, 2]], dtype=complex)
    e1 = np.array([1, 0, 0], dtype=complex)
    with pytest.raises(K.KrylovBreakdown) as ei:
        K.lanczos2(M2.dot, M2.conj().T.dot, e1, e1, 3)
    assert ei.value.step == 1


@pytest.mark.slow
def test_config_4x4_no_deflation():
    """4^4, eps = 0.5, mu = 0.3, kappa = 0.2, k = 200, no deflation: both
    methods approximate the dense sgn(A) b, Arnoldi somewhat better than
    two-sided Lanczos at equal k (Sec. 5)."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.5, 1000)
    A = W.a_operator(U, dims, 0.3, 0.2)
    Ad = A.conj().T.tocsr()
    b = synth.gaussian_source(dims, 2000)
    ref = S.sign_spectral(A.toarray()) @ b
    ea = _rel(K.sign_arnoldi(A.dot, b, 200), ref)
    el = _rel(K.sign_lanczos2(A.dot, Ad.dot, b, 200), ref)
    assert ea < 1e-6 and el < 1e-5
    assert ea < el
    # at k = 300 both are far below 1e-8
    assert _rel(K.sign_lanczos2(A.dot, Ad.dot, b, 300), ref) < 1e-8
