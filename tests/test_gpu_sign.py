"""GPU parity of sgn(A) b and D_ov(mu) b (Secs. 1-5) through the C ABI against
the FP64 oracle: the dense spectral sign on 4^4 (N = 3072), the oracle's own
Krylov runs of the same algorithm, LR deflation with the oracle's exact
eigenpairs, the mixed-precision two-pass form, closed forms on free and
gauge-transformed free fields at 8^4, and the degenerate cases."""
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


@pytest.fixture(scope="module")
def c4():
    return config4()


def _ctx(ovl, dims, U):
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    return ctx


def _solve(ovl, ctx, method, k, mu, b, flags=0):
    out, info = ctx.sign_krylov(method, k, mu, KAPPA, torch_c128(b), flags=flags)
    return out.cpu().numpy(), info


def test_lanczos2_fp64_matches_dense(ovl, c4):
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    y, info = _solve(ovl, ctx, ovl.LANCZOS2, 400, c4["mu"], c4["b"])
    assert info["status"] == 0 and info["k_used"] == 400
    assert rel(y, c4["ref"]) < 1e-10


def test_arnoldi_fp64_matches_dense(ovl, c4):
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    y, info = _solve(ovl, ctx, ovl.ARNOLDI, 300, c4["mu"], c4["b"])
    assert info["status"] == 0
    assert rel(y, c4["ref"]) < 1e-10


def test_arnoldi_doublefloat_matches_dense_and_fp64(ovl, c4):
    """Arnoldi with the basis and the Gram-Schmidt sweeps in double-float arithmetic (about 48
    significant bits): the same process as the FP64 run, so within 1e-10 of the dense sgn(A) b at
    k = 300 and within 1e-11 of the FP64 Arnoldi result at equal k."""
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    y, info = _solve(ovl, ctx, ovl.ARNOLDI, 300, c4["mu"], c4["b"], flags=ovl.MIXED)
    assert info["status"] == 0 and info["k_used"] == 300
    assert rel(y, c4["ref"]) < 1e-10
    y64, _ = _solve(ovl, ctx, ovl.ARNOLDI, 300, c4["mu"], c4["b"])
    assert rel(y, y64) < 1e-11
    yo, _ = _solve(ovl, ctx, ovl.ARNOLDI, 300, c4["mu"], c4["b"], flags=ovl.MIXED | ovl.OVERLAP)
    g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), 256)
    assert rel(yo, c4["b"] + g5 * y) < 1e-14


@pytest.mark.parametrize("method", ["arnoldi", "arnoldi_df", "lanczos2"])
@pytest.mark.parametrize("k", [1, 2, 7, 60])
def test_same_algorithm_parity(ovl, c4, method, k):
    """At equal k the GPU and the oracle run the same algorithm; before the
    two-sided Lanczos loses bi-orthogonality their results agree far below the
    approximation error itself."""
    A = c4["A"]
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    if method.startswith("arnoldi"):
        yo = K.sign_arnoldi(A.dot, c4["b"], k)
        y, _ = _solve(ovl, ctx, ovl.ARNOLDI, k, c4["mu"], c4["b"], flags=ovl.MIXED if method == "arnoldi_df" else 0)
    else:
        Ad = A.conj().T.tocsr()
        yo = K.sign_lanczos2(A.dot, Ad.dot, c4["b"], k)
        y, _ = _solve(ovl, ctx, ovl.LANCZOS2, k, c4["mu"], c4["b"])
    assert rel(y, yo) < 1e-9


@pytest.mark.parametrize("k", [150, 200, 250])
def test_lanczos2_error_matches_oracle_error(ovl, c4, k):
    """Past the loss of bi-orthogonality the recurrence amplifies rounding (a
    1e-15 change of b moves the oracle's own k = 200 result by ~6e-8), so the
    comparison is of the distance to the dense sgn(A) b, which both runs share."""
    A = c4["A"]
    yo = K.sign_lanczos2(A.dot, A.conj().T.tocsr().dot, c4["b"], k)
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    y, _ = _solve(ovl, ctx, ovl.LANCZOS2, k, c4["mu"], c4["b"])
    eo, eg = rel(yo, c4["ref"]), rel(y, c4["ref"])
    assert eg <= 3 * eo + 1e-12 and eo <= 3 * eg + 1e-12, (eg, eo)


def test_overlap_output(ovl, c4):
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    y, _ = _solve(ovl, ctx, ovl.LANCZOS2, 400, c4["mu"], c4["b"], flags=ovl.OVERLAP)
    g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), 256)
    ref = c4["b"] + g5 * c4["ref"]
    assert rel(y, ref) < 1e-10


@pytest.mark.parametrize("method", ["arnoldi", "arnoldi_df", "lanczos2"])
def test_deflated_matches_dense(ovl, c4, method):
    """m = 20 exact eigenpairs of smallest |Re lambda| (Sec. 3, Eq. 3.4; Sec. 4, Eq. 4.5)."""
    lam, X, Xi = c4["lam"], c4["X"], c4["Xi"]
    idx = np.argsort(np.abs(lam.real))[:20]
    R = np.ascontiguousarray(X[:, idx].T)
    L = np.ascontiguousarray(Xi[idx, :].conj())
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    ctx.set_deflation(c4["mu"], KAPPA, lam[idx], torch_c128(R), torch_c128(L))
    m = ovl.LANCZOS2 if method == "lanczos2" else ovl.ARNOLDI
    fl = ovl.MIXED if method == "arnoldi_df" else 0
    y, info = _solve(ovl, ctx, m, 300, c4["mu"], c4["b"], flags=fl)
    assert info["status"] == 0
    assert rel(y, c4["ref"]) < 1e-10
    # same algorithm at small k
    defl = Dm.Deflation(lam=lam[idx], R=X[:, idx], L=Xi[idx, :].conj().T)
    A = c4["A"]
    if m == ovl.ARNOLDI:
        yo = K.sign_arnoldi(A.dot, c4["b"], 40, defl)
    else:
        yo = K.sign_lanczos2(A.dot, A.conj().T.tocsr().dot, c4["b"], 40, defl)
    y40, _ = _solve(ovl, ctx, m, 40, c4["mu"], c4["b"], flags=fl)
    assert rel(y40, yo) < 1e-9


def test_deflation_biorthonormalises(ovl, c4):
    """L is rescaled internally so that L^dag R = I: scaling the given left
    vectors must not change the result."""
    lam, X, Xi = c4["lam"], c4["X"], c4["Xi"]
    idx = np.argsort(np.abs(lam.real))[:8]
    R = np.ascontiguousarray(X[:, idx].T)
    L = np.ascontiguousarray(Xi[idx, :].conj()) * (1.7 - 0.4j)
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    ctx.set_deflation(c4["mu"], KAPPA, lam[idx], torch_c128(R), torch_c128(L))
    y, _ = _solve(ovl, ctx, ovl.LANCZOS2, 400, c4["mu"], c4["b"])
    assert rel(y, c4["ref"]) < 1e-10


_METHODS = {"lanczos2": ("LANCZOS2", 0), "arnoldi": ("ARNOLDI", 0), "arnoldi_df": ("ARNOLDI", "MIXED")}


def _method(ovl, name):
    m, f = _METHODS[name]
    return getattr(ovl, m), (getattr(ovl, f) if f else 0)


@pytest.mark.parametrize("method", list(_METHODS))
def test_fully_deflated_source(ovl, c4, method):
    """b an eigenvector in the deflated set: b_perp = 0 and sgn(A) b is exact."""
    lam, X, Xi = c4["lam"], c4["X"], c4["Xi"]
    idx = np.argsort(np.abs(lam.real))[:4]
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    ctx.set_deflation(c4["mu"], KAPPA, lam[idx], torch_c128(X[:, idx].T.copy()), torch_c128(Xi[idx, :].conj().copy()))
    b = X[:, idx[1]].copy()
    m, fl = _method(ovl, method)
    y, info = _solve(ovl, ctx, m, 10, c4["mu"], b, flags=fl)
    assert info["k_used"] == 0 and info["bperp_norm"] < 1e-12
    assert rel(y, np.sign(lam[idx[1]].real) * b) < 1e-12


@pytest.mark.parametrize("method", list(_METHODS))
def test_zero_source(ovl, c4, method):
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    m, fl = _method(ovl, method)
    y, info = _solve(ovl, ctx, m, 10, c4["mu"], np.zeros_like(c4["b"]), flags=fl)
    assert np.abs(y).max() == 0.0


def test_arnoldi_lucky_breakdown(ovl):
    """A source spanned by a few plane waves of the free field (U = 1) has a Krylov space of
    small dimension: the Arnoldi process stops early (H[j+1, j] ~ 0, Sec. 2) in FP64 and in
    double-float, and the result is the closed form."""
    dims, mu = (4, 4, 4, 4), 0.3
    V = 256
    x = np.arange(V)
    t = x % 4  # t fastest
    rng = np.random.default_rng(77)
    spin = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    b = (np.exp(1j * np.pi * (2 * 1 + 1) * t / 4)[:, None] * spin[None, :]).reshape(-1)  # one momentum
    ref = F.overlap_free_apply(dims, mu, KAPPA, b) - b
    g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), V)
    ref = g5 * ref
    ctx = _ctx(ovl, dims, synth.free_gauge_field(dims))
    for fl in (0, ovl.MIXED):
        y, info = _solve(ovl, ctx, ovl.ARNOLDI, 60, mu, b, flags=fl)
        assert info["status"] == 0 and info["k_used"] <= 4, info
        assert rel(y, ref) < 1e-10


@pytest.mark.parametrize("k", [1, 2, 7, 60, 300])
def test_arnoldi_delayed_cgs2_matches_classical(ovl, c4, k):
    """The double-float Arnoldi's default delayed Gram-Schmidt (two basis sweeps per step, the
    second pass of step j fused with the first of step j + 1) and the classical form (four sweeps,
    OVL_ARNOLDI_CGS2) build the same Arnoldi process (Sec. 2, Eq. 2.2-2.3): equal results to
    1e-12 from k = 1 on, and the oracle's Arnoldi (CGS2) result at small k; with 20 deflated
    eigenpairs as well."""
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    yd, infod = _solve(ovl, ctx, ovl.ARNOLDI, k, c4["mu"], c4["b"], flags=ovl.MIXED)
    yc, infoc = _solve(ovl, ctx, ovl.ARNOLDI, k, c4["mu"], c4["b"], flags=ovl.MIXED | ovl.ARNOLDI_CGS2)
    assert infod["status"] == 0 and infod["k_used"] == infoc["k_used"] == k
    assert rel(yd, yc) < 1e-12
    if k <= 60:
        assert rel(yd, K.sign_arnoldi(c4["A"].dot, c4["b"], k)) < 1e-10
    if k == 300:
        assert rel(yd, c4["ref"]) < 1e-10
        d = Dm.eigenpairs_dense(c4["A"].toarray(), 20)
        ctx.set_deflation(c4["mu"], KAPPA, d.lam, torch_c128(d.R.T.copy()), torch_c128(d.L.T.copy()))
        yd, _ = _solve(ovl, ctx, ovl.ARNOLDI, 300, c4["mu"], c4["b"], flags=ovl.MIXED)
        yc, _ = _solve(ovl, ctx, ovl.ARNOLDI, 300, c4["mu"], c4["b"], flags=ovl.MIXED | ovl.ARNOLDI_CGS2)
        assert rel(yd, yc) < 1e-12 and rel(yd, c4["ref"]) < 1e-10


@pytest.mark.parametrize("flags,tol", [("TWO_PASS", 1e-10), ("MIXED", 1e-8), ("MIXED|STEPWISE", 1e-8)])
def test_two_pass(ovl, c4, flags, tol):
    """Two-pass 2sL (Sec. 5): FP64 or FP32 pass 1 for the coefficients, FP64
    regeneration of the basis in pass 2 (persistent kernels, or one kernel per step)."""
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    fl = 0
    for f in flags.split("|"):
        fl |= getattr(ovl, f)
    y, info = _solve(ovl, ctx, ovl.LANCZOS2, 400, c4["mu"], c4["b"], flags=fl)
    assert info["status"] == 0
    assert rel(y, c4["ref"]) < tol


def test_inner_newton_equals_quadrature(ovl, c4):
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    y1, i1 = _solve(ovl, ctx, ovl.LANCZOS2, 250, c4["mu"], c4["b"])
    y2, i2 = _solve(ovl, ctx, ovl.LANCZOS2, 250, c4["mu"], c4["b"], flags=ovl.INNER_NEWTON)
    assert i1["inner_method"] == 0 and i2["inner_method"] == 1
    assert rel(y1, y2) < 1e-11


@pytest.mark.parametrize("method", ["arnoldi", "arnoldi_df"])
def test_arnoldi_quadrature_equals_newton(ovl, c4, method):
    """The inner sign of the Hessenberg H_k by the resolvent quadrature (Givens-rotation solves of the
    shifted systems) and by Roberts' iteration (Sec. 2) agree far below the 1e-10 target."""
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    m, fl = _method(ovl, method)
    for k in (1, 2, 40, 250):
        y1, i1 = _solve(ovl, ctx, m, k, c4["mu"], c4["b"], flags=fl)
        y2, i2 = _solve(ovl, ctx, m, k, c4["mu"], c4["b"], flags=fl | ovl.INNER_NEWTON)
        assert i1["inner_method"] == 0 and i2["inner_method"] == 1, (k, i1, i2)
        assert rel(y1, y2) < 1e-11, k


def test_host_buffers_and_no_graph(ovl, c4):
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    y1, _ = ctx.sign_krylov(ovl.LANCZOS2, 120, c4["mu"], KAPPA, np.ascontiguousarray(c4["b"]))
    y2, _ = _solve(ovl, ctx, ovl.LANCZOS2, 120, c4["mu"], c4["b"], flags=ovl.NO_GRAPH)
    assert isinstance(y1, np.ndarray)
    assert rel(y1, y2) < 1e-14


def test_repeat_is_deterministic(ovl, c4):
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    y1, _ = _solve(ovl, ctx, ovl.LANCZOS2, 150, c4["mu"], c4["b"], flags=ovl.MIXED)
    y2, _ = _solve(ovl, ctx, ovl.LANCZOS2, 150, c4["mu"], c4["b"], flags=ovl.MIXED)
    assert np.array_equal(y1, y2)
    # the persistent and the per-step kernels run the same FP32 recurrence (their
    # reductions add in different orders, so compare before rounding is amplified)
    y4, _ = _solve(ovl, ctx, ovl.LANCZOS2, 30, c4["mu"], c4["b"], flags=ovl.MIXED)
    y3, _ = _solve(ovl, ctx, ovl.LANCZOS2, 30, c4["mu"], c4["b"], flags=ovl.MIXED | ovl.STEPWISE)
    assert rel(y3, y4) < 1e-6


@pytest.mark.parametrize("gauge", [False, True])
def test_free_field_8x4_closed_form(ovl, gauge):
    """8^4, U = 1 or a random gauge transform of it: D_ov b from the momentum-
    space closed form (FFT), at a volume the dense oracle cannot reach."""
    dims, mu = (8, 8, 8, 8), 0.3
    V = 4096
    b = synth.gaussian_source(dims, 31)
    ref = F.overlap_free_apply(dims, mu, KAPPA, b)
    if gauge:
        g = synth.gauge_transformation(dims, 32)
        fwd, _, _, _ = W.neighbours(dims)
        U = np.einsum("vab,vndb->vnad", g, g[fwd].conj())
        b = np.einsum("vab,vsb->vsa", g, b.reshape(V, 4, 3)).reshape(-1)
        ref = np.einsum("vab,vsb->vsa", g, ref.reshape(V, 4, 3)).reshape(-1)
    else:
        U = synth.free_gauge_field(dims)
    ctx = _ctx(ovl, dims, U)
    for flags in (ovl.OVERLAP, ovl.OVERLAP | ovl.MIXED):
        y, info = _solve(ovl, ctx, ovl.LANCZOS2, 300, mu, b, flags=flags)
        assert rel(y, ref) < (1e-10 if not flags & ovl.MIXED else 1e-8)


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (3, 2, 5, 4)])
def test_small_ragged_lattices(ovl, dims):
    """Lattices smaller than one thread block and with odd spatial extents."""
    from oracle import sign as S
    U = synth.gauge_field(dims, 0.4, 41)
    A = W.a_operator(U, dims, 0.3, KAPPA)
    Ad = A.conj().T.tocsr()
    b = synth.gaussian_source(dims, 42)
    ctx = _ctx(ovl, dims, U)
    N = A.shape[0]
    for fl in (0, ovl.MIXED):  # FP64 and double-float Arnoldi
        if N <= 400:  # Krylov space exhausted: exact (Sec. 2, Eq. 2.1)
            ref = S.sign_spectral(A.toarray()) @ b
            y, _ = _solve(ovl, ctx, ovl.ARNOLDI, N, 0.3, b, flags=fl)
            assert rel(y, ref) < 1e-9
        k = 150
        y, _ = _solve(ovl, ctx, ovl.ARNOLDI, k, 0.3, b, flags=fl)
        assert rel(y, K.sign_arnoldi(A.dot, b, k)) < 1e-9
    k = 40
    yl, _ = _solve(ovl, ctx, ovl.LANCZOS2, k, 0.3, b)
    assert rel(yl, K.sign_lanczos2(A.dot, Ad.dot, b, k)) < 1e-8


@pytest.mark.parametrize("k", [5, 20, 60])
def test_mixed_pass1_matches_fp64(ovl, c4, k):
    """Before loss of bi-orthogonality the FP32 pass 1 runs the same process as the
    FP64 one (same start vectors in the FP32 device layout): the two-pass mixed
    result equals the FP64 result to FP32 rounding."""
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    y64, _ = _solve(ovl, ctx, ovl.LANCZOS2, k, c4["mu"], c4["b"])
    y32, _ = _solve(ovl, ctx, ovl.LANCZOS2, k, c4["mu"], c4["b"], flags=ovl.MIXED)
    assert rel(y32, y64) < 1e-5


def test_mixed_deflated_matches_dense(ovl, c4):
    lam, X, Xi = c4["lam"], c4["X"], c4["Xi"]
    idx = np.argsort(np.abs(lam.real))[:20]
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    ctx.set_deflation(c4["mu"], KAPPA, lam[idx], torch_c128(X[:, idx].T.copy()), torch_c128(Xi[idx, :].conj().copy()))
    y, info = _solve(ovl, ctx, ovl.LANCZOS2, 300, c4["mu"], c4["b"], flags=ovl.MIXED)
    assert info["status"] == 0
    assert rel(y, c4["ref"]) < 1e-8


def test_mixed_deflated_reprojection_option(ovl, c4):
    """Re-projection of the deflated directions in the FP32 pass (optional): the
    result stays within the FP32 bound of the projected operator."""
    lam, X, Xi = c4["lam"], c4["X"], c4["Xi"]
    idx = np.argsort(np.abs(lam.real))[:20]
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    ctx.set_deflation(c4["mu"], KAPPA, lam[idx], torch_c128(X[:, idx].T.copy()), torch_c128(Xi[idx, :].conj().copy()))
    y, info = _solve(ovl, ctx, ovl.LANCZOS2, 300, c4["mu"], c4["b"], flags=ovl.MIXED | ovl.REPROJ)
    assert rel(y, c4["ref"]) < 1e-6


def test_mixed_reprojection_period(ovl, c4):
    """Re-projection every p-th step (stepwise kernels): p = 1 is the every-step re-projection,
    bitwise; a period beyond k projects nothing, bitwise the stepwise solve without it; p = 5 stays
    within the same bound as p = 1."""
    lam, X, Xi = c4["lam"], c4["X"], c4["Xi"]
    idx = np.argsort(np.abs(lam.real))[:20]
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    ctx.set_deflation(c4["mu"], KAPPA, lam[idx], torch_c128(X[:, idx].T.copy()), torch_c128(Xi[idx, :].conj().copy()))
    mu, b = c4["mu"], c4["b"]
    st = ovl.MIXED | ovl.STEPWISE
    y1, _ = _solve(ovl, ctx, ovl.LANCZOS2, 120, mu, b, flags=st | ovl.REPROJ)
    y1p, _ = _solve(ovl, ctx, ovl.LANCZOS2, 120, mu, b, flags=st | ovl.REPROJ_PERIOD(1))
    assert np.array_equal(y1, y1p)
    y0, _ = _solve(ovl, ctx, ovl.LANCZOS2, 120, mu, b, flags=st)
    yinf, _ = _solve(ovl, ctx, ovl.LANCZOS2, 120, mu, b, flags=ovl.MIXED | ovl.REPROJ_PERIOD(127))
    assert np.array_equal(y0, yinf)
    assert not np.array_equal(y0, y1)
    y5, info = _solve(ovl, ctx, ovl.LANCZOS2, 300, mu, b, flags=ovl.MIXED | ovl.REPROJ_PERIOD(5))
    assert info["status"] == 0
    assert rel(y5, c4["ref"]) < 1e-6


def test_newton_fallback_on_hard_spectrum(ovl):
    """Ritz values close to the imaginary axis (2^3 x 4, eps = 1.0, min |Re lambda| ~ 0.03):
    whatever inner method finishes, the result matches the dense sign."""
    from oracle import sign as S
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 1.0, 31)
    A = W.a_operator(U, dims, 0.3, KAPPA)
    b = synth.gaussian_source(dims, 7)
    ref = S.sign_spectral(A.toarray()) @ b
    ctx = _ctx(ovl, dims, U)
    y, info = _solve(ovl, ctx, ovl.LANCZOS2, 300, 0.3, b)
    yn, infon = _solve(ovl, ctx, ovl.LANCZOS2, 300, 0.3, b, flags=ovl.INNER_NEWTON)
    assert rel(yn, y) < 1e-9
    assert rel(y, ref) < 1e-5
    for fl in (0, ovl.MIXED):  # Arnoldi: exhausted Krylov space (k = N = 384), exact up to rounding
        ya, _ = _solve(ovl, ctx, ovl.ARNOLDI, 384, 0.3, b, flags=fl)
        yan, _ = _solve(ovl, ctx, ovl.ARNOLDI, 384, 0.3, b, flags=fl | ovl.INNER_NEWTON)
        assert rel(ya, ref) < 1e-8 and rel(yan, ref) < 1e-8


@pytest.mark.parametrize("k", [60, 400])
def test_double_float_pass2_matches_fp64_pass2(ovl, c4, k):
    """The regeneration pass in double-float arithmetic (FP32 pairs) and in native FP64 follow the
    same pass-1 coefficients: their results agree far below the 1e-8 target."""
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    y_df, _ = _solve(ovl, ctx, ovl.LANCZOS2, k, c4["mu"], c4["b"], flags=ovl.MIXED | ovl.PASS2_DF)
    y_64, _ = _solve(ovl, ctx, ovl.LANCZOS2, k, c4["mu"], c4["b"], flags=ovl.MIXED)
    assert rel(y_df, y_64) < 1e-11
