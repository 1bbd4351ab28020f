"""Batched two-sided Lanczos solves (several right-hand sides on several lattices
of different sizes in one graph-captured launch sequence) against the dense
oracle, against the single-sequence solve, and on the edge cases of a batch."""
import numpy as np
import pytest

from gpu_common import KAPPA, config4, rel, torch_c128
from oracle import sign as S
from oracle import wilson as W
from paper_0810_4228_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ovl():
    from paper_0810_4228_gb300 import ovl as O
    O.load()
    return O


@pytest.fixture(scope="module")
def mid():
    """A lattice of 192 sites (one full and one partial block) with its dense sign."""
    dims, mu = (4, 4, 2, 6), 0.3
    U = synth.gauge_field(dims, 0.5, 3050)
    A = W.a_operator(U, dims, mu, KAPPA).toarray()
    return dict(dims=dims, U=U, mu=mu, sgn=S.sign_spectral(A))


@pytest.fixture(scope="module")
def small():
    """A ragged lattice smaller than one block (V = 72) with its dense sign."""
    dims, mu = (2, 3, 2, 6), 0.3
    U = synth.gauge_field(dims, 0.5, 3000)
    A = W.a_operator(U, dims, mu, KAPPA).toarray()
    return dict(dims=dims, U=U, mu=mu, sgn=S.sign_spectral(A))


def _ctx(O, dims, U):
    c = O.Context(dims)
    c.set_gauge(torch_c128(U))
    return c


def _sources(dims, seed, nrhs):
    return synth.gaussian_source(dims, seed, nrhs=nrhs)


@pytest.mark.parametrize("mode", ["fp64", "fp64_two_pass", "mixed"])
def test_batch_matches_dense(ovl, mid, mode):
    """Two lattices (4^4 and 4^2 x 2 x 6), 3 + 2 sources, every result against the dense oracle."""
    c4 = config4()
    assert c4["mu"] == mid["mu"]
    ca, cb = _ctx(ovl, c4["dims"], c4["U"]), _ctx(ovl, mid["dims"], mid["U"])
    ba = _sources(c4["dims"], 3100, 3)
    bb = _sources(mid["dims"], 3101, 2)
    bt = ovl.Batch([ca, cb], [3, 2])
    flags = {"fp64": 0, "fp64_two_pass": ovl.TWO_PASS, "mixed": ovl.MIXED}[mode]
    outs, infos, st = bt.solve(500, c4["mu"], KAPPA, [torch_c128(ba), torch_c128(bb)], flags=flags)
    assert st == 0 and len(infos) == 5
    tol = 1e-8 if mode == "mixed" else 1e-10
    ya, yb = outs[0].cpu().numpy(), outs[1].cpu().numpy()
    sgn4 = c4["X"] @ (S.csign(c4["lam"])[:, None] * c4["Xi"])
    for r in range(3):
        assert rel(ya[r], sgn4 @ ba[r]) < tol
    for r in range(2):
        assert rel(yb[r], mid["sgn"] @ bb[r]) < tol
    bt.close()


def test_batch_equals_single_solves(ovl, small):
    """Each sequence of an FP64 batch equals the single-sequence FP64 solve of the same source
    (both converged; the kernels differ, so rounding differs)."""
    c4 = config4()
    ca = _ctx(ovl, c4["dims"], c4["U"])
    ba = _sources(c4["dims"], 3200, 2)
    bt = ovl.Batch([ca], [2])
    outs, _, _ = bt.solve(300, c4["mu"], KAPPA, [torch_c128(ba)])
    for r in range(2):
        y1, _ = ca.sign_krylov(ovl.LANCZOS2, 300, c4["mu"], KAPPA, torch_c128(ba[r]))
        assert rel(outs[0][r].cpu().numpy(), y1.cpu().numpy()) < 1e-11
    bt.close()


@pytest.mark.parametrize("k", [3, 25])
def test_batch_same_process_small_k(ovl, small, k):
    """Before loss of bi-orthogonality the batched FP64 process and the oracle's two-sided
    Lanczos agree to rounding."""
    from oracle import krylov as K
    dims = small["dims"]
    U = small["U"]
    A = W.a_operator(U, dims, small["mu"], KAPPA)
    Ad = A.conj().T.tocsr()
    b = _sources(dims, 3300, 1)
    c = _ctx(ovl, dims, U)
    bt = ovl.Batch([c], [1])
    outs, infos, _ = bt.solve(k, small["mu"], KAPPA, [torch_c128(b)])
    assert infos[0]["k_used"] == k
    assert rel(outs[0][0].cpu().numpy(), K.sign_lanczos2(A.dot, Ad.dot, b[0], k)) < 1e-11
    bt.close()


def test_batch_deflated_overlap_host(ovl):
    """Deflation installed on the context, D_ov output, host buffers, mixed precision."""
    c4 = config4()
    lam, X, Xi = c4["lam"], c4["X"], c4["Xi"]
    idx = np.argsort(np.abs(lam.real))[:20]
    ca = _ctx(ovl, c4["dims"], c4["U"])
    ca.set_deflation(c4["mu"], KAPPA, lam[idx], torch_c128(X[:, idx].T.copy()), torch_c128(Xi[idx, :].conj().copy()))
    ba = _sources(c4["dims"], 3400, 2)
    bt = ovl.Batch([ca], [2])
    outs, infos, st = bt.solve(300, c4["mu"], KAPPA, [np.ascontiguousarray(ba)], flags=ovl.MIXED | ovl.OVERLAP)
    assert st == 0
    sgn4 = X @ (S.csign(lam)[:, None] * Xi)
    g5 = np.tile(np.array([1, 1, 1, 1, 1, 1, -1, -1, -1, -1, -1, -1.0]), c4["A"].shape[0] // 12)
    for r in range(2):
        ref = ba[r] + g5 * (sgn4 @ ba[r])
        assert rel(outs[0][r], ref) < 1e-8
    bt.close()


def test_batch_graph_replay_and_recapture(ovl, small):
    """Replaying the captured graph gives identical results; a new k captures a new graph."""
    dims, U = small["dims"], small["U"]
    c = _ctx(ovl, dims, U)
    b = torch_c128(_sources(dims, 3500, 3))
    bt = ovl.Batch([c], [3])
    y1 = bt.solve(60, small["mu"], KAPPA, [b])[0][0].clone()
    y2 = bt.solve(60, small["mu"], KAPPA, [b])[0][0].clone()
    y3 = bt.solve(80, small["mu"], KAPPA, [b])[0][0].clone()
    y4 = bt.solve(60, small["mu"], KAPPA, [b], flags=ovl.NO_GRAPH)[0][0].clone()
    y5 = bt.solve(80, small["mu"], KAPPA, [b], flags=ovl.NO_GRAPH)[0][0].clone()
    assert bool((y1 == y2).all()) and bool((y1 == y4).all()) and bool((y3 == y5).all())
    assert not bool((y1 == y3).all())
    bt.close()


def _oracle_2sl(small, b, k):
    from oracle import krylov as K
    A = W.a_operator(small["U"], small["dims"], small["mu"], KAPPA)
    return K.sign_lanczos2(A.dot, A.conj().T.tocsr().dot, b, k)


def test_batch_zero_source_among_others(ovl, small):
    dims, U = small["dims"], small["U"]
    c = _ctx(ovl, dims, U)
    b = _sources(dims, 3600, 3)
    b[1] = 0
    bt = ovl.Batch([c], [3])
    outs, infos, st = bt.solve(25, small["mu"], KAPPA, [torch_c128(b)])
    y = outs[0].cpu().numpy()
    assert st == 0 and infos[1]["k_used"] == 0
    assert not np.any(y[1])
    for q in (0, 2):
        assert rel(y[q], _oracle_2sl(small, b[q], 25)) < 1e-11
    bt.close()


def test_one_shot_batched_call(ovl, small):
    import ctypes
    dims, U = small["dims"], small["U"]
    c = _ctx(ovl, dims, U)
    b = torch_c128(_sources(dims, 3700, 2))
    out = torch_c128(np.zeros((2, 12 * 72)))
    lib = ovl.load()
    ctxs = (ctypes.c_void_p * 1)(c._h.value)
    nr = (ctypes.c_int * 1)(2)
    bp = (ctypes.c_void_p * 1)(b.data_ptr())
    op = (ctypes.c_void_p * 1)(out.data_ptr())
    r = lib.ovl_sign_krylov_batched(ctxs, 1, nr, 25, small["mu"], KAPPA, bp, op, 0, None)
    assert r == 0
    y = out.cpu().numpy()
    bh = b.cpu().numpy()
    for q in range(2):
        assert rel(y[q], _oracle_2sl(small, bh[q], 25)) < 1e-11


def test_batch_uneven_lattices_point_sources(ovl):
    """12 point sources on each of three lattices of different sizes (6^4, 4^3 x 6, 2^2 x 4 x 6),
    mixed precision at k = 700, against single FP64 solves of the same sources at k = 1000 (point
    sources need a larger k than Gaussian ones)."""
    mu = 0.2
    dims_list = [(6, 6, 6, 6), (4, 4, 4, 6), (2, 2, 4, 6)]
    ctxs, srcs = [], []
    for j, d in enumerate(dims_list):
        ctxs.append(_ctx(ovl, d, synth.gauge_field(d, 1.0, 3800 + j)))
        srcs.append(synth.point_sources(d, site=0))
    bt = ovl.Batch(ctxs, [12] * 3)
    outs, infos, st = bt.solve(700, mu, KAPPA, [torch_c128(s) for s in srcs], flags=ovl.MIXED)
    assert st == 0 and len(infos) == 36
    for j in range(3):
        for r in (0, 5, 11):
            y1, _ = ctxs[j].sign_krylov(ovl.LANCZOS2, 1000, mu, KAPPA, torch_c128(srcs[j][r]))
            e = rel(outs[j][r].cpu().numpy(), y1.cpu().numpy())
            assert e < 1e-8, (j, r, e)
    bt.close()


def test_batch_double_float_pass2_matches_fp64_pass2(ovl, mid):
    c = _ctx(ovl, mid["dims"], mid["U"])
    b = torch_c128(_sources(mid["dims"], 3900, 3))
    bt = ovl.Batch([c], [3])
    y_df = bt.solve(300, mid["mu"], KAPPA, [b], flags=ovl.MIXED)[0][0].cpu().numpy()
    y_64 = bt.solve(300, mid["mu"], KAPPA, [b], flags=ovl.MIXED | ovl.PASS2_F64)[0][0].cpu().numpy()
    for r in range(3):
        assert rel(y_df[r], y_64[r]) < 1e-11
    bt.close()


def test_batch_autotuner_picks_shapes(ovl, small):
    """The first solve times the launch-shape candidates and keeps one; OVL_NO_TUNE keeps the defaults."""
    c = _ctx(ovl, small["dims"], small["U"])
    b = torch_c128(_sources(small["dims"], 4000, 2))
    bt = ovl.Batch([c], [2])
    assert bt.tuning() is None
    y1 = bt.solve(25, small["mu"], KAPPA, [b])[0][0].cpu().numpy()
    sites, minb, seqs = bt.tuning()
    assert sites in (64, 128, 256) and minb in (2, 3, 4, 5, 6) and seqs in (1, 2)
    bt2 = ovl.Batch([c], [2])
    y2 = bt2.solve(25, small["mu"], KAPPA, [b], flags=ovl.NO_TUNE)[0][0].cpu().numpy()
    assert bt2.tuning() is None
    for r in range(2):
        assert rel(y1[r], y2[r]) < 1e-12
        assert rel(y1[r], _oracle_2sl(small, b.cpu().numpy()[r], 25)) < 1e-11
    bt.close()
    bt2.close()


@pytest.mark.parametrize("sites,minb,seqs", [(64, 2, 1), (128, 3, 1), (256, 4, 1), (64, 5, 1), (256, 6, 1),
                                             (128, 2, 2), (128, 3, 2), (64, 4, 2)])
def test_batch_every_pinned_shape(ovl, small, mid, sites, minb, seqs):
    """Each pinned launch shape: FP64 two-pass at k = 25 against the oracle's two-sided Lanczos on
    a lattice smaller than one block, and mixed precision on two lattices against the dense sign."""
    dims, U = small["dims"], small["U"]
    c = _ctx(ovl, dims, U)
    b = _sources(dims, 4100, 3)
    bt = ovl.Batch([c], [3])
    bt.set_tuning(sites, minb, seqs)
    assert bt.tuning() == (sites, minb, seqs)
    y = bt.solve(25, small["mu"], KAPPA, [torch_c128(b)], flags=ovl.TWO_PASS)[0][0].cpu().numpy()
    for r in range(3):
        assert rel(y[r], _oracle_2sl(small, b[r], 25)) < 1e-11, r
    bt.close()
    c4 = config4()
    ca, cb = _ctx(ovl, c4["dims"], c4["U"]), _ctx(ovl, mid["dims"], mid["U"])
    ba, bb = _sources(c4["dims"], 4101, 2), _sources(mid["dims"], 4102, 2)
    bt = ovl.Batch([ca, cb], [2, 3])
    bt.set_tuning(sites, minb, seqs)
    bb = _sources(mid["dims"], 4102, 3)
    outs, _, st = bt.solve(500, c4["mu"], KAPPA, [torch_c128(ba), torch_c128(bb)], flags=ovl.MIXED)
    assert st == 0 and bt.tuning() == (sites, minb, seqs)
    sgn4 = c4["X"] @ (S.csign(c4["lam"])[:, None] * c4["Xi"])
    for r in range(2):
        assert rel(outs[0][r].cpu().numpy(), sgn4 @ ba[r]) < 1e-8
    for r in range(3):  # an odd count: the last sequence has no partner in the two-sequence blocks
        assert rel(outs[1][r].cpu().numpy(), mid["sgn"] @ bb[r]) < 1e-8
    bt.close()


def test_batch_two_sequence_regeneration_equals_one(ovl, mid):
    """Two sequences per regeneration block do each sequence's arithmetic as one per block."""
    c = _ctx(ovl, mid["dims"], mid["U"])
    b = torch_c128(_sources(mid["dims"], 4300, 5))
    bt = ovl.Batch([c], [5])
    bt.set_tuning(128, 2, 1)
    y1 = bt.solve(300, mid["mu"], KAPPA, [b], flags=ovl.MIXED)[0][0].cpu().numpy()
    bt.set_tuning(128, 2, 2)
    y2 = bt.solve(300, mid["mu"], KAPPA, [b], flags=ovl.MIXED)[0][0].cpu().numpy()
    assert np.array_equal(y1, y2)
    bt.close()


def test_batch_rejects_unknown_shape(ovl, small):
    c = _ctx(ovl, small["dims"], small["U"])
    bt = ovl.Batch([c], [1])
    with pytest.raises(ovl.OvlError):
        bt.set_tuning(96, 3)
    with pytest.raises(ovl.OvlError):
        bt.set_tuning(128, 7)
    with pytest.raises(ovl.OvlError):
        bt.set_tuning(128, 3, 3)
    assert bt.tuning() is None
    bt.close()


def test_batch_persistent_pass1_equals_stepwise(ovl, mid):
    """The persistent pass 1 (one cooperative launch) and the stepwise kernels with the same block
    shape (128 sites) do the same arithmetic in the same order: equal results."""
    c4 = config4()
    ca, cb = _ctx(ovl, c4["dims"], c4["U"]), _ctx(ovl, mid["dims"], mid["U"])
    ba, bb = _sources(c4["dims"], 4200, 2), _sources(mid["dims"], 4201, 3)
    srcs = [torch_c128(ba), torch_c128(bb)]
    bt = ovl.Batch([ca, cb], [2, 3])
    bt.set_tuning(128, 3)
    yp = [o.cpu().numpy() for o in bt.solve(400, c4["mu"], KAPPA, srcs, flags=ovl.MIXED)[0]]
    ys = [o.cpu().numpy() for o in bt.solve(400, c4["mu"], KAPPA, srcs, flags=ovl.MIXED | ovl.STEPWISE)[0]]
    for a, b in zip(yp, ys):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
    sgn4 = c4["X"] @ (S.csign(c4["lam"])[:, None] * c4["Xi"])
    for r in range(2):
        assert rel(yp[0][r], sgn4 @ ba[r]) < 1e-8
    bt.close()


def test_batch_tuning_cache(ovl, small, tmp_path, monkeypatch):
    """A second batch of the same shape takes the first one's tuned launch shapes from the cache
    (no timing) and gives bitwise the same result; with OVL_TUNE_CACHE set the choice is also
    appended to that file for later processes."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("OVL_TUNE_CACHE", str(path))
    c = _ctx(ovl, small["dims"], small["U"])
    b = torch_c128(_sources(small["dims"], 4400, 4))  # a batch shape no other test tunes
    bt = ovl.Batch([c], [4])
    bt.solve(40, small["mu"], KAPPA, [b], flags=ovl.MIXED)
    first = bt.tuning()
    assert first is not None
    lines = path.read_text().splitlines()
    assert any(ln.split()[1:] == [str({64: 0, 128: 1, 256: 2}[first[0]]), str(first[1]), str(first[2] - 1)]
               for ln in lines), (lines, first)
    bt2 = ovl.Batch([c], [4])
    y2 = bt2.solve(40, small["mu"], KAPPA, [b], flags=ovl.MIXED)[0][0].cpu().numpy()
    assert bt2.tuning() == first
    y1 = bt.solve(40, small["mu"], KAPPA, [b], flags=ovl.MIXED)[0][0].cpu().numpy()
    assert np.array_equal(y1, y2)
    bt.close()
    bt2.close()


@pytest.fixture(scope="module")
def big(ovl):
    """16^3 x 12 (49152 sites): more tiles than the persistent passes hold on chip on 152 SMs
    (at most 8 tiles of 32 sites per block), so single-source mixed solves take the batched
    kernels as a batch of one."""
    dims, mu = (16, 16, 16, 12), 0.2
    U = synth.gauge_field(dims, 1.0, 3300)
    return dict(dims=dims, mu=mu, U=U, b=synth.gaussian_source(dims, 3301))


def test_single_source_mixed_routed_through_batch_of_one(ovl, big):
    """A mixed two-sided Lanczos solve of one source on a lattice above the persistent limit runs the
    batched kernels (double-float regeneration): bitwise the result of a user batch of one, and at
    small k the same process as the stepwise mixed path and the FP64 solve (Sec. 5)."""
    ctx = _ctx(ovl, big["dims"], big["U"])
    b = torch_c128(big["b"])
    mu = big["mu"]
    y_r, i_r = ctx.sign_krylov(ovl.LANCZOS2, 30, mu, KAPPA, b, flags=ovl.MIXED)
    assert i_r["status"] == 0 and i_r["k_used"] == 30
    bt = ovl.Batch([ctx], [1])
    y_b = bt.solve(30, mu, KAPPA, [b.reshape(1, -1)], flags=ovl.MIXED)[0][0].cpu().numpy()[0]
    bt.close()
    y_r = y_r.cpu().numpy()
    assert np.array_equal(y_r, y_b)
    y_s, _ = ctx.sign_krylov(ovl.LANCZOS2, 30, mu, KAPPA, b, flags=ovl.MIXED | ovl.STEPWISE)
    y_64, _ = ctx.sign_krylov(ovl.LANCZOS2, 30, mu, KAPPA, b)
    assert rel(y_r, y_s.cpu().numpy()) < 1e-6
    assert rel(y_r, y_64.cpu().numpy()) < 1e-5


def test_single_source_mixed_routed_deflated_converged(ovl, big):
    """With 20 deflated critical pairs the routed mixed solve reaches the FP64 two-pass result of the
    same k to 1e-8 (the accuracy target of Sec. 5); D_ov b with host buffers equals b + gamma5 y; a
    changed deflation set (m = 20 -> 8) is taken up by the next solve."""
    ctx = _ctx(ovl, big["dims"], big["U"])
    mu, k = big["mu"], 600
    e = ctx.deflation_eigs(mu, KAPPA, 20)
    assert e["m"] == 20
    b = torch_c128(big["b"])
    y_r, i_r = ctx.sign_krylov(ovl.LANCZOS2, k, mu, KAPPA, b, flags=ovl.MIXED)
    y_64, i_64 = ctx.sign_krylov(ovl.LANCZOS2, k, mu, KAPPA, b, flags=ovl.TWO_PASS)
    assert i_r["status"] == 0 and i_64["status"] == 0
    # |b_perp^R| after the oblique split (Eq. 4.5): the same in both paths, not |b|
    assert abs(i_r["bperp_norm"] - i_64["bperp_norm"]) < 1e-6 * i_64["bperp_norm"]
    assert abs(i_r["bperp_norm"] - np.linalg.norm(big["b"])) > 1e-6 * i_64["bperp_norm"]
    y_r, y_64 = y_r.cpu().numpy(), y_64.cpu().numpy()
    assert rel(y_r, y_64) < 1e-8
    bh = np.ascontiguousarray(big["b"])
    yo, _ = ctx.sign_krylov(ovl.LANCZOS2, k, mu, KAPPA, bh, flags=ovl.MIXED | ovl.OVERLAP)
    g5 = np.tile(np.repeat([1.0, 1, -1, -1], 3), synth.volume(big["dims"]))
    assert isinstance(yo, np.ndarray)
    assert rel(yo, bh + g5 * y_r) < 1e-14
    lam, R, L = ctx.get_deflation()
    ctx.set_deflation(mu, KAPPA, lam[:8], R[:8].contiguous(), L[:8].contiguous())
    y8, _ = ctx.sign_krylov(ovl.LANCZOS2, 40, mu, KAPPA, b, flags=ovl.MIXED)
    y8s, _ = ctx.sign_krylov(ovl.LANCZOS2, 40, mu, KAPPA, b, flags=ovl.MIXED | ovl.STEPWISE)
    assert rel(y8.cpu().numpy(), y8s.cpu().numpy()) < 1e-6


def test_user_batch_recaptures_on_deflation_change(ovl):
    """A batch's captured graph holds each context's deflation size: after set_deflation changes
    it (m = 8 -> 4) the next solve re-captures and equals a fresh batch's solve."""
    c4 = config4()
    ctx = _ctx(ovl, c4["dims"], c4["U"])
    lam, X, Xi = c4["lam"], c4["X"], c4["Xi"]
    idx = np.argsort(np.abs(lam.real))[:8]
    R, L = X[:, idx].T.copy(), Xi[idx, :].conj().copy()
    ctx.set_deflation(c4["mu"], KAPPA, lam[idx], torch_c128(R), torch_c128(L))
    b = torch_c128(_sources(c4["dims"], 4500, 1))
    bt = ovl.Batch([ctx], [1])
    y8 = bt.solve(30, c4["mu"], KAPPA, [b], flags=ovl.MIXED)[0][0].cpu().numpy()
    ctx.set_deflation(c4["mu"], KAPPA, lam[idx[:4]], torch_c128(R[:4]), torch_c128(L[:4]))
    y4 = bt.solve(30, c4["mu"], KAPPA, [b], flags=ovl.MIXED)[0][0].cpu().numpy()
    bt2 = ovl.Batch([ctx], [1])
    y4f = bt2.solve(30, c4["mu"], KAPPA, [b], flags=ovl.MIXED)[0][0].cpu().numpy()
    assert np.array_equal(y4, y4f)
    assert rel(y4, y8) > 1e-6  # the deflation size changes the k = 30 result
    bt.close()
    bt2.close()
