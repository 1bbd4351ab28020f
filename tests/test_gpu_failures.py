"""The library's failure statuses on the GPU, produced without a fault: a bounded device wait
that runs out (the persistent pass 1's grid barrier made unreachable by the test-only
ovl_set_wait_limit, so every wait gives up after a few polls) returns OVL_ETIMEOUT and leaves the
context usable; a rank-deficient set of left eigenvectors gives OVL_ESINGULAR (L^dag R singular,
Sec. 3, Eq. 3.1); a solve at another mu than the installed deflation gives OVL_EINVAL; and a
gradient whose upstream vector is orthogonal to the source (g^dag b = 0: the two-sided process
cannot start, Sec. 4) gives OVL_EBREAKDOWN."""
import numpy as np
import pytest

from gpu_common import KAPPA, config4, rel, torch_c128
from oracle import deflation as Dm
from paper_0810_4228_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ovl():
    from paper_0810_4228_gb300 import ovl as O
    O.load()
    return O


def _ctx(ovl, c4):
    ctx = ovl.Context(c4["dims"])
    ctx.set_gauge(torch_c128(c4["U"]))
    return ctx


def test_timeout_then_usable(ovl):
    c4 = config4()
    ctx = _ctx(ovl, c4)
    b = torch_c128(c4["b"])
    ctx.set_wait_limit(1000, unreachable=True)
    with pytest.raises(ovl.OvlError) as e:
        ctx.sign_krylov(ovl.LANCZOS2, 200, c4["mu"], KAPPA, b, flags=ovl.MIXED)
    assert e.value.code == ovl.ETIMEOUT
    # the same context, default limits: the persistent solve runs to the dense result
    ctx.set_wait_limit(0)
    y, info = ctx.sign_krylov(ovl.LANCZOS2, 400, c4["mu"], KAPPA, b, flags=ovl.MIXED)
    assert info["status"] == 0 and rel(y.cpu().numpy(), c4["ref"]) < 1e-8
    # and once more captured in a graph (the default path)
    y2, _ = ctx.sign_krylov(ovl.LANCZOS2, 400, c4["mu"], KAPPA, b, flags=ovl.MIXED)
    assert rel(y2.cpu().numpy(), c4["ref"]) < 1e-8


def test_singular_left_vectors(ovl):
    c4 = config4()
    ctx = _ctx(ovl, c4)
    d = Dm.eigenpairs_dense(c4["A"].toarray(), 4)
    R = np.ascontiguousarray(d.R.T)
    L = np.ascontiguousarray(d.L.T).copy()
    L[1] = L[0]  # two equal left vectors: L^dag R has two equal rows
    with pytest.raises(ovl.OvlError) as e:
        ctx.set_deflation(c4["mu"], KAPPA, d.lam, torch_c128(R), torch_c128(L))
    assert e.value.code == ovl.ESINGULAR
    # a valid set afterwards is accepted and used
    ctx.set_deflation(c4["mu"], KAPPA, d.lam, torch_c128(R), torch_c128(np.ascontiguousarray(d.L.T)))
    y, info = ctx.sign_krylov(ovl.LANCZOS2, 400, c4["mu"], KAPPA, torch_c128(c4["b"]))
    assert info["status"] == 0 and rel(y.cpu().numpy(), c4["ref"]) < 1e-10


def test_mu_mismatch_with_deflation(ovl):
    c4 = config4()
    ctx = _ctx(ovl, c4)
    d = Dm.eigenpairs_dense(c4["A"].toarray(), 4)
    ctx.set_deflation(c4["mu"], KAPPA, d.lam, torch_c128(np.ascontiguousarray(d.R.T)),
                      torch_c128(np.ascontiguousarray(d.L.T)))
    for mu, kappa in ((c4["mu"] + 0.1, KAPPA), (c4["mu"], KAPPA + 0.01)):
        with pytest.raises(ovl.OvlError) as e:
            ctx.sign_krylov(ovl.LANCZOS2, 50, mu, kappa, torch_c128(c4["b"]))
        assert e.value.code == ovl.EINVAL


def test_gradient_breakdown_orthogonal_upstream(ovl):
    c4 = config4()
    ctx = _ctx(ovl, c4)
    b = c4["b"]
    x = synth.gaussian_source(c4["dims"], 77)
    g = x - (np.vdot(b, x) / np.vdot(b, b)) * b  # g^dag b = 0
    assert abs(np.vdot(g, b)) < 1e-10 * np.linalg.norm(g) * np.linalg.norm(b)
    with pytest.raises(ovl.OvlError) as e:
        ctx.sign_grad(100, c4["mu"], KAPPA, torch_c128(b), torch_c128(g))
    assert e.value.code == ovl.EBREAKDOWN
