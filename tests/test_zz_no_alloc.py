"""The allocation-free pair entry point (for callers that must not call
cudaMalloc when they call it, e.g. while capturing a CUDA graph): through the
C ABI, two calls in a row must give what ovl_apply_pair gives, within the
tolerances the stencil tests use.  Kept in a file of its own, collected last."""
import numpy as np
import pytest

from gpu_common import KAPPA, torch_c128
from paper_0810_4228_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ovl():
    from paper_0810_4228_gb300 import ovl as O
    O.load()
    return O


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (24, 24, 24, 24)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-14), (1, 1e-6)])
def test_noalloc_pair_matches_pair(ovl, dims, prec, tol):
    import torch
    mu = 0.3
    U = synth.gauge_field(dims, 1.0, 51)
    v = synth.gaussian_source(dims, 52)
    w = synth.gaussian_source(dims, 53)
    ctx = ovl.Context(dims)
    ctx.set_gauge(torch_c128(U))
    nv, nw = ctx.empty_native(prec), ctx.empty_native(prec)
    ctx.pack(torch_c128(v), nv, prec)
    ctx.pack(torch_c128(w), nw, prec)
    t0, s0 = ctx.empty_native(prec), ctx.empty_native(prec)
    a0 = ctx.apply_pair(mu, KAPPA, nv, nw, t0, s0, prec)
    for _ in range(2):  # two calls in a row share the static scratch
        t1, s1 = ctx.empty_native(prec), ctx.empty_native(prec)
        alpha = torch.zeros(2, dtype=torch.float64, device="cuda")
        ctx.apply_pair_noalloc(mu, KAPPA, nv, nw, t1, s1, alpha, prec)
        torch.cuda.synchronize()
        a1 = complex(alpha[0].item(), alpha[1].item())
        scale = t0.abs().max().item()
        assert (t1 - t0).abs().max().item() <= tol * scale
        assert (s1 - s0).abs().max().item() <= tol * s0.abs().max().item()
        assert abs(a1 - a0) <= tol * abs(a0)


# (48, 48, 48, 64) = 7077888 and (64, 64, 32, 40) = 5242880 sites lie between the true limit
# (4194304: 32768 blocks of 64 sites per parity) and twice it; (64, 64, 64, 80) far above
@pytest.mark.parametrize("dims", [(48, 48, 48, 64), (64, 64, 32, 40), (32, 32, 32, 130), (64, 64, 64, 80)])
def test_noalloc_rejects_oversized_lattice(ovl, dims):
    """Rejected with OVL_EINVAL before any launch (creating the context allocates nothing, and the
    undersized buffers are never touched)."""
    import torch
    ctx = ovl.Context(dims)
    x = torch.zeros(2, dtype=torch.complex128, device="cuda")
    a = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(ovl.OvlError) as e:
        ctx.apply_pair_noalloc(0.3, KAPPA, x, x, x, x, a, 1)
    assert e.value.code == ovl.EINVAL
    assert "too large" in str(e.value)


def test_noalloc_accepts_the_largest_lattice_without_launching(ovl):
    """At exactly the limit (32^3 x 128 = 4194304 sites) the size check passes: with null
    buffers the call then stops at the null-argument check, before any launch."""
    ctx = ovl.Context((32, 32, 32, 128))
    with pytest.raises(ovl.OvlError) as e:
        ctx._check(ctx._lib.ovl_apply_pair_noalloc(ctx._h, 0.3, KAPPA, 1, None, None, None, None, None))
    assert e.value.code == ovl.EINVAL
    assert "null argument" in str(e.value)
