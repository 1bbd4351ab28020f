"""Host-only check of the size rule of the allocation-free pair entry point: the thread blocks
its kernel launches, from the same function the launcher uses, against the static scratch's
32768 partial-sum slots.  No GPU call."""
import pytest


@pytest.fixture(scope="module")
def ovl():
    from paper_0810_4228_gb300 import build
    build.build()
    from paper_0810_4228_gb300 import ovl as O
    O.load()
    return O


@pytest.mark.parametrize("dims,blocks,fits", [
    ((32, 32, 32, 128), 32768, True),      # 4194304 sites: one block per 64 sites of each parity
    ((32, 32, 32, 130), 33280, False),     # just above the limit
    ((64, 64, 32, 40), 40960, False),      # between the limit and twice it
    ((48, 48, 48, 64), 55296, False),
    ((24, 24, 24, 24), 2592, True),
    ((16, 16, 16, 8), 1024, True),         # below 155648 sites: one block per 32 sites
    ((4, 4, 4, 4), 8, True),
])
def test_pair_block_count(ovl, dims, blocks, fits):
    ok, nb, mx = ovl.noalloc_pair_blocks(dims)
    assert mx == 32768
    assert nb == blocks
    assert ok == fits


def test_pair_block_count_rejects_invalid_lattice(ovl):
    for dims in ((4, 4, 4, 3), (1, 4, 4, 4)):
        ok, nb, _ = ovl.noalloc_pair_blocks(dims)
        assert not ok and nb == 0
