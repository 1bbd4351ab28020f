"""CPU checks of the stored full-size oracle references (tests/golden/oracle_refs.npz, written by
tests/golden/make_oracle_refs.py from oracle/ only) and of the comparison the GPU tests make with
them: every case is present with its workload, the oracle's eigenpairs have small residuals, its
deflated Arnoldi result is self-converged (k_lo against k_hi), the stored projections are those of
the seeded vectors, and the comparison recovers a planted error of known size."""
import numpy as np
import pytest

from gpu_common import assert_oracle_close, oracle_distance, oracle_refs
from paper_0810_4228_gb300 import synth

CASES = {"gauss8_mu0.1": ((8, 8, 8, 8), 1001, 0.1), "gauss8_mu0.3": ((8, 8, 8, 8), 1001, 0.3),
         "gauss8_mu0.5": ((8, 8, 8, 8), 1001, 0.5)}
CASES.update({f"batch6_r{r}": ((6, 6, 6, 6), 1003, 0.2) for r in (0, 5, 11)})
CASES.update({f"batch8_r{r}": ((8, 8, 8, 8), 1004, 0.2) for r in (0, 5, 11)})


def test_every_case_present_and_converged():
    refs = oracle_refs()
    for name, (dims, seed, mu) in CASES.items():
        r = refs[name]
        assert tuple(r["dims"]) == dims and int(r["seed"]) == seed and float(r["mu"]) == mu, name
        assert int(r["m"]) == 20 and str(r["method"]) == "arnoldi"
        assert float(r["eig_residual"]) < 1e-12, name
        assert float(r["selfdiff"]) < 1e-11, (name, float(r["selfdiff"]))
        N = 12 * int(np.prod(dims))
        assert len(r["idx"]) == 4096 and r["idx"].max() < N and np.all(np.diff(r["idx"]) > 0)
        # the sampled values are a part of a vector of the stored norm
        assert np.sum(np.abs(r["val"]) ** 2) <= float(r["norm"]) ** 2 * (1 + 1e-12), name
        if str(r["source_kind"]) == "gauss":
            # spread over the lattice (a point source's result is concentrated near its site):
            # the mean square agrees within the sampling spread
            ms = np.mean(np.abs(r["val"]) ** 2) * N
            assert 0.5 < ms / float(r["norm"]) ** 2 < 2.0, name


def test_projections_bounded_by_cauchy_schwarz():
    refs = oracle_refs()
    for name, (dims, _, _) in CASES.items():
        r = refs[name]
        for j, p in enumerate(r["proj"]):
            g = synth.gaussian_source(dims, 9000 + j)
            assert abs(p) <= np.linalg.norm(g) * float(r["norm"]) * (1 + 1e-12)


@pytest.mark.parametrize("eps", [1e-9, 1e-6])
def test_comparison_recovers_a_planted_error(eps):
    """A vector y and a reference built from it the way the script stores one; y perturbed by a
    random relative error eps reads as about eps on the samples and through the projections."""
    dims = (4, 4, 4, 4)
    N = 12 * 256
    rng = np.random.default_rng(3)
    y = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    idx = np.sort(rng.choice(N, 1024, replace=False))
    G = np.stack([synth.gaussian_source(dims, 9000 + j) for j in range(8)])
    ref = {"dims": np.array(dims), "idx": idx, "val": y[idx], "norm": np.linalg.norm(y), "proj": G.conj() @ y}
    assert max(oracle_distance(y, ref)) == 0.0
    e = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    yp = y + eps * np.linalg.norm(y) * e / np.linalg.norm(e)
    rs, mx, rp = oracle_distance(yp, ref)
    assert 0.7 * eps < rs < 1.4 * eps and mx < 10 * eps and 0.3 * eps < rp < 3 * eps, (rs, mx, rp)
    assert_oracle_close(yp, ref, 3 * eps)
    with pytest.raises(AssertionError):
        assert_oracle_close(yp, ref, 0.3 * eps)
