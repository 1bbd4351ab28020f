"""Writes tests/golden/oracle_refs.npz: the FP64 oracle's sgn(A) b on the full-size workloads
that the dense oracle cannot reach, for the GPU parity tests and the benchmark's accuracy gate.

Only ``oracle/`` computes here; the inputs come from the seeded generators of
``paper_0810_4228_gb300.synth``.  For each case the oracle builds A = gamma5 D_w(mu) (Sec. 1,
Eq. 1.2), finds its own critical eigenpairs with ARPACK in shift-invert mode (Sec. 3 and Sec. 5:
the m eigenvalues of smallest |Re lambda| and their left/right eigenvectors), and runs the deflated
Arnoldi approximation (Sec. 3, Eq. 3.4) at two Krylov sizes; the difference of the two is stored
as the oracle's own error estimate.  Arnoldi rather than two-sided Lanczos: both converge to the
same sgn(A) b, but the oracle's two-sided Lanczos at k of about 1000 carries a rounding floor near
1e-10 (loss of bi-orthogonality amplifies rounding), while Arnoldi with Gram-Schmidt applied twice
keeps its basis orthonormal and reaches 1e-12.

Stored per case (a vector of N = 12 V complex entries is too large to keep whole):
  * ``idx``: 4096 sampled component indices (seeded), ``val``: sgn(A) b at those indices;
  * ``norm``: |sgn(A) b|_2;
  * ``proj``: g_j^dag sgn(A) b for the eight seeded Gaussian vectors g_j =
    synth.gaussian_source(dims, 9000 + j), a check on the whole vector;
  * ``selfdiff``: |y(k_hi) - y(k_lo)| / |y(k_hi)|, and the eigenpairs' largest residual.

Workloads (fields U = exp(i eps H), seeds as named; kappa = 0.2, antiperiodic time):
  * ``gauss8_mu{0.1,0.3,0.5}``: 8^4, eps = 1.0, U seed 1001, Gaussian b seed 2001, m = 20;
  * ``batch{6,8}_r{0,5,11}``: 6^4 (U seed 1003) and 8^4 (U seed 1004), eps = 1.0, mu = 0.2,
    the point sources of spin-colour index r at site 0, m = 20 (two of the four lattices of the
    batched workload; the oracle's LU-based eigensolver does not reach 12^4 and 16^3 x 8).

Usage: ``python tests/golden/make_oracle_refs.py [--jobs J] [--cache DIR]`` (about an hour on 8
cores; ``--cache`` keeps each field's eigenpairs in DIR and reuses them on a later run).
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "oracle_refs.npz")

KAPPA, EPS, M = 0.2, 1.0, 20
K_LO, K_HI = 800, 1000  # default Krylov sizes (a group may set its own "k")
NSAMPLE, NPROJ, PROJ_SEED = 4096, 8, 9000

# one field + chemical potential + sources per group (groups of the same field share the
# eigenpairs through --cache once the first has computed them)
GROUPS = [
    {"dims": (8, 8, 8, 8), "seed": 1001, "mu": 0.1, "sources": [("gauss8_mu0.1", "gauss", 2001)]},
    {"dims": (8, 8, 8, 8), "seed": 1001, "mu": 0.3, "sources": [("gauss8_mu0.3", "gauss", 2001)]},
    # mu = 0.5 converges more slowly: 3e-9 between k = 800 and 1000
    {"dims": (8, 8, 8, 8), "seed": 1001, "mu": 0.5, "sources": [("gauss8_mu0.5", "gauss", 2001)], "k": (1300, 1600)},
] + [{"dims": (6, 6, 6, 6), "seed": 1003, "mu": 0.2, "sources": [(f"batch6_r{r}", "point", r)]} for r in (0, 5, 11)] \
  + [{"dims": (8, 8, 8, 8), "seed": 1004, "mu": 0.2, "sources": [(f"batch8_r{r}", "point", r)]} for r in (0, 5, 11)]


def _run_group(args):
    gr, cache = args
    sys.path.insert(0, ROOT)
    from oracle import deflation as D
    from oracle import krylov as K
    from oracle import wilson as W
    from paper_0810_4228_gb300 import synth

    dims, mu = gr["dims"], gr["mu"]
    t0 = time.time()
    U = synth.gauge_field(dims, EPS, gr["seed"])
    A = W.a_operator(U, dims, mu, KAPPA)
    Ah = A.conj().T.tocsr()
    cfile = (os.path.join(cache, f"defl_{'x'.join(map(str, dims))}_s{gr['seed']}_mu{mu}_m{M}.npz")
             if cache else None)
    if cfile and os.path.exists(cfile):
        z = np.load(cfile)
        defl = K.Deflation(lam=z["lam"], R=z["R"], L=z["L"])
    else:
        defl = D.eigenpairs_arpack(A, M)
        if cfile:
            np.savez(cfile, lam=defl.lam, R=defl.R, L=defl.L)
    res = max(np.linalg.norm(A @ defl.R - defl.R * defl.lam, axis=0).max(),
              np.linalg.norm(Ah @ defl.L - defl.L * np.conj(defl.lam), axis=0).max())
    t_eig = time.time() - t0
    N = A.shape[0]
    idx = np.sort(np.random.default_rng(7).choice(N, NSAMPLE, replace=False)).astype(np.int64)
    G = np.stack([synth.gaussian_source(dims, PROJ_SEED + j) for j in range(NPROJ)])
    out = {}
    k_lo, k_hi = gr.get("k", (K_LO, K_HI))
    for name, kind, arg in gr["sources"]:
        b = synth.gaussian_source(dims, arg) if kind == "gauss" else synth.point_sources(dims, site=0)[arg]
        y_hi, inf = K.sign_arnoldi(A.dot, b, k_hi, defl=defl, return_info=True)
        # the k_lo approximation from the same process: its first k_lo steps are the k_lo-step run
        nb = np.linalg.norm(b - defl.R @ (defl.L.conj().T @ b))
        y_lo = (y_hi - inf["V"] @ inf["c"]
                + nb * (inf["V"][:, :k_lo] @ K.inner_sign_e1(inf["H"][:k_lo, :k_lo])))
        del inf
        nrm = np.linalg.norm(y_hi)
        out[name] = {
            "dims": np.array(dims), "seed": gr["seed"], "eps": EPS, "mu": mu, "kappa": KAPPA, "m": defl.m,
            "source_kind": kind, "source_arg": arg, "k_lo": k_lo, "k_hi": k_hi, "method": "arnoldi",
            "idx": idx, "val": y_hi[idx], "norm": nrm, "proj": G.conj() @ y_hi,
            "selfdiff": np.linalg.norm(y_hi - y_lo) / nrm, "eig_residual": res,
            "lam": defl.lam,
        }
        print(f"{name}: m={defl.m} eig {t_eig:.0f}s residual {res:.1e} selfdiff "
              f"{out[name]['selfdiff']:.2e} total {time.time() - t0:.0f}s", flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=3)
    ap.add_argument("--cache", default="", help="directory for the fields' eigenpairs (reused when present)")
    ap.add_argument("--only", default="", help="comma-separated cases to recompute; the others are kept from the file")
    args = ap.parse_args()
    if args.cache:
        os.makedirs(args.cache, exist_ok=True)
    threads = max(1, (os.cpu_count() or 1) // args.jobs)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = str(threads)
    ctx = mp.get_context("spawn")
    only = set(x for x in args.only.split(",") if x)
    groups = [g for g in GROUPS if not only or any(src[0] in only for src in g["sources"])]
    with ctx.Pool(args.jobs) as pool:
        parts = pool.map(_run_group, [(g, args.cache) for g in groups], chunksize=1)
    flat = {}
    if only and os.path.exists(OUT):  # keep the cases not recomputed
        z = np.load(OUT)
        flat = {key: z[key] for key in z.files if key.split("/", 1)[0] not in only}
    for part in parts:
        for name, d in part.items():
            for key, v in d.items():
                flat[f"{name}/{key}"] = v
    np.savez_compressed(OUT, **flat)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
