"""Shared helpers of the GPU parity tests: seeded inputs (from the input
generator module) and cached oracle references."""
import functools

import numpy as np

from paper_0810_4228_gb300 import synth

KAPPA = 0.2  # m_w = -1.5


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@functools.lru_cache(maxsize=4)
def config4(eps=0.5, seed=1000, mu=0.3):
    """4^4, U = exp(i eps H), mu, kappa = 0.2, Gaussian b: the small workload
    the oracle diagonalises densely (N = 3072)."""
    from oracle import sign as S
    from oracle import wilson as W
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, eps, seed)
    A = W.a_operator(U, dims, mu, KAPPA)
    Ad = A.toarray()
    lam, X = np.linalg.eig(Ad)
    Xi = np.linalg.inv(X)
    sg = S.csign(lam)
    b = synth.gaussian_source(dims, 2000)
    ref = X @ (sg * (Xi @ b))
    return dict(dims=dims, U=U, A=A, mu=mu, b=b, ref=ref, lam=lam, X=X, Xi=Xi)


def torch_c128(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


REFS_PATH = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.abspath(__file__)),
                                       "golden", "oracle_refs.npz")


@functools.lru_cache(maxsize=1)
def oracle_refs():
    """The FP64 oracle's sgn(A) b on the full-size workloads, as written by
    tests/golden/make_oracle_refs.py: {case: {field: array}}."""
    z = np.load(REFS_PATH)
    out = {}
    for key in z.files:
        case, field = key.split("/", 1)
        out.setdefault(case, {})[field] = z[key]
    return out


@functools.lru_cache(maxsize=4)
def _proj_vectors(dims, n):
    return np.stack([synth.gaussian_source(dims, 9000 + j) for j in range(n)])


def oracle_distance(y, ref):
    """(relative 2-norm over the sampled components, largest sampled difference relative to the
    largest sampled magnitude, relative error estimated from the stored projections
    g_j^dag sgn(A) b) of a full vector y against the oracle's stored sgn(A) b.  The g_j have
    i.i.d. N(0, 1) real and imaginary parts, so E|g^dag e|^2 = 2 |e|^2."""
    y = np.asarray(y).ravel()
    G = _proj_vectors(tuple(int(d) for d in ref["dims"]), len(ref["proj"]))
    d = y[ref["idx"]] - ref["val"]
    pe = G.conj() @ y - ref["proj"]
    return (float(np.linalg.norm(d) / np.linalg.norm(ref["val"])),
            float(np.abs(d).max() / np.abs(ref["val"]).max()),
            float(np.sqrt(np.mean(np.abs(pe) ** 2) / 2.0) / float(ref["norm"])))


def assert_oracle_close(y, ref, tol, what=""):
    """Element by element on the sampled components and on the whole vector through the
    projections (which estimate the relative 2-norm error to within a factor of about two with
    eight projections; the bound below allows three)."""
    rel_s, max_s, rel_p = oracle_distance(y, ref)
    assert rel_s <= tol and max_s <= tol and rel_p <= 3 * tol, (what, rel_s, max_s, rel_p)
    return rel_s, max_s, rel_p


def gamma5_diag(V):
    """Chiral gamma5 = diag(1, 1, -1, -1) in spin, on the flattened index 12 s + 3 spin + colour."""
    return np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)
