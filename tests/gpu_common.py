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
