"""Pins of the oracle to statements the paper prints (fixtures under tests/golden/, each with its
citation).  The paper gives no worked numerical example; what it does state about the methods'
behaviour is checked here against the oracle's Arnoldi (Sec. 2) and two-sided Lanczos (Sec. 4)."""
import os

import numpy as np

from oracle import krylov as K
from oracle import sign as S
from oracle import wilson as W
from paper_0810_4228_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _fixture(name):
    vals = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                key, *rest = line.split()
                vals[key] = [float(x) for x in rest]
    return vals


def _k_needed(solve, ref, eps, ks):
    for k in ks:
        if np.linalg.norm(solve(k) - ref) <= eps * np.linalg.norm(ref):
            return k
    return None


def test_lanczos2_needs_about_20_percent_larger_subspace():
    """Sec. 5: two-sided Lanczos needs a Krylov subspace about 20 % larger than Arnoldi for the
    same accuracy, with and without deflation."""
    g = _fixture("krylov_size_ratio.txt")
    eps = g["eps"][0]
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.5, 1000)
    A = W.a_operator(U, dims, 0.3, 0.2)
    Ad = A.conj().T.tocsr()
    b = synth.gaussian_source(dims, 2000)
    # one eigendecomposition serves the exact result (Eq. 1.3) and the deflation sets (Eq. 3.1)
    lam, X = np.linalg.eig(A.toarray())
    Xi = np.linalg.inv(X)
    ref = X @ (S.csign(lam) * (Xi @ b))
    order = np.argsort(np.abs(lam.real), kind="stable")
    for m in g["deflation_sizes"]:
        m = int(m)
        idx = order[:m]
        defl = K.Deflation(lam=lam[idx].copy(), R=X[:, idx].copy(), L=Xi[idx, :].conj().T.copy()) if m else None
        ks = range(160, 400, 10)
        ka = _k_needed(lambda k: K.sign_arnoldi(A.dot, b, k, defl), ref, eps, ks)
        kl = _k_needed(lambda k: K.sign_lanczos2(A.dot, Ad.dot, b, k, defl), ref, eps, ks)
        assert ka is not None and kl is not None, (m, ka, kl)
        assert g["ratio_min"][0] <= kl / ka <= g["ratio_max"][0], (m, ka, kl)
