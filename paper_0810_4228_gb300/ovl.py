"""Python binding of the C ABI in include/ovl.h (argument marshalling only).

Every computation runs in libovl.so's CUDA kernels; this module passes
torch device pointers, sizes and the current CUDA stream.  It raises if the
library is missing: there is no CPU fallback.

Names follow the C functions: ``Context.apply_Dw``, ``Context.apply_pair``,
``Context.set_deflation``, ``Context.sign_krylov``.  Tensors are complex128
in the canonical layout [V, 4, 3] (spinors) and [V, 4, 3, 3] (links) unless a
``native=True`` argument says otherwise; see include/ovl.h for the layout and
the physics conventions.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libovl.so")

OK, EINVAL, ENOMEM, ECUDA, EBREAKDOWN, ESINGULAR, ENOCONV, ETIMEOUT, ESTATE = range(9)
ARNOLDI, LANCZOS2 = 0, 1
GAMMA5, DAGGER, NATIVE, HOST, F32, F32_FULL = 0x1, 0x2, 0x4, 0x8, 0x10, 0x20
OVERLAP, MIXED, TWO_PASS, INNER_NEWTON, NO_GRAPH, PROFILE = 0x100, 0x200, 0x400, 0x1000, 0x2000, 0x4000
STENCIL_SITE, STENCIL_SPLIT, REPROJ, STEPWISE, PASS2_F64, PASS2_DF = 0x10000, 0x20000, 0x8000, 0x40000, 0x80000, 0x100000
NO_TUNE, ARNOLDI_CGS2 = 0x200000, 0x400000


def REPROJ_PERIOD(p: int) -> int:
    """REPROJ applied every p-th step of the FP32 pass (1 <= p <= 127; p = 1 is REPROJ)."""
    if not 1 <= int(p) <= 127:
        raise ValueError("re-projection period must be within 1..127")
    return REPROJ | ((int(p) & 0x7F) << 24)

_ERRNAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", EBREAKDOWN: "EBREAKDOWN",
             ESINGULAR: "ESINGULAR", ENOCONV: "ENOCONV", ETIMEOUT: "ETIMEOUT", ESTATE: "ESTATE"}

EXPORTS = ["ovl_create", "ovl_destroy", "ovl_last_error", "ovl_set_stream", "ovl_vector_bytes",
           "ovl_set_gauge", "ovl_apply_Dw", "ovl_apply_pair", "ovl_apply_pair_noalloc",
           "ovl_apply_pair_noalloc_blocks", "ovl_pack", "ovl_unpack",
           "ovl_set_deflation", "ovl_get_deflation", "ovl_deflation_eigs", "ovl_sign_krylov",
           "ovl_profile_get", "ovl_profile_reset", "ovl_dw_grad", "ovl_sign_grad", "ovl_batch_create",
           "ovl_batch_destroy", "ovl_batch_last_error", "ovl_batch_solve", "ovl_batch_profile", "ovl_batch_tuning",
           "ovl_batch_set_tuning",
           "ovl_sign_krylov_batched", "ovl_overlap_eigs", "ovl_sign_arnoldi_restarted",
           "ovl_set_wait_limit"]


class OvlError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class KStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int), ("kernels", ctypes.c_longlong),
                ("ms", ctypes.c_double)]


class EigInfo(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("iterations", ctypes.c_int), ("matvecs", ctypes.c_longlong),
                ("max_residual", ctypes.c_double), ("lambda_cut", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class OvInfo(ctypes.Structure):
    _fields_ = [("nconv", ctypes.c_int), ("restarts", ctypes.c_int), ("sign_solves", ctypes.c_longlong),
                ("ritz_residual", ctypes.c_double), ("max_residual", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [("k_used", ctypes.c_int), ("breakdown_step", ctypes.c_int),
                ("inner_iters", ctypes.c_int), ("inner_method", ctypes.c_int),
                ("bperp_norm", ctypes.c_double), ("inner_err", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libovl.so (once).  Raises ImportError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_0810_4228_gb300.build`")
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "ovl_create": (I, [ctypes.POINTER(P), ctypes.POINTER(I), I, P]),
        "ovl_destroy": (I, [P]),
        "ovl_last_error": (ctypes.c_char_p, [P]),
        "ovl_set_stream": (I, [P, P]),
        "ovl_vector_bytes": (ctypes.c_size_t, [P, I]),
        "ovl_set_gauge": (I, [P, P, I]),
        "ovl_apply_Dw": (I, [P, D, D, P, P, I]),
        "ovl_apply_pair": (I, [P, D, D, I, P, P, P, P, ctypes.POINTER(D)]),
        "ovl_apply_pair_noalloc": (I, [P, D, D, I, P, P, P, P, P]),
        "ovl_apply_pair_noalloc_blocks": (I, [ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "ovl_pack": (I, [P, P, P, I]),
        "ovl_unpack": (I, [P, P, P, I]),
        "ovl_set_deflation": (I, [P, D, D, I, ctypes.POINTER(D), P, P, I]),
        "ovl_sign_krylov": (I, [P, I, I, D, D, P, P, I, ctypes.POINTER(Info)]),
        "ovl_profile_get": (I, [P, ctypes.POINTER(KStat), I, ctypes.POINTER(I)]),
        "ovl_get_deflation": (I, [P, ctypes.POINTER(I), ctypes.POINTER(D), P, P, I]),
        "ovl_deflation_eigs": (I, [P, D, D, I, I, D, I, I, ctypes.POINTER(EigInfo)]),
        "ovl_dw_grad": (I, [P, D, D, P, P, P, ctypes.POINTER(D), I]),
        "ovl_sign_grad": (I, [P, I, D, D, P, P, P, P, ctypes.POINTER(D), P, I, ctypes.POINTER(Info)]),
        "ovl_profile_reset": (I, [P]),
        "ovl_batch_create": (I, [ctypes.POINTER(P), ctypes.POINTER(P), I, ctypes.POINTER(I)]),
        "ovl_batch_destroy": (I, [P]),
        "ovl_batch_last_error": (ctypes.c_char_p, [P]),
        "ovl_batch_solve": (I, [P, I, D, D, ctypes.POINTER(P), ctypes.POINTER(P), I, ctypes.POINTER(Info)]),
        "ovl_batch_profile": (I, [P, ctypes.POINTER(D), ctypes.POINTER(I), I]),
        "ovl_batch_tuning": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "ovl_batch_set_tuning": (I, [P, I, I, I]),
        "ovl_set_wait_limit": (I, [P, ctypes.c_longlong, I]),
        "ovl_sign_arnoldi_restarted": (I, [P, I, I, D, D, P, P, I, ctypes.POINTER(Info)]),
        "ovl_overlap_eigs": (I, [P, I, I, D, D, I, I, I, D, I, ctypes.POINTER(D), P, ctypes.POINTER(OvInfo)]),
        "ovl_sign_krylov_batched": (I, [ctypes.POINTER(P), I, ctypes.POINTER(I), I, D, D, ctypes.POINTER(P),
                                        ctypes.POINTER(P), I, ctypes.POINTER(Info)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def noalloc_pair_blocks(dims):
    """(fits, blocks, max_blocks): the thread blocks ovl_apply_pair_noalloc's kernel launches on
    a lattice of extents dims and the most its static scratch holds (host only, no GPU call)."""
    lib = load()
    arr = (ctypes.c_int * 4)(*[int(d) for d in dims])
    nb, mx = ctypes.c_int(), ctypes.c_int()
    r = lib.ovl_apply_pair_noalloc_blocks(arr, ctypes.byref(nb), ctypes.byref(mx))
    return r == OK, nb.value, mx.value


def _ptr(t) -> int:
    import torch
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if not t.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return t.ctypes.data
    raise TypeError(type(t))


def _is_host(t) -> bool:
    import torch
    return isinstance(t, np.ndarray) or (isinstance(t, torch.Tensor) and not t.is_cuda)


def _stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


@dataclass
class Lattice:
    dims: tuple
    bc_t: int = -1

    @property
    def volume(self) -> int:
        L = self.dims
        return L[0] * L[1] * L[2] * L[3]


class Context:
    """One lattice (and gauge field) on the current CUDA device."""

    def __init__(self, dims, bc_t: int = -1, stream=None):
        self._lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.bc_t = int(bc_t)
        self.V = int(np.prod(self.dims))
        self.n = 12 * self.V
        h = ctypes.c_void_p()
        arr = (ctypes.c_int * 4)(*self.dims)
        self._stream = stream
        r = self._lib.ovl_create(ctypes.byref(h), arr, self.bc_t, _stream_handle(stream))
        if r:
            raise OvlError(r, f"ovl_create failed for dims={self.dims}, bc_t={bc_t}")
        self._h = h

    # -- helpers
    def _check(self, r):
        if r:
            raise OvlError(r, self._lib.ovl_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ovl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        self._check(self._lib.ovl_set_stream(self._h, _stream_handle(stream)))

    def vector_bytes(self, prec: int = 0) -> int:
        return int(self._lib.ovl_vector_bytes(self._h, prec))

    def empty_native(self, prec: int = 0):
        import torch
        return torch.empty(self.n, dtype=torch.complex128 if prec == 0 else torch.complex64, device="cuda")

    # -- C ABI
    def set_gauge(self, U):
        flags = HOST if _is_host(U) else 0
        self._check(self._lib.ovl_set_gauge(self._h, _ptr(U), flags))

    def pack(self, canon, native, prec: int = 0):
        self._check(self._lib.ovl_pack(self._h, _ptr(canon), _ptr(native), prec))

    def unpack(self, native, canon, prec: int = 0):
        self._check(self._lib.ovl_unpack(self._h, _ptr(native), _ptr(canon), prec))

    def apply_Dw(self, mu: float, kappa: float, x, y=None, flags: int = GAMMA5):
        """y = D_w(mu) x, gamma5 D_w(mu) x (GAMMA5, default) or A^dag x (DAGGER)."""
        import torch
        if y is None:
            if _is_host(x):
                y = np.empty_like(x) if isinstance(x, np.ndarray) else torch.empty_like(x)
            else:
                y = torch.empty_like(x)
        if _is_host(x):
            flags |= HOST
        self._check(self._lib.ovl_apply_Dw(self._h, mu, kappa, _ptr(x), _ptr(y), flags))
        return y

    def apply_pair(self, mu: float, kappa: float, v, w, t, s, prec: int = 0):
        """t = A v, s = A^dag w on device-layout vectors; returns alpha = w^dag t."""
        a = (ctypes.c_double * 2)()
        self._check(self._lib.ovl_apply_pair(self._h, mu, kappa, prec, _ptr(v), _ptr(w), _ptr(t), _ptr(s), a))
        return complex(a[0], a[1])

    def apply_pair_noalloc(self, mu: float, kappa: float, v, w, t, s, alpha_dev, prec: int = 0):
        """As apply_pair, without any device allocation: alpha = w^dag t is written to the
        device tensor alpha_dev (2 float64) and nothing is synchronised."""
        self._check(self._lib.ovl_apply_pair_noalloc(self._h, mu, kappa, prec, _ptr(v), _ptr(w), _ptr(t), _ptr(s),
                                                      _ptr(alpha_dev)))

    def dw_grad(self, mu: float, kappa: float, x, g, grad_U=None, flags: int = 0):
        """(grad_U, grad_mu) of a real l(y), y = A x, from g = dl/dy*; canonical device tensors.
        flags: 0 (FP64) or F32 (the link force in FP32)."""
        gm = ctypes.c_double()
        self._check(self._lib.ovl_dw_grad(self._h, mu, kappa, _ptr(x), _ptr(g),
                                          _ptr(grad_U) if grad_U is not None else None, ctypes.byref(gm), flags))
        return grad_U, gm.value

    def sign_grad(self, k: int, mu: float, kappa: float, b, g, y=None, grad_U=None, grad_b=None, flags: int = 0):
        """Derivatives of Re <g, sgn(A) b> with respect to mu, U and b (k-step two-sided Lanczos from
        (b, g), no deflation; FP64, or FP32 with flags=MIXED); canonical device tensors.  Returns
        (grad_mu, info); y, grad_U, grad_b are written when given."""
        gm = ctypes.c_double()
        info = Info()
        r = self._lib.ovl_sign_grad(self._h, int(k), mu, kappa, _ptr(b), _ptr(g),
                                    _ptr(y) if y is not None else None,
                                    _ptr(grad_U) if grad_U is not None else None, ctypes.byref(gm),
                                    _ptr(grad_b) if grad_b is not None else None, int(flags), ctypes.byref(info))
        self._check(r)
        return gm.value, info.as_dict()

    def set_deflation(self, mu: float, kappa: float, lam, R, L):
        """Install m critical eigenpairs: lam (m,) complex, R and L (m, 12V) complex128."""
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.complex128))
        m = int(lam.shape[0])
        if m == 0:
            self._check(self._lib.ovl_set_deflation(self._h, mu, kappa, 0, None, None, None, 0))
            return
        lam_d = np.ascontiguousarray(np.stack([lam.real, lam.imag], axis=1).ravel())
        flags = HOST if _is_host(R) else 0
        self._keep = (R, L)
        self._check(self._lib.ovl_set_deflation(
            self._h, mu, kappa, m, lam_d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            _ptr(R), _ptr(L), flags))

    def deflation_eigs(self, mu: float, kappa: float, m: int, nextra: int = 10, tol: float = 1e-10,
                       nkrylov: int = 0, maxit: int = 400):
        """Compute and install the m critical eigenpairs on the GPU (thick-restart Arnoldi on A^2,
        basis of nkrylov vectors, 0 = automatic, at most maxit restart cycles); returns info dict."""
        info = EigInfo()
        r = self._lib.ovl_deflation_eigs(self._h, mu, kappa, m, nextra, tol, nkrylov, maxit, ctypes.byref(info))
        if r == ENOCONV:
            raise OvlError(r, f"{self._lib.ovl_last_error(self._h).decode()} {info.as_dict()}")
        self._check(r)
        return info.as_dict()

    def get_deflation(self, device: bool = True):
        """(lam, R, L) of the installed deflation; R, L canonical (m, 12V) complex128."""
        import torch
        m = ctypes.c_int()
        self._check(self._lib.ovl_get_deflation(self._h, ctypes.byref(m), None, None, None, 0))
        m = m.value
        lam = np.empty(2 * max(m, 1))
        if device:
            R = torch.empty((m, self.n), dtype=torch.complex128, device="cuda")
            L = torch.empty_like(R)
            flags = 0
        else:
            R = np.empty((m, self.n), dtype=np.complex128)
            L = np.empty_like(R)
            flags = HOST
        self._check(self._lib.ovl_get_deflation(self._h, None, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                _ptr(R) if m else None, _ptr(L) if m else None, flags))
        return lam[0:2 * m:2] + 1j * lam[1:2 * m:2], R, L

    def set_wait_limit(self, polls: int = 0, unreachable: bool = False):
        """Bounded device waits of the persistent pass 1 give up after `polls` polls (0: default);
        unreachable=True makes every such wait run out (tests of the OVL_ETIMEOUT path)."""
        self._check(self._lib.ovl_set_wait_limit(self._h, int(polls), 1 if unreachable else 0))

    def sign_arnoldi_restarted(self, m: int, cycles: int, mu: float, kappa: float, b, out=None, flags: int = 0):
        """out = sgn(A) b (D_ov b with OVERLAP) by Arnoldi restarted every m steps, at most `cycles`
        cycles (a basis of m + 1 double-float vectors).  Returns (out, info dict)."""
        import torch
        if out is None:
            out = (np.empty_like(b) if isinstance(b, np.ndarray) else torch.empty_like(b))
        if _is_host(b):
            flags |= HOST
        info = Info()
        r = self._lib.ovl_sign_arnoldi_restarted(self._h, int(m), int(cycles), mu, kappa, _ptr(b), _ptr(out),
                                                 int(flags), ctypes.byref(info))
        self._check(r)
        d = info.as_dict()
        d["status"] = r
        return out, d

    def overlap_eigs(self, method: int, k: int, mu: float, kappa: float, nev: int, flags: int = 0,
                     nkrylov: int = 0, tol: float = 1e-10, maxit: int = 200, vecs=None):
        """The nev eigenvalues of D_ov(mu) nearest 0 (thick-restart Arnoldi, D_ov applied by sign solves
        of `method` with Krylov size k); returns (eigenvalues as a complex numpy array, nearest 0 first,
        info dict).  vecs: optional device tensor (nev, 12V) complex128 receiving the eigenvectors."""
        lam = (ctypes.c_double * (2 * nev))()
        info = OvInfo()
        r = self._lib.ovl_overlap_eigs(self._h, int(method), int(k), mu, kappa, int(flags), int(nev), int(nkrylov),
                                       float(tol), int(maxit), lam, _ptr(vecs) if vecs is not None else None,
                                       ctypes.byref(info))
        if r:
            raise OvlError(r, f"{self._lib.ovl_last_error(self._h).decode()} {info.as_dict()}")
        return np.array(lam[0::2]) + 1j * np.array(lam[1::2]), info.as_dict()

    def profile(self, reset: bool = True):
        """Per-kernel-class totals of the OVL_PROFILE solves since the last reset."""
        arr = (KStat * 32)()
        cnt = ctypes.c_int()
        self._check(self._lib.ovl_profile_get(self._h, arr, 32, ctypes.byref(cnt)))
        out = {arr[i].name.decode(): {"launches": arr[i].launches, "kernels": int(arr[i].kernels),
                                      "ms": arr[i].ms} for i in range(min(cnt.value, 32))}
        if reset:
            self._check(self._lib.ovl_profile_reset(self._h))
        return out

    def sign_krylov(self, method: int, k: int, mu: float, kappa: float, b, out=None, flags: int = 0):
        """out = sgn(gamma5 D_w(mu)) b, or D_ov(mu) b with flags |= OVERLAP, by ARNOLDI or LANCZOS2.
        flags |= MIXED: two-sided Lanczos in two passes (FP32 pass 1, FP64-accurate regeneration;
        on lattices above the persistent kernels' limit run as a batch of one with double-float
        regeneration); Arnoldi with its basis and Gram-Schmidt sweeps in double-float arithmetic.
        REPROJ_PERIOD(p): re-projection of the deflated directions every p-th FP32 step.
        Returns (out, info dict).  b may be a CUDA tensor or host memory."""
        import torch
        if out is None:
            out = (np.empty_like(b) if isinstance(b, np.ndarray) else torch.empty_like(b))
        if _is_host(b) != _is_host(out):
            raise ValueError("b and out must both be host or both be device memory")
        if _is_host(b):
            flags |= HOST
        info = Info()
        r = self._lib.ovl_sign_krylov(self._h, method, int(k), mu, kappa, _ptr(b), _ptr(out), flags,
                                      ctypes.byref(info))
        if r and r != EBREAKDOWN:
            self._check(r)
        d = info.as_dict()
        d["status"] = r
        return out, d


class Batch:
    """Batched two-sided Lanczos solves over several contexts (lattices) and right-hand sides:
    ``nrhs[j]`` sources for ``contexts[j]``, solved together (one captured graph)."""

    def __init__(self, contexts, nrhs):
        self._lib = load()
        self.contexts = list(contexts)
        self.nrhs = [int(r) for r in nrhs]
        h = ctypes.c_void_p()
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        nr = (ctypes.c_int * len(self.nrhs))(*self.nrhs)
        r = self._lib.ovl_batch_create(ctypes.byref(h), arr, len(self.contexts), nr)
        if r:
            raise OvlError(r, "ovl_batch_create failed")
        self._h = h

    @property
    def nseq(self) -> int:
        return sum(self.nrhs)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.ovl_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, k: int, mu: float, kappa: float, sources, outs=None, flags: int = 0):
        """sources[j]: (nrhs[j], 12 V_j) complex128 (CUDA tensors or host arrays); returns
        (outs, infos, status) with one info dict per sequence in (context, rhs) order."""
        import torch
        if outs is None:
            outs = [np.empty_like(b) if isinstance(b, np.ndarray) else torch.empty_like(b) for b in sources]
        if any(_is_host(b) for b in sources):
            flags |= HOST
        bp = (ctypes.c_void_p * len(sources))(*[_ptr(b) for b in sources])
        op = (ctypes.c_void_p * len(outs))(*[_ptr(o) for o in outs])
        infos = (Info * self.nseq)()
        r = self._lib.ovl_batch_solve(self._h, int(k), mu, kappa, bp, op, flags, infos)
        if r and r != EBREAKDOWN:
            raise OvlError(r, self._lib.ovl_batch_last_error(self._h).decode())
        return outs, [i.as_dict() for i in infos], r

    def profile(self, reset: bool = True):
        """Per-phase totals of the OVL_PROFILE solves: {'pass1', 'inner_sign', 'pass2_or_combine'} in ms,
        and the number of solves."""
        ms = (ctypes.c_double * 3)()
        n = ctypes.c_int()
        self._lib.ovl_batch_profile(self._h, ms, ctypes.byref(n), 1 if reset else 0)
        return {"pass1": ms[0], "inner_sign": ms[1], "pass2_or_combine": ms[2]}, n.value

    def tuning(self):
        """(pass-1 sites per block, regeneration blocks per SM, sequences per regeneration block) chosen
        by the autotuner, or None."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        r = self._lib.ovl_batch_tuning(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return (a.value, b.value, c.value) if r == 0 else None

    def set_tuning(self, pass1_block_sites: int, regen_blocks_per_sm: int, regen_seqs_per_block: int = 1):
        """Pin the launch shapes (64/128/256 sites per pass-1 block, 2..6 regeneration blocks per SM,
        1/2 sequences per regeneration block); the autotuner is then skipped."""
        r = self._lib.ovl_batch_set_tuning(self._h, int(pass1_block_sites), int(regen_blocks_per_sm),
                                           int(regen_seqs_per_block))
        if r:
            raise OvlError(r, self._lib.ovl_batch_last_error(self._h).decode())
