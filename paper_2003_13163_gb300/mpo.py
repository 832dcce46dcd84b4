"""Python binding of the C ABI in include/mpo.h (argument marshalling only).

Every step of the simulation runs in the CUDA library; this module converts
arrays and handles. There is no CPU fallback: if the library is missing or no
GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MPO_FP64, MPO_FP32, MPO_MIXED_FP32 = 0, 1, 2
PRECISIONS = {"fp64": MPO_FP64, "fp32": MPO_FP32, "mixed": MPO_MIXED_FP32}
MPO_S_ALL_BONDS, MPO_S_CENTRE = 0, 1
ERRORS = {0: "MPO_OK", -1: "MPO_ERR_ARG", -2: "MPO_ERR_CUDA", -3: "MPO_ERR_OOM", -4: "MPO_ERR_NOCONV",
          -5: "MPO_ERR_TIMEOUT", -6: "MPO_ERR_STATE"}
EXPORTS = ["mpo_default_opts", "mpo_init", "mpo_apply_layer", "mpo_apply_gate", "mpo_apply_superop", "mpo_sweep",
           "mpo_entropy", "mpo_schmidt", "mpo_bond_dims", "mpo_get_site", "mpo_to_dense", "mpo_centre",
           "mpo_device_bytes", "mpo_free", "mpo_last_error", "mpo_eigh", "mpo_svd", "mpo_version",
           "mpo_profile", "mpo_profile_read", "mpo_profile_sweeps", "mpo_profile_steps", "mpo_profile_phases", "mpo_svd_static",
           "mpo_probability", "mpo_sample", "mpo_gemm", "mpo_svd_last_stats",
           "mpo_init_batch", "mpo_apply_layer_batch", "mpo_batch_instance", "mpo_svd_truncated", "mpo_gemm_ex",
           "mpo_theta", "mpo_check_superop"]


class MPOError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("eig_max_sweeps", ctypes.c_int), ("sv_rel_cutoff", ctypes.c_double),
                ("arena_cap_bytes", ctypes.c_size_t), ("smode", ctypes.c_int),
                ("barrier_timeout_s", ctypes.c_double), ("block_jacobi_min_rows", ctypes.c_int),
                ("tensor_cores", ctypes.c_int), ("oversample", ctypes.c_int), ("refine_steps", ctypes.c_int)]


_lib = None


def load_library(path: str | None = None):
    """Load the built library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built ({path}); run paper_2003_13163_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, D, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    IP, DP = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    sig = {
        "mpo_default_opts": (None, [ctypes.POINTER(Opts)]),
        "mpo_init": (I, [ctypes.POINTER(P), I, I, I, P, ctypes.POINTER(Opts)]),
        "mpo_apply_layer": (I, [P, I, P, P, I]),
        "mpo_apply_gate": (I, [P, I, P, D]),
        "mpo_apply_superop": (I, [P, I, P]),
        "mpo_sweep": (I, [P]),
        "mpo_entropy": (I, [P, DP, DP, DP]),
        "mpo_schmidt": (I, [P, I, DP, IP]),
        "mpo_bond_dims": (I, [P, IP]),
        "mpo_get_site": (I, [P, I, P, IP, IP]),
        "mpo_to_dense": (I, [P, P]),
        "mpo_centre": (I, [P, IP]),
        "mpo_device_bytes": (Z, [P]),
        "mpo_free": (None, [P]),
        "mpo_last_error": (ctypes.c_char_p, [P]),
        "mpo_eigh": (I, [I, P, P, P, I, I, P]),
        "mpo_svd": (I, [I, I, P, P, P, I, I, I, P]),
        "mpo_version": (ctypes.c_char_p, []),
        "mpo_profile": (I, [P, I]),
        "mpo_profile_read": (I, [P, I, ctypes.POINTER(ctypes.c_char_p), DP, ctypes.POINTER(ctypes.c_longlong), DP, DP]),
        "mpo_profile_sweeps": (ctypes.c_longlong, [P]),
        "mpo_profile_steps": (ctypes.c_longlong, [P]),
        "mpo_profile_phases": (I, [P, DP]),
        "mpo_svd_static": (I, [I, I, P, P, P, I, I, P]),
        "mpo_probability": (I, [P, I, P, P]),
        "mpo_sample": (I, [P, I, P, P, P]),
        "mpo_gemm": (I, [I, I, I, P, P, P, I, I, P]),
        "mpo_svd_last_stats": (I, [IP, DP]),
        "mpo_init_batch": (I, [ctypes.POINTER(P), I, IP, I, I, P, ctypes.POINTER(Opts), I]),
        "mpo_apply_layer_batch": (I, [P, I, P, DP, IP, DP, DP, DP]),
        "mpo_batch_instance": (I, [P, I, ctypes.POINTER(P)]),
        "mpo_svd_truncated": (I, [I, I, P, I, I, ctypes.POINTER(Opts), P, P, DP, IP, P]),
        "mpo_gemm_ex": (I, [I, I, I, P, I, I, P, I, I, P, I, I, I, P]),
        "mpo_theta": (I, [P, I, P, D, P, IP, IP]),
        "mpo_check_superop": (I, [P, D, DP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a) -> int:
    """Raw address of a numpy array or a torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def default_opts() -> Opts:
    o = Opts()
    load_library().mpo_default_opts(ctypes.byref(o))
    return o


def _make_opts(cutoff=0.0, eig_max_sweeps=0, arena_cap_bytes=0, centre_only=False, barrier_timeout_s=0.0,
               block_jacobi_min_rows=0, tensor_cores=False, oversample=0, refine_steps=0) -> Opts:
    o = default_opts()
    if cutoff > 0:
        o.sv_rel_cutoff = cutoff
    if eig_max_sweeps > 0:
        o.eig_max_sweeps = eig_max_sweeps
    o.arena_cap_bytes = arena_cap_bytes
    o.smode = MPO_S_CENTRE if centre_only else MPO_S_ALL_BONDS
    if barrier_timeout_s > 0:
        o.barrier_timeout_s = barrier_timeout_s
    o.block_jacobi_min_rows = block_jacobi_min_rows
    o.tensor_cores = 1 if tensor_cores else 0
    o.oversample = int(oversample)
    o.refine_steps = int(refine_steps)
    return o


class MPO:
    """Handle on one device-resident MPO (see include/mpo.h)."""

    def __init__(self, n: int, chi_max: int, precision: str = "fp64", *, cutoff: float = 0.0,
                 eig_max_sweeps: int = 0, arena_cap_bytes: int = 0, centre_only: bool = False,
                 barrier_timeout_s: float = 0.0, block_jacobi_min_rows: int = 0, tensor_cores: bool = False,
                 oversample: int = 0, refine_steps: int = 0, stream=None, _borrowed=None):
        lib = load_library()
        self._lib = lib
        self.n, self.chi_max = n, chi_max
        self.prec = PRECISIONS[precision]
        self._owned = _borrowed is None
        if _borrowed is not None:        # an instance of a batch: the batch owns it
            self.h = _borrowed
            return
        o = _make_opts(cutoff, eig_max_sweeps, arena_cap_bytes, centre_only, barrier_timeout_s,
                       block_jacobi_min_rows, tensor_cores, oversample, refine_steps)
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream is not None else _current_stream()
        rc = lib.mpo_init(ctypes.byref(h), n, chi_max, self.prec, st, ctypes.byref(o))
        if rc != 0:
            raise MPOError(rc, lib.mpo_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != 0:
            raise MPOError(rc, self._lib.mpo_last_error(self.h).decode())

    def apply_layer(self, parity: int, gates, p) -> None:
        """gates: (n_gates, 4, 4) complex128 (numpy, or a CUDA tensor viewed as
        float64 pairs); p: scalar or (n_gates,) float64."""
        if isinstance(gates, np.ndarray):
            gates = np.ascontiguousarray(gates, dtype=np.complex128)
        if np.isscalar(p):
            pa, stride = np.array([float(p)]), 0
        elif isinstance(p, np.ndarray):
            pa, stride = np.ascontiguousarray(p, dtype=np.float64), 1
        else:
            pa, stride = p, 1
        self._check(self._lib.mpo_apply_layer(self.h, parity, _ptr(gates), _ptr(pa), stride))

    def apply_gate(self, bond: int, U, p: float) -> None:
        """One noisy gate on ABI bond `bond` (no sweep). U: (4, 4) complex128
        numpy array, or a CUDA / pinned tensor of 32 float64 (re, im pairs)."""
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.complex128)
        self._check(self._lib.mpo_apply_gate(self.h, bond, _ptr(U), float(p)))

    def theta(self, bond: int, U, p: float):
        """theta' = M (A_b A_{b+1}) of a noisy gate on ABI bond b, untruncated,
        as a CUDA tensor (4 chi_b, 4 chi_{b+2}) (mpo_theta); the centre moves
        onto the bond."""
        import torch
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.complex128)
        r, c = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.mpo_theta(self.h, bond, _ptr(U), float(p), None, ctypes.byref(r), ctypes.byref(c)))
        dt = torch.complex64 if self.prec == MPO_FP32 else torch.complex128
        out = torch.empty((r.value, c.value), dtype=dt, device="cuda")
        self._check(self._lib.mpo_theta(self.h, bond, _ptr(U), float(p), ctypes.c_void_p(out.data_ptr()),
                                        ctypes.byref(r), ctypes.byref(c)))
        return out

    def apply_superop(self, bond: int, M: np.ndarray) -> None:
        M = np.ascontiguousarray(M, dtype=np.complex128)
        self._check(self._lib.mpo_apply_superop(self.h, bond, _ptr(M)))

    def sweep(self) -> None:
        self._check(self._lib.mpo_sweep(self.h))

    def entropy(self, with_trace: bool = True):
        S = np.empty(self.n - 1)
        tr, dw = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.mpo_entropy(self.h, S.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          ctypes.byref(tr) if with_trace else None, ctypes.byref(dw)))
        return S, (tr.value if with_trace else None), dw.value

    def schmidt(self, bond: int) -> np.ndarray:
        lam = np.empty(self.chi_max)
        ln = ctypes.c_int()
        self._check(self._lib.mpo_schmidt(self.h, bond, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          ctypes.byref(ln)))
        return lam[: ln.value].copy()

    def bond_dims(self) -> np.ndarray:
        d = np.empty(self.n + 1, dtype=np.int32)
        self._check(self._lib.mpo_bond_dims(self.h, d.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return d

    def site(self, k: int) -> np.ndarray:
        cl, cr = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.mpo_get_site(self.h, k, None, ctypes.byref(cl), ctypes.byref(cr)))
        buf = np.empty((cl.value, 4, cr.value), dtype=np.complex128)
        self._check(self._lib.mpo_get_site(self.h, k, _ptr(buf), ctypes.byref(cl), ctypes.byref(cr)))
        return buf

    def to_dense(self) -> np.ndarray:
        out = np.empty((4,) * self.n, dtype=np.complex128)
        self._check(self._lib.mpo_to_dense(self.h, _ptr(out)))
        return out

    def probability(self, bits) -> np.ndarray:
        """P(x) = <<X|rho>> (Sec. 3.4) of bit strings bits: (S, n) of 0/1."""
        bits = np.ascontiguousarray(bits, dtype=np.uint8)
        if bits.ndim == 1:
            bits = bits[None, :]
        P = np.empty(bits.shape[0])
        self._check(self._lib.mpo_probability(self.h, bits.shape[0], _ptr(bits), _ptr(P)))
        return P

    def sample(self, uniforms) -> tuple:
        """Samples by sequential conditionals (Sec. 3.4) from caller uniforms
        (S, n) in [0, 1). Returns (bits (S, n) uint8, P(bits) (S,))."""
        u = np.ascontiguousarray(uniforms, dtype=np.float64)
        bits = np.empty(u.shape, dtype=np.uint8)
        P = np.empty(u.shape[0])
        self._check(self._lib.mpo_sample(self.h, u.shape[0], _ptr(u), _ptr(bits), _ptr(P)))
        return bits, P

    def centre(self) -> int:
        c = ctypes.c_int()
        self._check(self._lib.mpo_centre(self.h, ctypes.byref(c)))
        return c.value

    def profile(self, enable: bool = True) -> None:
        self._check(self._lib.mpo_profile(self.h, int(enable)))

    def profile_read(self) -> dict:
        """{kernel class: {ms, launches, flops, bytes}} since profile(True)."""
        out = {}
        for cls in range(16):
            nm = ctypes.c_char_p()
            ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            n = ctypes.c_longlong()
            rc = self._lib.mpo_profile_read(self.h, cls, ctypes.byref(nm), ctypes.byref(ms), ctypes.byref(n),
                                            ctypes.byref(fl), ctypes.byref(by))
            if rc != 0:
                break
            out[nm.value.decode()] = {"ms": ms.value, "launches": n.value, "flops": fl.value, "bytes": by.value}
        out["_sweeps"] = int(self._lib.mpo_profile_sweeps(self.h))
        out["_steps"] = int(self._lib.mpo_profile_steps(self.h))
        ph = (ctypes.c_double * 3)()
        self._check(self._lib.mpo_profile_phases(self.h, ph))
        out["_block_jacobi_phase_ms"] = {"gram": ph[0], "pair_eig": ph[1], "apply": ph[2]}
        return out

    def device_bytes(self) -> int:
        return int(self._lib.mpo_device_bytes(self.h))

    def close(self) -> None:
        if getattr(self, "h", None) and getattr(self, "_owned", True):
            self._lib.mpo_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()



class MPOBatch:
    """k independent circuits held and advanced together (the batching form,
    see mpo_init_batch in include/mpo.h)."""

    def __init__(self, n_list, chi_max: int, precision: str = "fp32", *, workers: int = 0, stream=None, **opts):
        lib = load_library()
        self._lib = lib
        self.n_list = [int(n) for n in n_list]
        self.k = len(self.n_list)
        self.chi_max = chi_max
        self.precision = precision
        self.prec = PRECISIONS[precision]
        self.offsets = np.concatenate([[0], np.cumsum([n - 1 for n in self.n_list])]).astype(np.int64)
        o = _make_opts(**opts)
        nn = np.ascontiguousarray(self.n_list, dtype=np.int32)
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream is not None else _current_stream()
        rc = lib.mpo_init_batch(ctypes.byref(h), self.k, nn.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                chi_max, self.prec, st, ctypes.byref(o), int(workers))
        if rc != 0:
            raise MPOError(rc, lib.mpo_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != 0:
            raise MPOError(rc, self._lib.mpo_last_error(self.h).decode())

    def apply_layer(self, t: int, gates, p, active=None, *, with_trace: bool = True):
        """Step t (1-based) on the active instances. gates: list over the
        active instances (index order) of (n_gates, 4, 4) complex arrays, or
        one concatenated complex128 array; p: (k,) rates. Returns (S list of
        per-instance entropy arrays, trace (k,), discarded (k,)); entries of
        inactive instances are NaN."""
        if isinstance(gates, (list, tuple)):
            gates = (np.concatenate([np.asarray(g, dtype=np.complex128).reshape(-1) for g in gates])
                     if len(gates) else np.zeros(0, dtype=np.complex128))
        if isinstance(gates, np.ndarray):
            gates = np.ascontiguousarray(gates, dtype=np.complex128)
        pa = np.ascontiguousarray(np.broadcast_to(np.asarray(p, dtype=np.float64), (self.k,)))
        act = None if active is None else np.ascontiguousarray(active, dtype=np.int32)
        S = np.full(int(self.offsets[-1]), np.nan)
        tr = np.full(self.k, np.nan)
        dw = np.full(self.k, np.nan)
        DP = ctypes.POINTER(ctypes.c_double)
        self._check(self._lib.mpo_apply_layer_batch(
            self.h, int(t), _ptr(gates) if (gates.size if isinstance(gates, np.ndarray) else gates.numel()) else None,
            pa.ctypes.data_as(DP),
            None if act is None else act.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            S.ctypes.data_as(DP), tr.ctypes.data_as(DP) if with_trace else None, dw.ctypes.data_as(DP)))
        return [S[self.offsets[i]:self.offsets[i + 1]] for i in range(self.k)], tr, dw

    def instance(self, i: int) -> "MPO":
        """The instance's context for diagnostics (owned by the batch)."""
        q = ctypes.c_void_p()
        self._check(self._lib.mpo_batch_instance(self.h, int(i), ctypes.byref(q)))
        return MPO(self.n_list[i], self.chi_max, self.precision, _borrowed=q)

    def close(self) -> None:
        if getattr(self, "h", None):
            self._lib.mpo_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

def eigh(A, precision: str = "fp64", max_sweeps: int = 0):
    """Hermitian eigen-solve on the device through the C ABI (test export).

    A: CUDA torch tensor (m, m) complex128/complex64, overwritten. Returns
    (w, V) torch tensors (unsorted)."""
    import torch
    lib = load_library()
    m = A.shape[0]
    prec = {"fp64": MPO_FP64, "fp32": MPO_FP32}[precision]
    rdt = torch.float64 if prec == MPO_FP64 else torch.float32
    w = torch.empty(m, dtype=rdt, device=A.device)
    V = torch.empty_like(A)
    rc = lib.mpo_eigh(m, A.data_ptr(), w.data_ptr(), V.data_ptr(), prec, max_sweeps,
                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise MPOError(rc, "mpo_eigh failed")
    return w, V


def svd_rows(X, precision: str = "fp64", max_sweeps: int = 0, block: bool = False):
    """One-sided Jacobi SVD on the device (test export). X: CUDA tensor (r, c),
    overwritten with U^H X. Returns (w, Ut): squared row norms and U^T."""
    import torch
    lib = load_library()
    r, c = X.shape
    prec = {"fp64": MPO_FP64, "fp32": MPO_FP32}[precision]
    rdt = torch.float64 if prec == MPO_FP64 else torch.float32
    w = torch.empty(r, dtype=rdt, device=X.device)
    Ut = torch.empty((r, r), dtype=X.dtype, device=X.device)
    rc = lib.mpo_svd(r, c, X.data_ptr(), w.data_ptr(), Ut.data_ptr(), prec, max_sweeps, int(block),
                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise MPOError(rc, "mpo_svd failed")
    return w, Ut


def svd_last_stats() -> dict:
    """Sweeps and block-Jacobi phase times (ms) of the last svd_rows call on
    this thread."""
    lib = load_library()
    sw = ctypes.c_int()
    ph = (ctypes.c_double * 3)()
    lib.mpo_svd_last_stats(ctypes.byref(sw), ph)
    return {"sweeps": sw.value, "gram_ms": ph[0], "pair_eig_ms": ph[1], "apply_ms": ph[2]}


def svd_rows_static(X, precision: str = "fp64", max_sweeps: int = 0):
    """Block one-sided Jacobi SVD through the entry point that allocates
    nothing (r <= 512, c <= 2048). Same outputs as svd_rows(..., block=True)."""
    import torch
    lib = load_library()
    r, c = X.shape
    prec = {"fp64": MPO_FP64, "fp32": MPO_FP32}[precision]
    rdt = torch.float64 if prec == MPO_FP64 else torch.float32
    w = torch.empty(r, dtype=rdt, device=X.device)
    Ut = torch.empty((r, r), dtype=X.dtype, device=X.device)
    rc = lib.mpo_svd_static(r, c, X.data_ptr(), w.data_ptr(), Ut.data_ptr(), prec, max_sweeps,
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise MPOError(rc, lib.mpo_last_error(None).decode())
    return w, Ut


def gemm(A, B, precision: str = "fp32", tensor_cores: bool = True):
    """C = A B on the device through the C ABI (test export); A (M, K), B (K, N)
    CUDA complex tensors, contiguous."""
    import torch
    lib = load_library()
    M, K = A.shape
    N = B.shape[1]
    C = torch.empty((M, N), dtype=A.dtype, device=A.device)
    prec = {"fp64": MPO_FP64, "fp32": MPO_FP32}[precision]
    rc = lib.mpo_gemm(M, N, K, A.data_ptr(), B.data_ptr(), C.data_ptr(), prec, int(tensor_cores),
                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise MPOError(rc, "mpo_gemm failed")
    return C


def svd_truncated(A, cap: int, precision: str = "mixed", **opts):
    """Truncated SVD of one matrix in the arithmetic of a precision form
    (mpo_svd_truncated, test export). A: CUDA tensor (r, c), r <= c,
    complex128 (fp64 / mixed) or complex64 (fp32); not modified. Returns
    (U (r, k), X (k, c), lam2 (k,) numpy) with U X the kept part of A."""
    import torch
    lib = load_library()
    r, c = A.shape
    prec = PRECISIONS[precision]
    U = torch.zeros((r, cap), dtype=A.dtype, device=A.device)
    X = torch.zeros((cap, c), dtype=A.dtype, device=A.device)
    lam2 = np.zeros(cap)
    k = ctypes.c_int()
    o = _make_opts(**opts)
    rc = lib.mpo_svd_truncated(r, c, A.contiguous().data_ptr(), cap, prec, ctypes.byref(o), U.data_ptr(),
                               X.data_ptr(), lam2.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(k),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise MPOError(rc, lib.mpo_last_error(None).decode())
    kk = k.value
    return U[:, :kk], X[:kk], lam2[:kk]


def check_superop(M, tol: float = 0.0):
    """(is_channel, defect) of a 16x16 two-qubit superoperator in the App. A
    convention (mpo_check_superop): trace preserving and completely positive
    to tol times its largest entry."""
    M = np.ascontiguousarray(M, dtype=np.complex128)
    d = ctypes.c_double()
    rc = load_library().mpo_check_superop(_ptr(M), float(tol), ctypes.byref(d))
    if rc not in (0, -1):
        raise MPOError(rc, "mpo_check_superop failed")
    return rc == 0, d.value


def gemm_ex(A, B, opA: int = 0, opB: int = 0, precision: str = "fp64", engine: int = 1):
    """C = op(A) op(B) through mpo_gemm_ex (test export); op 1 = conjugate
    transpose. A, B: contiguous CUDA complex tensors."""
    import torch
    lib = load_library()
    M = A.shape[1] if opA else A.shape[0]
    K = A.shape[0] if opA else A.shape[1]
    N = B.shape[0] if opB else B.shape[1]
    C = torch.zeros((M, N), dtype=A.dtype, device=A.device)
    rc = lib.mpo_gemm_ex(M, N, K, A.data_ptr(), A.shape[1], opA, B.data_ptr(), B.shape[1], opB, C.data_ptr(), N,
                         PRECISIONS[precision], engine, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise MPOError(rc, lib.mpo_last_error(None).decode())
    return C
