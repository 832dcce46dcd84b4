"""Oracle D: the vectorised density matrix as a dense 4^n tensor (n <= 10).

Oracle code: test infrastructure only, see ``oracle/__init__.py``.

What it computes, gate by gate in circuit order (Sec. 4.1: the gates of a
step are applied sequentially, bond ascending):
  1. |rho>> <- M |rho>> with M the 16x16 superoperator on sites (l, l+1)
     (App. A, the B = M . (...) step);
  2. truncation: the operator-Schmidt decomposition of |rho>> across the cut
     [1..l]:[(l+1)..n] (App. A, SVD of B), keeping the chi_max largest
     Schmidt values and, of those, the ones above cutoff * lambda_max; no
     renormalisation (Sec. 3.4 uses Tr rho < 1 as the truncation diagnostic).
After every step it records S_l (Sec. 3.3) at every cut from the exact
Schmidt values of the current |rho>>, Tr rho (Sec. 3.4) and the discarded
weight of each gate. No MPO is involved, so this pins the truncation
semantics independently of any canonical-form bookkeeping.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .channels import noisy_gate_superop
from .entropy import mpo_entropy


def initial_vec(n: int) -> np.ndarray:
    """|0..0><0..0| vectorised: only I_k = 0 for every k (Sec. 4.1)."""
    T = np.zeros((4,) * n, dtype=np.complex128)
    T[(0,) * n] = 1.0
    return T


def apply_superop(T: np.ndarray, M: np.ndarray, l: int) -> np.ndarray:
    """Apply a 16x16 superoperator on sites (l, l+1), paper bond l (1-based)."""
    n = T.ndim
    t = T.reshape(4 ** (l - 1), 16, 4 ** (n - l - 1))
    return np.einsum("ij,ajb->aib", M, t).reshape((4,) * n)


def schmidt_values(T: np.ndarray, l: int) -> np.ndarray:
    """Operator-Schmidt values of |rho>> across the cut after site l (descending)."""
    n = T.ndim
    return np.linalg.svd(T.reshape(4 ** l, 4 ** (n - l)), compute_uv=False)


def truncate(T: np.ndarray, l: int, chi_max: int, cutoff: float):
    """Keep the chi_max largest Schmidt terms across cut l (App. A); also drop
    values <= cutoff * lambda_max. Returns (T', discarded weight)."""
    n = T.ndim
    mat = T.reshape(4 ** l, 4 ** (n - l))
    U, s, Vh = np.linalg.svd(mat, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return T, 0.0
    k = int(min(chi_max, np.count_nonzero(s > cutoff * s[0])))
    k = max(k, 1)
    tot = float((s * s).sum())
    w = float((s[k:] ** 2).sum() / tot) if tot > 0 else 0.0
    mat2 = (U[:, :k] * s[:k][None, :]) @ Vh[:k]
    return mat2.reshape((4,) * n), w


def trace(T: np.ndarray) -> complex:
    """Tr rho = sum over I_k in {0, 3} of |rho>> (Sec. 3.4, I = (d+1) x)."""
    t1 = np.array([1.0, 0.0, 0.0, 1.0])
    out = T
    for _ in range(T.ndim):
        out = np.tensordot(t1, out, axes=(0, 0))
    return complex(out)


@dataclass
class DenseResult:
    S: np.ndarray                      # (depth, n-1) MPO entropies after every step
    trace: np.ndarray                  # (depth,) Tr rho after every step
    discarded: list = field(default_factory=list)   # per step: array of per-gate weights
    schmidt: list = field(default_factory=list)     # per step: list of n-1 Schmidt vectors
    final: np.ndarray = None           # final |rho>> tensor


def run(circuit, chi_max: int, cutoff: float = 0.0, keep_schmidt: bool = False) -> DenseResult:
    from paper_2003_13163_gb300.circuits import layer_bonds

    n = circuit.n
    T = initial_vec(n)
    S_rows, tr, disc, sch = [], [], [], []
    for t in range(1, circuit.depth + 1):
        ws = []
        for U, p, l in zip(circuit.gates[t - 1], circuit.p[t - 1], layer_bonds(n, circuit.parity(t))):
            T = apply_superop(T, noisy_gate_superop(U, p), l)
            T, w = truncate(T, l, chi_max, cutoff)
            ws.append(w)
        lams = [schmidt_values(T, l) for l in range(1, n)]
        S_rows.append([mpo_entropy(lm) for lm in lams])
        tr.append(trace(T).real)
        disc.append(np.array(ws))
        if keep_schmidt:
            sch.append(lams)
    return DenseResult(S=np.array(S_rows), trace=np.array(tr), discarded=disc, schmidt=sch, final=T)
