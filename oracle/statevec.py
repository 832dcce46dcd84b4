"""Pure-state simulator for the noiseless (p = 0) pin of Sec. 3.3:
S_l(|psi><psi|) = 2 S_l(|psi>).

Oracle code: test infrastructure only, see ``oracle/__init__.py``.
"""
from __future__ import annotations

import numpy as np

from .entropy import von_neumann_from_schmidt


def initial_psi(n: int) -> np.ndarray:
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply_gate(psi: np.ndarray, U: np.ndarray, l: int) -> np.ndarray:
    """Apply a 4x4 U to qubits (l, l+1) (paper bond l, 1-based)."""
    n = int(np.log2(psi.size))
    t = psi.reshape(2 ** (l - 1), 4, 2 ** (n - l - 1))
    return np.einsum("ij,ajb->aib", U, t).reshape(-1)


def entropies(psi: np.ndarray) -> np.ndarray:
    """S_l(|psi>) for l = 1..n-1 (von Neumann entropy of the left block, bits)."""
    n = int(np.log2(psi.size))
    out = np.empty(n - 1)
    for l in range(1, n):
        s = np.linalg.svd(psi.reshape(2 ** l, 2 ** (n - l)), compute_uv=False)
        out[l - 1] = von_neumann_from_schmidt(s)
    return out


def run(circuit) -> np.ndarray:
    """Entropies after every step of a noiseless circuit: array (depth, n-1)."""
    from paper_2003_13163_gb300.circuits import layer_bonds

    psi = initial_psi(circuit.n)
    rows = []
    for t in range(1, circuit.depth + 1):
        for U, l in zip(circuit.gates[t - 1], layer_bonds(circuit.n, circuit.parity(t))):
            psi = apply_gate(psi, U, l)
        rows.append(entropies(psi))
    return np.array(rows)
