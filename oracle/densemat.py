"""Plain 2^n x 2^n density-matrix simulator of the noisy brickwork (Sec. 2.1-2.2).

Oracle code: test infrastructure only, see ``oracle/__init__.py``.
Qubit 1 is the most significant bit of the computational-basis index. Each
noisy gate on qubits (l, l+1) maps rho -> N_2[p](U rho U^dagger) with U and
the Paulis embedded as I (x) G (x) I; the channel is the Pauli-sum form of
Sec. 2.2. Intended for n <= 8.
"""
from __future__ import annotations

import numpy as np

from .channels import two_qubit_paulis_nontrivial


def _embed(G: np.ndarray, n: int, l: int) -> np.ndarray:
    """I_{2^(l-1)} (x) G (x) I_{2^(n-l-1)} for a two-qubit G on paper bond l."""
    return np.kron(np.kron(np.eye(2 ** (l - 1)), G), np.eye(2 ** (n - l - 1)))


def initial_rho(n: int) -> np.ndarray:
    """|0...0><0...0| (Sec. 2.1)."""
    rho = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
    rho[0, 0] = 1.0
    return rho


def apply_noisy_gate(rho: np.ndarray, U: np.ndarray, p: float, l: int) -> np.ndarray:
    n = int(np.log2(rho.shape[0]))
    Uf = _embed(U, n, l)
    r = Uf @ rho @ Uf.conj().T
    out = (1.0 - p) * r
    for P in two_qubit_paulis_nontrivial():
        Pf = _embed(P, n, l)
        out = out + (p / 15.0) * (Pf @ r @ Pf)
    return out


def rho_to_vec(rho: np.ndarray) -> np.ndarray:
    """|rho>> of Sec. 3.1 as a (4,)*n tensor with I_k = 2 i_k + i'_k."""
    n = int(np.log2(rho.shape[0]))
    t = rho.reshape((2,) * (2 * n))
    perm = []
    for k in range(n):
        perm += [k, n + k]
    return t.transpose(perm).reshape((4,) * n)


def vec_to_rho(T: np.ndarray) -> np.ndarray:
    n = T.ndim
    t = T.reshape((2,) * (2 * n))
    perm = [2 * k for k in range(n)] + [2 * k + 1 for k in range(n)]
    return t.transpose(perm).reshape(2 ** n, 2 ** n)
