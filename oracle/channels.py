"""Two-qubit channels of Sec. 2.2 and their 16x16 superoperators (App. A).

Oracle code: test infrastructure only, see ``oracle/__init__.py``.

Conventions (Sec. 3.1 and App. A):
  * two-qubit kets |i_l i_{l+1}> have basis index 2*i_l + i_{l+1};
  * the vectorised local index is I = d*i + i' (ket digit high, bra digit
    low), d = 2, so I in {0,1,2,3};
  * M[(I_l, I_{l+1}), (J_l, J_{l+1})] = <i_l i_{l+1}| M(|j_l j_{l+1}><j'_l j'_{l+1}|) |i'_l i'_{l+1}>
    with row index 4*I_l + I_{l+1} and column index 4*J_l + J_{l+1}
    (App. A, definition of M; the printed symbol there is N, the text means
    the noisy gate M = N o U of Sec. 3.2).
"""
from __future__ import annotations

import itertools

import numpy as np

_I2 = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULIS = (_I2, _X, _Y, _Z)


def two_qubit_paulis_nontrivial():
    """The 15 non-trivial two-qubit Paulis E_2 = {I,X,Y,Z}^(x2) - {I (x) I} (Sec. 2.2)."""
    out = []
    for a, b in itertools.product(range(4), range(4)):
        if a == 0 and b == 0:
            continue
        out.append(np.kron(PAULIS[a], PAULIS[b]))
    return out


def depolarize2(rho: np.ndarray, p: float) -> np.ndarray:
    """N_2[p](rho) = (1-p) rho + p/15 sum_{P in E_2} P rho P (Sec. 2.2, first form),
    rho a 4x4 operator on the two qubits."""
    acc = (1.0 - p) * rho
    for P in two_qubit_paulis_nontrivial():
        acc = acc + (p / 15.0) * (P @ rho @ P)
    return acc


def depolarize2_closed(rho: np.ndarray, p: float) -> np.ndarray:
    """Second form of Sec. 2.2: (1 - 16p/15) rho + (16p/15) (I (x) I / 4) Tr rho."""
    lam = 16.0 * p / 15.0
    return (1.0 - lam) * rho + lam * np.trace(rho) * np.eye(4) / 4.0


def noisy_gate(U: np.ndarray, p: float):
    """The map M = N_2[p] o U with U(rho) = U rho U^dagger (Sec. 3.2)."""
    def apply(rho):
        return depolarize2(U @ rho @ U.conj().T, p)
    return apply


def superop(channel) -> np.ndarray:
    """16x16 matrix of a two-qubit map in the index convention of App. A.

    Column (J_l, J_{l+1}) is the image of the matrix unit
    |j_l j_{l+1}><j'_l j'_{l+1}|; row (I_l, I_{l+1}) reads the entry
    <i_l i_{l+1}| . |i'_l i'_{l+1}> of that image."""
    M = np.zeros((16, 16), dtype=np.complex128)
    for Jl, Jr in itertools.product(range(4), range(4)):
        jl, jlp = divmod(Jl, 2)
        jr, jrp = divmod(Jr, 2)
        E = np.zeros((4, 4), dtype=np.complex128)
        E[2 * jl + jr, 2 * jlp + jrp] = 1.0
        img = channel(E)
        for Il, Ir in itertools.product(range(4), range(4)):
            il, ilp = divmod(Il, 2)
            ir, irp = divmod(Ir, 2)
            M[4 * Il + Ir, 4 * Jl + Jr] = img[2 * il + ir, 2 * ilp + irp]
    return M


def noisy_gate_superop(U: np.ndarray, p: float) -> np.ndarray:
    """Superoperator of the noisy Haar gate M = N_2[p] o U (Sec. 3.2, App. A)."""
    return superop(noisy_gate(U, p))


def trace_vector() -> np.ndarray:
    """t with t[(I_l, I_{l+1})] = delta_{i_l i'_l} delta_{i_{l+1} i'_{l+1}}: t^T vec(rho) = Tr rho
    (the vectorised trace of Sec. 3.4; I = 3x for x in {0,1} picks the diagonal)."""
    t1 = np.array([1.0, 0.0, 0.0, 1.0])
    return np.kron(t1, t1)


def choi(M: np.ndarray) -> np.ndarray:
    """Choi matrix C = sum_{jk} M(|j><k|) (x) |j><k| of a two-qubit map given by its
    superoperator M (rows/cols in the App. A convention), as a 16x16 matrix
    with row (i, j) and column (i', k). CPTP maps have C >= 0."""
    C = np.zeros((4, 4, 4, 4), dtype=np.complex128)  # [i, j, i', k]
    for j in range(4):
        for k in range(4):
            jl, jr = divmod(j, 2)
            kl, kr = divmod(k, 2)
            col = 4 * (2 * jl + kl) + (2 * jr + kr)
            img = np.zeros((4, 4), dtype=np.complex128)
            for i in range(4):
                for ip in range(4):
                    il, ir = divmod(i, 2)
                    ipl, ipr = divmod(ip, 2)
                    row = 4 * (2 * il + ipl) + (2 * ir + ipr)
                    img[i, ip] = M[row, col]
            C[:, j, :, k] = img
    return C.reshape(16, 16)
