"""MPO entanglement entropy (Sec. 3.3) and Page's mean entanglement entropy.

Oracle code: test infrastructure only, see ``oracle/__init__.py``.
"""
from __future__ import annotations

import numpy as np


def mpo_entropy(lam) -> float:
    """S_l = -sum_a p_a log2 p_a with p_a = lambda_a^2 / sum_b lambda_b^2
    (Sec. 3.3, definition of the MPO entanglement entropy). Terms with
    p_a = 0 contribute 0 (the limit p log p -> 0)."""
    lam = np.asarray(lam, dtype=np.float64)
    w = lam * lam
    tot = w.sum()
    if tot <= 0.0:
        return 0.0
    p = w / tot
    p = p[p > 0.0]
    return float(-(p * np.log2(p)).sum())


def von_neumann_from_schmidt(s) -> float:
    """Entanglement entropy of a pure state from its Schmidt coefficients s:
    S = -sum s^2 log2 s^2 (the S_l(|psi>) of Sec. 3.3), normalised."""
    s = np.asarray(s, dtype=np.float64)
    w = s * s
    w = w / w.sum()
    w = w[w > 0.0]
    return float(-(w * np.log2(w)).sum())


def page_entropy_bits(m: int, n: int) -> float:
    """Page's average entanglement entropy of an m x n bipartite Haar state,
    m <= n: S = sum_{k=n+1}^{mn} 1/k - (m-1)/(2n) nats (Page 1993), in bits.
    Sec. 4.1 quotes 2*S_{16,16} = 6.56 for n = 8 qubits at p = 0."""
    if m > n:
        m, n = n, m
    s = sum(1.0 / k for k in range(n + 1, m * n + 1)) - (m - 1) / (2.0 * n)
    return s / np.log(2.0)
