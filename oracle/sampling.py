"""Output probabilities and sampling of Sec. 3.4, from the dense |rho>>.

Oracle code: test infrastructure only, see ``oracle/__init__.py``.

P(x) = <<X|rho>> with X_k = (d+1) x_k = 3 x_k: the diagonal entry
rho[x, x] read from the vectorised tensor (Sec. 3.4). Sampling follows the
sequential-conditional rule of Sec. 3.4 with marginals formed by brute-force
summation of P over the undetermined bits (no MPO contraction, so this pins
the GPU's environment-based chain independently).
"""
from __future__ import annotations

import itertools

import numpy as np


def probabilities(T: np.ndarray, bits: np.ndarray) -> np.ndarray:
    """P(x) for each row x of bits (shape (S, n), entries 0/1)."""
    bits = np.atleast_2d(bits)
    return np.array([T[tuple(3 * int(b) for b in row)].real for row in bits])


def all_probabilities(T: np.ndarray) -> np.ndarray:
    """P over all 2^n strings, index = integer with x_1 as the high bit."""
    n = T.ndim
    return np.array([T[tuple(3 * b for b in x)].real for x in itertools.product((0, 1), repeat=n)])


def sample(T: np.ndarray, uniforms: np.ndarray) -> np.ndarray:
    """Sequential conditionals (Sec. 3.4): bit k is 0 iff
    u_k < P(x_1..x_{k-1}, 0) / (P(.., 0) + P(.., 1)), marginals by summation."""
    n = T.ndim
    Pall = all_probabilities(T).reshape((2,) * n)
    out = np.zeros(uniforms.shape, dtype=np.uint8)
    for s in range(uniforms.shape[0]):
        prefix = ()
        for k in range(n):
            m0 = Pall[prefix + (0,)].sum()
            m1 = Pall[prefix + (1,)].sum()
            m0, m1 = max(m0, 0.0), max(m1, 0.0)
            x = 0 if (m0 + m1 > 0.0 and uniforms[s, k] < m0 / (m0 + m1)) or m0 + m1 <= 0.0 else 1
            out[s, k] = x
            prefix = prefix + (x,)
    return out
