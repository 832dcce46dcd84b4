"""Seeded synthetic inputs for the 1D noisy brickwork circuit (Sec. 2.1, Sec. 4.1).

This module only draws random numbers and lays out the brickwork schedule; it
holds none of the simulation arithmetic (no superoperator, no contraction, no
SVD). Both the CUDA path and the CPU oracle take their gates from here, so a
parity test never depends on two random-number generators agreeing.

Haar-random 4x4 unitaries (Sec. 4.1: "n/2 Haar-random two-qubit unitary
operators" per odd time step, "(n-2)/2" per even one) are drawn with the
QR-of-a-complex-Gaussian recipe with the phase fix of Mezzadri (2007):
Z = (X + iY)/sqrt(2) with X, Y i.i.d. N(0,1); Z = QR; U = Q diag(R_jj/|R_jj|).
Each gate consumes exactly one ``standard_normal((2, 4, 4))`` draw from a
``numpy.random.Generator(PCG64(seed))`` stream, gates in circuit order
(time step ascending, bond ascending).

Brickwork (Sec. 2.1, Fig. 2): qubits 1..n (n even). Odd time steps t act on
the bonds l = 1, 3, ..., n-1 (parity 0); even time steps on l = 2, 4, ..., n-2
(parity 1). Gate i of a layer of parity q acts on paper bond l = 2i + 1 + q,
i.e. sites (l, l+1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def layer_parity(t: int) -> int:
    """Parity of time step t (1-based): 0 for odd t, 1 for even t (Sec. 2.1)."""
    if t < 1:
        raise ValueError("time steps are 1-based")
    return (t + 1) % 2


def layer_bonds(n: int, parity: int) -> list[int]:
    """Paper bonds l (1-based; gate acts on qubits l, l+1) of one brickwork layer."""
    if n < 2 or n % 2:
        raise ValueError("n must be even and >= 2")
    return list(range(1 + parity, n, 2))


def n_gates(n: int, parity: int) -> int:
    return len(layer_bonds(n, parity))


def haar_unitary(rng: np.random.Generator) -> np.ndarray:
    """One 4x4 Haar-random unitary (Mezzadri 2007), complex128."""
    g = rng.standard_normal((2, 4, 4))
    z = (g[0] + 1j * g[1]) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    return q * (d / np.abs(d))[None, :]


@dataclass
class Circuit:
    """A depth-D noisy brickwork circuit on n qubits.

    gates[t-1]  : complex128 array (n_gates(n, parity(t)), 4, 4), row-major,
                  basis index 2*i_l + i_{l+1} (qubit l is the high digit).
    p[t-1]      : float64 array (n_gates,), the depolarising rate of Sec. 2.2
                  applied after each gate.
    """

    n: int
    depth: int
    seed: int
    gates: list = field(default_factory=list)
    p: list = field(default_factory=list)

    def parity(self, t: int) -> int:
        return layer_parity(t)

    def total_gates(self) -> int:
        return sum(len(g) for g in self.gates)


def random_circuit(n: int, depth: int, p: float, seed: int) -> Circuit:
    """Seeded Haar brickwork circuit with a uniform depolarising rate p."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = Circuit(n=n, depth=depth, seed=seed)
    for t in range(1, depth + 1):
        k = n_gates(n, layer_parity(t))
        us = np.empty((k, 4, 4), dtype=np.complex128)
        for i in range(k):
            us[i] = haar_unitary(rng)
        c.gates.append(us)
        c.p.append(np.full(k, float(p)))
    return c


def ensemble_instances(k: int, seed: int = 4, n_choices=(16, 24, 32, 40, 48, 56, 64),
                       p_choices=(0.005, 0.01, 0.02, 0.05), depth_per_qubit: int = 2,
                       gate_seed0: int = 1000) -> list[Circuit]:
    """k independent instances for the batching form: (n_i, p_i) drawn
    uniformly from the choices with PCG64(seed) (n first, then p, per
    instance), depth D_i = depth_per_qubit * n_i, and instance i's gates from
    PCG64(gate_seed0 + i)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(k):
        n = int(n_choices[rng.integers(len(n_choices))])
        p = float(p_choices[rng.integers(len(p_choices))])
        out.append(random_circuit(n, depth_per_qubit * n, p, gate_seed0 + i))
    return out


def random_hermitian_psd(m: int, decay: float, seed: int, dtype=np.complex128) -> np.ndarray:
    """Seeded Hermitian positive semidefinite m x m matrix with spectrum
    exp(-decay * k), k = 0..m-1 (a test input for the eigensolver; the
    exponentially decaying spectrum mirrors the Schmidt spectra of Fig. 7)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    q = q * (np.diagonal(r) / np.abs(np.diagonal(r)))[None, :]
    w = np.exp(-decay * np.arange(m))
    return ((q * w[None, :]) @ q.conj().T).astype(dtype)


def random_complex(shape, seed: int) -> np.ndarray:
    """Seeded complex Gaussian array, entries CN(0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal((2,) + tuple(shape))
    return (g[0] + 1j * g[1]) / np.sqrt(2.0)


def sampling_uniforms(n_samples: int, n: int, seed: int) -> np.ndarray:
    """Seeded uniforms in [0, 1), shape (n_samples, n): the random input of the
    sequential-conditional sampler (Sec. 3.4), one per sample and qubit."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((n_samples, n))
