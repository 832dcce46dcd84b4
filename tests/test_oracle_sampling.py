"""Pins of the oracle's output probabilities and sampler (Sec. 3.4)."""
import itertools

import numpy as np

from oracle import dense, sampling, statevec
from paper_2003_13163_gb300.circuits import random_circuit, sampling_uniforms


def test_probabilities_sum_to_trace_and_match_pure_state():
    c = random_circuit(6, 4, 0.0, seed=3)
    T = dense.run(c, 64).final
    Pall = sampling.all_probabilities(T)
    psi = statevec.initial_psi(6)
    from paper_2003_13163_gb300.circuits import layer_bonds
    for t in range(1, c.depth + 1):
        for U, l in zip(c.gates[t - 1], layer_bonds(6, c.parity(t))):
            psi = statevec.apply_gate(psi, U, l)
    np.testing.assert_allclose(Pall, np.abs(psi) ** 2, atol=1e-13)        # p = 0: P(x) = |psi(x)|^2
    np.testing.assert_allclose(Pall.sum(), dense.trace(T).real, atol=1e-13)


def test_noisy_truncated_probabilities_sum_to_trace():
    c = random_circuit(8, 5, 0.05, seed=4)
    d = dense.run(c, 8, 1e-12)
    np.testing.assert_allclose(sampling.all_probabilities(d.final).sum(), d.trace[-1], atol=1e-12)
    assert d.trace[-1] < 1.0


def test_product_state_and_maximally_mixed():
    T = dense.initial_vec(4)
    P = sampling.all_probabilities(T)
    assert P[0] == 1.0 and P[1:].sum() == 0.0
    c = random_circuit(4, 1, 15 / 16, seed=1)
    P = sampling.all_probabilities(dense.run(c, 16).final)
    np.testing.assert_allclose(P, 1 / 16, atol=1e-14)


def test_sampler_frequencies_follow_P():
    c = random_circuit(4, 3, 0.02, seed=9)
    T = dense.run(c, 16).final
    P = sampling.all_probabilities(T)
    S = 20000
    bits = sampling.sample(T, sampling_uniforms(S, 4, seed=11))
    idx = (bits * (1 << np.arange(3, -1, -1))).sum(axis=1)
    freq = np.bincount(idx, minlength=16) / S
    sigma = np.sqrt(P * (1 - P) / S)
    assert np.all(np.abs(freq - P) <= 5 * sigma + 1e-12)


def test_sampler_is_inverse_cdf_in_lexicographic_order():
    """With conditionals in bit order, the sampler is the inverse CDF of P over
    strings ordered x_1 high: u in the first bit picks the half, and so on."""
    c = random_circuit(4, 2, 0.0, seed=2)
    T = dense.run(c, 16).final
    P = sampling.all_probabilities(T)
    cdf = np.cumsum(P)
    rng = np.random.default_rng(0)
    for _ in range(50):
        u1 = rng.random()
        bits = sampling.sample(T, np.array([[u1, 0.0, 0.0, 0.0]]))[0]
        # with later uniforms 0 the string is the first one of its prefix class
        # whose mass makes the first-bit choice consistent with u1
        first = 0 if u1 < P[:8].sum() / P.sum() else 1
        assert bits[0] == first
