"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU (no GPU marker). Each check is chosen so that a
plausible mistake in the oracle (a wrong sign, a transposed superoperator
index, a dropped term, a mis-ordered site) breaks at least one of them.
"""
import json
import os

import numpy as np
import pytest

from oracle import channels, dense, densemat, mpo, statevec
from oracle.entropy import mpo_entropy, page_entropy_bits
from paper_2003_13163_gb300.circuits import haar_unitary, layer_bonds, random_circuit

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def rand_rho(d, seed):
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    r = z @ z.conj().T
    return r / np.trace(r)


def rand_u(seed):
    return haar_unitary(np.random.Generator(np.random.PCG64(seed)))


# ---------------------------------------------------------------- channels --
@pytest.mark.parametrize("p", [0.0, 0.01, 0.3, 15 / 16, 1.0])
def test_depolarising_two_forms_agree(p):
    """Sec. 2.2 states the Pauli-sum form equals (1-16p/15) rho + 16p/15 I/4 Tr rho."""
    rho = rand_rho(4, 1)
    np.testing.assert_allclose(channels.depolarize2(rho, p), channels.depolarize2_closed(rho, p), atol=1e-14)


def test_superop_is_trace_preserving_and_cp():
    t = channels.trace_vector()
    for s in range(5):
        M = channels.noisy_gate_superop(rand_u(s), 0.1 * s)
        np.testing.assert_allclose(t @ M, t, atol=1e-13)
        C = channels.choi(M)
        np.testing.assert_allclose(C, C.conj().T, atol=1e-13)
        assert np.linalg.eigvalsh(C).min() > -1e-12
        assert abs(np.trace(C) - 4.0) < 1e-12


def _vec2(rho):
    """Vectorise a two-qubit operator independently of oracle.channels: entry
    4*I_l + I_r with I = 2 i + i' (Sec. 3.1)."""
    v = np.zeros(16, dtype=complex)
    for il in range(2):
        for ilp in range(2):
            for ir in range(2):
                for irp in range(2):
                    v[4 * (2 * il + ilp) + (2 * ir + irp)] = rho[2 * il + ir, 2 * ilp + irp]
    return v


@pytest.mark.parametrize("p", [0.0, 0.05, 0.5])
def test_superop_acts_as_channel_on_vectorised_rho(p):
    """M vec(rho) == vec(N(U rho U^dag)) for the App. A index convention."""
    U = rand_u(7)
    M = channels.noisy_gate_superop(U, p)
    rho = rand_rho(4, 3)
    lhs = M @ _vec2(rho)
    rhs = _vec2(channels.depolarize2_closed(U @ rho @ U.conj().T, p))
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def test_superop_closed_forms():
    """p = 15/16 is the fully depolarising map t t^T / 4; p = 1 is not."""
    t = channels.trace_vector()
    U = rand_u(11)
    np.testing.assert_allclose(channels.noisy_gate_superop(U, 15 / 16), np.outer(t, t) / 4, atol=1e-13)
    assert np.abs(channels.noisy_gate_superop(U, 1.0) - np.outer(t, t) / 4).max() > 1e-3


def test_haar_inputs_are_unitary_and_haar_moment():
    rng = np.random.Generator(np.random.PCG64(5))
    acc = 0.0
    N = 4000
    for _ in range(N):
        U = haar_unitary(rng)
        acc += abs(U[0, 0]) ** 2
    np.testing.assert_allclose(U.conj().T @ U, np.eye(4), atol=1e-13)
    # E|U_11|^2 = 1/4, variance of |U_11|^2 is 3/80 for Haar U(4): 5 sigma bound
    assert abs(acc / N - 0.25) < 5 * np.sqrt(3 / 80 / N)


# ----------------------------------------------------------------- entropy --
def test_entropy_closed_forms():
    assert mpo_entropy([1.0, 0.0, 0.0]) == 0.0
    np.testing.assert_allclose(mpo_entropy(np.ones(16)), 4.0, atol=1e-14)
    np.testing.assert_allclose(mpo_entropy([3.0, 3.0, 0.0]), 1.0, atol=1e-14)
    # scale invariance (Sec. 3.3 normalises by sum lambda^2)
    lam = np.array([0.9, 0.3, 0.1, 1e-3])
    np.testing.assert_allclose(mpo_entropy(lam), mpo_entropy(7.5 * lam), atol=1e-14)
    np.testing.assert_allclose(2 * page_entropy_bits(16, 16), 6.5638757, atol=1e-6)


# ---------------------------------------------------- dense vs rho matrices --
@pytest.mark.parametrize("n", [4, 6])
def test_dense_oracle_matches_density_matrix_simulation(n):
    """Vectorised superoperator simulation == plain rho -> N(U rho U^dag)."""
    c = random_circuit(n, 4, 0.07, seed=n)
    rho = densemat.initial_rho(n)
    T = dense.initial_vec(n)
    for t in range(1, c.depth + 1):
        for U, p, l in zip(c.gates[t - 1], c.p[t - 1], layer_bonds(n, c.parity(t))):
            rho = densemat.apply_noisy_gate(rho, U, p, l)
            T = dense.apply_superop(T, channels.noisy_gate_superop(U, p), l)
        np.testing.assert_allclose(densemat.vec_to_rho(T), rho, atol=1e-13)
        np.testing.assert_allclose(np.trace(rho), 1.0, atol=1e-13)
        np.testing.assert_allclose(rho, rho.conj().T, atol=1e-13)
        np.testing.assert_allclose(dense.trace(T), 1.0, atol=1e-13)
    np.testing.assert_allclose(densemat.rho_to_vec(rho), T, atol=1e-13)


# ---------------------------------------------------------- pure states -----
def test_pure_state_doubling_mpo_and_dense():
    """p = 0: S_l(|psi><psi|) = 2 S_l(|psi>) (Sec. 3.3)."""
    c = random_circuit(8, 8, 0.0, seed=1)
    sv = statevec.run(c)
    m = mpo.run(c, 256, 1e-14)
    np.testing.assert_allclose(m.S, 2 * sv, atol=1e-10)
    c6 = random_circuit(6, 6, 0.0, seed=2)
    d = dense.run(c6, 64)
    np.testing.assert_allclose(d.S, 2 * statevec.run(c6), atol=1e-10)


def test_page_value_statevector_ensemble():
    """Noiseless n = 8 deep circuits: mean max entropy -> 6.56 (Sec. 4.1, Fig. 3).

    Uses the state-vector oracle, tied to the MPO oracle by the doubling test."""
    g = GOLD["page_smax_n8_p0"]
    finals = []
    for s in range(24):
        c = random_circuit(8, 40, 0.0, seed=s)
        S = 2 * statevec.run(c)
        finals.append(S[-10:].mean(axis=0))
    mean = np.mean(finals, axis=0)
    assert abs(mean.max() - g["value"]) < 0.05
    assert int(np.argmax(mean)) == 3          # the middle cut l = 4


# ------------------------------------------------------ special states ------
def test_ghz_has_entropy_two_at_every_cut():
    """GHZ_n (Sec. 3.2) prepared by H then a CNOT chain; S_l = 2 for all l."""
    n = 6
    H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    first = CNOT @ np.kron(H, np.eye(2))
    m = mpo.MPO(n, 64, 1e-14)
    T = dense.initial_vec(n)
    for l in range(1, n):
        U = first if l == 1 else CNOT
        M = channels.noisy_gate_superop(U, 0.0)
        m.apply_superop(M, l)
        T = dense.apply_superop(T, M, l)
    lams = m.sweep()
    for lam in lams:
        assert abs(mpo_entropy(lam) - GOLD["ghz_mpo_entropy"]["value"]) < 1e-12
    for l in range(1, n):
        assert abs(mpo_entropy(dense.schmidt_values(T, l)) - 2.0) < 1e-12


def test_classically_correlated_pair_has_entropy_one():
    """1/2 |00><00| + 1/2 |11><11| (Sec. 3.3, LOCC example) has S = 1."""
    H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    U = CNOT @ np.kron(H, np.eye(2))
    Z1 = np.kron(np.diag([1.0, -1.0]), np.eye(2))

    def chan(r):  # Bell preparation, then full dephasing of qubit 1 (an LOCC map)
        r = U @ r @ U.conj().T
        return 0.5 * r + 0.5 * Z1 @ r @ Z1

    M = channels.superop(chan)
    m = mpo.MPO(2, 16, 1e-14)
    m.apply_superop(M, 1)
    lam = m.sweep()[0]
    assert abs(mpo_entropy(lam) - GOLD["classical_pair_mpo_entropy"]["value"]) < 1e-12


def test_full_depolarisation_gives_zero_entropy_and_p1_does_not():
    """p = 15/16 maps every pair to I/4: after one odd step rho = I/2^n, S = 0 (Sec. 3.3)."""
    n = 6
    c = random_circuit(n, 1, 15 / 16, seed=3)
    m = mpo.run(c, 64, 1e-12)
    d = dense.run(c, 64)
    assert np.abs(m.S).max() < 1e-12 and np.abs(d.S).max() < 1e-12
    np.testing.assert_allclose(m.trace, 1.0, atol=1e-13)
    c1 = random_circuit(n, 1, 1.0, seed=3)
    S1 = mpo.run(c1, 64, 1e-12).S[0]
    assert S1[0] > 1e-2           # intra-pair cut: (1/15) sum P rho P is not I/4


def test_product_state_initial():
    m = mpo.MPO(8, 16)
    lams = m.sweep()
    assert all(mpo_entropy(lm) == 0.0 for lm in lams)
    assert abs(m.trace() - 1.0) < 1e-15


# ------------------------------------------------- truncation semantics -----
@pytest.mark.parametrize("chi,n", [(4, 8), (16, 8), (16, 10)])
def test_mpo_oracle_matches_dense_truncation(chi, n):
    """Two independent realisations of the truncated dynamics (global SVD of the
    dense |rho>> vs local mixed-canonical MPO update) agree."""
    c = random_circuit(n, 6, 0.05, seed=10 + chi)
    d = dense.run(c, chi, 1e-12)
    m = mpo.run(c, chi, 1e-12)
    np.testing.assert_allclose(m.S, d.S, atol=1e-9)
    np.testing.assert_allclose(m.trace, d.trace, atol=1e-10)
    for wd, wm in zip(d.discarded, m.discarded):
        np.testing.assert_allclose(wm, wd, atol=1e-10)
    assert sum(w.sum() for w in d.discarded) > 0   # the case really truncates
    np.testing.assert_allclose(m.mpo.to_dense(), d.final, atol=1e-10)


def test_exact_at_full_bond_dimension():
    """chi = 4^(n/2) represents any state exactly (Sec. 3.1): no discarded weight, Tr = 1."""
    c = random_circuit(8, 10, 0.02, seed=0)
    m = mpo.run(c, 256, 1e-14)
    assert max(w.max() for w in m.discarded) < 1e-20
    np.testing.assert_allclose(m.trace, 1.0, atol=1e-12)


def test_schmidt_weight_is_bond_invariant():
    """sum_a (lambda^[l]_a)^2 = <<rho|rho>> = Tr rho^2 at every bond l."""
    c = random_circuit(10, 6, 0.03, seed=4)
    m = mpo.run(c, 32, 1e-12, keep_schmidt=True)
    for lams in m.schmidt:
        w = [float((lm ** 2).sum()) for lm in lams]
        np.testing.assert_allclose(w, w[0], rtol=1e-11)
    for a in m.mpo.A[1:]:          # after the sweep every site but the first is a right isometry
        R = a.reshape(a.shape[0], -1)
        np.testing.assert_allclose(R @ R.conj().T, np.eye(a.shape[0]), atol=1e-12)


# ------------------------------------------------- paper statistics ---------
@pytest.mark.parametrize("key", ["fig5_p015", "fig5_p010"])
def test_peak_depth_and_height_fig5(key):
    """n = 8, N_s = 24: the mean maximum MPO entropy peaks at the printed D*
    with the printed S* (Sec. 4.1, Fig. 5); Tr rho stays above the printed band."""
    g = GOLD[key]
    n, D = 8, g["D_star"] + 3
    S, tr = [], []
    for s in range(24):
        r = mpo.run(random_circuit(n, D, g["p"], s), g["chi"], 1e-12)
        S.append(r.S)
        tr.append(r.trace.min())
    smax = np.mean(S, axis=0).max(axis=1)
    assert int(np.argmax(smax)) + 1 == g["D_star"]
    assert abs(smax.max() - g["S_star"]) < 0.2
    assert min(tr) >= g["trace_min"]


def test_ensemble_instances_recipe():
    """The batching workload's inputs: (n_i, p_i) from the stated choices,
    depth 2 n_i, brickwork gate counts per step, reproducible per seed, and
    instance i's gates equal to a single circuit drawn with seed 1000 + i."""
    from paper_2003_13163_gb300.circuits import ensemble_instances, n_gates
    a = ensemble_instances(12, seed=4)
    b = ensemble_instances(12, seed=4)
    assert [c.n for c in a] == [c.n for c in b]
    for i, c in enumerate(a):
        assert c.n in (16, 24, 32, 40, 48, 56, 64)
        assert float(c.p[0][0]) in (0.005, 0.01, 0.02, 0.05)
        assert c.depth == 2 * c.n
        assert [len(g) for g in c.gates[:2]] == [n_gates(c.n, 0), n_gates(c.n, 1)]
        ref = random_circuit(c.n, c.depth, float(c.p[0][0]), 1000 + i)
        assert np.array_equal(ref.gates[0], c.gates[0]) and np.array_equal(ref.gates[-1], c.gates[-1])
    assert len({c.n for c in ensemble_instances(64, seed=4)}) > 3      # the sizes are mixed


# ------------------------------------------------ Oracle V (App. A, literal) --
@pytest.mark.parametrize("n,chi,p,seed,depth", [(6, 64, 0.02, 31, 8), (8, 256, 0.05, 32, 8)])
def test_vidal_update_matches_dense_exact(n, chi, p, seed, depth):
    """App. A's global (Gamma, lambda) update and the dense route agree when
    nothing is truncated: every S_l after every step and the final |rho>>."""
    from oracle import vidal
    c = random_circuit(n, depth, p, seed=seed)
    v = vidal.run(c, chi)
    d = dense.run(c, chi)
    assert np.abs(v.S - d.S).max() < 1e-10
    assert np.abs(v.final.to_dense() - d.final).max() < 1e-12


@pytest.mark.parametrize("n,chi,p,seed,depth", [(8, 16, 0.05, 2, 6), (8, 4, 0.02, 5, 6), (10, 16, 0.05, 3, 4)])
def test_vidal_update_matches_dense_truncated(n, chi, p, seed, depth):
    """With truncation: App. A keeps the chi largest values at the gate's bond
    and only re-canonicalises elsewhere, so it reproduces the dense
    truncation, the discarded weights included (the equivalence of App. A and
    the local update of the Note added)."""
    from oracle import vidal
    c = random_circuit(n, depth, p, seed=seed)
    v = vidal.run(c, chi, 1e-10)
    d = dense.run(c, chi, 1e-10)
    assert sum(w.sum() for w in d.discarded) > 0.0
    assert np.abs(v.S - d.S).max() < 1e-9
    np.testing.assert_allclose(np.concatenate(v.discarded), np.concatenate(d.discarded), atol=1e-12)
    assert np.abs(v.final.to_dense() - d.final).max() < 1e-11


def test_vidal_lambdas_are_the_schmidt_values():
    """After every gate the lambda vectors App. A maintains are the exact
    operator-Schmidt values of |rho>> at every cut (the canonical form)."""
    from oracle import vidal
    c = random_circuit(8, 5, 0.03, seed=9)
    m = vidal.VidalMPO(8)
    for t in range(1, c.depth + 1):
        for U, p, l in zip(c.gates[t - 1], c.p[t - 1], layer_bonds(8, c.parity(t))):
            m.apply(l, channels.noisy_gate_superop(U, p), 256, 1e-12)
            T = m.to_dense()
            for b in range(1, 8):
                ref = dense.schmidt_values(T, b)
                k = len(m.lam[b])
                np.testing.assert_allclose(m.lam[b], ref[:k], atol=1e-11 * ref[0])
                assert ref[k:].sum() < 1e-9 * ref[0] if k < len(ref) else True
