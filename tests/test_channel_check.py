"""mpo_check_superop, the host-side validation mpo_apply_superop applies to a
caller's map (Sec. 2.2: the method takes any two-qubit error model, which
must be a quantum channel): trace preservation and complete positivity,
checked against maps whose properties are known in closed form."""
import numpy as np
import pytest

from oracle import channels
from paper_2003_13163_gb300 import build as B
from paper_2003_13163_gb300 import mpo
from paper_2003_13163_gb300.circuits import haar_unitary


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


@pytest.mark.parametrize("p", [0.0, 0.013, 0.4, 15 / 16, 1.0])
def test_noisy_gates_are_channels(p):
    rng = np.random.Generator(np.random.PCG64(3))
    ok, defect = mpo.check_superop(channels.noisy_gate_superop(haar_unitary(rng), p))
    assert ok and defect < 1e-12


def test_dephasing_and_amplitude_damping_are_channels():
    Z1 = np.kron(np.diag([1.0, -1.0]), np.eye(2))
    ok, _ = mpo.check_superop(channels.superop(lambda r: 0.8 * r + 0.2 * Z1 @ r @ Z1))
    assert ok
    g = 0.3                                   # amplitude damping on the second qubit
    K0 = np.kron(np.eye(2), np.array([[1, 0], [0, np.sqrt(1 - g)]]))
    K1 = np.kron(np.eye(2), np.array([[0, np.sqrt(g)], [0, 0]]))
    ok, _ = mpo.check_superop(channels.superop(lambda r: K0 @ r @ K0.conj().T + K1 @ r @ K1.conj().T))
    assert ok


def test_trace_decreasing_map_is_rejected():
    ok, defect = mpo.check_superop(0.5 * channels.superop(lambda r: r))
    assert not ok and abs(defect - 0.5) < 1e-12


def test_partial_transpose_is_rejected():
    """The partial transpose on one qubit preserves the trace but is not
    completely positive: its Choi matrix is a swap with eigenvalue -1."""
    def pt(r):
        t = r.reshape(2, 2, 2, 2)                         # (a, b, a', b')
        return t.transpose(2, 1, 0, 3).reshape(4, 4)      # transpose qubit l
    M = channels.superop(pt)
    ok, defect = mpo.check_superop(M)
    assert not ok and defect > 0.5


def test_tolerance_scales_with_the_map():
    rng = np.random.Generator(np.random.PCG64(5))
    M = channels.noisy_gate_superop(haar_unitary(rng), 0.02)
    E = np.zeros_like(M)
    E[0, 0] = 1e-6                               # breaks trace preservation by 1e-6
    assert mpo.check_superop(M + E, tol=1e-5)[0]
    assert not mpo.check_superop(M + E, tol=1e-8)[0]
