"""The batching form (mpo_init_batch / mpo_apply_layer_batch): k independent
circuits advanced together on worker threads and streams.

Every instance must produce exactly what the same circuit gives through the
single-instance calls (the batch changes only where the work runs, never its
arithmetic), and the FP64 batch must match the dense oracle to 1e-10.
"""
import numpy as np
import pytest

from oracle import dense
from paper_2003_13163_gb300.circuits import ensemble_instances, random_circuit
from tests.gpu_util import need_gpu, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    return need_gpu()


def _run_batch(M, circuits, chi, precision, workers, active_of=None, cutoff=0.0):
    """Advance the circuits as one batch up to the deepest; instance i takes
    part in step t when t <= its depth and active_of(i, t) (default True)."""
    b = M.MPOBatch([c.n for c in circuits], chi, precision, workers=workers, cutoff=cutoff)
    D = max(c.depth for c in circuits)
    S = [[] for _ in circuits]
    tr = [[] for _ in circuits]
    dw = [[] for _ in circuits]
    for t in range(1, D + 1):
        act = [int(t <= c.depth and (active_of is None or active_of(i, t))) for i, c in enumerate(circuits)]
        gates = [c.gates[t - 1] for i, c in enumerate(circuits) if act[i]]
        p = [float(c.p[t - 1][0]) if t <= c.depth and len(c.p[t - 1]) else 0.0 for c in circuits]
        s, trace, d = b.apply_layer(t, gates, p, act)
        for i in range(len(circuits)):
            if act[i]:
                S[i].append(s[i].copy())
                tr[i].append(trace[i])
                dw[i].append(d[i])
    return b, [np.array(x) for x in S], [np.array(x) for x in tr], [np.array(x) for x in dw]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_equals_single_instances(M, precision):
    circuits = [random_circuit(n, d, p, seed=s)
                for n, d, p, s in [(8, 6, 0.02, 11), (10, 5, 0.05, 12), (6, 7, 0.01, 13), (12, 4, 0.02, 14)]]
    chi = 16
    b, S, tr, dw = _run_batch(M, circuits, chi, precision, workers=3)
    for i, c in enumerate(circuits):
        S1, tr1, dw1, m = run_gpu(M, c, chi, precision)
        assert np.array_equal(S[i], S1), f"instance {i}"
        assert np.array_equal(tr[i], tr1), f"instance {i}"
        assert np.array_equal(dw[i], dw1), f"instance {i}"
        assert list(b.instance(i).bond_dims()) == list(m.bond_dims())
        m.close()
    b.close()


def test_batch_inactive_instances_are_left_alone(M):
    """An instance that sits out step 3 equals the single-instance run of its
    circuit without that step's gates (the later steps keep their parity)."""
    circuits = [random_circuit(8, 6, 0.02, seed=21), random_circuit(8, 6, 0.03, seed=22)]
    skip = lambda i, t: not (i == 1 and t == 3)
    b, S, tr, dw = _run_batch(M, circuits, 16, "fp64", workers=2, active_of=skip)
    c = circuits[1]
    m = M.MPO(c.n, 16, "fp64")
    ref = []
    for t in range(1, c.depth + 1):
        if t == 3:
            continue
        m.apply_layer(c.parity(t), c.gates[t - 1], c.p[t - 1])
        ref.append(m.entropy()[0])
    assert len(S[1]) == c.depth - 1
    assert np.array_equal(S[1], np.array(ref))
    m.close()
    b.close()


def test_batch_fp64_matches_dense_oracle(M):
    """Exact (untruncated) instances of different sizes against oracle D."""
    circuits = [random_circuit(n, d, p, seed=s) for n, d, p, s in [(6, 8, 0.02, 31), (8, 10, 0.05, 32),
                                                                  (4, 6, 0.1, 33)]]
    b, S, tr, dw = _run_batch(M, circuits, 256, "fp64", workers=3)
    for i, c in enumerate(circuits):
        d = dense.run(c, 256)
        assert np.abs(S[i] - d.S).max() < 1e-10, f"instance {i}"
        np.testing.assert_allclose(tr[i], d.trace, atol=1e-12)
    b.close()


def test_batch_truncated_matches_dense_oracle(M):
    circuits = [random_circuit(8, 8, 0.02, seed=41), random_circuit(10, 8, 0.05, seed=42)]
    b, S, tr, dw = _run_batch(M, circuits, 16, "fp64", workers=2, cutoff=1e-7)
    for i, c in enumerate(circuits):
        d = dense.run(c, 16, 1e-7)
        assert np.abs(S[i] - d.S).max() < 1e-9, f"instance {i}"
        assert dw[i].sum() > 0.0
    b.close()


def test_batch_worker_count_does_not_change_results(M):
    circuits = ensemble_instances(6, seed=4, n_choices=(6, 8, 10), depth_per_qubit=1)
    _, S1, tr1, _ = _run_batch(M, circuits, 32, "fp32", workers=1)
    _, S4, tr4, _ = _run_batch(M, circuits, 32, "fp32", workers=4)
    for i in range(len(circuits)):
        assert np.array_equal(S1[i], S4[i])
        assert np.array_equal(tr1[i], tr4[i])


def test_batch_rejects_single_instance_calls(M):
    import ctypes
    b = M.MPOBatch([6, 8], 8, "fp64", workers=2)
    S = np.zeros(8)
    assert b._lib.mpo_entropy(b.h, S.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, None) == -1
    assert b"batch" in b._lib.mpo_last_error(b.h)
    b.close()


def test_batch_many_mixed_instances_threads(M):
    """Many instances of different sizes (so their kernels ask for different
    launch resources) on eight worker threads give the one-thread results."""
    circuits = [random_circuit(n, 4, 0.02, seed=50 + i) for i, n in enumerate([4, 6, 8, 10, 12, 14, 16] * 4)]
    _, S1, tr1, _ = _run_batch(M, circuits, 32, "fp32", workers=1)
    _, S8, tr8, _ = _run_batch(M, circuits, 32, "fp32", workers=8)
    for i in range(len(circuits)):
        assert np.array_equal(S1[i], S8[i]), f"instance {i}"
        assert np.array_equal(tr1[i], tr8[i]), f"instance {i}"
