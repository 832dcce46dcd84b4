"""Host logic of bench.py (no GPU): the gate schedule a timed step walks and
the algorithmic work the roofline divides by."""
import numpy as np

import bench
from paper_2003_13163_gb300.circuits import layer_bonds, random_circuit


def test_gate_schedule_walks_the_brickwork_in_order():
    n = 8
    c = random_circuit(n, 6, 0.01, seed=1)
    sched = bench.gate_schedule(c, n, 2, 10)
    assert len(sched) == 10
    expect = []
    for t in range(2, 7):
        bonds = layer_bonds(n, c.parity(t))                  # paper bonds, ascending
        for g, l in enumerate(bonds):
            expect.append((t, g, l - 1, g == len(bonds) - 1))
    assert sched == expect[:10]
    # every step end is flagged once, on the step's last gate
    assert [e for e in sched if e[3]] == [e for e in expect[:10] if e[3]]


def test_gate_work_closed_forms_at_a_saturated_bond():
    chi, n = 1024, 64
    dims = np.array([1] + [chi] * (n - 1) + [1])
    x = 4 * chi
    # theta (4chi x chi)(chi x 4chi), superoperator, Gram 4 x^3, projection
    # 8 chi x^2, centre move 12 chi^2 (4 chi)
    gemm = 8 * x * x * chi + 2048 * chi * chi + 4 * x ** 3 + 8 * chi * x * x + 48 * chi ** 3
    w = bench.gate_work(dims, 20, chi, "mixed")
    assert w["gemm"] == gemm
    assert np.isclose(w["solve"], 13.3 * (chi + bench.MIXED_MARGIN) ** 3)
    assert w["bytes"] == 2 * (chi * 4 * chi * 2) * 16
    assert np.isclose(bench.gate_work(dims, 20, chi, "fp64")["solve"], 13.3 * x ** 3)
    assert bench.gate_work(dims, 20, chi, "fp32")["bytes"] == w["bytes"] / 2


def test_sweep_work_counts_the_recorded_bonds():
    dims = np.array([1, 4, 16, 16, 4, 1])
    centre = bench.sweep_work(dims, 5, True)
    r, c = dims[2], 4 * dims[3]
    assert centre["gemm"] == 12 * r * r * c and np.isclose(centre["solve"], 13.3 * r ** 3)
    full = bench.sweep_work(dims, 5, False)
    assert full["gemm"] == sum(12 * dims[b] ** 2 * 4 * dims[b + 1] for b in range(1, 5))
