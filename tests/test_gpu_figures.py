"""Paper statistics reproduced by the GPU engine through the batching form:
ensembles of seeded circuits (N_s = 24, Sec. 4.1) run as one batch, against
the values printed in the paper (tests/golden/paper_values.json).

- Fig. 5, p = 0.1 (chi = 150) and p = 0.15 (chi = 80): the mean maximum MPO
  entropy over the circuits peaks at the printed depth D* with the printed
  height S*, and the trace stays above the printed band (Sec. 4.1).
- Fig. 3: noiseless n = 8 deep circuits, the maximum MPO entropy approaches
  twice the Page value, 6.56, at the middle cut (Sec. 4.1).
"""
import json
import os

import numpy as np
import pytest

from paper_2003_13163_gb300.circuits import random_circuit
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.fixture(scope="module")
def M():
    return need_gpu()


def run_ensemble(M, circs, chi, precision):
    """Every circuit stepped together through one batch; returns the
    entropies (circuits x steps x bonds) and the traces (circuits x steps)."""
    b = M.MPOBatch([c.n for c in circs], chi, precision, workers=8)
    p = np.array([float(c.p[0][0]) for c in circs])
    S, tr = [], []
    for t in range(1, circs[0].depth + 1):
        s, trace, _ = b.apply_layer(t, [c.gates[t - 1] for c in circs], p)
        S.append(np.array(s))
        tr.append(trace)
    b.close()
    return np.transpose(np.array(S), (1, 0, 2)), np.array(tr).T


@pytest.mark.parametrize("key,precision", [("fig5_p010", "fp64"), ("fig5_p010", "mixed"), ("fig5_p015", "mixed")])
def test_fig5_peak_depth_and_height(M, key, precision):
    g = GOLD[key]
    circs = [random_circuit(8, g["D_star"] + 3, g["p"], s) for s in range(24)]
    S, tr = run_ensemble(M, circs, g["chi"], precision)
    smax = S.mean(axis=0).max(axis=1)
    assert int(np.argmax(smax)) + 1 == g["D_star"]
    assert abs(smax.max() - g["S_star"]) < 0.2
    assert tr.min() >= g["trace_min"]


def test_fig3_page_limit(M):
    g = GOLD["page_smax_n8_p0"]
    circs = [random_circuit(8, 30, 0.0, s) for s in range(12)]
    S, _ = run_ensemble(M, circs, g["chi"], "fp64")
    late = S[:, -8:, :].mean(axis=(0, 1))            # mean over circuits and the last 8 steps
    assert int(np.argmax(late)) == 3                 # the middle cut
    assert abs(late.max() - g["value"]) < 0.1
