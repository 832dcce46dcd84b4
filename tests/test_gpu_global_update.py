"""App. A's global update on the GPU: after every gate the whole chain is
re-canonicalised (a sweep of factorisations over every bond, O(n) per gate,
as App. A's left and right sweeps are), through mpo_apply_gate + mpo_sweep,
against Oracle V, which implements App. A literally in the (Gamma, lambda)
form: S_l at every cut after every gate."""
import numpy as np
import pytest

from oracle import vidal
from oracle.channels import noisy_gate_superop
from paper_2003_13163_gb300.circuits import layer_bonds, random_circuit
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    return need_gpu()


@pytest.mark.parametrize("n,chi,p,seed,depth", [(8, 256, 0.01, 3, 4), (8, 16, 0.01, 4, 5), (10, 16, 0.02, 5, 4)])
def test_global_update_matches_oracle_v_after_every_gate(M, n, chi, p, seed, depth):
    c = random_circuit(n, depth, p, seed)
    m = M.MPO(n, chi, "fp64")
    v = vidal.VidalMPO(n)
    worst = 0.0
    for t in range(1, depth + 1):
        for U, pp, l in zip(c.gates[t - 1], c.p[t - 1], layer_bonds(n, c.parity(t))):
            m.apply_gate(l - 1, U, float(pp))
            m.sweep()
            S, _, _ = m.entropy(with_trace=False)
            v.apply(l, noisy_gate_superop(U, pp), chi, 1e-12)
            worst = max(worst, float(np.abs(S - np.array(v.entropies())).max()))
    m.close()
    assert worst < 1e-9, worst
