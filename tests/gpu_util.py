"""Helpers shared by the GPU tests: build/load the library, skip without a GPU."""
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_13163_gb300 import build as B
    B.build()
    from paper_2003_13163_gb300 import mpo
    mpo.load_library()
    return mpo


def run_gpu(mpo_mod, circuit, chi, precision="fp64", cutoff=0.0, steps=None, **kw):
    """Run a circuit through the C ABI; returns (S (D, n-1), trace (D,), disc (D,), handle)."""
    import numpy as np
    m = mpo_mod.MPO(circuit.n, chi, precision, cutoff=cutoff, **kw)
    S, tr, dw = [], [], []
    D = circuit.depth if steps is None else steps
    for t in range(1, D + 1):
        m.apply_layer(circuit.parity(t), circuit.gates[t - 1], circuit.p[t - 1])
        s, trace, d = m.entropy()
        S.append(s)
        tr.append(trace)
        dw.append(d)
    return np.array(S), np.array(tr), np.array(dw), m
