"""Single-kernel cases for profiler captures (ncu) of the engine's kernels.

    python -m paper_2003_13163_gb300.profile_cases svd R C fp32|fp64 REPS [block|rows]
    python -m paper_2003_13163_gb300.profile_cases gemm M N K REPS [tc|simt]

`svd` factorises a seeded R x C complex matrix with a flat spectrum (the shape
of a centre move at chi = C/4, or of a gate SVD when R = C) through mpo_svd;
`gemm` runs the FP32 complex product through mpo_gemm. Each repetition prints
its wall time. Small shapes keep a profiler capture short.
"""
from __future__ import annotations

import sys
import time


def main(argv):
    import numpy as np
    import torch

    from . import build as B
    from . import mpo
    from .circuits import random_complex

    B.build()
    what = argv[0]
    if what == "svd":
        r, c, prec, reps = int(argv[1]), int(argv[2]), argv[3], int(argv[4])
        block = (argv[5] if len(argv) > 5 else "block") == "block"
        dt = torch.complex64 if prec == "fp32" else torch.complex128
        k = min(r, c)
        U = np.linalg.qr(random_complex((r, k), seed=1))[0]
        Vh = np.linalg.qr(random_complex((c, k), seed=2))[0].conj().T
        X0 = torch.tensor((U * np.linspace(1, 0.05, k)[None, :]) @ Vh, dtype=dt, device="cuda")
        for _ in range(reps):
            X = X0.clone()
            torch.cuda.synchronize()
            t = time.time()
            mpo.svd_rows(X, prec, block=block)
            torch.cuda.synchronize()
            el = time.time() - t
            st = mpo.svd_last_stats()
            print(f"svd {prec} {r}x{c} block={block}: {el:.4f} s, {st['sweeps']} sweeps, phases G/E/A "
                  f"{st['gram_ms']:.1f}/{st['pair_eig_ms']:.1f}/{st['apply_ms']:.1f} ms", flush=True)
    elif what == "gemm":
        m, n, kk, reps = int(argv[1]), int(argv[2]), int(argv[3]), int(argv[4])
        tc = (argv[5] if len(argv) > 5 else "tc") == "tc"
        A = torch.tensor(random_complex((m, kk), seed=3), dtype=torch.complex64, device="cuda")
        Bm = torch.tensor(random_complex((kk, n), seed=4), dtype=torch.complex64, device="cuda")
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.time()
            mpo.gemm(A, Bm, "fp32", tensor_cores=tc)
            torch.cuda.synchronize()
            dt_ = time.time() - t
            print(f"gemm {m}x{n}x{kk} tc={tc}: {dt_ * 1e3:.3f} ms, {8.0 * m * n * kk / dt_ / 1e12:.2f} TFLOP/s", flush=True)
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv[1:])
