"""Plain FP64 CPU oracle for the noisy-MPO simulation of arXiv:2003.13163.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it. It shares no code with the
CUDA library; its only common input is the seeded gate stream of
``paper_2003_13163_gb300.circuits`` (random numbers, no method arithmetic).

Modules (each function cites the passage it follows):
  channels  - Pauli-sum depolarising channel (Sec. 2.2) and the 16x16
              superoperator of a noisy gate (App. A definition of M).
  densemat  - 2^n x 2^n density-matrix simulator (Sec. 2.1-2.2), n <= 8.
  dense     - Oracle D: vectorised |rho>> as a 4^n tensor (Sec. 3.1), exact
              per-gate truncation by the operator-Schmidt decomposition across
              the gate's cut (App. A, bulk case), entropies at every cut.
  statevec  - pure-state simulator for the p = 0 identity of Sec. 3.3.
  mpo       - Oracle M: the MPO in mixed canonical form updated gate by gate
              with QR/SVD centre moves and local truncation (Note added), plus
              the end-of-step Schmidt sweep giving lambda at every bond.
  vidal     - Oracle V: App. A's canonical (Gamma, lambda) update taken
              literally, with its global left and right re-factorisation after
              every gate and the divisions by lambda; a third route to the
              same truncated dynamics, for untruncated or mildly truncated
              cases.
  entropy   - MPO entanglement entropy (Sec. 3.3) and Page's mean entropy.

Parity status: every function is pinned by a ``-m "not gpu"`` test against
closed forms, paper-printed values or an independent second formulation;
none is "parity unpinned".
"""
