"""Oracle M: the MPO of Sec. 3.1 in mixed canonical form, updated gate by gate.

Oracle code: test infrastructure only, see ``oracle/__init__.py``.

Site k (0-based) holds A[k] with shape (chi_k, 4, chi_{k+1}), chi_0 = chi_n = 1,
index order [alpha_left, I, alpha_right] with I = 2 i + i' (Sec. 3.1). Bond b
(1 <= b <= n-1) sits between sites b-1 and b and is the paper's cut
[1..b]:[(b+1)..n].

Update scheme (Note added: move the orthogonality centre by a local
factorisation, then apply the gate and truncate locally), which in exact
arithmetic reproduces App. A's canonical update:
  * sites left of the centre are left isometries, sites right of it right
    isometries; the centre carries the whole norm (no renormalisation);
  * centre moves factorise one site with numpy's SVD (LAPACK gesdd), so the
    Schmidt values at the crossed bond are visible and the same drop rule
    (lambda <= cutoff * lambda_max) applies at every factorisation;
  * gate on paper bond l (sites i = l-1, i+1): theta = A[i] A[i+1]
    contracted over the shared bond, theta' = M theta on (I_l, I_{l+1}), SVD of
    theta' as a (chi_i*4) x (4*chi_{i+2}) matrix, keep the chi_max largest
    Schmidt values (App. A), left factor -> A[i], S V^dagger -> A[i+1];
  * after every step a right-to-left sweep of SVDs yields lambda^[b] at every
    bond (the Schmidt values S_l of Sec. 3.3 are defined on) and leaves the
    MPO with the centre at site 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .channels import noisy_gate_superop
from .entropy import mpo_entropy


def _keep(s: np.ndarray, cap: int, cutoff: float) -> int:
    if s.size == 0 or s[0] <= 0.0:
        return 1
    return max(1, int(min(cap, np.count_nonzero(s > cutoff * s[0]))))


class MPO:
    def __init__(self, n: int, chi_max: int, cutoff: float = 0.0):
        if n < 2 or n % 2:
            raise ValueError("n must be even and >= 2")
        self.n, self.chi_max, self.cutoff = n, chi_max, cutoff
        # |0..0><0..0|: every site one-hot at I = 0 with bond dimension 1 (Sec. 4.1;
        # the paper pads the bonds to chi with zero singular values, which is the
        # same state).
        self.A = []
        for _ in range(n):
            a = np.zeros((1, 4, 1), dtype=np.complex128)
            a[0, 0, 0] = 1.0
            self.A.append(a)
        self.centre = 0

    # -- factorisations -------------------------------------------------
    def _move_right(self, k: int) -> np.ndarray:
        """Make site k a left isometry; push the rest into site k+1. Returns
        the singular values at bond k+1."""
        a = self.A[k]
        cl, _, cr = a.shape
        U, s, Vh = np.linalg.svd(a.reshape(cl * 4, cr), full_matrices=False)
        r = _keep(s, s.size, self.cutoff)
        self.A[k] = U[:, :r].reshape(cl, 4, r)
        self.A[k + 1] = np.tensordot(s[:r, None] * Vh[:r], self.A[k + 1], axes=(1, 0))
        return s

    def _move_left(self, k: int) -> np.ndarray:
        """Make site k a right isometry; push the rest into site k-1. Returns
        the singular values at bond k."""
        a = self.A[k]
        cl, _, cr = a.shape
        U, s, Vh = np.linalg.svd(a.reshape(cl, 4 * cr), full_matrices=False)
        r = _keep(s, s.size, self.cutoff)
        self.A[k] = Vh[:r].reshape(r, 4, cr)
        self.A[k - 1] = np.tensordot(self.A[k - 1], U[:, :r] * s[None, :r], axes=(2, 0))
        return s

    def move_centre(self, target: int) -> None:
        while self.centre < target:
            self._move_right(self.centre)
            self.centre += 1
        while self.centre > target:
            self._move_left(self.centre)
            self.centre -= 1

    # -- the noisy gate (App. A, with the local update of the Note added) --
    def apply_superop(self, M: np.ndarray, l: int) -> float:
        """Apply a 16x16 superoperator on paper bond l; returns the discarded
        weight sum_{beta >= kept} lambda'^2 / sum_beta lambda'^2."""
        i = l - 1
        if self.centre < i:
            self.move_centre(i)
        elif self.centre > i + 1:
            self.move_centre(i + 1)
        a, b = self.A[i], self.A[i + 1]
        cl, cr = a.shape[0], b.shape[2]
        theta = np.tensordot(a, b, axes=(2, 0))                 # [a, I, J, c]
        Mt = M.reshape(4, 4, 4, 4)                              # [I', J', I, J]
        thetap = np.einsum("xyij,aijc->axyc", Mt, theta)
        U, s, Vh = np.linalg.svd(thetap.reshape(cl * 4, 4 * cr), full_matrices=False)
        k = _keep(s, self.chi_max, self.cutoff)
        tot = float((s * s).sum())
        w = float((s[k:] ** 2).sum() / tot) if tot > 0 else 0.0
        self.A[i] = U[:, :k].reshape(cl, 4, k)
        self.A[i + 1] = (s[:k, None] * Vh[:k]).reshape(k, 4, cr)
        self.centre = i + 1
        return w

    def sweep(self) -> list:
        """Right-to-left Schmidt sweep. Returns lambda^[b] for b = 1..n-1."""
        self.move_centre(self.n - 1)
        lams = [None] * (self.n - 1)
        for k in range(self.n - 1, 0, -1):
            s = self._move_left(k)
            lams[k - 1] = s
            self.centre = k - 1
        return lams

    # -- observables ----------------------------------------------------
    def trace(self) -> complex:
        """Tr rho by contracting every site with the trace vector (Sec. 3.4)."""
        v = np.ones(1, dtype=np.complex128)
        for a in self.A:
            v = v @ (a[:, 0, :] + a[:, 3, :])
        return complex(v[0])

    def to_dense(self) -> np.ndarray:
        T = self.A[0]
        for a in self.A[1:]:
            T = np.tensordot(T, a, axes=(T.ndim - 1, 0))
        return T.reshape((4,) * self.n)

    def bond_dims(self) -> list:
        return [a.shape[2] for a in self.A[:-1]]


@dataclass
class MPOResult:
    S: np.ndarray
    trace: np.ndarray
    discarded: list = field(default_factory=list)
    schmidt: list = field(default_factory=list)
    bond_dims: list = field(default_factory=list)
    mpo: MPO = None


def run(circuit, chi_max: int, cutoff: float = 0.0, keep_schmidt: bool = False,
        steps: int | None = None) -> MPOResult:
    """Run the first ``steps`` (default: all) time steps of a circuit; record
    S_l at every bond, Tr rho and per-gate discarded weights after every step
    (Sec. 4.1)."""
    from paper_2003_13163_gb300.circuits import layer_bonds

    n = circuit.n
    mpo = MPO(n, chi_max, cutoff)
    S_rows, tr, disc, sch, dims = [], [], [], [], []
    depth = circuit.depth if steps is None else steps
    for t in range(1, depth + 1):
        ws = []
        for U, p, l in zip(circuit.gates[t - 1], circuit.p[t - 1], layer_bonds(n, circuit.parity(t))):
            ws.append(mpo.apply_superop(noisy_gate_superop(U, p), l))
        lams = mpo.sweep()
        S_rows.append([mpo_entropy(lm) for lm in lams])
        tr.append(mpo.trace().real)
        disc.append(np.array(ws))
        dims.append(mpo.bond_dims())
        if keep_schmidt:
            sch.append(lams)
    return MPOResult(S=np.array(S_rows), trace=np.array(tr), discarded=disc, schmidt=sch,
                     bond_dims=dims, mpo=mpo)
