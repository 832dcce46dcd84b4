"""Oracle V: the canonical (Gamma, lambda) update of App. A, literally.

Oracle code: test infrastructure only, see ``oracle/__init__.py``.

This is the paper's own update scheme, kept as a third, independent route to
the same truncated dynamics as Oracle D (dense) and Oracle M (mixed-canonical
QR/TEBD, the scheme of the Note added). The state is held in the form of
Sec. 3.1 / App. A:

    |rho>> = sum Gamma[1]^{I_1} lambda[1] Gamma[2]^{I_2} lambda[2] ... Gamma[n]^{I_n}

with Gamma[k] of shape (chi_{k-1}, 4, chi_k) (index order [alpha_{k-1}, I_k,
alpha_k], I = 2 i + i') and lambda[b] the operator-Schmidt values across the
cut [1..b]:[(b+1)..n] (lambda[0] = lambda[n] = [1]). Nothing is renormalised.

A gate on paper bond l (sites l, l+1, 1-based) follows App. A step by step:
  1. B = M . (lambda[l-1] Gamma[l] lambda[l] Gamma[l+1] lambda[l+1]), the
     16 x 16 superoperator acting on (I_l, I_{l+1}), as a matrix with rows
     (alpha_{l-1}, I_l) and columns (I_{l+1}, alpha_{l+1});
  2. SVD B = V diag(lambda') W; keep the chi_max largest values (and, of
     those, the ones above cutoff * lambda'_max): lambda[l] <- lambda';
  3. global update to the left: B_left = V lambda' as a matrix
     alpha_{l-1} x (I_l, alpha_l); its SVD V1 lambda'' W1 gives the new
     Schmidt values at bond l-1 and Gamma[l] <- W1 / lambda[l] (divided on
     its right index); the next B_left is lambda[l-2] Gamma[l-1] V1 lambda'',
     and so on down to site 1, where Gamma[1] <- Gamma[1] V1;
  4. global update to the right, the mirror image: B_right = lambda' W as a
     matrix (alpha_l, I_{l+1}) x alpha_{l+1}; its SVD V2 lambda'' W2 gives
     Gamma[l+1] <- V2 / lambda[l] (divided on its left index) and the new
     values at bond l+1, and so on up to site n, where Gamma[n] <- W2 Gamma[n].

The divisions by lambda are the paper's; they lose precision when a kept
value is tiny, so this oracle is for untruncated or mildly truncated cases.
Values below cutoff * max in the sweep factorisations are rank-zero
directions (those matrices have at most chi_{k-1} rows) and are dropped.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .channels import noisy_gate_superop
from .entropy import mpo_entropy


def _keep(s: np.ndarray, cap: int, cutoff: float) -> int:
    if s.size == 0 or s[0] == 0.0:
        return 1
    return max(1, int(min(cap, np.count_nonzero(s > cutoff * s[0]))))


class VidalMPO:
    """Gamma / lambda form of |rho>> (App. A) for n sites."""

    def __init__(self, n: int):
        self.n = n
        g = np.zeros((1, 4, 1), dtype=np.complex128)
        g[0, 0, 0] = 1.0                               # |0><0| at every site: I = 0
        self.G = [g.copy() for _ in range(n)]          # Gamma[k], k = 0 .. n-1 (site k+1)
        self.lam = [np.ones(1) for _ in range(n + 1)]  # lam[b]: cut after site b (0 and n trivial)

    def apply(self, l: int, M: np.ndarray, chi_max: int, cutoff: float) -> float:
        """App. A update for the 16x16 superoperator M on paper bond l.
        Returns the discarded weight sum_{dropped} lambda'^2 / sum lambda'^2."""
        n, G, lam = self.n, self.G, self.lam
        a, b = l - 1, l                                # 0-based sites l, l+1
        T = np.einsum("x,xiy,y,yjz,z->xijz", lam[a], G[a], lam[a + 1], G[b], lam[b + 1])
        T = np.einsum("pqij,xijz->xpqz", M.reshape(4, 4, 4, 4), T)
        cl, cr = T.shape[0], T.shape[3]
        V, s, W = np.linalg.svd(T.reshape(cl * 4, 4 * cr), full_matrices=False)
        k = _keep(s, chi_max, cutoff)
        tot = float((s * s).sum())
        disc = float((s[k:] ** 2).sum() / tot) if tot > 0 else 0.0
        V, s, W = V[:, :k], s[:k], W[:k]
        lam[b] = s.copy()

        # left: B_left[alpha_{l-1}, (I_l, alpha_l)] = V[(alpha_{l-1}, I_l), alpha_l] s[alpha_l]
        Bl = (V * s[None, :]).reshape(cl, 4 * k)
        right_lam = s
        for site in range(a, 0, -1):
            V1, s1, W1 = np.linalg.svd(Bl, full_matrices=False)
            k1 = _keep(s1, chi_max, cutoff)
            V1, s1, W1 = V1[:, :k1], s1[:k1], W1[:k1]
            G[site] = W1.reshape(k1, 4, -1) / right_lam[None, None, :]
            lam[site] = s1.copy()
            # next: lambda[site-1] Gamma[site-1] V1 lambda''
            Bl = np.einsum("x,xiy,yz,z->xiz", lam[site - 1], G[site - 1], V1, s1).reshape(G[site - 1].shape[0], -1)
            right_lam = s1
        # site 1 (no bond to its left): Gamma[1] <- Gamma[1] V1, i.e. B_left / lambda''
        G[0] = Bl.reshape(1, 4, -1) / right_lam[None, None, :]

        # right: B_right[(alpha_l, I_{l+1}), alpha_{l+1}] = s[alpha_l] W[alpha_l, (I_{l+1}, alpha_{l+1})]
        Br = (s[:, None] * W).reshape(k * 4, cr)
        left_lam = s
        for site in range(b, n - 1):
            V2, s2, W2 = np.linalg.svd(Br, full_matrices=False)
            k2 = _keep(s2, chi_max, cutoff)
            V2, s2, W2 = V2[:, :k2], s2[:k2], W2[:k2]
            G[site] = V2.reshape(-1, 4, k2) / left_lam[:, None, None]
            lam[site + 1] = s2.copy()
            # next: lambda'' W2 Gamma[site+1] lambda[site+2]
            Br = np.einsum("x,xy,yiz,z->xiz", s2, W2, G[site + 1], lam[site + 2]).reshape(-1, G[site + 1].shape[2])
            left_lam = s2
        # site n (no bond to its right): Gamma[n] <- W2 Gamma[n], i.e. B_right / lambda''
        G[n - 1] = Br.reshape(-1, 4, 1) / left_lam[:, None, None]
        return disc

    def to_dense(self) -> np.ndarray:
        """Contract Gamma[1] lambda[1] ... Gamma[n] into the 4^n tensor |rho>>."""
        out = self.G[0].reshape(4, -1)
        for k in range(1, self.n):
            out = (out * self.lam[k][None, :]) @ self.G[k].reshape(self.G[k].shape[0], -1)
            out = out.reshape(-1, self.G[k].shape[2])
        return out.reshape((4,) * self.n)

    def entropies(self) -> list:
        """S_l (Sec. 3.3) from lambda[l], l = 1 .. n-1."""
        return [mpo_entropy(self.lam[b]) for b in range(1, self.n)]


@dataclass
class VidalResult:
    S: np.ndarray
    discarded: list = field(default_factory=list)
    final: VidalMPO = None


def run(circuit, chi_max: int, cutoff: float = 1e-12) -> VidalResult:
    """The circuit in order (step t ascending, bond ascending within a step,
    Sec. 4.1), S_l at every cut after every step."""
    from paper_2003_13163_gb300.circuits import layer_bonds

    m = VidalMPO(circuit.n)
    S_rows, disc = [], []
    for t in range(1, circuit.depth + 1):
        ws = [m.apply(l, noisy_gate_superop(U, p), chi_max, cutoff)
              for U, p, l in zip(circuit.gates[t - 1], circuit.p[t - 1], layer_bonds(circuit.n, circuit.parity(t)))]
        S_rows.append(m.entropies())
        disc.append(np.array(ws))
    return VidalResult(S=np.array(S_rows), discarded=disc, final=m)
