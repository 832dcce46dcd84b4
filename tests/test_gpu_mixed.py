"""The precision form (MPO_MIXED_FP32) against the FP64 form and the oracles.

Targets: |dS| <= 1e-6 against the FP64 form on the same seed, at every bond
and step, and a relative Frobenius error of the kept theta <= 1e-7 per gate
on an identical FP64 input (the one-step error). The inputs theta' are taken
from Oracle M trajectories of the paper's workload (Haar brickwork with
two-qubit depolarising noise, Sec. 4.1) at the point where the bond
dimensions sit at chi_max, so every truncation bites.
"""
import numpy as np
import pytest

from oracle import dense, mpo as ompo
from oracle.channels import noisy_gate_superop
from paper_2003_13163_gb300.circuits import layer_bonds, random_circuit, random_complex
from tests.gpu_util import need_gpu, run_gpu

pytestmark = pytest.mark.gpu

KEPT_TOL = 1e-7
DS_TOL = 1e-6


@pytest.fixture(scope="module")
def M():
    return need_gpu()


def oracle_thetas(n, chi, p, seed, depth):
    """theta' (FP64) of every gate of step depth + 1 of an Oracle M run."""
    c = random_circuit(n, depth + 1, p, seed)
    m = ompo.MPO(n, chi, 1e-12)
    for t in range(1, depth + 1):
        for U, pp, l in zip(c.gates[t - 1], c.p[t - 1], layer_bonds(n, c.parity(t))):
            m.apply_superop(noisy_gate_superop(U, pp), l)
        m.sweep()
    out = []
    t = depth + 1
    for U, pp, l in zip(c.gates[t - 1], c.p[t - 1], layer_bonds(n, c.parity(t))):
        Mg = noisy_gate_superop(U, pp)
        i = l - 1
        if m.centre < i:
            m.move_centre(i)
        elif m.centre > i + 1:
            m.move_centre(i + 1)
        a, b = m.A[i], m.A[i + 1]
        th = np.einsum("xyij,aijc->axyc", Mg.reshape(4, 4, 4, 4), np.tensordot(a, b, axes=(2, 0)))
        out.append(th.reshape(a.shape[0] * 4, 4 * b.shape[2]))
        m.apply_superop(Mg, l)
    return out


def lapack_truncation(A, cap, cutoff):
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    k = max(1, int(min(cap, np.count_nonzero(s > cutoff * s[0]))))
    return (U[:, :k] * s[:k]) @ Vh[:k], s[:k] ** 2


def check_kept(M, A, cap, precision="mixed", **opts):
    import torch
    if A.shape[0] > A.shape[1]:
        A = A.conj().T
    At = torch.tensor(A, device="cuda")
    U, X, lam2 = M.svd_truncated(At, cap, precision, **opts)
    U, X = U.cpu().numpy(), X.cpu().numpy()
    ref, l2ref = lapack_truncation(A, cap, 1e-12)
    got = U @ X
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    # the left factor is an isometry to the accuracy of the FP64-class
    # products (tensor-core split products: about 1e-11)
    iso = np.abs(U.conj().T @ U - np.eye(U.shape[1])).max()
    return err, iso, lam2, l2ref


@pytest.mark.parametrize("n,chi,depth,seed", [(16, 64, 10, 2), (16, 64, 12, 0), (16, 256, 9, 2)])
def test_mixed_kept_theta_per_gate(M, n, chi, depth, seed):
    """One-step error of the precision form's truncated SVD on identical FP64
    theta' (the saturated gates of a trajectory): kept theta within 1e-7 of
    the FP64 truncation, left factor orthonormal, kept squared singular values
    to 1e-9 relative (the large ones) or 1e-14 absolute."""
    thetas = oracle_thetas(n, chi, 0.005, seed, depth)
    worst = 0.0
    bulk = [th for th in thetas if min(th.shape) > chi]
    assert bulk, "the workload must contain truncating gates"
    for th in thetas:
        err, iso, lam2, l2ref = check_kept(M, th, chi)
        worst = max(worst, err)
        assert err <= KEPT_TOL, f"kept-theta error {err:.2e} on a {th.shape} gate"
        assert iso < 1e-10
        kk = min(len(lam2), len(l2ref))
        # the precision form drops lambda <= 1e-7 lambda_max (its cutoff), the
        # FP64 reference only lambda <= 1e-12 lambda_max
        assert len(lam2) <= len(l2ref) and np.all(l2ref[kk:] <= 1e-14 * l2ref[0])
        np.testing.assert_allclose(lam2[:kk], l2ref[:kk], rtol=1e-9, atol=1e-14 * l2ref[0])
    print(f"worst kept-theta error {worst:.2e}")


def test_mixed_exact_when_nothing_is_truncated(M):
    """With m = r the refined basis spans the whole row space: the mixed SVD
    equals the FP64 one to the accuracy of its FP64-class products (a
    synthetic matrix whose spectrum decays exponentially over six decades,
    the shape of Fig. 7, staying above the precision form's cutoff of
    1e-7 sigma_max)."""
    r, c = 300, 700
    U = np.linalg.qr(random_complex((r, r), 5))[0]
    Vh = np.linalg.qr(random_complex((c, r), 6))[0].conj().T
    s = np.exp(-np.linspace(0, 13.8, r))
    A = (U * s) @ Vh
    err, iso, lam2, l2ref = check_kept(M, A, r)
    assert err < 1e-10
    assert len(lam2) == r
    # squared singular values from the FP64 Gram of the projection: to ~1e-13
    # of the largest (eps_64 times a few sqrt(m)), so relative 1e-9 down to
    # 1e-5 of it
    big = l2ref > 1e-5 * l2ref[0]
    np.testing.assert_allclose(lam2[big], l2ref[big], rtol=1e-9)
    np.testing.assert_allclose(lam2, l2ref, rtol=0, atol=1e-12 * l2ref[0])


def test_rayleigh_ritz_is_what_meets_the_bar(M):
    """The FP32 SVD alone (the FP32 form's truncation of fl32(theta')) misses
    the kept-theta bar on a saturated gate; the precision form, whose FP64
    Rayleigh-Ritz starts from the same FP32 singular vectors, meets it."""
    import torch
    th = max(oracle_thetas(16, 64, 0.005, 2, 10), key=lambda a: min(a.shape))
    if th.shape[0] > th.shape[1]:
        th = th.conj().T
    U, X, _ = M.svd_truncated(torch.tensor(th.astype(np.complex64), device="cuda"), 64, "fp32")
    ref, _ = lapack_truncation(th, 64, 1e-12)
    got = U.cpu().numpy().astype(np.complex128) @ X.cpu().numpy().astype(np.complex128)
    err32 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    errmx, _, _, _ = check_kept(M, th, 64)
    print(f"kept-theta error: FP32 form {err32:.2e}, precision form {errmx:.2e}")
    assert errmx <= KEPT_TOL < err32


@pytest.mark.parametrize("steps,over", [(1, 32), (8, 64)])
def test_mixed_oversampling_and_steps(M, steps, over):
    """Other subspace sizes (chi_max + oversample) and initial step counts: the
    convergence check adds steps until the FP32 Ritz values show the kept
    directions resolved, so every setting meets the bar, with an isometric
    left factor and the FP64 squared singular values."""
    thetas = [th for th in oracle_thetas(16, 64, 0.005, 0, 12) if min(th.shape) > 64]
    for th in thetas[:6]:
        e1, iso, lam2, l2ref = check_kept(M, th, 64, oversample=over, refine_steps=steps)
        assert e1 <= KEPT_TOL and iso < 1e-10
        kk = min(len(lam2), len(l2ref))
        np.testing.assert_allclose(lam2[:kk], l2ref[:kk], rtol=1e-9, atol=1e-14 * l2ref[0])


def test_mixed_config_n8_exact_vs_dense_oracle(M):
    """n = 8, chi = 256 (no truncation by chi_max), p = 0.02: against the
    dense oracle. The precision form drops Schmidt values below 1e-7 of the
    largest at every factorisation (the resolution of its FP64 Gram
    eigen-solve); that moves S at second order in the dropped amplitude
    (~1e-14) but Tr rho at first order (a few 1e-8)."""
    c = random_circuit(8, 10, 0.02, seed=0)
    ref = dense.run(c, 256)
    S, tr, dw, m = run_gpu(M, c, 256, "mixed")
    m.close()
    assert np.abs(S - ref.S).max() < 1e-8
    assert np.abs(tr - ref.trace).max() < 1e-7


def test_mixed_truncated_vs_dense_oracle(M):
    """Truncation semantics (App. A) at n = 10, chi = 16 against Oracle D."""
    c = random_circuit(10, 8, 0.01, seed=3)
    ref = dense.run(c, 16)
    S, tr, dw, m = run_gpu(M, c, 16, "mixed")
    m.close()
    assert np.abs(S - ref.S).max() < DS_TOL
    assert np.abs(tr - ref.trace).max() < DS_TOL


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mixed_vs_fp64_trajectory(M, seed):
    """n = 16, chi = 64, p = 0.005, 12 steps, the same seeded gates through the
    precision form and the FP64 form: |dS| <= 1e-6 at every bond after every
    step, traces and discarded weights alike."""
    c = random_circuit(16, 12, 0.005, seed=seed)
    S64, tr64, dw64, m64 = run_gpu(M, c, 64, "fp64")
    m64.close()
    Smx, trmx, dwmx, mmx = run_gpu(M, c, 64, "mixed")
    mmx.close()
    dS = np.abs(Smx - S64)
    print(f"seed {seed}: max |dS| per step {dS.max(axis=1)}")
    assert dS.max() <= DS_TOL
    assert np.abs(trmx - tr64).max() <= DS_TOL * np.abs(tr64).max()
    assert np.abs(dwmx - dw64).max() <= DS_TOL


def test_mixed_centre_mode_and_schmidt_values(M):
    """Centre-only entropy mode of the precision form, and the Schmidt values
    it records, against the FP64 form."""
    c = random_circuit(16, 10, 0.005, seed=4)
    S64, _, _, m64 = run_gpu(M, c, 64, "fp64", centre_only=True)
    Smx, _, _, mmx = run_gpu(M, c, 64, "mixed", centre_only=True)
    b = 16 // 2 - 1
    assert np.all(np.isnan(Smx[:, :b])) and np.all(np.isnan(Smx[:, b + 1:]))
    assert np.abs(Smx[:, b] - S64[:, b]).max() <= DS_TOL
    l64, lmx = m64.schmidt(b), mmx.schmidt(b)
    n = min(len(l64), len(lmx))
    assert np.abs(l64[:n] - lmx[:n]).max() < 1e-7
    m64.close()
    mmx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_theta_export_matches_oracle(M, precision):
    """mpo_theta (App. A: the superoperator applied to the contracted sites,
    before truncation) against Oracle M's theta' for the first gate of step
    11 of the same seeded circuit. The bond bases are fixed only up to
    unitaries and the scalar factor is kept apart, so the gauge-invariant
    normalised singular values are compared."""
    c = random_circuit(16, 11, 0.005, 2)
    m = M.MPO(16, 64, precision)
    for t in range(1, 11):
        m.apply_layer(c.parity(t), c.gates[t - 1], c.p[t - 1])
    l0 = layer_bonds(16, c.parity(11))[0]
    th = m.theta(l0 - 1, c.gates[10][0], float(c.p[10][0])).cpu().numpy()
    m.close()
    ref = oracle_thetas(16, 64, 0.005, 2, 10)[0]
    if precision == "fp64":
        assert th.shape == ref.shape
    s, sr = np.linalg.svd(th, compute_uv=False), np.linalg.svd(ref, compute_uv=False)
    # the handle keeps the MPO's scalar factor apart (its log-norm): compare
    # the spectra normalised to unit Frobenius norm
    s, sr = s / np.linalg.norm(s), sr / np.linalg.norm(sr)
    # the precision form drops Schmidt values below 1e-7 of the largest at
    # every factorisation, so its bonds may be narrower by those directions
    k = min(len(s), len(sr))
    np.testing.assert_allclose(s[:k], sr[:k], rtol=0, atol=(1e-10 if precision == "fp64" else 1e-7) * sr[0])
    assert np.all(sr[k:] <= 1e-6 * sr[0])
