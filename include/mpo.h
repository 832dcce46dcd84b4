/*
 * mpo.h - C ABI of the GB300 noisy-MPO engine.
 *
 * The engine simulates 1D brickwork circuits of noisy two-qubit gates on a
 * density matrix stored as a matrix product operator (MPO), following
 * Noh, Jiang & Fefferman, "Efficient classical simulation of noisy random
 * quantum circuits in one dimension" (arXiv:2003.13163):
 *
 *   - state: the vectorised density matrix |rho>> of Sec. 3.1 with local
 *     index I = 2 i + i' (ket digit high, bra digit low), kept as an MPO in
 *     mixed canonical form (the local QR/TEBD update of the "Note added",
 *     equivalent in exact arithmetic to the canonical update of App. A);
 *   - gate: the noisy two-qubit map M = N_2[p] o U of Sec. 3.2 with the
 *     two-qubit depolarising channel N_2[p] of Sec. 2.2, applied as its
 *     16x16 superoperator (App. A) to the two-site tensor theta, followed by
 *     the truncated SVD that keeps the chi_max largest Schmidt values (App. A);
 *   - output: the MPO entanglement entropy S_l of Sec. 3.3 at every bond after
 *     every step, Tr rho (Sec. 3.4) and the discarded weight.
 *
 * Conventions shared by every call:
 *   - qubits/sites are 1..n in the paper; the ABI numbers bonds 0..n-2, ABI
 *     bond b = paper bond l - 1 (the cut between paper sites l and l+1);
 *   - a gate U is a 4x4 complex128 matrix, row-major, basis index
 *     2 i_l + i_{l+1} (qubit l is the high digit), stored as interleaved
 *     (re, im) doubles: double[4][4][2];
 *   - p is the paper's two-qubit depolarising rate (Sec. 2.2): the channel is
 *     (1 - 16p/15) rho + (16p/15) (I/4) Tr rho, fully depolarising at p = 15/16;
 *   - all device work is issued on the stream given to mpo_init. Calls on one
 *     handle must not run concurrently from several host threads.
 *
 * Errors: every int-returning call returns MPO_OK (0) or a negative MPO_ERR_*
 * code; mpo_last_error() gives a message. After an error the handle refuses
 * further work with MPO_ERR_STATE until mpo_free. There is no CPU fallback:
 * without a usable CUDA device mpo_init returns MPO_ERR_CUDA.
 */
#ifndef GB300_MPO_H
#define GB300_MPO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpo_ctx *mpo_handle;

/* Arithmetic of the path.
 *   MPO_FP64:       complex128 site tensors, every contraction and eigen-solve in
 *                   FP64 (the plain form).
 *   MPO_FP32:       complex64 site tensors and FP32 contractions and eigen-solves;
 *                   Schmidt-value normalisation, entropy and log-norm stay FP64.
 *                   Fast, but its entropies differ from the FP64 form by ~1e-3.
 *   MPO_MIXED_FP32: the precision form. complex128 site tensors; every truncated
 *                   SVD (App. A) and centre move starts from the FP32 one-sided
 *                   Jacobi SVD of an FP32 copy, whose m = chi_max + oversample
 *                   leading left singular vectors Q are refined in FP64 by one
 *                   Rayleigh-Ritz step: B = Q^H theta' and H = B B^H by
 *                   FP64-accurate products, and the FP64 Hermitian Jacobi
 *                   eigen-solve of H (optionally preceded by refine_steps FP64
 *                   subspace-iteration steps); the singular values, their
 *                   normalisation and the entropy are FP64. Matches the FP64
 *                   form to |dS| <= 1e-6 and a kept-theta relative Frobenius
 *                   error <= 1e-7 per gate. */
typedef enum { MPO_FP64 = 0, MPO_FP32 = 1, MPO_MIXED_FP32 = 2 } mpo_precision;

/* Which bonds mpo_entropy reports.
 *   MPO_S_ALL_BONDS: the end-of-step Schmidt sweep computes lambda at every bond.
 *   MPO_S_CENTRE:    only the centre bond (ABI bond n/2 - 1); other entries NaN. */
typedef enum { MPO_S_ALL_BONDS = 0, MPO_S_CENTRE = 1 } mpo_entropy_mode;

enum {
  MPO_OK = 0,
  MPO_ERR_ARG = -1,     /* invalid argument (sizes, parity, NULL)              */
  MPO_ERR_CUDA = -2,    /* a CUDA call failed, or no device                    */
  MPO_ERR_OOM = -3,     /* device allocation failed or exceeded arena_cap_bytes */
  MPO_ERR_NOCONV = -4,  /* an SVD / eigen-solve hit its sweep cap unconverged   */
  MPO_ERR_TIMEOUT = -5, /* a bounded device-side wait gave up                   */
  MPO_ERR_STATE = -6    /* handle is in an error state or call order is wrong   */
};

/* Options; pass NULL for the defaults given in brackets. */
typedef struct {
  int eig_max_sweeps;       /* cap on Jacobi sweeps per SVD [40, at most 64]; reaching it -> MPO_ERR_NOCONV */
  double sv_rel_cutoff;     /* drop Schmidt values lambda <= cutoff * lambda_max at every
                               factorisation [1e-12 for FP64, 1e-6 for FP32: the rounding
                               floor of the one-sided Jacobi SVD; 1e-7 for MPO_MIXED_FP32]; <= 0
                               selects the default */
  size_t arena_cap_bytes;   /* refuse device allocations above this total [0 = no cap] */
  mpo_entropy_mode smode;   /* [MPO_S_ALL_BONDS] */
  double barrier_timeout_s; /* limit of each device-side grid-barrier wait [5.0] */
  int block_jacobi_min_rows;/* factorisations with at least this many rows use the block
                               one-sided Jacobi SVD (pairs of 16-row blocks) instead of the
                               row-pair one [0 = default: 64 for FP32, never for FP64;
                               < 0 = never]. The block form needs far fewer passes over
                               the matrix but resolves singular values only to about
                               sqrt(eps) * sigma_max relative accuracy per row pair. */
  int tensor_cores;         /* MPO_FP32: > 0 runs the plain complex products (theta, centre
                               moves) on the tcgen05 tensor cores with 3 x TF32 split products
                               [0 = off: the SIMT FP32 kernel, currently the faster one].
                               MPO_MIXED_FP32: >= 0 runs its FP64 products (theta, the
                               refinement and the projections) on the tensor cores as
                               FP64-accurate BF16 split products [0 = on; < 0 = SIMT FP64] */
  int oversample;           /* MPO_MIXED_FP32: extra FP32 singular vectors carried into the FP64
                               Rayleigh-Ritz step of a truncating SVD, beyond chi_max [0 = 64;
                               < 0 = none] */
  int refine_steps;         /* MPO_MIXED_FP32: FP64 subspace-iteration steps (shifted CholeskyQR3
                               after each product) before the Rayleigh-Ritz step of a truncating
                               SVD [0 or < 0 = none, the default; at most 7] */
} mpo_opts;

/* Fill *o with the defaults. */
void mpo_default_opts(mpo_opts *o);

/* Create an n-qubit MPO in the product state |0..0><0..0| (Sec. 4.1, initial
 * lambda = (1,0,..), one-hot Gamma at I = 0).
 *   out        : receives the handle (set to NULL on failure).
 *   n_qubits   : even, 2 <= n_qubits <= 4096 (Sec. 2.1 takes n even).
 *   chi_max    : bond-dimension cap of the truncation (App. A), 1 <= chi_max <= 4096.
 *   prec       : MPO_FP64, MPO_FP32 or MPO_MIXED_FP32.
 *   cuda_stream: a cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream),
 *                or NULL for the legacy default stream.
 *   opts       : NULL for defaults.
 * Allocates all device memory up front for the worst-case bond dimensions
 * min(chi_max, 4^b, 4^(n-b)); returns MPO_ERR_OOM if that exceeds the device
 * or arena_cap_bytes. */
int mpo_init(mpo_handle *out, int n_qubits, int chi_max, mpo_precision prec,
             void *cuda_stream, const mpo_opts *opts);

/* Apply one brickwork step (Sec. 2.1, Sec. 4.1): the noisy gates of one layer
 * in ascending bond order, each followed by its truncation to chi_max, then
 * the end-of-step Schmidt sweep and entropy reduction.
 *   parity : 0 = paper bonds 1,3,..,n-1 (odd time step, n/2 gates);
 *            1 = paper bonds 2,4,..,n-2 (even time step, n/2-1 gates).
 *   gates  : [n_gates][4][4][2] doubles (complex128 U, see conventions);
 *            host or device pointer (detected); gate i acts on paper bond
 *            2 i + 1 + parity. Host memory is copied before the call returns.
 *   p      : depolarising rates, host or device; p[i * p_stride] for gate i
 *            (p_stride = 0 applies p[0] to every gate). 0 <= p <= 1.
 * The call may synchronise the stream (it reads back kept bond dimensions). */
int mpo_apply_layer(mpo_handle h, int parity, const double *gates, const double *p, int p_stride);

/* Apply one noisy gate on ABI bond b (paper bond b+1) without the end-of-step
 * sweep; for tests and custom schedules. Same gate / p formats as above. */
int mpo_apply_gate(mpo_handle h, int bond, const double *gate, double p);

/* The two-site block theta' = M (A_b A_{b+1}) of a noisy gate on ABI bond b
 * (App. A: the superoperator applied to the contracted sites, before the
 * truncated SVD), (4 chi_b) x (4 chi_{b+2}) row-major, row (a, I_b) =
 * 4 a + I_b, column (I_{b+1}, c) = chi_{b+2} I_{b+1} + c; complex128 for
 * MPO_FP64 / MPO_MIXED_FP32 handles, complex64 for MPO_FP32, in the handle's
 * normalisation (the MPO's scalar factor, kept apart as a log-norm, is not
 * applied: multiply by exp(log-norm) for the block of rho). The centre is
 * moved onto the bond (the state is unchanged otherwise) and nothing is
 * truncated. gate / p as for mpo_apply_gate; out: host or device buffer of
 * rows x cols entries, or NULL to query *rows, *cols only. Synchronises. */
int mpo_theta(mpo_handle h, int bond, const double *gate, double p, void *out, int *rows, int *cols);

/* Apply a general 16x16 two-site superoperator (row 4*I_l + I_{l+1}, column
 * 4*J_l + J_{l+1}, App. A convention), complex128 interleaved [16][16][2],
 * host or device pointer, on ABI bond b. Sec. 2.2 notes the method covers
 * any two-qubit error model; this entry takes the map directly. A map that
 * mpo_check_superop rejects (tolerance 1e-9) returns MPO_ERR_ARG and leaves
 * the state untouched. */
int mpo_apply_superop(mpo_handle h, int bond, const double *M);

/* Is M (as for mpo_apply_superop) a quantum channel (Sec. 2.2)? Checks trace
 * preservation, t^T M = t^T with t the vectorised two-qubit trace (t_I = 1
 * for I in {0, 3} on each qubit), and complete positivity, the 16x16 Choi
 * matrix C[(a, j), (b, k)] = (M(|j><k|))_{ab} Hermitian positive
 * semidefinite (host FP64 Jacobi eigenvalues), each to tol (<= 0: 1e-9)
 * times the largest |M_ij|. Returns MPO_OK or MPO_ERR_ARG (MPO_ERR_CUDA if a
 * device M cannot be read); *defect (may be NULL) receives the larger
 * violation. Host code only: runs without a GPU for host M. */
int mpo_check_superop(const double *M, double tol, double *defect);

/* Run the Schmidt sweep now (normally done at the end of mpo_apply_layer). */
int mpo_sweep(mpo_handle h);

/* Read the results of the last step. Synchronises the stream.
 *   S         : host [n-1]: MPO entanglement entropy (Sec. 3.3, base 2) at ABI
 *               bond b (NaN where not computed).
 *   trace     : nullable; Tr rho (Sec. 3.4) including the tracked log-norm.
 *   discarded : nullable; sum over the step's gates of the discarded weight
 *               w = sum_{dropped} lambda'^2 / sum_all lambda'^2. */
int mpo_entropy(mpo_handle h, double *S, double *trace, double *discarded);

/* Schmidt values lambda^[b] of ABI bond b from the last sweep, normalised so
 * that sum lambda^2 = 1, descending. lam: host [chi_max]; *len receives the
 * count. */
int mpo_schmidt(mpo_handle h, int bond, double *lam, int *len);

/* Current bond dimensions: dims host [n+1], dims[0] = dims[n] = 1. */
int mpo_bond_dims(mpo_handle h, int *dims);

/* Copy site k (0-based) to host as complex128 interleaved [chiL][4][chiR][2],
 * scaled so that the MPO's product of sites equals rho (the log-norm is
 * folded into the centre site). *chiL / *chiR receive the dims; buf may be
 * NULL to query them. */
int mpo_get_site(mpo_handle h, int k, double *buf, int *chiL, int *chiR);

/* Output probabilities (Sec. 3.4): P(x) = <<X|rho>> with X_k = (d+1) x_k, i.e.
 * the product over sites of the I = 3 x_k slices, times the tracked scale.
 *   bits: host [n_strings][n] bytes, each 0 or 1 (x_1 first);
 *   P   : host [n_strings] out. With truncation P sums to Tr rho <= 1 over all
 *         x (Sec. 3.4), and single entries can dip slightly below zero.
 * Synchronises the stream; allocates its scratch per call. */
int mpo_probability(mpo_handle h, int n_strings, const unsigned char *bits, double *P);

/* Samples from P(x) / Tr rho by sequential conditionals (Sec. 3.4): bit k is 0
 * when u_k < P(x_1..x_{k-1}, 0) / (P(.., 0) + P(.., 1)), the marginals taken
 * with the trace vector on the remaining sites; the comparison is made in FP64.
 *   uniforms: host [n_samples][n] doubles in [0, 1) supplied by the caller
 *             (the randomness is an input, so runs are reproducible);
 *   bits    : host [n_samples][n] out;
 *   P       : nullable host [n_samples] out, P(x) of each drawn string.
 * Synchronises the stream; allocates its scratch per call. */
int mpo_sample(mpo_handle h, int n_samples, const double *uniforms, unsigned char *bits, double *P);

/* ---- Batching form -------------------------------------------------------
 * k independent circuits (the ensembles of circuit instances the paper runs
 * per (n, p) point, Sec. 4) held and advanced together. Each instance is an
 * engine context of its own (n_i qubits, the shared chi_max, precision and
 * options) on a stream the library creates; n_workers host threads (<= 0:
 * min(8, k)) drive the instances of a call concurrently, longest chains
 * first. A batch handle accepts only the calls of this block, mpo_free and
 * mpo_last_error; the other calls return MPO_ERR_ARG on it.
 *   n_i        : host [k], each even, 2..4096.
 *   cuda_stream: the caller's stream; each call's work starts after the work
 *                already queued on it (so device gate arrays written there
 *                are safe to read).
 * Errors as mpo_init; the message names the failing instance. */
int mpo_init_batch(mpo_handle *out, int k, const int *n_i, int chi_max, mpo_precision prec, void *cuda_stream,
                   const mpo_opts *opts, int n_workers);

/* One step t (1-based; odd t acts on paper bonds 1, 3, ..., even t on 2, 4,
 * ..., in ascending order, Sec. 3.3) on every instance i with active[i] != 0
 * (active NULL: all). Synchronous: returns when every instance has finished.
 *   gates_all : host or device; for each active instance in index order, its
 *               (n_i - parity) / 2 gates as [4][4] complex128 (row-major,
 *               interleaved), where parity = (t + 1) % 2;
 *   p_all     : host [k], the paper's p of each instance (one per instance);
 *   S_all     : nullable host out, the n_i - 1 bond entropies (bits) of
 *               instance i at offset sum_{j<i} (n_j - 1), as mpo_entropy;
 *   trace_all : nullable host [k] out, Tr rho of each active instance;
 *   discarded_all: nullable host [k] out, the step's summed discarded weight.
 * Outputs of inactive instances are left untouched. On an instance's error
 * the call returns its code and the batch handle enters the error state. */
int mpo_apply_layer_batch(mpo_handle h, int t, const double *gates_all, const double *p_all, const int *active,
                          double *S_all, double *trace_all, double *discarded_all);

/* The context of instance i of a batch (owned by the batch: do not free),
 * for the diagnostic calls (mpo_schmidt, mpo_to_dense, mpo_bond_dims, ...).
 * Do not use it while mpo_apply_layer_batch runs. */
int mpo_batch_instance(mpo_handle h, int i, mpo_handle *inst);

/* Contract the MPO into |rho>> (4^n complex128, interleaved, index
 * I_1 I_2 .. I_n with I_1 most significant). n <= 12. Test export. */
int mpo_to_dense(mpo_handle h, double *rho_vec);

/* Orthogonality-centre site (0-based). */
int mpo_centre(mpo_handle h, int *centre);

/* Device bytes held by the handle. */
size_t mpo_device_bytes(mpo_handle h);

/* Kernel timing. enable = 1 clears the counters and starts recording a CUDA
 * event pair on the handle's stream around every kernel launch of the path;
 * enable = 0 stops. Adds a little launch overhead while on; the paper has no
 * counterpart (it is a measurement aid). */
int mpo_profile(mpo_handle h, int enable);

/* Totals for kernel class cls (0 .. 11: svd_gate (the truncated SVD of a
 * gate), svd_sweep (the SVDs of centre moves and Schmidt sweeps), cgemm,
 * superop, select, gather, transpose, trace, tc_cgemm, refine_gemm (the FP64
 * products of the precision form's refinement), eig_fp64 (its FP64 Hermitian
 * eigen-solves), convert (its FP32 copies)) since the last mpo_profile(h, 1):
 * summed event durations in ms, launch count, and the algorithmic flops and
 * bytes of those launches as the library counts them: an SVD of an r x c
 * matrix (r <= c) keeping k values counts the Hermitian Gram 4 r^2 c, the
 * projection 8 k r c and, unless the eigen-solve is a launch of its own
 * (eig_fp64, 13.3 m^3), 13.3 r^3; a complex GEMM 8 M N K. Returns
 * MPO_ERR_ARG past the last class. Synchronises the stream. */
int mpo_profile_read(mpo_handle h, int cls, const char **name, double *ms, long long *launches, double *flops,
                     double *bytes);

/* Jacobi sweeps summed over the SVD launches recorded since mpo_profile(h, 1). */
long long mpo_profile_sweeps(mpo_handle h);

/* MPO_MIXED_FP32: subspace-iteration steps summed over the truncated SVDs
 * recorded since mpo_profile(h, 1) (0 for the other forms). */
long long mpo_profile_steps(mpo_handle h);

/* Wall time (ms) spent by the block Jacobi SVD in its three phases (Gram
 * partials, pair eigen-solves, rotation apply; grid-barrier waits included),
 * summed since mpo_profile(h, 1). ms3: host [3]. */
int mpo_profile_phases(mpo_handle h, double *ms3);

/* Release everything; NULL is a no-op. */
void mpo_free(mpo_handle h);

/* Message of the last error on h (or of the last failed mpo_init when h is
 * NULL); thread-local storage, valid until the next call. */
const char *mpo_last_error(mpo_handle h);

/* Stand-alone Hermitian eigen-solver used by the path (cyclic parallel
 * Jacobi), exported for tests: A is m x m complex (interleaved, row-major,
 * leading dimension m), device pointer, overwritten. On return w (device,
 * [m]) holds eigenvalues and V (device, m x m row-major) the eigenvectors as
 * columns, unsorted. prec selects FP64 (double) or FP32 (float) buffers.
 * Returns MPO_ERR_NOCONV when max_sweeps is reached. */
int mpo_eigh(int m, void *A, void *w, void *V, mpo_precision prec, int max_sweeps, void *cuda_stream);

/* Stand-alone one-sided Jacobi SVD used by every factorisation of the path
 * (App. A's SVD of B, and the centre moves), exported for tests. block = 0
 * selects the row-pair (Hestenes) form, block = 1 the 16-row block form. X is r x c
 * complex (interleaved, row-major, leading dimension c), device pointer,
 * overwritten with U^H X, whose rows are mutually orthogonal. On return w
 * (device, [r]) holds the squared row norms (the squared singular values of
 * the input, unsorted) and Ut (device, r x r row-major) the transpose of the
 * unitary U, so input = U * output. Returns MPO_ERR_NOCONV when max_sweeps
 * (<= 64) is reached. */
int mpo_svd(int r, int c, void *X, void *w, void *Ut, mpo_precision prec, int max_sweeps, int block,
            void *cuda_stream);

/* The truncated SVD of every gate (App. A: keep the cap largest singular
 * values, and only those above sv_rel_cutoff * the largest) in the arithmetic
 * of precision prec, exported for tests: for MPO_MIXED_FP32 it is the FP32
 * Jacobi SVD plus FP64 subspace refinement and Rayleigh-Ritz projection that
 * the precision form applies to every theta'.
 *   A     : device, r x c complex (complex128 for MPO_FP64 / MPO_MIXED_FP32,
 *           complex64 for MPO_FP32), row-major, 1 <= r <= c, r <= 8192; not
 *           modified.
 *   cap   : the bond-dimension cap chi_max.
 *   opts  : NULL for the defaults (sv_rel_cutoff, oversample, refine_steps,
 *           eig_max_sweeps, block_jacobi_min_rows as in mpo_opts).
 *   U     : device, r x cap complex (leading dimension cap): columns 0..k-1
 *           receive the left singular vectors in descending order.
 *   X     : device, cap x c complex: rows 0..k-1 receive lambda_j w_j^H, so
 *           that U[:, :k] X[:k] is the kept part of A.
 *   lam2  : host [cap]: the k kept squared singular values, descending.
 *   k     : host: the kept count.
 * Allocates its workspace per call and waits for the stream. Errors as
 * mpo_svd; the message is in mpo_last_error(NULL). */
int mpo_svd_truncated(int r, int c, const void *A, int cap, mpo_precision prec, const mpo_opts *opts, void *U,
                      void *X, double *lam2, int *k, void *cuda_stream);

/* Statistics of the last mpo_svd call made on the calling thread: the sweeps
 * it ran and, for the block variant, the wall time (ms) of its three phases
 * (Gram partials, pair solves, rotation apply; grid-barrier waits included,
 * zeros for the row-pair variant). Either pointer may be NULL (host). */
int mpo_svd_last_stats(int *sweeps, double *phase_ms3);

/* Block one-sided Jacobi SVD that allocates nothing (the paper has no
 * counterpart; this is a deployment aid).
 *
 * Same contract and result as mpo_svd(r, c, X, w, Ut, prec, max_sweeps, 1,
 * stream) for r <= 512 and c <= 2048, but every piece of scratch the solver
 * needs lives in one device array built into the library (about 1.7 MB per
 * GPU that uses it, held until the process exits). It is meant for callers
 * that must not call cudaMalloc when they need the factorisation: code that
 * runs inside a memory allocator's own hooks (a framework's custom-allocator
 * callback, where allocating again would re-enter the allocator), or a host
 * that grants the library a fixed memory budget ahead of time and accounts
 * for every byte it hands out.
 *
 *   - Larger matrices are rejected with MPO_ERR_ARG; mpo_last_error(NULL) says
 *     which limit was hit. Other errors as for mpo_svd.
 *   - The first call on a device loads the library's device code (CUDA loads
 *     modules lazily by default) and maps the array, so that call itself
 *     takes device memory (about 1.7 MB plus the module) and looks up the
 *     array's address. Callers inside allocator hooks or under a fixed budget
 *     make one warm-up call at initialisation (any size, e.g. 1 x 1), before
 *     any stream capture; later calls allocate nothing.
 *   - mpo_svd_last_stats reports the sweeps and phase times of the last call,
 *     as for mpo_svd(..., block = 1).
 *   - All calls on a device share the one array, which keeps the last call's
 *     contents. Calls whose work overlaps on the GPU (several streams, several
 *     host threads) race on it and must be serialised by the caller.
 *   - The call waits for the stream before it returns (it reads the solver's
 *     status). */
int mpo_svd_static(int r, int c, void *X, void *w, void *Ut, mpo_precision prec, int max_sweeps,
                   void *cuda_stream);

/* Stand-alone complex GEMM used by the path, exported for tests:
 * C (M x N) = A (M x K) B (K x N), row-major, interleaved complex, device
 * pointers. tensor_cores = 1 (FP32 only) runs the tcgen05 kernel with 3 x TF32
 * split products, 0 the SIMT kernel of the given precision. */
int mpo_gemm(int M, int N, int K, const void *A, const void *B, void *C, mpo_precision prec, int tensor_cores,
             void *cuda_stream);

/* The same product with explicit operand forms and engines, exported for
 * tests: C (M x N, leading dimension ldc) = op(A) op(B), op 0 = as stored,
 * op 1 = conjugate transpose (A is then stored K x M with leading dimension
 * lda, B N x K with ldb), device pointers. engine 0 runs the SIMT kernel of
 * the given precision; engine 1 the tensor cores: for MPO_FP32 the 3 x TF32
 * kernel (opA = opB = 0 only, as mpo_gemm), for MPO_FP64 the FP64-accurate
 * product from BF16 slices with FP32 accumulation that the precision form
 * uses (each operand split into 6 slices of 7 bits under a power-of-two
 * scale per row / column; relative error about 2^-42 of |row| |column|).
 * Allocates its scratch per call and waits for the stream. */
int mpo_gemm_ex(int M, int N, int K, const void *A, int lda, int opA, const void *B, int ldb, int opB, void *C,
                int ldc, mpo_precision prec, int engine, void *cuda_stream);

/* Library version string. */
const char *mpo_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_MPO_H */
