// mpo_api.cu - the C ABI of include/mpo.h: device store, per-gate update,
// end-of-step Schmidt sweep and observables of the noisy-MPO simulation of
// arXiv:2003.13163, on one GB300.
//
// State layout (device, one buffer per site, all of the same capacity so that
// results can be produced in a spare buffer and swapped in by pointer):
//   site k holds A_k[alpha][I][beta], row-major, chi[k] x 4 x chi[k+1],
//   complex (double2 or float2). Its left matricisation L(A_k) is the plain
//   row-major (4 chi[k]) x chi[k+1] matrix, its right matricisation R(A_k) the
//   plain row-major chi[k] x (4 chi[k+1]) matrix: both are views of the same
//   memory. Sites left of the centre are left isometries, sites right of it
//   right isometries; the centre has unit Frobenius norm and the true scale
//   is exp(lognorm) (device FP64), so rho = exp(lognorm) * A_1 ... A_n.
//
// Per noisy gate on sites (i, i+1) (App. A bulk/edge cases, with the local
// update of the Note added):
//   1. move the centre to i or i+1 (QR-type moves, below);
//   2. theta = L(A_i) R(A_{i+1})                       (complex GEMM)
//   3. theta' = M theta on (I, J)                      (superoperator kernel)
//   4. Gram of the smaller side, Hermitian eigen-solve (Jacobi), select the
//      chi_max largest lambda'^2 (App. A truncation), discarded weight;
//   5. write back: left isometry -> site i, Lambda W^H / ||kept|| -> site i+1.
// Centre moves and the sweep use the same Gram/eigen route: for the centre C,
// G = C^H C (or C C^H) = V diag(sigma^2) V^H, the isometry is C V Sigma^-1 (or
// Sigma^-1 V^H C) and Sigma V^H (or V Sigma) is pushed into the neighbour;
// sigma <= cutoff * sigma_max are dropped (they are below the rounding floor
// of the Gram). The sweep's sigma at bond b are the Schmidt values lambda^[b].
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <complex>
#include <string>
#include <vector>
#include <algorithm>
#include <type_traits>
#include <atomic>
#include <map>
#include <mutex>
#include <thread>

#include "../../include/mpo.h"
#include "common.cuh"
#include "linalg.cuh"
#include "mpo_kernels.cuh"
#include "mixed.cuh"
#include "tcgemm.cuh"
#include "ozgemm.cuh"

namespace {

thread_local std::string g_last_init_error;
thread_local int g_last_svd_sweeps = 0;           // statistics of the last mpo_svd on this thread
thread_local double g_last_svd_phase_ms[3] = {0.0, 0.0, 0.0};

struct HostSync {   // pinned read-back of the last select + eigen-solve
  SelectInfo info;
  GridCtl ctl;
  unsigned long long phase_ns[4];
  int tc_err;
  GridCtl eig[8];     // FP64 eigen-solves of the last mixed factorisation
  int chol_status;    // Cholesky QR pivot status of the last mixed factorisation
  int oz_err;         // the tensor-core FP64 GEMM's wait-limit flag
};

}  // namespace

struct BatchState;

// Scratch of the FP64-accurate tensor-core GEMM: the BF16 slices of both
// operands and their row / column exponents (sized for the largest product
// the handle issues).
struct OzWork {
  __nv_bfloat16 *a = nullptr, *b = nullptr;
  int *ea = nullptr, *eb = nullptr, *status = nullptr;
  size_t a_cap = 0, b_cap = 0;     // elements
  int e_cap = 0;
};

struct mpo_ctx {
  BatchState* batch = nullptr;     // set on handles made by mpo_init_batch
  int n = 0, chi_max = 0;
  mpo_precision prec = MPO_FP64;
  cudaStream_t st = nullptr;
  mpo_opts opts{};
  double cutoff = 0.0;
  bool failed = false;
  std::string msg;
  int device = 0, num_sms = 0;

  std::vector<int> cap, chi;       // bond caps / current dims, index 0..n
  std::vector<void*> site;         // n buffers, each site_cap elements
  void* spare = nullptr;
  size_t site_cap = 0, esz = 0;    // elements per site buffer, bytes per complex
  void* theta2 = nullptr;          // conjugate-transposed operand of the one-sided SVD
  void *theta = nullptr, *vecs = nullptr, *tmp = nullptr, *wv = nullptr, *Ms = nullptr;
  size_t theta_cap = 0, tmp_cap = 0;
  int m_cap = 0;
  int* perm = nullptr;
  double* lam2 = nullptr;
  SelectInfo* info = nullptr;
  GridCtl* ctl = nullptr;
  OSCtl* osctl = nullptr;          // control block of the Jacobi launches (barriers, status, counts)
  void *bj_gpart = nullptr, *bj_j = nullptr;   // block Jacobi partial Grams and pair rotations
  int* bj_act = nullptr;                        // block Jacobi integer state (bj_state_ints)
  size_t bj_slots = 0, bj_act_ints = 0;
  int block_min_rows = 0;
  bool tensor_cores = false;       // FP32 plain products on tcgen05
  int* tc_status = nullptr;        // set by the tensor-core GEMM if a wait timed out
  double* scal = nullptr;          // [0] lognorm, [1] discarded accumulator
  double* dS = nullptr;            // [n-1]
  double* dschmidt = nullptr;      // [(n-1) * chi_max]
  double2* dgates = nullptr;
  double2* dsup = nullptr;         // staging of a caller-given 16x16 superoperator
  double* dp = nullptr;
  double2 *tv0 = nullptr, *tv1 = nullptr;
  HostSync* hs = nullptr;          // pinned
  std::vector<int> schmidt_len;
  std::vector<char> s_valid;
  int centre = 0;
  size_t bytes = 0;
  int last_sweeps = 0;
  // kernel-class timing (mpo_profile): CUDA events recorded on h->st around
  // each launch, resolved lazily
  // precision form (MPO_MIXED_FP32): complex128 sites, FP32 approximate SVD,
  // FP64 refinement; buffers of the refinement (see msvd_select)
  bool mixed = false;
  bool vecs_conj = false;          // vecs holds rows conj(column of U) (mixed) instead of U^T
  int mx_over = 0, mx_steps = 0;   // oversampling and refinement steps
  int mx_mcap = 0;                 // largest m = min(r, chi_max + oversample)
  float2 *mx_a32 = nullptr, *mx_ut32 = nullptr;
  float* mx_w32 = nullptr;
  int* mx_perm32 = nullptr;
  double* mx_lam32 = nullptr;
  SelectInfo* mx_info32 = nullptr;
  double2 *mx_Q = nullptr, *mx_Q2 = nullptr, *mx_B = nullptr, *mx_T = nullptr;
  double2 *mx_V = nullptr, *mx_G = nullptr;
  double* mx_w = nullptr;
  double2* mx_W = nullptr;         // D L^{-H} of a Cholesky QR pass; the FP32 Ritz vectors, promoted
  double2* mx_Q0 = nullptr;        // the stage-2 basis (FP32 Ritz directions in FP64)
  float2 *mx_A32 = nullptr, *mx_Li32 = nullptr, *mx_t32 = nullptr;   // FP32 Cholesky: scaled Gram, L^{-1}, scratch
  double* mx_d = nullptr;          // column scales of a Cholesky QR pass
  unsigned long long mx_seed = 0;  // start-basis counter
  int mx_last_steps = 0;           // subspace steps taken by the last factorisation
  int mx_cur_bond = -1;            // bond of the gate being factorised (-1: not a gate)
  std::vector<int> mx_bond_steps;  // subspace steps the last gate on each bond needed
  long long prof_steps = 0;        // subspace steps since profiling was switched on
  OSCtl* mx_eosctl = nullptr;      // control block of the FP64 Rayleigh-Ritz eigen-solve
  int* mx_chst = nullptr;          // set when a Cholesky pivot was not positive
  OzWork oz;                       // FP64-accurate tensor-core GEMM scratch (precision form)
  bool use_oz = false;
  bool prof = false;
  struct Pending { int cls; cudaEvent_t a, b; double flops, bytes; };
  std::vector<Pending> pend;
  std::vector<cudaEvent_t> evpool;
  double prof_ms[16] = {0}, prof_flops[16] = {0}, prof_bytes[16] = {0};
  long long prof_n[16] = {0};
  long long prof_sweeps = 0;
  double prof_phase_ns[3] = {0, 0, 0};
};

enum { PK_SVD = 0, PK_SVD_SWEEP, PK_GEMM, PK_SUPEROP, PK_SELECT, PK_GATHER, PK_TRANSPOSE, PK_TRACE, PK_TCGEMM,
       PK_REFINE, PK_EIG64, PK_CONVERT, PK_OZ, PK_NCLASS };
static const char* kProfNames[PK_NCLASS] = {"svd_gate", "svd_sweep", "cgemm", "superop", "select", "gather", "transpose", "trace",
                                            "tc_cgemm", "refine_gemm", "eig_fp64", "convert", "oz_gemm"};

static cudaEvent_t prof_event(mpo_ctx* h) {
  if (!h->evpool.empty()) { cudaEvent_t e = h->evpool.back(); h->evpool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static void prof_resolve(mpo_ctx* h) {
  if (h->pend.empty()) return;
  cudaStreamSynchronize(h->st);
  for (auto& q : h->pend) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      h->prof_ms[q.cls] += ms;
      h->prof_n[q.cls] += 1;
      h->prof_flops[q.cls] += q.flops;
      h->prof_bytes[q.cls] += q.bytes;
    }
    h->evpool.push_back(q.a);
    h->evpool.push_back(q.b);
  }
  h->pend.clear();
}

// Bracket one launch with events when profiling is on.
struct ProfScope {
  mpo_ctx* h;
  int cls;
  double flops, bytes;
  cudaEvent_t a = nullptr;
  ProfScope(mpo_ctx* h_, int c, double f, double b) : h(h_), cls(c), flops(f), bytes(b) {
    if (h->prof) { a = prof_event(h); cudaEventRecord(a, h->st); }
  }
  void set(double f, double b) { flops = f; bytes = b; }
  ~ProfScope() {
    if (!h->prof || !a) return;
    cudaEvent_t b = prof_event(h);
    cudaEventRecord(b, h->st);
    h->pend.push_back({cls, a, b, flops, bytes});
    if (h->pend.size() > 2048) prof_resolve(h);
  }
};

// ------------------------------------------------------------------ errors --
static int fail(mpo_ctx* h, int code, const std::string& m) {
  h->failed = true;
  h->msg = m;
  return code;
}
#define CK(h, call)                                                                         \
  do {                                                                                      \
    cudaError_t e__ = (call);                                                               \
    if (e__ != cudaSuccess)                                                                 \
      return fail((h), MPO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
  } while (0)

// complex128 site tensors: the FP64 form and the precision form
static bool dsite(const mpo_ctx* h) { return h->prec != MPO_FP32; }

static int cap_of(int b, int n, int chi_max) {
  // min(chi_max, 4^b, 4^(n-b)) without overflow
  int e = std::min(b, n - b);
  long long v = 1;
  for (int i = 0; i < e && v < chi_max; ++i) v *= 4;
  return (int)std::min<long long>(v, chi_max);
}

// ------------------------------------------------------- eigen-solve launch --
// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device. The limit is a property of the function shared by every
// host thread (the batching form launches from several), so it only ever
// grows: a thread that needs less never lowers it under another's launch.
static cudaError_t ensure_dynamic_smem(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cur;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  int& c = cur[std::make_pair(fn, dev)];
  if (bytes <= c) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) c = bytes;
  return e;
}

template <typename T>
static cudaError_t launch_jacobi(cudaStream_t st, cplx<T>* G, int m, cplx<T>* V, T* w, GridCtl* ctl,
                                 int max_sweeps, double timeout_s, int num_sms) {
  const int N = m + (m & 1);
  const size_t smem = sizeof(JRot<T>) * (size_t)std::max(1, N / 2);
  cudaError_t e = ensure_dynamic_smem((const void*)jacobi_kernel<T>, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel<T>, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int coresident = per_sm * num_sms;
  int want = (2 * m + 7) / 8;   // one warp per row of G and V in phase B
  int blocks = std::max(1, std::min(coresident, want));
  e = cudaMemsetAsync(ctl, 0, sizeof(GridCtl), st);
  if (e != cudaSuccess) return e;
  const T tol_rel = std::is_same<T, double>::value ? (T)1e-14 : (T)2e-6;
  const T floor_rel = eps_of<T>::value;
  long long timeout_ns = (long long)(timeout_s * 1e9);
  void* args[] = {&G, &m, &V, &w, &ctl, &max_sweeps, (void*)&tol_rel, (void*)&floor_rel, &timeout_ns};
  return cudaLaunchCooperativeKernel((const void*)jacobi_kernel<T>, dim3(blocks), dim3(256), args, smem, st);
}

template <typename T>
static cudaError_t launch_select(cudaStream_t st, const T* w, int m, int cap, double cutoff2, int* perm,
                                 double* lam2, SelectInfo* info, double* disc, double* lognorm, double* S,
                                 double* sch, const double* total_in = nullptr) {
  int P = 1;
  while (P < m) P <<= 1;
  const size_t smem = (size_t)P * (sizeof(double) + sizeof(int));
  cudaError_t e = ensure_dynamic_smem((const void*)select_kernel<T>, (int)smem);
  if (e != cudaSuccess) return e;
  select_kernel<T><<<1, 1024, smem, st>>>(w, m, cap, cutoff2, perm, lam2, info, disc, lognorm, S, sch, total_in);
  return cudaGetLastError();
}

static int grid_for(size_t work, int num_sms) {
  size_t b = (work + 255) / 256;
  size_t mx = (size_t)num_sms * 16;
  return (int)std::max<size_t>(1, std::min(b, mx));
}

template <typename T>
static cudaError_t launch_onesided(cudaStream_t st, cplx<T>* X, int r, int c, int ldx, cplx<T>* Ut, T* w, OSCtl* ctl,
                                   int max_sweeps, double timeout_s, int num_sms, double tol_min = 0.0) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, onesided_jacobi_kernel<T>, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int N = r + (r & 1);
  // one warp per pair; at least one CTA per SM so that the FP64 units of every
  // SM take part even when the pairs are few
  const int want = std::max(num_sms, (N / 2 + 7) / 8);
  const int blocks = std::max(1, std::min(per_sm * num_sms, want));
  e = cudaMemsetAsync(ctl, 0, sizeof(OSCtl), st);
  if (e != cudaSuccess) return e;
  // rows count as orthogonal once |<x_p, x_q>| <= 2 eps sqrt(c) ||x_p|| ||x_q||,
  // the rounding level of the length-c dot product itself
  const T tol_rel = (T)std::max(tol_min, 2.0 * eps_of<T>::value * std::sqrt((double)std::max(c, 1)));
  const T floor_rel = eps_of<T>::value * eps_of<T>::value;
  long long timeout_ns = (long long)(timeout_s * 1e9);
  void* args[] = {&X, &r, &c, &ldx, &Ut, &w, &ctl, &max_sweeps, (void*)&tol_rel, (void*)&floor_rel, &timeout_ns};
  return cudaLaunchCooperativeKernel((const void*)onesided_jacobi_kernel<T>, dim3(blocks), dim3(256), args, 0, st);
}

template <typename T>
static cudaError_t launch_block_jacobi(cudaStream_t st, cplx<T>* X, int r, int c, int ldx, cplx<T>* Ut, T* w,
                                      cplx<T>* Gpart, size_t gpart_slots, cplx<T>* Jbuf, int* act, size_t act_ints,
                                      OSCtl* ctl, int max_sweeps, double timeout_s, int num_sms) {
  const int smem = block_jacobi_smem_bytes<T>();
  cudaError_t e = ensure_dynamic_smem((const void*)block_jacobi_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, block_jacobi_kernel<T>, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int nb = (r + JB - 1) / JB, npairs = (nb + (nb & 1)) / 2;
  const size_t nch = (size_t)(c + JCW - 1) / JCW;
  if ((size_t)npairs * nch > gpart_slots || bj_state_ints(r) > act_ints) return cudaErrorInvalidValue;   // workspace too small
  const int items = npairs * ((c + JCW - 1) / JCW + (r + JCW - 1) / JCW);
  const int blocks = std::max(1, std::min(per_sm * num_sms, items));
  e = cudaMemsetAsync(ctl, 0, sizeof(OSCtl), st);
  if (e != cudaSuccess) return e;
  // relative criterion at the rounding level of a length-c dot product, but
  // never below twice the stopping level of the in-CTA pair solve (4 eps
  // sqrt(JP)) plus the rounding of applying a JP-term rotation: with short
  // rows (c < 16 JP) a tighter outer test than the inner solve can meet
  // makes the sweeps rotate the same pairs for ever; the absolute floor sits
  // above the rounding of the pair Gram itself, which the block rotation
  // cannot resolve below
  const T tol_rel = (T)(2.0 * eps_of<T>::value * std::max(std::sqrt((double)std::max(c, 1)), 4.0 * std::sqrt((double)JP)));
  const T floor_rel = (T)(16.0 * eps_of<T>::value * std::max(std::sqrt((double)std::max(c, 1)), 4.0));
  long long timeout_ns = (long long)(timeout_s * 1e9);
  void* args[] = {&X, &r, &c, &ldx, &Ut, &w, &Gpart, &Jbuf, &act, &ctl, &max_sweeps, (void*)&tol_rel,
                  (void*)&floor_rel, &timeout_ns};
  return cudaLaunchCooperativeKernel((const void*)block_jacobi_kernel<T>, dim3(blocks), dim3(256), args, smem, st);
}

// ---------------------------------------------------------------------------
// Precision form: truncated SVD of a complex128 matrix X (r x c, r <= c,
// leading dimension ldx) keeping at most cap singular values (App. A), with
// the heavy lifting in FP32 and the accuracy won back in FP64.
//   1. FP32 one-sided Jacobi SVD of fl32(X) -> approximate U (r x r), w.
//   2. Q (r x m, FP64) = the m = min(r, cap + oversample) leading columns of U,
//      made orthonormal to FP64 rounding by Newton-Schulz steps.
//   3. Optional (refine_steps > 0, only when m < r): subspace-iteration steps
//      W <- orth(X^H Q), Q <- orth(X W) in FP64, each damping the components
//      of the leading singular vectors outside span(Q) by
//      (sigma_{m+1} / sigma_j)^2; orth is shifted Cholesky QR followed by two
//      Cholesky QR passes (shifted CholeskyQR3, stable for condition numbers
//      up to 1/u), applied after each product so that a basis never carries
//      more than the condition number sigma_1 / sigma_m; the refined basis is
//      then turned back towards the FP32 one (Q <- Q W, W the orthonormal
//      factor of Q^H Q_FP32) so that the Rayleigh-Ritz matrix stays nearly
//      diagonal.
//   4. Rayleigh-Ritz in FP64: B = Q^H X (m x c), H = B B^H (m x m), both by
//      the FP64-class products, and the FP64 Hermitian Jacobi eigen-solve
//      H = V diag(w) V^H. With Q from the FP32 singular vectors H is nearly
//      diagonal, so the solve ends after a few sweeps. The Ritz values w are
//      the squared singular values, Q V the left singular vectors and the rows
//      of V^H B = Lambda W^H the scaled right ones.
// Outputs follow the one-sided Jacobi convention of svd_select: rows 0..m-1
// of X are overwritten with V^H B, h->vecs holds V^H Q^H (m x r, row j = conj
// of left singular vector j: h->vecs_conj), h->mx_w the w; the select kernel
// then sorts and truncates, with the discarded weight taken against the
// squared Frobenius norm of X (the Ritz values cover span(Q) only).
// ---------------------------------------------------------------------------
constexpr int kMixedMargin = 64;      // Ritz directions carried into the FP64 step beyond cap
constexpr int kMixedMaxSteps = 24;    // cap on subspace-iteration steps of one factorisation
constexpr int kMixedSteps = 4;        // steps before the first convergence check

// C (M x N) = alpha op(A) op(B) (+ C), complex128, FP64-accurate on the
// tensor cores (ozgemm.cuh): exponents, BF16 slices of both operands, then
// the MMA kernel. Returns cudaErrorInvalidValue if the scratch is too small.
static cudaError_t oz_gemm(cudaStream_t st, int M, int N, int K, const double2* A, int lda, int opA, const double2* B,
                           int ldb, int opB, double2* C, int ldc, double alpha, int accumulate, const OzWork& w,
                           double timeout_s, int num_sms) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int K8 = (std::max(K, 1) + 31) / 32 * 32;
  const int Mp = (M + oz::BM - 1) / oz::BM * oz::BM, Nrp = (2 * N + oz::BN - 1) / oz::BN * oz::BN;
  const size_t Kp = 2 * (size_t)K8;
  if ((size_t)oz::S * Mp * Kp > w.a_cap || (size_t)oz::S * Nrp * Kp > w.b_cap || Mp > w.e_cap || Nrp / 2 > w.e_cap)
    return cudaErrorInvalidValue;
  // scaling exponents: rows of op(A) are stored rows of A (op 0) or stored
  // columns (op 1); columns of op(B) are stored columns of B (op 0) or rows
  cudaError_t e0 = cudaMemsetAsync(w.ea, 0, sizeof(int) * (size_t)M, st);
  if (e0 == cudaSuccess) e0 = cudaMemsetAsync(w.eb, 0, sizeof(int) * (size_t)N, st);
  if (e0 != cudaSuccess) return e0;
  {
    const int Ra = opA ? K : M, Ca = opA ? M : K, Rb = opB ? N : K, Cb = opB ? K : N;
    oz_exp_kernel<<<dim3((Ca + 31) / 32, (Ra + 255) / 256), dim3(32, 8), 0, st>>>(A, lda, Ra, Ca, opA ? 0 : 1, w.ea);
    oz_exp_kernel<<<dim3((Cb + 31) / 32, (Rb + 255) / 256), dim3(32, 8), 0, st>>>(B, ldb, Rb, Cb, opB ? 1 : 0, w.eb);
  }
  oz_split_a_kernel<<<dim3(K8 / 32, Mp / 32), dim3(32, 8), 0, st>>>(A, lda, opA, M, K, K8, Mp, w.ea, w.a);
  oz_split_b_kernel<<<dim3(K8 / 32, Nrp / 64), dim3(32, 8), 0, st>>>(B, ldb, opB, K, N, K8, Nrp, w.eb, w.b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = ensure_dynamic_smem((const void*)oz_mma_kernel, oz::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  oz_mma_kernel<<<dim3(Nrp / oz::BN, Mp / oz::BM), oz::NT, oz::SMEM_BYTES, st>>>(
      M, N, (int)Kp, w.a, (size_t)Mp * Kp, w.b, (size_t)Nrp * Kp, w.ea, w.eb, C, ldc, alpha, accumulate, w.status,
      (long long)(timeout_s * 1e9));
  return cudaGetLastError();
}

// Allocate the scratch for products whose operands have at most dmax rows,
// columns and inner dimension.
static bool alloc_oz(OzWork& w, int dmax, size_t* bytes) {
  const size_t Mp = (size_t)(dmax + oz::BM - 1) / oz::BM * oz::BM;
  const size_t Nrp = (size_t)(2 * dmax + oz::BN - 1) / oz::BN * oz::BN;
  const size_t Kp = 2 * (size_t)((dmax + 31) / 32 * 32);
  w.a_cap = (size_t)oz::S * Mp * Kp;
  w.b_cap = (size_t)oz::S * Nrp * Kp;
  w.e_cap = (int)std::max(Mp, Nrp);
  bool ok = cudaMalloc((void**)&w.a, w.a_cap * sizeof(__nv_bfloat16)) == cudaSuccess &&
            cudaMalloc((void**)&w.b, w.b_cap * sizeof(__nv_bfloat16)) == cudaSuccess &&
            cudaMalloc((void**)&w.ea, w.e_cap * sizeof(int)) == cudaSuccess &&
            cudaMalloc((void**)&w.eb, w.e_cap * sizeof(int)) == cudaSuccess &&
            cudaMalloc((void**)&w.status, sizeof(int)) == cudaSuccess &&
            cudaMemset(w.status, 0, sizeof(int)) == cudaSuccess;
  if (!ok) cudaGetLastError();
  if (bytes) *bytes += (w.a_cap + w.b_cap) * sizeof(__nv_bfloat16) + 2 * w.e_cap * sizeof(int);
  return ok;
}

static void free_oz(OzWork& w) {
  cudaFree(w.a); cudaFree(w.b); cudaFree(w.ea); cudaFree(w.eb); cudaFree(w.status);
  w = OzWork();
}

// Products large enough to fill 128 x 128 real tiles go to the tensor cores.
// (SIMT FP64 runs at about 8 GFLOP/s per SM on this part, so even small
// products with few tiles are faster as split BF16 products.)
static bool oz_worth(int M, int N, int K) { return (double)M * N * K >= 2.6e5 && M >= 16 && N >= 8 && K >= 16; }

static cudaError_t mx_gemm(mpo_ctx* h, int M, int N, int K, const double2* A, int lda, int opA, const double2* B,
                           int ldb, int opB, double2* C, int ldc, double alpha = 1.0, int accumulate = 0) {
  ProfScope ps(h, PK_REFINE, 8.0 * M * N * K, (double)((size_t)M * K + (size_t)K * N + (size_t)M * N) * sizeof(double2));
  if (h->use_oz && oz_worth(M, N, K)) {
    ps.cls = PK_OZ;
    return oz_gemm(h->st, M, N, K, A, lda, opA, B, ldb, opB, C, ldc, alpha, accumulate, h->oz,
                   h->opts.barrier_timeout_s, h->num_sms);
  }
  return cgemm<double>(h->st, M, N, K, A, lda, opA, B, ldb, opB, C, ldc, nullptr, alpha, accumulate);
}

// Y (rows x m, leading dimension m) <- Y (3 I - Y^H Y) / 2, iters times
// (Newton-Schulz iteration for the orthonormal polar factor, Higham,
// Functions of Matrices, Sec. 8.3): each step squares the defect
// |Y^H Y - I|, so a basis orthonormal to ~1e-3 reaches FP64 rounding in four
// steps. The result is left in Y (spare is scratch; the two are swapped).
static int mx_newton_schulz(mpo_ctx* h, double2*& Y, double2*& spare, int rows, int m, int iters,
                            double* defect_dev = nullptr) {
  for (int it = 0; it < iters; ++it) {
    CK(h, mx_gemm(h, m, m, rows, Y, m, 1, Y, m, 0, h->mx_G, m));
    if (defect_dev && it == iters - 1) {   // |Y^H Y - I| entering the last step
      CK(h, cudaMemsetAsync(defect_dev, 0, sizeof(double), h->st));
      defect_kernel<<<grid_for((size_t)m * m, h->num_sms), 256, 0, h->st>>>(h->mx_G, m, defect_dev);
      CK(h, cudaGetLastError());
    }
    {
      ProfScope ps(h, PK_REFINE, 0.0, 2.0 * m * m * sizeof(double2));
      ns_multiplier_kernel<<<grid_for((size_t)m * m, h->num_sms), 256, 0, h->st>>>(h->mx_G, m);
      CK(h, cudaGetLastError());
    }
    CK(h, mx_gemm(h, rows, m, m, Y, m, 0, h->mx_G, m, 0, spare, m));
    std::swap(Y, spare);
  }
  return MPO_OK;
}

// FP32 Cholesky factorisation of the Hermitian block A[k0:k0+s, k0:k0+s]
// (leading dimension m) into L (lower triangle, in place) and L^{-1} into the
// same block of Li, by recursive halving: with A = [[A11, .], [A21, A22]],
//   L11, L11^{-1} <- recursion on A11;  L21 = A21 L11^{-H};
//   A22 -= L21 L21^H;  L22, L22^{-1} <- recursion on A22;
//   (L^{-1})_21 = -L22^{-1} L21 L11^{-1}.
// Blocks of at most CHOL32_NB rows are factored by chol_diag_kernel, the rest
// by FP32 GEMMs. Li is zero above the diagonal blocks on entry.
static int chol32_rec(mpo_ctx* h, float2* A, float2* Li, int m, int k0, int s) {
  if (s <= CHOL32_NB) {
    chol_diag_kernel<float, CHOL32_NB><<<1, 256, chol_smem_bytes<float, CHOL32_NB>(), h->st>>>(
        A, m, k0, s, Li + (size_t)k0 * m + k0, m, h->mx_chst);
    CK(h, cudaGetLastError());
    return MPO_OK;
  }
  const int s1 = std::min(s - 1, (s / 2 + CHOL32_NB - 1) / CHOL32_NB * CHOL32_NB), s2 = s - s1;
  int rc = chol32_rec(h, A, Li, m, k0, s1);
  if (rc) return rc;
  float2* A21 = A + (size_t)(k0 + s1) * m + k0;
  float2* A22 = A21 + s1;
  const float2* Li11 = Li + (size_t)k0 * m + k0;
  float2* Li21 = Li + (size_t)(k0 + s1) * m + k0;
  const float2* Li22 = Li21 + s1;
  float2* T = h->mx_t32;                                                                // s2 x s1
  CK(h, cgemm<float>(h->st, s2, s1, s1, A21, m, 0, Li11, m, 1, T, s1));                 // L21 = A21 L11^{-H}
  CK(h, cudaMemcpy2DAsync(A21, (size_t)m * sizeof(float2), T, (size_t)s1 * sizeof(float2),
                          (size_t)s1 * sizeof(float2), s2, cudaMemcpyDeviceToDevice, h->st));
  CK(h, cgemm<float>(h->st, s2, s2, s1, A21, m, 0, A21, m, 1, A22, m, nullptr, -1.0, 1));   // A22 -= L21 L21^H
  rc = chol32_rec(h, A, Li, m, k0 + s1, s2);
  if (rc) return rc;
  CK(h, cgemm<float>(h->st, s2, s1, s1, A21, m, 0, Li11, m, 0, T, s1));                 // L21 L11^{-1}
  CK(h, cgemm<float>(h->st, s2, s1, s2, Li22, m, 0, T, s1, 0, Li21, m, nullptr, -1.0, 0));   // -L22^{-1} (.)
  return MPO_OK;
}

// One mixed-precision Cholesky QR pass on Y (rows x m, leading dimension m):
// G = Y^H Y by the FP64-class product, A = fl32(D G D) + shift I with
// D = diag(G)^{-1/2}, the FP32 factorisation A = L L^H with L^{-1}, and
// Y <- Y D L^{-H} by the FP64-class product (result in Y; spare is scratch).
// The shift, 8 m u_32, bounds the FP32 rounding of A and of its
// factorisation, so A stays positive definite whatever the conditioning of
// Y; a pass takes a condition number kappa of Y to about sqrt(shift) kappa
// (and no lower than 1 + shift). Mixed-precision Cholesky QR: Yamazaki,
// Tomov & Dongarra, SIAM J. Sci. Comput. 37 (2015); the shift: Fukaya,
// Kannan, Nakatsukasa, Yamamoto & Yanagisawa, SIAM J. Sci. Comput. 42 (2020).
static int mx_cholqr_pass(mpo_ctx* h, double2*& Y, double2*& spare, int rows, int m) {
  CK(h, mx_gemm(h, m, m, rows, Y, m, 1, Y, m, 0, h->mx_G, m));
  {
    ProfScope ps(h, PK_REFINE, 16.0 * m * m * m / 3.0, 6.0 * m * m * sizeof(float2));
    const float shift = (float)(8.0 * m * 5.9604644775390625e-08);
    scale_gram_fp32_kernel<<<grid_for((size_t)m * m, h->num_sms), 256, 0, h->st>>>(h->mx_G, m, shift, h->mx_A32,
                                                                                      h->mx_d);
    CK(h, cudaGetLastError());
    CK(h, cudaMemsetAsync(h->mx_Li32, 0, (size_t)m * m * sizeof(float2), h->st));
    int rc = chol32_rec(h, h->mx_A32, h->mx_Li32, m, 0, m);
    if (rc) return rc;
    form_w_kernel<<<grid_for((size_t)m * m, h->num_sms), 256, 0, h->st>>>(h->mx_Li32, h->mx_d, m, h->mx_W);
    CK(h, cudaGetLastError());
  }
  CK(h, mx_gemm(h, rows, m, m, Y, m, 0, h->mx_W, m, 0, spare, m));
  std::swap(Y, spare);
  return MPO_OK;
}

static int mx_cholqr(mpo_ctx* h, double2*& Y, double2*& spare, int rows, int m, int passes) {
  for (int p = 0; p < passes; ++p) {
    int rc = mx_cholqr_pass(h, Y, spare, rows, m);
    if (rc) return rc;
  }
  return MPO_OK;
}

// Subspace-iteration steps Q <- orth(X orth(X^H Q)) on Q (r x m). Each half
// step is followed by three Cholesky QR passes, which hold the basis
// condition number near 1 although every product multiplies it by up to
// sigma_1 / sigma_m (each pass divides it by about 30).
static int mx_subspace_steps(mpo_ctx* h, const double2* X, int r, int c, int ldx, int m, int steps) {
  const int passes = 3;
  for (int it = 0; it < steps; ++it) {
    CK(h, mx_gemm(h, c, m, r, X, ldx, 1, h->mx_Q, m, 0, h->mx_T, m));     // T = X^H Q (c x m)
    int rc = mx_cholqr(h, h->mx_T, h->mx_B, c, m, passes);
    if (rc) return rc;
    CK(h, mx_gemm(h, r, m, c, X, ldx, 0, h->mx_T, m, 0, h->mx_Q, m));     // Q = X T (r x m)
    rc = mx_cholqr(h, h->mx_Q, h->mx_Q2, r, m, passes);
    if (rc) return rc;
  }
  return MPO_OK;
}

static int msvd_status(mpo_ctx* h) {
  if (h->hs->ctl.err) return fail(h, MPO_ERR_TIMEOUT, "grid barrier wait timed out in the FP32 Rayleigh-Ritz SVD");
  if (h->hs->ctl.status) return fail(h, MPO_ERR_NOCONV, "FP32 Rayleigh-Ritz SVD reached eig_max_sweeps");
  if (h->use_oz && h->hs->oz_err) return fail(h, MPO_ERR_TIMEOUT, "an mbarrier wait timed out in the tensor-core FP64 GEMM");
  if (h->hs->chol_status) return fail(h, MPO_ERR_NOCONV, "Cholesky QR met a non-positive pivot");
  return MPO_OK;
}

static int msvd_select(mpo_ctx* h, double2* X, int r, int c, int ldx, int cap, bool disc, double* S, double* sch, int* k) {
  const int m = std::min(r, cap + h->mx_over);          // dimension of the iterated subspace
  const int mp = std::min(m, cap + kMixedMargin);        // dimension of the FP64 Rayleigh-Ritz step
  if (m > h->mx_mcap || r > h->m_cap) return fail(h, MPO_ERR_STATE, "mixed factorisation larger than its workspace");
  const bool iterate = m < r;
  CK(h, cudaMemsetAsync(h->mx_chst, 0, sizeof(int), h->st));
  {
    ProfScope ps(h, PK_CONVERT, 0.0, (double)r * c * sizeof(double2));
    CK(h, cudaMemsetAsync(h->scal + 2, 0, sizeof(double), h->st));
    frob2_kernel<<<grid_for((size_t)r * c, h->num_sms), 256, 0, h->st>>>(X, r, c, ldx, h->scal + 2);   // ||X||_F^2
    CK(h, cudaGetLastError());
  }
  int rc = MPO_OK, steps = 0;
  // the step count this bond needed last time, plus one (the spectra of
  // successive gates on a bond change slowly, and a step costs far less than
  // the second FP32 Rayleigh-Ritz step that too few steps force)
  const int remembered = (h->mx_cur_bond >= 0 && h->mx_cur_bond < (int)h->mx_bond_steps.size())
                             ? h->mx_bond_steps[h->mx_cur_bond] : 0;
  if (iterate) {
    // 1. seeded Gaussian start and the first steps of the subspace iteration
    {
      ProfScope ps(h, PK_CONVERT, 0.0, (double)c * m * sizeof(double2));
      h->mx_seed += 0x9E3779B97F4A7C15ull;
      gauss_start_kernel<<<grid_for((size_t)c * m, h->num_sms), 256, 0, h->st>>>(h->mx_T, (size_t)c * m, h->mx_seed);
      CK(h, cudaGetLastError());
    }
    CK(h, mx_gemm(h, r, m, c, X, ldx, 0, h->mx_T, m, 0, h->mx_Q, m));     // Q = X Omega
    rc = mx_cholqr(h, h->mx_Q, h->mx_Q2, r, m, 3);
    if (rc) return rc;
    steps = std::max(std::max(1, h->mx_steps), remembered > 0 ? remembered + 1 : 0);
    rc = mx_subspace_steps(h, X, r, c, ldx, m, steps);
    if (rc) return rc;
  }
  // 2. FP32 Rayleigh-Ritz (stage 1). The leading cap directions keep
  // components outside span(Q) of order (sigma_{m+1} / sigma_cap)^(2 steps),
  // estimated from the FP32 Ritz values as (w_m / w_cap)^steps; above 1e-7
  // the iteration takes the steps that bring the estimate to 1e-8 and the
  // FP32 step is repeated (the kept-theta error is about 2e-2 of the estimate)
  for (;;) {
    // the FP32 solve runs on M = Q^H X T (m x m; T the orthonormal basis of
    // the last half step, so M M^H = Q^H X X^H Q up to the iteration's
    // residual) rather than on B = Q^H X (m x c), and stops at relative
    // couplings of 3e-5: the first-order correction below and the FP64 step
    // remove what the FP32 solve leaves
    const int c1 = iterate ? m : c;
    if (iterate) {
      rc = mx_newton_schulz(h, h->mx_Q, h->mx_Q2, r, m, 2, h->scal + 3);
      if (rc) return rc;
      rc = mx_newton_schulz(h, h->mx_T, h->mx_B, c, m, 2, h->scal + 4);
      if (rc) return rc;
      CK(h, mx_gemm(h, m, c, r, h->mx_Q, m, 1, X, ldx, 0, h->mx_B, c));   // B = Q^H X (m x c)
      CK(h, mx_gemm(h, m, m, c, h->mx_B, c, 0, h->mx_T, m, 0, h->mx_W, m));  // M = B T (m x m)
    }
    {
      ProfScope ps(h, PK_CONVERT, 0.0, (double)m * c1 * (sizeof(double2) + sizeof(float2)));
      to_fp32_kernel<<<grid_for((size_t)m * c1, h->num_sms), 256, 0, h->st>>>(iterate ? h->mx_W : X, m, c1,
                                                                              iterate ? m : ldx, h->mx_a32);
      CK(h, cudaGetLastError());
    }
    {
      const double fm = m, fc = c1;
      ProfScope ps(h, disc ? PK_SVD : PK_SVD_SWEEP, 4.0 * fm * fm * fc, (2.0 * fm * fc + fm * fm) * sizeof(float2));
      CK(h, launch_onesided<float>(h->st, h->mx_a32, m, c1, c1, h->mx_ut32, h->mx_w32, h->osctl,
                                   h->opts.eig_max_sweeps, h->opts.barrier_timeout_s, h->num_sms, 3e-5));
    }
    {
      ProfScope ps(h, PK_SELECT, 0.0, (double)m * (sizeof(float) + sizeof(int) + sizeof(double)));
      CK(h, launch_select<float>(h->st, h->mx_w32, m, m, -1.0, h->mx_perm32, h->mx_lam32, h->mx_info32, nullptr,
                                 nullptr, nullptr, nullptr));
    }
    if (!iterate) break;
    double rd[4];   // w_cap, w_m, the two orthonormality defects
    CK(h, cudaMemcpyAsync(&rd[0], h->mx_lam32 + (cap - 1), sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaMemcpyAsync(&rd[1], h->mx_lam32 + (m - 1), sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaMemcpyAsync(&rd[2], h->scal + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaMemcpyAsync(&h->hs->ctl, &h->osctl->g, sizeof(GridCtl), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaMemcpyAsync(&h->hs->chol_status, h->mx_chst, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    if (h->use_oz) CK(h, cudaMemcpyAsync(&h->hs->oz_err, h->oz.status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    rc = msvd_status(h);
    if (rc) return rc;
    if (!(std::max(rd[2], rd[3]) <= 1e-3))
      return fail(h, MPO_ERR_NOCONV, "subspace basis not orthonormal after Cholesky QR");
    const double rho2 = rd[0] > 0.0 ? std::max(0.0, rd[1]) / rd[0] : 0.0;
    if (steps >= kMixedMaxSteps || rho2 <= 0.0 || std::pow(rho2, steps) <= 1e-7) break;
    const int need = rho2 < 1.0 ? (int)std::ceil(std::log(1e-8) / std::log(rho2)) : kMixedMaxSteps;
    const int more = std::max(1, std::min(need, kMixedMaxSteps) - steps);
    rc = mx_subspace_steps(h, X, r, c, ldx, m, more);
    if (rc) return rc;
    steps += more;
  }
  h->mx_last_steps = steps;
  if (h->prof) h->prof_steps += steps;
  if (iterate && h->mx_cur_bond >= 0 && h->mx_cur_bond < (int)h->mx_bond_steps.size())
    h->mx_bond_steps[h->mx_cur_bond] = steps;
  // 3. the mp leading FP32 Ritz directions V_P (V = U32 in descending order,
  // promoted), corrected to first order for their error along the other
  // m - mp directions (the FP32 solve leaves couplings of 2 eps_32 sqrt(c)
  // relative, which would otherwise leak into the kept subspace), then
  // Q' = Q V_P made orthonormal in FP64
  double2* Qp = h->mx_Q0;
  double2* Qsp = h->mx_Q2;
  {
    ProfScope ps(h, PK_CONVERT, 0.0, (double)m * m * (sizeof(double2) + sizeof(float2)));
    promote_columns_kernel<<<grid_for((size_t)m * m, h->num_sms), 256, 0, h->st>>>(h->mx_ut32, m, h->mx_perm32, m,
                                                                                      h->mx_W);
    CK(h, cudaGetLastError());
  }
  if (mp < m) {
    const double2* Bs = iterate ? h->mx_B : X;
    const int ldbs = iterate ? c : ldx;
    CK(h, mx_gemm(h, m, c, m, h->mx_W, m, 1, Bs, ldbs, 0, h->mx_T, c));        // V^H B (m x c)
    CK(h, mx_gemm(h, m, m, c, h->mx_T, c, 0, h->mx_T, c, 1, h->mx_G, m));      // S = V^H H V
    CK(h, mx_gemm(h, m, m, m, h->mx_W, m, 1, h->mx_W, m, 0, h->mx_V, m));      // G = V^H V
    {
      ProfScope ps(h, PK_REFINE, 0.0, 3.0 * (double)m * mp * sizeof(double2));
      partition_correction_kernel<<<grid_for((size_t)(m - mp) * mp, h->num_sms), 256, 0, h->st>>>(
          h->mx_G, h->mx_V, m, mp, h->mx_B);
      CK(h, cudaGetLastError());
    }
    CK(h, mx_gemm(h, m, mp, m - mp, h->mx_W + mp, m, 0, h->mx_B, mp, 0, h->mx_W, m, 1.0, 1));   // V_P += V_R E
  }
  if (iterate) {
    CK(h, mx_gemm(h, r, mp, m, h->mx_Q, m, 0, h->mx_W, m, 0, Qp, mp));
  } else {
    CK(h, cudaMemcpy2DAsync(Qp, (size_t)mp * sizeof(double2), h->mx_W, (size_t)m * sizeof(double2),
                            (size_t)mp * sizeof(double2), r, cudaMemcpyDeviceToDevice, h->st));
  }
  rc = mx_newton_schulz(h, Qp, Qsp, r, mp, 3);
  if (rc) return rc;
  // 4. FP64 Rayleigh-Ritz (stage 2): B' = Q'^H X, H' = B' B'^H, nearly
  // diagonal, and the FP64 Hermitian Jacobi eigen-solve H' = V diag(w) V^H
  CK(h, mx_gemm(h, mp, c, r, Qp, mp, 1, X, ldx, 0, h->mx_B, c));            // B' (mp x c)
  CK(h, mx_gemm(h, mp, mp, c, h->mx_B, c, 0, h->mx_B, c, 1, h->mx_G, mp));  // H' (mp x mp)
  {
    ProfScope ps(h, PK_EIG64, 13.3 * (double)mp * mp * mp, 3.0 * (double)mp * mp * sizeof(double2));
    hermitise_kernel<<<grid_for((size_t)mp * mp, h->num_sms), 256, 0, h->st>>>(h->mx_G, mp);
    CK(h, cudaGetLastError());
    CK(h, launch_jacobi<double>(h->st, h->mx_G, mp, h->mx_V, h->mx_w, &h->mx_eosctl->g, h->opts.eig_max_sweeps,
                                h->opts.barrier_timeout_s, h->num_sms));
  }
  // left factor Q' V, stored as rows conj(column j) = V^H Q'^H; the rows
  // V^H B' = Lambda W^H go to X
  CK(h, mx_gemm(h, mp, c, mp, h->mx_V, mp, 1, h->mx_B, c, 0, X, ldx));
  CK(h, mx_gemm(h, mp, r, mp, h->mx_V, mp, 1, Qp, mp, 1, (double2*)h->vecs, r));
  h->vecs_conj = true;
  {
    ProfScope ps(h, PK_SELECT, 0.0, (double)mp * (sizeof(double) + sizeof(int) + sizeof(double)));
    CK(h, launch_select<double>(h->st, h->mx_w, mp, cap, h->cutoff * h->cutoff, h->perm, h->lam2, h->info,
                                disc ? h->scal + 1 : nullptr, h->scal, S, sch, h->scal + 2));
  }
  CK(h, cudaMemcpyAsync(&h->hs->info, h->info, sizeof(SelectInfo), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaMemcpyAsync(&h->hs->ctl, &h->osctl->g, sizeof(GridCtl), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaMemcpyAsync(&h->hs->chol_status, h->mx_chst, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaMemcpyAsync(h->hs->eig, &h->mx_eosctl->g, sizeof(GridCtl), cudaMemcpyDeviceToHost, h->st));
  if (h->use_oz) CK(h, cudaMemcpyAsync(&h->hs->oz_err, h->oz.status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  rc = msvd_status(h);
  if (rc) return rc;
  h->last_sweeps = h->hs->ctl.sweeps;
  h->prof_sweeps += h->prof ? h->hs->ctl.sweeps : 0;
  if (h->hs->eig[0].err) return fail(h, MPO_ERR_TIMEOUT, "grid barrier wait timed out in the FP64 Rayleigh-Ritz eigen-solve");
  if (h->hs->eig[0].status)
    return fail(h, MPO_ERR_NOCONV, "FP64 Rayleigh-Ritz eigen-solve reached eig_max_sweeps (m = " + std::to_string(mp) + ")");
  *k = h->hs->info.k;
  return MPO_OK;
}

// One-sided Jacobi SVD of X (r x c, rows orthogonalised in place; left factor
// transposed in h->vecs), then select the kept squared singular values; waits
// for the stream and returns the kept count in *k (or an error code).
template <typename T>
static int svd_select(mpo_ctx* h, cplx<T>* X, int r, int c, int ldx, int cap, bool disc, double* S, double* sch, int* k) {
  if constexpr (std::is_same<T, double>::value) {
    if (h->mixed) return msvd_select(h, X, r, c, ldx, cap, disc, S, sch, k);
  }
  h->vecs_conj = false;
  T* w = (T*)h->wv;
  {
    // algorithmic work of the factorisation: Hermitian Gram of the short side
    // (4 mn^2 mx real flops), projection onto the kept vectors (8 k mn mx) and
    // the dense Hermitian eigen-decomposition (13.3 mn^3); bytes: read and
    // write X, write U
    const double mn = std::min(r, c), mx = std::max(r, c), kk = std::min(cap, (int)mn);
    ProfScope ps(h, disc ? PK_SVD : PK_SVD_SWEEP, 4.0 * mn * mn * mx + 8.0 * kk * mn * mx + 13.3 * mn * mn * mn,
                 (2.0 * r * c + (double)r * r) * sizeof(cplx<T>));
    if (h->block_min_rows > 0 && r >= h->block_min_rows)
      CK(h, launch_block_jacobi<T>(h->st, X, r, c, ldx, (cplx<T>*)h->vecs, w, (cplx<T>*)h->bj_gpart, h->bj_slots,
                                   (cplx<T>*)h->bj_j, h->bj_act, h->bj_act_ints, h->osctl, h->opts.eig_max_sweeps,
                                   h->opts.barrier_timeout_s, h->num_sms));
    else
      CK(h, launch_onesided<T>(h->st, X, r, c, ldx, (cplx<T>*)h->vecs, w, h->osctl, h->opts.eig_max_sweeps,
                               h->opts.barrier_timeout_s, h->num_sms));
  }
  {
    ProfScope ps(h, PK_SELECT, 0.0, (double)r * (sizeof(T) + sizeof(int) + sizeof(double)));
    CK(h, launch_select<T>(h->st, w, r, cap, h->cutoff * h->cutoff, h->perm, h->lam2, h->info,
                           disc ? h->scal + 1 : nullptr, h->scal, S, sch));
  }
  CK(h, cudaMemcpyAsync(&h->hs->info, h->info, sizeof(SelectInfo), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaMemcpyAsync(&h->hs->ctl, &h->osctl->g, sizeof(GridCtl), cudaMemcpyDeviceToHost, h->st));
  if (h->prof) CK(h, cudaMemcpyAsync(h->hs->phase_ns, h->osctl->phase_ns, sizeof(h->hs->phase_ns), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaMemcpyAsync(&h->hs->tc_err, h->tc_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  if (h->hs->tc_err) return fail(h, MPO_ERR_TIMEOUT, "an mbarrier wait timed out in the tensor-core GEMM");
  if (h->prof) for (int i = 0; i < 3; ++i) h->prof_phase_ns[i] += h->hs->phase_ns[i];
  if (h->hs->ctl.err) return fail(h, MPO_ERR_TIMEOUT, "grid barrier wait timed out in the SVD");
  h->last_sweeps = h->hs->ctl.sweeps;
  h->prof_sweeps += h->prof ? h->hs->ctl.sweeps : 0;
  if (h->hs->ctl.status)
    return fail(h, MPO_ERR_NOCONV, "Jacobi SVD reached eig_max_sweeps (" + std::to_string(r) + " x " + std::to_string(c) + ")");
  *k = h->hs->info.k;
  return MPO_OK;
}

template <typename T> static cplx<T>* S_(mpo_ctx* h, int k) { return (cplx<T>*)h->site[k]; }

// Plain complex64 products large enough to fill a 128 x 64 tile go to the
// tensor cores (tcgen05, 3 x TF32); everything else runs on the SIMT kernel.
static cudaError_t tc_cgemm(cudaStream_t st, int M, int N, int K, const float2* A, int lda, const float2* B, int ldb,
                            float2* C, int ldc, const double* alpha_dev, double alpha_host, int* status,
                            double timeout_s) {
  {
    cudaError_t e = ensure_dynamic_smem((const void*)tc_cgemm_kernel, tcg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((N + tcg::BNC - 1) / tcg::BNC, (M + tcg::BM - 1) / tcg::BM);
  tc_cgemm_kernel<<<grid, 128, tcg::SMEM_BYTES, st>>>(M, N, K, A, lda, B, ldb, C, ldc, alpha_dev, alpha_host, status,
                                                        (long long)(timeout_s * 1e9));
  return cudaGetLastError();
}

static bool use_tensor_cores(int M, int N, int K) { return M >= 64 && N >= 32 && K >= 16; }

template <typename T>
static cudaError_t gemm_p(mpo_ctx* h, int M, int N, int K, const cplx<T>* A, int lda, int opA, const cplx<T>* B,
                          int ldb, int opB, cplx<T>* C, int ldc, const double* alpha_dev = nullptr) {
  ProfScope ps(h, PK_GEMM, 8.0 * M * N * K, (double)((size_t)M * K + (size_t)K * N + (size_t)M * N) * sizeof(cplx<T>));
  if constexpr (std::is_same<T, double>::value) {
    if (h->use_oz && !alpha_dev && oz_worth(M, N, K)) {
      ps.cls = PK_OZ;
      return oz_gemm(h->st, M, N, K, A, lda, opA, B, ldb, opB, C, ldc, 1.0, 0, h->oz, h->opts.barrier_timeout_s,
                     h->num_sms);
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    if (h->tensor_cores && opA == 0 && opB == 0 && use_tensor_cores(M, N, K)) {
      ps.cls = PK_TCGEMM;
      return tc_cgemm(h->st, M, N, K, A, lda, B, ldb, C, ldc, alpha_dev, 1.0, h->tc_status, h->opts.barrier_timeout_s);
    }
  }
  return cgemm<T>(h->st, M, N, K, A, lda, opA, B, ldb, opB, C, ldc, alpha_dev, 1.0);
}

static void swap_spare(mpo_ctx* h, int k) { std::swap(h->site[k], h->spare); }

template <typename T>
static cudaError_t gather_rows(mpo_ctx* h, const cplx<T>* src, int lds, int len, int k, int transpose, int conj_,
                               int mode, cplx<T>* out, int ldo) {
  ProfScope ps(h, PK_GATHER, 0.0, 2.0 * len * k * sizeof(cplx<T>));
  gather_rows_kernel<T><<<grid_for((size_t)len * k, h->num_sms), 256, 0, h->st>>>(
      src, lds, len, h->perm, h->lam2, h->info, k, transpose, conj_, mode, out, ldo);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t conj_transpose(mpo_ctx* h, const cplx<T>* in, int r, int c, int ldi, cplx<T>* out, int ldo) {
  ProfScope ps(h, PK_TRANSPOSE, 0.0, 2.0 * r * c * sizeof(cplx<T>));
  dim3 grid((c + 31) / 32, (r + 31) / 32);
  conj_transpose_kernel<T><<<grid, dim3(32, 8), 0, h->st>>>(in, r, c, ldi, out, ldo);
  return cudaGetLastError();
}

// Centre at site k -> site k becomes a left isometry, centre moves to k+1.
// L(C) = Y^H with Y = U X' (one-sided SVD of Y): Q = X'^H Sigma^-1 -> site k,
// R = Sigma U^H / ||kept|| pushed into site k+1.
// Precision form, centre moves that record nothing: the centre C becomes an
// isometry by Cholesky QR instead of an SVD (the move needs a basis of the
// bond space, not its Schmidt decomposition; the state C = Q (Q^H C) is
// unchanged up to rounding). Y (rows x r) is orthonormalised by
// kMovePasses mixed-precision Cholesky QR passes, which take a condition
// number up to ~1e7 (the cutoff's 1e-7 floor on the bond weights) to about
// 1, and three Newton-Schulz steps to FP64 orthonormality. The orthonormality
// defect entering the last Newton-Schulz step (its Gram matrix) is read back:
// above 1e-5 the move falls back to the SVD route and returns 1.
constexpr int kMovePasses = 5;

static int mx_isometry(mpo_ctx* h, double2*& Y, int rows, int r, bool* ok) {
  double2* sp = h->mx_Q2;
  CK(h, cudaMemsetAsync(h->mx_chst, 0, sizeof(int), h->st));
  int rc = mx_cholqr(h, Y, sp, rows, r, kMovePasses);
  if (rc) return rc;
  rc = mx_newton_schulz(h, Y, sp, rows, r, 2);
  if (rc) return rc;
  CK(h, mx_gemm(h, r, r, rows, Y, r, 1, Y, r, 0, h->mx_G, r));
  CK(h, cudaMemsetAsync(h->scal + 3, 0, sizeof(double), h->st));
  defect_kernel<<<grid_for((size_t)r * r, h->num_sms), 256, 0, h->st>>>(h->mx_G, r, h->scal + 3);
  CK(h, cudaGetLastError());
  rc = mx_newton_schulz(h, Y, sp, rows, r, 1);
  if (rc) return rc;
  double defect = 1.0;
  CK(h, cudaMemcpyAsync(&defect, h->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaMemcpyAsync(&h->hs->chol_status, h->mx_chst, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  if (h->use_oz) CK(h, cudaMemcpyAsync(&h->hs->oz_err, h->oz.status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  if (h->use_oz && h->hs->oz_err) return fail(h, MPO_ERR_TIMEOUT, "an mbarrier wait timed out in the tensor-core FP64 GEMM");
  *ok = !h->hs->chol_status && defect <= 1e-5;
  return MPO_OK;
}

static int mx_move_right(mpo_ctx* h, int k, bool* done) {
  const int mX = 4 * h->chi[k], r = h->chi[k + 1], mR = 4 * h->chi[k + 2];
  double2* C = (double2*)h->site[k];                                          // mX x r
  double2* Y = h->mx_Q;
  CK(h, cudaMemcpyAsync(Y, C, (size_t)mX * r * sizeof(double2), cudaMemcpyDeviceToDevice, h->st));
  int rc = mx_isometry(h, Y, mX, r, done);
  if (rc || !*done) return rc;
  CK(h, mx_gemm(h, r, r, mX, Y, r, 1, C, r, 0, h->mx_W, r));                 // R = Q^H C
  CK(h, mx_gemm(h, r, mR, r, h->mx_W, r, 0, (const double2*)h->site[k + 1], mR, 0, (double2*)h->spare, mR));
  swap_spare(h, k + 1);
  CK(h, cudaMemcpyAsync(h->spare, Y, (size_t)mX * r * sizeof(double2), cudaMemcpyDeviceToDevice, h->st));
  swap_spare(h, k);
  h->centre = k + 1;
  return MPO_OK;
}

static int mx_move_left(mpo_ctx* h, int k, bool* done) {
  const int r = h->chi[k], mR = 4 * h->chi[k + 1], mL = 4 * h->chi[k - 1];
  double2* C = (double2*)h->site[k];                                          // r x mR
  double2* Y = h->mx_Q;
  CK(h, conj_transpose<double>(h, C, r, mR, mR, Y, r));                       // C^H (mR x r)
  int rc = mx_isometry(h, Y, mR, r, done);
  if (rc || !*done) return rc;
  CK(h, mx_gemm(h, r, r, mR, C, mR, 0, Y, r, 0, h->mx_W, r));                // L = C Q
  CK(h, mx_gemm(h, mL, r, r, (const double2*)h->site[k - 1], r, 0, h->mx_W, r, 0, (double2*)h->spare, r));
  swap_spare(h, k - 1);
  CK(h, conj_transpose<double>(h, Y, mR, r, r, (double2*)h->spare, mR));     // Q^H (r x mR)
  swap_spare(h, k);
  h->centre = k - 1;
  return MPO_OK;
}

template <typename T>
static int move_right(mpo_ctx* h, int k) {
  if constexpr (std::is_same<T, double>::value) {
    if (h->mixed) {
      bool done = false;
      int rc0 = mx_move_right(h, k, &done);
      if (rc0 || done) return rc0;
    }
  }
  const int mX = 4 * h->chi[k], r = h->chi[k + 1], mR = 4 * h->chi[k + 2];
  cplx<T>* Y = (cplx<T>*)h->theta2;
  cplx<T>* tmp = (cplx<T>*)h->tmp;
  CK(h, conj_transpose<T>(h, S_<T>(h, k), mX, r, r, Y, mX));                   // Y = L(C)^H (r x mX)
  int rk = 0;
  int rc = svd_select<T>(h, Y, r, mX, mX, r, false, nullptr, nullptr, &rk);
  if (rc) return rc;
  CK(h, gather_rows<T>(h, Y, mX, mX, rk, 1, 1, 1, (cplx<T>*)h->spare, rk));     // Q (mX x rk)
  swap_spare(h, k);
  CK(h, gather_rows<T>(h, (cplx<T>*)h->vecs, r, r, rk, 0, 1 ^ (int)h->vecs_conj, 2, tmp, r));   // R (rk x r)
  CK(h, gemm_p<T>(h, rk, mR, r, tmp, r, 0, S_<T>(h, k + 1), mR, 0, (cplx<T>*)h->spare, mR));
  swap_spare(h, k + 1);
  h->chi[k + 1] = rk;
  h->centre = k + 1;
  return MPO_OK;
}

// Centre at site k -> site k becomes a right isometry, centre moves to k-1.
// R(C) = U X' (one-sided SVD in place): Lambda^-1 X' -> site k,
// U Lambda / ||kept|| pushed into site k-1. The row norms of X' are the
// Schmidt values of bond k; with record they and the entropy are stored.
template <typename T>
static int move_left(mpo_ctx* h, int k, bool record) {
  if constexpr (std::is_same<T, double>::value) {
    if (h->mixed && !record) {
      bool done = false;
      int rc0 = mx_move_left(h, k, &done);
      if (rc0 || done) return rc0;
    }
  }
  const int r = h->chi[k], mR = 4 * h->chi[k + 1], mL = 4 * h->chi[k - 1];
  cplx<T>* Y = S_<T>(h, k);
  cplx<T>* tmp = (cplx<T>*)h->tmp;
  int rk = 0;
  double* S = record ? h->dS + (k - 1) : nullptr;
  double* sch = record ? h->dschmidt + (size_t)(k - 1) * h->chi_max : nullptr;
  int rc = svd_select<T>(h, Y, r, mR, mR, r, false, S, sch, &rk);
  if (rc) return rc;
  CK(h, gather_rows<T>(h, Y, mR, mR, rk, 0, 0, 1, (cplx<T>*)h->spare, mR));        // Lambda^-1 X'
  swap_spare(h, k);
  CK(h, gather_rows<T>(h, (cplx<T>*)h->vecs, r, r, rk, 1, (int)h->vecs_conj, 2, tmp, rk));   // U Lambda / ||kept||
  CK(h, gemm_p<T>(h, mL, rk, r, S_<T>(h, k - 1), r, 0, tmp, rk, 0, (cplx<T>*)h->spare, rk));
  swap_spare(h, k - 1);
  h->chi[k] = rk;
  h->centre = k - 1;
  if (record) {
    h->schmidt_len[k - 1] = rk;
    h->s_valid[k - 1] = 1;
  }
  return MPO_OK;
}

template <typename T>
static int move_centre(mpo_ctx* h, int lo, int hi) {
  while (h->centre < lo) { int rc = move_right<T>(h, h->centre); if (rc) return rc; }
  while (h->centre > hi) { int rc = move_left<T>(h, h->centre, false); if (rc) return rc; }
  return MPO_OK;
}

// One noisy gate on sites (i, i+1), superoperator M on the device.
template <typename T>
static int gate_update(mpo_ctx* h, int i, const cplx<T>* M) {
  int rc = move_centre<T>(h, i, i + 1);
  if (rc) return rc;
  const int chiL = h->chi[i], chiM = h->chi[i + 1], chiR = h->chi[i + 2];
  const int mL = 4 * chiL, mR = 4 * chiR;
  cplx<T>* A0 = S_<T>(h, i);
  cplx<T>* A1 = S_<T>(h, i + 1);
  cplx<T>* th = (cplx<T>*)h->theta;
  CK(h, gemm_p<T>(h, mL, mR, chiM, A0, chiM, 0, A1, mR, 0, th, mR));        // theta
  {
    ProfScope ps(h, PK_SUPEROP, 2048.0 * chiL * chiR, 32.0 * chiL * chiR * sizeof(cplx<T>));
    apply_superop_kernel<T><<<grid_for((size_t)chiL * chiR, h->num_sms), 256, 0, h->st>>>(th, chiL, chiR, M);
    CK(h, cudaGetLastError());
  }
  int k = 0;
  h->mx_cur_bond = i;
  if (mL <= mR) {
    // theta' = U X', rows of X' = Lambda W^H
    rc = svd_select<T>(h, th, mL, mR, mR, h->chi_max, true, nullptr, nullptr, &k);
    h->mx_cur_bond = -1;
    if (rc) return rc;
    CK(h, gather_rows<T>(h, (cplx<T>*)h->vecs, mL, mL, k, 1, (int)h->vecs_conj, 0, A0, k));   // U_k -> site i
    CK(h, gather_rows<T>(h, th, mR, mR, k, 0, 0, 3, A1, mR));                    // Lambda W^H / ||kept||
  } else {
    // theta'^H = U X'  =>  theta' = X'^H U^H
    cplx<T>* Y = (cplx<T>*)h->theta2;
    CK(h, conj_transpose<T>(h, th, mL, mR, mR, Y, mL));
    rc = svd_select<T>(h, Y, mR, mL, mL, h->chi_max, true, nullptr, nullptr, &k);
    h->mx_cur_bond = -1;
    if (rc) return rc;
    CK(h, gather_rows<T>(h, (cplx<T>*)h->vecs, mR, mR, k, 0, 1 ^ (int)h->vecs_conj, 2, A1, mR));   // Lambda U^H / ||kept||
    CK(h, gather_rows<T>(h, Y, mL, mL, k, 1, 1, 1, A0, k));                      // X'^H Lambda^-1
  }
  h->chi[i + 1] = k;
  h->centre = i + 1;
  return MPO_OK;
}

template <typename T>
static int sweep_all(mpo_ctx* h) {
  std::fill(h->s_valid.begin(), h->s_valid.end(), 0);
  if (h->opts.smode == MPO_S_CENTRE) {
    const int k = h->n / 2;
    int rc = move_centre<T>(h, k, k);
    if (rc) return rc;
    return move_left<T>(h, k, true);
  }
  int rc = move_centre<T>(h, h->n - 1, h->n - 1);
  if (rc) return rc;
  for (int k = h->n - 1; k >= 1; --k) {
    rc = move_left<T>(h, k, true);
    if (rc) return rc;
  }
  return MPO_OK;
}

// ---------------------------------------------------------- gate staging ----
static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Stage ng gates and rates on the device and build their superoperators into h->Ms.
template <typename T>
static int stage_gates(mpo_ctx* h, int ng, const double* gates, const double* p, int p_stride) {
  const double2* dg = (const double2*)gates;
  if (!is_device_ptr(gates)) {
    CK(h, cudaMemcpyAsync(h->dgates, gates, sizeof(double2) * 16 * ng, cudaMemcpyHostToDevice, h->st));
    dg = h->dgates;
  }
  const double* dp = p;
  int stride = p_stride;
  if (!is_device_ptr(p)) {
    std::vector<double> hp(ng);
    for (int i = 0; i < ng; ++i) {
      hp[i] = p[(size_t)i * p_stride];
      if (!(hp[i] >= 0.0 && hp[i] <= 1.0)) return fail(h, MPO_ERR_ARG, "p must lie in [0, 1]");
    }
    CK(h, cudaMemcpyAsync(h->dp, hp.data(), sizeof(double) * ng, cudaMemcpyHostToDevice, h->st));
    CK(h, cudaStreamSynchronize(h->st));   // hp is a pageable temporary
    dp = h->dp;
    stride = 1;
  }
  build_superop_kernel<T><<<ng, 256, 0, h->st>>>(dg, dp, stride, (cplx<T>*)h->Ms);
  CK(h, cudaGetLastError());
  return MPO_OK;
}

// theta' = M (A_i A_{i+1}) of a noisy gate on ABI bond i, formed by the
// kernels of gate_update (centre move, contraction, superoperator) and copied
// to out without truncation; the state keeps its centre on the bond.
template <typename T>
static int theta_t(mpo_ctx* h, int i, const double* gate, double p, void* out, int* rows, int* cols) {
  int rc = move_centre<T>(h, i, i + 1);
  if (rc) return rc;
  const int chiL = h->chi[i], chiM = h->chi[i + 1], chiR = h->chi[i + 2];
  *rows = 4 * chiL;
  *cols = 4 * chiR;
  if (!out) return MPO_OK;
  rc = stage_gates<T>(h, 1, gate, &p, 0);
  if (rc) return rc;
  cplx<T>* th = (cplx<T>*)h->theta;
  CK(h, gemm_p<T>(h, 4 * chiL, 4 * chiR, chiM, S_<T>(h, i), chiM, 0, S_<T>(h, i + 1), 4 * chiR, 0, th, 4 * chiR));
  apply_superop_kernel<T><<<grid_for((size_t)chiL * chiR, h->num_sms), 256, 0, h->st>>>(th, chiL, chiR,
                                                                                         (const cplx<T>*)h->Ms);
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpyAsync(out, th, (size_t)16 * chiL * chiR * sizeof(cplx<T>), cudaMemcpyDefault, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  return MPO_OK;
}

template <typename T>
static int apply_layer_t(mpo_ctx* h, int parity, const double* gates, const double* p, int p_stride) {
  const int ng = (h->n - parity) / 2;   // parity 0: n/2 gates; parity 1: n/2 - 1
  CK(h, cudaMemsetAsync(h->scal + 1, 0, sizeof(double), h->st));
  if (ng > 0) {
    int rc = stage_gates<T>(h, ng, gates, p, p_stride);
    if (rc) return rc;
    for (int g = 0; g < ng; ++g) {
      rc = gate_update<T>(h, 2 * g + parity, (const cplx<T>*)h->Ms + (size_t)g * 256);
      if (rc) return rc;
    }
  }
  return sweep_all<T>(h);
}

template <typename T>
static int trace_t(mpo_ctx* h, double* tr) {
  double2 one = make_double2(1.0, 0.0);
  CK(h, cudaMemcpyAsync(h->tv0, &one, sizeof(double2), cudaMemcpyHostToDevice, h->st));
  double2 *a = h->tv0, *b = h->tv1;
  for (int k = 0; k < h->n; ++k) {
    const int cl = h->chi[k], cr = h->chi[k + 1];
    {
      ProfScope ps(h, PK_TRACE, 8.0 * cl * cr, (2.0 * cl * cr) * sizeof(cplx<T>));
      trace_step_kernel<T><<<(cr + 127) / 128, 128, 0, h->st>>>(S_<T>(h, k), cl, cr, a, b);
      CK(h, cudaGetLastError());
    }
    std::swap(a, b);
  }
  double2 v;
  double ln;
  CK(h, cudaMemcpyAsync(&v, a, sizeof(double2), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaMemcpyAsync(&ln, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  *tr = v.x * std::exp(ln);
  return MPO_OK;
}

// ---------------------------------------------------------- P(x), sampling --
// Output probabilities P(x) = <<X|rho>> with X = (d+1) x (Sec. 3.4) of S bit
// strings, or S samples drawn by sequential conditionals (Sec. 3.4) from the
// caller's uniforms. Scratch is allocated per call (a diagnostic path).
template <typename T>
static int chain_t(mpo_ctx* h, int S, const double* uniforms, unsigned char* bits, double* P) {
  const int n = h->n, cm = h->chi_max;
  const bool sample = uniforms != nullptr;
  std::vector<void*> owned;
  auto dalloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    owned.push_back(p);
    return p;
  };
  auto release = [&]() { for (void* p : owned) cudaFree(p); owned.clear(); };
  cplx<T>* L = (cplx<T>*)dalloc(sizeof(cplx<T>) * (size_t)S * cm);
  cplx<T>* L2 = (cplx<T>*)dalloc(sizeof(cplx<T>) * (size_t)S * cm);
  cplx<T>* t0 = (cplx<T>*)dalloc(sizeof(cplx<T>) * (size_t)S * cm);
  cplx<T>* t1 = (cplx<T>*)dalloc(sizeof(cplx<T>) * (size_t)S * cm);
  double* ls = (double*)dalloc(sizeof(double) * S);
  unsigned char* dbits = (unsigned char*)dalloc((size_t)S * n);
  double* du = sample ? (double*)dalloc(sizeof(double) * (size_t)S * n) : nullptr;
  double2* R = sample ? (double2*)dalloc(sizeof(double2) * (size_t)(n + 1) * (cm + 1)) : nullptr;
  if (!L || !L2 || !t0 || !t1 || !ls || !dbits || (sample && (!du || !R))) { release(); return fail(h, MPO_ERR_OOM, "chain scratch"); }
  auto ck = [&](cudaError_t e) -> bool { if (e != cudaSuccess) { release(); fail(h, MPO_ERR_CUDA, cudaGetErrorString(e)); return false; } return true; };
  if (!ck(cudaMemsetAsync(ls, 0, sizeof(double) * S, h->st))) return MPO_ERR_CUDA;
  if (sample) {
    if (!ck(cudaMemcpyAsync(du, uniforms, sizeof(double) * (size_t)S * n, cudaMemcpyHostToDevice, h->st))) return MPO_ERR_CUDA;
    // right environments R_k (k = n .. 0), R_n = (1)
    const double2 one = make_double2(1.0, 0.0);
    if (!ck(cudaMemcpyAsync(R + (size_t)n * (cm + 1), &one, sizeof(double2), cudaMemcpyHostToDevice, h->st))) return MPO_ERR_CUDA;
    for (int k = n - 1; k >= 0; --k) {
      trace_right_kernel<T><<<(h->chi[k] + 127) / 128, 128, 0, h->st>>>(S_<T>(h, k), h->chi[k], h->chi[k + 1],
                                                                      R + (size_t)(k + 1) * (cm + 1), R + (size_t)k * (cm + 1));
      if (!ck(cudaGetLastError())) return MPO_ERR_CUDA;
    }
  } else {
    if (!ck(cudaMemcpyAsync(dbits, bits, (size_t)S * n, cudaMemcpyHostToDevice, h->st))) return MPO_ERR_CUDA;
  }
  {  // L = 1 for every string (left bond dimension 1)
    std::vector<cplx<T>> ones(S, mk<T>(T(1), T(0)));
    if (!ck(cudaMemcpyAsync(L, ones.data(), sizeof(cplx<T>) * S, cudaMemcpyHostToDevice, h->st))) return MPO_ERR_CUDA;
    if (!ck(cudaStreamSynchronize(h->st))) return MPO_ERR_CUDA;
  }
  for (int k = 0; k < n; ++k) {
    const int cl = h->chi[k], cr = h->chi[k + 1];
    const cplx<T>* A = S_<T>(h, k);
    if (!ck(cgemm<T>(h->st, S, cr, cl, L, cl, 0, A, 4 * cr, 0, t0, cr))) return MPO_ERR_CUDA;            // I = 0
    if (!ck(cgemm<T>(h->st, S, cr, cl, L, cl, 0, A + 3 * (size_t)cr, 4 * cr, 0, t1, cr))) return MPO_ERR_CUDA; // I = 3
    chain_select_kernel<T><<<(S * 32 + 255) / 256, 256, 0, h->st>>>(t0, t1, S, cr, sample ? R + (size_t)(k + 1) * (cm + 1) : nullptr,
                                                                   du, dbits, n, k, L2, ls);
    if (!ck(cudaGetLastError())) return MPO_ERR_CUDA;
    std::swap(L, L2);
  }
  std::vector<cplx<T>> fin(S);
  std::vector<double> hls(S);
  double ln = 0.0;
  if (!ck(cudaMemcpyAsync(fin.data(), L, sizeof(cplx<T>) * S, cudaMemcpyDeviceToHost, h->st))) return MPO_ERR_CUDA;
  if (!ck(cudaMemcpyAsync(hls.data(), ls, sizeof(double) * S, cudaMemcpyDeviceToHost, h->st))) return MPO_ERR_CUDA;
  if (!ck(cudaMemcpyAsync(&ln, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->st))) return MPO_ERR_CUDA;
  if (sample && !ck(cudaMemcpyAsync(bits, dbits, (size_t)S * n, cudaMemcpyDeviceToHost, h->st))) return MPO_ERR_CUDA;
  if (!ck(cudaStreamSynchronize(h->st))) return MPO_ERR_CUDA;
  if (P)
    for (int s = 0; s < S; ++s) P[s] = (double)fin[s].x * std::exp(hls[s] + ln);
  release();
  return MPO_OK;
}

// ================================================================ C ABI ====
// ------------------------------------------------------ map validation ----
// Eigenvalues of an n x n Hermitian matrix (row-major complex, n <= 16) by
// the cyclic Jacobi method in FP64 on the host (Golub & Van Loan, Sec. 8.5):
// rotations until every off-diagonal entry is below 1e-15 of the Frobenius
// norm. Returns the smallest eigenvalue.
static double hermitian_min_eig(std::vector<std::complex<double>> A, int n) {
  double fro = 0.0;
  for (const auto& z : A) fro += std::norm(z);
  fro = std::sqrt(fro);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off = std::max(off, std::abs(A[p * n + q]));
    if (off <= 1e-15 * fro) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const std::complex<double> g = A[p * n + q];
        const double ag = std::abs(g);
        if (ag <= 1e-300) continue;
        const double a = A[p * n + p].real(), b = A[q * n + q].real();
        const double zeta = (b - a) / (2.0 * ag);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = t * c;
        const std::complex<double> u = g / ag;
        // J = [[c, s], [-conj(u) s, conj(u) c]] on columns p, q; A <- J^H A J
        for (int k = 0; k < n; ++k) {          // A <- A J
          const std::complex<double> x = A[k * n + p], y = A[k * n + q];
          A[k * n + p] = c * x - sn * std::conj(u) * y;
          A[k * n + q] = sn * x + c * std::conj(u) * y;
        }
        for (int k = 0; k < n; ++k) {          // A <- J^H A
          const std::complex<double> x = A[p * n + k], y = A[q * n + k];
          A[p * n + k] = c * x - sn * u * y;
          A[q * n + k] = sn * x + c * u * y;
        }
        A[p * n + q] = A[q * n + p] = 0.0;
      }
  }
  double mn = A[0].real();
  for (int i = 1; i < n; ++i) mn = std::min(mn, A[i * n + i].real());
  return mn;
}

// Checks a two-qubit superoperator M (App. A convention: row 4 I_l + I_r,
// I = 2 ket + bra) for the two properties of a quantum channel (Sec. 2.2):
// trace preservation, t^T M = t^T with t_I = 1 for I in {0, 3} on each qubit;
// complete positivity, the Choi matrix C[(a, j), (b, k)] = (M(|j><k|))_{ab}
// (two-qubit indices a, b, j, k = 2 q_l + q_r) positive semidefinite. The
// tolerance is tol times the largest |M_ij|. Returns 0, 1 (not trace
// preserving) or 2 (not completely positive); *defect receives the larger
// violation (the largest |t^T M - t^T| entry or minus the smallest Choi
// eigenvalue).
static int check_superop(const std::complex<double>* M, double tol, double* defect) {
  double mx = 0.0;
  for (int e = 0; e < 256; ++e) mx = std::max(mx, std::abs(M[e]));
  const double lim = tol * std::max(mx, 1e-300);
  auto t = [](int I) { return (I == 0 || I == 3) ? 1.0 : 0.0; };
  double tp = 0.0;
  for (int col = 0; col < 16; ++col) {
    std::complex<double> v = 0.0;
    for (int row = 0; row < 16; ++row) v += t(row / 4) * t(row % 4) * M[row * 16 + col];
    tp = std::max(tp, std::abs(v - t(col / 4) * t(col % 4)));
  }
  std::vector<std::complex<double>> C(256);
  for (int a = 0; a < 4; ++a)
    for (int j = 0; j < 4; ++j)
      for (int b = 0; b < 4; ++b)
        for (int k = 0; k < 4; ++k) {
          const int row = 4 * (2 * (a >> 1) + (b >> 1)) + (2 * (a & 1) + (b & 1));
          const int col = 4 * (2 * (j >> 1) + (k >> 1)) + (2 * (j & 1) + (k & 1));
          C[(4 * a + j) * 16 + (4 * b + k)] = M[row * 16 + col];
        }
  // the Choi matrix of a Hermiticity-preserving map is Hermitian; use its
  // Hermitian part and count the rest as a defect
  double herm = 0.0;
  for (int x = 0; x < 16; ++x)
    for (int y = x; y < 16; ++y) {
      herm = std::max(herm, std::abs(C[x * 16 + y] - std::conj(C[y * 16 + x])));
      const std::complex<double> h = 0.5 * (C[x * 16 + y] + std::conj(C[y * 16 + x]));
      C[x * 16 + y] = h;
      C[y * 16 + x] = std::conj(h);
    }
  const double cp = std::max(herm, -hermitian_min_eig(C, 16));
  if (defect) *defect = std::max(tp, cp);
  if (tp > lim) return 1;
  if (cp > lim) return 2;
  return 0;
}

extern "C" {

void mpo_default_opts(mpo_opts* o) {
  if (!o) return;
  o->eig_max_sweeps = 40;
  o->sv_rel_cutoff = 0.0;
  o->arena_cap_bytes = 0;
  o->smode = MPO_S_ALL_BONDS;
  o->barrier_timeout_s = 5.0;
  o->block_jacobi_min_rows = 0;
  o->tensor_cores = 0;
  o->oversample = 0;
  o->refine_steps = 0;
}

const char* mpo_version(void) { return "gb300-mpo 0.1 (sm_103a)"; }

static int init_fail(mpo_ctx* h, int code, const std::string& m) {
  g_last_init_error = m;
  if (h) mpo_free(h);
  return code;
}

// Device allocation that counts towards the handle's bytes.
static bool ws_alloc(mpo_ctx* h, void** p, size_t bytes) {
  if (cudaMalloc(p, std::max<size_t>(bytes, 256)) != cudaSuccess) { cudaGetLastError(); *p = nullptr; return false; }
  h->bytes += bytes;
  return true;
}

// Workspace of the factorisations (svd_select / msvd_select) for matrices of
// at most m rows and ccap columns: left factor, values, selection, control
// blocks, the block Jacobi's partial Grams and rotations, and for the
// precision form its FP32 copy and FP64 refinement buffers.
static bool alloc_factor_ws(mpo_ctx* h, int m, int ccap, size_t bj_nch) {
  auto alloc = [&](void** p, size_t bytes) -> bool { return ws_alloc(h, p, bytes); };
  const size_t rsz = h->prec != MPO_FP32 ? sizeof(double) : sizeof(float);
  const size_t bj_pairs = (size_t)((m + JB - 1) / JB + 1) / 2 + 1;
  bool ok = true;
  ok = ok && alloc(&h->vecs, (size_t)m * m * h->esz);
  ok = ok && alloc(&h->wv, (size_t)m * rsz);
  ok = ok && alloc((void**)&h->perm, (size_t)m * sizeof(int));
  ok = ok && alloc((void**)&h->lam2, (size_t)m * sizeof(double));
  ok = ok && alloc((void**)&h->info, sizeof(SelectInfo));
  ok = ok && alloc((void**)&h->ctl, sizeof(GridCtl));
  ok = ok && alloc((void**)&h->osctl, sizeof(OSCtl));
  ok = ok && alloc((void**)&h->tc_status, sizeof(int));
  if (h->block_min_rows > 0) {
    h->bj_slots = bj_pairs * bj_nch;
    ok = ok && alloc(&h->bj_gpart, h->bj_slots * JP * JP * h->esz);
    ok = ok && alloc(&h->bj_j, bj_pairs * JP * JP * h->esz);
    h->bj_act_ints = bj_state_ints(m);
    ok = ok && alloc((void**)&h->bj_act, h->bj_act_ints * sizeof(int));
  }
  if (h->mixed) {
    const size_t mm = (size_t)h->mx_mcap;
    ok = ok && alloc((void**)&h->mx_a32, (size_t)m * ccap * sizeof(float2));
    ok = ok && alloc((void**)&h->mx_ut32, (size_t)m * m * sizeof(float2));
    ok = ok && alloc((void**)&h->mx_w32, (size_t)m * sizeof(float));
    ok = ok && alloc((void**)&h->mx_perm32, (size_t)m * sizeof(int));
    ok = ok && alloc((void**)&h->mx_lam32, (size_t)m * sizeof(double));
    ok = ok && alloc((void**)&h->mx_info32, sizeof(SelectInfo));
    ok = ok && alloc((void**)&h->mx_Q, (size_t)m * mm * sizeof(double2));
    ok = ok && alloc((void**)&h->mx_Q2, (size_t)m * mm * sizeof(double2));
    ok = ok && alloc((void**)&h->mx_B, (size_t)ccap * mm * sizeof(double2));
    ok = ok && alloc((void**)&h->mx_T, (size_t)ccap * mm * sizeof(double2));
    ok = ok && alloc((void**)&h->mx_V, mm * mm * sizeof(double2));
    ok = ok && alloc((void**)&h->mx_G, mm * mm * sizeof(double2));
    ok = ok && alloc((void**)&h->mx_w, mm * sizeof(double));
    ok = ok && alloc((void**)&h->mx_W, mm * mm * sizeof(double2));
    ok = ok && alloc((void**)&h->mx_eosctl, sizeof(OSCtl));
    ok = ok && alloc((void**)&h->mx_Q0, (size_t)m * mm * sizeof(double2));
    ok = ok && alloc((void**)&h->mx_A32, mm * mm * sizeof(float2));
    ok = ok && alloc((void**)&h->mx_Li32, mm * mm * sizeof(float2));
    ok = ok && alloc((void**)&h->mx_t32, mm * mm * sizeof(float2));
    ok = ok && alloc((void**)&h->mx_d, mm * sizeof(double));
    ok = ok && alloc((void**)&h->mx_chst, sizeof(int));
    if (ok) ok = ensure_dynamic_smem((const void*)chol_diag_kernel<float, CHOL32_NB>, chol_smem_bytes<float, CHOL32_NB>()) == cudaSuccess;
  }
  return ok;
}

int mpo_init(mpo_handle* out, int n, int chi_max, mpo_precision prec, void* stream, const mpo_opts* opts) {
  if (!out) { g_last_init_error = "out is NULL"; return MPO_ERR_ARG; }
  *out = nullptr;
  if (n < 2 || n % 2 || n > 4096) { g_last_init_error = "n_qubits must be even, 2..4096"; return MPO_ERR_ARG; }
  if (chi_max < 1 || chi_max > 4096) { g_last_init_error = "chi_max must be 1..4096"; return MPO_ERR_ARG; }
  if (prec != MPO_FP64 && prec != MPO_FP32 && prec != MPO_MIXED_FP32) { g_last_init_error = "unknown precision"; return MPO_ERR_ARG; }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    g_last_init_error = "no CUDA device";
    return MPO_ERR_CUDA;
  }
  mpo_ctx* h = new mpo_ctx();
  h->n = n;
  h->chi_max = chi_max;
  h->prec = prec;
  h->st = (cudaStream_t)stream;
  mpo_default_opts(&h->opts);
  if (opts) h->opts = *opts;
  if (h->opts.eig_max_sweeps <= 0) h->opts.eig_max_sweeps = 40;
  if (!(h->opts.barrier_timeout_s > 0.0)) h->opts.barrier_timeout_s = 5.0;
  h->mixed = prec == MPO_MIXED_FP32;
  h->cutoff = h->opts.sv_rel_cutoff > 0.0 ? h->opts.sv_rel_cutoff
                                          : (prec == MPO_FP64 ? 1e-12 : (h->mixed ? 1e-7 : 1e-6));
  if (cudaGetDevice(&h->device) != cudaSuccess) return init_fail(h, MPO_ERR_CUDA, "cudaGetDevice failed");
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
  if (!coop) return init_fail(h, MPO_ERR_CUDA, "device lacks cooperative launch");

  h->esz = prec != MPO_FP32 ? sizeof(double2) : sizeof(float2);
  const size_t rsz = prec != MPO_FP32 ? sizeof(double) : sizeof(float);
  h->cap.resize(n + 1);
  for (int b = 0; b <= n; ++b) h->cap[b] = cap_of(b, n, chi_max);
  h->chi.assign(n + 1, 1);
  h->site_cap = 0;
  for (int k = 0; k < n; ++k) h->site_cap = std::max(h->site_cap, (size_t)h->cap[k] * 4 * h->cap[k + 1]);
  size_t th = 0;
  int m = 1;
  for (int i = 0; i + 1 < n; ++i) {
    th = std::max(th, (size_t)16 * h->cap[i] * h->cap[i + 2]);
    m = std::max(m, 4 * std::min(h->cap[i], h->cap[i + 2]));
  }
  for (int b = 0; b <= n; ++b) m = std::max(m, h->cap[b]);
  h->theta_cap = th;
  h->m_cap = m;
  const int jac_limit = prec != MPO_FP32 ? 8192 : 16384;   // rotation table must fit shared memory
  if (m > jac_limit) return init_fail(h, MPO_ERR_ARG, "bond dimension too large for the eigen-solver's shared-memory table");
  h->tmp_cap = (size_t)m * chi_max;
  h->tensor_cores = prec == MPO_FP32 && h->opts.tensor_cores > 0;
  h->block_min_rows = h->opts.block_jacobi_min_rows < 0 ? 0
                      : (h->opts.block_jacobi_min_rows > 0 ? h->opts.block_jacobi_min_rows : (prec != MPO_FP64 ? 64 : 0));
  // precision form: subspace iteration on chi_max + oversample directions,
  // FP32 and FP64 Rayleigh-Ritz steps
  h->mx_over = h->opts.oversample > 0 ? h->opts.oversample : (h->opts.oversample < 0 ? 0 : chi_max);
  h->mx_bond_steps.assign(n, 0);
  h->mx_steps = h->opts.refine_steps > 0 ? std::min(h->opts.refine_steps, kMixedMaxSteps) : (h->opts.refine_steps < 0 ? 1 : kMixedSteps);
  h->mx_mcap = std::min(m, chi_max + h->mx_over);
  // FP64-accurate products on the tensor cores (BF16 slices) unless switched off
  h->use_oz = h->mixed && h->opts.tensor_cores >= 0;
  int mx_ccap = 1;   // longest row of a factorised matrix
  for (int i = 0; i + 1 < n; ++i) mx_ccap = std::max(mx_ccap, 4 * std::max(h->cap[i], h->cap[i + 2]));
  for (int b = 0; b + 1 <= n; ++b) mx_ccap = std::max(mx_ccap, 4 * h->cap[std::min(b + 1, n)]);
  const size_t bj_nch = (size_t)(4 * chi_max + JCW - 1) / JCW + 1;
  const int ngmax = n / 2;
  const size_t need = (size_t)(n + 1) * h->site_cap * h->esz + 2 * th * h->esz + (size_t)m * m * h->esz +
                      h->tmp_cap * h->esz + (size_t)m * (rsz + sizeof(int) + sizeof(double)) +
                      (size_t)ngmax * 256 * h->esz + (size_t)ngmax * (16 * sizeof(double2) + sizeof(double)) +
                      (size_t)(n - 1) * (1 + chi_max) * sizeof(double) + 2 * (size_t)chi_max * sizeof(double2) + 4096 +
                      (h->mixed ? (size_t)m * mx_ccap * sizeof(float2) + (size_t)m * m * sizeof(float2) +
                                      (size_t)m * (sizeof(float) + sizeof(int) + sizeof(double)) +
                                      2 * (size_t)m * h->mx_mcap * sizeof(double2) +
                                      2 * (size_t)mx_ccap * h->mx_mcap * sizeof(double2) +
                                      2 * (size_t)h->mx_mcap * h->mx_mcap * sizeof(double2) +
                                      2 * (size_t)h->mx_mcap * h->mx_mcap * sizeof(double2) +
                                      3 * (size_t)h->mx_mcap * h->mx_mcap * sizeof(float2) +
                                      (size_t)m * h->mx_mcap * sizeof(double2) + (size_t)h->mx_mcap * sizeof(double)
                                : 0) +
                      (h->use_oz ? (size_t)oz::S * 2 * 3 * (size_t)std::max(m, mx_ccap) * 2 *
                                       (size_t)((std::max(m, mx_ccap) + 127) / 128 * 128)
                                 : 0);
  if (h->opts.arena_cap_bytes > 0 && need > h->opts.arena_cap_bytes)
    return init_fail(h, MPO_ERR_OOM, "device memory needed (" + std::to_string(need) + " B) exceeds arena_cap_bytes");
  size_t freeb = 0, totb = 0;
  if (cudaMemGetInfo(&freeb, &totb) == cudaSuccess && need > freeb)
    return init_fail(h, MPO_ERR_OOM, "device memory needed (" + std::to_string(need) + " B) exceeds free memory");

  auto alloc = [&](void** p, size_t bytes) -> bool { return ws_alloc(h, p, bytes); };
  h->site.assign(n, nullptr);
  bool ok = true;
  for (int k = 0; k < n && ok; ++k) ok = alloc(&h->site[k], h->site_cap * h->esz);
  ok = ok && alloc(&h->spare, h->site_cap * h->esz);
  ok = ok && alloc(&h->theta, th * h->esz);
  ok = ok && alloc(&h->theta2, th * h->esz);
  ok = ok && alloc(&h->tmp, h->tmp_cap * h->esz);
  ok = ok && alloc(&h->Ms, (size_t)std::max(1, ngmax) * 256 * h->esz);
  ok = ok && alloc((void**)&h->dgates, (size_t)std::max(1, ngmax) * 16 * sizeof(double2));
  ok = ok && alloc((void**)&h->dp, (size_t)std::max(1, ngmax) * sizeof(double));
  ok = ok && alloc((void**)&h->dsup, 256 * sizeof(double2));
  ok = ok && alloc_factor_ws(h, m, mx_ccap, bj_nch);
  if (ok && h->use_oz) ok = alloc_oz(h->oz, std::max(m, mx_ccap), &h->bytes);
  ok = ok && alloc((void**)&h->scal, 8 * sizeof(double));
  ok = ok && alloc((void**)&h->dS, (size_t)(n - 1) * sizeof(double));
  ok = ok && alloc((void**)&h->dschmidt, (size_t)(n - 1) * chi_max * sizeof(double));
  ok = ok && alloc((void**)&h->tv0, (size_t)(chi_max + 1) * sizeof(double2));
  ok = ok && alloc((void**)&h->tv1, (size_t)(chi_max + 1) * sizeof(double2));
  if (!ok) return init_fail(h, MPO_ERR_OOM, "cudaMalloc failed");
  if (cudaMallocHost((void**)&h->hs, sizeof(HostSync)) != cudaSuccess) {
    cudaGetLastError();
    h->hs = nullptr;
    return init_fail(h, MPO_ERR_CUDA, "cudaMallocHost failed");
  }
  // product state |0..0><0..0|: every site 1 x 4 x 1 with A[0][0][0] = 1 (Sec. 4.1)
  std::vector<unsigned char> one(h->esz, 0);
  if (prec != MPO_FP32) { double v = 1.0; memcpy(one.data(), &v, sizeof v); }
  else { float v = 1.0f; memcpy(one.data(), &v, sizeof v); }
  for (int k = 0; k < n; ++k) {
    if (cudaMemsetAsync(h->site[k], 0, 4 * h->esz, h->st) != cudaSuccess ||
        cudaMemcpyAsync(h->site[k], one.data(), h->esz, cudaMemcpyHostToDevice, h->st) != cudaSuccess)
      return init_fail(h, MPO_ERR_CUDA, "initial state upload failed");
  }
  if (cudaMemsetAsync(h->tc_status, 0, sizeof(int), h->st) != cudaSuccess ||
      cudaMemsetAsync(h->scal, 0, 8 * sizeof(double), h->st) != cudaSuccess ||
      cudaMemsetAsync(h->dS, 0, (size_t)(n - 1) * sizeof(double), h->st) != cudaSuccess ||
      cudaStreamSynchronize(h->st) != cudaSuccess)
    return init_fail(h, MPO_ERR_CUDA, "initial state upload failed");
  h->schmidt_len.assign(n - 1, 1);
  h->s_valid.assign(n - 1, 0);
  // the product state's Schmidt values are (1): S = 0 at every bond
  std::vector<double> s1((size_t)(n - 1) * chi_max, 0.0);
  for (int b = 0; b < n - 1; ++b) s1[(size_t)b * chi_max] = 1.0;
  if (cudaMemcpy(h->dschmidt, s1.data(), s1.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return init_fail(h, MPO_ERR_CUDA, "initial state upload failed");
  std::fill(h->s_valid.begin(), h->s_valid.end(), 1);
  h->centre = 0;
  *out = h;
  return MPO_OK;
}

static void batch_free(mpo_ctx* h);

void mpo_free(mpo_handle h) {
  if (!h) return;
  if (h->batch) { batch_free(h); return; }
  for (void* p : h->site) if (p) cudaFree(p);
  void* ps[] = {h->spare, h->theta, h->theta2, h->osctl, h->tc_status, h->bj_gpart, h->bj_j, h->bj_act, h->vecs, h->tmp, h->wv, h->perm, h->lam2, h->Ms, h->dgates,
                h->dsup, h->dp, h->info, h->ctl, h->scal, h->dS, h->dschmidt, h->tv0, h->tv1,
                h->mx_a32, h->mx_ut32, h->mx_w32, h->mx_perm32, h->mx_lam32, h->mx_info32, h->mx_Q, h->mx_Q2,
                h->mx_B, h->mx_T, h->mx_V, h->mx_G, h->mx_w,
                h->mx_W, h->mx_A32, h->mx_Li32, h->mx_t32, h->mx_d, h->mx_chst, h->mx_eosctl, h->mx_Q0};
  for (void* p : ps) if (p) cudaFree(p);
  if (h->hs) cudaFreeHost(h->hs);
  free_oz(h->oz);
  for (auto& q : h->pend) { cudaEventDestroy(q.a); cudaEventDestroy(q.b); }
  for (auto e : h->evpool) cudaEventDestroy(e);
  delete h;
}

const char* mpo_last_error(mpo_handle h) {
  if (!h) return g_last_init_error.c_str();
  return h->msg.c_str();
}

#define GUARD(h)                                                        \
  do {                                                                  \
    if (!(h)) return MPO_ERR_ARG;                                       \
    if ((h)->batch) {                                                   \
      (h)->msg = "a batch handle takes only the batch calls";           \
      return MPO_ERR_ARG;                                               \
    }                                                                   \
    if ((h)->failed) return MPO_ERR_STATE;                              \
    cudaSetDevice((h)->device);                                         \
  } while (0)

int mpo_apply_layer(mpo_handle h, int parity, const double* gates, const double* p, int p_stride) {
  GUARD(h);
  if (parity != 0 && parity != 1) return fail(h, MPO_ERR_ARG, "parity must be 0 or 1");
  const int ng = (h->n - parity) / 2;
  if (ng > 0 && (!gates || !p || p_stride < 0)) return fail(h, MPO_ERR_ARG, "gates/p must be non-NULL, p_stride >= 0");
  return dsite(h) ? apply_layer_t<double>(h, parity, gates, p, p_stride)
                             : apply_layer_t<float>(h, parity, gates, p, p_stride);
}

int mpo_apply_gate(mpo_handle h, int bond, const double* gate, double p) {
  GUARD(h);
  if (bond < 0 || bond > h->n - 2 || !gate) return fail(h, MPO_ERR_ARG, "bad bond or gate");
  if (dsite(h)) {
    int rc = stage_gates<double>(h, 1, gate, &p, 0);
    return rc ? rc : gate_update<double>(h, bond, (const double2*)h->Ms);
  }
  int rc = stage_gates<float>(h, 1, gate, &p, 0);
  return rc ? rc : gate_update<float>(h, bond, (const float2*)h->Ms);
}

int mpo_theta(mpo_handle h, int bond, const double* gate, double p, void* out, int* rows, int* cols) {
  GUARD(h);
  if (bond < 0 || bond > h->n - 2 || !gate || !rows || !cols) return fail(h, MPO_ERR_ARG, "bad bond, gate or dims");
  if (!(p >= 0.0 && p <= 1.0)) return fail(h, MPO_ERR_ARG, "p must lie in [0, 1]");
  return dsite(h) ? theta_t<double>(h, bond, gate, p, out, rows, cols)
                  : theta_t<float>(h, bond, gate, p, out, rows, cols);
}

int mpo_check_superop(const double* M, double tol, double* defect) {
  if (!M) return MPO_ERR_ARG;
  std::complex<double> hm[256];
  if (is_device_ptr(M)) {
    if (cudaMemcpy(hm, M, sizeof(hm), cudaMemcpyDeviceToHost) != cudaSuccess) { cudaGetLastError(); return MPO_ERR_CUDA; }
  } else {
    std::memcpy(hm, M, sizeof(hm));
  }
  return check_superop(hm, tol > 0.0 ? tol : 1e-9, defect) ? MPO_ERR_ARG : MPO_OK;
}

int mpo_apply_superop(mpo_handle h, int bond, const double* M) {
  GUARD(h);
  if (bond < 0 || bond > h->n - 2 || !M) return fail(h, MPO_ERR_ARG, "bad bond or superoperator");
  {
    double defect = 0.0;
    const int rc = mpo_check_superop(M, 1e-9, &defect);
    if (rc == MPO_ERR_CUDA) return fail(h, rc, "could not read the superoperator");
    if (rc) return fail(h, MPO_ERR_ARG, "superoperator is not trace preserving and completely positive (defect " +
                                            std::to_string(defect) + ")");
  }
  const double2* src = (const double2*)M;
  if (!is_device_ptr(M)) {
    CK(h, cudaMemcpyAsync(h->dsup, M, sizeof(double2) * 256, cudaMemcpyHostToDevice, h->st));
    src = h->dsup;
  }
  if (dsite(h)) cast_superop_kernel<double><<<1, 256, 0, h->st>>>(src, (double2*)h->Ms);
  else cast_superop_kernel<float><<<1, 256, 0, h->st>>>(src, (float2*)h->Ms);
  CK(h, cudaGetLastError());
  return dsite(h) ? gate_update<double>(h, bond, (const double2*)h->Ms)
                             : gate_update<float>(h, bond, (const float2*)h->Ms);
}

int mpo_sweep(mpo_handle h) {
  GUARD(h);
  return dsite(h) ? sweep_all<double>(h) : sweep_all<float>(h);
}

int mpo_entropy(mpo_handle h, double* S, double* trace, double* discarded) {
  GUARD(h);
  if (!S) return fail(h, MPO_ERR_ARG, "S is NULL");
  std::vector<double> hS(h->n - 1);
  double disc = 0.0;
  CK(h, cudaMemcpyAsync(hS.data(), h->dS, sizeof(double) * (h->n - 1), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaMemcpyAsync(&disc, h->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  for (int b = 0; b < h->n - 1; ++b) S[b] = h->s_valid[b] ? hS[b] : NAN;
  if (discarded) *discarded = disc;
  if (trace) {
    int rc = dsite(h) ? trace_t<double>(h, trace) : trace_t<float>(h, trace);
    if (rc) return rc;
  }
  return MPO_OK;
}

int mpo_schmidt(mpo_handle h, int bond, double* lam, int* len) {
  GUARD(h);
  if (bond < 0 || bond > h->n - 2 || !lam || !len) return fail(h, MPO_ERR_ARG, "bad bond or NULL output");
  if (!h->s_valid[bond]) return fail(h, MPO_ERR_STATE, "no Schmidt values recorded for this bond");
  const int L = h->schmidt_len[bond];
  std::vector<double> p(L);
  CK(h, cudaMemcpyAsync(p.data(), h->dschmidt + (size_t)bond * h->chi_max, sizeof(double) * L,
                        cudaMemcpyDeviceToHost, h->st));
  CK(h, cudaStreamSynchronize(h->st));
  for (int i = 0; i < L; ++i) lam[i] = std::sqrt(std::max(0.0, p[i]));
  *len = L;
  return MPO_OK;
}

int mpo_bond_dims(mpo_handle h, int* dims) {
  GUARD(h);
  if (!dims) return fail(h, MPO_ERR_ARG, "dims is NULL");
  for (int b = 0; b <= h->n; ++b) dims[b] = h->chi[b];
  return MPO_OK;
}

int mpo_centre(mpo_handle h, int* c) {
  GUARD(h);
  if (!c) return fail(h, MPO_ERR_ARG, "NULL");
  *c = h->centre;
  return MPO_OK;
}

size_t mpo_device_bytes(mpo_handle h) { return h ? h->bytes : 0; }

int mpo_probability(mpo_handle h, int n_strings, const unsigned char* bits, double* P) {
  GUARD(h);
  if (n_strings < 1 || !bits || !P) return fail(h, MPO_ERR_ARG, "mpo_probability: bad arguments");
  for (size_t i = 0; i < (size_t)n_strings * h->n; ++i)
    if (bits[i] > 1) return fail(h, MPO_ERR_ARG, "mpo_probability: bits must be 0 or 1");
  return dsite(h) ? chain_t<double>(h, n_strings, nullptr, const_cast<unsigned char*>(bits), P)
                             : chain_t<float>(h, n_strings, nullptr, const_cast<unsigned char*>(bits), P);
}

int mpo_sample(mpo_handle h, int n_samples, const double* uniforms, unsigned char* bits, double* P) {
  GUARD(h);
  if (n_samples < 1 || !uniforms || !bits) return fail(h, MPO_ERR_ARG, "mpo_sample: bad arguments");
  for (size_t i = 0; i < (size_t)n_samples * h->n; ++i)
    if (!(uniforms[i] >= 0.0 && uniforms[i] < 1.0)) return fail(h, MPO_ERR_ARG, "mpo_sample: uniforms must lie in [0, 1)");
  return dsite(h) ? chain_t<double>(h, n_samples, uniforms, bits, P)
                             : chain_t<float>(h, n_samples, uniforms, bits, P);
}

int mpo_profile(mpo_handle h, int enable) {
  GUARD(h);
  prof_resolve(h);
  if (enable) {
    for (int i = 0; i < PK_NCLASS; ++i) { h->prof_ms[i] = 0; h->prof_n[i] = 0; h->prof_flops[i] = 0; h->prof_bytes[i] = 0; }
    h->prof_sweeps = 0;
    h->prof_steps = 0;
    for (int i = 0; i < 3; ++i) h->prof_phase_ns[i] = 0;
  }
  h->prof = enable != 0;
  return MPO_OK;
}

int mpo_profile_read(mpo_handle h, int cls, const char** name, double* ms, long long* launches, double* flops,
                     double* bytes) {
  GUARD(h);
  if (cls < 0 || cls >= PK_NCLASS) return MPO_ERR_ARG;
  prof_resolve(h);
  if (name) *name = kProfNames[cls];
  if (ms) *ms = h->prof_ms[cls];
  if (launches) *launches = h->prof_n[cls];
  if (flops) *flops = h->prof_flops[cls];
  if (bytes) *bytes = h->prof_bytes[cls];
  return MPO_OK;
}

long long mpo_profile_sweeps(mpo_handle h) { return h ? h->prof_sweeps : 0; }

long long mpo_profile_steps(mpo_handle h) { return h ? h->prof_steps : 0; }

int mpo_profile_phases(mpo_handle h, double* ms3) {
  GUARD(h);
  if (!ms3) return MPO_ERR_ARG;
  for (int i = 0; i < 3; ++i) ms3[i] = h->prof_phase_ns[i] * 1e-6;
  return MPO_OK;
}

int mpo_get_site(mpo_handle h, int k, double* buf, int* chiL, int* chiR) {
  GUARD(h);
  if (k < 0 || k >= h->n || !chiL || !chiR) return fail(h, MPO_ERR_ARG, "bad site index");
  *chiL = h->chi[k];
  *chiR = h->chi[k + 1];
  if (!buf) return MPO_OK;
  const size_t cnt = (size_t)h->chi[k] * 4 * h->chi[k + 1];
  double ln = 0.0;
  CK(h, cudaMemcpyAsync(&ln, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  if (dsite(h)) {
    CK(h, cudaMemcpyAsync(buf, h->site[k], cnt * sizeof(double2), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
  } else {
    std::vector<float> f(2 * cnt);
    CK(h, cudaMemcpyAsync(f.data(), h->site[k], cnt * sizeof(float2), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    for (size_t i = 0; i < 2 * cnt; ++i) buf[i] = f[i];
  }
  if (k == h->centre) {
    const double s = std::exp(ln);
    for (size_t i = 0; i < 2 * cnt; ++i) buf[i] *= s;
  }
  return MPO_OK;
}

int mpo_to_dense(mpo_handle h, double* rho_vec) {
  GUARD(h);
  if (!rho_vec || h->n > 12) return fail(h, MPO_ERR_ARG, "to_dense needs n <= 12 and a buffer");
  // T: rows = 4^j combined physical index, cols = current bond
  std::vector<double> T(2, 0.0);
  T[0] = 1.0;
  size_t rows = 1;
  int bond = 1;
  for (int k = 0; k < h->n; ++k) {
    int cl, cr;
    mpo_get_site(h, k, nullptr, &cl, &cr);
    std::vector<double> A((size_t)cl * 4 * cr * 2);
    int rc = mpo_get_site(h, k, A.data(), &cl, &cr);
    if (rc) return rc;
    if (cl != bond) return fail(h, MPO_ERR_STATE, "inconsistent bond dimensions");
    std::vector<double> Tn(rows * 4 * cr * 2, 0.0);
    for (size_t r = 0; r < rows; ++r)
      for (int a = 0; a < cl; ++a) {
        const double tr = T[(r * cl + a) * 2], ti = T[(r * cl + a) * 2 + 1];
        if (tr == 0.0 && ti == 0.0) continue;
        for (int I = 0; I < 4; ++I)
          for (int c = 0; c < cr; ++c) {
            const double ar = A[(((size_t)a * 4 + I) * cr + c) * 2], ai = A[(((size_t)a * 4 + I) * cr + c) * 2 + 1];
            const size_t o = ((r * 4 + I) * cr + c) * 2;
            Tn[o] += tr * ar - ti * ai;
            Tn[o + 1] += tr * ai + ti * ar;
          }
      }
    T.swap(Tn);
    rows *= 4;
    bond = cr;
  }
  memcpy(rho_vec, T.data(), rows * 2 * sizeof(double));
  return MPO_OK;
}

int mpo_svd_last_stats(int* sweeps, double* phase_ms3) {
  if (sweeps) *sweeps = g_last_svd_sweeps;
  if (phase_ms3) for (int i = 0; i < 3; ++i) phase_ms3[i] = g_last_svd_phase_ms[i];
  return MPO_OK;
}

int mpo_svd(int r, int c, void* X, void* w, void* Ut, mpo_precision prec, int max_sweeps, int block, void* stream) {
  if (r < 1 || c < 1 || !X || !w || !Ut || (prec != MPO_FP64 && prec != MPO_FP32)) return MPO_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPO_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  OSCtl* ctl = nullptr;
  void *gp = nullptr, *jb = nullptr;
  int* act = nullptr;
  const size_t esz = prec == MPO_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t pairs = (size_t)((r + JB - 1) / JB + 1) / 2 + 1, nch = (size_t)(c + JCW - 1) / JCW + 1;
  bool ok = cudaMalloc(&ctl, sizeof(OSCtl)) == cudaSuccess;
  if (block) {
    ok = ok && cudaMalloc(&gp, pairs * nch * JP * JP * esz) == cudaSuccess;
    ok = ok && cudaMalloc(&jb, pairs * JP * JP * esz) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&act, bj_state_ints(r) * sizeof(int)) == cudaSuccess;
  }
  if (!ok) { cudaGetLastError(); cudaFree(ctl); cudaFree(gp); cudaFree(jb); cudaFree(act); return MPO_ERR_OOM; }
  const int ms = max_sweeps > 0 ? max_sweeps : 40;
  cudaError_t e;
  if (block)
    e = prec == MPO_FP64
        ? launch_block_jacobi<double>(st, (double2*)X, r, c, c, (double2*)Ut, (double*)w, (double2*)gp, pairs * nch,
                                      (double2*)jb, act, bj_state_ints(r), ctl, ms, 5.0, sms)
        : launch_block_jacobi<float>(st, (float2*)X, r, c, c, (float2*)Ut, (float*)w, (float2*)gp, pairs * nch,
                                     (float2*)jb, act, bj_state_ints(r), ctl, ms, 5.0, sms);
  else
    e = prec == MPO_FP64
        ? launch_onesided<double>(st, (double2*)X, r, c, c, (double2*)Ut, (double*)w, ctl, ms, 5.0, sms)
        : launch_onesided<float>(st, (float2*)X, r, c, c, (float2*)Ut, (float*)w, ctl, ms, 5.0, sms);
  OSCtl hctl{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hctl, ctl, sizeof(OSCtl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(ctl); cudaFree(gp); cudaFree(jb); cudaFree(act);
  if (e != cudaSuccess) { g_last_init_error = cudaGetErrorString(e); return MPO_ERR_CUDA; }
  const GridCtl& hc = hctl.g;
  g_last_svd_sweeps = hc.sweeps;
  for (int i = 0; i < 3; ++i) g_last_svd_phase_ms[i] = block ? 1e-6 * (double)hctl.phase_ns[i] : 0.0;
  if (hc.err) return MPO_ERR_TIMEOUT;
  if (hc.status) return MPO_ERR_NOCONV;
  return MPO_OK;
}

int mpo_svd_truncated(int r, int c, const void* A, int cap, mpo_precision prec, const mpo_opts* opts, void* U,
                      void* X, double* lam2, int* k, void* stream) {
  if (r < 1 || c < 1 || r > c || cap < 1 || !A || !U || !X || !lam2 || !k ||
      (prec != MPO_FP64 && prec != MPO_FP32 && prec != MPO_MIXED_FP32)) {
    g_last_init_error = "mpo_svd_truncated: bad argument (needs 1 <= r <= c, cap >= 1, non-NULL buffers)";
    return MPO_ERR_ARG;
  }
  if (r > 8192) { g_last_init_error = "mpo_svd_truncated: r > 8192"; return MPO_ERR_ARG; }
  mpo_ctx* h = new mpo_ctx();
  h->n = 2;
  h->chi_max = cap;
  h->prec = prec;
  h->st = (cudaStream_t)stream;
  mpo_default_opts(&h->opts);
  if (opts) h->opts = *opts;
  if (h->opts.eig_max_sweeps <= 0) h->opts.eig_max_sweeps = 40;
  if (!(h->opts.barrier_timeout_s > 0.0)) h->opts.barrier_timeout_s = 5.0;
  h->mixed = prec == MPO_MIXED_FP32;
  h->cutoff = h->opts.sv_rel_cutoff > 0.0 ? h->opts.sv_rel_cutoff : (prec == MPO_FP64 ? 1e-12 : (h->mixed ? 1e-7 : 1e-6));
  h->esz = prec != MPO_FP32 ? sizeof(double2) : sizeof(float2);
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return MPO_ERR_CUDA; }
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  h->m_cap = r;
  h->block_min_rows = h->opts.block_jacobi_min_rows < 0 ? 0
                      : (h->opts.block_jacobi_min_rows > 0 ? h->opts.block_jacobi_min_rows : (prec != MPO_FP64 ? 64 : 0));
  h->mx_over = h->opts.oversample > 0 ? h->opts.oversample : (h->opts.oversample < 0 ? 0 : cap);
  h->mx_steps = h->opts.refine_steps > 0 ? std::min(h->opts.refine_steps, kMixedMaxSteps) : (h->opts.refine_steps < 0 ? 1 : kMixedSteps);
  h->mx_mcap = std::min(r, cap + h->mx_over);
  h->use_oz = h->mixed && h->opts.tensor_cores >= 0;
  const size_t nch = (size_t)(c + JCW - 1) / JCW + 1;
  bool ok = ws_alloc(h, &h->theta, (size_t)r * c * h->esz) && alloc_factor_ws(h, r, c, nch) &&
            ws_alloc(h, (void**)&h->scal, 8 * sizeof(double));
  if (ok && h->use_oz) ok = alloc_oz(h->oz, c, &h->bytes);
  if (ok && cudaMallocHost((void**)&h->hs, sizeof(HostSync)) != cudaSuccess) { cudaGetLastError(); h->hs = nullptr; ok = false; }
  if (!ok) { mpo_free(h); g_last_init_error = "mpo_svd_truncated: allocation failed"; return MPO_ERR_OOM; }
  int rc = MPO_OK, kk = 0;
  auto ck = [&](cudaError_t e) { if (rc == MPO_OK && e != cudaSuccess) { rc = MPO_ERR_CUDA; g_last_init_error = cudaGetErrorString(e); } };
  ck(cudaMemcpyAsync(h->theta, A, (size_t)r * c * h->esz, cudaMemcpyDeviceToDevice, h->st));
  ck(cudaMemsetAsync(h->scal, 0, 8 * sizeof(double), h->st));
  ck(cudaMemsetAsync(h->tc_status, 0, sizeof(int), h->st));
  if (rc == MPO_OK) {
    rc = prec != MPO_FP32 ? svd_select<double>(h, (double2*)h->theta, r, c, c, cap, true, nullptr, nullptr, &kk)
                          : svd_select<float>(h, (float2*)h->theta, r, c, c, cap, true, nullptr, nullptr, &kk);
    if (rc) g_last_init_error = h->msg;
  }
  if (rc == MPO_OK) {
    if (prec != MPO_FP32) {
      ck(gather_rows<double>(h, (double2*)h->vecs, r, r, kk, 1, (int)h->vecs_conj, 0, (double2*)U, cap));
      ck(gather_rows<double>(h, (double2*)h->theta, c, c, kk, 0, 0, 0, (double2*)X, c));
    } else {
      ck(gather_rows<float>(h, (float2*)h->vecs, r, r, kk, 1, 0, 0, (float2*)U, cap));
      ck(gather_rows<float>(h, (float2*)h->theta, c, c, kk, 0, 0, 0, (float2*)X, c));
    }
    ck(cudaMemcpyAsync(lam2, h->lam2, sizeof(double) * kk, cudaMemcpyDeviceToHost, h->st));
    ck(cudaStreamSynchronize(h->st));
    *k = kk;
  }
  mpo_free(h);
  return rc;
}

// ---------------------------------------------------------------------------
// Block-Jacobi SVD with built-in scratch (mpo_svd_static).
//
// Some callers cannot allocate device memory at the point where they need an
// SVD: code running inside an allocator's own callbacks (allocating again
// would re-enter the allocator), or hosts that hand out a fixed memory budget
// up front and account for every byte. For them this entry point keeps the block
// Jacobi's scratch (barrier/status block, pair Gram partials, rotations) in
// one file-scope device array that exists for as long as the library is
// loaded on each GPU that uses it. The caller only passes the matrix and the
// two outputs; nothing is allocated or freed.
// ---------------------------------------------------------------------------
namespace {
constexpr int kStaticMaxRows = 512;
constexpr int kStaticMaxCols = 2048;
constexpr size_t kStaticPairs = (size_t)(((kStaticMaxRows + JB - 1) / JB + 1) / 2 + 1);
constexpr size_t kStaticChunks = (size_t)((kStaticMaxCols + JCW - 1) / JCW + 1);
constexpr size_t kStaticSlots = kStaticPairs * kStaticChunks;
struct StaticSvdScratch {       // laid out for the widest element (complex128)
  OSCtl ctl;
  int act[bj_state_ints(kStaticMaxRows)];
  double2 jbuf[kStaticPairs * JP * JP];
  double2 gpart[kStaticSlots * JP * JP];
};
}  // namespace

// Shared by every call on a device; keeps the previous call's contents.
static __device__ __align__(256) unsigned char g_static_svd_scratch[sizeof(StaticSvdScratch)];

static int static_scratch_address(StaticSvdScratch** out) {
  // one lookup per device, done with that device current (the symbol's host
  // name is only a stand-in; the device address comes from the runtime)
  static void* addr[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MPO_ERR_CUDA;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_svd_scratch);
    if (e != cudaSuccess || !p) {
      g_last_init_error = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return MPO_ERR_CUDA;
    }
    addr[dev] = p;
  }
  *out = reinterpret_cast<StaticSvdScratch*>(addr[dev]);
  return MPO_OK;
}

int mpo_svd_static(int r, int c, void* X, void* w, void* Ut, mpo_precision prec, int max_sweeps, void* stream) {
  if (!X || !w || !Ut || r < 1 || c < 1 || (prec != MPO_FP64 && prec != MPO_FP32)) {
    g_last_init_error = "mpo_svd_static: bad argument";
    return MPO_ERR_ARG;
  }
  if (r > kStaticMaxRows || c > kStaticMaxCols) {
    g_last_init_error = "mpo_svd_static: matrix " + std::to_string(r) + " x " + std::to_string(c) +
                        " exceeds the built-in scratch limit of " + std::to_string(kStaticMaxRows) + " x " +
                        std::to_string(kStaticMaxCols);
    return MPO_ERR_ARG;
  }
  StaticSvdScratch* s = nullptr;
  int rc = static_scratch_address(&s);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPO_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ms = max_sweeps > 0 ? max_sweeps : 40;
  // launch_block_jacobi clears the control block (barrier counters, status,
  // per-sweep counts) before the launch; the kernel clears its round stamps
  // first, and the Gram partials, rotations and pair flags are fully written
  // before they are read in every round
  cudaError_t e = prec == MPO_FP64
      ? launch_block_jacobi<double>(st, (double2*)X, r, c, c, (double2*)Ut, (double*)w, (double2*)s->gpart,
                                    kStaticSlots, (double2*)s->jbuf, s->act, bj_state_ints(kStaticMaxRows), &s->ctl,
                                    ms, 5.0, sms)
      : launch_block_jacobi<float>(st, (float2*)X, r, c, c, (float2*)Ut, (float*)w, (float2*)s->gpart,
                                   kStaticSlots, (float2*)s->jbuf, s->act, bj_state_ints(kStaticMaxRows), &s->ctl,
                                   ms, 5.0, sms);
  OSCtl hctl{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hctl, &s->ctl, sizeof(OSCtl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { g_last_init_error = cudaGetErrorString(e); return MPO_ERR_CUDA; }
  // the same statistics as mpo_svd(..., block = 1) for mpo_svd_last_stats
  g_last_svd_sweeps = hctl.g.sweeps;
  for (int i = 0; i < 3; ++i) g_last_svd_phase_ms[i] = 1e-6 * (double)hctl.phase_ns[i];
  if (hctl.g.err) return MPO_ERR_TIMEOUT;
  if (hctl.g.status) return MPO_ERR_NOCONV;
  return MPO_OK;
}

int mpo_gemm(int M, int N, int K, const void* A, const void* B, void* C, mpo_precision prec, int tensor_cores,
             void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || (prec != MPO_FP64 && prec != MPO_FP32)) return MPO_ERR_ARG;
  if (tensor_cores && prec != MPO_FP32) return MPO_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  int* status = nullptr;
  if (tensor_cores) {
    if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) return MPO_ERR_OOM;
    cudaMemsetAsync(status, 0, sizeof(int), st);
    e = tc_cgemm(st, M, N, K, (const float2*)A, K, (const float2*)B, N, (float2*)C, N, nullptr, 1.0, status, 5.0);
  } else if (prec == MPO_FP64) {
    e = cgemm<double>(st, M, N, K, (const double2*)A, K, 0, (const double2*)B, N, 0, (double2*)C, N);
  } else {
    e = cgemm<float>(st, M, N, K, (const float2*)A, K, 0, (const float2*)B, N, 0, (float2*)C, N);
  }
  int hs = 0;
  if (e == cudaSuccess && status) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (status) cudaFree(status);
  if (e != cudaSuccess) { g_last_init_error = cudaGetErrorString(e); return MPO_ERR_CUDA; }
  return hs ? MPO_ERR_TIMEOUT : MPO_OK;
}

int mpo_gemm_ex(int M, int N, int K, const void* A, int lda, int opA, const void* B, int ldb, int opB, void* C,
                int ldc, mpo_precision prec, int engine, void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || (opA != 0 && opA != 1) || (opB != 0 && opB != 1) ||
      (prec != MPO_FP64 && prec != MPO_FP32) || (engine != 0 && engine != 1))
    return MPO_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPO_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaSuccess;
  int hs = 0;
  if (prec == MPO_FP64 && engine == 1) {
    OzWork w;
    if (!alloc_oz(w, std::max(M, std::max(N, K)), nullptr)) { free_oz(w); return MPO_ERR_OOM; }
    e = oz_gemm(st, M, N, K, (const double2*)A, lda, opA, (const double2*)B, ldb, opB, (double2*)C, ldc, 1.0, 0, w,
                5.0, sms);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, w.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    free_oz(w);
  } else if (engine == 1) {
    return mpo_gemm(M, N, K, A, B, C, prec, 1, stream);
  } else {
    e = prec == MPO_FP64 ? cgemm<double>(st, M, N, K, (const double2*)A, lda, opA, (const double2*)B, ldb, opB,
                                         (double2*)C, ldc)
                         : cgemm<float>(st, M, N, K, (const float2*)A, lda, opA, (const float2*)B, ldb, opB,
                                        (float2*)C, ldc);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) { g_last_init_error = cudaGetErrorString(e); return MPO_ERR_CUDA; }
  return hs ? MPO_ERR_TIMEOUT : MPO_OK;
}

int mpo_eigh(int m, void* A, void* w, void* V, mpo_precision prec, int max_sweeps, void* stream) {
  if (m < 1 || !A || !w || !V || (prec != MPO_FP64 && prec != MPO_FP32)) return MPO_ERR_ARG;
  const int lim = prec == MPO_FP64 ? 8192 : 16384;
  if (m > lim) return MPO_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPO_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  GridCtl* ctl = nullptr;
  if (cudaMalloc(&ctl, sizeof(GridCtl)) != cudaSuccess) return MPO_ERR_OOM;
  cudaError_t e = prec == MPO_FP64
      ? launch_jacobi<double>(st, (double2*)A, m, (double2*)V, (double*)w, ctl, max_sweeps > 0 ? max_sweeps : 40, 5.0, sms)
      : launch_jacobi<float>(st, (float2*)A, m, (float2*)V, (float*)w, ctl, max_sweeps > 0 ? max_sweeps : 40, 5.0, sms);
  GridCtl hc{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctl, sizeof(GridCtl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(ctl);
  if (e != cudaSuccess) { g_last_init_error = cudaGetErrorString(e); return MPO_ERR_CUDA; }
  if (hc.err) return MPO_ERR_TIMEOUT;
  if (hc.status) return MPO_ERR_NOCONV;
  return MPO_OK;
}


// ---------------------------------------------------------------------------
// Batching form: k independent circuits (the paper's ensembles of circuit
// instances per (n, p) point, Sec. 4) advanced one step per call. Every
// instance is an ordinary engine context on a stream of its own; a call hands
// the instances to n_workers host threads, longest chains first, each thread
// driving its instances' layers (whose Jacobi factorisations wait on the host
// for the kept rank) while the others keep the GPU busy with theirs.
// ---------------------------------------------------------------------------
struct BatchState {
  std::vector<mpo_ctx*> inst;
  std::vector<cudaStream_t> streams;
  std::vector<int> n_i, order;     // order: instance indices by decreasing n
  std::vector<size_t> s_off;       // offset of instance i's n_i - 1 entropies
  int workers = 1;
  cudaStream_t caller = nullptr;
  cudaEvent_t ready = nullptr;
};

static void batch_free(mpo_ctx* h) {
  BatchState* B = h->batch;
  cudaSetDevice(h->device);
  for (mpo_ctx* q : B->inst) mpo_free(q);
  for (cudaStream_t s : B->streams) if (s) cudaStreamDestroy(s);
  if (B->ready) cudaEventDestroy(B->ready);
  delete B;
  delete h;
}

int mpo_init_batch(mpo_handle* out, int k, const int* n_i, int chi_max, mpo_precision prec, void* stream,
                   const mpo_opts* opts, int n_workers) {
  if (!out) { g_last_init_error = "out is NULL"; return MPO_ERR_ARG; }
  *out = nullptr;
  if (k < 1 || !n_i) { g_last_init_error = "k must be >= 1 and n_i non-NULL"; return MPO_ERR_ARG; }
  for (int i = 0; i < k; ++i)
    if (n_i[i] < 2 || n_i[i] % 2 || n_i[i] > 4096) {
      g_last_init_error = "n_i[" + std::to_string(i) + "] must be even, 2..4096";
      return MPO_ERR_ARG;
    }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    g_last_init_error = "no CUDA device";
    return MPO_ERR_CUDA;
  }
  mpo_ctx* h = new mpo_ctx();
  h->batch = new BatchState();
  BatchState& B = *h->batch;
  h->chi_max = chi_max;
  h->prec = prec;
  cudaGetDevice(&h->device);
  B.caller = (cudaStream_t)stream;
  B.workers = std::max(1, std::min(n_workers > 0 ? n_workers : 8, k));
  if (cudaEventCreateWithFlags(&B.ready, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    batch_free(h);
    g_last_init_error = "cudaEventCreate failed";
    return MPO_ERR_CUDA;
  }
  size_t off = 0;
  for (int i = 0; i < k; ++i) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      batch_free(h);
      g_last_init_error = "cudaStreamCreate failed";
      return MPO_ERR_CUDA;
    }
    B.streams.push_back(s);
    mpo_handle q = nullptr;
    const int rc = mpo_init(&q, n_i[i], chi_max, prec, s, opts);
    if (rc) {
      const std::string m = "instance " + std::to_string(i) + ": " + g_last_init_error;
      batch_free(h);
      g_last_init_error = m;
      return rc;
    }
    B.inst.push_back(q);
    B.n_i.push_back(n_i[i]);
    B.s_off.push_back(off);
    off += (size_t)(n_i[i] - 1);
  }
  B.order.resize(k);
  for (int i = 0; i < k; ++i) B.order[i] = i;
  std::stable_sort(B.order.begin(), B.order.end(), [&](int x, int y) { return B.n_i[x] > B.n_i[y]; });
  *out = h;
  return MPO_OK;
}

int mpo_apply_layer_batch(mpo_handle h, int t, const double* gates_all, const double* p_all, const int* active,
                          double* S_all, double* trace_all, double* discarded_all) {
  if (!h || !h->batch) return MPO_ERR_ARG;
  if (h->failed) return MPO_ERR_STATE;
  if (t < 1 || !p_all) { h->msg = "t must be >= 1 and p_all non-NULL"; return MPO_ERR_ARG; }
  BatchState& B = *h->batch;
  const int k = (int)B.inst.size();
  const int parity = (t % 2 == 1) ? 0 : 1;   // odd steps: paper bonds 1, 3, ...; even steps: 2, 4, ...
  std::vector<size_t> goff(k, 0);
  size_t acc = 0;
  for (int i = 0; i < k; ++i) {
    if (active && !active[i]) continue;
    goff[i] = acc;
    acc += (size_t)((B.n_i[i] - parity) / 2) * 32;   // gates x 4 x 4 complex128
  }
  if (acc > 0 && !gates_all) { h->msg = "gates_all is NULL"; return MPO_ERR_ARG; }
  cudaSetDevice(h->device);
  if (cudaEventRecord(B.ready, B.caller) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, MPO_ERR_CUDA, "cudaEventRecord on the caller's stream failed");
  }
  std::atomic<int> next{0};
  std::vector<int> rcs(k, MPO_OK);
  auto work = [&]() {
    cudaSetDevice(h->device);
    std::vector<double> scratch;
    for (;;) {
      const int j = next.fetch_add(1);
      if (j >= k) break;
      const int i = B.order[j];
      if (active && !active[i]) continue;
      mpo_ctx* q = B.inst[i];
      if (cudaStreamWaitEvent(q->st, B.ready, 0) != cudaSuccess) { cudaGetLastError(); rcs[i] = MPO_ERR_CUDA; continue; }
      int rc = mpo_apply_layer(q, parity, gates_all + goff[i], p_all + i, 0);
      if (rc == MPO_OK && (S_all || trace_all || discarded_all)) {
        scratch.resize(B.n_i[i] - 1);
        double tr = 0.0, dw = 0.0;
        rc = mpo_entropy(q, S_all ? S_all + B.s_off[i] : scratch.data(), trace_all ? &tr : nullptr, &dw);
        if (rc == MPO_OK) {
          if (trace_all) trace_all[i] = tr;
          if (discarded_all) discarded_all[i] = dw;
        }
      }
      rcs[i] = rc;
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < B.workers; ++w) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  for (int i = 0; i < k; ++i)
    if (rcs[i] != MPO_OK) return fail(h, rcs[i], "instance " + std::to_string(i) + ": " + B.inst[i]->msg);
  return MPO_OK;
}

int mpo_batch_instance(mpo_handle h, int i, mpo_handle* inst) {
  if (!h || !h->batch || !inst) return MPO_ERR_ARG;
  if (i < 0 || i >= (int)h->batch->inst.size()) { h->msg = "instance index out of range"; return MPO_ERR_ARG; }
  *inst = h->batch->inst[i];
  return MPO_OK;
}

}  // extern "C"
