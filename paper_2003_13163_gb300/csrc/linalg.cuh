// linalg.cuh - dense complex linear algebra of the MPO update, written for
// one GB300: a tiled SIMT complex GEMM, a persistent cooperative parallel
// Jacobi eigen-solver for Hermitian matrices, and the single-CTA
// sort/select/entropy kernel that turns eigenvalues into kept Schmidt values.
#pragma once
#include "common.cuh"

// ---------------------------------------------------------------------------
// Complex GEMM: C (M x N) = alpha * op(A) * op(B), all row-major.
//   op == 0: plain; op == 1: conjugate transpose.
//   op(A)(i,k) = A[i*lda + k]      or conj(A[k*lda + i])
//   op(B)(k,j) = B[k*ldb + j]      or conj(B[j*ldb + k])
// alpha = alpha_host * (alpha_dev ? *alpha_dev : 1); accumulate != 0 adds the
// product to C instead of overwriting it (C and A / B must not overlap then).
// CTA tile BM x BN, K-slab BK, 256 threads, each thread TM x TN outputs spaced
// by 16 rows / 16 columns so that shared-memory reads broadcast along rows.
// ---------------------------------------------------------------------------
template <typename T, int BM, int BN, int BK>
__global__ void __launch_bounds__(256) cgemm_kernel(int M, int N, int K,
    const cplx<T>* __restrict__ A, int lda, int opA,
    const cplx<T>* __restrict__ B, int ldb, int opB,
    cplx<T>* __restrict__ C, int ldc, const double* __restrict__ alpha_dev, double alpha_host, int accumulate) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ cplx<T> As[BK][BM];
  __shared__ cplx<T> Bs[BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  cplx<T> acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = czero<T>();

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int s = 0; s < (BM * BK) / 256; ++s) {
      int idx = tid + 256 * s, i, k;
      cplx<T> v = czero<T>();
      if (opA == 0) {
        i = idx / BK; k = idx % BK;
        if (row0 + i < M && k0 + k < K) v = A[(size_t)(row0 + i) * lda + (k0 + k)];
      } else {
        i = idx % BM; k = idx / BM;
        if (row0 + i < M && k0 + k < K) v = cconj<T>(A[(size_t)(k0 + k) * lda + (row0 + i)]);
      }
      As[k][i] = v;
    }
#pragma unroll
    for (int s = 0; s < (BN * BK) / 256; ++s) {
      int idx = tid + 256 * s, j, k;
      cplx<T> v = czero<T>();
      if (opB == 0) {
        j = idx % BN; k = idx / BN;
        if (col0 + j < N && k0 + k < K) v = B[(size_t)(k0 + k) * ldb + (col0 + j)];
      } else {
        k = idx % BK; j = idx / BK;
        if (col0 + j < N && k0 + k < K) v = cconj<T>(B[(size_t)(col0 + j) * ldb + (k0 + k)]);
      }
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cplx<T> a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cfma<T>(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  const T alpha = (T)(alpha_host * (alpha_dev ? *alpha_dev : 1.0));
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = col0 + tx + 16 * j;
      if (c < N) {
        cplx<T> v = cscale<T>(acc[i][j], alpha);
        if (accumulate) v = cadd<T>(v, C[(size_t)r * ldc + c]);
        C[(size_t)r * ldc + c] = v;
      }
    }
  }
}

template <typename T>
inline cudaError_t cgemm(cudaStream_t st, int M, int N, int K, const cplx<T>* A, int lda, int opA,
                         const cplx<T>* B, int ldb, int opB, cplx<T>* C, int ldc,
                         const double* alpha_dev = nullptr, double alpha_host = 1.0, int accumulate = 0) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  constexpr int BM = 64, BN = 64, BK = 8;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  if (K <= 0 && accumulate) return cudaSuccess;
  if (K <= 0) {  // empty contraction: C = 0
    for (int r = 0; r < M; ++r) {
      cudaError_t e = cudaMemsetAsync(C + (size_t)r * ldc, 0, sizeof(cplx<T>) * N, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cgemm_kernel<T, BM, BN, BK><<<grid, 256, 0, st>>>(M, N, K, A, lda, opA, B, ldb, opB, C, ldc, alpha_dev, alpha_host,
                                                     accumulate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Parallel cyclic Jacobi eigen-solver for an m x m Hermitian matrix G
// (row-major, leading dimension m), in place: on exit G is diagonal to
// within the stopping rule, w[i] = G_ii and V (row-major) holds the
// eigenvectors as columns, G_in = V diag(w) V^H.
//
// Ordering: round-robin (circle method) over N = m + (m odd) players, so each
// round rotates N/2 disjoint pairs (p, q) and a sweep of N-1 rounds visits
// every pair once; an odd m gives one pair a bye per round.
// Rotation of pair (p, q) with a = G_pp, b = G_qq, g = G_pq = |g| u:
//   zeta = (b - a) / (2|g|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1/sqrt(1 + t^2), s = t c, J = [[c, s], [-conj(u) s, conj(u) c]],
// the complex form of the symmetric Schur rotation (Golub & Van Loan,
// Matrix Computations, Sec. 8.5); J^H G J zeroes G_pq.
// A pair is skipped when |g| <= max(tol_rel sqrt(|a b|), floor_rel max_i|G_ii|)
// (the relative criterion of Demmel & Veselic 1992 plus an absolute floor at
// the rounding level of the input). The solve stops after a sweep without a
// rotation; status = 1 if max_sweeps is reached first.
//
// Each round runs as three phases of one persistent cooperative launch:
//   A (every CTA, redundantly): the rotation table of the round -> smem;
//                                                                  barrier
//   B (G <- G J, V <- V J): one warp per row, lanes over pairs;   barrier
//   C (G <- J^H G): one warp per pair, lanes over columns;           barrier
// All G/V traffic uses L2-only loads/stores because other CTAs write it.
// ---------------------------------------------------------------------------
template <typename T> struct JRot { T c, s, ur, ui; };

__device__ __forceinline__ int rr_player(int pos, int r, int N) {
  return pos == 0 ? 0 : 1 + ((pos - 1 + r) % (N - 1));
}

template <typename T>
__global__ void __launch_bounds__(256) jacobi_kernel(cplx<T>* G, int m, cplx<T>* V, T* w, GridCtl* ctl,
                                                      int max_sweeps, T tol_rel, T floor_rel, long long timeout_ns) {
  extern __shared__ unsigned char jsmem[];
  JRot<T>* rot = reinterpret_cast<JRot<T>*>(jsmem);
  __shared__ int s_active;
  __shared__ T s_red[32];
  const int N = m + (m & 1), npairs = N / 2;
  const unsigned nblk = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarp_blk = blockDim.x >> 5;
  const long gwarp = (long)blockIdx.x * nwarp_blk + warp, nwarps = (long)nblk * nwarp_blk;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, gthreads = (size_t)nblk * blockDim.x;

  // V = I
  for (size_t e = gtid; e < (size_t)m * m; e += gthreads) {
    size_t r = e / m, c = e % m;
    stcg(&V[e], mk<T>(r == c ? T(1) : T(0), T(0)));
  }
  // scale = max_i |G_ii| (each CTA redundantly)
  T loc = T(0);
  for (int i = threadIdx.x; i < m; i += blockDim.x) loc = fmax(loc, fabs(ldcg(&G[(size_t)i * m + i]).x));
  for (int o = 16; o > 0; o >>= 1) loc = fmax(loc, __shfl_xor_sync(0xffffffffu, loc, o));
  if (lane == 0) s_red[warp] = loc;
  __syncthreads();
  if (threadIdx.x == 0) {
    T mx = T(0);
    for (int i = 0; i < nwarp_blk; ++i) mx = fmax(mx, s_red[i]);
    s_red[0] = mx;
  }
  __syncthreads();
  const T floor_abs = floor_rel * s_red[0];
  if (!grid_barrier(ctl, nblk, timeout_ns)) return;

  int sweep = 0;
  bool converged = (m <= 1);
  for (; sweep < max_sweeps && !converged; ++sweep) {
    long sweep_active = 0;
    for (int r = 0; r < N - 1; ++r) {
      // ---- phase A: rotation table -------------------------------------
      if (threadIdx.x == 0) s_active = 0;
      __syncthreads();
      int my_active = 0;
      for (int pi = threadIdx.x; pi < npairs; pi += blockDim.x) {
        int p = rr_player(pi, r, N), q = rr_player(N - 1 - pi, r, N);
        if (p > q) { int t_ = p; p = q; q = t_; }
        JRot<T> R; R.c = T(1); R.s = T(0); R.ur = T(1); R.ui = T(0);
        if (q < m) {
          const T a = ldcg(&G[(size_t)p * m + p]).x, b = ldcg(&G[(size_t)q * m + q]).x;
          const cplx<T> g = ldcg(&G[(size_t)p * m + q]);
          const T ag = hypot(g.x, g.y);
          const T thr = fmax(tol_rel * sqrt(fabs(a * b)), floor_abs);
          if (ag > thr && ag > T(0)) {
            const T zeta = (b - a) / (T(2) * ag);
            T t;
            if (fabs(zeta) > T(1) / eps_of<T>::value) t = T(0.5) / zeta;
            else t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
            const T c = T(1) / sqrt(T(1) + t * t);
            R.c = c; R.s = t * c; R.ur = g.x / ag; R.ui = g.y / ag;
            if (R.s != T(0)) ++my_active;
          }
        }
        rot[pi] = R;
      }
      if (my_active) atomicAdd(&s_active, my_active);
      __syncthreads();
      const int act = s_active;   // identical in every CTA: same inputs, same code
      sweep_active += act;
      if (act == 0) continue;
      // phase B rewrites the pivots (G_pp, G_qq, G_pq) that phase A reads:
      // no CTA rotates before every CTA has built its table from the same G
      if (!grid_barrier(ctl, nblk, timeout_ns)) return;
      // ---- phase B: column rotations, G <- G J and V <- V J ---------------
      for (long row = gwarp; row < 2L * m; row += nwarps) {
        cplx<T>* Rw = row < m ? G + (size_t)row * m : V + (size_t)(row - m) * m;
        for (int pi = lane; pi < npairs; pi += 32) {
          const JRot<T> R = rot[pi];
          if (R.s == T(0)) continue;
          int p = rr_player(pi, r, N), q = rr_player(N - 1 - pi, r, N);
          if (p > q) { int t_ = p; p = q; q = t_; }
          const cplx<T> x = ldcg(&Rw[p]), y = ldcg(&Rw[q]);
          const cplx<T> uy = cmul<T>(mk<T>(R.ur, -R.ui), y);   // conj(u) y
          stcg(&Rw[p], mk<T>(R.c * x.x - R.s * uy.x, R.c * x.y - R.s * uy.y));
          stcg(&Rw[q], mk<T>(R.s * x.x + R.c * uy.x, R.s * x.y + R.c * uy.y));
        }
      }
      if (!grid_barrier(ctl, nblk, timeout_ns)) return;
      // ---- phase C: row rotations, G <- J^H G ----------------------------
      for (long pi = gwarp; pi < npairs; pi += nwarps) {
        const JRot<T> R = rot[pi];
        if (R.s == T(0)) continue;
        int p = rr_player((int)pi, r, N), q = rr_player(N - 1 - (int)pi, r, N);
        if (p > q) { int t_ = p; p = q; q = t_; }
        cplx<T>* Rp = G + (size_t)p * m;
        cplx<T>* Rq = G + (size_t)q * m;
        for (int j = lane; j < m; j += 32) {
          const cplx<T> x = ldcg(&Rp[j]), y = ldcg(&Rq[j]);
          const cplx<T> uy = cmul<T>(mk<T>(R.ur, R.ui), y);    // u y
          cplx<T> np_ = mk<T>(R.c * x.x - R.s * uy.x, R.c * x.y - R.s * uy.y);
          cplx<T> nq_ = mk<T>(R.s * x.x + R.c * uy.x, R.s * x.y + R.c * uy.y);
          if (j == q) np_ = czero<T>();
          if (j == p) { nq_ = czero<T>(); np_.y = T(0); }
          if (j == q) nq_.y = T(0);
          stcg(&Rp[j], np_);
          stcg(&Rq[j], nq_);
        }
      }
      if (!grid_barrier(ctl, nblk, timeout_ns)) return;
    }
    if (sweep_active == 0) converged = true;
  }
  for (size_t i = gtid; i < (size_t)m; i += gthreads) w[i] = ldcg(&G[i * m + i]).x;
  if (gtid == 0) {
    ctl->sweeps = sweep;
    ctl->status = converged ? 0 : 1;
  }
}

// ---------------------------------------------------------------------------
// Select kernel (one CTA): turn the m eigenvalues w of a Gram matrix (the
// squared Schmidt values lambda'^2 of the factorised bond) into the kept set.
//   - bitonic sort of (value desc, index asc) in shared memory (stable order
//     for exact ties), negative rounding values clamped to 0;
//   - k = min(cap, #{lambda^2 > cutoff^2 * lambda_max^2}), at least 1;
//   - sums in FP64: total = sum lambda^2 (or *total_in, the squared Frobenius
//     norm of the factorised matrix, when w holds Ritz values of a subspace
//     only), kept = sum of the k largest;
//   - outputs perm[0..k), lam2[0..k) (descending), info->k, info->kept,
//     info->total; adds (total-kept)/total to *disc_acc and 0.5 log(kept) to
//     *lognorm when those are non-null;
//   - with S_out: the MPO entanglement entropy -sum p log2 p, p = lam2/kept
//     (Sec. 3.3), and the normalised lam2/kept into schmidt_out.
// ---------------------------------------------------------------------------
struct SelectInfo {
  int k;
  int status;
  int pad[2];
  double kept;
  double total;
  double inv_sqrt_kept;
  double pad2;
};

template <typename T>
__global__ void __launch_bounds__(1024) select_kernel(const T* __restrict__ w, int m, int cap, double cutoff2,
                                                       int* __restrict__ perm, double* __restrict__ lam2,
                                                       SelectInfo* info, double* disc_acc, double* lognorm,
                                                       double* S_out, double* schmidt_out,
                                                       const double* __restrict__ total_in) {
  extern __shared__ unsigned char ssm[];
  int P = 1;
  while (P < m) P <<= 1;
  double* key = reinterpret_cast<double*>(ssm);
  int* idx = reinterpret_cast<int*>(key + P);
  __shared__ double red[32];
  __shared__ double s_tot, s_kept, s_max;
  __shared__ int s_k;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wp = tid >> 5;
  for (int i = tid; i < P; i += nt) {
    if (i < m) { double v = (double)w[i]; key[i] = v > 0.0 ? v : 0.0; idx[i] = i; }
    else { key[i] = -1.0; idx[i] = 0x7fffffff; }
  }
  __syncthreads();
  // bitonic sort, descending by key, ascending index on ties
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < P; i += nt) {
        int j = i ^ stride;
        if (j > i) {
          bool desc = ((i & size) == 0);
          double ki = key[i], kj = key[j];
          int ii = idx[i], ij = idx[j];
          bool i_first = (ki > kj) || (ki == kj && ii < ij);   // i belongs before j in descending order
          bool swap = desc ? !i_first : i_first;
          if (swap) { key[i] = kj; key[j] = ki; idx[i] = ij; idx[j] = ii; }
        }
      }
      __syncthreads();
    }
  }
  // total and max
  double loc = 0.0;
  for (int i = tid; i < m; i += nt) loc += key[i];
  for (int o = 16; o > 0; o >>= 1) loc += __shfl_xor_sync(0xffffffffu, loc, o);
  if (lane == 0) red[wp] = loc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int i = 0; i < (nt + 31) / 32; ++i) s += red[i];
    s_tot = total_in ? *total_in : s;   // the factorised matrix's squared norm when w covers a subspace only
    s_max = key[0];
    const double thr = cutoff2 * key[0];
    int k = 0;
    const int lim = cap < m ? cap : m;
    while (k < lim && key[k] > thr) ++k;
    if (k == 0) k = 1;
    s_k = k;
  }
  __syncthreads();
  const int k = s_k;
  loc = 0.0;
  for (int i = tid; i < k; i += nt) loc += key[i];
  for (int o = 16; o > 0; o >>= 1) loc += __shfl_xor_sync(0xffffffffu, loc, o);
  __syncthreads();
  if (lane == 0) red[wp] = loc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int i = 0; i < (nt + 31) / 32; ++i) s += red[i];
    s_kept = s;
  }
  __syncthreads();
  const double kept = s_kept;
  for (int i = tid; i < k; i += nt) { perm[i] = idx[i]; lam2[i] = key[i]; }
  if (S_out) {
    loc = 0.0;
    for (int i = tid; i < k; i += nt) {
      const double pz = kept > 0.0 ? key[i] / kept : 0.0;
      if (schmidt_out) schmidt_out[i] = pz;
      if (pz > 0.0) loc -= pz * log2(pz);
    }
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_xor_sync(0xffffffffu, loc, o);
    __syncthreads();
    if (lane == 0) red[wp] = loc;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int i = 0; i < (nt + 31) / 32; ++i) s += red[i];
      *S_out = s;
    }
  }
  if (tid == 0) {
    info->k = k;
    info->kept = kept;
    info->total = s_tot;
    info->inv_sqrt_kept = kept > 0.0 ? 1.0 / sqrt(kept) : 0.0;
    if (disc_acc && s_tot > 0.0) *disc_acc += (s_tot - kept) / s_tot;
    if (lognorm && kept > 0.0) *lognorm += 0.5 * log(kept);
  }
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi SVD by row orthogonalisation.
// Input X (r x c, row-major, leading dimension ldx), in place. On exit the
// rows of X are mutually orthogonal, X_out = U^H X_in with U unitary (r x r),
// returned transposed as Ut (row p of Ut = column p of U, leading dim r), and
// w[i] = ||row i of X_out||^2: X_in = U X_out, so the squared singular values
// of X_in are w and its left singular vectors the columns of U
// (Hestenes 1958; Demmel & Veselic 1992 for the relative-accuracy stopping
// rule). No Gram matrix is formed, so small singular values keep their
// relative accuracy instead of being lost below eps * sigma_max^2.
//
// Pair (p, q) with a = ||x_p||^2, b = ||x_q||^2, g = <x_p, x_q> = sum_j
// x_p[j] conj(x_q[j]) is rotated by the same J as in the two-sided solver:
// rows  x_p <- c x_p - u s x_q,   x_q <- s x_p + u c x_q      (X <- J^H X)
// Ut    t_p <- c t_p - u* s t_q,  t_q <- s t_p + u* c t_q      (U <- U J)
// Ordering is round-robin as above; pairs of one round touch disjoint rows,
// so a round is one phase (one warp per pair) followed by one grid barrier.
// A sweep with no rotation (|g| <= max(tol sqrt(ab), floor)) ends the solve.
// ---------------------------------------------------------------------------
struct OSCtl {
  GridCtl g;
  int active[64];   // rotations per sweep (grid-wide atomic counts)
  double scale;
  double pad;
  unsigned long long phase_ns[4];   // CTA 0: wall time per phase (G, E, A), barrier waits included
};

template <typename T>
__device__ __forceinline__ void warp_sum3(T& a, T& b, T& c, T& d) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) onesided_jacobi_kernel(cplx<T>* X, int r, int c, int ldx, cplx<T>* Ut, T* w,
                                                               OSCtl* ctl, int max_sweeps, T tol_rel, T floor_rel,
                                                               long long timeout_ns) {
  const int N = r + (r & 1), npairs = N / 2;
  const unsigned nblk = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwb = blockDim.x >> 5;
  const long gwarp = (long)blockIdx.x * nwb + warp, nwarps = (long)nblk * nwb;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, gthreads = (size_t)nblk * blockDim.x;
  if (max_sweeps > 64) max_sweeps = 64;

  for (size_t e = gtid; e < (size_t)r * r; e += gthreads) {
    const size_t i = e / r, j = e % r;
    stcg(&Ut[e], mk<T>(i == j ? T(1) : T(0), T(0)));
  }
  // squared row norms -> w, then the largest one sets the absolute floor
  for (long i = gwarp; i < r; i += nwarps) {
    T s = T(0);
    for (int j = lane; j < c; j += 32) { const cplx<T> x = ldcg(&X[(size_t)i * ldx + j]); s += x.x * x.x + x.y * x.y; }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[i] = s;
  }
  if (!grid_barrier(&ctl->g, nblk, timeout_ns)) return;
  __shared__ T s_floor;
  if (threadIdx.x == 0) {
    T mx = T(0);
    for (int i = 0; i < r; ++i) mx = fmax(mx, __ldcg(&w[i]));
    s_floor = floor_rel * mx;
  }
  __syncthreads();
  const T floor_abs = s_floor;

  int sweep = 0;
  bool converged = (r <= 1);
  for (; sweep < max_sweeps && !converged; ++sweep) {
    for (int rd = 0; rd < N - 1; ++rd) {
      for (long pi = gwarp; pi < npairs; pi += nwarps) {
        int p = rr_player((int)pi, rd, N), q = rr_player(N - 1 - (int)pi, rd, N);
        if (p > q) { int t_ = p; p = q; q = t_; }
        if (q >= r) continue;
        cplx<T>* xp = X + (size_t)p * ldx;
        cplx<T>* xq = X + (size_t)q * ldx;
        T a = T(0), b = T(0), gr = T(0), gi = T(0);
#pragma unroll 16
        for (int j = lane; j < c; j += 32) {
          const cplx<T> x = ldcg(&xp[j]), y = ldcg(&xq[j]);
          a = fma(x.x, x.x, fma(x.y, x.y, a));
          b = fma(y.x, y.x, fma(y.y, y.y, b));
          gr = fma(x.x, y.x, fma(x.y, y.y, gr));     // x conj(y)
          gi = fma(x.y, y.x, fma(-x.x, y.y, gi));
        }
        warp_sum3<T>(a, b, gr, gi);
        // rotation parameters in FP64 whatever T is: unbiased c, s, u keep
        // the accumulated U unitary over many sweeps
        const double agd = hypot((double)gr, (double)gi);
        const double thr = fmax((double)tol_rel * sqrt((double)a * (double)b), (double)floor_abs);
        if (!(agd > thr) || agd == 0.0) continue;
        const double zeta = ((double)b - (double)a) / (2.0 * agd);
        double td;
        if (fabs(zeta) > 1e16) td = 0.5 / zeta;
        else td = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double csd = 1.0 / sqrt(1.0 + td * td);
        const T cs = (T)csd, sn = (T)(td * csd);
        if (sn == T(0)) continue;
        const T ur = (T)((double)gr / agd), ui = (T)((double)gi / agd);
        if (lane == 0) atomicAdd(&ctl->active[sweep], 1);
#pragma unroll 16
        for (int j = lane; j < c; j += 32) {
          const cplx<T> x = ldcg(&xp[j]), y = ldcg(&xq[j]);
          const cplx<T> uy = cmul<T>(mk<T>(ur, ui), y);
          stcg(&xp[j], mk<T>(cs * x.x - sn * uy.x, cs * x.y - sn * uy.y));
          stcg(&xq[j], mk<T>(sn * x.x + cs * uy.x, sn * x.y + cs * uy.y));
        }
        cplx<T>* tp = Ut + (size_t)p * r;
        cplx<T>* tq = Ut + (size_t)q * r;
#pragma unroll 16
        for (int j = lane; j < r; j += 32) {
          const cplx<T> x = ldcg(&tp[j]), y = ldcg(&tq[j]);
          const cplx<T> uy = cmul<T>(mk<T>(ur, -ui), y);
          stcg(&tp[j], mk<T>(cs * x.x - sn * uy.x, cs * x.y - sn * uy.y));
          stcg(&tq[j], mk<T>(sn * x.x + cs * uy.x, sn * x.y + cs * uy.y));
        }
      }
      if (!grid_barrier(&ctl->g, nblk, timeout_ns)) return;
    }
    if (atomicAdd(&ctl->active[sweep], 0) == 0) converged = true;
  }
  for (long i = gwarp; i < r; i += nwarps) {
    T s = T(0);
    for (int j = lane; j < c; j += 32) { const cplx<T> x = ldcg(&X[(size_t)i * ldx + j]); s += x.x * x.x + x.y * x.y; }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[i] = s;
  }
  if (gtid == 0) {
    ctl->g.sweeps = sweep;
    ctl->g.status = converged ? 0 : 1;
  }
}

// ---------------------------------------------------------------------------
// Gather of selected rows: element (j, i) = f_j * op(src[perm[j] * lds + i]),
// i < len, j < k (k = min(info->k, k_cap)), op = conj if conj_ else identity;
// written to out[j * ldo + i] (transpose == 0) or out[i * ldo + j] (== 1).
// f_j by mode: 0 -> 1; 1 -> 1/sqrt(lam2_j); 2 -> sqrt(lam2_j / kept);
//              3 -> 1/sqrt(kept).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void gather_rows_kernel(const cplx<T>* __restrict__ src, int lds, int len, const int* __restrict__ perm,
                                  const double* __restrict__ lam2, const SelectInfo* __restrict__ info, int k_cap,
                                  int transpose, int conj_, int mode, cplx<T>* __restrict__ out, int ldo) {
  const int k = info->k < k_cap ? info->k : k_cap;
  const size_t total = (size_t)len * k;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i, j;
    if (transpose) { i = (int)(e / k); j = (int)(e % k); }
    else { j = (int)(e / len); i = (int)(e % len); }
    double f = 1.0;
    if (mode == 1) f = lam2[j] > 0.0 ? 1.0 / sqrt(lam2[j]) : 0.0;
    else if (mode == 2) f = info->kept > 0.0 ? sqrt(lam2[j] / info->kept) : 0.0;
    else if (mode == 3) f = info->inv_sqrt_kept;
    cplx<T> v = src[(size_t)perm[j] * lds + i];
    if (conj_) v = cconj<T>(v);
    v = cscale<T>(v, (T)f);
    if (transpose) out[(size_t)i * ldo + j] = v;
    else out[(size_t)j * ldo + i] = v;
  }
}

// out (c x r) = in (r x c)^H, 32 x 32 tiles through shared memory.
template <typename T>
__global__ void conj_transpose_kernel(const cplx<T>* __restrict__ in, int r, int c, int ldi, cplx<T>* __restrict__ out, int ldo) {
  __shared__ cplx<T> tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int i = by + yy, j = bx + threadIdx.x;
    if (i < r && j < c) tile[yy][threadIdx.x] = in[(size_t)i * ldi + j];
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int j = bx + yy, i = by + threadIdx.x;
    if (j < c && i < r) out[(size_t)j * ldo + i] = cconj<T>(tile[threadIdx.x][yy]);
  }
}


// Shared-memory address of a generic pointer (for cp.async).
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------------------
// Block one-sided Jacobi SVD (row blocks of JB rows; a pair holds 2 JB rows).
// Same contract as onesided_jacobi_kernel: X (r x c) <- U^H X with rows
// mutually orthogonal, Ut = U^T, w = squared row norms.
//
// Rows are grouped in nb = ceil(r / JB) blocks, paired round-robin (bye for
// odd nb). For the pair (P, Q) of a round:
//   G = X_PQ X_PQ^H (2JB x 2JB), diagonalised as G = J diag J^H by an in-CTA
//   cyclic Jacobi, then X_PQ <- J^H X_PQ and Ut_PQ <- J^T Ut_PQ;
// this orthogonalises all 2JB rows of the pair at once (block Jacobi; the
// rotations are applied as small dense products, so each round streams X once
// instead of once per row pair). A pair is left alone when every cross entry
// satisfies |G_ij| <= max(tol sqrt(G_ii G_jj), floor * max_k G_kk).
// One round = three phases of a persistent cooperative launch:
//   G: Gram partials over column chunks (pair x chunk work items)   barrier
//   E: per pair, sum partials, skip test, inner Jacobi -> J         barrier
//   A: per pair x chunk, apply J to X and to Ut                     barrier
// ---------------------------------------------------------------------------
constexpr int JB = 16;           // rows per block
constexpr int JP = 2 * JB;       // rows per pair
constexpr int JCW = 512;         // columns per Gram / apply work item

// Integer state of the block Jacobi for r rows: the per-pair rotate flags of
// a round, then for each block the round stamp of its last rotation, then
// for each block a flag "own rows not known orthogonal", then for each block
// pair (P, Q) the stamp of the round that last found it orthogonal (N x N,
// N = the padded block count).
__host__ __device__ constexpr size_t bj_state_ints(int r) {
  return (size_t)(((r + JB - 1) / JB + (((r + JB - 1) / JB) & 1)) / 2) +
         2 * (size_t)((r + JB - 1) / JB + (((r + JB - 1) / JB) & 1)) +
         (size_t)((r + JB - 1) / JB + (((r + JB - 1) / JB) & 1)) * (size_t)((r + JB - 1) / JB + (((r + JB - 1) / JB) & 1));
}


// In-CTA cyclic Jacobi of the pair's 2JB x 2JB Gram in the working precision
// TI (FP64 arithmetic runs at 1/64 of the FP32 rate on this part, so nothing
// here is promoted). The tolerance is set at the rounding level of TI and the
// sweep count is capped, because J is re-derived in every outer round and an
// inexact inner solve only costs outer sweeps. The rounding drift of the
// accumulated rotations is removed afterwards by bj_polish_unitary.
template <typename TI> __device__ __forceinline__ TI rsqrt_fast(TI x);
template <> __device__ __forceinline__ float rsqrt_fast<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_fast<double>(double x) { return rsqrt(x); }

// Rotation parameters of the 2 x 2 Hermitian block [[a, g], [conj g, b]]
// (rows p, q of G): c, s real and u = g / |g|, chosen so that the rotation
// R = [[c, s], [-s conj(u), c conj(u)]] zeroes the off-diagonal entry of
// R^H G R; s = 0 when |g|^2 <= max(tol^2 |a b|, floor^2) (square-root free
// skip test).
template <typename TI>
__device__ __forceinline__ void bj_rot_params(const cplx<TI>* G, int p, int q, TI tol2, TI flo2, TI& c_, TI& s_,
                                              TI& ur, TI& ui) {
  constexpr int LD = JP + 1;
  const TI a_ = G[p * LD + p].x, b_ = G[q * LD + q].x;
  const TI gx = G[p * LD + q].x, gy = G[p * LD + q].y;
  const TI g2 = gx * gx + gy * gy;
  c_ = TI(1); s_ = TI(0); ur = TI(1); ui = TI(0);
  if (g2 > fmax(tol2 * fabs(a_ * b_), flo2) && g2 > TI(0)) {
    const TI inv = rsqrt_fast<TI>(g2);                              // 1 / |g|
    const TI zeta = (b_ - a_) * TI(0.5) * inv;
    TI t;
    if constexpr (sizeof(TI) == 4) {
      // FP32: approximate divide and square root (a few ulp); any t gives
      // an exactly normalised (c, s) up to rsqrt rounding, and an inexact
      // angle only leaves a slightly larger off-diagonal for later rounds
      const float az = fabsf(zeta);
      if (az > 1.0f / eps_of<float>::value) t = __fdividef(0.5f, zeta);
      else {
        const float q = fmaf(zeta, zeta, 1.0f);
        t = __fdividef(1.0f, az + q * rsqrtf(q));
        if (!(zeta >= 0.0f)) t = -t;
      }
    } else {
      if (fabs(zeta) > TI(1) / eps_of<TI>::value) t = TI(0.5) / zeta;
      else t = (zeta >= TI(0) ? TI(1) : TI(-1)) / (fabs(zeta) + sqrt(TI(1) + zeta * zeta));
    }
    c_ = rsqrt_fast<TI>(TI(1) + t * t);
    s_ = t * c_;
    ur = gx * inv; ui = gy * inv;
  }
}

// One round of the cyclic parallel Jacobi as 2 x 2 block updates: the round's
// JP/2 disjoint rotations partition the indices into pairs, so the JP x JP
// matrix splits into (JP/2)^2 blocks B_ab = G[{p_a, q_a}][{p_b, q_b}], each
// updated on its own as B_ab <- R_a^H B_ab R_b. Thread (a, b) derives both
// rotations from the old matrix and writes the new block into the other
// buffer, so a round needs one barrier instead of three (parameters, column
// pass, row pass). Requires blockDim.x == (JP/2)^2.
//
// In-CTA cyclic Jacobi of the pair's 2JB x 2JB Gram in the working precision
// TI (FP64 arithmetic runs at 1/64 of the FP32 rate on this part, so nothing
// here is promoted). The tolerance is set at the rounding level of TI and the
// sweep count is capped, because J is re-derived in every outer round and an
// inexact inner solve only costs outer sweeps. The rounding drift of the
// accumulated rotations is removed afterwards by bj_polish_unitary. G0 holds
// the input; G1 is scratch of the same shape; both are overwritten. Returns
// 1 when a sweep found nothing left to rotate (the result is diagonal to the
// tolerance), 0 when max_sweeps ran out first.
template <typename TI>
__device__ int bj_inner_eig(cplx<TI>* G0, cplx<TI>* G1, cplx<TI>* Vs /*JP x JP, ld JP+1*/, double tol,
                             double floor_abs, int max_sweeps) {
  constexpr int LD = JP + 1, NR = JP / 2;
  static_assert(NR * NR == 256, "one thread per 2 x 2 block");
  const int tid = threadIdx.x, ia = tid / NR, ib = tid % NR;
  for (int e = tid; e < JP * JP; e += blockDim.x) {
    const int i = e / JP, j = e % JP;
    Vs[i * LD + j] = mk<TI>(i == j ? TI(1) : TI(0), TI(0));
  }
  __syncthreads();
  const TI tol2 = (TI)(tol * tol), flo2 = (TI)(floor_abs * floor_abs);
  cplx<TI>* Gc = G0;
  cplx<TI>* Gn = G1;
  for (int sw = 0; sw < max_sweeps; ++sw) {
    int any = 0;
    for (int rd = 0; rd < JP - 1; ++rd) {
      int pa = rr_player(ia, rd, JP), qa = rr_player(JP - 1 - ia, rd, JP);
      if (pa > qa) { const int t_ = pa; pa = qa; qa = t_; }
      int pb = rr_player(ib, rd, JP), qb = rr_player(JP - 1 - ib, rd, JP);
      if (pb > qb) { const int t_ = pb; pb = qb; qb = t_; }
      // lane l of every warp derives rotation l % NR; threads fetch the two
      // they need by shuffle (no block barrier for a shared table)
      TI cl, sl, url, uil;
      {
        const int lr = (tid & 31) % NR;
        int pl = rr_player(lr, rd, JP), ql = rr_player(JP - 1 - lr, rd, JP);
        if (pl > ql) { const int t_ = pl; pl = ql; ql = t_; }
        bj_rot_params<TI>(Gc, pl, ql, tol2, flo2, cl, sl, url, uil);
      }
      // every warp derives the same table from the same matrix, so a round
      // with nothing to rotate is skipped by all threads alike (no writes,
      // no barrier); the function therefore ends with a barrier, so that no
      // thread reuses G0 / G1 (the caller's polish scratch) while another is
      // still reading the last skipped rounds' table
      if (!__any_sync(0xffffffffu, sl != TI(0))) continue;
      const TI ca = __shfl_sync(0xffffffffu, cl, ia), sa = __shfl_sync(0xffffffffu, sl, ia);
      const TI ura = __shfl_sync(0xffffffffu, url, ia), uia = __shfl_sync(0xffffffffu, uil, ia);
      const TI cb = __shfl_sync(0xffffffffu, cl, ib), sb = __shfl_sync(0xffffffffu, sl, ib);
      const TI urb = __shfl_sync(0xffffffffu, url, ib), uib = __shfl_sync(0xffffffffu, uil, ib);
      cplx<TI> b00 = Gc[pa * LD + pb], b01 = Gc[pa * LD + qb], b10 = Gc[qa * LD + pb], b11 = Gc[qa * LD + qb];
      if (sb != TI(0)) {        // columns: [x y] <- [c x - s conj(u) y, s x + c conj(u) y]
        const cplx<TI> ub = mk<TI>(urb, -uib);
        const cplx<TI> y0 = cmul<TI>(ub, b01), y1 = cmul<TI>(ub, b11);
        b01 = mk<TI>(sb * b00.x + cb * y0.x, sb * b00.y + cb * y0.y);
        b00 = mk<TI>(cb * b00.x - sb * y0.x, cb * b00.y - sb * y0.y);
        b11 = mk<TI>(sb * b10.x + cb * y1.x, sb * b10.y + cb * y1.y);
        b10 = mk<TI>(cb * b10.x - sb * y1.x, cb * b10.y - sb * y1.y);
      }
      if (sa != TI(0)) {        // rows: [x; y] <- [c x - s u y; s x + c u y]
        const cplx<TI> ua = mk<TI>(ura, uia);
        const cplx<TI> y0 = cmul<TI>(ua, b10), y1 = cmul<TI>(ua, b11);
        b10 = mk<TI>(sa * b00.x + ca * y0.x, sa * b00.y + ca * y0.y);
        b00 = mk<TI>(ca * b00.x - sa * y0.x, ca * b00.y - sa * y0.y);
        b11 = mk<TI>(sa * b01.x + ca * y1.x, sa * b01.y + ca * y1.y);
        b01 = mk<TI>(ca * b01.x - sa * y1.x, ca * b01.y - sa * y1.y);
        if (ia == ib) {         // the rotated diagonal block: exact zeros, real diagonal
          b01 = czero<TI>(); b10 = czero<TI>(); b00.y = TI(0); b11.y = TI(0);
        }
      }
      Gn[pa * LD + pb] = b00; Gn[pa * LD + qb] = b01; Gn[qa * LD + pb] = b10; Gn[qa * LD + qb] = b11;
      if (sb != TI(0)) {        // V <- V R_b on rows ia and ia + NR
        const cplx<TI> ub = mk<TI>(urb, -uib);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          cplx<TI>* R = Vs + (ia + h * NR) * LD;
          const cplx<TI> x = R[pb], uy = cmul<TI>(ub, R[qb]);
          R[pb] = mk<TI>(cb * x.x - sb * uy.x, cb * x.y - sb * uy.y);
          R[qb] = mk<TI>(sb * x.x + cb * uy.x, sb * x.y + cb * uy.y);
        }
      }
      any |= __syncthreads_or(sb != TI(0));
      cplx<TI>* t_ = Gc; Gc = Gn; Gn = t_;
    }
    if (!any) {
      __syncthreads();   // rounds skipped without a barrier: no thread may leave while others still read Gc
      return 1;
    }
  }
  __syncthreads();
  return 0;
}

// One Newton-Schulz step V <- V (3 I - V^H V) / 2 (Higham, Functions of
// Matrices, Sec. 8.3): for V = Q (I + E) with small Hermitian E the result is
// unitary to O(|E|^2) + rounding, so the per-pair rotation J carries no
// accumulated drift into the U of the SVD. S and W are JP x JP scratch
// (leading dimension JP+1) in shared memory.
template <typename TI>
__device__ void bj_polish_unitary(cplx<TI>* Vs, cplx<TI>* S, cplx<TI>* W) {
  constexpr int LD = JP + 1;
  const int tid = threadIdx.x;
  for (int e = tid; e < JP * JP; e += blockDim.x) {      // S = V^H V
    const int i = e / JP, j = e % JP;
    cplx<TI> acc = czero<TI>();
#pragma unroll 8
    for (int k = 0; k < JP; ++k) cfma<TI>(acc, cconj<TI>(Vs[k * LD + i]), Vs[k * LD + j]);
    S[i * LD + j] = acc;
  }
  __syncthreads();
  for (int e = tid; e < JP * JP; e += blockDim.x) {      // W = V (3 I - S) / 2
    const int i = e / JP, j = e % JP;
    cplx<TI> acc = czero<TI>();
#pragma unroll 8
    for (int k = 0; k < JP; ++k) {
      cplx<TI> m = cscale<TI>(S[k * LD + j], TI(-0.5));
      if (k == j) m.x += TI(1.5);
      cfma<TI>(acc, Vs[i * LD + k], m);
    }
    W[i * LD + j] = acc;
  }
  __syncthreads();
  for (int e = tid; e < JP * JP; e += blockDim.x) Vs[(e / JP) * LD + (e % JP)] = W[(e / JP) * LD + (e % JP)];
  __syncthreads();
}

// Newton-Schulz steps until V is unitary to rounding: each step first forms
// S = V^H V and tests max |S - I| <= tol, then applies the step; the loop
// ends after the first step taken from a state that passed the test (leaving
// a defect of about tol^2 plus rounding) or after max_steps steps. The
// iteration converges for |S - I| < 1 (Higham, Functions of Matrices, 8.3).
template <typename TI>
__device__ void bj_polish_unitary_to(cplx<TI>* Vs, cplx<TI>* S, cplx<TI>* W, TI tol, int max_steps) {
  constexpr int LD = JP + 1;
  const int tid = threadIdx.x;
  for (int it = 0; it < max_steps; ++it) {
    int bad = 0;
    for (int e = tid; e < JP * JP; e += blockDim.x) {
      const int i = e / JP, j = e % JP;
      cplx<TI> acc = czero<TI>();
#pragma unroll 8
      for (int k = 0; k < JP; ++k) cfma<TI>(acc, cconj<TI>(Vs[k * LD + i]), Vs[k * LD + j]);
      S[i * LD + j] = acc;
      if (!(fabs(acc.x - (i == j ? TI(1) : TI(0))) <= tol && fabs(acc.y) <= tol)) bad = 1;
    }
    const int any_bad = __syncthreads_or(bad);
    for (int e = tid; e < JP * JP; e += blockDim.x) {
      const int i = e / JP, j = e % JP;
      cplx<TI> acc = czero<TI>();
#pragma unroll 8
      for (int k = 0; k < JP; ++k) {
        cplx<TI> m = cscale<TI>(S[k * LD + j], TI(-0.5));
        if (k == j) m.x += TI(1.5);
        cfma<TI>(acc, Vs[i * LD + k], m);
      }
      W[i * LD + j] = acc;
    }
    __syncthreads();
    for (int e = tid; e < JP * JP; e += blockDim.x) Vs[(e / JP) * LD + (e % JP)] = W[(e / JP) * LD + (e % JP)];
    __syncthreads();
    if (!any_bad) break;
  }
}

// Asynchronous global -> shared copies (cp.async): BYTES per copy, the tail
// beyond src_bytes zero-filled, so rows past the matrix read as zeros.
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void* dst, const void* src, int src_bytes) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" :: "r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" :: "r"(smem_addr(dst)), "l"(src), "n"(BYTES),
                 "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" :: "n"(N) : "memory"); }

template <typename T> struct BJ_GW { static constexpr int value = sizeof(T) == 4 ? 128 : 64; };
constexpr int BJ_NB = 4;   // phase-G staging ring: sub-chunks in flight per CTA
__device__ __forceinline__ bool tid_is_zero() { return threadIdx.x == 0; }

// Dynamic shared memory of block_jacobi_kernel<T>: the larger of the phase-G
// staging ring and the phase E/A matrices, then the cross-block reduction
// buffer.
template <typename T>
constexpr int block_jacobi_smem_bytes() {
  constexpr int GW = BJ_GW<T>::value;
  constexpr int TS = GW + 1;
  constexpr int RING = BJ_NB * JP * TS * (int)sizeof(cplx<T>);
  constexpr int GV = 3 * JP * (JP + 1) * (int)sizeof(cplx<T>);
  constexpr int RED = 8 * 16 * 40 * (int)sizeof(T);
  return (RING > GV ? RING : GV) + RED;
}

template <typename T>
__global__ void __launch_bounds__(256) block_jacobi_kernel(cplx<T>* X, int r, int c, int ldx, cplx<T>* Ut, T* w,
                                                            cplx<T>* Gpart, cplx<T>* Jbuf, int* act_flag, OSCtl* ctl,
                                                            int max_sweeps, T tol_rel, T floor_rel, long long timeout_ns) {
  constexpr int LD = JP + 1;
  // Dynamic shared memory (block_jacobi_smem_bytes<T>()): a ring of BJ_NB
  // phase-G tiles of JP rows x TS columns; phases E and A reuse the same
  // bytes for the pair Gram Gs, the rotation Vs and the polish scratch; the
  // cross-block reduction buffer follows.
  constexpr int GW = BJ_GW<T>::value;                    // staged columns in phase G
  // padded row stride: GW + 1 puts the rows that one warp reads at the same
  // column in distinct banks (8-byte rows at 2 x 129 words, 16-byte at 4 x 65)
  constexpr int TS = GW + 1;
  constexpr int RING = BJ_NB * JP * TS * (int)sizeof(cplx<T>), GV = 3 * JP * (JP + 1) * (int)sizeof(cplx<T>);
  extern __shared__ __align__(128) unsigned char smraw[];
  cplx<T>* ring = reinterpret_cast<cplx<T>*>(smraw);
  T* red = reinterpret_cast<T*>(smraw + (RING > GV ? RING : GV));   // [8][16][40]
  cplx<T>* Gs = reinterpret_cast<cplx<T>*>(smraw);     // phase E: the pair Gram; phase A: J^H or J^T
  cplx<T>* Vs = Gs + JP * LD;

  __shared__ T s_gmax;
  cplx<T>* Js = reinterpret_cast<cplx<T>*>(red);        // phase A: J^H or J^T (ld JP+1)
  __shared__ T s_floor;
  const int nb = (r + JB - 1) / JB, N = nb + (nb & 1), npairs = N / 2;
  const int nch = (c + JCW - 1) / JCW, nchu = (r + JCW - 1) / JCW;
  const unsigned nblk = gridDim.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwb = blockDim.x >> 5;
  const long gwarp = (long)blockIdx.x * nwb + warp, nwarps = (long)nblk * nwb;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + tid, gthreads = (size_t)nblk * blockDim.x;
  if (max_sweeps > 64) max_sweeps = 64;

  for (size_t e = gtid; e < (size_t)r * r; e += gthreads) {
    const size_t i = e / r, j = e % r;
    stcg(&Ut[e], mk<T>(i == j ? T(1) : T(0), T(0)));
  }
  // round stamps (round g = sweep (N - 1) + rd + 1): a pair whose blocks are
  // both unchanged since the round that found it orthogonal stays orthogonal,
  // so cross-only sweeps skip its Gram and its test
  int* last_mod = act_flag + npairs;
  int* wdirty = last_mod + N;   // 1: the block's own rows were left by an inexact pair solve
  int* last_clean = wdirty + N;
  // every block starts unverified: its first pair forms the full Gram
  for (size_t e = gtid; e < 2 * (size_t)N + (size_t)N * N; e += gthreads) last_mod[e] = (e >= (size_t)N && e < 2 * (size_t)N) ? 1 : 0;
  for (long i = gwarp; i < r; i += nwarps) {
    T s = T(0);
    for (int j = lane; j < c; j += 32) { const cplx<T> x = ldcg(&X[(size_t)i * ldx + j]); s += x.x * x.x + x.y * x.y; }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[i] = s;
  }
  if (!grid_barrier(&ctl->g, nblk, timeout_ns)) return;
  if (tid == 0) {
    T mx = T(0);
    for (int i = 0; i < r; ++i) mx = fmax(mx, __ldcg(&w[i]));
    s_floor = floor_rel * mx;
  }
  __syncthreads();
  const T floor_abs = s_floor;

  int sweep = 0;
  bool converged = (r <= 1);
  bool verify = false;   // this sweep forms full Grams to confirm convergence
  for (; sweep < max_sweeps && !converged; ++sweep) {
    // a verification pass is one round of full Grams (two when a block sits
    // out round 0): every round pairs each block once, so it re-checks the
    // rows inside every block; the cross blocks were just found orthogonal
    const int nrounds = verify ? ((nb & 1) ? 2 : 1) : N - 1;
    for (int rd = 0; rd < nrounds; ++rd) {
      unsigned long long tph = (blockIdx.x == 0 && tid == 0) ? global_timer_ns() : 0ull;
      // ---- phase G: partial Grams of each pair over column chunks ---------
      // A pair with an unverified block (every block until its first pair
      // solve, and after an inexact one) and every pair of a verification
      // pass form the full 2JB x 2JB Gram. Otherwise each block's own rows
      // are mutually orthogonal (a pair solve orthogonalises all its rows,
      // and a block's rows change only when it is paired), so only the
      // JB x JB cross block X_P X_Q^H and the row norms are formed; the
      // diagonal blocks are taken as diagonal.
      const bool full_gram = verify;
      const long nitems = (long)npairs * nch;
      // The CTA's work is the sequence of (item, sub-chunk) stages of its
      // items; a ring of BJ_NB tiles keeps BJ_NB stages in flight (cp.async,
      // no register staging), refilling each tile as soon as its stage has
      // been consumed, across item boundaries.
      const int gstamp = sweep * (N - 1) + rd + 1;
      auto pair_dirty = [&](int P_, int Q_) -> bool {
        return __ldcg(&last_clean[(size_t)P_ * N + Q_]) <= max(__ldcg(&last_mod[P_]), __ldcg(&last_mod[Q_]));
      };
      // a pair forms its full Gram in full sweeps, and whenever one of its
      // blocks was left by a pair solve that ran out of inner sweeps (its own
      // rows are then not known to be orthogonal, which cross-only Grams
      // assume)
      auto pair_full = [&](int P_, int Q_) -> bool {
        return full_gram || __ldcg(&wdirty[P_]) != 0 || __ldcg(&wdirty[Q_]) != 0;
      };
      auto item_valid = [&](long it) -> bool {
        const int pi_ = (int)(it / nch);
        int P_ = rr_player(pi_, rd, N), Q_ = rr_player(N - 1 - pi_, rd, N);
        if (P_ > Q_) { const int t_ = P_; P_ = Q_; Q_ = t_; }
        return Q_ < nb && (pair_full(P_, Q_) || pair_dirty(P_, Q_));
      };
      long p_item = blockIdx.x;   // producer cursor
      int p_sub = 0;
      while (p_item < nitems && !item_valid(p_item)) p_item += nblk;
      auto issue = [&](int buf) {
        if (p_item >= nitems) return;
        const int pi_ = (int)(p_item / nch), ch_ = (int)(p_item % nch);
        int P_ = rr_player(pi_, rd, N), Q_ = rr_player(N - 1 - pi_, rd, N);
        if (P_ > Q_) { const int t_ = P_; P_ = Q_; Q_ = t_; }
        const int c0_ = ch_ * JCW, c1_ = min(c, c0_ + JCW), k0 = c0_ + p_sub * GW;
        cplx<T>* tile = ring + buf * JP * TS;
        constexpr int PER = JP * GW / 256;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int e_ = tid + 256 * u, i = e_ / GW, k = e_ % GW;
          const int row = (i < JB ? P_ * JB + i : Q_ * JB + (i - JB));
          const bool in = row < r && k0 + k < c1_;
          cp_async_zfill<(int)sizeof(cplx<T>)>(&tile[i * TS + k], in ? (const void*)&X[(size_t)row * ldx + k0 + k]
                                                                     : (const void*)X,
                                               in ? (int)sizeof(cplx<T>) : 0);
        }
        if (++p_sub == (c1_ - c0_ + GW - 1) / GW) {
          p_sub = 0;
          do { p_item += nblk; } while (p_item < nitems && !item_valid(p_item));
        }
      };
#pragma unroll
      for (int q = 0; q < BJ_NB; ++q) { issue(q); cp_async_commit(); }
      int jseq = 0;               // consumer position in the stage sequence
      for (long item = blockIdx.x; item < nitems; item += nblk) {
        if (!item_valid(item)) continue;
        const int pi = (int)(item / nch), ch = (int)(item % nch);
        int P = rr_player(pi, rd, N), Q = rr_player(N - 1 - pi, rd, N);
        if (P > Q) { int t_ = P; P = Q; Q = t_; }
        const bool fullp = pair_full(P, Q);
        // full: thread (ti, tj) owns G[ti + 16a][tj + 16b];
        // cross: k-slice g = tid / 16 (k = g, g + 16, ...), member m = tid % 16
        // owns C[4 mi + i][4 mj + j], mi = m / 4, mj = m % 4, and the norms of
        // rows 4 mi + mj and JB + 4 mj + mi (each row's norm on one member)
        const int ti = tid >> 4, tj = tid & 15;
        const int mi = (tid & 15) >> 2, mj = tid & 3;
        cplx<T> acc[4][4];
        T nrmP = T(0), nrmQ = T(0);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = czero<T>();
        const int c0 = ch * JCW, c1 = min(c, c0 + JCW);
        const int nsub = (c1 - c0 + GW - 1) / GW;
        for (int s = 0; s < nsub; ++s, ++jseq) {
          cp_async_wait<BJ_NB - 1>();
          __syncthreads();
          const cplx<T>* tile = ring + (jseq % BJ_NB) * JP * TS;
          const int kn = min(GW, c1 - (c0 + s * GW));
          if (fullp) {
#pragma unroll 4
            for (int k = 0; k < kn; ++k) {
              const cplx<T> a0 = tile[ti * TS + k], a1 = tile[(ti + 16) * TS + k];
              const cplx<T> b0 = cconj<T>(tile[tj * TS + k]), b1 = cconj<T>(tile[(tj + 16) * TS + k]);
              cfma<T>(acc[0][0], a0, b0); cfma<T>(acc[0][1], a0, b1);
              cfma<T>(acc[1][0], a1, b0); cfma<T>(acc[1][1], a1, b1);
            }
          } else {
            for (int k = (tid >> 4); k < kn; k += 16) {
              cplx<T> av[4], bv[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                av[i] = tile[(4 * mi + i) * TS + k];
                bv[i] = tile[(JB + 4 * mj + i) * TS + k];
              }
              const cplx<T> np_ = tile[(4 * mi + mj) * TS + k], nq_ = tile[(JB + 4 * mj + mi) * TS + k];
              nrmP += np_.x * np_.x + np_.y * np_.y;
              nrmQ += nq_.x * nq_.x + nq_.y * nq_.y;
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma<T>(acc[i][j], av[i], cconj<T>(bv[j]));
            }
          }
          __syncthreads();                      // the tile is free: refill it
          issue(jseq % BJ_NB);
          cp_async_commit();
        }
        cplx<T>* Gp = Gpart + ((size_t)pi * nch + ch) * JP * JP;
        if (fullp) {
#pragma unroll
          for (int a_ = 0; a_ < 2; ++a_)
#pragma unroll
            for (int b_ = 0; b_ < 2; ++b_) stcg(&Gp[(ti + 16 * a_) * JP + tj + 16 * b_], acc[a_][b_]);
        } else {
          // reduce the 16 k-slices in a fixed order (deterministic, so the
          // same input always gives the same factorisation): half-warp pairs
          // by shuffle, then the 8 warps through shared memory
          constexpr int NV = 34;                                 // 16 complex + 2 norms
          T vals[NV];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) { vals[2 * (4 * i + j)] = acc[i][j].x; vals[2 * (4 * i + j) + 1] = acc[i][j].y; }
          vals[32] = nrmP;
          vals[33] = nrmQ;
#pragma unroll
          for (int v = 0; v < NV; ++v) vals[v] += __shfl_xor_sync(0xffffffffu, vals[v], 16);
          if ((tid & 31) < 16) {
#pragma unroll
            for (int v = 0; v < NV; ++v) red[((tid >> 5) * 16 + (tid & 15)) * NV + v] = vals[v];
          }
          __syncthreads();
          for (int e = tid; e < JP * JP; e += blockDim.x) {
            const int i = e / JP, j = e % JP;
            cplx<T> v = czero<T>();
            if ((i < JB) != (j < JB)) {
              const bool upper = i < JB;
              const int pi_ = upper ? i : j, qj = upper ? j - JB : i - JB;
              const int m = (pi_ >> 2) * 4 + (qj >> 2), o = 2 * (4 * (pi_ & 3) + (qj & 3));
              T sr = T(0), si = T(0);
              for (int w = 0; w < 8; ++w) { sr += red[(w * 16 + m) * NV + o]; si += red[(w * 16 + m) * NV + o + 1]; }
              v = mk<T>(sr, upper ? si : -si);
            } else if (i == j) {
              T s = T(0);
              if (i < JB) { for (int w = 0; w < 8; ++w) s += red[(w * 16 + i) * NV + 32]; }        // member i
              else {
                const int q = i - JB, m = 4 * (q & 3) + (q >> 2);                                   // 4 mi + mj, mj = q / 4, mi = q % 4
                for (int w = 0; w < 8; ++w) s += red[(w * 16 + m) * NV + 33];
              }
              v = mk<T>(s, T(0));
            }
            stcg(&Gp[e], v);
          }
          __syncthreads();
        }
      }
      cp_async_wait<0>();
      __syncthreads();
      if (!grid_barrier(&ctl->g, nblk, timeout_ns)) return;
      if (blockIdx.x == 0 && tid == 0) { unsigned long long t2 = global_timer_ns(); ctl->phase_ns[0] += t2 - tph; tph = t2; }
      // ---- phase E: per pair, reduce, test, inner eigen-solve ---------------
      for (long pi = blockIdx.x; pi < npairs; pi += nblk) {
        int P = rr_player((int)pi, rd, N), Q = rr_player(N - 1 - (int)pi, rd, N);
        if (P > Q) { int t_ = P; P = Q; Q = t_; }
        const bool full_e = Q < nb && pair_full(P, Q);
        if (Q >= nb || (!full_e && !pair_dirty(P, Q))) { if (tid == 0) act_flag[pi] = 0; continue; }
        for (int e = tid; e < JP * JP; e += blockDim.x) {
          double sr = 0.0, si = 0.0;
          const cplx<T>* src = Gpart + (size_t)pi * nch * JP * JP + e;
          for (int ch0 = 0; ch0 < nch; ch0 += 8) {   // up to eight loads in flight
            cplx<T> v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = ch0 + u < nch ? ldcg(src + (size_t)(ch0 + u) * JP * JP) : czero<T>();
#pragma unroll
            for (int u = 0; u < 8; ++u) { sr += (double)v[u].x; si += (double)v[u].y; }
          }
          Gs[(e / JP) * LD + (e % JP)] = mk<T>((T)sr, (T)si);
        }
        __shared__ int s_need;
        if (tid == 0) s_need = 0;
        __syncthreads();
        // the test: |G_ij| > max(tol sqrt(G_ii G_jj), floor); the floor is
        // the larger of the global one (initial largest row) and floor_rel
        // times the pair's largest row norm, the level to which a rotation
        // derived from this pair's Gram resolves its entries (rows gain norm
        // as the sweeps concentrate it, so the initial scale alone can sit
        // below what the pair solve can reach and the sweeps never end)
        double gpmax = 0.0;
        for (int i = 0; i < JP; ++i) gpmax = fmax(gpmax, (double)Gs[i * LD + i].x);
        const double pfloor = fmax((double)floor_abs, (double)floor_rel * gpmax);
        for (int e = tid; e < (full_e ? JP * JP : JB * JB); e += blockDim.x) {
          const int i = full_e ? e / JP : e / JB, j = full_e ? e % JP : JB + e % JB;
          if (i >= j) continue;
          const double aij = hypot(Gs[i * LD + j].x, Gs[i * LD + j].y);
          const double thr = fmax((double)tol_rel * sqrt(fabs(Gs[i * LD + i].x * Gs[j * LD + j].x)), pfloor);
          if (aij > thr) s_need = 1;
        }
        __syncthreads();
        const int need = s_need;
        if (need) {
          // Near convergence the pair Gram is diag + a small cross block: one
          // first-order step J = I + E, E_ij = G_ij / (G_jj - G_ii) on the
          // cross entries (E skew-Hermitian), made unitary to rounding by
          // Newton-Schulz steps (J^H J = I - E^2 to start), leaves O(|E|^2)
          // off-diagonals -- quadratic like the Jacobi endgame but with O(1)
          // sequential steps. Those O(|E|^2) residues also land inside the
          // blocks, which cross-only sweeps assume orthogonal, so the step is
          // taken only where they stay below the convergence test: every
          // cross |E_ij| < 0.01 (so |J^H J - I| <= 512 * 1e-4 and the polish
          // converges in a few steps) and JB max|E|^2 max_k G_kk <=
          // max(tol min_k G_kk, floor); outside full-Gram sweeps; else the
          // inner solve.
          int first_order = 0, exact = 1;
          if (!full_e) {
            double gmin = 1e300, gmax = 0.0;
            for (int i = 0; i < JP; ++i) {
              const double d = (double)Gs[i * LD + i].x;
              gmin = fmin(gmin, d);
              gmax = fmax(gmax, d);
            }
            const double e2lim = gmax > 0.0 ? fmax((double)tol_rel * gmin, pfloor) / (JB * gmax) : 0.0;
            int ok = 1;
            for (int e = tid; e < JB * JB; e += blockDim.x) {
              const int i = e / JB, j = JB + e % JB;
              const double gap = fabs((double)Gs[j * LD + j].x - (double)Gs[i * LD + i].x);
              const double gx = (double)Gs[i * LD + j].x, gy = (double)Gs[i * LD + j].y;
              const double g2 = gx * gx + gy * gy;
              if (!(g2 < 1e-4 * gap * gap && g2 <= e2lim * gap * gap)) ok = 0;
            }
            first_order = __syncthreads_and(ok);
          }
          if (first_order) {
            for (int e = tid; e < JP * JP; e += blockDim.x) {
              const int i = e / JP, j = e % JP;
              cplx<T> v = mk<T>(i == j ? T(1) : T(0), T(0));
              if (i < JB && j >= JB) {                 // E_ij = G_ij / (G_jj - G_ii)
                const T den = Gs[j * LD + j].x - Gs[i * LD + i].x;
                v = cscale<T>(Gs[i * LD + j], T(1) / den);
              } else if (i >= JB && j < JB) {          // E_ij = -conj(E_ji)
                const T den = Gs[i * LD + i].x - Gs[j * LD + j].x;
                v = cscale<T>(cconj<T>(Gs[j * LD + i]), T(-1) / den);
              }
              Vs[i * LD + j] = v;
            }
            __syncthreads();
            bj_polish_unitary_to<T>(Vs, Gs, Vs + JP * LD, T(8.0 * eps_of<T>::value * 5.66), 6);
          } else {
            if (tid == 0) {
              T gm = T(0);
              for (int i = 0; i < JP; ++i) gm = fmax(gm, Gs[i * LD + i].x);
              s_gmax = gm;
            }
            __syncthreads();
            exact = bj_inner_eig<T>(Gs, Vs + JP * LD, Vs, 4.0 * (double)eps_of<T>::value * sqrt((double)JP),
                                    32.0 * (double)eps_of<T>::value * (double)s_gmax, 3);
            // FP32: remove the rounding drift of J (FP64 rotations keep it at 1e-16)
            if constexpr (sizeof(T) == 4) bj_polish_unitary<T>(Vs, Gs, Vs + JP * LD);
          }
          for (int e = tid; e < JP * JP; e += blockDim.x) stcg(&Jbuf[(size_t)pi * JP * JP + e], Vs[(e / JP) * LD + (e % JP)]);
          if (tid == 0) {
            act_flag[pi] = 1;
            last_mod[P] = gstamp;
            last_mod[Q] = gstamp;
            wdirty[P] = wdirty[Q] = exact ? 0 : 1;
            atomicAdd(&ctl->active[sweep], 1);
          }
        } else if (tid == 0) {
          act_flag[pi] = 0;
          last_clean[(size_t)P * N + Q] = gstamp;
          if (full_e) wdirty[P] = wdirty[Q] = 0;   // verified by the full Gram
        }
        __syncthreads();
      }
      if (!grid_barrier(&ctl->g, nblk, timeout_ns)) return;
      if (blockIdx.x == 0 && tid == 0) { unsigned long long t2 = global_timer_ns(); ctl->phase_ns[1] += t2 - tph; tph = t2; }
      // ---- phase A: X_PQ <- J^H X_PQ, Ut_PQ <- J^T Ut_PQ -----------------
      // Work items are (active pair, 512-column chunk of X or of Ut), staged
      // GW columns at a time through the same cp.async ring as phase G. Each
      // thread forms a 4 x (GW/32) complex micro-tile of the product: rows
      // 4 ty .. 4 ty + 3 (J from shared memory, a broadcast within the warp)
      // by columns tx + 32 b (consecutive across the warp), eight shared
      // loads per 16 (FP32) complex multiply-adds.
      {
        constexpr int NBC = GW / 32;                         // columns per thread
        const long aitems = (long)npairs * (nch + nchu);
        auto a_valid = [&](long it) -> bool { return __ldcg(&act_flag[(int)(it / (nch + nchu))]) != 0; };
        long p_item = blockIdx.x;
        int p_sub = 0;
        while (p_item < aitems && !a_valid(p_item)) p_item += nblk;
        auto issue = [&](int buf) {
          if (p_item >= aitems) return;
          const int pi_ = (int)(p_item / (nch + nchu)), ch_ = (int)(p_item % (nch + nchu));
          int P_ = rr_player(pi_, rd, N), Q_ = rr_player(N - 1 - pi_, rd, N);
          if (P_ > Q_) { const int t_ = P_; P_ = Q_; Q_ = t_; }
          const bool onU_ = ch_ >= nch;
          const cplx<T>* M_ = onU_ ? Ut : X;
          const int ld_ = onU_ ? r : ldx, ncol_ = onU_ ? r : c;
          const int c0_ = (onU_ ? ch_ - nch : ch_) * JCW, c1_ = min(ncol_, c0_ + JCW), k0 = c0_ + p_sub * GW;
          cplx<T>* tile = ring + buf * JP * TS;
          constexpr int PER = JP * GW / 256;
#pragma unroll
          for (int u = 0; u < PER; ++u) {
            const int e_ = tid + 256 * u, i = e_ / GW, k = e_ % GW;
            const int row = (i < JB ? P_ * JB + i : Q_ * JB + (i - JB));
            const bool in = row < r && k0 + k < c1_;
            cp_async_zfill<(int)sizeof(cplx<T>)>(&tile[i * TS + k],
                                                 in ? (const void*)&M_[(size_t)row * ld_ + k0 + k] : (const void*)M_,
                                                 in ? (int)sizeof(cplx<T>) : 0);
          }
          if (++p_sub == (c1_ - c0_ + GW - 1) / GW) {
            p_sub = 0;
            do { p_item += nblk; } while (p_item < aitems && !a_valid(p_item));
          }
        };
#pragma unroll
        for (int q = 0; q < BJ_NB; ++q) { issue(q); cp_async_commit(); }
        const int ty = tid >> 5, tx = tid & 31;
        int jseq = 0;
        // J of the CTA's next item is loaded into registers while the current
        // item computes, so its L2 round trip is off the critical path
        constexpr int JPER = JP * JP / 256;
        cplx<T> jpre[JPER];
        auto load_j = [&](long it) {
          const int pi_ = (int)(it / (nch + nchu));
#pragma unroll
          for (int u = 0; u < JPER; ++u) {
            const int e = tid + 256 * u, i = e / JP, k = e % JP;
            jpre[u] = ldcg(&Jbuf[(size_t)pi_ * JP * JP + k * JP + i]);
          }
        };
        long item = blockIdx.x;
        while (item < aitems && !a_valid(item)) item += nblk;
        if (item < aitems) load_j(item);
        for (; item < aitems;) {
          const int pi = (int)(item / (nch + nchu)), ch = (int)(item % (nch + nchu));
          int P = rr_player(pi, rd, N), Q = rr_player(N - 1 - pi, rd, N);
          if (P > Q) { int t_ = P; P = Q; Q = t_; }
          const bool onU = ch >= nch;
          cplx<T>* M = onU ? Ut : X;
          const int ld = onU ? r : ldx, ncol = onU ? r : c;
          const int c0 = (onU ? ch - nch : ch) * JCW, c1 = min(ncol, c0 + JCW);
#pragma unroll
          for (int u = 0; u < JPER; ++u) {
            // Js[i][k] = (J^H)[i][k] = conj(J[k][i])  or  (J^T)[i][k] = J[k][i]
            const int e = tid + 256 * u, i = e / JP, k = e % JP;
            Js[i * LD + k] = onU ? jpre[u] : cconj<T>(jpre[u]);
          }
          long next = item + nblk;
          while (next < aitems && !a_valid(next)) next += nblk;
          if (next < aitems) load_j(next);
          int orow[4];
#pragma unroll
          for (int a_ = 0; a_ < 4; ++a_) {
            const int i = 4 * ty + a_;
            orow[a_] = i < JB ? P * JB + i : Q * JB + (i - JB);
          }
          const int nsub = (c1 - c0 + GW - 1) / GW;
          for (int s = 0; s < nsub; ++s, ++jseq) {
            cp_async_wait<BJ_NB - 1>();
            __syncthreads();                    // the stage (and, first time, Js) is visible
            const cplx<T>* tile = ring + (jseq % BJ_NB) * JP * TS;
            cplx<T> acc[4][NBC];
#pragma unroll
            for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
              for (int b_ = 0; b_ < NBC; ++b_) acc[a_][b_] = czero<T>();
#pragma unroll 4
            for (int k = 0; k < JP; ++k) {
              cplx<T> jv[4], xv[NBC];
#pragma unroll
              for (int a_ = 0; a_ < 4; ++a_) jv[a_] = Js[(4 * ty + a_) * LD + k];
#pragma unroll
              for (int b_ = 0; b_ < NBC; ++b_) xv[b_] = tile[k * TS + tx + 32 * b_];
#pragma unroll
              for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
                for (int b_ = 0; b_ < NBC; ++b_) cfma<T>(acc[a_][b_], jv[a_], xv[b_]);
            }
            const int k0 = c0 + s * GW;
#pragma unroll
            for (int a_ = 0; a_ < 4; ++a_) {
              if (orow[a_] >= r) continue;
#pragma unroll
              for (int b_ = 0; b_ < NBC; ++b_) {
                const int col = k0 + tx + 32 * b_;
                if (col < c1) stcg(&M[(size_t)orow[a_] * ld + col], acc[a_][b_]);
              }
            }
            __syncthreads();                    // stage consumed: refill it
            issue(jseq % BJ_NB);
            cp_async_commit();
          }
          item = next;
        }
        cp_async_wait<0>();
        __syncthreads();
      }
      if (!grid_barrier(&ctl->g, nblk, timeout_ns)) return;
      if (blockIdx.x == 0 && tid == 0) ctl->phase_ns[2] += global_timer_ns() - tph;
    }
    // a quiet sweep ends the solve only if it checked every block's own rows:
    // sweep 0 (each block's first pair forms its full Gram) or a verification
    // pass; a quiet cross-only sweep triggers a verification pass
    const bool quiet = atomicAdd(&ctl->active[sweep], 0) == 0;
    const bool was_full = (sweep == 0) || verify;
    if (quiet && was_full) converged = true;
    verify = quiet && !was_full;
  }
  for (long i = gwarp; i < r; i += nwarps) {
    T s = T(0);
    for (int j = lane; j < c; j += 32) { const cplx<T> x = ldcg(&X[(size_t)i * ldx + j]); s += x.x * x.x + x.y * x.y; }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) w[i] = s;
  }
  if (gtid == 0) {
    ctl->g.sweeps = sweep;
    ctl->g.status = converged ? 0 : 1;
  }
}
