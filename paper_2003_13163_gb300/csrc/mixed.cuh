// mixed.cuh - kernels of the precision form ("mixed"): the truncated SVD of
// a complex128 matrix A whose approximate left singular basis comes from the
// FP32 one-sided Jacobi SVD of fl32(A) and is refined in FP64:
//
//   Q <- the m leading columns of the FP32 left factor, promoted to FP64 and
//        made orthonormal by Newton-Schulz steps Q <- Q (3 I - Q^H Q) / 2;
//   subspace iteration Q <- orth(A A^H Q), orth = shifted CholeskyQR3;
//   Rayleigh-Ritz: Q turned towards the FP32 basis, B = Q^H A, FP64 one-sided
//        Jacobi SVD B = U_B Lambda W^H, left factor Q U_B, rows Lambda W^H.
//
// The products are the engine's complex GEMM; these kernels convert, gather,
// form the Newton-Schulz multiplier, factor the diagonal blocks of the
// blocked Cholesky factorisation and shift a Gram matrix.
#pragma once
#include "common.cuh"

// out (r x c, FP32, ld c) = fl32(in (r x c, FP64, ld ldi)).
__global__ void to_fp32_kernel(const double2* __restrict__ in, int r, int c, int ldi, float2* __restrict__ out) {
  const size_t total = (size_t)r * c;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / c, j = e % c;
    const double2 v = in[i * ldi + j];
    out[e] = make_float2((float)v.x, (float)v.y);
  }
}

// Q (r x m, FP64, row-major) column j = column perm[j] of U, where the FP32
// one-sided Jacobi returns Ut = U^T (row p of Ut = column p of U, ld r).
__global__ void promote_columns_kernel(const float2* __restrict__ Ut, int r, const int* __restrict__ perm, int m,
                                       double2* __restrict__ Q) {
  const size_t total = (size_t)r * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    const float2 v = Ut[(size_t)perm[j] * r + i];
    Q[e] = make_double2((double)v.x, (double)v.y);
  }
}

// G (m x m) <- (3 I - G) / 2 in place: the Newton-Schulz multiplier
// (Higham, Functions of Matrices, Sec. 8.3).
__global__ void ns_multiplier_kernel(double2* __restrict__ G, int m) {
  const size_t total = (size_t)m * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    double2 g = G[e];
    g.x = (i == j ? 1.5 : 0.0) - 0.5 * g.x;
    g.y = -0.5 * g.y;
    G[e] = g;
  }
}

// ---------------------------------------------------------------------------
// Cholesky factorisation G = L L^H of a Hermitian positive definite
// complex128 matrix with the inverse L^{-1} alongside, by recursive halving
// (the host issues the off-diagonal GEMMs): this kernel is the base case, a
// diagonal block of at most CHOL_NB rows factored in shared memory (Golub &
// Van Loan, Matrix Computations, Sec. 4.2) whose triangular factor is then
// inverted by forward substitution; L goes to the lower triangle of the
// block in G (leading dimension ldg), L^{-1} to Linv (leading dimension ldl,
// zeros above the diagonal). A non-positive pivot sets *status (the
// factorisation then continues with a tiny pivot so that no NaN is
// produced).
// ---------------------------------------------------------------------------
constexpr int CHOL_NB = 32;
constexpr int CHOL_LD = CHOL_NB + 1;
constexpr int CHOL_SMEM = 2 * CHOL_NB * CHOL_LD * (int)sizeof(double2);

__global__ void __launch_bounds__(256) chol_diag_kernel(double2* __restrict__ G, int ldg, int k0, int b,
                                                        double2* __restrict__ Linv, int ldl, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char csm[];
  double2* Ls = reinterpret_cast<double2*>(csm);            // [NB][LD]
  double2* Xs = Ls + CHOL_NB * CHOL_LD;                      // [NB][LD]
  __shared__ double s_inv;
  const int tid = threadIdx.x;
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    Ls[i * CHOL_LD + j] = i >= j ? G[(size_t)(k0 + i) * ldg + k0 + j] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      double d = Ls[j * CHOL_LD + j].x;
      if (!(d > 0.0)) { atomicExch(status, 1); d = 1e-300; }
      d = sqrt(d);
      Ls[j * CHOL_LD + j] = make_double2(d, 0.0);
      s_inv = 1.0 / d;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < b; i += blockDim.x) {
      const double2 v = Ls[i * CHOL_LD + j];
      Ls[i * CHOL_LD + j] = make_double2(v.x * s_inv, v.y * s_inv);
    }
    __syncthreads();
    const int t = b - j - 1;   // trailing block (j+1 .. b-1), lower triangle
    for (int e = tid; e < t * t; e += blockDim.x) {
      const int i = j + 1 + e / t, l = j + 1 + e % t;
      if (l > i) continue;
      const double2 a = Ls[i * CHOL_LD + j], c = Ls[l * CHOL_LD + j];
      double2 v = Ls[i * CHOL_LD + l];
      v.x -= a.x * c.x + a.y * c.y;        // a * conj(c)
      v.y -= a.y * c.x - a.x * c.y;
      Ls[i * CHOL_LD + l] = v;
    }
    __syncthreads();
  }
  // X = L^{-1} by forward substitution, one column per thread
  for (int c = tid; c < b; c += blockDim.x) {
    for (int i = 0; i < b; ++i) {
      if (i < c) { Xs[i * CHOL_LD + c] = make_double2(0.0, 0.0); continue; }
      double xr = (i == c) ? 1.0 : 0.0, xi = 0.0;
      for (int l = c; l < i; ++l) {
        const double2 L_ = Ls[i * CHOL_LD + l], x = Xs[l * CHOL_LD + c];
        xr -= L_.x * x.x - L_.y * x.y;
        xi -= L_.x * x.y + L_.y * x.x;
      }
      const double inv = 1.0 / Ls[i * CHOL_LD + i].x;
      Xs[i * CHOL_LD + c] = make_double2(xr * inv, xi * inv);
    }
  }
  __syncthreads();
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    if (i >= j) G[(size_t)(k0 + i) * ldg + k0 + j] = Ls[i * CHOL_LD + j];
    Linv[(size_t)i * ldl + j] = Xs[i * CHOL_LD + j];
  }
}

// G (m x m) diagonal += rel * trace(G) (the shift of shifted Cholesky QR).
// One CTA.
__global__ void add_trace_shift_kernel(double2* __restrict__ G, int m, double rel) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += G[(size_t)i * m + i].x;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < (blockDim.x + 31) / 32; ++i) v += red[i];
    red[0] = v;
  }
  __syncthreads();
  const double sh = rel * red[0];
  for (int i = threadIdx.x; i < m; i += blockDim.x) G[(size_t)i * m + i].x += sh;
}

// *out = sum |A_ij|^2 over an r x c complex128 matrix (leading dimension lda),
// accumulated in FP64. One CTA (the matrices are at most a few tens of MB).
__global__ void __launch_bounds__(1024) frob2_kernel(const double2* __restrict__ A, int r, int c, int lda,
                                                     double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  const size_t total = (size_t)r * c;
  for (size_t e = threadIdx.x; e < total; e += blockDim.x) {
    const double2 v = A[(e / c) * lda + e % c];
    s += v.x * v.x + v.y * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < (blockDim.x + 31) / 32; ++i) v += red[i];
    *out = v;
  }
}

// x <- conj(x) for n complex128 entries.
__global__ void conj_inplace_kernel(double2* __restrict__ x, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    x[e].y = -x[e].y;
}
