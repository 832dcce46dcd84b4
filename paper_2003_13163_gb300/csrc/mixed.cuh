// mixed.cuh - kernels of the precision form ("mixed"): the truncated SVD of
// a complex128 matrix A (App. A) with FP64-class products on the tensor cores
// and FP32 solves, refined to FP64 accuracy:
//
//   subspace iteration from a seeded Gaussian start, Q <- orth(A orth(A^H Q)),
//        orth = mixed-precision Cholesky QR (FP64-class Gram, FP32 Cholesky of
//        the diagonally scaled Gram, FP64-class product), Newton-Schulz steps
//        Q <- Q (3 I - Q^H Q) / 2 for the final orthonormality;
//   FP32 Rayleigh-Ritz (one-sided Jacobi) on the iterated subspace, and a
//        first-order correction of its leading directions for the coupling
//        the FP32 solve leaves to the rest of the subspace;
//   FP64 Rayleigh-Ritz on those directions: B = Q'^H A, H = B B^H and the FP64
//        Hermitian Jacobi eigen-solve H = V Lambda^2 V^H; left factor Q' V,
//        rows V^H B.
//
// The products are the engine's complex GEMM; these kernels convert, gather,
// draw the start basis, form the Newton-Schulz multiplier and the Cholesky QR
// factors, reduce norms and defects, make a Gram matrix Hermitian and form
// the first-order correction.
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
// Cholesky factorisation G = L L^H of a Hermitian positive definite complex
// matrix with the inverse L^{-1} alongside, by recursive halving (the host
// issues the off-diagonal GEMMs): this kernel is the base case, a diagonal
// block of at most NB rows factored in shared memory (Golub & Van Loan,
// Matrix Computations, Sec. 4.2) whose triangular factor is then inverted by
// forward substitution; L goes to the lower triangle of the block in G
// (leading dimension ldg), L^{-1} to Linv (leading dimension ldl, zeros above
// the diagonal). A non-positive pivot sets *status (the factorisation then
// continues with a tiny pivot so that no NaN is produced). The precision
// form instantiates it in FP32 with NB = 64.
// ---------------------------------------------------------------------------
template <typename T, int NB>
constexpr int chol_smem_bytes() { return 2 * NB * (NB + 1) * (int)sizeof(cplx<T>); }
constexpr int CHOL32_NB = 64;     // FP32 base block

template <typename T, int NB>
__global__ void __launch_bounds__(256) chol_diag_kernel(cplx<T>* __restrict__ G, int ldg, int k0, int b,
                                                        cplx<T>* __restrict__ Linv, int ldl, int* __restrict__ status) {
  constexpr int LD = NB + 1;
  extern __shared__ __align__(16) unsigned char csm[];
  cplx<T>* Ls = reinterpret_cast<cplx<T>*>(csm);            // [NB][LD]
  cplx<T>* Xs = Ls + NB * LD;                                // [NB][LD]
  __shared__ T s_inv;
  const int tid = threadIdx.x;
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    Ls[i * LD + j] = i >= j ? G[(size_t)(k0 + i) * ldg + k0 + j] : czero<T>();
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      T d = Ls[j * LD + j].x;
      if (!(d > T(0))) { atomicExch(status, 1); d = sizeof(T) == 8 ? T(1e-300) : T(1e-30); }
      d = sqrt(d);
      Ls[j * LD + j] = mk<T>(d, T(0));
      s_inv = T(1) / d;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < b; i += blockDim.x) Ls[i * LD + j] = cscale<T>(Ls[i * LD + j], s_inv);
    __syncthreads();
    const int t = b - j - 1;   // trailing block (j+1 .. b-1), lower triangle
    for (int e = tid; e < t * t; e += blockDim.x) {
      const int i = j + 1 + e / t, l = j + 1 + e % t;
      if (l > i) continue;
      Ls[i * LD + l] = csub<T>(Ls[i * LD + l], cmul<T>(Ls[i * LD + j], cconj<T>(Ls[l * LD + j])));
    }
    __syncthreads();
  }
  // X = L^{-1} by forward substitution, one column per thread
  for (int c = tid; c < b; c += blockDim.x) {
    for (int i = 0; i < b; ++i) {
      if (i < c) { Xs[i * LD + c] = czero<T>(); continue; }
      cplx<T> x = mk<T>(i == c ? T(1) : T(0), T(0));
      for (int l = c; l < i; ++l) x = csub<T>(x, cmul<T>(Ls[i * LD + l], Xs[l * LD + c]));
      Xs[i * LD + c] = cscale<T>(x, T(1) / Ls[i * LD + i].x);
    }
  }
  __syncthreads();
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    if (i >= j) G[(size_t)(k0 + i) * ldg + k0 + j] = Ls[i * LD + j];
    Linv[(size_t)i * ldl + j] = Xs[i * LD + j];
  }
}

// Mixed-precision Cholesky QR, first half: A (m x m, FP32) = fl32(D G D) +
// shift I with D = diag(G)^{-1/2} (a zero column gets d = 0), so that the
// FP32 Cholesky factors a unit-diagonal matrix whatever the column scales;
// d goes to dvec.
__global__ void scale_gram_fp32_kernel(const double2* __restrict__ G, int m, float shift, float2* __restrict__ A,
                                       double* __restrict__ dvec) {
  const size_t total = (size_t)m * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    const double gi = G[(size_t)i * m + i].x, gj = G[(size_t)j * m + j].x;
    const double di = gi > 1e-300 ? rsqrt(gi) : 0.0, dj = gj > 1e-300 ? rsqrt(gj) : 0.0;
    const double2 g = G[e];
    A[e] = make_float2((float)(di * dj * g.x) + (i == j ? shift : 0.0f), (float)(di * dj * g.y));
    if (i == j) dvec[i] = di;
  }
}

// Second half: W (m x m, FP64) = D L^{-H} from the FP32 inverse factor
// Linv = L^{-1} (lower triangular): W_ij = d_i conj(Linv_ji), upper triangle.
// Y W then has Gram L^{-1} (D G D) L^{-H}, close to the identity.
__global__ void form_w_kernel(const float2* __restrict__ Linv, const double* __restrict__ dvec, int m,
                              double2* __restrict__ W) {
  const size_t total = (size_t)m * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    const float2 l = Linv[(size_t)j * m + i];
    W[e] = j >= i ? make_double2(dvec[i] * (double)l.x, -dvec[i] * (double)l.y) : make_double2(0.0, 0.0);
  }
}

// Seeded complex Gaussian start basis for the subspace iteration: entry e
// draws two uniforms from the SplitMix64 sequence (Steele, Lea & Flood 2014)
// at counter 2e, 2e+1 of the given seed and turns them into a standard
// complex normal by the Box-Muller transform.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void gauss_start_kernel(double2* __restrict__ out, size_t n, unsigned long long seed) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long a = splitmix64(seed + 2 * e), b = splitmix64(seed + 2 * e + 1);
    const double u1 = ((double)(a >> 11) + 1.0) * (1.0 / 9007199254740993.0);   // (0, 1]
    const double u2 = (double)(b >> 11) * (1.0 / 9007199254740992.0);           // [0, 1)
    const double rad = sqrt(-log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[e] = make_double2(rad * cs, rad * sn);
  }
}

// *out += sum |A_ij|^2 over an r x c complex128 matrix (leading dimension
// lda), accumulated in FP64: grid-stride partial sums, one atomicAdd per CTA
// (*out zeroed beforehand).
__global__ void __launch_bounds__(256) frob2_kernel(const double2* __restrict__ A, int r, int c, int lda,
                                                    double* __restrict__ out) {
  __shared__ double red[8];
  double s = 0.0;
  const size_t total = (size_t)r * c;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const double2 v = A[(e / c) * lda + e % c];
    s += v.x * v.x + v.y * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < 8; ++i) v += red[i];
    atomicAdd(out, v);
  }
}

// H (m x m) <- (H + H^H) / 2 in place: the Gram matrix of the Rayleigh-Ritz
// step made exactly Hermitian (its two triangles come from separately rounded
// products) before the Hermitian eigen-solver, which reads one triangle.
__global__ void hermitise_kernel(double2* __restrict__ H, int m) {
  const size_t total = (size_t)m * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    if (j < i) continue;
    if (j == i) { H[e].y = 0.0; continue; }
    const double2 a = H[e], b = H[(size_t)j * m + i];
    const double2 v = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    H[e] = v;
    H[(size_t)j * m + i] = make_double2(v.x, -v.y);
  }
}

// First-order correction of a partition of approximate eigenvectors
// (one refinement step of Ogita & Aishima, Japan J. Indust. Appl. Math. 35
// (2018), restricted to the coupling between the leading mp directions P and
// the remaining ones R): with the approximate eigenvector matrix V (m x m),
// S = V^H H V and G = V^H V (both FP64-accurate), R = I - G and
// lambda_i = S_ii / (1 - R_ii), the columns i in P gain the components
//   E_ji = (S_ji + lambda_i R_ji) / (lambda_i - lambda_j),   j in R,
// which removes their error along R to first order; pairs whose relative gap
// is below 1e-2 (P and R meet inside a cluster, only in the margin beyond the
// kept directions) get the orthogonality term R_ji / 2 alone.
// Output E ((m - mp) x mp, row j - mp, column i).
__global__ void partition_correction_kernel(const double2* __restrict__ S, const double2* __restrict__ G, int m, int mp,
                                            double2* __restrict__ E) {
  const size_t total = (size_t)(m - mp) * mp;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = mp + (int)(e / mp), i = (int)(e % mp);
    const double li = S[(size_t)i * m + i].x / G[(size_t)i * m + i].x;
    const double lj = S[(size_t)j * m + j].x / G[(size_t)j * m + j].x;
    const double2 s = S[(size_t)j * m + i];
    const double2 g = G[(size_t)j * m + i];
    const double2 rji = make_double2(-g.x, -g.y);      // (I - G)_ji, j != i
    const double gap = li - lj;
    double2 v;
    if (fabs(gap) > 1e-2 * fmax(fabs(li), fabs(lj)))
      v = make_double2((s.x + li * rji.x) / gap, (s.y + li * rji.y) / gap);
    else
      v = make_double2(0.5 * rji.x, 0.5 * rji.y);
    E[e] = v;
  }
}

// *out = max_ij |G_ij - delta_ij| over an m x m complex128 matrix: the
// orthonormality defect of a basis whose Gram matrix is G. Grid-stride
// maxima, one atomicMax per CTA on the bit pattern (order-preserving for
// non-negative doubles); *out zeroed beforehand.
__global__ void __launch_bounds__(256) defect_kernel(const double2* __restrict__ G, int m, double* __restrict__ out) {
  __shared__ double red[8];
  double s = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)m * m; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / m, j = e % m;
    const double2 g = G[e];
    s = fmax(s, hypot(g.x - (i == j ? 1.0 : 0.0), g.y));
  }
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < 8; ++i) v = fmax(v, red[i]);
    atomicMax((unsigned long long*)out, (unsigned long long)__double_as_longlong(v));
  }
}
