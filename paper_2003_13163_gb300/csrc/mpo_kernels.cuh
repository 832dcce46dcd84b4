// mpo_kernels.cuh - the noisy-gate specific kernels: building the 16x16
// superoperator of each gate, applying it to the two-site tensor theta, and
// the transfer-vector contraction that gives Tr rho.
#pragma once
#include "common.cuh"

// ---------------------------------------------------------------------------
// Superoperator of the noisy gate M = N_2[p] o U (Sec. 3.2) in the App. A
// index convention: row 4*I_l + I_{l+1}, column 4*J_l + J_{l+1}, I = 2 i + i'.
//   (U (x) U*) part: M_U[(I_l,I_r),(J_l,J_r)] = U[2 i_l + i_r, 2 j_l + j_r]
//                                             * conj(U[2 i'_l + i'_r, 2 j'_l + j'_r])
//   depolarising part (Sec. 2.2, second form): with lam = 16 p / 15,
//     N = (1 - lam) 1 + (lam / 4) t t^T, t[(I_l, I_r)] = [i_l = i'_l][i_r = i'_r];
//   since t^T M_U = t^T (unitary conjugation preserves the trace),
//     M = (1 - lam) M_U + (lam / 4) t t^T.
// One CTA per gate, one thread per entry; built in FP64, stored in T.
// gates: [g][4][4] complex128; p: p[g * p_stride].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void build_superop_kernel(const double2* __restrict__ gates, const double* __restrict__ p, int p_stride,
                                     cplx<T>* __restrict__ Ms) {
  const int g = blockIdx.x, e = threadIdx.x;   // e in [0, 256)
  const double2* U = gates + (size_t)g * 16;
  const int row = e >> 4, col = e & 15;
  const int Il = row >> 2, Ir = row & 3, Jl = col >> 2, Jr = col & 3;
  const int il = Il >> 1, ilp = Il & 1, ir = Ir >> 1, irp = Ir & 1;
  const int jl = Jl >> 1, jlp = Jl & 1, jr = Jr >> 1, jrp = Jr & 1;
  const double2 a = U[(2 * il + ir) * 4 + (2 * jl + jr)];
  const double2 b = U[(2 * ilp + irp) * 4 + (2 * jlp + jrp)];
  // a * conj(b)
  double re = a.x * b.x + a.y * b.y;
  double im = a.y * b.x - a.x * b.y;
  const double lam = 16.0 * p[(size_t)g * p_stride] / 15.0;
  const double trow = (il == ilp && ir == irp) ? 1.0 : 0.0;
  const double tcol = (jl == jlp && jr == jrp) ? 1.0 : 0.0;
  re = (1.0 - lam) * re + 0.25 * lam * trow * tcol;
  im = (1.0 - lam) * im;
  Ms[(size_t)g * 256 + e] = mk<T>((T)re, (T)im);
}

// Cast a caller-given complex128 16x16 superoperator into the working type.
template <typename T>
__global__ void cast_superop_kernel(const double2* __restrict__ src, cplx<T>* __restrict__ dst) {
  const int e = threadIdx.x;
  dst[e] = mk<T>((T)src[e].x, (T)src[e].y);
}

// ---------------------------------------------------------------------------
// theta'[(a,I'),(J',c)] = sum_{I,J} M[4I'+J', 4I+J] theta[(a,I),(J,c)]
// (App. A: B = M . (lambda Gamma lambda Gamma lambda)), in place.
// theta is (4 chiL) x (4 chiR) row-major, row a*4+I, column J*chiR + c.
// One thread per (a, c); M staged in shared memory; consecutive threads take
// consecutive c so every one of the 16 loads and stores is coalesced.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) apply_superop_kernel(cplx<T>* __restrict__ theta, int chiL, int chiR,
                                                             const cplx<T>* __restrict__ M) {
  __shared__ cplx<T> Ms[256];
  for (int e = threadIdx.x; e < 256; e += blockDim.x) Ms[e] = M[e];
  __syncthreads();
  const size_t ld = (size_t)4 * chiR;
  const size_t total = (size_t)chiL * chiR;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / chiR), c = (int)(e % chiR);
    cplx<T> in[16];
#pragma unroll
    for (int I = 0; I < 4; ++I)
#pragma unroll
      for (int J = 0; J < 4; ++J) in[4 * I + J] = theta[(size_t)(4 * a + I) * ld + (size_t)J * chiR + c];
#pragma unroll
    for (int o = 0; o < 16; ++o) {
      cplx<T> acc = czero<T>();
#pragma unroll
      for (int i = 0; i < 16; ++i) cfma<T>(acc, Ms[o * 16 + i], in[i]);
      const int Ip = o >> 2, Jp = o & 3;
      theta[(size_t)(4 * a + Ip) * ld + (size_t)Jp * chiR + c] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Trace transfer step (Sec. 3.4): v_out[c] = sum_a v_in[a] (A[a,0,c] + A[a,3,c]),
// the contraction of one site with the vectorised identity (I = (d+1) x).
// v in complex128 regardless of T. One thread per output column.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void trace_step_kernel(const cplx<T>* __restrict__ A, int chiL, int chiR,
                                  const double2* __restrict__ vin, double2* __restrict__ vout) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= chiR) return;
  double re = 0.0, im = 0.0;
#pragma unroll 4
  for (int a = 0; a < chiL; ++a) {
    const cplx<T> x0 = A[(size_t)(4 * a + 0) * chiR + c];
    const cplx<T> x3 = A[(size_t)(4 * a + 3) * chiR + c];
    const double tr = (double)x0.x + (double)x3.x, ti = (double)x0.y + (double)x3.y;
    const double2 v = vin[a];
    re += v.x * tr - v.y * ti;
    im += v.x * ti + v.y * tr;
  }
  vout[c] = make_double2(re, im);
}

// ---------------------------------------------------------------------------
// Right trace environments (Sec. 3.4): R_k[a] = sum_c (A_k[a,0,c] + A_k[a,3,c]) R_{k+1}[c],
// R_n = (1): the contraction of sites k..n-1 with the vectorised identity.
// One thread per row a.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void trace_right_kernel(const cplx<T>* __restrict__ A, int chiL, int chiR,
                                   const double2* __restrict__ rin, double2* __restrict__ rout) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= chiL) return;
  double re = 0.0, im = 0.0;
  const cplx<T>* r0 = A + (size_t)(4 * a + 0) * chiR;
  const cplx<T>* r3 = A + (size_t)(4 * a + 3) * chiR;
#pragma unroll 4
  for (int c = 0; c < chiR; ++c) {
    const double tr = (double)r0[c].x + (double)r3[c].x, ti = (double)r0[c].y + (double)r3[c].y;
    const double2 v = rin[c];
    re += tr * v.x - ti * v.y;
    im += tr * v.y + ti * v.x;
  }
  rout[a] = make_double2(re, im);
}

// ---------------------------------------------------------------------------
// One site of the probability / sampling chain for S strings at once.
// t0 = L A_k[:,0,:] and t1 = L A_k[:,3,:] (S x chiR each, computed by GEMM)
// hold the two continuations x_k = 0, 1 (I = (d+1) x, Sec. 3.4).
//   sampling (uniforms != null): p_x = Re(t_x . R_{k+1}) is proportional to
//     the marginal of the first k bits (Sec. 3.4, sequential conditionals);
//     x_k = 0 if u < p0 / (p0 + p1) else 1 (decided in FP64);
//   probability (bits given): x_k = bits[s * n + k].
// The chosen row is rescaled by its largest |entry| and the log of that
// factor is added to logscale[s], so long chains neither underflow nor
// overflow. One warp per string.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void chain_select_kernel(const cplx<T>* __restrict__ t0, const cplx<T>* __restrict__ t1, int S, int chiR,
                                    const double2* __restrict__ Rnext, const double* __restrict__ uniforms,
                                    unsigned char* __restrict__ bits, int n, int k, cplx<T>* __restrict__ Lout,
                                    double* __restrict__ logscale) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= S) return;
  const cplx<T>* a0 = t0 + (size_t)warp * chiR;
  const cplx<T>* a1 = t1 + (size_t)warp * chiR;
  int x;
  if (uniforms) {
    double p0 = 0.0, p1 = 0.0;
    for (int c = lane; c < chiR; c += 32) {
      const double2 r = Rnext[c];
      p0 += (double)a0[c].x * r.x - (double)a0[c].y * r.y;
      p1 += (double)a1[c].x * r.x - (double)a1[c].y * r.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      p0 += __shfl_xor_sync(0xffffffffu, p0, o);
      p1 += __shfl_xor_sync(0xffffffffu, p1, o);
    }
    p0 = p0 > 0.0 ? p0 : 0.0;   // truncation can leave tiny negative marginals
    p1 = p1 > 0.0 ? p1 : 0.0;
    const double u = uniforms[(size_t)warp * n + k];
    x = (p0 + p1 > 0.0 && u < p0 / (p0 + p1)) ? 0 : 1;
    if (p0 + p1 <= 0.0) x = 0;
    if (lane == 0) bits[(size_t)warp * n + k] = (unsigned char)x;
  } else {
    x = bits[(size_t)warp * n + k] ? 1 : 0;
  }
  const cplx<T>* src = x ? a1 : a0;
  double mx = 0.0;
  for (int c = lane; c < chiR; c += 32) mx = fmax(mx, fmax(fabs((double)src[c].x), fabs((double)src[c].y)));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const double f = mx > 0.0 ? 1.0 / mx : 1.0;
  for (int c = lane; c < chiR; c += 32) Lout[(size_t)warp * chiR + c] = cscale<T>(src[c], (T)f);
  if (lane == 0 && mx > 0.0) logscale[warp] += log(mx);
}
