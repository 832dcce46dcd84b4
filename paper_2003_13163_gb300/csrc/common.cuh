// common.cuh - complex arithmetic and small device helpers shared by the
// engine's kernels. Complex numbers are interleaved (re, im) pairs: double2 for
// the FP64 form, float2 for the FP32 form.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

template <typename T> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };
template <typename T> using cplx = typename cplx_t<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T re, T im) { cplx<T> z; z.x = re; z.y = im; return z; }
template <typename T> __host__ __device__ __forceinline__ cplx<T> czero() { return mk<T>(T(0), T(0)); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) { return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __host__ __device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// acc += a * b
template <typename T> __device__ __forceinline__ void cfma(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}

// L2-only loads/stores (bypass the non-coherent L1) for data that other CTAs
// of the same persistent kernel write between grid barriers.
__device__ __forceinline__ double2 ldcg(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ldcg(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ void stcg(double2* p, double2 v) { __stcg(p, v); }
__device__ __forceinline__ void stcg(float2* p, float2 v) { __stcg(p, v); }

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Control block of a persistent cooperative kernel: a sense-counting grid
// barrier plus status words. Zeroed by the host before every launch.
struct GridCtl {
  unsigned int count;
  unsigned int gen;
  int err;        // 1: a barrier wait ran past its time limit
  int status;     // kernel-specific status (e.g. not converged)
  int sweeps;     // kernel-specific counter
  int pad[3];
};

// Grid-wide barrier for a cooperatively launched kernel (all CTAs resident).
// Every wait is bounded by timeout_ns of wall time: on expiry the CTA sets
// ctl->err and every CTA leaves at its next barrier, so a broken launch ends
// with an error status instead of hanging the GPU. Returns false on error.
__device__ __forceinline__ bool grid_barrier(GridCtl* ctl, unsigned int nblocks, long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = &ctl->gen;
    volatile int* verr = &ctl->err;
    unsigned int g = *vgen;
    __threadfence();
    unsigned int arrived = atomicAdd(&ctl->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&ctl->count, 0u);
      __threadfence();
      atomicAdd(&ctl->gen, 1u);
    } else {
      unsigned long long t0 = global_timer_ns();
      while (*vgen == g) {
        if (*verr) { ok = 0; break; }
        if ((long long)(global_timer_ns() - t0) > timeout_ns) { atomicExch(&ctl->err, 1); ok = 0; break; }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (*verr) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T> struct eps_of;
template <> struct eps_of<double> { static constexpr double value = 2.220446049250313e-16; };
template <> struct eps_of<float> { static constexpr float value = 1.1920929e-07f; };
