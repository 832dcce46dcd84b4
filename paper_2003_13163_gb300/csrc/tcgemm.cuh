// tcgemm.cuh - complex GEMM on the 5th-generation tensor cores (tcgen05) for
// the FP32 form: C (M x N) = alpha * A (M x K) * B (K x N), all row-major
// complex64, no transposes (the theta contraction L(A_i) R(A_{i+1}) and the
// centre-move products).
//
// Complex as real: with A' = [Ar | Ai] (M x 2K) and
//   B' = [[Br, Bi], [-Bi, Br]] (2K x 2N),  A' B' = [Re C | Im C].
// A CTA computes a 128 x 64 complex tile as one 128 x 128 real accumulator in
// tensor memory (columns 0..63 real parts, 64..127 imaginary parts).
// FP32 accuracy from TF32 inputs: x = hi + lo with hi = tf32(x),
// lo = tf32(x - hi); D = Ah Bh + Ah Bl + Al Bh (the lo*lo term is below FP32
// rounding), accumulated in FP32 by the tensor cores.
//
// Operands are staged by the CTA's threads into shared memory in the K-major,
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix; LBO =
// byte step between core matrices along K, SBO = step between 8-row groups),
// two stages deep; one elected thread issues tcgen05.mma and commits each
// stage to an mbarrier; four warps read the accumulator back with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows).
#pragma once
#include <stdint.h>
#include "common.cuh"

namespace tcg {

constexpr int BM = 128;          // tile rows (TMEM lanes)
constexpr int BNC = 64;          // tile complex columns -> 128 real accumulator columns
constexpr int BN = 2 * BNC;      // real N of the MMA
constexpr int BK = 32;           // real K per stage (4 MMAs of K = 8)
constexpr int OP_BYTES = BM * BK * 4;             // one 128 x 32 tf32 operand (A or B^T): 16 KB
constexpr int STAGE_BYTES = 4 * OP_BYTES;         // Ah, Al, Bh, Bl
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 1024; // two stages + alignment slack

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// (row, k) -> byte offset in a 128-row K-major no-swizzle operand of BK columns
__device__ __forceinline__ uint32_t kmaj(int row, int k) {
  return (uint32_t)((row >> 3) * 128 + (row & 7) * 16 + (k >> 2) * (BM * 16) + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(((BM * 16) >> 4) & 0x3FFF) << 16;   // LBO: next core matrix along K
  d |= (uint64_t)((128 >> 4) & 0x3FFF) << 32;         // SBO: next 8-row group
  d |= (uint64_t)1 << 46;                             // descriptor version
  return d;                                           // no swizzle, base offset 0
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity, long long timeout_ns) {
  unsigned long long t0 = 0;
  for (long it = 0;; ++it) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
    if (it == 0) t0 = global_timer_ns();
    else if ((it & 255) == 0 && (long long)(global_timer_ns() - t0) > timeout_ns) return false;
  }
}

#define TCG_LD32(v, base, taddr)                                                                               \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15," \
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                      \
               : "=r"(v[base + 0]), "=r"(v[base + 1]), "=r"(v[base + 2]), "=r"(v[base + 3]),                   \
                 "=r"(v[base + 4]), "=r"(v[base + 5]), "=r"(v[base + 6]), "=r"(v[base + 7]),                   \
                 "=r"(v[base + 8]), "=r"(v[base + 9]), "=r"(v[base + 10]), "=r"(v[base + 11]),                 \
                 "=r"(v[base + 12]), "=r"(v[base + 13]), "=r"(v[base + 14]), "=r"(v[base + 15]),               \
                 "=r"(v[base + 16]), "=r"(v[base + 17]), "=r"(v[base + 18]), "=r"(v[base + 19]),               \
                 "=r"(v[base + 20]), "=r"(v[base + 21]), "=r"(v[base + 22]), "=r"(v[base + 23]),               \
                 "=r"(v[base + 24]), "=r"(v[base + 25]), "=r"(v[base + 26]), "=r"(v[base + 27]),               \
                 "=r"(v[base + 28]), "=r"(v[base + 29]), "=r"(v[base + 30]), "=r"(v[base + 31])                \
               : "r"(taddr))

}  // namespace tcg

// grid: (ceil(N / 64), ceil(M / 128)); 128 threads; dynamic smem tcg::SMEM_BYTES.
// status: set to 1 if an mbarrier wait ran past timeout_ns (the tile is then
// left unwritten).
__global__ void __launch_bounds__(128) tc_cgemm_kernel(int M, int N, int K, const float2* __restrict__ A, int lda,
                                                      const float2* __restrict__ B, int ldb, float2* __restrict__ C,
                                                      int ldc, const double* __restrict__ alpha_dev, double alpha_host,
                                                      int* status, long long timeout_ns) {
  using namespace tcg;
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BNC;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" :: "r"(saddr(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&bars[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&bars[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tacc = tmem_base;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

  // real K runs over [0, Kp) for the real parts and [Kp, 2 Kp) for the
  // imaginary parts, Kp = K rounded up to BK (zero padded)
  const int Kp = (K + BK - 1) / BK * BK;
  const int nstage = 2 * Kp / BK;
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;

  for (int s = 0; s < nstage && ok; ++s) {
    const int b = s & 1;
    unsigned char* Ah = sm + b * STAGE_BYTES;
    unsigned char* Al = Ah + OP_BYTES;
    unsigned char* Bh = Al + OP_BYTES;
    unsigned char* Bl = Bh + OP_BYTES;
    if (s >= 2) {   // the MMAs that read this buffer two stages ago must be done
      if (!wait_parity(saddr(&bars[b]), phase[b], timeout_ns)) { ok = false; break; }
      phase[b] ^= 1u;
    }
    const int kr = s * BK;                      // real-K start of this stage
    const bool imag_half = kr >= Kp;
    const int kc0 = imag_half ? kr - Kp : kr;   // complex column of A / row of B
    // A' rows: [Ar | Ai]; 128 rows x 32 real columns. All loads of a thread
    // are issued before the first conversion (blockDim.x == 128).
    {
      constexpr int PER = BM * BK / 128;
      float xa[PER];
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + 128 * u, rr = e / BK, kk = e % BK;
        const int gr = row0 + rr, gk = kc0 + kk;
        xa[u] = 0.f;
        if (gr < M && gk < K) { const float2 v = A[(size_t)gr * lda + gk]; xa[u] = imag_half ? v.y : v.x; }
      }
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + 128 * u, rr = e / BK, kk = e % BK;
        const uint32_t h = tf32_rna(xa[u]);
        const uint32_t l = tf32_rna(xa[u] - __uint_as_float(h));
        *reinterpret_cast<uint32_t*>(Ah + kmaj(rr, kk)) = h;
        *reinterpret_cast<uint32_t*>(Al + kmaj(rr, kk)) = l;
      }
    }
    // B'^T rows t: t < 64 -> Re column j (Br over the real half, -Bi over the
    // imaginary half); t >= 64 -> Im column j (Bi, then Br)
    {
      constexpr int PER = BN * BK / 128;
      float xb[PER];
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + 128 * u, kk = e / BN, t = e % BN;   // consecutive threads: consecutive columns
        const int j = col0 + (t & (BNC - 1)), gk = kc0 + kk;
        const bool imcol = t >= BNC;
        xb[u] = 0.f;
        if (j < N && gk < K) {
          const float2 v = B[(size_t)gk * ldb + j];
          xb[u] = imcol ? (imag_half ? v.x : v.y) : (imag_half ? -v.y : v.x);
        }
      }
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + 128 * u, kk = e / BN, t = e % BN;
        const uint32_t h = tf32_rna(xb[u]);
        const uint32_t l = tf32_rna(xb[u] - __uint_as_float(h));
        *reinterpret_cast<uint32_t*>(Bh + kmaj(t, kk)) = h;
        *reinterpret_cast<uint32_t*>(Bl + kmaj(t, kk)) = l;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int q = 0; q < BK / 8; ++q) {
        const uint32_t off = (uint32_t)(2 * q * (BM * 16));   // two core matrices along K per MMA
        const uint64_t dAh = tcg::desc(saddr(Ah) + off), dAl = tcg::desc(saddr(Al) + off);
        const uint64_t dBh = tcg::desc(saddr(Bh) + off), dBl = tcg::desc(saddr(Bl) + off);
        const uint32_t acc0 = (s > 0 || q > 0) ? 1u : 0u;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(tacc), "l"(dAh), "l"(dBh), "r"(idesc), "r"(acc0));
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(tacc), "l"(dAh), "l"(dBl), "r"(idesc), "r"(1u));
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(tacc), "l"(dAl), "l"(dBh), "r"(idesc), "r"(1u));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(saddr(&bars[b])) : "memory");
    }
  }
  // drain: wait for the last commit of each buffer still pending
  for (int b = 0; b < 2 && ok; ++b) {
    const int uses = (nstage - b + 1) / 2;        // commits made on buffer b; all but the last were waited for
    if (uses > 0) {
      if (!wait_parity(saddr(&bars[b]), phase[b], timeout_ns)) ok = false;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const double al = alpha_host * (alpha_dev ? *alpha_dev : 1.0);
    const int rr = 32 * warp + lane, gr = row0 + rr;
    uint32_t v[64];
    const uint32_t tw = tacc + ((uint32_t)(32 * warp) << 16);
    for (int half = 0; half < 2; ++half) {      // complex columns [32 half, 32 half + 32)
      TCG_LD32(v, 0, tw + 32 * half);            // real parts
      TCG_LD32(v, 32, tw + 64 + 32 * half);      // imaginary parts
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (gr < M) {
        for (int jj = 0; jj < 32; ++jj) {
          const int j = col0 + 32 * half + jj;
          if (j < N)
            C[(size_t)gr * ldc + j] = make_float2((float)(__uint_as_float(v[jj]) * al), (float)(__uint_as_float(v[32 + jj]) * al));
        }
      }
    }
  } else {
    if (tid == 0) atomicExch(status, 1);
    // best effort: let MMAs still in flight finish (bounded) before TMEM is freed
    for (int b = 0; b < 2; ++b) (void)wait_parity(saddr(&bars[b]), phase[b], timeout_ns);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" :: "r"(tacc));
}
