// ozgemm.cuh - FP64-accurate complex GEMM on the tcgen05 tensor cores from
// BF16 split products with FP32 accumulation (the error-free splitting
// scheme of Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012):
//
//   C (M x N, complex128) = alpha op(A) op(B) (+ C),  op = plain or ^H.
//
// Splitting. Every row i of op(A) (every column j of op(B)) gets a power of
// two 2^e_i bounding its entries; each real entry x = v / 2^e_i in (-1, 1)
// is written as sum_{t=1..S} a_t 2^{-7t} with integers |a_1| <= 128,
// |a_t| <= 64 for t >= 2 (the balanced base-128 digits of round(x 2^{7S})),
// so every slice value a_t 2^{-7t} is exact in BF16 and every product
// a_t b_u 2^{-7(t+u)} is exact in FP32. Keeping the products with
// t + u <= S + 1 leaves a relative error of about 2^{-7S} of |row| |column|.
//
// Complex as real: op(A)' = [Re | Im] (M x 2K), and the rows of op(B)'^T
// interleave the output's real and imaginary parts: row 2j = [Re b_j | -Im
// b_j], row 2j+1 = [Im b_j | Re b_j], so a real output column pair
// (2j, 2j+1) is the complex column j.
//
// Accumulation. The products of one level L = t + u are summed in their own
// TMEM accumulator: within a level every product is an integer multiple of
// 2^{-7L}, and over a K chunk of KC real terms those integer sums stay far
// below 2^24, so each chunk's sum is exact whatever the alignment and
// rounding inside the tensor core's FP32 accumulation (levels of different
// units must not share an accumulator: their small terms would fall below
// the accumulator's resolution, an error growing with K). After each chunk
// every level is drained to double-float (hi, lo) FP32 registers; the tile's
// value (hi + lo) 2^{e_i + f_j} is formed in FP64 once at the end.
//
// One CTA computes a 128 x 64 real tile (128 rows x 32 complex columns) with
// S 64-column FP32 accumulators (512 TMEM columns allocated). Operand slices are
// staged by cp.async into the K-major no-swizzle core-matrix layout (8 rows x
// 16 bytes per core matrix, SBO = 128 B between 8-row groups, LBO = rows x
// 16 B between the K groups of 8), two stages of 32 real K; one thread
// issues tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulate, M = 128,
// N = 64) and commits each stage to an mbarrier; every wait is bounded.
#pragma once
#include <cuda_bf16.h>
#include "common.cuh"
#include "tcgemm.cuh"

// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes -> v[base .. base + 15]
#define OZ_LD16(v, base, taddr)                                                                               \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
               : "=r"(v[base + 0]), "=r"(v[base + 1]), "=r"(v[base + 2]), "=r"(v[base + 3]),                 \
                 "=r"(v[base + 4]), "=r"(v[base + 5]), "=r"(v[base + 6]), "=r"(v[base + 7]),                 \
                 "=r"(v[base + 8]), "=r"(v[base + 9]), "=r"(v[base + 10]), "=r"(v[base + 11]),               \
                 "=r"(v[base + 12]), "=r"(v[base + 13]), "=r"(v[base + 14]), "=r"(v[base + 15])              \
               : "r"(taddr))

namespace oz {
constexpr int S = 6;                         // slices per operand (about 43 bits)
constexpr int BM = 128, BN = 64;             // real tile: 128 rows x 64 real (32 complex) columns
constexpr int KS = 32;                       // real K per stage (two MMAs of K = 16)
constexpr int KC = 256;                      // real K per exact chunk
constexpr int SPC = KC / KS;                 // stages per chunk
constexpr int A_SLICE = BM * KS * 2;         // 8 KB: one A slice, 128 rows x 32 K
constexpr int B_SLICE = BN * KS * 2;         // 4 KB: one B slice, 64 rows x 32 K
constexpr int A_LBO = BM * 16, B_LBO = BN * 16;   // bytes between the K groups of 8
constexpr int B_OFF = S * A_SLICE;           // B slices follow the A slices in a stage
constexpr int STAGE_BYTES = S * (A_SLICE + B_SLICE);   // 72 KB
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 1024;
constexpr int NT = 512;                      // 16 warps: 4 TMEM lane groups x 4 column groups of 16
constexpr int NACC = S;                      // one accumulator per level L = 2 .. S + 1
constexpr int TCOLS = 512;                   // TMEM allocation (power of two >= NACC * BN)
static_assert(NACC * BN <= TCOLS, "accumulators exceed the TMEM allocation");

// Shared-memory matrix descriptor, K-major, no swizzle: start address, LBO
// (byte step between the core matrices of consecutive K groups), SBO = 128 B
// (step between 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((128 >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
}  // namespace oz

// Scaling exponents. raw[i] = the largest biased FP64 exponent field among
// the real and imaginary parts of row i of op(A) (or column j of op(B)),
// gathered with integer atomicMax (raw zeroed beforehand); the scaling
// exponent is then oz_ex(raw) = raw - 1022 (the frexp exponent of the row's
// largest entry, so every |x| < 2^oz_ex), or 0 for a zero row.
__device__ __forceinline__ int oz_ex(int raw) { return raw > 0 ? raw - 1022 : 0; }
__device__ __forceinline__ int oz_bexp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7FF); }

// The stored matrix (R rows x C columns, leading dimension ld) is scanned in
// 32-column x 256-row tiles, block (32, 8); by_row = 1 reduces along each
// stored row (raw indexed by stored row), 0 along each stored column (raw
// indexed by stored column). One atomic per warp-row or per tile column.
__global__ void oz_exp_kernel(const double2* __restrict__ X, int ld, int R, int C, int by_row, int* __restrict__ raw) {
  __shared__ int red[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 256, ty = threadIdx.y;
  int mcol = 0;
  for (int r = r0 + ty; r < min(R, r0 + 256); r += 8) {
    int v = 0;
    if (c < C) {
      const double2 x = X[(size_t)r * ld + c];
      v = max(oz_bexp(x.x), oz_bexp(x.y));
    }
    if (by_row) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (threadIdx.x == 0 && v > 0) atomicMax(&raw[r], v);
    } else {
      mcol = max(mcol, v);
    }
  }
  if (!by_row) {
    red[ty][threadIdx.x] = mcol;
    __syncthreads();
    if (ty == 0) {
      int v = red[0][threadIdx.x];
#pragma unroll
      for (int i = 1; i < 8; ++i) v = max(v, red[i][threadIdx.x]);
      if (c < C && v > 0) atomicMax(&raw[c], v);
    }
  }
}

// The S slices of x / 2^ex (|x| < 2^ex) by integer arithmetic on the FP64
// bits: N = round(x 2^(7S - ex)), |N| <= 2^(7S), written in balanced base-128
// digits N = sum_t a_t 2^(7(S - t)) (a_t in [-64, 63] for t >= 2 and
// |a_1| <= 128); out[t] = a_{t+1} 2^{-7(t+1)}, exact in BF16. The error
// |x / 2^ex - sum| <= 2^(-7S - 1). No FP64 arithmetic (that unit runs at
// 1/64 of the FP32 rate on this part).
__device__ __forceinline__ void oz_slices(double v, int ex, float* out) {
  const long long bits = __double_as_longlong(v);
  const int be = (int)((bits >> 52) & 0x7FF);
  long long n = 0;
  if (be > 0) {
    const long long mant = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
    const int sh = 1075 - 7 * oz::S + ex - be;     // right shift taking mant 2^(be-1075) to units of 2^(ex - 7S)
    if (sh < 63) {
      const long long mag = sh > 0 ? (mant + (1ll << (sh - 1))) >> sh : mant << (-sh);
      n = bits < 0 ? -mag : mag;
    }
  }
#pragma unroll
  for (int t = oz::S - 1; t >= 1; --t) {
    const long long d = ((n + 64) & 127) - 64;
    out[t] = __int2float_rn((int)d) * __int_as_float((127 - 7 * (t + 1)) << 23);
    n = (n - d) >> 7;
  }
  out[0] = __int2float_rn((int)n) * __int_as_float((127 - 7) << 23);
}

// Slices of op(A)' = [Re | Im] into Asl[t][i][c] (S x Mp x Kp, row-major,
// Kp = 2 K8): c < K8 real parts, K8 <= c < 2 K8 imaginary parts; zero
// outside M x K. Tiles of 32 rows x 32 K through shared memory so that
// both the reads (either op) and the writes are coalesced. grid (K8/32, Mp/32), block (32, 8).
__global__ void oz_split_a_kernel(const double2* __restrict__ A, int lda, int op, int M, int K, int K8, int Mp,
                                  const int* __restrict__ e, __nv_bfloat16* __restrict__ Asl) {
  __shared__ double2 tile[32][33];
  const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    double2 v = make_double2(0.0, 0.0);
    if (op == 0) {                       // tile[i][k] from row i0 + r
      const int i = i0 + r, k = k0 + tx;
      if (i < M && k < K) v = A[(size_t)i * lda + k];
      tile[r][tx] = v;
    } else {                             // tile[i][k] = conj(A[k][i]) from row k0 + r of A
      const int k = k0 + r, i = i0 + tx;
      if (i < M && k < K) { v = A[(size_t)k * lda + i]; v.y = -v.y; }
      tile[tx][r] = v;
    }
  }
  __syncthreads();
  const size_t Kp = 2 * (size_t)K8, sstride = (size_t)Mp * Kp;
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, k = k0 + tx;
    const double2 v = tile[r][tx];
    const int ex = i < M ? oz_ex(e[i]) : 0;
    float sr[oz::S], si[oz::S];
    oz_slices(v.x, ex, sr);
    oz_slices(v.y, ex, si);
#pragma unroll
    for (int t = 0; t < oz::S; ++t) {
      Asl[t * sstride + (size_t)i * Kp + k] = __float2bfloat16_rn(sr[t]);
      Asl[t * sstride + (size_t)i * Kp + K8 + k] = __float2bfloat16_rn(si[t]);
    }
  }
}

// Slices of the interleaved rows of op(B)'^T into Bsl[t][q][c] (S x Nrp x Kp):
// row 2j = [Re b_j | -Im b_j], row 2j + 1 = [Im b_j | Re b_j] (b_j = column j
// of op(B)); zero outside. grid (K8/32, Nrp/64), block (32, 8): 32 complex
// columns (64 rows of Bsl) x 32 K per CTA.
__global__ void oz_split_b_kernel(const double2* __restrict__ B, int ldb, int op, int K, int N, int K8, int Nrp,
                                  const int* __restrict__ f, __nv_bfloat16* __restrict__ Bsl) {
  __shared__ double2 tile[32][33];   // tile[j][k]
  const int j0 = blockIdx.y * 32, k0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    double2 v = make_double2(0.0, 0.0);
    if (op == 0) {                       // row k0 + r of B holds op(B)[k][j0 + tx]
      const int k = k0 + r, j = j0 + tx;
      if (j < N && k < K) v = B[(size_t)k * ldb + j];
      tile[tx][r] = v;
    } else {                             // op(B)[k][j] = conj(B[j][k]): row j0 + r of B
      const int j = j0 + r, k = k0 + tx;
      if (j < N && k < K) { v = B[(size_t)j * ldb + k]; v.y = -v.y; }
      tile[r][tx] = v;
    }
  }
  __syncthreads();
  const size_t Kp = 2 * (size_t)K8, sstride = (size_t)Nrp * Kp;
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, k = k0 + tx;
    const double2 v = tile[r][tx];
    const int ex = j < N ? oz_ex(f[j]) : 0;
    float sr[oz::S], si[oz::S];
    oz_slices(v.x, ex, sr);
    oz_slices(v.y, ex, si);
    const size_t q0 = (size_t)(2 * j) * Kp, q1 = (size_t)(2 * j + 1) * Kp;
#pragma unroll
    for (int t = 0; t < oz::S; ++t) {
      __nv_bfloat16* base = Bsl + t * sstride;
      base[q0 + k] = __float2bfloat16_rn(sr[t]);
      base[q0 + K8 + k] = __float2bfloat16_rn(-si[t]);
      base[q1 + k] = __float2bfloat16_rn(si[t]);
      base[q1 + K8 + k] = __float2bfloat16_rn(sr[t]);
    }
  }
}

// (hi, lo) += x for exact x (Knuth's two-sum; the rounding error of hi + x
// goes to lo).
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// grid (Nrp / 64, Mp / 128), 512 threads, dynamic smem oz::SMEM_BYTES.
// Kp: real K (2 K8), a multiple of oz::KS. status: set to 1 if an mbarrier
// wait ran past timeout_ns (the tile is then left unwritten).
__global__ void __launch_bounds__(512, 1) oz_mma_kernel(int M, int N, int Kp, const __nv_bfloat16* __restrict__ Asl,
                                                        size_t a_sstride, const __nv_bfloat16* __restrict__ Bsl,
                                                        size_t b_sstride, const int* __restrict__ eA,
                                                        const int* __restrict__ eB, double2* __restrict__ C, int ldc,
                                                        double alpha, int accumulate, int* status, long long timeout_ns) {
  using namespace oz;
  extern __shared__ __align__(1024) unsigned char oz_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)oz_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bars[3];   // [0], [1]: stage buffers; [2]: chunk drained-ready
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.y * BM, rcol0 = blockIdx.x * BN;
  const int lg = warp & 3, cg = warp >> 2;   // TMEM lane group (rows 32 lg ..), accumulator column group

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(tcg::saddr(&tmem_base)), "n"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tcg::saddr(&bars[b])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;
  // kind::f16 instruction descriptor: D FP32 (bit 4), A and B BF16 (bits 7, 10), K-major, N >> 3, M >> 4
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

  const int nst = Kp / KS;
  // A stage holds, per slice, the 128 A rows and the 64 B rows of 32 real K
  // as 16-byte pieces (row, K group c) in the core-matrix layout.
  auto load_stage = [&](int s) {
    const uint32_t st = tcg::saddr(sm) + (uint32_t)((s & 1) * STAGE_BYTES);
    const size_t k0 = (size_t)s * KS;
    for (int q = tid; q < S * (BM + BN) * 4; q += NT) {
      const int c = q & 3, rr = q >> 2;            // rr over S x (BM + BN) rows
      const int t = rr / (BM + BN), r = rr % (BM + BN);
      const bool isA = r < BM;
      const int rb = isA ? r : r - BM;
      const __nv_bfloat16* src = isA ? Asl + (size_t)t * a_sstride + (size_t)(row0 + rb) * Kp
                                     : Bsl + (size_t)t * b_sstride + (size_t)(rcol0 + rb) * Kp;
      src += k0 + 8 * c;
      const uint32_t dst = st + (isA ? t * A_SLICE + c * A_LBO : B_OFF + t * B_SLICE + c * B_LBO) +
                           (rb >> 3) * 128 + (rb & 7) * 16;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" :: "r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  // double-float sums of all levels for this thread's 16 accumulator columns
  float hi[16], lo[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) { hi[j] = 0.f; lo[j] = 0.f; }
  uint32_t phase[2] = {0u, 0u}, cphase = 0u;
  uint32_t fresh = (1u << NACC) - 1u;   // accumulators whose next MMA overwrites
  const uint32_t tl = tbase + ((uint32_t)(32 * lg) << 16) + 16 * cg;
  bool ok = true;

  // Per stage s: wait for its operands, issue its MMAs (they run while the
  // next stage is loaded), then wait for the MMAs of stage s - 1 (the other
  // buffer) and refill that buffer with stage s + 1. At the end of a K chunk
  // every thread waits for the chunk's MMAs and drains levels 2..4.
  load_stage(0);
  for (int s = 0; s < nst; ++s) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!ok) s_fail = 1;
    __syncthreads();
    if (s_fail) break;
    const bool chunk_end = ((s + 1) % SPC == 0) || (s + 1 == nst);
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = tcg::saddr(sm + (s & 1) * STAGE_BYTES);
#pragma unroll
      for (int kk = 0; kk < KS / 16; ++kk) {
        for (int t = 0; t < S; ++t) {
          for (int u = 0; t + u + 2 <= S + 1; ++u) {
            const int acc = t + u;           // level L = t + u + 2
            const uint32_t en = (fresh >> acc) & 1u ? 0u : 1u;
            fresh &= ~(1u << acc);
            const uint64_t da = oz::desc(st + t * A_SLICE + kk * 2 * A_LBO, A_LBO);
            const uint64_t db = oz::desc(st + B_OFF + u * B_SLICE + kk * 2 * B_LBO, B_LBO);
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                         :: "r"(tbase + BN * acc), "l"(da), "l"(db), "r"(idesc), "r"(en));
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(tcg::saddr(&bars[s & 1])) : "memory");
      if (chunk_end)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(tcg::saddr(&bars[2])) : "memory");
      if (chunk_end) fresh = (1u << NACC) - 1u;   // every level restarts after the drain
    }
    if (s + 1 < nst) {
      if (s >= 1) {   // the other buffer was read by the MMAs of stage s - 1
        const int b = (s + 1) & 1;
        if (!tcg::wait_parity(tcg::saddr(&bars[b]), phase[b], timeout_ns)) ok = false;
        phase[b] ^= 1u;
      }
      load_stage(s + 1);
    }
    if (chunk_end) {
      if (!tcg::wait_parity(tcg::saddr(&bars[2]), cphase, timeout_ns)) ok = false;
      cphase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (ok) {
        uint32_t v[16];
#pragma unroll
        for (int acc = 0; acc < NACC; ++acc) {
          OZ_LD16(v, 0, tl + BN * acc);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; ++j) df_add(hi[j], lo[j], __uint_as_float(v[j]));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (!ok) s_fail = 1;
      __syncthreads();
      if (s_fail) break;
    }
  }
  if (!s_fail) {
    const int row = row0 + 32 * lg + lane;
    const int er = row < M ? oz_ex(eA[row]) : 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = (rcol0 >> 1) + 8 * cg + q;     // complex column: real part 2q, imaginary 2q + 1
      if (row >= M || j >= N) continue;
      const int sc = er + oz_ex(eB[j]);
      double re = (double)hi[2 * q] + (double)lo[2 * q];
      double im = (double)hi[2 * q + 1] + (double)lo[2 * q + 1];
      re = ldexp(re, sc) * alpha;
      im = ldexp(im, sc) * alpha;
      if (accumulate) { const double2 cv = C[(size_t)row * ldc + j]; re += cv.x; im += cv.y; }
      C[(size_t)row * ldc + j] = make_double2(re, im);
    }
  } else {
    if (tid == 0) atomicExch(status, 1);
    // let MMAs still in flight finish (bounded) before TMEM is released
    (void)tcg::wait_parity(tcg::saddr(&bars[2]), cphase, timeout_ns);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "n"(TCOLS));
}
