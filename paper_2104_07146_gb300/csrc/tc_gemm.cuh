// Tensor-core tile products of the mixed forms (a14): one CTA of 128 threads
// computes C(i, j) = sum_k A(i, k) B(k, j) on the tensor cores with
// tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation in tensor memory).
//
// Operand precision.  Each operand value is split into NS BF16 slices,
// a = a_0 + a_1 + ... (a_0 the BF16 rounding of a, a_1 that of the remainder,
// and so on), and the products a_p b_q with p + q < NS are accumulated in
// FP32.  NS = 1 is the plain BF16 product; NS = 2 adds the two cross terms of
// the high and low halves (three products, operands carried to 16 bits);
// NS = 3 carries the operands to 24 bits, the FP32 significand, with six
// products.  This is the split-BF16 scheme of Henry, Tang and Heinecke
// ("Leveraging the bfloat16 artificial intelligence datatype for
// higher-precision computations", ARITH 2019).  The operands are first
// rounded to FP32 with integer operations (round to nearest even; values below
// the FP32 normal range become zero), so no FP64 instruction is spent on them.
//
// Layout.  The MMA tile is 128 x 64 (M x N), K advances 16 per instruction.
// Both operands are staged K-major without swizzling: the canonical layout is
// made of 8-row x 16-byte "core matrices" (8 BF16 values of one row, rows
// 16 bytes apart, 128 contiguous bytes).  A chunk of KC values of k holds
// KC / 8 core matrices per group of 8 rows, so core matrix (row group g,
// k group q) starts at g * 16 KC + 128 q: the leading-dimension byte offset
// (between K-adjacent core matrices) is 128 and the stride-dimension byte
// offset (between 8-row groups) is 16 KC.  One instruction reads two
// K-adjacent core matrices, so the k-th instruction of a chunk starts 256 k
// bytes in.
//
// Flow per output tile: the 4 warps gather a chunk of A (128 rows) and B
// (64 rows, that is 64 columns of the result) through the caller's accessors
// into one of two stages; one thread issues the chunk's MMAs and commits them
// to that stage's mbarrier, and the warps go on to gather the next chunk into
// the other stage, waiting on a stage's mbarrier before overwriting it.
// After the last chunk, warp w reads TMEM lanes 32w..32w+31 (rows of the
// tile) with tcgen05.ld and hands every element to the caller's fc(i, j, v).
//
// Every wait on an mbarrier is bounded: a wait that runs out raises
// kFlagTimeout in the caller's flag word, the CTA waits (again bounded) for
// the MMAs it issued, frees its tensor memory and returns without output.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace hmle {
namespace tc {

// Tag type selecting the tensor-core products with NS BF16 slices per
// operand (the Tc template parameter of the sweep's product kernels).
template <int NS>
struct Split {
  static_assert(NS >= 1 && NS <= 3, "one to three BF16 slices");
};

constexpr int kTM = 128;                      // rows of the MMA tile = TMEM lanes
constexpr int kTN = 64;                       // columns of the MMA tile = FP32 TMEM columns
constexpr uint32_t kTmemCols = 64;            // power of two >= 32
constexpr unsigned long long kWaitNs = 1000000000ull;   // a wait gives up after one second

// values of k per staged chunk, and the shared memory of the two stages
template <int NS> __host__ __device__ constexpr int chunk_k() { return NS == 1 ? 64 : 32; }
template <int NS> __host__ __device__ constexpr int a_bytes() { return kTM * chunk_k<NS>() * 2; }   // one slice of A
template <int NS> __host__ __device__ constexpr int b_bytes() { return kTN * chunk_k<NS>() * 2; }   // one slice of B
template <int NS> __host__ __device__ constexpr int stage_bytes() { return NS * (a_bytes<NS>() + b_bytes<NS>()); }
template <int NS> __host__ __device__ constexpr int smem_words() { return (2 * stage_bytes<NS>() + 128 + 7) / 8; }

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits
// 4-5 = 1), A and B BF16 (bits 7-9 and 10-12 = 1), both K-major (bits 15,
// 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset 128 >> 4 (bits 16-29), stride byte offset sbo >> 4 (bits
// 32-45), the fixed version bits 46-48 = 0b001, no swizzling (bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// FP32 rounding of a double by integer operations: round to nearest even,
// |x| below 2^-126 to a signed zero, beyond the FP32 range to infinity, NaN
// stays NaN.
__device__ __forceinline__ float to_f32(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(bits >> 32), lo = (uint32_t)bits;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
  const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // top 23 of the 52 fraction bits
  const uint32_t rest = lo & 0x1FFFFFFFu;                   // the 29 bits rounded away
  uint32_t r = ((uint32_t)(e & 0xFF) << 23) | m;
  if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) r += 1u;   // a carry moves to the next binade
  if (e <= 0) r = 0u;
  if (e >= 255)
    r = ((hi & 0x7FF00000u) == 0x7FF00000u && ((hi & 0xFFFFFu) | lo)) ? 0x7FC00000u : 0x7F800000u;
  return __uint_as_float(sign | r);
}

// The NS BF16 slices of eight values, packed two per 32-bit word (the lower
// k in the low half): w[p] holds slice p of the eight values.
template <int NS>
__device__ __forceinline__ void slices8(const double *v, uint4 *w) {
  uint32_t o[NS][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float a = to_f32(v[2 * e]), b = to_f32(v[2 * e + 1]);
#pragma unroll
    for (int p = 0; p < NS; ++p) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
      o[p][e] = *reinterpret_cast<const uint32_t *>(&h);
      if (p + 1 < NS) {
        a -= __bfloat162float(h.x);   // exact: the remainder fits in FP32
        b -= __bfloat162float(h.y);
      }
    }
  }
#pragma unroll
  for (int p = 0; p < NS; ++p) w[p] = make_uint4(o[p][0], o[p][1], o[p][2], o[p][3]);
}

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the completion of phase `parity` of the mbarrier: false
// after kWaitNs of global time.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity) {
  if (try_wait(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (!try_wait(bar, parity))
    if (now_ns() - t0 > kWaitNs) return false;
  return true;
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int x = 0; x < 16; ++x) v[x] = __uint_as_float(r[x]);
}

// Stage rows [r0, r0 + ROWS) x k [k0, k0 + KC) of an operand given by
// f(row, k) (rows >= nrows and k >= K are zero) as NS slices, slice p at
// dst + p * ROWS * KC * 2.  KFAST: the operand is contiguous along k in
// memory, so a thread reads 8 consecutive k of a row and 8 threads cover
// 8 rows of one k group; otherwise consecutive threads take consecutive rows.
// Both orders store 8 threads' 16-byte pieces into 128 contiguous bytes.
template <int NS, bool KFAST, int ROWS, class F>
__device__ __forceinline__ void stage(uint8_t *dst, int r0, int nrows, int k0, int K, F f) {
  constexpr int KC = chunk_k<NS>(), QN = KC / 8, kUnits = ROWS * QN;
  constexpr int kSlice = ROWS * KC * 2;
  for (int u = threadIdx.x; u < kUnits; u += 128) {
    int row, q;
    if (KFAST) { row = (u / (8 * QN)) * 8 + (u & 7); q = (u >> 3) % QN; }
    else { row = u % ROWS; q = u / ROWS; }
    const int gr = r0 + row, kb = k0 + q * 8;
    uint4 w[NS];
#pragma unroll
    for (int p = 0; p < NS; ++p) w[p] = make_uint4(0u, 0u, 0u, 0u);
    if (gr < nrows && kb < K) {
      double v[8];
      if (kb + 8 <= K) {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = f(gr, kb + e);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (kb + e < K) ? f(gr, kb + e) : 0.0;
      }
      slices8<NS>(v, w);
    }
    const uint32_t off = (uint32_t)((row >> 3) * (16 * KC) + q * 128 + (row & 7) * 16);
#pragma unroll
    for (int p = 0; p < NS; ++p) *reinterpret_cast<uint4 *>(dst + p * kSlice + off) = w[p];
  }
}

// C(i, j) = sum_k A(i, k) B(k, j), i < M, j < N, k < K, delivered once per
// element to fc(i, j, value).  fa(i, k), fb(k, j) return doubles; A_KFAST /
// B_KFAST: the operand is contiguous along k in memory.  smem: at least
// smem_words<NS>() doubles of dynamic shared memory.  128 threads.  flags:
// the caller's error word (kFlagTimeout).
// Compensated addition (TwoSum): hi + lo holds the running sum to about
// twice the FP32 precision.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float v) {
  const float s = hi + v;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}

template <int NS, bool A_KFAST, bool B_KFAST, class FA, class FB, class FC>
__device__ void gemm(int M, int N, int K, FA fa, FB fb, FC fc, double *smem, int *flags) {
  constexpr int KC = chunk_k<NS>();
  constexpr uint32_t kSbo = 16 * KC;
  // With several slices (the mixed forms' long sums) every group of kGroup
  // chunks (128 values of k) is accumulated in its own TMEM region (two,
  // alternating) and read out into compensated FP32 registers, so the FP32
  // rounding of the tensor cores' accumulation spans 128 terms, not the whole
  // of K, while a product with K <= 128 reads its tile out once.
  constexpr bool kChunked = NS >= 2;
  constexpr int kGroup = kChunked ? 128 / KC : 1;
  constexpr uint32_t kCols = kChunked ? 2 * kTmemCols : kTmemCols;
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5;
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem) + 127) & ~(uintptr_t)127);
  const uint32_t bar0 = smem_addr(&s_bar[0]);   // stage s: bar0 + 8 s
  if (M <= 0 || N <= 0) return;
  __syncthreads();   // earlier users of this shared memory are done
  if (warp == 0)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                 "r"(kCols)
                 : "memory");
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8u), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;   // this warp's TMEM lanes
  uint32_t phase = 0u, pending = 0u;   // bit s: parity to wait for / MMAs in flight on stage s
  // bounded wait for the MMAs of stage s; false if it ran out
  auto drain = [&](int s) -> bool {
    if (!((pending >> s) & 1u)) return true;
    if (!wait_bar(bar0 + 8u * s, (phase >> s) & 1u)) return false;
    phase ^= 1u << s;
    pending &= ~(1u << s);
    return true;
  };
  float hi[kChunked ? kTN : 1], lo[kChunked ? kTN : 1];
  uint32_t unread = 0u;                // bit r: TMEM region r holds a group not yet added
  // add TMEM region s (one group's partial products) into hi / lo
  auto absorb = [&](int s) {
    if constexpr (kChunked) {
      if (!((unread >> s) & 1u)) return;
      unread &= ~(1u << s);
      fence_after();
#pragma unroll
      for (int j0 = 0; j0 < kTN; j0 += 16) {
        float v[16];
        ld16(tmem + lane_base + (uint32_t)(s * kTN + j0), v);
#pragma unroll
        for (int x = 0; x < 16; ++x) two_sum_add(hi[j0 + x], lo[j0 + x], v[x]);
      }
      fence_before();
    }
  };
  bool failed = false;
  const int nk = K > 0 ? (K + KC - 1) / KC : 1;   // K = 0: one chunk of zeros
  for (int m0 = 0; m0 < M && !failed; m0 += kTM) {
    for (int n0 = 0; n0 < N && !failed; n0 += kTN) {
      if constexpr (kChunked) {
#pragma unroll
        for (int x = 0; x < kTN; ++x) { hi[x] = 0.0f; lo[x] = 0.0f; }
      }
      for (int c = 0; c < nk; ++c) {
        const int s = c & 1;
        const bool late = !drain(s);
        if (__syncthreads_or(late)) { failed = true; break; }
        // chunks up to c - 2 are complete: if c - 2 ends its group, add the
        // group's region (chunk c - 1 and this chunk write the other one)
        if (c >= 2 && (c - 2) % kGroup == kGroup - 1) absorb(((c - 2) / kGroup) & 1);
        uint8_t *sa = base + s * stage_bytes<NS>();
        uint8_t *sb = sa + NS * a_bytes<NS>();
        const int k0 = c * KC;
        stage<NS, A_KFAST, kTM>(sa, m0, M, k0, K, fa);
        stage<NS, B_KFAST, kTN>(sb, n0, N, k0, K, [&](int j, int k) { return fb(k, j); });
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          fence_after();
          const uint32_t a0 = smem_addr(sa), b0 = smem_addr(sb);
          const int rg = (c / kGroup) & 1;   // this chunk's TMEM region
          const uint32_t dst = tmem + (kChunked ? (uint32_t)(rg * kTN) : 0u);
#pragma unroll
          for (int kk = 0; kk < KC / 16; ++kk) {
            // the small cross terms first, the product of the leading slices last
#pragma unroll
            for (int w = NS - 1; w >= 0; --w)
#pragma unroll
              for (int p = 0; p <= w; ++p) {
                const uint32_t ao = a0 + (uint32_t)(p * a_bytes<NS>()) + 256u * kk;
                const uint32_t bo = b0 + (uint32_t)((w - p) * b_bytes<NS>()) + 256u * kk;
                const bool first = ((kChunked ? c % kGroup == 0 : c == 0) && kk == 0 && w == NS - 1 && p == 0);
                mma(dst, sdesc(ao, kSbo), sdesc(bo, kSbo), first ? 0u : 1u);
              }
          }
          commit(bar0 + 8u * s);
        }
        pending |= 1u << s;
        unread |= 1u << ((c / kGroup) & 1);
      }
      if (failed) break;
      const int last = (nk - 1) & 1;   // the last two chunks, older first
      bool late = !drain(last ^ 1);
      late |= !drain(last);
      if (__syncthreads_or(late)) { failed = true; break; }
      fence_after();
      const int i = m0 + warp * 32 + (tid & 31);
      if constexpr (kChunked) {
        const int g = (nk - 1) / kGroup;   // the last group, and the one before it if not yet added
        absorb((g + 1) & 1);
        absorb(g & 1);
        if (i < M) {
#pragma unroll
          for (int x = 0; x < kTN; ++x)
            if (n0 + x < N) fc(i, n0 + x, (double)hi[x] + (double)lo[x]);
        }
      } else {
        for (int j0 = 0; j0 < kTN && n0 + j0 < N; j0 += 16) {
          float v[16];
          ld16(tmem + lane_base + (uint32_t)j0, v);
          if (i < M) {
#pragma unroll
            for (int x = 0; x < 16; ++x)
              if (n0 + j0 + x < N) fc(i, n0 + j0 + x, (double)v[x]);
          }
        }
      }
      fence_before();
      __syncthreads();   // TMEM read before the next tile's MMAs overwrite it
    }
  }
  if (failed) {
    if (tid == 0) raise_flag(flags, kFlagTimeout);
    drain(0);   // bounded: the MMAs this CTA issued and has not seen complete
    drain(1);
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
  if (tid == 0) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar0 + 8u) : "memory");
  }
  __syncthreads();
}

}  // namespace tc
}  // namespace hmle
