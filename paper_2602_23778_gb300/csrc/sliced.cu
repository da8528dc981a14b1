// Split-precision (error-free sliced) product W = (A - shift I) X on the
// tcgen05 tensor cores, F16 operands, FP32 accumulation in TMEM.
//
// Slicing (Ozaki, Ogita, Oishi and Rump's error-free splitting, BIT 2012):
// every row i of A is scaled by 2^-e_i (e_i = exponent of the row's largest
// |a_il|, so |a_il 2^-e_i| < 1), rounded to a 63-bit integer M (at S = 8) and
// written as S balanced base-256 digits, a_il 2^-e_i = sum_s d_s 2^-(8s+7) + r
// with d_0 in [0, 128], d_s in [-128, 127] (s >= 1), |r| <= 2^-(8S) .  Every
// column j of X gets the same treatment with its own exponent f_j.  Each
// digit has at most 8 significant bits, hence is exact in F16, and a digit
// product (at most 2^14) is exact in FP32.  The product keeps the S(S+1)/2
// digit pairs with s + t <= S - 1 (triangular truncation):
//     W_ij = 2^(e_i + f_j) sum_w 2^-(8w+14) C_w,   C_w = sum_{s+t=w} A_s X_t
// (0-based s, t, w).  C_w is accumulated in FP32 over K chunks of 128: a
// weight group has at most S = 8 pairs, so every partial sum is at most
// 8 x 2^14 x 128 = 2^24 in magnitude and every FP32 addition is exact.  After
// each chunk the epilogue warps move C_w into two int64 registers per output
// (hi = sum_{w<4} C_w 2^8(3-w), lo = sum_{w>=4} C_w 2^8(S-1-w)), exact
// integer arithmetic; at the end W_ij = 2^(e_i+f_j) (hi 2^-38 + lo
// 2^-(8S+6)) with one rounding.  The only errors are the rounding of M and
// the truncated digit pairs: per product term about (S + 2) 2^-8S of the
// scaled operands.  (Eight-bit digits: 36 plane pairs for 63 bits, against
// 45 with seven-bit digits.)
//
// Kernel: a CTA owns 128 rows x 32 columns of W over a range of K (the
// product's equal-work plan: a range of (row tile, K block) units, at most
// two tiles; the row update: a persistent list of tiles).  Warp 0 issues TMA loads
// (A digit tiles 128 x 64 per plane, X digit tiles of all S planes stacked:
// 32 S rows x 64), warp 1 issues tcgen05.mma (M = 128, N = 32 (S - s) for A
// plane s: one instruction covers every X plane that pairs with it, writing
// the accumulators of weights s..S-1, which sit side by side in TMEM),
// warps 2-9 drain TMEM (two per lane group, 16 columns each).  The
// accumulators are double-buffered (2 x S x 32 FP32 columns <= 512) so
// draining overlaps the next chunk.  All waits are bounded (globaltimer); on
// expiry the CTA records a timeout, drains what it started and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sliced.cuh"

namespace eigref {

namespace sl {

constexpr int kBits = 8;           // bits per digit plane (a digit has at most 8 significant bits)
constexpr int kMaxS = 8;           // digit planes per operand (at most)
constexpr int kDefaultS = 8;       // default digit planes (63 bits: FP64-level accuracy at n = 16384)
constexpr int kBM = 128;           // rows of W per CTA
constexpr int kBN = 32;            // columns of W per CTA
constexpr int kBK = 64;            // K per pipeline stage (128 bytes of F16)
constexpr int kChunkBlocks = 2;    // K blocks per exact accumulation chunk (128: 8 pairs x 2^14 x 128 <= 2^24)
constexpr int kRA = 9;             // A ring stages (a K block of planes and one more)
constexpr int kRAProduct = 10;     // the product's ring: one stage deeper (its epilogue keeps no sums in shared memory)
constexpr int kRAUpdate = 7;       // the update's ring: two stages give way to the epilogue's transpose blocks
// Digit weights: a = 2^e sum_s d_s 2^-(kBits s + 7), so the pairs of weight
// group w = s + t carry 2^-(kBits w + 14); the epilogue keeps
// hi = sum_(w<4) C_w 2^(kBits (3 - w)) and lo = sum_(w>=4) C_w 2^(kBits (S-1-w)).
constexpr int kHiExp = 3 * kBits + 14;                  // hi carries 2^-kHiExp
template <int S>
struct LoExp {
  static constexpr int value = kBits * (S - 1) + 14;    // lo carries 2^-value
};
constexpr int kRX = 2;             // X ring stages (Gram products, update)
constexpr int kRXProduct = 2;      // the product's X ring (a third stage in place of two A stages measured the same)
constexpr int kRXMax = 2;
constexpr int kATile = kBM * kBK * 2;                // 16 KiB
constexpr int kXTile = kMaxS * kBN * kBK * 2;        // 32 KiB (all planes of a K block)
constexpr int kEpiWarps = 8;       // two warps per TMEM lane group, 16 columns each
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kNonFinite = -100000;  // exponent marking a row / column holding Inf or NaN
constexpr uint64_t kTimeoutNs = 2000000000ull;       // 2 s: no legitimate wait comes close
constexpr int kSmemBytes = kRA * kATile + kRX * kXTile + 1024 /*barriers*/ + 1024 /*alignment*/;
constexpr int kSmemBytesProduct = kRAProduct * kATile + kRXProduct * kXTile + 1024 + 1024;
// The row update's epilogue: 16 warps, four a TMEM lane group, 8 of the 32
// tile columns each (the other modes keep 8 warps of 16 columns)
constexpr int kEpiWarpsU = 16;
constexpr int kThreadsU = 64 + 32 * kEpiWarpsU;
constexpr int kTrStride = kBN * 4 / kEpiWarpsU + 1;   // doubles a row of a warp's 32 x 8 transpose block (no bank conflicts)
constexpr int kTrBytes = kEpiWarpsU * 32 * kTrStride * 8;   // 36 KiB
constexpr int kSmemBytesUpdate = kRAUpdate * kATile + kRX * kXTile + 1024 + kTrBytes + 1024;
__host__ __device__ constexpr int ring_a(int mode) { return mode == 0 ? kRAProduct : (mode == 2 ? kRAUpdate : kRA); }
__host__ __device__ constexpr int ring_x(int mode) { return mode == 0 ? kRXProduct : kRX; }
__host__ __device__ constexpr int threads_of(int mode) { return mode == 2 ? kThreadsU : kThreads; }
__host__ __device__ constexpr int smem_bytes(int mode) {
  return mode == 0 ? kSmemBytesProduct : (mode == 2 ? kSmemBytesUpdate : kSmemBytes);
}

// A CTA's abort flag (shared memory).  Every bounded wait takes its limit in
// a register (the launch's wait_ns, 0: kTimeoutNs) and reads the clock every
// 64 polls (16 for the sleeping form); a limit under kShortWaitNs is checked
// at every poll instead, so that a tiny one gives up at the first wait that
// is not already complete.
struct WaitState {
  volatile int abort;
};
constexpr unsigned long long kShortWaitNs = 100000ull;

struct __align__(8) Bars {
  uint64_t a_full[kRAProduct], a_empty[kRAProduct], x_full[kRXMax], x_empty[kRXMax], acc_full[2], acc_empty[2], drain;
  uint32_t tmem_base;
  WaitState wait;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long wait_limit(unsigned long long wait_ns) {
  return wait_ns ? wait_ns : kTimeoutNs;
}
// Bounded wait: false when the CTA is aborting or the wait ran past the limit.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, WaitState* w, unsigned long long lim) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  const bool every = lim < kShortWaitNs;
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 0 || every) {
      if (w->abort) return false;
      if (globaltimer() - t0 > lim) {
        w->abort = 1;
        return false;
      }
    }
  }
}
// The same with a short sleep between polls after the first few: for waits
// that are long against the work of the other warps on the SM (the spinning
// lanes would take their issue slots).
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t bar, uint32_t parity, WaitState* w, unsigned long long lim) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  const bool every = lim < kShortWaitNs;
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 8) __nanosleep(128);
    if ((it & 15) == 0 || every) {
      if (w->abort) return false;
      if (globaltimer() - t0 > lim) {
        w->abort = 1;
        return false;
      }
    }
  }
}
// Bounded wait used while leaving after an abort: lets work already issued
// complete, gives up after 100 ms.
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > 100000000ull) return;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
// K-major operand in the 128-byte swizzled layout TMA writes: rows of 128 B,
// 8-row groups 1024 B apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// kind::f16 instruction descriptor: D = F32, A = B = F16, both K-major.
// (Every digit is an integer of at most 8 significant bits, exact in F16.)
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

#define TC_LD8(taddr, r)                                                                             \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"               \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), \
                 "=r"(r[7])                                                                          \
               : "r"(taddr))

#define TC_LD16(taddr, r)                                                                                   \
  asm volatile(                                                                                             \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),     \
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),          \
        "=r"(r[15])                                                                                         \
      : "r"(taddr))

#define TC_LD32(taddr, r)                                                                                     \
  asm volatile(                                                                                               \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17," \
      "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                      \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),       \
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), \
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),           \
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),           \
        "=r"(r[30]), "=r"(r[31])                                                                             \
      : "r"(taddr))

// ---------------------------------------------------------------------------
// The tensor-core kernel, for three products that share its structure:
//   PRODUCT  W = (A - shift I) X       A-planes (rows of A)   x  column planes of X
//   GRAM     G = X^T X, S = X^T W      column planes of X     x  column planes of X / W
//   UPDATE   X' = X + (W - X D) D^-1 - X F  (rows >= k)       row planes of X  x  column planes of F
// An A-side plane s holds 128 rows of a "row-scaled" operand (one exponent per
// row), a B-side plane t 32 rows of a "column-scaled" operand; both are K-major
// (the contraction index runs along the 128-byte rows TMA writes).
// ---------------------------------------------------------------------------


// The value of one output from its two exact int64 sums (digit-pair groups
// w < 4 and w >= 4, see the epilogue) and the row / column exponents:
// 2^(er + fc) (hi 2^-kHiExp + lo 2^-LoExp), rounded once to nearest-even.  The
// exact sum V = hi 2^(m-kHiExp) + lo (value V 2^-m) is formed as a 128-bit
// integer and rounded to 53 bits with integer arithmetic up to the bit
// pattern: no FP64 instruction (FP64 runs at a small fraction of the integer
// rate on this part), and the same value as rounding the exact sum once.
template <int S>
__device__ __forceinline__ double recombine128(long long hi, long long lo, int er, int fc) {
  if (er == kNonFinite || fc == kNonFinite) return __longlong_as_double(0x7FF8000000000000ll);  // Inf / NaN operand
  constexpr int m = LoExp<S>::value > kHiExp ? LoExp<S>::value : kHiExp;
  constexpr int K = m - kHiExp;                 // lo = 0 when S < 4 (no weight group >= 4)
  // V as a 128-bit two's complement (vh, vl); |V| < 2^98
  const unsigned long long a = K ? ((unsigned long long)hi << K) : (unsigned long long)hi;
  const long long ah = K ? (hi >> (64 - K)) : (hi >> 63);
  const unsigned long long vl0 = a + (unsigned long long)lo;
  long long vh = ah + (lo >> 63) + (vl0 < a ? 1 : 0);
  unsigned long long vl = vl0;
  const bool neg = vh < 0;
  if (neg) {
    vl = 0ull - vl0;
    vh = ~vh + (vl0 == 0ull ? 1 : 0);
  }
  if ((vh | (long long)vl) == 0) return 0.0;
  const unsigned long long uh = (unsigned long long)vh;
  const int nb = uh ? 128 - __clzll((long long)uh) : 64 - __clzll((long long)vl);   // bit length, <= 98
  unsigned long long mant;
  int e2 = nb - 53;
  if (nb <= 53) {
    mant = vl << (53 - nb);
  } else {
    const int sh = nb - 53;                                 // 1 .. 45
    mant = (vl >> sh) | (uh << (64 - sh));
    const unsigned long long rem = vl & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    mant += (rem > half || (rem == half && (mant & 1ull))) ? 1ull : 0ull;
    if (mant >> 53) {
      mant >>= 1;
      ++e2;
    }
  }
  const int ex = e2 - m + er + fc;
  const int be = ex + 52 + 1023;
  if (be >= 1 && be <= 2046)
    return __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)be << 52) |
                                            (mant & 0xFFFFFFFFFFFFFull)));
  const double v = ldexp((double)mant, ex);   // outside the normal range (not met in practice)
  return neg ? -v : v;
}

// The same, out of line: the rare case of the two-word route below, kept out
// of its callers' instruction stream.
template <int S>
__device__ __noinline__ double recombine_wide(long long hi, long long lo, int er, int fc) {
  return recombine128<S>(hi, lo, er, fc);
}

// The same value by a shorter route where |hi|, |lo| < 2^61 and the exact sum
// has at most 52 + K bits above the 2^K boundary (the case met in practice):
// with t = hi + floor(lo / 2^K) and low = lo mod 2^K, V = t 2^K + low and
// 0 <= low < 2^K, so the sign of V is the sign of t, and |V| = T 2^K + low'
// with T = |t| (less one, and low' = 2^K - low, when t < 0 and low != 0).
// The 53 bits kept are then T shifted left and the top of low', the bits
// rounded off all lie in low' (K <= 32: 32-bit arithmetic), and the rounding
// is to nearest, ties to even, as above.  Anything else takes the 128-bit route.
template <int S>
__device__ __forceinline__ double recombine(long long hi, long long lo, int er, int fc) {
  if (er == kNonFinite || fc == kNonFinite) return __longlong_as_double(0x7FF8000000000000ll);  // Inf / NaN operand
  constexpr int m = LoExp<S>::value > kHiExp ? LoExp<S>::value : kHiExp;
  constexpr int K = m - kHiExp;                 // 0, 8, 16, 24 or 32
  static_assert(K >= 0 && K <= 32, "two-word recombination needs K <= 32");
  constexpr long long kLim = 1ll << 61;
  if (hi > -kLim && hi < kLim && lo > -kLim && lo < kLim) {
    const long long t = hi + (lo >> K);
    constexpr uint32_t lowm = (uint32_t)((1ull << K) - 1ull);
    uint32_t low = (uint32_t)lo & lowm;
    const bool neg = t < 0;
    const unsigned long long T = neg ? (unsigned long long)(-t) - (low != 0u ? 1ull : 0ull) : (unsigned long long)t;
    low = neg ? ((0u - low) & lowm) : low;
    if (T < (1ull << 52)) {
      if (T == 0ull && low == 0u) return 0.0;
      const int nb = T ? 64 - __clzll((long long)T) + K : 32 - __clz((int)low);   // bits of |V|
      int sh = nb - 53;
      unsigned long long mant;
      if (sh <= 0) {
        mant = ((T << K) | (unsigned long long)low) << (-sh);
      } else {                                   // 1 <= sh <= K - 1
        mant = (T << (K - sh)) | (unsigned long long)(low >> sh);
        const uint32_t rem = low & ((1u << sh) - 1u), half = 1u << (sh - 1);
        mant += (rem > half || (rem == half && (mant & 1ull))) ? 1ull : 0ull;
        if (mant >> 53) {
          mant >>= 1;
          ++sh;
        }
      }
      const int be = sh - m + er + fc + 52 + 1023;
      if (be >= 1 && be <= 2046)
        return __longlong_as_double(
            (long long)(((unsigned long long)neg << 63) | (((unsigned long long)(be - 1) << 52) + mant)));
    }
  }
  return recombine_wide<S>(hi, lo, er, fc);
}

// One CTA's tile: output column block nb, row tile mb, K split / job zb.
// tiles > 0 (UPDATE only): persistent, the CTA takes tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... of tiles (column block fastest, tgx of them;
// nb and mb unused).  Ring, stage and accumulator counters run on across
// the CTA's tiles, so the MMAs of one tile fill the second accumulator set
// while the epilogue warps finish the previous one.
// ITEMS false (the grouped kernels): one tile a CTA only, the code for the
// persistent and equal-work item lists left out (it costs registers).
template <int S, int MODE, bool ITEMS = true>
__device__ __forceinline__ void sliced_mma_body(const CUtensorMap* tmA, const CUtensorMap* tmB,
                                                const CUtensorMap* tmB2, const MmaArgs& g, int nb, int mb, int zb,
                                                int tgx = 0, int tiles = 0) {
  // one read of the stop flag per CTA: an aborting CTA of this grid may set it
  __shared__ int s_skip;
  __shared__ double s_colsum[2][3][4][kBN / 2];     // UPDATE: per lane-group column sums, by tile parity
  if (threadIdx.x == 0) s_skip = (g.ctl && g.ctl->done) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int RA = ring_a(MODE);                   // A ring stages
  unsigned char* sa = smem;                          // RA x 16 KiB
  constexpr int RX = ring_x(MODE);                   // X ring stages
  unsigned char* sx = smem + RA * kATile;            // RX x 32 KiB
  Bars* bars = reinterpret_cast<Bars*>(sx + RX * kXTile);
  static_assert(sizeof(Bars) <= 1024, "barrier block");
  double* s_tr = reinterpret_cast<double*>(sx + RX * kXTile + 1024);    // UPDATE: 16 warps x 32 x kTrStride
  constexpr int EW = MODE == MODE_UPDATE ? kEpiWarpsU : kEpiWarps;       // epilogue warps
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // column blocks vary fastest, so the CTAs sharing A-side rows run together
  const int job = MODE == MODE_GRAM ? (zb & 1) : 0;
  const int split = MODE == MODE_GRAM ? (zb >> 1) : (MODE == MODE_PRODUCT ? zb : 0);
  const int nsplit = MODE == MODE_UPDATE ? 1 : g.ksplit;
  const bool persist = ITEMS && MODE == MODE_UPDATE && tiles > 0;
  const bool ranged = ITEMS && MODE == MODE_PRODUCT && g.sk_ranges > 0;
  // Work items of this CTA in order: column block, row tile, first K block,
  // K blocks and the slot of its exact partial.  By default one item: the
  // CTA's tile, K split `split` of nsplit.  Persistent update: tiles
  // blockIdx.x, blockIdx.x + gridDim.x, ...  Equal-work product: range mb
  // (of sk_ranges equal ranges) of the (row tile, K block) units of column
  // block nb, cut at row-tile boundaries (at most two items); an item's slot
  // is mb less the range holding its tile's first unit.
  struct Item {
    int nb, mb, kb_lo, kb, slot;
  };
  auto item = [&](int w, Item& it) -> bool {
    if (persist) {
      const int t = (int)blockIdx.x + w * (int)gridDim.x;
      if (t >= tiles) return false;
      it = Item{t % tgx, t / tgx, 0, g.kb_total, 0};
      return true;
    }
    if (ranged) {
      const int64_t U = g.sk_units, R = g.sk_ranges, KBt = g.kb_total;
      const int64_t u0 = (int64_t)mb * U / R, u1 = ((int64_t)mb + 1) * U / R;
      const int64_t s0 = w == 0 ? u0 : (u0 / KBt + w) * KBt;
      if (s0 >= u1) return false;
      const int64_t e0 = min((s0 / KBt + 1) * KBt, u1);
      const int64_t first = (((s0 / KBt) * KBt + 1) * R - 1) / U;
      it = Item{nb, (int)(s0 / KBt), (int)(s0 % KBt), (int)(e0 - s0), (int)(mb - first)};
      return true;
    }
    if (w > 0) return false;
    const int lo = (int)((int64_t)g.kb_total * split / nsplit);
    it = Item{nb, mb, lo, (int)((int64_t)g.kb_total * (split + 1) / nsplit) - lo, split};
    return true;
  };
  constexpr int NBUF = 2;                            // TMEM accumulator sets: 2 x S x 32 <= 512 columns
  static_assert(2 * kMaxS * kBN <= 512, "two accumulator sets must fit in TMEM");
  const CUtensorMap* tB = job ? tmB2 : tmB;
  WaitState* wst = &bars->wait;
  const unsigned long long wlim = wait_limit(g.wait_ns);

  if (threadIdx.x == 0) {
    for (int i = 0; i < RA; ++i) {
      mbar_init(smem_u32(&bars->a_full[i]), 1);
      mbar_init(smem_u32(&bars->a_empty[i]), 1);
    }
    for (int i = 0; i < RX; ++i) {
      mbar_init(smem_u32(&bars->x_full[i]), 1);
      mbar_init(smem_u32(&bars->x_empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&bars->acc_full[i]), 1);
      mbar_init(smem_u32(&bars->acc_empty[i]), EW);  // one arrival per epilogue warp
    }
    mbar_init(smem_u32(&bars->drain), 1);
    bars->wait.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&bars->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = bars->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(tB) : "memory");
      int issued_a = 0, issued_x = 0;
      bool ok = true;
      int as = 0;
      uint32_t aph = 0;                              // lap parity of the A ring
      int gkb = 0;                                   // K blocks over the CTA's tiles (X stage and parity)
      Item it;
      for (int w = 0; ok && item(w, it); ++w) {
        const int nbt = it.nb;
        const int m0 = it.mb * kBM;
        for (int kb = 0; kb < it.kb && ok; ++kb, ++gkb) {
          const int kx = (it.kb_lo + kb) * kBK;      // K coordinate (elements)
          const int xs = gkb % RX;
          ok = mbar_wait(smem_u32(&bars->x_empty[xs]), ((gkb / RX) & 1) ^ 1, wst, wlim);
          if (!ok) break;
          mbar_expect_tx(smem_u32(&bars->x_full[xs]), (uint32_t)(S * kBN * kBK * 2));
#pragma unroll
          for (int t = 0; t < S; ++t)
            tma_load_2d(smem_u32(sx + xs * kXTile + t * kBN * kBK * 2), tB, smem_u32(&bars->x_full[xs]), kx,
                        t * g.b_plane_rows + nbt * kBN);
          ++issued_x;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            ok = mbar_wait(smem_u32(&bars->a_empty[as]), aph ^ 1, wst, wlim);
            if (!ok) break;
            mbar_expect_tx(smem_u32(&bars->a_full[as]), (uint32_t)kATile);
            tma_load_2d(smem_u32(sa + as * kATile), tmA, smem_u32(&bars->a_full[as]), kx, s * g.a_plane_rows + m0);
            ++issued_a;
            if (++as == RA) {
              as = 0;
              aph ^= 1;
            }
          }
        }
      }
      if (!ok) {
        // let the copies this thread started land before the CTA leaves
        for (int i = (issued_a > RA ? issued_a - RA : 0); i < issued_a; ++i)
          mbar_drain(smem_u32(&bars->a_full[i % RA]), (i / RA) & 1);
        for (int i = (issued_x > RX ? issued_x - RX : 0); i < issued_x; ++i)
          mbar_drain(smem_u32(&bars->x_full[i % RX]), (i / RX) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint64_t a_desc0 = smem_desc(smem_u32(sa));
      const uint64_t x_desc0 = smem_desc(smem_u32(sx));
      bool ok = true;
      int as = 0;
      uint32_t aph = 0;
      int gkb = 0, gc = 0;                           // K blocks and chunks over the CTA's tiles
      Item it;
      for (int w = 0; ok && item(w, it); ++w) {
        const int KB = it.kb;
        const int NC = (KB + kChunkBlocks - 1) / kChunkBlocks;
        for (int kb = 0; kb < KB && ok; ++kb, ++gkb) {
          const int c = gc + kb / kChunkBlocks;
          const int buf = NBUF == 2 ? (c & 1) : 0;
          const bool first = (kb % kChunkBlocks) == 0;
          const bool last = (kb % kChunkBlocks) == kChunkBlocks - 1 || kb == KB - 1;
          if (first) {
            ok = mbar_wait(smem_u32(&bars->acc_empty[buf]), ((c / NBUF) & 1) ^ 1, wst, wlim);
            if (!ok) break;
            tc_fence_after();
          }
          const int xs = gkb % RX;
          ok = mbar_wait(smem_u32(&bars->x_full[xs]), (gkb / RX) & 1, wst, wlim);
          if (!ok) break;
          tc_fence_after();
          const uint64_t xd = x_desc0 + (uint64_t)(xs * (kXTile >> 4));
          const uint32_t cbase = (uint32_t)(buf * S * kBN);
          const uint32_t acc0 = first ? 0u : 1u;       // the chunk's first MMA overwrites every accumulator
#pragma unroll
          for (int s = 0; s < S; ++s) {
            ok = mbar_wait(smem_u32(&bars->a_full[as]), aph, wst, wlim);
            if (!ok) break;
            tc_fence_after();
            const uint64_t ad = a_desc0 + (uint64_t)(as * (kATile >> 4));
            // B = B-side planes 0 .. S-1-s stacked: N = 32 (S - s) rows (weight
            // groups w = s .. S-1 at columns cbase + 32 w), issued as pieces of
            // at most 256 (the M = 128 limit); +2 in the address field steps 32
            // bytes (16 K) inside the 128-byte swizzle row
            const int N = kBN * (S - s);
            const int N1 = N < 256 ? N : 256;
            const uint32_t dt = tbase + cbase + (uint32_t)(s * kBN);
            tc_mma(dt, ad, xd, idesc_f16(kBM, N1), s == 0 ? acc0 : 1u);
            tc_mma(dt, ad + 2, xd + 2, idesc_f16(kBM, N1), 1u);
            tc_mma(dt, ad + 4, xd + 4, idesc_f16(kBM, N1), 1u);
            tc_mma(dt, ad + 6, xd + 6, idesc_f16(kBM, N1), 1u);
            if (N > 256) {
              const uint64_t xd2 = xd + (uint64_t)((256 * kBK * 2) >> 4);
              const uint32_t id2 = idesc_f16(kBM, N - 256);
              tc_mma(dt + 256u, ad, xd2, id2, s == 0 ? acc0 : 1u);
              tc_mma(dt + 256u, ad + 2, xd2 + 2, id2, 1u);
              tc_mma(dt + 256u, ad + 4, xd2 + 4, id2, 1u);
              tc_mma(dt + 256u, ad + 6, xd2 + 6, id2, 1u);
            }
            tc_commit(smem_u32(&bars->a_empty[as]));
            if (++as == RA) {
              as = 0;
              aph ^= 1;
            }
          }
          if (!ok) break;
          tc_commit(smem_u32(&bars->x_empty[xs]));
          if (last) tc_commit(smem_u32(&bars->acc_full[buf]));
        }
        gc += NC;
      }
      if (!ok) {
        // wait for the MMAs already issued before the CTA releases TMEM
        tc_commit(smem_u32(&bars->drain));
        mbar_drain(smem_u32(&bars->drain), 0);
      }
    }
  } else {
    // ---------------- epilogue: drain chunks into exact int64 sums ----------------
    const int lg = warp & 3;                           // TMEM lane group of this warp
    constexpr int kC = kBN * 4 / EW;                   // columns of a warp: 16 (8 warps) or 8 (16 warps)
    const int half = (warp - 2) >> 2;                  // which kC of the 32 columns
    bool ok = true;
    int gc = 0;                                        // chunks over the CTA's tiles
    Item it;
    for (int w = 0; item(w, it); ++w) {
      const int nbt = it.nb;
      const int mbt = it.mb;
      const int NC = (it.kb + kChunkBlocks - 1) / kChunkBlocks;
      const int64_t row = (int64_t)mbt * kBM + lg * 32 + lane;
      long long hi[kC], lo[kC];
#pragma unroll
      for (int j = 0; j < kC; ++j) hi[j] = lo[j] = 0;
      if (MODE == MODE_UPDATE && row < g.m_valid && row >= g.row_begin) {
        // the row's X and W values the update reads after the drain: into L1
        // while the MMAs run (128 contiguous bytes each)
        const int64_t e0 = row * g.k + nbt * (kBN / 2);
        asm volatile("prefetch.global.L1 [%0];" ::"l"(g.X + e0));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(g.W + e0));
      }
      for (int cl = 0; cl < NC && ok; ++cl) {
        const int c = gc + cl;
        const int buf = NBUF == 2 ? (c & 1) : 0;
        // one lane waits, the warp follows (the TMEM loads below are warp-collective);
        // it sleeps between polls, leaving issue slots to the MMA warp
        int w_ok = 0;
        if (lane == 0) w_ok = mbar_wait_sleep(smem_u32(&bars->acc_full[buf]), (c / NBUF) & 1, wst, wlim);
        ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
        __syncwarp();
        if (!ok) break;
        tc_fence_after();
        const uint32_t cbase = (uint32_t)(buf * S * kBN);
        const uint32_t tw = tbase + ((uint32_t)(lg * 32) << 16) + cbase + (uint32_t)(half * kC);
        // several weights per round trip to TMEM (two at S >= 8, within the register budget)
        constexpr int GW = S >= 8 ? 2 : 3;
#pragma unroll
        for (int w0 = 0; w0 < S; w0 += GW) {
          uint32_t r[GW][kC];
#pragma unroll
          for (int q = 0; q < GW; ++q)
            if (w0 + q < S) {
              if constexpr (kC == 16)
                TC_LD16(tw + (uint32_t)((w0 + q) * kBN), r[q]);
              else
                TC_LD8(tw + (uint32_t)((w0 + q) * kBN), r[q]);
            }
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < GW; ++q) {
            if (w0 + q >= S) continue;
            const int w = w0 + q;
            if (w < 4) {
              const int sh = kBits * (3 - w);
#pragma unroll
              for (int j = 0; j < kC; ++j) hi[j] += (long long)__float2int_rn(__uint_as_float(r[q][j])) << sh;
            } else {
              const int sh = kBits * (S - 1 - w);
#pragma unroll
              for (int j = 0; j < kC; ++j) lo[j] += (long long)__float2int_rn(__uint_as_float(r[q][j])) << sh;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->acc_empty[buf]));
      }
      gc += NC;
      const int er = (ok && row < g.m_valid) ? g.rowexp[row] : 0;
      const int* cexp = job ? g.colexp2 : g.colexp;
      if constexpr (MODE == MODE_UPDATE) {
        // The B operand interleaves F and M by 16 columns, so column block nbt
        // covers the real columns c0 .. c0 + 15 with X F in the first half of
        // the tile and X M in the second; four warps share each lane group's
        // 32 rows, 8 columns each (part = half: 0, 1 X F, 2, 3 X M):
        //   X F:  X' = X + (W - X D) D^-1 - X F   (written), sums of X'^2 and R^2
        //   X M:  V2 = R2 - X2 M                  (the rows of E21 D), sums of V2^2
        // Each lane recombines its row of 8 columns; the warp's 32 x 8 block
        // then turns through shared memory, so that 8 lanes hold 8 consecutive
        // columns of one row and every global load and store of X, W and X'
        // moves 64-byte row segments.  X, W, d and 1/d are read-only in this
        // launch (X' is another buffer).
        constexpr int kR = kBN / 2;                      // real columns of a tile
        constexpr int kL = 32 / kC;                      // rows a step after the turn
        const bool isF = half < 2;
        const int c0 = nbt * kR;
        const int cf = c0 + (half & 1) * kC;             // this warp's first real column
        const int cl = cf + (lane & (kC - 1));           // this lane's column after the turn
        const bool cok = cl < g.k;
        const int e_l = cok ? __ldg(cexp + nbt * kBN + half * kC + (lane & (kC - 1))) : 0;
        double* tr = s_tr + (warp - 2) * 32 * kTrStride;
        __syncwarp();                                    // the last tile's reads of tr are done
#pragma unroll
        for (int j = 0; j < kC; ++j) {
          const int ej = __shfl_sync(0xffffffffu, e_l, j);
          const bool lv = ok && row < g.m_valid && row >= g.row_begin && cf + j < g.k;
          tr[lane * kTrStride + j] = lv ? recombine<S>(hi[j], lo[j], er, ej) : 0.0;
        }
        __syncwarp();
        // lane L: column cl of rows r0 + kL i, i = 0 .. kC - 1
        const int64_t r0 = (int64_t)mbt * kBM + lg * 32 + (lane / kC);
        const double dj = cok ? __ldg(g.d + cl) : 0.0, dij = cok ? __ldg(g.dinv + cl) : 0.0;
        double xv[kC], wv[kC];
#pragma unroll
        for (int i = 0; i < kC; ++i) {
          const int64_t r = r0 + kL * i;
          const bool lv = ok && cok && r < g.m_valid && r >= g.row_begin;
          xv[i] = lv ? __ldg(g.X + r * g.k + cl) : 0.0;
          wv[i] = lv ? __ldg(g.W + r * g.k + cl) : 0.0;
        }
        // column sums, rows in order: X F warps of X'^2 and (W - X D)^2, X M warps of V2^2
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int i = 0; i < kC; ++i) {
          const int64_t r = r0 + kL * i;
          if (ok && cok && r < g.m_valid && r >= g.row_begin) {
            const double rr = wv[i] - xv[i] * dj;
            const double t = tr[(kL * i + lane / kC) * kTrStride + (lane & (kC - 1))];
            if (isF) {
              const double xn = xv[i] + rr * dij - t;
              g.Xn[r * g.k + cl] = xn;
              s0 = fma(xn, xn, s0);
              s1 = fma(rr, rr, s1);
            } else {
              const double v = rr - t;
              s0 = fma(v, v, s0);
            }
          }
        }
        // the lanes that share a column (lane % kC), in a fixed order
#pragma unroll
        for (int o = kC; o < 32; o <<= 1) {
          s0 += __shfl_xor_sync(0xffffffffu, s0, o);
          s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        const int tp = w & 1;                            // tile parity: the buffer of this tile's sums
        if (lane < kC) {
          const int cc = (half & 1) * kC + lane;        // real column within the tile
          if (isF) {
            s_colsum[tp][0][lg][cc] = s0;
            s_colsum[tp][1][lg][cc] = s1;
          } else {
            s_colsum[tp][2][lg][cc] = s0;
          }
        }
        // the epilogue warps meet; the first two add the four lane groups'
        // sums of the tile.  A warp writes buffer tp again two tiles later,
        // after the next meeting, which every reader of this one has passed.
        asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
        const int et = (int)threadIdx.x - 64;
        if (et < 3 * kR) {
          const int which = et / kR, cc = et % kR;
          const int col = c0 + cc;
          if (col < g.k) {
            const double v = s_colsum[tp][which][0][cc] + s_colsum[tp][which][1][cc] + s_colsum[tp][which][2][cc] +
                             s_colsum[tp][which][3][cc];
            g.upart[(int64_t)mbt * 3 * g.k + which * g.k + col] = v;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < kC; ++j) {
          const int col = nbt * kBN + half * kC + j;
          const bool live = ok && row < g.m_valid && col < g.k;
          // split-K partials stay exact int64 pairs: the sum over splits is exact,
          // so the result does not depend on how K was split
          const bool raw = (MODE == MODE_GRAM) || (MODE == MODE_PRODUCT && (nsplit > 1 || ranged));
          const double w = (live && !raw) ? recombine<S>(hi[j], lo[j], er, cexp[col]) : 0.0;
          if (MODE == MODE_PRODUCT) {
            if (live) {
              if (nsplit == 1 && !ranged)
                g.P[row * g.k + col] = w - g.shift * g.Xs[row * g.k + col];
              else
                g.ppart[(int64_t)it.slot * g.m_valid * g.k + row * g.k + col] = make_longlong2(hi[j], lo[j]);
            }
          } else {
            if (live) g.gpart[((int64_t)(job * nsplit + split) * g.k + col) * g.k + row] = make_longlong2(hi[j], lo[j]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (bars->wait.abort && threadIdx.x == 0) {
    atomicExch(g.err, 1);
    if (g.ctl) {
      Control* c = const_cast<Control*>(g.ctl);
      c->status = EIGREF_E_TIMEOUT;
      c->done = 1;
    }
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
  }
}

template <int S, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    sliced_mma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ CUtensorMap tmB2, MmaArgs g) {
  sliced_mma_body<S, MODE>(&tmA, &tmB, &tmB2, g, blockIdx.x, blockIdx.y, blockIdx.z);
}

// The row update over a persistent grid (one CTA per SM): tiles = gx column
// blocks x row tiles, column block fastest.  With one tile a CTA, load, MMAs
// and the FP64 epilogue of a CTA run one after another and nothing else
// shares the SM; here the MMAs of a CTA's next tile overlap the epilogue of
// its current one.
template <int S>
__global__ void __launch_bounds__(kThreadsU, 1)
    sliced_update_persistent_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                                    MmaArgs g, int gx, int tiles) {
  sliced_mma_body<S, MODE_UPDATE>(&tmA, &tmB, &tmB, g, 0, 0, 0, gx, tiles);
}

// ---------------------------------------------------------------------------
// The product W = (A - shift I) X on 128 x 64 tiles (column blocks of 64 when
// k is a multiple of 64).  A 64-deep K block of a tile moves the same 128 KiB
// of A planes as a 128 x 32 tile but does twice the MMA work, so the bytes a
// flop that TMA brings into one SM's shared memory drop by 40 % and the
// tensor pipe, not the TMA feed, sets the pace.  The 8 weight groups of a
// 128 x 64 tile take all 512 TMEM columns (group w at columns 64 w), so
// there is one accumulator set, drained group by group:
//   * every MMA accumulates (the epilogue clears a group in TMEM after
//     reading it, and before the first chunk);
//   * the MMA for A plane s (B = X planes 0 .. S-1-s, groups s .. S-1) is
//     issued as pieces p1 = groups s .. s+3 and p2 = groups s+4 .. S-1, in
//     the order s0p1, s1p1, s0p2, s1p2, s2p1, s2p2, s3p1, ... so that group
//     w takes its last contribution of a chunk from piece "w p1" and groups
//     finish in the order 0, 1, .., S-1;
//   * in a chunk's last K block the MMA warp commits group w's barrier
//     after piece "w p1"; the epilogue drains (and clears) groups in that
//     order while the rest of the block runs;
//   * in a chunk's first K block the MMA warp waits for a group to be
//     drained only before the first piece that touches it: the two pieces
//     that open a block touch groups 0 .. 4 only, and the last groups to be
//     drained (S-3 .. S-1) are first needed about 1200 clocks of tensor work
//     later.
// One thread issues every MMA, and each barrier operation costs it tens of
// clocks of latency, so the pipeline is cut to keep those few: A stages of
// two planes (one wait and one release per two planes), drain barriers per
// pair of weight groups, and the barrier of the next A stage (and of the
// next K block's X stage and first A stage) tested without blocking before
// the current piece's MMAs are issued, so that its latency overlaps them.
// Same exactness as the 128 x 32 kernel (a group of a 128-deep chunk stays
// below 2^24), same items (fixed K splits or equal-work ranges) and partials.
// ---------------------------------------------------------------------------
constexpr int kWBN = 64;                                  // columns of W per CTA
constexpr int kWPS = 2;                                   // A planes a stage
constexpr int kWAStage = kWPS * kATile;                   // 32 KiB
constexpr int kWRA = 3;                                   // A ring stages
constexpr int kWRX = 2;                                   // X ring (all planes of a K block, 64 KiB)
constexpr int kWXTile = kMaxS * kWBN * kBK * 2;           // 64 KiB
constexpr int kWPairs = (kMaxS + 1) / 2;                  // drain barriers: one per pair of weight groups
constexpr int kSmemBytesWide = kWRA * kWAStage + kWRX * kWXTile + 1024 /*barriers*/ + 1024 /*alignment*/;
static_assert(kSmemBytesWide <= 232448, "shared memory of the wide product");
static_assert(kMaxS * kWBN <= 512, "the weight groups of a 128 x 64 tile must fit in TMEM");

struct __align__(8) WideBars {
  uint64_t a_full[kWRA], a_empty[kWRA], x_full[kWRX], x_empty[kWRX], g_full[kWPairs], g_empty[kWPairs], drain;
  uint32_t tmem_base;
  WaitState wait;
};

// Piece i of a K block for S planes: plane s, first and last weight group.
struct WPiece {
  int s, glo, ghi;
};
template <int S>
__host__ __device__ constexpr WPiece wide_piece(int i) {
  // s0p1, s1p1, s0p2, s1p2, then p1 (and p2) of s = 2 .. S-1
  if (S >= 6 && i < 4) {
    const int s = i & 1;
    return (i < 2) ? WPiece{s, s, s + 3} : WPiece{s, s + 4, S - 1};
  }
  int j = (S >= 6) ? 4 : 0;
  for (int s = (S >= 6) ? 2 : 0; s < S; ++s) {
    const int hi1 = s + 3 < S - 1 ? s + 3 : S - 1;
    if (j == i) return WPiece{s, s, hi1};
    ++j;
    if (s + 4 <= S - 1) {
      if (j == i) return WPiece{s, s + 4, S - 1};
      ++j;
    }
  }
  return WPiece{-1, 0, -1};
}
template <int S>
__host__ __device__ constexpr int wide_pieces() {
  int c = 0;
  for (int s = 0; s < S; ++s) c += (s + 4 <= S - 1) ? 2 : 1;
  return c;
}
template <int S>
__host__ __device__ constexpr int wide_stages() {
  return (S + kWPS - 1) / kWPS;
}
// the last piece of a K block that reads A stage s / 2 (the stage is then released)
template <int S>
__host__ __device__ constexpr bool wide_last_of_stage(int i) {
  const WPiece p = wide_piece<S>(i);
  for (int j = i + 1; j < wide_pieces<S>(); ++j)
    if (wide_piece<S>(j).s / kWPS == p.s / kWPS) return false;
  return true;
}
template <int S>
__host__ __device__ constexpr bool wide_first_of_stage(int i) {
  if (i >= wide_pieces<S>()) return false;
  const WPiece p = wide_piece<S>(i);
  for (int j = 0; j < i; ++j)
    if (wide_piece<S>(j).s / kWPS == p.s / kWPS) return false;
  return true;
}
// piece i finishes both groups of pair s / 2 (in a chunk's last block): it is
// "s p1" for the pair's higher group (group S - 1 when the pair has one)
template <int S>
__host__ __device__ constexpr bool wide_ends_pair(int i) {
  const WPiece p = wide_piece<S>(i);
  return p.glo == p.s && (p.s % 2 == 1 || p.s == S - 1);
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// The MMA warp's work for piece I .. of one K block, unrolled at compile
// time so that the piece table costs the issuing thread no instructions.
// pre: the stage of piece I was seen complete by an earlier test.  Every
// test names a phase whose predecessor on that slot this thread has already
// waited for, so a true result can only mean that phase.
struct WideIssue {
  WideBars* bars;
  uint32_t tbase;
  uint64_t a_desc0, xd;
  int gkb, c;
  bool last;
  WaitState* wst;
  unsigned long long wlim;
};
struct WideNext {
  bool a0, x;      // the next K block's first A stage and X stage, seen complete
};
template <int S, int I>
__device__ __forceinline__ bool wide_issue(const WideIssue& q, int& ready, bool pre, WideNext& nx) {
  if constexpr (I < wide_pieces<S>()) {
    constexpr WPiece p = wide_piece<S>(I);
    constexpr int NST = wide_stages<S>();
    const int ia = q.gkb * NST + p.s / kWPS;          // the stage's place in the A ring's sequence
    const int slot = ia % kWRA;
    if constexpr (wide_first_of_stage<S>(I)) {
      if (!pre && !mbar_wait(smem_u32(&q.bars->a_full[slot]), (ia / kWRA) & 1, q.wst, q.wlim)) return false;
      tc_fence_after();
    }
    while (ready < p.ghi / 2) {
      ++ready;
      if (!mbar_wait(smem_u32(&q.bars->g_empty[ready]), q.c & 1, q.wst, q.wlim)) return false;
      tc_fence_after();
    }
    // look ahead without blocking: the next stage of this block, or after the
    // last piece the next K block's X stage and first A stage
    bool nxt = false;
    if constexpr (wide_first_of_stage<S>(I + 1)) {
      const int ib = q.gkb * NST + wide_piece<S>(I + 1).s / kWPS;
      nxt = mbar_test(smem_u32(&q.bars->a_full[ib % kWRA]), (ib / kWRA) & 1);
    }
    if constexpr (I + 1 == wide_pieces<S>()) {
      const int ib = (q.gkb + 1) * NST, xb = q.gkb + 1;
      nx.a0 = mbar_test(smem_u32(&q.bars->a_full[ib % kWRA]), (ib / kWRA) & 1);
      nx.x = mbar_test(smem_u32(&q.bars->x_full[xb % kWRX]), (xb / kWRX) & 1);
    }
    const uint64_t ad = q.a_desc0 + (uint64_t)((slot * kWAStage + (p.s % kWPS) * kATile) >> 4);
    // B rows: X planes t = glo - s .. ghi - s (64 rows each, 128 B a row);
    // TMEM columns 64 glo ..; +2 in the address field steps 16 K
    const uint64_t bd = q.xd + (uint64_t)(((p.glo - p.s) * kWBN * kBK * 2) >> 4);
    constexpr uint32_t id = idesc_f16(kBM, kWBN * (p.ghi - p.glo + 1));
    const uint32_t dt = q.tbase + (uint32_t)(p.glo * kWBN);
    tc_mma(dt, ad, bd, id, 1u);
    tc_mma(dt, ad + 2, bd + 2, id, 1u);
    tc_mma(dt, ad + 4, bd + 4, id, 1u);
    tc_mma(dt, ad + 6, bd + 6, id, 1u);
    if constexpr (wide_last_of_stage<S>(I)) tc_commit(smem_u32(&q.bars->a_empty[slot]));
    if constexpr (wide_ends_pair<S>(I))
      if (q.last) tc_commit(smem_u32(&q.bars->g_full[p.s / 2]));
    return wide_issue<S, I + 1>(q, ready, nxt, nx);
  } else {
    return true;
  }
}

#define TC_ST32_ZERO(taddr)                                                                                  \
  asm volatile(                                                                                              \
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1," \
      "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),                                                  \
      "r"(0u)                                                                                                \
      : "memory")

template <int S>
__global__ void __launch_bounds__(kThreads, 1)
    sliced_wide_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, MmaArgs g) {
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = (g.ctl && g.ctl->done) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sa = smem;                          // kWRA x 32 KiB
  unsigned char* sx = smem + kWRA * kWAStage;        // kWRX x 64 KiB
  WideBars* bars = reinterpret_cast<WideBars*>(sx + kWRX * kWXTile);
  static_assert(sizeof(WideBars) <= 1024, "barrier block");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nb = blockIdx.x, mb = blockIdx.y, split = blockIdx.z;
  const int nsplit = g.ksplit;
  const bool ranged = g.sk_ranges > 0;
  // Work items of this CTA, as in the 128 x 32 kernel: one K split of one
  // tile, or the tiles an equal-work range crosses (an item a tile).
  struct Item {
    int nb, mb, kb_lo, kb, slot;
  };
  auto item = [&](int w, Item& it) -> bool {
    if (ranged) {
      const int64_t U = g.sk_units, R = g.sk_ranges, KBt = g.kb_total;
      const int64_t u0 = (int64_t)mb * U / R, u1 = ((int64_t)mb + 1) * U / R;
      const int64_t s0 = w == 0 ? u0 : (u0 / KBt + w) * KBt;
      if (s0 >= u1) return false;
      const int64_t e0 = min((s0 / KBt + 1) * KBt, u1);
      const int64_t first = (((s0 / KBt) * KBt + 1) * R - 1) / U;
      it = Item{nb, (int)(s0 / KBt), (int)(s0 % KBt), (int)(e0 - s0), (int)(mb - first)};
      return true;
    }
    if (w > 0) return false;
    const int lo = (int)((int64_t)g.kb_total * split / nsplit);
    it = Item{nb, mb, lo, (int)((int64_t)g.kb_total * (split + 1) / nsplit) - lo, split};
    return true;
  };
  WaitState* wst = &bars->wait;
  const unsigned long long wlim = wait_limit(g.wait_ns);

  if (threadIdx.x == 0) {
    for (int i = 0; i < kWRA; ++i) {
      mbar_init(smem_u32(&bars->a_full[i]), 1);
      mbar_init(smem_u32(&bars->a_empty[i]), 1);
    }
    for (int i = 0; i < kWRX; ++i) {
      mbar_init(smem_u32(&bars->x_full[i]), 1);
      mbar_init(smem_u32(&bars->x_empty[i]), 1);
    }
    for (int i = 0; i < kWPairs; ++i) {
      mbar_init(smem_u32(&bars->g_full[i]), 1);
      // one arrival per epilogue warp and group of the pair
      mbar_init(smem_u32(&bars->g_empty[i]), kEpiWarps * (2 * i + 1 < S ? 2 : 1));
    }
    mbar_init(smem_u32(&bars->drain), 1);
    bars->wait.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&bars->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = bars->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
      int issued_a = 0, issued_x = 0;
      bool ok = true;
      int as = 0;
      uint32_t aph = 0;
      int gkb = 0;
      Item it;
      for (int w = 0; ok && item(w, it); ++w) {
        const int m0 = it.mb * kBM;
        for (int kb = 0; kb < it.kb && ok; ++kb, ++gkb) {
          const int kx = (it.kb_lo + kb) * kBK;
          const int xs = gkb % kWRX;
          ok = mbar_wait(smem_u32(&bars->x_empty[xs]), ((gkb / kWRX) & 1) ^ 1, wst, wlim);
          if (!ok) break;
          mbar_expect_tx(smem_u32(&bars->x_full[xs]), (uint32_t)(S * kWBN * kBK * 2));
#pragma unroll
          for (int t = 0; t < S; ++t)
            tma_load_2d(smem_u32(sx + xs * kWXTile + t * kWBN * kBK * 2), &tmB, smem_u32(&bars->x_full[xs]), kx,
                        t * g.b_plane_rows + it.nb * kWBN);
          ++issued_x;
#pragma unroll
          for (int j = 0; j < wide_stages<S>(); ++j) {
            constexpr int kLast = S - kWPS * (wide_stages<S>() - 1);   // planes of the last stage
            const int np = j == wide_stages<S>() - 1 ? kLast : kWPS;
            ok = mbar_wait(smem_u32(&bars->a_empty[as]), aph ^ 1, wst, wlim);
            if (!ok) break;
            mbar_expect_tx(smem_u32(&bars->a_full[as]), (uint32_t)(np * kATile));
            for (int h = 0; h < np; ++h)
              tma_load_2d(smem_u32(sa + as * kWAStage + h * kATile), &tmA, smem_u32(&bars->a_full[as]), kx,
                          (kWPS * j + h) * g.a_plane_rows + m0);
            ++issued_a;
            if (++as == kWRA) {
              as = 0;
              aph ^= 1;
            }
          }
        }
      }
      if (!ok) {
        for (int i = (issued_a > kWRA ? issued_a - kWRA : 0); i < issued_a; ++i)
          mbar_drain(smem_u32(&bars->a_full[i % kWRA]), (i / kWRA) & 1);
        for (int i = (issued_x > kWRX ? issued_x - kWRX : 0); i < issued_x; ++i)
          mbar_drain(smem_u32(&bars->x_full[i % kWRX]), (i / kWRX) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint64_t a_desc0 = smem_desc(smem_u32(sa));
      const uint64_t x_desc0 = smem_desc(smem_u32(sx));
      bool ok = true;
      int gkb = 0, gc = 0;
      WideNext nx{false, false};
      Item it;
      for (int w = 0; ok && item(w, it); ++w) {
        const int KB = it.kb;
        const int NC = (KB + kChunkBlocks - 1) / kChunkBlocks;
        for (int kb = 0; kb < KB && ok; ++kb, ++gkb) {
          const int c = gc + kb / kChunkBlocks;
          const bool first = (kb % kChunkBlocks) == 0;
          const bool last = (kb % kChunkBlocks) == kChunkBlocks - 1 || kb == KB - 1;
          const int xs = gkb % kWRX;
          if (!nx.x) {
            ok = mbar_wait(smem_u32(&bars->x_full[xs]), (gkb / kWRX) & 1, wst, wlim);
            if (!ok) break;
          }
          tc_fence_after();
          const uint64_t xd = x_desc0 + (uint64_t)(xs * (kWXTile >> 4));
          int ready = first ? -1 : (S - 1) / 2;          // group pairs known drained for this chunk
          const WideIssue q{bars, tbase, a_desc0, xd, gkb, c, last, wst, wlim};
          const bool pre = nx.a0;
          ok = wide_issue<S, 0>(q, ready, pre, nx);
          if (!ok) break;
          tc_commit(smem_u32(&bars->x_empty[xs]));
        }
        gc += NC;
      }
      if (!ok) {
        tc_commit(smem_u32(&bars->drain));
        mbar_drain(smem_u32(&bars->drain), 0);
      }
    }
  } else {
    // ---------------- epilogue: drain groups into exact int64 sums ----------------
    const int lg = warp & 3;                           // TMEM lane group of this warp
    const int half = (warp - 2) >> 2;                  // which 32 of the 64 columns
    constexpr int kC = kWBN / 2;
    const uint32_t tw = tbase + ((uint32_t)(lg * 32) << 16) + (uint32_t)(half * kC);
    // every group starts cleared
#pragma unroll
    for (int w = 0; w < S; ++w) TC_ST32_ZERO(tw + (uint32_t)(w * kWBN));
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_fence_before();
    __syncwarp();
    if (lane == 0)
      for (int w = 0; w < S; ++w) mbar_arrive(smem_u32(&bars->g_empty[w / 2]));
    bool ok = true;
    int gc = 0;
    Item it;
    for (int wi = 0; item(wi, it); ++wi) {
      const int NC = (it.kb + kChunkBlocks - 1) / kChunkBlocks;
      const int64_t row = (int64_t)it.mb * kBM + lg * 32 + lane;
      long long hi[kC], lo[kC];
#pragma unroll
      for (int j = 0; j < kC; ++j) hi[j] = lo[j] = 0;
      for (int cl = 0; cl < NC && ok; ++cl) {
        const int c = gc + cl;
#pragma unroll
        for (int w = 0; w < S; ++w) {
          // one barrier a pair of groups: wait at the pair's first group; each
          // group, once read and cleared, adds one arrival a warp to the
          // pair's release barrier (which completes with the pair's last)
          if (w % 2 == 0) {
            int w_ok = 0;
            if (lane == 0) w_ok = mbar_wait_sleep(smem_u32(&bars->g_full[w / 2]), c & 1, wst, wlim);
            ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
            __syncwarp();
            if (!ok) break;
            tc_fence_after();
          }
          // two halves of 16 columns (the register budget holds the 64 sums
          // and one half); the group is cleared and released after the second
          // half is in registers
          const int sh = w < 4 ? kBits * (3 - w) : kBits * (S - 1 - w);
          long long* acc = w < 4 ? hi : lo;
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            uint32_t r[kC / 2];
            TC_LD16(tw + (uint32_t)(w * kWBN + hh * (kC / 2)), r);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (hh == 1) {
              TC_ST32_ZERO(tw + (uint32_t)(w * kWBN));
              asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(smem_u32(&bars->g_empty[w / 2]));
            }
#pragma unroll
            for (int j = 0; j < kC / 2; ++j)
              acc[hh * (kC / 2) + j] += (long long)__float2int_rn(__uint_as_float(r[j])) << sh;
          }
        }
      }
      gc += NC;
      const int er = (ok && row < g.m_valid) ? g.rowexp[row] : 0;
      const bool raw = nsplit > 1 || ranged;
#pragma unroll
      for (int j = 0; j < kC; ++j) {
        const int col = it.nb * kWBN + half * kC + j;
        const bool live = ok && row < g.m_valid && col < g.k;
        if (!live) continue;
        if (raw)
          g.ppart[(int64_t)it.slot * g.m_valid * g.k + row * g.k + col] = make_longlong2(hi[j], lo[j]);
        else
          g.P[row * g.k + col] = recombine128<S>(hi[j], lo[j], er, g.colexp[col]) - g.shift * g.Xs[row * g.k + col];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (bars->wait.abort && threadIdx.x == 0) {
    atomicExch(g.err, 1);
    if (g.ctl) {
      Control* c = const_cast<Control*>(g.ctl);
      c->status = EIGREF_E_TIMEOUT;
      c->done = 1;
    }
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
  }
}

// Many problems' tiles in one launch (a batch).  The tensor maps travel in
// the kernel's parameter block, as for the single-problem kernel; CTA c
// takes tile c - cta_begin[t] of task t, ordered column block fastest, then
// row tile, then split.
constexpr int kGroupMax = 40;
struct GroupMma {
  CUtensorMap tmA[kGroupMax];
  CUtensorMap tmB[kGroupMax];
  CUtensorMap tmB2[kGroupMax];
  MmaArgs args[kGroupMax];
  int cta_begin[kGroupMax + 1];
  int gx[kGroupMax], gy[kGroupMax];
  int count;
};

template <int S, int MODE>
__global__ void __launch_bounds__(threads_of(MODE), 1) sliced_mma_grouped_kernel(const __grid_constant__ GroupMma p) {
  const int c = blockIdx.x;
  int t = 0;
  while (t + 1 < p.count && c >= p.cta_begin[t + 1]) ++t;
  const int local = c - p.cta_begin[t];
  const int gx = p.gx[t], gy = p.gy[t];
  sliced_mma_body<S, MODE, false>(&p.tmA[t], &p.tmB[t], &p.tmB2[t], p.args[t], local % gx, (local / gx) % gy,
                                  local / (gx * gy));
}

// ---------------------------------------------------------------------------
// Gram products G = X^T X and S = X^T W for k <= 16 columns over very many
// rows (the sparse workloads).  With 16-row planes, S planes of a K block
// stack into one tile of 16 S rows: the MMA takes A = planes 0..7 of X
// (128 rows) and B = all S planes of Y (N = 16 S), so one instruction forms
// every plane pair (s, t) -- each TMEM element holds exactly one pair, at
// lane 16 s + i, column 16 t + j (S < 8: lanes past the planes read zeros or
// stale rows and are never drained).  One CTA per K split forms both products from
// one load of each tile.  A single pair's sum stays below 2^24 for 960 K
// (960 x 128 x 128 < 2^24), so chunks are 15 K blocks long.  The epilogue
// keeps, per thread, the int64 (hi, lo) sums of its plane row s for 16
// columns j and weights w = s + t <= S - 1; at the end the 16 threads that
// hold a row i add their sums in shared memory, and one exact int64 pair per
// output and split is written.
// ---------------------------------------------------------------------------
constexpr int kG16Stages = 5;
constexpr int kG16Chunk = 15;                       // K blocks per exact chunk (960)
constexpr int kG16Tile = 16 * kMaxS * kBK * 2;      // 16 S rows x 64 K, F16 (S = 8: 16 KiB)
constexpr int kG16Stage = 2 * kG16Tile;             // X tile + Y tile
constexpr int kG16Smem = kG16Stages * kG16Stage + 1024 + 1024;

struct Gram16Args {
  int kb_total;            // K blocks of 64 over all rows
  int ksplit;              // CTAs (K splits)
  int k;                   // columns that exist (<= 16)
  longlong2* part;         // [2][ksplit][k k] exact partials, column-major k x k
  const Control* ctl;
  int* err;
  unsigned long long wait_ns;   // limit of every bounded wait (0: the default)
};

struct __align__(8) Bars16 {
  uint64_t full[kG16Stages], empty[kG16Stages], acc_full, acc_empty, drain;
  uint32_t tmem_base;
  WaitState wait;
};

template <int S>
__global__ void __launch_bounds__(kThreads, 1) sgram16_kernel(const __grid_constant__ CUtensorMap tmX,
                                                             const __grid_constant__ CUtensorMap tmY,
                                                             Gram16Args g) {
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = (g.ctl && g.ctl->done) ? 1 : 0;
  __syncthreads();
  if (s_skip) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Bars16* bars = reinterpret_cast<Bars16*>(smem + kG16Stages * kG16Stage);
  constexpr int kRows = 16 * S;                      // rows of a stacked tile
  constexpr int kTileBytes = kRows * kBK * 2;
  constexpr int kColsJob = kRows;                    // TMEM columns per product
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int split = blockIdx.x;
  const int kb_lo = (int)((int64_t)g.kb_total * split / g.ksplit);
  const int kb_hi = (int)((int64_t)g.kb_total * (split + 1) / g.ksplit);
  const int KB = kb_hi - kb_lo;
  const int NC = (KB + kG16Chunk - 1) / kG16Chunk;
  WaitState* wst = &bars->wait;
  const unsigned long long wlim = wait_limit(g.wait_ns);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kG16Stages; ++i) {
      mbar_init(smem_u32(&bars->full[i]), 1);
      mbar_init(smem_u32(&bars->empty[i]), 1);
    }
    mbar_init(smem_u32(&bars->acc_full), 1);
    mbar_init(smem_u32(&bars->acc_empty), kEpiWarps);
    mbar_init(smem_u32(&bars->drain), 1);
    bars->wait.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&bars->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = bars->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer: the X and Y tiles of each K block ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmX) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmY) : "memory");
      bool ok = true;
      int issued = 0;
      for (int kb = 0; kb < KB && ok; ++kb) {
        const int st = kb % kG16Stages, lap = kb / kG16Stages;
        ok = mbar_wait(smem_u32(&bars->empty[st]), (uint32_t)((lap & 1) ^ 1), wst, wlim);
        if (!ok) break;
        const int kx = (kb_lo + kb) * kBK;
        mbar_expect_tx(smem_u32(&bars->full[st]), (uint32_t)(2 * kTileBytes));
        tma_load_2d(smem_u32(smem + st * kG16Stage), &tmX, smem_u32(&bars->full[st]), kx, 0);
        tma_load_2d(smem_u32(smem + st * kG16Stage + kG16Tile), &tmY, smem_u32(&bars->full[st]), kx, 0);
        ++issued;
      }
      if (!ok)
        for (int i = (issued > kG16Stages ? issued - kG16Stages : 0); i < issued; ++i)
          mbar_drain(smem_u32(&bars->full[i % kG16Stages]), (uint32_t)((i / kG16Stages) & 1));
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      for (int kb = 0; kb < KB && ok; ++kb) {
        const int c = kb / kG16Chunk;
        const bool first = (kb % kG16Chunk) == 0;
        const bool last = (kb % kG16Chunk) == kG16Chunk - 1 || kb == KB - 1;
        if (first && c > 0) {   // one accumulator set: the previous chunk must be drained
          ok = mbar_wait(smem_u32(&bars->acc_empty), (uint32_t)((c - 1) & 1), wst, wlim);
          if (!ok) break;
          tc_fence_after();
        }
        const int st = kb % kG16Stages, lap = kb / kG16Stages;
        ok = mbar_wait(smem_u32(&bars->full[st]), (uint32_t)(lap & 1), wst, wlim);
        if (!ok) break;
        tc_fence_after();
        const uint64_t xd = smem_desc(smem_u32(smem + st * kG16Stage));
        const uint64_t yd = smem_desc(smem_u32(smem + st * kG16Stage + kG16Tile));
        constexpr uint32_t id1 = idesc_f16(kBM, kRows);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t acc = (first && q == 0) ? 0u : 1u;
          const uint64_t o = (uint64_t)(2 * q);    // 16 K per step inside the 128-byte swizzle row
          tc_mma(tbase, xd + o, xd + o, id1, acc);                                 // G: X planes x X planes
          tc_mma(tbase + kColsJob, xd + o, yd + o, id1, acc);                      // S: X planes x Y planes
        }
        tc_commit(smem_u32(&bars->empty[st]));
        if (last) tc_commit(smem_u32(&bars->acc_full));
      }
      if (!ok) {
        tc_commit(smem_u32(&bars->drain));
        mbar_drain(smem_u32(&bars->drain), 0);
      }
    }
  } else {
    // ---------------- epilogue ----------------
    const int lg = warp & 3;                     // TMEM lane group
    const int half = (warp - 2) >> 2;            // which plane columns t of the row
    const int r = lg * 32 + lane;                // TMEM lane = 16 s + i
    const int sp = r >> 4;                       // plane s of X this lane holds
    long long hi[2][16], lo[2][16];
#pragma unroll
    for (int jb = 0; jb < 2; ++jb)
#pragma unroll
      for (int j = 0; j < 16; ++j) hi[jb][j] = lo[jb][j] = 0;
    bool ok = true;
    constexpr int kT0 = (S + 1) / 2;             // half 0 takes planes t < kT0, half 1 the rest
    for (int c = 0; c < NC && ok; ++c) {
      int w_ok = 0;
      if (lane == 0) w_ok = mbar_wait(smem_u32(&bars->acc_full), (uint32_t)(c & 1), wst, wlim);
      ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
      __syncwarp();
      if (!ok) break;
      tc_fence_after();
      const uint32_t tl = tbase + ((uint32_t)(lg * 32) << 16);
#pragma unroll
      for (int jb = 0; jb < 2; ++jb) {
#pragma unroll
        for (int b = 0; b < (S + 2) / 2; ++b) {
          // which 16 columns: plane t of Y (half 0: t < kT0, half 1: t >= kT0)
          const int t = half == 0 ? b : kT0 + b;
          if (half == 0 && t >= kT0) continue;
          if (half == 1 && t > S - 1) continue;
          const uint32_t col = (uint32_t)(jb * kColsJob + 16 * t);
          const int w = sp + t;
          uint32_t v[16];
          TC_LD16(tl + col, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (w <= S - 1) {
            if (w < 4) {
              const int sh = kBits * (3 - w);
#pragma unroll
              for (int j = 0; j < 16; ++j) hi[jb][j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh;
            } else {
              const int sh = kBits * (S - 1 - w);
#pragma unroll
              for (int j = 0; j < 16; ++j) lo[jb][j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->acc_empty));
    }
    // the 16 threads holding row i (4 lane groups x 2 lanes x 2 halves) add their sums
    asm volatile("bar.sync 1, 256;" ::: "memory");   // every epilogue warp is past its last TMEM read
    longlong2* red = reinterpret_cast<longlong2*>(smem);   // [16 contributors][16 i][16 j] (the ring is idle now)
    const int i = r & 15;
    const int qc = lg * 4 + (lane >> 4) * 2 + half;
    const int te = threadIdx.x - 64;             // 0..255 over the epilogue warps
    for (int jb = 0; jb < 2; ++jb) {
#pragma unroll
      for (int j = 0; j < 16; ++j) red[(qc * 16 + i) * 16 + j] = make_longlong2(hi[jb][j], lo[jb][j]);
      asm volatile("bar.sync 1, 256;" ::: "memory");
      {
        const int oi = te & 15, oj = te >> 4;
        long long h = 0, l = 0;
        for (int q = 0; q < 16; ++q) {
          const longlong2 e = red[(q * 16 + oi) * 16 + oj];
          h += e.x;
          l += e.y;
        }
        if (ok && oi < g.k && oj < g.k)
          g.part[((int64_t)(jb * g.ksplit + split) * g.k + oj) * g.k + oi] = make_longlong2(h, l);
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (bars->wait.abort && threadIdx.x == 0) {
    atomicExch(g.err, 1);
    if (g.ctl) {
      Control* c = const_cast<Control*>(g.ctl);
      c->status = EIGREF_E_TIMEOUT;
      c->done = 1;
    }
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
  }
}

// G (job 0), S (job 1) from the split partials of sgram16: the exact sum over
// any number of splits (128-bit), then the one FP64 recombination.
template <int S>
__global__ void sgram16_reduce_kernel(const longlong2* __restrict__ part, int k, int nsplit,
                                      const int* __restrict__ xexp, const int* __restrict__ wexp,
                                      double* __restrict__ out, const Control* ctl) {
  if (ctl && ctl->done) return;
  const int64_t kk = (int64_t)k * k;
  const int lane = threadIdx.x & 31;
  for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < 2 * kk;
       e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int z = (int)(e / kk);
    const int64_t o = e % kk;
    const longlong2* p = part + (int64_t)z * nsplit * kk + o;
    __int128 hi = 0, lo = 0;
    for (int c = lane; c < nsplit; c += 32) {
      const longlong2 v = p[(int64_t)c * kk];
      hi += v.x;
      lo += v.y;
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      const long long hh = (long long)(hi >> 64), hl = (long long)(unsigned long long)hi;
      const long long lh = (long long)(lo >> 64), ll = (long long)(unsigned long long)lo;
      const long long ohh = __shfl_xor_sync(0xffffffffu, hh, m), ohl = __shfl_xor_sync(0xffffffffu, hl, m);
      const long long olh = __shfl_xor_sync(0xffffffffu, lh, m), oll = __shfl_xor_sync(0xffffffffu, ll, m);
      hi += ((__int128)ohh << 64) | (__int128)(unsigned long long)ohl;
      lo += ((__int128)olh << 64) | (__int128)(unsigned long long)oll;
    }
    if (lane == 0) {
      const int row = (int)(o % k), col = (int)(o / k);
      const int er = xexp[row], fc = z ? wexp[col] : xexp[col];
      if (er == kNonFinite || fc == kNonFinite) {
        out[e] = __longlong_as_double(0x7FF8000000000000ll);
      } else {
        // a 128-bit sum x = x_h 2^32 + x_l with x_l in [0, 2^32): both parts are
        // exact doubles (|x| < 2^84), so the sum rounds once, for either sign
        auto to_double = [](__int128 x) {
          return (double)(long long)(x >> 32) * 0x1p32 + (double)(unsigned int)(x & 0xFFFFFFFF);
        };
        const double hd = to_double(hi);
        const double ld = to_double(lo);
        out[e] = ldexp(fma(ld, ldexp(1.0, -LoExp<S>::value), hd * ldexp(1.0, -kHiExp)), er + fc);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Digit planes.  GB300 runs FP64 at ~1/64 of FP32, so the digits are cut
// with integer arithmetic: |a| 2^-e (< 1) is rounded once to an integer M of
// 8S - 1 bits (the same information the S digits keep), then M is split into
// balanced base-256 digits, the first in [0, 128], the others in [-128, 127];
// the sign of a is applied to all of them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int row_exponent(double amax) {
  if (!(amax > 0.0) || !isfinite(amax)) return 0;
  int e;
  frexp(amax, &e);       // amax = m 2^e, m in [0.5, 1): |a| < 2^e
  return e;
}

// The same from the bit pattern of a non-negative double (integer work only):
// a normal value 1.f 2^(x - 1023) has e = x - 1022, a subnormal m 2^-1074
// with m of L bits has e = L - 1074; zero, Inf and NaN give 0.
__device__ __forceinline__ int exponent_of_bits(unsigned long long u) {
  if (u == 0ull || u >= 0x7FF0000000000000ull) return 0;
  const int x = (int)(u >> 52);
  return x ? x - 1022 : (64 - __clzll((long long)u)) - 1074;
}

// |a| as its bit pattern: non-negative doubles order like these integers, and
// integer compares stay off the FP64 pipe (a small fraction of the integer
// rate on this part).  Inf is 0x7FF0..., NaN above it.
__device__ __forceinline__ unsigned long long abs_bits(double a) {
  return (unsigned long long)__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFull;
}
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

// The exponent e of the largest |a| of a 128-byte FP64 row r in a swizzled
// tile (|a| < 2^e for every value of the row), with 32-bit integer work: the
// largest high word of |a| carries the largest exponent field; only a row
// whose largest value is subnormal or zero needs the full bit patterns.
// kNonFinite when the row holds Inf or NaN.
__device__ __forceinline__ int row_exponent16(const unsigned char* tile, int r) {
  uint32_t hw = 0u;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint4 v = *reinterpret_cast<const uint4*>(tile + (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)));
    hw = max(hw, max(v.y & 0x7FFFFFFFu, v.w & 0x7FFFFFFFu));
  }
  if (hw >= 0x7FF00000u) return kNonFinite;
  if (hw >= 0x00100000u) return (int)(hw >> 20) - 1022;
  unsigned long long am = 0ull;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const double2 v = *reinterpret_cast<const double2*>(tile + (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)));
    am = umax64(am, umax64(abs_bits(v.x), abs_bits(v.y)));
  }
  return exponent_of_bits(am);
}

// An integer-valued FP32 (|x| < 2^22) as an int: one add at the 1.5 x 2^23
// offset, no conversion instruction.
__device__ __forceinline__ int int_of_f32(uint32_t u) {
  return __float_as_int(__uint_as_float(u) + 12582912.0f) - 0x4B400000;
}

// round(|a| 2^(kBits (S - 1) + 7 - e)) (half up) for |a| < 2^e: the
// magnitude the digits represent (63 bits at S = 8).
template <int S>
__device__ __forceinline__ unsigned long long magnitude_bits(unsigned long long bits, int e) {
  const int exr = (int)((bits >> 52) & 0x7FF);
  const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (exr ? (1ull << 52) : 0ull);
  // |a| 2^(kBits (S - 1) + 7 - e) = mant 2^sh; below 2^(kBits (S - 1) + 7) <= 2^63
  const int sh = (exr ? exr : 1) - 1075 - e + kBits * (S - 1) + 7;
  const int rs = -sh;
  const unsigned long long up = mant << (sh > 0 ? sh : 0);
  const unsigned long long dn = rs > 0 && rs < 64 ? (mant + (1ull << (rs - 1))) >> rs : 0ull;
  return sh >= 0 ? up : dn;
}

// Balanced digits by one offset: with b = 2^kBits (256) and
// B = (b/2)(1 + b + ... + b^(S-2)), the base-b fields g_s of M + B (most
// significant first) give M = g_0 b^(S-1) + sum_(s>=1) (g_s - b/2) b^(S-1-s):
// digit 0 is g_0 in [0, 128] (M <= 2^63), digit s >= 1 is g_s - 128 in
// [-128, 127].  Every digit has at most 8 significant bits, so it is exact
// in F16 (and in BF16), and a product of two is at most 2^14.  Carries are the one 64-bit
// addition; each digit is a shift and a mask.
template <int S>
struct DigitBias {
  static constexpr unsigned long long value =
      (1ull << (kBits - 1)) + (1ull << kBits) * DigitBias<S - 1>::value;
};
template <>
struct DigitBias<1> {
  static constexpr unsigned long long value = 0ull;
};
template <int S>
__device__ __forceinline__ unsigned long long biased_magnitude(unsigned long long bits, int e) {
  return magnitude_bits<S>(bits, e) + DigitBias<S>::value;
}
template <int S>
__device__ __forceinline__ int bal_digit(unsigned long long Mb, int s) {
  const int sh = kBits * (S - 1 - s);
  return s == 0 ? (int)(Mb >> sh) : (int)((Mb >> sh) & ((1ull << kBits) - 1ull)) - (1 << (kBits - 1));
}

template <int S>
__device__ __forceinline__ void digits_of(double a, int e, int* d) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  const unsigned long long Mb = biased_magnitude<S>(bits, e);
  const int sg = (long long)bits < 0 ? -1 : 1;
#pragma unroll
  for (int s = 0; s < S; ++s) d[s] = sg * bal_digit<S>(Mb, s);
}

// Eight values' S digit planes as F16, one 16-byte chunk (eight values) per
// plane: out[s] holds digit s of values 0..7, all scaled by 2^-e.  The
// digits come straight from the bytes of the biased magnitudes: for a pair
// of values, one byte permute gathers byte s of both, a mask and an offset
// make them the F16 numbers 1024 + g, and one F16 fused multiply-add with
// (+-1, -+1152) (-+1024 for the first digit, which has no offset) gives the
// signed digits exactly.
template <int S>
__device__ __forceinline__ void planes_of8(const unsigned long long (&bits)[8], int e, uint4 (&out)[S]) {
  unsigned long long M[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) M[q] = biased_magnitude<S>(bits[q], e);
  uint32_t sg[4], ctop[4], clow[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool n0 = (long long)bits[2 * q] < 0, n1 = (long long)bits[2 * q + 1] < 0;
    sg[q] = (n0 ? 0xBC00u : 0x3C00u) | ((n1 ? 0xBC00u : 0x3C00u) << 16);     // +-1
    ctop[q] = (n0 ? 0x6400u : 0xE400u) | ((n1 ? 0x6400u : 0xE400u) << 16);   // -+1024
    clow[q] = (n0 ? 0x6480u : 0xE480u) | ((n1 ? 0x6480u : 0xE480u) << 16);   // -+1152
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int bi = S - 1 - s;                          // byte of the magnitude holding digit s
    const uint32_t sel = (uint32_t)(bi & 3) | ((uint32_t)((bi & 3) + 4) << 8);
    uint32_t w4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t a = bi < 4 ? (uint32_t)M[2 * q] : (uint32_t)(M[2 * q] >> 32);
      const uint32_t b = bi < 4 ? (uint32_t)M[2 * q + 1] : (uint32_t)(M[2 * q + 1] >> 32);
      const uint32_t w = (__byte_perm(a, b, sel) & 0x00FF00FFu) | 0x64006400u;
      const __half2 h = __hfma2(*reinterpret_cast<const __half2*>(&w), *reinterpret_cast<const __half2*>(&sg[q]),
                                *reinterpret_cast<const __half2*>(s == 0 ? &ctop[q] : &clow[q]));
      w4[q] = *reinterpret_cast<const uint32_t*>(&h);
    }
    out[s] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
  }
}

template <int S>
__global__ void slice_a_kernel(const double* __restrict__ A, int64_t n, int64_t lda, int n_pad,
                               __half* __restrict__ As, int* __restrict__ rowexp) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t plane = (int64_t)n_pad * n_pad;
  for (int64_t i = wid; i < n_pad; i += nw) {
    unsigned long long amax = 0ull;
    if (i < n)
      for (int64_t l = lane; l < n; l += 32) amax = umax64(amax, abs_bits(A[i * lda + l]));
    for (int o = 16; o > 0; o >>= 1) amax = umax64(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const bool finite = amax < kInfBits;
    const int e = exponent_of_bits(amax);
    if (lane == 0) rowexp[i] = finite ? e : kNonFinite;
    for (int64_t l0 = (int64_t)lane * 8; l0 < n_pad; l0 += 32 * 8) {
      unsigned long long b[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t l = l0 + q;
        b[q] = (i < n && l < n && finite) ? (unsigned long long)__double_as_longlong(A[i * lda + l]) : 0ull;
      }
      uint4 pl[S];
      planes_of8<S>(b, e, pl);
#pragma unroll
      for (int s = 0; s < S; ++s) *reinterpret_cast<uint4*>(As + s * plane + i * n_pad + l0) = pl[s];
    }
  }
}

// Column maxima of a strided n x k operand (element (l, j) at Y[l rs + j cs])
// as non-negative double bit patterns; NaN survives (fmax would drop it).
__device__ __forceinline__ void colmax_body(const double* __restrict__ Y, int64_t rows, int k, int64_t rs, int64_t cs,
                                            unsigned long long* __restrict__ cmax, int bx, int nbx) {
  __shared__ unsigned long long part[256];
  const int rpb = blockDim.x / k;  // threads beyond rpb k idle
  const bool live = (int)threadIdx.x < rpb * k;
  const int j = threadIdx.x % k;
  // four independent loads in flight per thread (the max is order-free)
  unsigned long long m[4] = {0ull, 0ull, 0ull, 0ull};
  const int64_t stride = (int64_t)nbx * rpb;
  for (int64_t i = bx * (int64_t)rpb + threadIdx.x / k; live && i < rows; i += 4 * stride) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t iu = i + u * stride;
      if (iu < rows) m[u] = umax64(m[u], abs_bits(Y[iu * rs + j * cs]));
    }
  }
  const unsigned long long mm = umax64(umax64(m[0], m[1]), umax64(m[2], m[3]));
  // one atomic per column and block
  part[threadIdx.x] = live ? mm : 0ull;
  __syncthreads();
  if ((int)threadIdx.x < k) {
    unsigned long long b = 0;
    for (int r = 0; r < rpb; ++r) b = max(b, part[r * k + threadIdx.x]);
    atomicMax(cmax + threadIdx.x, b);
  }
}

// Column maxima of a contiguous row-major rows x k operand, read as a flat
// array of 16-byte pairs (half the load instructions of the strided form).
// The grid is sized so that 2 x (threads) is a multiple of k: each thread
// then meets the same two columns on every step.
__global__ void __launch_bounds__(256) colmax_flat_kernel(const double* __restrict__ Y, int64_t total, int k,
                                                          unsigned long long* __restrict__ cmax, const Control* ctl) {
  if (ctl && ctl->done) return;
  __shared__ unsigned long long colm[kMaxK];
  for (int j = threadIdx.x; j < k; j += blockDim.x) colm[j] = 0ull;
  __syncthreads();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const double2* Y2 = reinterpret_cast<const double2*>(Y);
  const int64_t pairs = total / 2;
  unsigned long long m0[2] = {0ull, 0ull}, m1[2] = {0ull, 0ull};
  for (int64_t q = t; q < pairs; q += 2 * T) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t qu = q + u * T;
      if (qu < pairs) {
        const double2 v = Y2[qu];
        m0[u] = umax64(m0[u], abs_bits(v.x));
        m1[u] = umax64(m1[u], abs_bits(v.y));
      }
    }
  }
  if (t < pairs) {
    atomicMax(&colm[(2 * t) % k], umax64(m0[0], m0[1]));
    atomicMax(&colm[(2 * t + 1) % k], umax64(m1[0], m1[1]));
  }
  if (t == 0 && (total & 1))   // odd total: the last element
    atomicMax(&colm[(total - 1) % k], abs_bits(Y[total - 1]));
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x)
    if (colm[j]) atomicMax(cmax + j, colm[j]);
}

void launch_colmax_rowmajor(const double* Y, int64_t rows, int k, unsigned long long* cmax, const Control* ctl,
                            cudaStream_t s) {
  // blocks: about 8 per SM, a multiple of k / gcd(k, 512) so that 2 x threads is a multiple of k
  int g = 512, kk = k;
  while (kk % 2 == 0 && g % 2 == 0) { kk /= 2; g /= 2; }
  const int unit = kk;                                  // k / gcd(k, 512)
  const int blocks = ((152 * 8 + unit - 1) / unit) * unit;
  colmax_flat_kernel<<<blocks, 256, 0, s>>>(Y, rows * (int64_t)k, k, cmax, ctl);
}

__global__ void colmax_kernel(const double* __restrict__ Y, int64_t rows, int k, int64_t rs, int64_t cs,
                              unsigned long long* __restrict__ cmax, const Control* ctl) {
  if (ctl && ctl->done) return;
  colmax_body(Y, rows, k, rs, cs, cmax, blockIdx.x, gridDim.x);
}

// Column digit planes: planes[(t kp + j) K + l] (F16) for column j of the
// strided operand, scaled by its column exponent.  A CTA takes 64 rows x 32
// columns through shared memory, so the plane writes are contiguous.
template <int S>
__device__ __forceinline__ void slice_cols_body(const double* __restrict__ Y, int64_t rows, int k, int64_t rs,
                                                int64_t cs, int K, int kp, const unsigned long long* __restrict__ cmax,
                                                __half* __restrict__ planes, int* __restrict__ colexp, int bx,
                                                int cb) {
  __shared__ double tile[64][33];
  __shared__ int fexp[32];
  const int l0 = bx * 64;
  const int tid = threadIdx.x;
  if (tid < 32) {
    const int j = cb * 32 + tid;
    const double cm = j < k ? __longlong_as_double((long long)cmax[j]) : 0.0;
    const int f = row_exponent(cm);
    fexp[tid] = isfinite(cm) ? f : 0;
    if (bx == 0 && j < k) colexp[j] = isfinite(cm) ? f : kNonFinite;
  }
  for (int e = tid; e < 64 * 32; e += 256) {
    const int rr = e >> 5, jj = e & 31;
    const int64_t l = l0 + rr;
    const int j = cb * 32 + jj;
    tile[rr][jj] = (l < rows && j < k) ? Y[l * rs + j * cs] : 0.0;
  }
  __syncthreads();
  // thread -> (jj, 8 consecutive rows); writes 16 bytes per plane
  const int jj = tid >> 3, r0 = (tid & 7) * 8;
  unsigned long long b[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) b[q] = (unsigned long long)__double_as_longlong(tile[r0 + q][jj]);
  uint4 pl[S];
  planes_of8<S>(b, fexp[jj], pl);
#pragma unroll
  for (int t = 0; t < S; ++t) {
    const int64_t rowid = (int64_t)t * kp + cb * 32 + jj;
    if (cb * 32 + jj < kp)   // kp = 16: half the block's columns are padding
      *reinterpret_cast<uint4*>(planes + rowid * K + l0 + r0) = pl[t];
  }
}

template <int S>
__global__ void __launch_bounds__(256) slice_cols_kernel(const double* __restrict__ Y, int64_t rows, int k, int64_t rs,
                                                         int64_t cs, int K, int kp,
                                                         const unsigned long long* __restrict__ cmax,
                                                         __half* __restrict__ planes, int* __restrict__ colexp,
                                                         const Control* ctl, unsigned long long* clear = nullptr,
                                                         int nclear = 0) {
  if (ctl && ctl->done) return;
  // another operand's column maxima, read by an earlier kernel: cleared for
  // the kernel that forms them next
  if (clear && blockIdx.x == 0 && blockIdx.y == 0)
    for (int j = threadIdx.x; j < nclear; j += blockDim.x) clear[j] = 0ull;
  slice_cols_body<S>(Y, rows, k, rs, cs, K, kp, cmax, planes, colexp, blockIdx.x, blockIdx.y);
}

// Column digit planes for k <= 16 (planes of 16 rows): planes[(t 16 + j) K + l].
// A CTA takes 128 rows x 16 columns, so every thread cuts digits of a
// column that exists in the plane layout.
template <int S>
__global__ void __launch_bounds__(256) slice_cols16_kernel(const double* __restrict__ Y, int64_t rows, int k,
                                                           int64_t rs, int64_t cs, int K,
                                                           const unsigned long long* __restrict__ cmax,
                                                           __half* __restrict__ planes,
                                                           int* __restrict__ colexp, const Control* ctl) {
  if (ctl && ctl->done) return;
  __shared__ double tile[128][17];
  __shared__ int fexp[16];
  const int l0 = blockIdx.x * 128;
  const int tid = threadIdx.x;
  if (tid < 16) {
    const unsigned long long cm = tid < k ? cmax[tid] : 0ull;
    const int f = exponent_of_bits(cm);
    fexp[tid] = cm < kInfBits ? f : kNonFinite;
    if (blockIdx.x == 0 && tid < k) colexp[tid] = cm < kInfBits ? f : kNonFinite;
  }
  for (int e = tid; e < 128 * 16; e += 256) {
    const int rr = e >> 4, jj = e & 15;
    const int64_t l = l0 + rr;
    tile[rr][jj] = (l < rows && jj < k) ? Y[l * rs + jj * cs] : 0.0;
  }
  __syncthreads();
  // the digit planes of eight rows of column jj
  const int jj = tid >> 4, r0 = (tid & 15) * 8;
  const int fe = fexp[jj];
  unsigned long long b[8];
#pragma unroll
  for (int q = 0; q < 8; ++q)
    b[q] = fe != kNonFinite ? (unsigned long long)__double_as_longlong(tile[r0 + q][jj]) : 0ull;
  uint4 pl[S];
  planes_of8<S>(b, fe != kNonFinite ? fe : 0, pl);
#pragma unroll
  for (int t = 0; t < S; ++t) *reinterpret_cast<uint4*>(planes + ((int64_t)t * 16 + jj) * K + l0 + r0) = pl[t];
}

// Row digit planes of a row-major n x k operand: planes[(s n_pad + i) K + l],
// one exponent per row.  One warp per row; lane c takes elements 8c..8c+7.
template <int S>
__device__ __forceinline__ void slice_rows_body(const double* __restrict__ Y, int64_t n, int k, int n_pad, int K,
                                                __half* __restrict__ planes, int* __restrict__ rowexp,
                                                int64_t wid, int64_t nw) {
  const int lane = threadIdx.x & 31;
  const int64_t plane = (int64_t)n_pad * K;
  for (int64_t i = wid; i < n_pad; i += nw) {
    unsigned long long amax = 0ull;
    if (i < n)
      for (int l = lane; l < k; l += 32) amax = umax64(amax, abs_bits(Y[i * k + l]));
    for (int o = 16; o > 0; o >>= 1) amax = umax64(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const bool finite = amax < kInfBits;
    const int e = exponent_of_bits(amax);
    if (lane == 0) rowexp[i] = finite ? e : kNonFinite;
    for (int c = lane; c < K / 8; c += 32) {
      unsigned long long b[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int l = c * 8 + q;
        b[q] = (i < n && l < k && finite) ? (unsigned long long)__double_as_longlong(Y[i * k + l]) : 0ull;
      }
      uint4 pl[S];
      planes_of8<S>(b, e, pl);
#pragma unroll
      for (int s = 0; s < S; ++s) *reinterpret_cast<uint4*>(planes + s * plane + i * K + c * 8) = pl[s];
    }
  }
}

template <int S>
__global__ void slice_rows_kernel(const double* __restrict__ Y, int64_t n, int k, int n_pad, int K,
                                  __half* __restrict__ planes, int* __restrict__ rowexp, const Control* ctl) {
  if (ctl && ctl->done) return;
  slice_rows_body<S>(Y, n, k, n_pad, K, planes, rowexp, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5,
                     ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// ---- the same slicing for a batch: blockIdx.z selects the problem ----
enum { OPD_XCOLS = 0, OPD_PCOLS = 1, OPD_FCOLS = 2 };

__global__ void zero_cmax_grouped_kernel(const GroupItem* __restrict__ items) {
  const GroupItem& it = items[blockIdx.x];
  if (it.b[0].ctl->done) return;
  for (int j = threadIdx.x; j < it.k; j += blockDim.x) it.x_cmax[j] = it.p_cmax[j] = 0ull;
  for (int j = threadIdx.x; j < kfm_cols(it.k); j += blockDim.x) it.f_cmax[j] = 0ull;
}

// Columns of operand OP and the plane rows between its digit planes: the
// [F | M] panel of the row update has kfm_cols(k) of both, X and P have k
// columns in planes of k_pad rows.
__device__ __forceinline__ int grouped_cols(const GroupItem& it, int op) { return op == OPD_FCOLS ? kfm_cols(it.k) : it.k; }
__device__ __forceinline__ int grouped_kp(const GroupItem& it, int op) { return op == OPD_FCOLS ? kfm_cols(it.k) : it.k_pad; }

// Operand OP of problem `it` in sweep parity `parity`: rows, row / column strides.
__device__ __forceinline__ const double* grouped_operand(const GroupItem& it, int parity, int op, int64_t* rows,
                                                        int64_t* rs, int64_t* cs, unsigned long long** cmax,
                                                        __half** planes, int** colexp, int* K) {
  const SweepBufs& b = it.b[parity];
  if (op == OPD_FCOLS) {   // the [F | M] panel, k x kfm column-major: element (l, c) at FM[l + c k]
    *rows = it.k; *rs = 1; *cs = it.k; *cmax = it.f_cmax;
    *planes = static_cast<__half*>(it.f_planes); *colexp = it.f_colexp; *K = it.kr;
    return b.fm;
  }
  *rows = it.n; *rs = it.k; *cs = 1;
  *K = it.n_pad;
  if (op == OPD_XCOLS) {
    *cmax = it.x_cmax; *planes = static_cast<__half*>(it.x_planes); *colexp = it.x_colexp;
    return b.x;
  }
  *cmax = it.p_cmax; *planes = static_cast<__half*>(it.p_planes); *colexp = it.p_colexp;
  return b.p;
}

template <int OP>
__global__ void colmax_grouped_kernel(const GroupItem* __restrict__ items, int parity) {
  const GroupItem& it = items[blockIdx.z];
  if (it.b[0].ctl->done) return;
  int64_t rows, rs, cs;
  unsigned long long* cmax;
  __half* planes;
  int* colexp;
  int K;
  const double* Y = grouped_operand(it, parity, OP, &rows, &rs, &cs, &cmax, &planes, &colexp, &K);
  colmax_body(Y, rows, grouped_cols(it, OP), rs, cs, cmax, blockIdx.x, gridDim.x);
}

template <int S, int OP>
__global__ void __launch_bounds__(256) slice_cols_grouped_kernel(const GroupItem* __restrict__ items, int parity) {
  const GroupItem& it = items[blockIdx.z];
  int64_t rows, rs, cs;
  unsigned long long* cmax;
  __half* planes;
  int* colexp;
  int K;
  const double* Y = grouped_operand(it, parity, OP, &rows, &rs, &cs, &cmax, &planes, &colexp, &K);
  const int kp = grouped_kp(it, OP);
  if ((int)blockIdx.x * 64 >= K || (int)blockIdx.y * 32 >= kp || it.b[0].ctl->done) return;
  slice_cols_body<S>(Y, rows, grouped_cols(it, OP), rs, cs, K, kp, cmax, planes, colexp, blockIdx.x, blockIdx.y);
}

template <int S>
__global__ void slice_rows_grouped_kernel(const GroupItem* __restrict__ items, int parity) {
  const GroupItem& it = items[blockIdx.z];
  if (it.b[0].ctl->done) return;
  slice_rows_body<S>(it.b[parity].x, it.n, it.k, it.n_pad, it.kr, static_cast<__half*>(it.xr_planes),
                     it.xr_rowexp, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5,
                     ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// P = (exact sum of the split partial products) - shift Xs.  Fixed splits:
// ksplit partials an element.  Equal-work ranges (R > 0): the ranges that
// touch the element's row tile (U units of kbt K blocks a column block).
template <int S>
// P = recombined sum of a tile's exact partial slots - shift Xs.  One CTA per
// (row tile, 32-column block): the tile's slot count is worked out once, a
// warp covers 32 consecutive columns of a row (coalesced), 8 rows a step.
__global__ void __launch_bounds__(256) product_reduce_kernel(const longlong2* __restrict__ part, int ksplit,
                                                             const int* __restrict__ rowexp,
                                                             const int* __restrict__ colexp, int k,
                                                             const double* __restrict__ Xs, double* __restrict__ P,
                                                             int64_t n, double shift, const Control* ctl, int64_t R,
                                                             int64_t U, int64_t kbt,
                                                             unsigned long long* __restrict__ pmax = nullptr,
                                                             unsigned long long* clear = nullptr, int nclear = 0) {
  if (ctl && ctl->done) return;
  if (clear && blockIdx.x == 0 && blockIdx.y == 0)   // maxima read by an earlier kernel, formed again later
    for (int j = threadIdx.x; j < nclear; j += blockDim.x) clear[j] = 0ull;
  __shared__ unsigned long long wmax[8][32];
  const int64_t tile = blockIdx.x;
  int nq = ksplit;
  if (R > 0) {
    const int64_t u = tile * kbt;   // first unit of the row tile
    nq = (int)(((u + kbt) * R - 1) / U - ((u + 1) * R - 1) / U) + 1;
  }
  const int c = (int)blockIdx.y * 32 + (int)(threadIdx.x & 31);
  const int64_t total = n * k;
  const int64_t r0 = tile * kBM;
  unsigned long long m = 0ull;   // max |P| of this thread's rows, as an ordered bit pattern
  if (c < k) {
    const int fc = colexp[c];
#pragma unroll 4
    for (int lr = (int)(threadIdx.x >> 5); lr < kBM; lr += 8) {
      const int64_t row = r0 + lr;
      if (row >= n) break;
      const int64_t e = row * k + c;
      long long hi = 0, lo = 0;
      for (int q = 0; q < nq; ++q) {
        const longlong2 v = part[(int64_t)q * total + e];
        hi += v.x;
        lo += v.y;
      }
      const double w = recombine<S>(hi, lo, rowexp[row], fc) - shift * Xs[e];
      P[e] = w;
      m = umax64(m, abs_bits(w));
    }
  }
  if (pmax) {
    // the eight warps' maxima of each column, then one atomic a column and CTA
    wmax[threadIdx.x >> 5][threadIdx.x & 31] = m;
    __syncthreads();
    if (threadIdx.x < 32 && c < k) {
      unsigned long long mm = 0ull;
#pragma unroll
      for (int w = 0; w < 8; ++w) mm = umax64(mm, wmax[w][threadIdx.x]);
      atomicMax(pmax + c, mm);
    }
  }
}

// G = X^T X (z = 0), S = X^T W (z = 1) from the exact split partials; one
// warp per output, lanes over the splits.
template <int S>
__device__ __forceinline__ void sgram_reduce_body(const longlong2* __restrict__ part, int k, int nsplit,
                                                  const int* __restrict__ xexp, const int* __restrict__ wexp,
                                                  double* __restrict__ out, int64_t w0, int64_t nw) {
  const int64_t kk = (int64_t)k * k;
  const int lane = threadIdx.x & 31;
  for (int64_t e = w0; e < 2 * kk; e += nw) {
    const int z = (int)(e / kk);
    const int64_t o = e % kk;
    const longlong2* p = part + (int64_t)z * nsplit * kk + o;
    long long hi = 0, lo = 0;
    for (int c = lane; c < nsplit; c += 32) {
      const longlong2 v = p[(int64_t)c * kk];
      hi += v.x;
      lo += v.y;
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      hi += __shfl_xor_sync(0xffffffffu, hi, m);
      lo += __shfl_xor_sync(0xffffffffu, lo, m);
    }
    const int row = (int)(o % k), col = (int)(o / k);
    if (lane == 0) out[e] = recombine<S>(hi, lo, xexp[row], z ? wexp[col] : xexp[col]);
  }
}

template <int S>
__global__ void sgram_reduce_kernel(const longlong2* __restrict__ part, int k, int nsplit, const int* __restrict__ xexp,
                                    const int* __restrict__ wexp, double* __restrict__ out, const Control* ctl) {
  if (ctl && ctl->done) return;
  sgram_reduce_body<S>(part, k, nsplit, xexp, wexp, out, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5,
                       ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// Few splits (the batch's small problems): one thread per output, the splits
// added in order -- the same exact sum as the warp form.
template <int S>
__device__ __forceinline__ void sgram_reduce_thread_body(const longlong2* __restrict__ part, int k, int nsplit,
                                                         const int* __restrict__ xexp, const int* __restrict__ wexp,
                                                         double* __restrict__ out, int64_t t0, int64_t nt) {
  const int64_t kk = (int64_t)k * k;
  for (int64_t e = t0; e < 2 * kk; e += nt) {
    const int z = (int)(e / kk);
    const int64_t o = e % kk;
    const longlong2* p = part + (int64_t)z * nsplit * kk + o;
    long long hi = 0, lo = 0;
#pragma unroll 4
    for (int c = 0; c < nsplit; ++c) {
      const longlong2 v = p[(int64_t)c * kk];
      hi += v.x;
      lo += v.y;
    }
    const int row = (int)(o % k), col = (int)(o / k);
    out[e] = recombine<S>(hi, lo, xexp[row], z ? wexp[col] : xexp[col]);
  }
}

// The thread form for one problem with many outputs: consecutive threads read
// consecutive partials of a split (the warp form reads one sector per lane).
template <int S>
__global__ void sgram_reduce_thread_kernel(const longlong2* __restrict__ part, int k, int nsplit,
                                           const int* __restrict__ xexp, const int* __restrict__ wexp,
                                           double* __restrict__ out, const Control* ctl) {
  if (ctl && ctl->done) return;
  sgram_reduce_thread_body<S>(part, k, nsplit, xexp, wexp, out, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                              (int64_t)gridDim.x * blockDim.x);
}

template <int S>
__global__ void sgram_reduce_grouped_kernel(const GroupItem* __restrict__ items) {
  const GroupItem& it = items[blockIdx.z];
  if (it.b[0].ctl->done) return;
  if (it.ksplit <= 8)
    sgram_reduce_thread_body<S>(static_cast<const longlong2*>(it.sgpart), it.k, it.ksplit, it.x_colexp, it.p_colexp,
                                it.b[0].g2, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                                (int64_t)gridDim.x * blockDim.x);
  else
    sgram_reduce_body<S>(static_cast<const longlong2*>(it.sgpart), it.k, it.ksplit, it.x_colexp, it.p_colexp,
                         it.b[0].g2, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5,
                         ((int64_t)gridDim.x * blockDim.x) >> 5);
}

template <int S>
void launch_slice_a(const double* A, int64_t n, int64_t lda, int n_pad, __half* As, int* rowexp,
                    cudaStream_t s) {
  slice_a_kernel<S><<<152 * 8, 256, 0, s>>>(A, n, lda, n_pad, As, rowexp);
}

// Column planes of Y with its column maxima already in cmax (formed by the
// kernel that wrote Y); `clear` (nclear entries) is zeroed on the way.
template <int S>
void launch_slice_cols_ready(const double* Y, int64_t rows, int k, int64_t rs, int64_t cs, int K, int kp,
                             const unsigned long long* cmax, __half* planes, int* colexp, const Control* ctl,
                             cudaStream_t s, unsigned long long* clear = nullptr, int nclear = 0) {
  dim3 gx((unsigned)(K / 64), (unsigned)((kp + 31) / 32));
  slice_cols_kernel<S><<<gx, 256, 0, s>>>(Y, rows, k, rs, cs, K, kp, cmax, planes, colexp, ctl, clear, nclear);
}

template <int S>
void launch_slice_cols(const double* Y, int64_t rows, int k, int64_t rs, int64_t cs, int K, int kp,
                       unsigned long long* cmax, __half* planes, int* colexp, const Control* ctl,
                       cudaStream_t s) {
  cudaMemsetAsync(cmax, 0, (size_t)k * 8, s);
  if (rs == k && cs == 1) {
    launch_colmax_rowmajor(Y, rows, k, cmax, ctl, s);
  } else {
    const int rpb = 256 / k > 0 ? 256 / k : 1;
    colmax_kernel<<<152 * 8, rpb * k, 0, s>>>(Y, rows, k, rs, cs, cmax, ctl);
  }
  dim3 gx((unsigned)(K / 64), (unsigned)((kp + 31) / 32));
  slice_cols_kernel<S><<<gx, 256, 0, s>>>(Y, rows, k, rs, cs, K, kp, cmax, planes, colexp, ctl);
}

template <int S>
void launch_slice_cols16(const double* Y, int64_t rows, int k, int K, unsigned long long* cmax, __half* planes,
                         int* colexp, const Control* ctl, cudaStream_t s) {
  cudaMemsetAsync(cmax, 0, (size_t)k * 8, s);
  launch_colmax_rowmajor(Y, rows, k, cmax, ctl, s);
  slice_cols16_kernel<S><<<K / 128, 256, 0, s>>>(Y, rows, k, k, 1, K, cmax, planes, colexp, ctl);
}

template <int S>
void launch_slice_rows(const double* Y, int64_t n, int k, int n_pad, int K, __half* planes, int* rowexp,
                       const Control* ctl, cudaStream_t s) {
  slice_rows_kernel<S><<<152 * 8, 256, 0, s>>>(Y, n, k, n_pad, K, planes, rowexp, ctl);
}

// ---------------------------------------------------------------------------
// Row update X' = X + (W - X D) D^-1 - X F on the tensor cores, for an even
// k <= 16 over very many rows (the sparse workloads).  One CTA per SM,
// persistent over 128-row tiles; rows k.. are updated (the leading block is
// the k x k stage's).
//   warp 0     TMA loads of the X and W tiles: FP64, 128-byte rows (16
//              columns; those past k and rows past n read as zero), 128-byte
//              swizzle.
//   warp 1     tcgen05.mma.  A = the S row digit planes of the X tile stacked
//              along K (plane s at K = 16 s .. 16 s + 15, exponent e_i per
//              row); B = the S column digit planes of F stacked along N
//              (plane t at N = 16 t .., exponent f_j per column), then those
//              of M (rows 128 ..).  The instruction for plane s takes B rows
//              0 .. 16 (S - s) - 1 and writes TMEM columns 16 s ..: column
//              16 w + j then holds the sum of every pair (s, t) with s + t = w,
//              the pairs of one weight only, exact in FP32 (at most 8 pairs x
//              16 x 2^14 = 2^21); a second instruction does the same for M
//              into columns 128 + 16 s ...
//   warps 2-5  one thread per tile row: cut the X row into the A operand
//              (running up to two tiles ahead of the epilogue).
//   warps 6-21 four threads per tile row (warps w, w + 4, w + 8, w + 12 share
//              a TMEM lane group), four columns each: drain the accumulators,
//              rebuild each (X F)_ij with integer arithmetic up to its bit
//              pattern, form x' = x + (w - x d_j) / d_j - (X F)_ij in FP64 as
//              the one fused multiply-add w (1 / d_j) - (X F)_ij (the same
//              value in exact arithmetic; the rounding of 1 / d_j scales
//              column j as a whole, which the normalisation takes out), write it
//              over the X tile in shared memory and store it with TMA (32 rows
//              per lane group), keeping the column sums of x'^2,
//              (w - x d_j)^2 and v^2, v = (w - x d_j) - (X M)_ij the row of
//              V2 = R2 - X2 M (E21 = V2 D^-1, the lower block of E-tilde_L in Algorithm 4).
// Accumulators and A operands are double-
// buffered, the X / W tiles triple-buffered.  Every wait is bounded; on expiry
// the CTA records a timeout.  No FP64 instruction outside the update formula
// and its sums: this part runs FP64 at a small fraction of its integer rate.
// ---------------------------------------------------------------------------
constexpr int kU16Stages = 3;
constexpr int kU16Tile = 128 * 128;                // 128 rows x 16 FP64: 16 KiB
constexpr int kU16Stage = 2 * kU16Tile;           // X tile, W tile
constexpr int kU16ABlock = kBM * kBK * 2;         // 128 rows x 64 K F16 (four planes)
constexpr int kU16ABuf = ((kMaxS + 3) / 4) * kU16ABlock;   // planes 0..7, four per block
constexpr int kU16BRows = 16 * kMaxS;             // rows (t, j) of one operand's planes
constexpr int kU16BBytes = 2 * kU16BRows * 128;   // F's then M's rows of 128 B; K = l in the first 32 B
constexpr int kU16SliceWarps = 4;                 // one thread per tile row
constexpr int kU16EpiWarps = 16;                  // four threads per tile row, four columns each
constexpr int kU16Threads = 64 + 32 * (kU16SliceWarps + kU16EpiWarps);
constexpr int kU16Smem = kU16Stages * kU16Stage + 2 * kU16ABuf + kU16BBytes + 1024 + 1024;

struct Upd16Args {
  int64_t n;
  int k;
  int row_begin;        // rows below it (the leading block) are left alone
  int tiles;            // ceil(n / 128); the grid is at most this
  const double* F;      // k x k column-major
  const double* M;      // k x k column-major (V2 = R2 - X2 M)
  const double* d;
  const double* dinv;
  double* Xn;           // plain stores of the one tile that holds rows below row_begin
  double* upart;        // [gridDim.x][3k]: column sums of x'^2, of (w - x d)^2, of v^2
  const Control* ctl;
  int* err;
  unsigned long long wait_ns;   // limit of every bounded wait (0: the default)
};

struct __align__(8) BarsU16 {
  // sub[g][i & 3]: the four warps of lane group g have written tile i (a ring
  // of four: a warp can run at most two tiles ahead of its group's leader,
  // which releases the X stage and, with the others, the accumulators)
  uint64_t full[kU16Stages], empty[kU16Stages], a_full[2], a_empty[2], acc_full[2], acc_empty[2], sub[4][4], drain;
  uint32_t tmem_base;
  WaitState wait;
};

// Byte offset of 16-byte chunk c of row r in a tile of 128-byte rows with the
// 128-byte swizzle (the layout TMA writes and the MMA descriptors describe).
__device__ __forceinline__ uint32_t swz128(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map), "r"(src),
               "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

#define TC_LD4(taddr, r)                                                                     \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"                 \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])                            \
               : "r"(taddr))

// One weight group of update16's accumulators (weights W0 .. W0 + NW - 1, at
// most four) as exact int64 sums, one a column: weight w counts
// 2^(kBits (TOP - w)).  The group's TMEM columns are loaded together and
// waited for once.  Each accumulator C_w is an integer-valued FP32 with
// |C_w| <= (w + 1) 2^18 (at most 16 products of two digits of at most 2^7
// for each of the w + 1 plane pairs); adding 1.5 x 2^23 makes its bit
// pattern C_w + 0x4B400000, and two weights w, w + 1 are joined as
// C_w 2^kBits + C_(w+1) (below 2^30) in 32-bit arithmetic, the offsets taken
// off modulo 2^32 in the same step; the two halves of the group are then
// joined in 64 bits.
template <int W0, int NW, int TOP, int C>
__device__ __forceinline__ void drain_u16_group(uint32_t tl, long long (&out)[C]) {
  uint32_t v[NW][C];
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    if constexpr (C == 8)
      TC_LD8(tl + 16 * (W0 + w), v[w]);
    else
      TC_LD4(tl + 16 * (W0 + w), v[w]);
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  constexpr uint32_t kOff = 0x4B400000u;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    long long acc = 0;
#pragma unroll
    for (int a = 0; a < NW; a += 2) {
      const uint32_t ua = __float_as_uint(__uint_as_float(v[a][j]) + 12582912.0f);
      int h;
      int last;
      if (a + 1 < NW) {
        const uint32_t ub = __float_as_uint(__uint_as_float(v[a + 1][j]) + 12582912.0f);
        h = (int)(ua * (1u << kBits) + ub - ((1u << kBits) + 1u) * kOff);
        last = a + 1;
      } else {
        h = (int)(ua - kOff);
        last = a;
      }
      acc += (long long)h * (1ll << (kBits * (TOP - (W0 + last))));
    }
    out[j] = acc;
  }
}

// One lane's C columns of one accumulator set of update16 into two exact int64
// sums: digit-pair groups w < 4 (hi, weight w counting 2^(kBits (3 - w))) and
// w >= 4 (lo, 2^(kBits (S - 1 - w))).
template <int S, int C = 8>
__device__ __forceinline__ void drain_u16(uint32_t tl, long long (&hi)[C], long long (&lo)[C]) {
  drain_u16_group<0, (S < 4 ? S : 4), 3, C>(tl, hi);
  if constexpr (S > 4) {
    drain_u16_group<4, S - 4, S - 1, C>(tl, lo);
  } else {
#pragma unroll
    for (int j = 0; j < C; ++j) lo[j] = 0;
  }
}

template <int S>
__global__ void __launch_bounds__(kU16Threads, 1) update16_kernel(const __grid_constant__ CUtensorMap tmX,
                                                                  const __grid_constant__ CUtensorMap tmW,
                                                                  const __grid_constant__ CUtensorMap tmXn,
                                                                  Upd16Args g) {
  if (g.ctl && g.ctl->done) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* stage0 = smem;
  unsigned char* abuf0 = smem + kU16Stages * kU16Stage;
  unsigned char* bop = abuf0 + 2 * kU16ABuf;
  BarsU16* bars = reinterpret_cast<BarsU16*>(bop + kU16BBytes);
  __shared__ int fexp_s[32];                 // column exponents of F (0 .. 15), of M (16 .. 31)
  __shared__ double d_s[16], dinv_s[16];
  __shared__ double colsum[3][4][16];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x;
  const int cnt = (g.tiles - (int)blockIdx.x + G - 1) / G;   // this CTA's tiles: blockIdx.x + i G
  WaitState* wst = &bars->wait;
  const unsigned long long wlim = wait_limit(g.wait_ns);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kU16Stages; ++i) {
      mbar_init(smem_u32(&bars->full[i]), 1);
      mbar_init(smem_u32(&bars->empty[i]), 4);                  // the four lane-group leaders
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&bars->a_full[i]), kU16SliceWarps);
      mbar_init(smem_u32(&bars->a_empty[i]), 1);
      mbar_init(smem_u32(&bars->acc_full[i]), 1);
      mbar_init(smem_u32(&bars->acc_empty[i]), kU16EpiWarps);
    }
    for (int i = 0; i < 16; ++i) mbar_init(smem_u32(&bars->sub[i >> 2][i & 3]), kU16EpiWarps / 4);
    mbar_init(smem_u32(&bars->drain), 1);
    bars->wait.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&bars->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    // column exponents of F and M, and d, 1/d (zero past k)
    const int j = threadIdx.x & 15;
    const double* Fm = threadIdx.x < 16 ? g.F : g.M;
    int fe = 0;
    if (j < g.k) {
      unsigned long long m = 0ull;
      for (int l = 0; l < g.k; ++l) m = umax64(m, abs_bits(Fm[(int64_t)j * g.k + l]));
      fe = m < kInfBits ? exponent_of_bits(m) : kNonFinite;
    }
    fexp_s[threadIdx.x] = fe;
    if (threadIdx.x < 16) {
      d_s[j] = j < g.k ? g.d[j] : 0.0;
      dinv_s[j] = j < g.k ? g.dinv[j] : 0.0;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = bars->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmX) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmW) : "memory");
      bool ok = true;
      int issued = 0;
      for (int i = 0; i < cnt && ok; ++i) {
        const int st = i % kU16Stages, lap = i / kU16Stages;
        ok = mbar_wait_sleep(smem_u32(&bars->empty[st]), (uint32_t)((lap & 1) ^ 1), wst, wlim);
        if (!ok) break;
        const int row0 = ((int)blockIdx.x + i * G) * 128;
        unsigned char* sx = stage0 + st * kU16Stage;
        mbar_expect_tx(smem_u32(&bars->full[st]), (uint32_t)kU16Stage);
        tma_load_2d(smem_u32(sx), &tmX, smem_u32(&bars->full[st]), 0, row0);
        tma_load_2d(smem_u32(sx + kU16Tile), &tmW, smem_u32(&bars->full[st]), 0, row0);
        ++issued;
      }
      if (!ok)
        for (int i = (issued > kU16Stages ? issued - kU16Stages : 0); i < issued; ++i)
          mbar_drain(smem_u32(&bars->full[i % kU16Stages]), (uint32_t)((i / kU16Stages) & 1));
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      const uint64_t bd = smem_desc(smem_u32(bop));
      for (int i = 0; i < cnt && ok; ++i) {
        const int a = i & 1, u = i >> 1;
        ok = mbar_wait_sleep(smem_u32(&bars->a_full[a]), (uint32_t)(u & 1), wst, wlim);
        if (ok) ok = mbar_wait_sleep(smem_u32(&bars->acc_empty[a]), (uint32_t)((u & 1) ^ 1), wst, wlim);
        if (!ok) break;
        tc_fence_after();
        const uint32_t ab = smem_u32(abuf0 + a * kU16ABuf);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const uint64_t ad = smem_desc(ab + (uint32_t)((s >> 2) * kU16ABlock)) + (uint64_t)(2 * (s & 3));
          tc_mma(tbase + (uint32_t)(a * 256 + 16 * s), ad, bd, idesc_f16(kBM, 16 * (S - s)), s == 0 ? 0u : 1u);
          // X M: M's planes from B row 128 on, accumulators from TMEM column 128 on
          tc_mma(tbase + (uint32_t)(a * 256 + 128 + 16 * s), ad, bd + (uint64_t)((kU16BRows * 128) >> 4),
                 idesc_f16(kBM, 16 * (S - s)), s == 0 ? 0u : 1u);
        }
        tc_commit(smem_u32(&bars->a_empty[a]));
        tc_commit(smem_u32(&bars->acc_full[a]));
      }
      if (!ok) {
        tc_commit(smem_u32(&bars->drain));
        mbar_drain(smem_u32(&bars->drain), 0);
      }
    }
  } else if (warp < 2 + kU16SliceWarps) {
    // ---------------- slicers: one thread per tile row, all 16 columns ----------------
    const int r = (warp - 2) * 32 + lane;
    // B operand first: digit t of F(l, j) at row 16 t + j, K = l, and of M(l, j)
    // at row 128 + 16 t + j (four (operand, j, l) a thread)
    for (int e = r; e < 512; e += 128) {
      const int op = e >> 8, j = (e >> 4) & 15, l = e & 15;
      const int fe = fexp_s[16 * op + j];
      const double* Fm = op ? g.M : g.F;
      const double v = (j < g.k && l < g.k && fe != kNonFinite) ? Fm[(int64_t)j * g.k + l] : 0.0;
      int dg[S];
      digits_of<S>(v, fe == kNonFinite ? 0 : fe, dg);
#pragma unroll
      for (int t = 0; t < S; ++t)
        *reinterpret_cast<uint16_t*>(bop + swz128(kU16BRows * op + 16 * t + j, l >> 3) + (l & 7) * 2) =
            __half_as_ushort(__int2half_rn(dg[t]));
    }
    bool ok = true;
    for (int i = 0; i < cnt && ok; ++i) {
      const int st = i % kU16Stages, lap = i / kU16Stages, a = i & 1;
      int w_ok = 1;
      if (lane == 0) {
        w_ok = mbar_wait_sleep(smem_u32(&bars->full[st]), (uint32_t)(lap & 1), wst, wlim);
        if (w_ok) w_ok = mbar_wait_sleep(smem_u32(&bars->a_empty[a]), (uint32_t)(((i >> 1) & 1) ^ 1), wst, wlim);
      }
      ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
      if (!ok) break;
      mbar_wait_sleep(smem_u32(&bars->full[st]), (uint32_t)(lap & 1), wst, wlim);   // complete: each lane acquires
      const unsigned char* xt = stage0 + st * kU16Stage;
      // the row's exponent first, then the planes half a row at a time (the
      // values are read from shared memory twice, to keep registers for the
      // sixteen epilogue warps)
      const int er = row_exponent16(xt, r);
      const bool fin = er != kNonFinite;
      const int e = fin ? er : 0;
      unsigned char* ab = abuf0 + a * kU16ABuf;
#pragma unroll
      for (int h = 0; h < 2; ++h) {   // columns 8 h .. 8 h + 7: one 16-byte chunk per plane
        unsigned long long bh[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const double2 v = *reinterpret_cast<const double2*>(xt + swz128(r, 4 * h + q));
          bh[2 * q] = fin ? (unsigned long long)__double_as_longlong(v.x) : 0ull;
          bh[2 * q + 1] = fin ? (unsigned long long)__double_as_longlong(v.y) : 0ull;
        }
        uint4 pl[S];
        planes_of8<S>(bh, e, pl);
#pragma unroll
        for (int s = 0; s < S; ++s)
          *reinterpret_cast<uint4*>(ab + (s >> 2) * kU16ABlock + swz128(r, 2 * (s & 3) + h)) = pl[s];
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->a_full[a]));
    }
  } else {
    // ---------------- epilogue: four threads per tile row, four columns each ----------------
    constexpr int kC = 4;                        // columns a thread
    const int ew = warp - 2 - kU16SliceWarps;   // 0..15
    const int lg = warp & 3;                     // TMEM lane group: tile rows 32 lg .. 32 lg + 31
    const int qt = ew >> 2;                      // columns kC qt .. kC qt + kC - 1
    const bool leader = qt == 0;                 // stores the lane group's 32 rows
    const int r = lg * 32 + lane;
    double sq[kC], rq[kC], vq[kC];
#pragma unroll
    for (int j = 0; j < kC; ++j) sq[j] = rq[j] = vq[j] = 0.0;
    bool ok = true;
    for (int i = 0; i < cnt && ok; ++i) {
      const int a = i & 1, u = i >> 1;
      int w_ok = 1;
      if (lane == 0) w_ok = mbar_wait_sleep(smem_u32(&bars->acc_full[a]), (uint32_t)(u & 1), wst, wlim);
      ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
      if (!ok) break;
      __syncwarp();
      tc_fence_after();
      // the X and W tiles of this tile: loaded (the slicers waited for them)
      // and not refilled before this warp's leader releases the stage
      const int st = i % kU16Stages;
      mbar_wait_sleep(smem_u32(&bars->full[st]), (uint32_t)((i / kU16Stages) & 1), wst, wlim);
      unsigned char* xt = stage0 + st * kU16Stage;
      const unsigned char* wt = xt + kU16Tile;
      // the row's exponent (as the slicers took it) and this thread's X values
      double2 xv[kC / 2];
      const int e_row = row_exponent16(xt, r);
#pragma unroll
      for (int q = 0; q < kC / 2; ++q) xv[q] = *reinterpret_cast<const double2*>(xt + swz128(r, (kC / 2) * qt + q));
      const uint32_t tl = tbase + ((uint32_t)(lg * 32) << 16) + (uint32_t)(a * 256 + kC * qt);
      // X M first (TMEM columns 128 ..), rounded at once, then X F
      double xm[kC];
      long long hi[kC], lo[kC];
      drain_u16<S, kC>(tl + 128u, hi, lo);
#pragma unroll
      for (int j = 0; j < kC; ++j) xm[j] = recombine<S>(hi[j], lo[j], e_row, fexp_s[16 + kC * qt + j]);
      drain_u16<S, kC>(tl, hi, lo);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->acc_empty[a]));
      const int64_t row0 = ((int64_t)blockIdx.x + (int64_t)i * G) * 128;
      const int64_t row = row0 + r;
      const bool live = row >= g.row_begin && row < g.n;
#pragma unroll
      for (int q = 0; q < kC / 2; ++q) {
        const int cc = (kC / 2) * qt + q;     // 16-byte chunk: columns 2 cc, 2 cc + 1
        const double2 x2 = xv[q];
        const double2 wv = *reinterpret_cast<const double2*>(wt + swz128(r, cc));
        const int j0 = 2 * cc, j1 = 2 * cc + 1;
        const double f0 = recombine<S>(hi[2 * q], lo[2 * q], e_row, fexp_s[j0]);
        const double f1 = recombine<S>(hi[2 * q + 1], lo[2 * q + 1], e_row, fexp_s[j1]);
        const double r0 = fma(-x2.x, d_s[j0], wv.x), r1 = fma(-x2.y, d_s[j1], wv.y);
        // x' = x + r / d - f = w / d - f, one fused multiply-add
        const double n0 = fma(wv.x, dinv_s[j0], -f0), n1 = fma(wv.y, dinv_s[j1], -f1);
        const double v0 = r0 - xm[2 * q], v1 = r1 - xm[2 * q + 1];   // rows of V2 = R2 - X2 M
        if (live) {
          sq[2 * q] = fma(n0, n0, sq[2 * q]);
          sq[2 * q + 1] = fma(n1, n1, sq[2 * q + 1]);
          rq[2 * q] = fma(r0, r0, rq[2 * q]);
          rq[2 * q + 1] = fma(r1, r1, rq[2 * q + 1]);
          vq[2 * q] = fma(v0, v0, vq[2 * q]);
          vq[2 * q + 1] = fma(v1, v1, vq[2 * q + 1]);
        }
        *reinterpret_cast<double2*>(xt + swz128(r, cc)) = make_double2(n0, n1);
      }
      const bool plain = row0 < g.row_begin;   // the tile with the leading block
      if (plain && live)
        for (int j = kC * qt; j < kC * qt + kC && j < g.k; ++j)
          g.Xn[row * g.k + j] = reinterpret_cast<const double*>(xt + swz128(r, j >> 1))[j & 1];
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars->sub[lg][i & 3]));
      if (leader) {
        int s_ok = 1;
        if (lane == 0) {
          s_ok = mbar_wait_sleep(smem_u32(&bars->sub[lg][i & 3]), (uint32_t)((i >> 2) & 1), wst, wlim);
          if (s_ok) {
            if (!plain && row0 + 32 * lg < g.n) {
              tma_store_2d(&tmXn, smem_u32(xt + lg * 32 * 128), 0, (int)(row0 + 32 * lg));
              bulk_commit();
              bulk_wait_read_all();   // the store has read the tile: the stage may be refilled
            }
            mbar_arrive(smem_u32(&bars->empty[st]));
          }
        }
        ok = __shfl_sync(0xffffffffu, s_ok, 0) != 0;
      }
    }
    if (lane == 0) bulk_wait_all();
    // column sums over this warp's rows, in a fixed order
#pragma unroll
    for (int j = 0; j < kC; ++j) {
      for (int o = 16; o > 0; o >>= 1) {
        sq[j] += __shfl_xor_sync(0xffffffffu, sq[j], o);
        rq[j] += __shfl_xor_sync(0xffffffffu, rq[j], o);
        vq[j] += __shfl_xor_sync(0xffffffffu, vq[j], o);
      }
      if (lane == 0) {
        colsum[0][lg][kC * qt + j] = sq[j];
        colsum[1][lg][kC * qt + j] = rq[j];
        colsum[2][lg][kC * qt + j] = vq[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if ((int)threadIdx.x < 3 * g.k) {
    const int which = threadIdx.x / g.k, j = threadIdx.x % g.k;
    g.upart[(int64_t)blockIdx.x * 3 * g.k + which * g.k + j] =
        colsum[which][0][j] + colsum[which][1][j] + colsum[which][2][j] + colsum[which][3][j];
  }
  if (bars->wait.abort && threadIdx.x == 0) {
    atomicExch(g.err, 1);
    if (g.ctl) {
      Control* c = const_cast<Control*>(g.ctl);
      c->status = EIGREF_E_TIMEOUT;
      c->done = 1;
    }
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
  }
}

// ---------------------------------------------------------------------------
// The same Gram products for an even k <= 16, cutting the digit planes in the
// kernel: each 64-row K block of X and W arrives by TMA as FP64 rows (128-byte
// swizzle, rows past n read as zero), the eight worker warps cut both into
// the stacked-plane tiles the MMA reads (one 16-byte chunk of 8 rows per
// thread, plane and operand), and the same warps drain the accumulators after
// the last K block of each exact chunk.  The column exponents come from
// column maxima formed before the launch.  HBM traffic is the FP64 operands,
// read once; the planes never leave shared memory.
// ---------------------------------------------------------------------------
constexpr int kG16FRaw = 4;                          // FP64 tile ring
constexpr int kG16FRawTile = 64 * 128;               // 64 rows x 16 FP64: 8 KiB
constexpr int kG16FPlanes = 3;                       // plane-tile ring (X planes, W planes)
constexpr int kG16FSmem = kG16FRaw * 2 * kG16FRawTile + kG16FPlanes * kG16Stage + 1024 + 1024;

struct Gram16FArgs {
  Gram16Args g;
  const unsigned long long* xmax;   // column maxima of |X|, |W| (ordered bits)
  const unsigned long long* wmax;
  int* xexp;                        // column exponents for the reduction (written by CTA 0)
  int* wexp;
};

struct __align__(8) Bars16F {
  uint64_t raw_full[kG16FRaw], raw_empty[kG16FRaw], pl_full[kG16FPlanes], pl_empty[kG16FPlanes], acc_full,
      acc_empty, drain;
  uint32_t tmem_base;
  WaitState wait;
};

template <int S>
__global__ void __launch_bounds__(kThreads, 1) sgram16f_kernel(const __grid_constant__ CUtensorMap tmX,
                                                              const __grid_constant__ CUtensorMap tmW,
                                                              Gram16FArgs fa) {
  const Gram16Args& g = fa.g;
  __shared__ int s_skip;
  __shared__ int fexp_s[2][16];
  if (threadIdx.x == 0) s_skip = (g.ctl && g.ctl->done) ? 1 : 0;
  if (threadIdx.x < 32) {
    // column exponents of X (0..15) and W (16..31); non-finite columns give NaN
    const int op = threadIdx.x >> 4, j = threadIdx.x & 15;
    const unsigned long long cm = j < g.k ? (op ? fa.wmax[j] : fa.xmax[j]) : 0ull;
    const int f = exponent_of_bits(cm);
    const int fe = cm < kInfBits ? f : kNonFinite;
    fexp_s[op][j] = fe;
    if (blockIdx.x == 0 && j < g.k) (op ? fa.wexp : fa.xexp)[j] = fe;
  }
  __syncthreads();
  if (s_skip) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* raw0 = smem;                                        // [kG16FRaw][X tile, W tile]
  unsigned char* pl0 = smem + kG16FRaw * 2 * kG16FRawTile;           // [kG16FPlanes][X planes, W planes]
  Bars16F* bars = reinterpret_cast<Bars16F*>(pl0 + kG16FPlanes * kG16Stage);
  constexpr int kRows = 16 * S;                      // rows of a stacked tile
  constexpr int kColsJob = kRows;                    // TMEM columns per product
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int split = blockIdx.x;
  const int kb_lo = (int)((int64_t)g.kb_total * split / g.ksplit);
  const int kb_hi = (int)((int64_t)g.kb_total * (split + 1) / g.ksplit);
  const int KB = kb_hi - kb_lo;
  WaitState* wst = &bars->wait;
  const unsigned long long wlim = wait_limit(g.wait_ns);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kG16FRaw; ++i) {
      mbar_init(smem_u32(&bars->raw_full[i]), 1);
      mbar_init(smem_u32(&bars->raw_empty[i]), kEpiWarps);
    }
    for (int i = 0; i < kG16FPlanes; ++i) {
      mbar_init(smem_u32(&bars->pl_full[i]), kEpiWarps);
      mbar_init(smem_u32(&bars->pl_empty[i]), 1);
    }
    mbar_init(smem_u32(&bars->acc_full), 1);
    mbar_init(smem_u32(&bars->acc_empty), kEpiWarps);
    mbar_init(smem_u32(&bars->drain), 1);
    bars->wait.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&bars->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = bars->tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer: the FP64 X and W rows of each K block ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmX) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmW) : "memory");
      bool ok = true;
      int issued = 0;
      for (int kb = 0; kb < KB && ok; ++kb) {
        const int st = kb % kG16FRaw, lap = kb / kG16FRaw;
        ok = mbar_wait_sleep(smem_u32(&bars->raw_empty[st]), (uint32_t)((lap & 1) ^ 1), wst, wlim);
        if (!ok) break;
        const int row = (kb_lo + kb) * kBK;
        unsigned char* rt = raw0 + st * 2 * kG16FRawTile;
        mbar_expect_tx(smem_u32(&bars->raw_full[st]), (uint32_t)(2 * kG16FRawTile));
        tma_load_2d(smem_u32(rt), &tmX, smem_u32(&bars->raw_full[st]), 0, row);
        tma_load_2d(smem_u32(rt + kG16FRawTile), &tmW, smem_u32(&bars->raw_full[st]), 0, row);
        ++issued;
      }
      if (!ok)
        for (int i = (issued > kG16FRaw ? issued - kG16FRaw : 0); i < issued; ++i)
          mbar_drain(smem_u32(&bars->raw_full[i % kG16FRaw]), (uint32_t)((i / kG16FRaw) & 1));
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = true;
      for (int kb = 0; kb < KB && ok; ++kb) {
        const int c = kb / kG16Chunk;
        const bool first = (kb % kG16Chunk) == 0;
        const bool last = (kb % kG16Chunk) == kG16Chunk - 1 || kb == KB - 1;
        if (first && c > 0) {   // one accumulator set: the previous chunk must be drained
          ok = mbar_wait_sleep(smem_u32(&bars->acc_empty), (uint32_t)((c - 1) & 1), wst, wlim);
          if (!ok) break;
          tc_fence_after();
        }
        const int pb = kb % kG16FPlanes;
        ok = mbar_wait_sleep(smem_u32(&bars->pl_full[pb]), (uint32_t)((kb / kG16FPlanes) & 1), wst, wlim);
        if (!ok) break;
        tc_fence_after();
        unsigned char* pt = pl0 + pb * kG16Stage;
        const uint64_t xd = smem_desc(smem_u32(pt));
        const uint64_t yd = smem_desc(smem_u32(pt + kG16Tile));
        constexpr uint32_t id1 = idesc_f16(kBM, kRows);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t acc = (first && q == 0) ? 0u : 1u;
          const uint64_t o = (uint64_t)(2 * q);    // 16 K per step inside the 128-byte swizzle row
          tc_mma(tbase, xd + o, xd + o, id1, acc);                                 // G: X planes x X planes
          tc_mma(tbase + kColsJob, xd + o, yd + o, id1, acc);                      // S: X planes x W planes
        }
        tc_commit(smem_u32(&bars->pl_empty[pb]));
        if (last) tc_commit(smem_u32(&bars->acc_full));
      }
      if (!ok) {
        tc_commit(smem_u32(&bars->drain));
        mbar_drain(smem_u32(&bars->drain), 0);
      }
    }
  } else {
    // ---------------- workers: cut the planes of every K block, drain every chunk ----------------
    const int te = threadIdx.x - 64;             // 0..255
    const int op = te >> 7;                      // slicing: 0 = X, 1 = W
    const int sj = te & 15, sig = (te >> 4) & 7; // column j, rows 8 sig .. 8 sig + 7 of the K block
    const int fe = fexp_s[op][sj];
    const int lg = warp & 3;                     // TMEM lane group
    const int job = (warp - 2) >> 2;             // 0: G = X^T X, 1: S = X^T W
    const int r = lg * 32 + lane;                // TMEM lane = 16 s + i
    const int sp = r >> 4;                       // plane s of X this lane holds
    long long hi[16], lo[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) hi[j] = lo[j] = 0;
    bool ok = true;
    for (int kb = 0; kb < KB && ok; ++kb) {
      const int st = kb % kG16FRaw, pb = kb % kG16FPlanes;
      int w_ok = 1;
      if (lane == 0) {
        w_ok = mbar_wait_sleep(smem_u32(&bars->raw_full[st]), (uint32_t)((kb / kG16FRaw) & 1), wst, wlim);
        if (w_ok)
          w_ok = mbar_wait_sleep(smem_u32(&bars->pl_empty[pb]), (uint32_t)(((kb / kG16FPlanes) & 1) ^ 1), wst, wlim);
      }
      ok = __shfl_sync(0xffffffffu, w_ok, 0) != 0;
      if (!ok) break;
      mbar_wait_sleep(smem_u32(&bars->raw_full[st]), (uint32_t)((kb / kG16FRaw) & 1), wst, wlim);   // each lane acquires
      {
        const unsigned char* rt = raw0 + (st * 2 + op) * kG16FRawTile;
        unsigned long long b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = 8 * sig + q;
          b[q] = fe != kNonFinite ? (unsigned long long)__double_as_longlong(
                                        *reinterpret_cast<const double*>(rt + swz128(i, sj >> 1) + (sj & 1) * 8))
                                  : 0ull;
        }
        uint4 pl[S];
        planes_of8<S>(b, fe != kNonFinite ? fe : 0, pl);
        unsigned char* pt = pl0 + pb * kG16Stage + op * kG16Tile;
#pragma unroll
        for (int t = 0; t < S; ++t) *reinterpret_cast<uint4*>(pt + swz128(16 * t + sj, sig)) = pl[t];
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&bars->pl_full[pb]));
        mbar_arrive(smem_u32(&bars->raw_empty[st]));
      }
      const bool last = (kb % kG16Chunk) == kG16Chunk - 1 || kb == KB - 1;
      if (last) {
        const int c = kb / kG16Chunk;
        int a_ok = 1;
        if (lane == 0) a_ok = mbar_wait_sleep(smem_u32(&bars->acc_full), (uint32_t)(c & 1), wst, wlim);
        ok = __shfl_sync(0xffffffffu, a_ok, 0) != 0;
        __syncwarp();
        if (!ok) break;
        tc_fence_after();
        const uint32_t tl = tbase + ((uint32_t)(lg * 32) << 16) + (uint32_t)(job * kColsJob);
#pragma unroll
        for (int t = 0; t < S; ++t) {
          // plane t of the right operand
          const uint32_t col = (uint32_t)(16 * t);
          const int w = sp + t;
          uint32_t v[16];
          TC_LD16(tl + col, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (w <= S - 1) {
            if (w < 4) {
              const int sh = kBits * (3 - w);
#pragma unroll
              for (int j = 0; j < 16; ++j) hi[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh;
            } else {
              const int sh = kBits * (S - 1 - w);
#pragma unroll
              for (int j = 0; j < 16; ++j) lo[j] += (long long)__float2int_rn(__uint_as_float(v[j])) << sh;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->acc_empty));
      }
    }
    // the 8 threads of a job holding row i (4 lane groups x 2 lanes) add their sums
    asm volatile("bar.sync 1, 256;" ::: "memory");   // every worker is past its last shared-memory use
    longlong2* red = reinterpret_cast<longlong2*>(pl0);   // [2 jobs][8 contributors][16 i][16 j]
    const int i = r & 15;
    const int qc = lg * 2 + (lane >> 4);
#pragma unroll
    for (int j = 0; j < 16; ++j) red[((job * 8 + qc) * 16 + i) * 16 + j] = make_longlong2(hi[j], lo[j]);
    asm volatile("bar.sync 1, 256;" ::: "memory");
    const int oi = te & 15, oj = (te >> 4) & 15;
#pragma unroll
    for (int jb = 0; jb < 2; ++jb) {
      long long h = 0, l = 0;
      for (int q = 0; q < 8; ++q) {
        const longlong2 e = red[((jb * 8 + q) * 16 + oi) * 16 + oj];
        h += e.x;
        l += e.y;
      }
      if (ok && oi < g.k && oj < g.k)
        g.part[((int64_t)(jb * g.ksplit + split) * g.k + oj) * g.k + oi] = make_longlong2(h, l);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (bars->wait.abort && threadIdx.x == 0) {
    atomicExch(g.err, 1);
    if (g.ctl) {
      Control* c = const_cast<Control*>(g.ctl);
      c->status = EIGREF_E_TIMEOUT;
      c->done = 1;
    }
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
  }
}

#define EIGREF_SLICE_DISPATCH(S_, CALL) \
  switch (S_) {                         \
    case 2: CALL(2); break;             \
    case 3: CALL(3); break;             \
    case 4: CALL(4); break;             \
    case 5: CALL(5); break;             \
    case 6: CALL(6); break;             \
    case 7: CALL(7); break;             \
    default: CALL(8); break;            \
  }

// ---------------------------------------------------------------------------
// Tensor maps (driver entry point fetched at run time; no -lcuda)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
              uint32_t box_outer) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Row-major rows x k FP64 operand in tiles of 16 columns (past k: zero) by
// box_rows rows, 128-byte swizzle (k even: rows are 16-byte multiples).
bool make_map_f64(CUtensorMap* m, const void* base, int k, int64_t rows, uint32_t box_rows) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)k * 8};
  cuuint32_t box[2] = {16, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace sl

cudaError_t init_sliced_attributes() {
  cudaError_t e = cudaSuccess;
#define EIGREF_SET_ATTR(S_)                                                                                        \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(sl::sliced_mma_kernel<S_, sl::MODE_PRODUCT>,                                        \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sl::kSmemBytesProduct);                  \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(sl::sliced_wide_kernel<S_>, cudaFuncAttributeMaxDynamicSharedMemorySize,               \
                             sl::kSmemBytesWide);                                                                  \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(sl::sliced_mma_kernel<S_, sl::MODE_GRAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             sl::kSmemBytes);                                                                      \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(sl::sliced_update_persistent_kernel<S_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             sl::kSmemBytesUpdate);                                                                \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(sl::sliced_mma_grouped_kernel<S_, sl::MODE_PRODUCT>,                                \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sl::kSmemBytesProduct);                  \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(sl::sliced_mma_grouped_kernel<S_, sl::MODE_GRAM>,                                   \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sl::kSmemBytes);                         \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(sl::sliced_mma_grouped_kernel<S_, sl::MODE_UPDATE>,                                 \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sl::kSmemBytesUpdate);                   \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(sl::sgram16_kernel<S_>, cudaFuncAttributeMaxDynamicSharedMemorySize, sl::kG16Smem); \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(sl::update16_kernel<S_>, cudaFuncAttributeMaxDynamicSharedMemorySize, sl::kU16Smem); \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(sl::sgram16f_kernel<S_>, cudaFuncAttributeMaxDynamicSharedMemorySize, sl::kG16FSmem);
  EIGREF_SET_ATTR(2) EIGREF_SET_ATTR(3) EIGREF_SET_ATTR(4) EIGREF_SET_ATTR(5) EIGREF_SET_ATTR(6)
  EIGREF_SET_ATTR(7) EIGREF_SET_ATTR(8)
#undef EIGREF_SET_ATTR
  return e;
}

// ---- plan / workspace ----
struct SlicedLayout {
  size_t a_planes, rowexp, x_planes, x_colexp, x_cmax, p_planes, p_colexp, p_cmax, xr_planes, xr_rowexp, f_planes,
      f_colexp, f_cmax, gpart, ppart, err, total;
};

static SlicedLayout sliced_layout(int64_t n_pad, int k_pad, int kr, int S, int ksplit, int k, int psplit = 1,
                                  int64_t n = 0) {
  SlicedLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 1023) & ~size_t(1023);
    size_t o = off;
    off += bytes;
    return o;
  };
  L.a_planes = take((size_t)S * n_pad * n_pad * 2);
  L.rowexp = take((size_t)n_pad * 4);
  L.x_planes = take((size_t)S * k_pad * n_pad * 2);
  L.x_colexp = take((size_t)k_pad * 4);
  L.x_cmax = take((size_t)k_pad * 8);
  L.p_planes = take((size_t)S * k_pad * n_pad * 2);
  L.p_colexp = take((size_t)k_pad * 4);
  L.p_cmax = take((size_t)k_pad * 8);
  L.xr_planes = take((size_t)S * n_pad * kr * 2);
  L.xr_rowexp = take((size_t)n_pad * 4);
  // the row update's B operand: the [F | M] panel (kfm_cols(k) columns)
  L.f_planes = take((size_t)S * kfm_cols(k) * kr * 2);
  L.f_colexp = take((size_t)kfm_cols(k) * 4);
  L.f_cmax = take((size_t)kfm_cols(k) * 8);
  L.gpart = take((size_t)2 * ksplit * k * k * 16);
  L.ppart = take(psplit > 1 ? (size_t)psplit * n * k * 16 : 64);
  L.err = take(64);
  L.total = off + 1024;
  return L;
}

size_t SlicedA::layout_total() const {
  return sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_).total;
}

int SlicedA::configure(const double* A, int64_t n, int64_t lda, int k, int precision, int slices) {
  A_ = A;
  n_ = n;
  lda_ = lda;
  k_ = k;
  precision_ = precision;
  slices_ = slices > 0 ? slices : sl::kDefaultS;
  if (precision != EIGREF_BF16_SLICES) {
    snprintf(err_, sizeof(err_), "split form %d not built (BF16 slices only)", precision);
    return EIGREF_E_UNSUPPORTED;
  }
  if (slices_ < 2 || slices_ > sl::kMaxS) {
    snprintf(err_, sizeof(err_), "slices must be in [2, %d]", sl::kMaxS);
    return EIGREF_E_INVALID;
  }
  // int64 headroom of the low group: (n / 256) 2^23.5 2^(7 (S - 5)) (S - 4) < 2^63
  const int64_t nmax = slices_ <= 8 ? ((int64_t)1 << 24) : ((int64_t)1 << 18);
  if (n > nmax) {
    snprintf(err_, sizeof(err_), "split form with %d slices limited to n <= %lld", slices_, (long long)nmax);
    return EIGREF_E_INVALID;
  }
  if (!sl::encode_fn()) {
    snprintf(err_, sizeof(err_), "cuTensorMapEncodeTiled unavailable");
    return EIGREF_E_CUDA;
  }
  n_pad_ = (int)((n + 255) / 256 * 256);
  k_pad_ = (k + 31) / 32 * 32;
  kr_ = (k + 63) / 64 * 64;
  // Gram split-K: about two CTAs per SM in total (2 jobs x k_pad/32 column blocks)
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_split = 2 * (k_pad_ / 32);
  ksplit_ = (304 + per_split - 1) / per_split;
  const int kbt = n_pad_ / sl::kBK;
  if (ksplit_ > kbt) ksplit_ = kbt;
  if (ksplit_ < 1) ksplit_ = 1;
  // the workspace holds partials for the largest split an autotuner may try
  psplit_max_ = 1;
  for (int p = 2; p <= 4; ++p)
    if ((n_pad_ / 64) / p >= 8) psplit_max_ = p;
  ksplit_max_ = std::min(kbt, 2 * ksplit_);
  // Equal-work product: each column block's gy x kbt (row tile, K block)
  // units cut into R equal ranges, R a whole number of rounds of one CTA per
  // SM with ranges no longer than a row tile (a range then covers at most two
  // tiles); small problems take at most 3 gy ranges, so that a tile meets at
  // most 4 ranges (the workspace's partial slots).
  {
    const int gx = k_pad_ / 32, gy = n_pad_ / sl::kBM;
    const int q = std::max(1, sms / gx);
    sk_units_ = (long long)gy * kbt;
    sk_ranges_ = gy < q ? std::min<long long>(q, 3LL * gy) : (long long)q * ((gy + q - 1) / q);
  }
  // The 128 x 64 product: one round of one CTA per SM, ranges of at least a
  // row tile (a tile then meets at most two ranges), or, for few row tiles,
  // at most 3 gy ranges (at most 4 a tile).
  if (k_pad_ % 64 == 0) {
    const int gx = k_pad_ / 64, gy = n_pad_ / sl::kBM;
    const int q = std::max(1, sms / gx);
    sk_units_w_ = (long long)gy * kbt;
    sk_ranges_w_ = gy < q ? std::min<long long>(q, 3LL * gy) : (long long)q;
  }
  wide_ = false;
  pslots_ = 4;
  psplit_ = kPsplitBalanced;
  return EIGREF_OK;
}

std::vector<int> SlicedA::psplit_candidates() const {
  std::vector<int> v;
  if (pslots_ >= 4) v.push_back(kPsplitBalanced);
  for (int p = 1; p <= psplit_max_; ++p) v.push_back(p);
  return v;
}

std::vector<int> SlicedA::ksplit_candidates() const {
  std::vector<int> v;
  const int h = ksplit_;
  for (int c : {std::max(1, h / 2), h, ksplit_max_})
    if (v.empty() || v.back() != c) v.push_back(c);
  return v;
}

int SlicedA::set_product_tile(int cols) {
  if (cols != 0 && cols != 32 && cols != 64) {
    snprintf(err_, sizeof(err_), "product_tile must be 0, 32 or 64 (%d)", cols);
    return EIGREF_E_INVALID;
  }
  if (cols == 64 && k_pad_ % 64 != 0) {
    snprintf(err_, sizeof(err_), "product_tile 64 needs k in (64 j - 32, 64 j] (k = %d)", k_);
    return EIGREF_E_INVALID;
  }
  wide_ = cols != 32 && k_pad_ % 64 == 0;
  return EIGREF_OK;
}

void SlicedA::set_splits(int psplit, int ksplit) {
  psplit_ = (psplit == kPsplitBalanced && pslots_ >= 4) ? kPsplitBalanced : std::max(1, std::min(psplit, psplit_max_));
  ksplit_ = std::max(1, std::min(ksplit, ksplit_max_));
}

size_t SlicedA::workspace_bytes() const { return layout_total(); }

void SlicedA::share_gpu(int problems) {
  if (problems <= 1) return;
  wide_ = false;
  psplit_ = psplit_max_ = pslots_ = 1;
  const int kbt = n_pad_ / sl::kBK;
  ksplit_ = ksplit_max_ = std::max(1, std::min(kbt, n_pad_ / 4096));
}

void SlicedA::bind_workspace(char* p) { ws_ = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023)); }

int SlicedA::prepare(cudaStream_t s) {
  const SlicedLayout L = sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_);
  auto* ap = reinterpret_cast<__half*>(ws_ + L.a_planes);
  // B-side and row planes: zero once, so padding rows and columns stay zero
  if (cudaMemsetAsync(ws_ + L.x_planes, 0, L.xr_rowexp - L.x_planes, s) != cudaSuccess ||
      cudaMemsetAsync(ws_ + L.f_planes, 0, L.f_colexp - L.f_planes, s) != cudaSuccess ||
      cudaMemsetAsync(ws_ + L.err, 0, 64, s) != cudaSuccess) {
    snprintf(err_, sizeof(err_), "memset of slice planes failed");
    return EIGREF_E_CUDA;
  }
  int* rowexp = reinterpret_cast<int*>(ws_ + L.rowexp);
#define EIGREF_CALL_SLICE_A(S_) sl::launch_slice_a<S_>(A_, n_, lda_, n_pad_, ap, rowexp, s)
  EIGREF_SLICE_DISPATCH(slices_, EIGREF_CALL_SLICE_A)
#undef EIGREF_CALL_SLICE_A
  const uint64_t S = (uint64_t)slices_;
  bool ok = sl::make_map(reinterpret_cast<CUtensorMap*>(tmA_), ap, (uint64_t)n_pad_, S * n_pad_, sl::kBK, sl::kBM);
  ok = ok && sl::make_map(reinterpret_cast<CUtensorMap*>(tmX_), ws_ + L.x_planes, (uint64_t)n_pad_, S * k_pad_,
                          sl::kBK, sl::kBN);
  ok = ok && sl::make_map(reinterpret_cast<CUtensorMap*>(tmXA_), ws_ + L.x_planes, (uint64_t)n_pad_, S * k_pad_,
                          sl::kBK, sl::kBM);
  ok = ok && sl::make_map(reinterpret_cast<CUtensorMap*>(tmP_), ws_ + L.p_planes, (uint64_t)n_pad_, S * k_pad_,
                          sl::kBK, sl::kBN);
  ok = ok && sl::make_map(reinterpret_cast<CUtensorMap*>(tmXR_), ws_ + L.xr_planes, (uint64_t)kr_, S * n_pad_,
                          sl::kBK, sl::kBM);
  if (k_pad_ % 64 == 0) {
    ok = ok && sl::make_map(reinterpret_cast<CUtensorMap*>(tmXw_), ws_ + L.x_planes, (uint64_t)n_pad_, S * k_pad_,
                            sl::kBK, sl::kWBN);
    ok = ok && sl::make_map(reinterpret_cast<CUtensorMap*>(tmPw_), ws_ + L.p_planes, (uint64_t)n_pad_, S * k_pad_,
                            sl::kBK, sl::kWBN);
  }
  ok = ok && sl::make_map(reinterpret_cast<CUtensorMap*>(tmF_), ws_ + L.f_planes, (uint64_t)kr_, S * kfm_cols(k_),
                          sl::kBK, sl::kBN);
  if (!ok) {
    snprintf(err_, sizeof(err_), "tensor map encoding failed");
    return EIGREF_E_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess) {
    snprintf(err_, sizeof(err_), "slicing A failed");
    return EIGREF_E_CUDA;
  }
  return EIGREF_OK;
}

static sl::MmaArgs base_args(const Control* ctl, int* err, unsigned long long wait_ns) {
  sl::MmaArgs g;
  memset(&g, 0, sizeof(g));
  g.ctl = ctl;
  g.err = err;
  g.ksplit = 1;
  g.wait_ns = wait_ns;
  return g;
}

template <int MODE>
static void launch_mma(int S, dim3 grid, const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& b2,
                       const sl::MmaArgs& g, cudaStream_t s) {
#define EIGREF_CALL_MMA(S_) \
  sl::sliced_mma_kernel<S_, MODE><<<grid, sl::kThreads, sl::smem_bytes(MODE), s>>>(a, b, b2, g)
  EIGREF_SLICE_DISPATCH(S, EIGREF_CALL_MMA)
#undef EIGREF_CALL_MMA
}

static void launch_product_reduce(int S, const MmaTask& t, int psplit, const double* Xs, double* P, int64_t total,
                                  double shift, const Control* ctl, cudaStream_t s,
                                  unsigned long long* pmax = nullptr, unsigned long long* clear = nullptr) {
  const int64_t n = total / t.g.k;
  const dim3 rg((unsigned)((n + sl::kBM - 1) / sl::kBM), (unsigned)((t.g.k + 31) / 32));
#define EIGREF_CALL_PR(S_)                                                                                   \
  sl::product_reduce_kernel<S_><<<rg, 256, 0, s>>>(t.g.ppart, psplit, t.g.rowexp, t.g.colexp, t.g.k, Xs, P, n, shift, \
                                                   ctl, t.g.sk_ranges, t.g.sk_units, t.g.kb_total, pmax, clear, \
                                                   clear ? t.g.k : 0)
  EIGREF_SLICE_DISPATCH(S, EIGREF_CALL_PR)
#undef EIGREF_CALL_PR
}

static void launch_task(int S, int mode, const MmaTask& t, cudaStream_t s) {
  const dim3 grid((unsigned)t.gx, (unsigned)t.gy, (unsigned)t.gz);
  if (mode == sl::MODE_PRODUCT && t.wide) {
#define EIGREF_CALL_WIDE(S_) sl::sliced_wide_kernel<S_><<<grid, sl::kThreads, sl::kSmemBytesWide, s>>>(t.a, t.b, t.g)
    EIGREF_SLICE_DISPATCH(S, EIGREF_CALL_WIDE)
#undef EIGREF_CALL_WIDE
  } else if (mode == sl::MODE_PRODUCT) {
    launch_mma<sl::MODE_PRODUCT>(S, grid, t.a, t.b, t.b2, t.g, s);
  } else if (mode == sl::MODE_GRAM) {
    launch_mma<sl::MODE_GRAM>(S, grid, t.a, t.b, t.b2, t.g, s);
  } else {
    // persistent: one CTA per SM (the kernel's shared memory allows one), at most one per tile
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = t.gx * t.gy;
    const int ctas = std::max(1, std::min(tiles, sms));
#define EIGREF_CALL_UPD(S_)                                                                                   \
  sl::sliced_update_persistent_kernel<S_><<<ctas, sl::kThreadsU, sl::kSmemBytesUpdate, s>>>(t.a, t.b, t.g, t.gx, tiles)
    EIGREF_SLICE_DISPATCH(S, EIGREF_CALL_UPD)
#undef EIGREF_CALL_UPD
  }
}

MmaTask SlicedA::product_task(const double* X, double* P, double shift, const Control* ctl, const double* Xs,
                              bool b_from_p) const {
  const SlicedLayout L = sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_);
  MmaTask t;
  t.a = *reinterpret_cast<const CUtensorMap*>(tmA_);
  t.b = t.b2 = *reinterpret_cast<const CUtensorMap*>(b_from_p ? tmP_ : tmX_);
  sl::MmaArgs& g = t.g;
  g = base_args(ctl, reinterpret_cast<int*>(ws_ + L.err), wait_ns_);
  g.a_plane_rows = n_pad_;
  g.b_plane_rows = k_pad_;
  g.kb_total = n_pad_ / sl::kBK;
  g.rowexp = reinterpret_cast<const int*>(ws_ + L.rowexp);
  g.colexp = reinterpret_cast<const int*>(ws_ + (b_from_p ? L.p_colexp : L.x_colexp));
  g.m_valid = n_;
  g.k = k_;
  g.X = X;
  g.Xs = Xs ? Xs : X;
  g.P = P;
  g.shift = shift;
  g.ppart = reinterpret_cast<longlong2*>(ws_ + L.ppart);
  t.wide = wide_ ? 1 : 0;
  if (wide_) t.b = t.b2 = *reinterpret_cast<const CUtensorMap*>(b_from_p ? tmPw_ : tmXw_);
  t.gx = k_pad_ / (wide_ ? sl::kWBN : sl::kBN);
  if (psplit_ == kPsplitBalanced) {
    // grid (column blocks, ranges): range blockIdx.y of column block blockIdx.x
    g.ksplit = 1;
    g.sk_ranges = (int)(wide_ ? sk_ranges_w_ : sk_ranges_);
    g.sk_units = wide_ ? sk_units_w_ : sk_units_;
    t.gy = g.sk_ranges;
    t.gz = 1;
  } else {
    g.ksplit = psplit_;
    t.gy = n_pad_ / sl::kBM;
    t.gz = psplit_;
  }
  return t;
}

MmaTask SlicedA::gram_task(double* part, const Control* ctl) const {
  const SlicedLayout L = sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_);
  MmaTask t;
  t.a = *reinterpret_cast<const CUtensorMap*>(tmXA_);
  t.b = *reinterpret_cast<const CUtensorMap*>(tmX_);
  t.b2 = *reinterpret_cast<const CUtensorMap*>(tmP_);
  sl::MmaArgs& g = t.g;
  g = base_args(ctl, reinterpret_cast<int*>(ws_ + L.err), wait_ns_);
  g.a_plane_rows = k_pad_;
  g.b_plane_rows = k_pad_;
  g.kb_total = n_pad_ / sl::kBK;
  g.ksplit = ksplit_;
  g.rowexp = reinterpret_cast<const int*>(ws_ + L.x_colexp);   // rows of G, S = columns of X
  g.colexp = reinterpret_cast<const int*>(ws_ + L.x_colexp);
  g.colexp2 = reinterpret_cast<const int*>(ws_ + L.p_colexp);
  g.m_valid = k_;
  g.k = k_;
  g.gpart = reinterpret_cast<longlong2*>(ws_ + L.gpart);
  (void)part;
  t.gx = k_pad_ / sl::kBN;
  t.gy = 1;
  t.gz = 2 * ksplit_;
  return t;
}

MmaTask SlicedA::update_task(const double* X, const double* W, const double* d, const double* dinv, double* Xn,
                             double* upart, const Control* ctl) const {
  const SlicedLayout L = sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_);
  MmaTask t;
  t.a = *reinterpret_cast<const CUtensorMap*>(tmXR_);
  t.b = t.b2 = *reinterpret_cast<const CUtensorMap*>(tmF_);
  sl::MmaArgs& g = t.g;
  g = base_args(ctl, reinterpret_cast<int*>(ws_ + L.err), wait_ns_);
  g.a_plane_rows = n_pad_;
  g.b_plane_rows = kfm_cols(k_);
  g.kb_total = kr_ / sl::kBK;
  g.rowexp = reinterpret_cast<const int*>(ws_ + L.xr_rowexp);
  g.colexp = reinterpret_cast<const int*>(ws_ + L.f_colexp);   // by column of the [F | M] panel
  g.m_valid = n_;
  g.k = k_;
  g.row_begin = k_;
  g.X = X;
  g.W = W;
  g.d = d;
  g.dinv = dinv;
  g.Xn = Xn;
  g.upart = upart;
  t.gx = kfm_cols(k_) / sl::kBN;   // a column block: 16 columns of X F and the same of X M
  t.gy = n_pad_ / sl::kBM;
  t.gz = 1;
  return t;
}

void SlicedA::fill_group_item(GroupItem* it) const {
  const SlicedLayout L = sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_);
  it->n_pad = n_pad_;
  it->k_pad = k_pad_;
  it->kr = kr_;
  it->ksplit = ksplit_;
  it->x_planes = ws_ + L.x_planes;
  it->p_planes = ws_ + L.p_planes;
  it->xr_planes = ws_ + L.xr_planes;
  it->f_planes = ws_ + L.f_planes;
  it->x_colexp = reinterpret_cast<int*>(ws_ + L.x_colexp);
  it->p_colexp = reinterpret_cast<int*>(ws_ + L.p_colexp);
  it->xr_rowexp = reinterpret_cast<int*>(ws_ + L.xr_rowexp);
  it->f_colexp = reinterpret_cast<int*>(ws_ + L.f_colexp);
  it->x_cmax = reinterpret_cast<unsigned long long*>(ws_ + L.x_cmax);
  it->p_cmax = reinterpret_cast<unsigned long long*>(ws_ + L.p_cmax);
  it->f_cmax = reinterpret_cast<unsigned long long*>(ws_ + L.f_cmax);
  it->sgpart = ws_ + L.gpart;
}

int SlicedA::product(const double* X, double* P, double shift, const Control* ctl, cudaStream_t s, cudaEvent_t ev0,
                     cudaEvent_t ev1, unsigned ev_flags) {
  const SlicedLayout L = sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_);
  auto* xp = reinterpret_cast<__half*>(ws_ + L.x_planes);
  auto* cmax = reinterpret_cast<unsigned long long*>(ws_ + L.x_cmax);
  auto* pmax = reinterpret_cast<unsigned long long*>(ws_ + L.p_cmax);
  int* colexp = reinterpret_cast<int*>(ws_ + L.x_colexp);
  // fused maxima: X's came from the normalisation; P's maxima (read by the
  // last Gram slicing) are cleared here and formed by the reduction, which
  // clears X's once this slicing has read them
  const bool fused = fused_max_ && psplit_ > 1;
#define EIGREF_CALL_SLICE_X(S_)                                                                              \
  if (fused)                                                                                                 \
    sl::launch_slice_cols_ready<S_>(X, n_, k_, k_, 1, n_pad_, k_pad_, cmax, xp, colexp, ctl, s, pmax, k_);   \
  else                                                                                                       \
    sl::launch_slice_cols<S_>(X, n_, k_, k_, 1, n_pad_, k_pad_, cmax, xp, colexp, ctl, s)
  EIGREF_SLICE_DISPATCH(slices_, EIGREF_CALL_SLICE_X)
#undef EIGREF_CALL_SLICE_X
  const MmaTask t = product_task(X, P, shift, ctl);
  if (ev0) cudaEventRecordWithFlags(ev0, s, ev_flags);
  launch_task(slices_, sl::MODE_PRODUCT, t, s);
  if (psplit_ > 1)
    launch_product_reduce(slices_, t, psplit_, X, P, n_ * k_, shift, ctl, s, fused ? pmax : nullptr,
                          fused ? cmax : nullptr);
  if (ev1) cudaEventRecordWithFlags(ev1, s, ev_flags);
  return psplit_ > 1 ? (fused ? 3 : 4) : 3;
}

bool SlicedA::fused_maxima() const { return fused_max_ && psplit_ > 1; }

unsigned long long* SlicedA::x_cmax() const {
  return reinterpret_cast<unsigned long long*>(
      ws_ + sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_).x_cmax);
}
unsigned long long* SlicedA::p_cmax() const {
  return reinterpret_cast<unsigned long long*>(
      ws_ + sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_).p_cmax);
}
unsigned long long* SlicedA::fm_cmax() const {
  return reinterpret_cast<unsigned long long*>(
      ws_ + sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_).f_cmax);
}

int SlicedA::product_sq(const double* X, double* T, double* P, double alpha, const Control* ctl, cudaStream_t s,
                        cudaEvent_t ev0, cudaEvent_t ev1, unsigned ev_flags) {
  const SlicedLayout L = sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_);
  const int64_t total = n_ * k_;
  const int rg = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  // T = A X: X's column planes in the X slot (kept for gram())
  auto* xp = reinterpret_cast<__half*>(ws_ + L.x_planes);
  auto* xmax = reinterpret_cast<unsigned long long*>(ws_ + L.x_cmax);
  int* xexp = reinterpret_cast<int*>(ws_ + L.x_colexp);
#define EIGREF_CALL_SLICE_X2(S_) \
  sl::launch_slice_cols<S_>(X, n_, k_, k_, 1, n_pad_, k_pad_, xmax, xp, xexp, ctl, s)
  EIGREF_SLICE_DISPATCH(slices_, EIGREF_CALL_SLICE_X2)
#undef EIGREF_CALL_SLICE_X2
  if (ev0) cudaEventRecordWithFlags(ev0, s, ev_flags);
  const MmaTask t1 = product_task(X, T, 0.0, ctl);
  launch_task(slices_, sl::MODE_PRODUCT, t1, s);
  if (psplit_ > 1) launch_product_reduce(slices_, t1, psplit_, X, T, total, 0.0, ctl, s);
  // P = A T - alpha X: T's column planes in the W slot (gram() re-slices W there)
  auto* pp = reinterpret_cast<__half*>(ws_ + L.p_planes);
  auto* pmax = reinterpret_cast<unsigned long long*>(ws_ + L.p_cmax);
  int* pexp = reinterpret_cast<int*>(ws_ + L.p_colexp);
#define EIGREF_CALL_SLICE_T(S_) \
  sl::launch_slice_cols<S_>(T, n_, k_, k_, 1, n_pad_, k_pad_, pmax, pp, pexp, ctl, s)
  EIGREF_SLICE_DISPATCH(slices_, EIGREF_CALL_SLICE_T)
#undef EIGREF_CALL_SLICE_T
  const MmaTask t2 = product_task(T, P, alpha, ctl, X, true);
  launch_task(slices_, sl::MODE_PRODUCT, t2, s);
  if (psplit_ > 1) launch_product_reduce(slices_, t2, psplit_, X, P, total, alpha, ctl, s);
  if (ev1) cudaEventRecordWithFlags(ev1, s, ev_flags);
  return psplit_ > 1 ? 10 : 8;
}

int SlicedA::gram(const double* P, double* part, double* out, const Control* ctl, cudaStream_t s) {
  const SlicedLayout L = sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_);
  auto* pp = reinterpret_cast<__half*>(ws_ + L.p_planes);
  auto* cmax = reinterpret_cast<unsigned long long*>(ws_ + L.p_cmax);
  int* pexp = reinterpret_cast<int*>(ws_ + L.p_colexp);
  const bool fused = fused_maxima();   // P's maxima formed by the product's reduction
#define EIGREF_CALL_SLICE_P(S_)                                                                   \
  if (fused)                                                                                      \
    sl::launch_slice_cols_ready<S_>(P, n_, k_, k_, 1, n_pad_, k_pad_, cmax, pp, pexp, ctl, s);    \
  else                                                                                            \
    sl::launch_slice_cols<S_>(P, n_, k_, k_, 1, n_pad_, k_pad_, cmax, pp, pexp, ctl, s)
  EIGREF_SLICE_DISPATCH(slices_, EIGREF_CALL_SLICE_P)
#undef EIGREF_CALL_SLICE_P
  const MmaTask t = gram_task(part, ctl);
  launch_task(slices_, sl::MODE_GRAM, t, s);
  // many outputs (k >= 32): a thread per output, coalesced over the splits;
  // otherwise a warp per output.  Both add the exact int64 partials.
  const bool per_thread = 2LL * k_ * k_ >= 2048;
  const int rg = per_thread ? (int)((2LL * k_ * k_ + 255) / 256) : (int)std::min<int64_t>((2LL * k_ * k_ + 7) / 8, 152 * 8);
#define EIGREF_CALL_SGR(S_)                                                                                          \
  if (per_thread)                                                                                                  \
    sl::sgram_reduce_thread_kernel<S_><<<rg, 256, 0, s>>>(t.g.gpart, k_, ksplit_, t.g.colexp, t.g.colexp2, out, ctl); \
  else                                                                                                             \
    sl::sgram_reduce_kernel<S_><<<rg, 256, 0, s>>>(t.g.gpart, k_, ksplit_, t.g.colexp, t.g.colexp2, out, ctl)
  EIGREF_SLICE_DISPATCH(slices_, EIGREF_CALL_SGR)
#undef EIGREF_CALL_SGR
  return 6;
}

int SlicedA::update(const double* X, const double* W, const double* FM, const double* d, const double* dinv,
                    double* Xn, double* upart, const Control* ctl, cudaStream_t s) {
  const SlicedLayout L = sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_);
  auto* xr = reinterpret_cast<__half*>(ws_ + L.xr_planes);
  auto* fp = reinterpret_cast<__half*>(ws_ + L.f_planes);
  int* xrexp = reinterpret_cast<int*>(ws_ + L.xr_rowexp);
  int* fexp = reinterpret_cast<int*>(ws_ + L.f_colexp);
  auto* fmax_ = reinterpret_cast<unsigned long long*>(ws_ + L.f_cmax);
  // FM is k x kfm column-major: element (l, c) at FM[l + c k]
  const int kfm = kfm_cols(k_);
  const bool fused = fused_max_;   // the [F | M] panel's maxima formed by the k x k stage
#define EIGREF_CALL_SLICE_UPD(S_)                                                                       \
  sl::launch_slice_rows<S_>(X, n_, k_, n_pad_, kr_, xr, xrexp, ctl, s);                                 \
  if (fused)                                                                                            \
    sl::launch_slice_cols_ready<S_>(FM, k_, kfm, 1, k_, kr_, kfm, fmax_, fp, fexp, ctl, s);             \
  else                                                                                                  \
    sl::launch_slice_cols<S_>(FM, k_, kfm, 1, k_, kr_, kfm, fmax_, fp, fexp, ctl, s)
  EIGREF_SLICE_DISPATCH(slices_, EIGREF_CALL_SLICE_UPD)
#undef EIGREF_CALL_SLICE_UPD
  const MmaTask t = update_task(X, W, d, dinv, Xn, upart, ctl);
  launch_task(slices_, sl::MODE_UPDATE, t, s);
  return 6;
}

// ---- grouped launches (a batch) ----
template <int MODE>
static void launch_mma_group(int S, const sl::GroupMma& p, int ctas, cudaStream_t s) {
#define EIGREF_CALL_MMA_G(S_) \
  sl::sliced_mma_grouped_kernel<S_, MODE><<<ctas, sl::threads_of(MODE), sl::smem_bytes(MODE), s>>>(p)
  EIGREF_SLICE_DISPATCH(S, EIGREF_CALL_MMA_G)
#undef EIGREF_CALL_MMA_G
}

void launch_mma_tasks(int S, int mode, const MmaTask* tasks, int count, cudaStream_t s, const cudaStream_t* side,
                      const cudaEvent_t* ev) {
  static sl::GroupMma p;   // host staging of the parameter block (copied at launch)
  const int groups = (count + sl::kGroupMax - 1) / sl::kGroupMax;
  // groups on side streams (forked from s, joined back): their tails overlap
  if (side) cudaEventRecord(ev[groups], s);
  for (int t0 = 0, gi = 0; t0 < count; t0 += sl::kGroupMax, ++gi) {
    const int nt = std::min(sl::kGroupMax, count - t0);
    cudaStream_t ls = s;
    if (side) {
      ls = side[gi];
      cudaStreamWaitEvent(ls, ev[groups], 0);
    }
    memset(&p, 0, sizeof(p));
    int ctas = 0;
    for (int i = 0; i < nt; ++i) {
      const MmaTask& t = tasks[t0 + i];
      p.tmA[i] = t.a;
      p.tmB[i] = t.b;
      p.tmB2[i] = t.b2;
      p.args[i] = t.g;
      p.gx[i] = t.gx;
      p.gy[i] = t.gy;
      p.cta_begin[i] = ctas;
      ctas += t.gx * t.gy * t.gz;
    }
    p.cta_begin[nt] = ctas;
    p.count = nt;
    if (mode == sl::MODE_PRODUCT) launch_mma_group<sl::MODE_PRODUCT>(S, p, ctas, ls);
    else if (mode == sl::MODE_GRAM) launch_mma_group<sl::MODE_GRAM>(S, p, ctas, ls);
    else launch_mma_group<sl::MODE_UPDATE>(S, p, ctas, ls);
    if (side) {
      cudaEventRecord(ev[gi], ls);
      cudaStreamWaitEvent(s, ev[gi], 0);
    }
  }
}

template <int S>
static void slice_grouped(int op, const GroupItem* items, const GroupDims& gd, int max_n_pad, int parity,
                          cudaStream_t s) {
  const int kp = (gd.max_k + 31) / 32;
  const int rpb = 256 / gd.max_k > 0 ? 256 / gd.max_k : 1;
  (void)rpb;
  switch (op) {
    case SLICE_ZERO_MAX:
      sl::zero_cmax_grouped_kernel<<<gd.count, 128, 0, s>>>(items);
      break;
    case SLICE_X_COLS:
      sl::colmax_grouped_kernel<sl::OPD_XCOLS><<<dim3(16, 1, gd.count), 256, 0, s>>>(items, parity);
      sl::slice_cols_grouped_kernel<S, sl::OPD_XCOLS><<<dim3(max_n_pad / 64, kp, gd.count), 256, 0, s>>>(items, parity);
      break;
    case SLICE_P_COLS:
      sl::colmax_grouped_kernel<sl::OPD_PCOLS><<<dim3(16, 1, gd.count), 256, 0, s>>>(items, parity);
      sl::slice_cols_grouped_kernel<S, sl::OPD_PCOLS><<<dim3(max_n_pad / 64, kp, gd.count), 256, 0, s>>>(items, parity);
      break;
    case SLICE_F_COLS: {
      const int kr = (gd.max_k + 63) / 64 * 64;
      sl::colmax_grouped_kernel<sl::OPD_FCOLS><<<dim3(1, 1, gd.count), 256, 0, s>>>(items, parity);
      sl::slice_cols_grouped_kernel<S, sl::OPD_FCOLS><<<dim3(kr / 64, kfm_cols(gd.max_k) / 32, gd.count), 256, 0, s>>>(
          items, parity);
      break;
    }
    default:
      sl::slice_rows_grouped_kernel<S><<<dim3(16, 1, gd.count), 256, 0, s>>>(items, parity);
      break;
  }
}

void launch_sgram_reduce_grouped(int S, const GroupItem* items, const GroupDims& gd, cudaStream_t s) {
  const int64_t warps = 2LL * gd.max_k * gd.max_k;
  const int rg = (int)std::min<int64_t>((warps + 7) / 8, 64);
#define EIGREF_CALL_SGRG(S_) sl::sgram_reduce_grouped_kernel<S_><<<dim3(rg, 1, gd.count), 256, 0, s>>>(items)
  EIGREF_SLICE_DISPATCH(S, EIGREF_CALL_SGRG)
#undef EIGREF_CALL_SGRG
}

void launch_slice_grouped(int S, int op, const GroupItem* items, const GroupDims& gd, int max_n_pad, int parity,
                          cudaStream_t s) {
#define EIGREF_CALL_SLICE_G(S_) slice_grouped<S_>(op, items, gd, max_n_pad, parity, s)
  EIGREF_SLICE_DISPATCH(S, EIGREF_CALL_SLICE_G)
#undef EIGREF_CALL_SLICE_G
}

int SlicedA::update_grid() const { return n_pad_ / sl::kBM; }

int SlicedA::timed_out(cudaStream_t s) const {
  const SlicedLayout L = sliced_layout(n_pad_, k_pad_, kr_, slices_, ksplit_max_, k_, pslots_, n_);
  int v = 0;
  cudaMemcpyAsync(&v, ws_ + L.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return v;
}

// ---------------------------------------------------------------------------
// SlicedGram: the tensor-core Gram products for k <= 16 without A (CSR).
// ---------------------------------------------------------------------------
struct Gram16Layout {
  size_t x_planes, x_colexp, x_cmax, p_planes, p_colexp, p_cmax, part, err, total;
};

static Gram16Layout gram16_layout(int64_t n_pad, int S, int ksplit, int k) {
  Gram16Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 1023) & ~size_t(1023);
    size_t o = off;
    off += bytes;
    return o;
  };
  L.x_planes = take((size_t)S * 16 * n_pad * 2);
  L.x_colexp = take(16 * 4);
  L.x_cmax = take(16 * 8);
  L.p_planes = take((size_t)S * 16 * n_pad * 2);
  L.p_colexp = take(16 * 4);
  L.p_cmax = take(16 * 8);
  L.part = take((size_t)2 * ksplit * k * k * 16);
  L.err = take(64);
  L.total = off + 1024;
  return L;
}

int SlicedGram::configure(int64_t n, int k, int slices) {
  n_ = n;
  k_ = k;
  slices_ = slices > 0 ? slices : sl::kDefaultS;
  if (k < 1 || k > 16) {
    snprintf(err_, sizeof(err_), "tensor-core Gram products for CSR need k <= 16 (k = %d)", k);
    return EIGREF_E_UNSUPPORTED;
  }
  if (slices_ < 2 || slices_ > sl::kMaxS) {
    snprintf(err_, sizeof(err_), "slices must be in [2, %d]", sl::kMaxS);
    return EIGREF_E_INVALID;
  }
  if (!sl::encode_fn()) {
    snprintf(err_, sizeof(err_), "cuTensorMapEncodeTiled unavailable");
    return EIGREF_E_CUDA;
  }
  n_pad_ = (n + 255) / 256 * 256;
  const int64_t kbt = n_pad_ / sl::kBK;
  // one CTA per SM, and at most 3500 K blocks per CTA (its int64 sums stay exact)
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  ksplit_ = (int)std::min<int64_t>(kbt, sms);
  while (kbt / ksplit_ > 3500) ksplit_ += sms;
  // the row update on the tensor cores: even k (16-byte rows for TMA), one
  // CTA per SM or per 128-row tile
  upd_grid_ = (int)std::min<int64_t>((n + 127) / 128, sms);
  upd_ok_ = false;
  if (k % 2 == 0) {
    alignas(64) CUtensorMap probe;
    const void* aligned = reinterpret_cast<const void*>(uintptr_t(1) << 20);
    upd_ok_ = sl::make_map_f64(&probe, aligned, k, n, 128) && sl::make_map_f64(&probe, aligned, k, n, 32);
  }
  return EIGREF_OK;
}

int SlicedGram::update(const double* X, const double* W, const double* F, const double* M, const double* d,
                       const double* dinv, double* Xn, double* upart, const Control* ctl, cudaStream_t s) {
  if (!upd_ok_) return -1;
  alignas(64) CUtensorMap mx, mw, mn;
  if (!sl::make_map_f64(&mx, X, k_, n_, 128) || !sl::make_map_f64(&mw, W, k_, n_, 128) ||
      !sl::make_map_f64(&mn, Xn, k_, n_, 32))
    return -1;
  const Gram16Layout L = gram16_layout(n_pad_, slices_, ksplit_, k_);
  sl::Upd16Args a;
  a.n = n_;
  a.k = k_;
  a.row_begin = k_;
  a.tiles = (int)((n_ + 127) / 128);
  a.F = F;
  a.M = M;
  a.d = d;
  a.dinv = dinv;
  a.Xn = Xn;
  a.upart = upart;
  a.ctl = ctl;
  a.err = reinterpret_cast<int*>(ws_ + L.err);
  a.wait_ns = wait_ns_;
#define EIGREF_CALL_U16(S_) sl::update16_kernel<S_><<<upd_grid_, sl::kU16Threads, sl::kU16Smem, s>>>(mx, mw, mn, a)
  EIGREF_SLICE_DISPATCH(slices_, EIGREF_CALL_U16)
#undef EIGREF_CALL_U16
  return 1;
}

size_t SlicedGram::workspace_bytes() const { return gram16_layout(n_pad_, slices_, ksplit_, k_).total; }

void SlicedGram::bind_workspace(char* p) {
  ws_ = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

int SlicedGram::prepare(cudaStream_t s) {
  const Gram16Layout L = gram16_layout(n_pad_, slices_, ksplit_, k_);
  if (cudaMemsetAsync(ws_ + L.x_planes, 0, L.part - L.x_planes, s) != cudaSuccess ||
      cudaMemsetAsync(ws_ + L.err, 0, 64, s) != cudaSuccess) {
    snprintf(err_, sizeof(err_), "memset of slice planes failed");
    return EIGREF_E_CUDA;
  }
  const uint64_t rows = (uint64_t)slices_ * 16;
  bool ok = sl::make_map(reinterpret_cast<CUtensorMap*>(tmX_), ws_ + L.x_planes, (uint64_t)n_pad_, rows, sl::kBK,
                         (uint32_t)rows);
  ok = ok && sl::make_map(reinterpret_cast<CUtensorMap*>(tmP_), ws_ + L.p_planes, (uint64_t)n_pad_, rows, sl::kBK,
                          (uint32_t)rows);
  if (!ok) {
    snprintf(err_, sizeof(err_), "tensor map encoding failed");
    return EIGREF_E_CUDA;
  }
  return EIGREF_OK;
}

// Even k: the fused kernel (planes cut in shared memory) from the column
// maxima in x_cmax() / p_cmax(), then the reduction.  Returns the launch
// count, or -1 when the operands cannot be mapped (then the plane path runs).
int SlicedGram::gram_fused(const double* X, const double* P, double* out, const Control* ctl, cudaStream_t s) {
  if (!upd_ok_) return -1;
  alignas(64) CUtensorMap mx, mp;
  if (!sl::make_map_f64(&mx, X, k_, n_, 64) || !sl::make_map_f64(&mp, P, k_, n_, 64)) return -1;
  const Gram16Layout L = gram16_layout(n_pad_, slices_, ksplit_, k_);
  int* xexp = reinterpret_cast<int*>(ws_ + L.x_colexp);
  int* pexp = reinterpret_cast<int*>(ws_ + L.p_colexp);
  sl::Gram16FArgs fa;
  fa.g.kb_total = (int)((n_ + sl::kBK - 1) / sl::kBK);
  fa.g.ksplit = ksplit_;
  fa.g.k = k_;
  fa.g.part = reinterpret_cast<longlong2*>(ws_ + L.part);
  fa.g.ctl = ctl;
  fa.g.err = reinterpret_cast<int*>(ws_ + L.err);
  fa.g.wait_ns = wait_ns_;
  fa.xmax = x_cmax();
  fa.wmax = p_cmax();
  fa.xexp = xexp;
  fa.wexp = pexp;
  const int rg = (int)std::min<int64_t>((2LL * k_ * k_ + 7) / 8, 152 * 8);
#define EIGREF_CALL_G16F(S_)                                                                                     \
  sl::sgram16f_kernel<S_><<<ksplit_, sl::kThreads, sl::kG16FSmem, s>>>(mx, mp, fa);                               \
  sl::sgram16_reduce_kernel<S_><<<rg, 256, 0, s>>>(fa.g.part, k_, ksplit_, xexp, pexp, out, ctl)
  EIGREF_SLICE_DISPATCH(slices_, EIGREF_CALL_G16F)
#undef EIGREF_CALL_G16F
  return 2;
}

int SlicedGram::gram(const double* X, const double* P, double* out, const Control* ctl, cudaStream_t s) {
  if (upd_ok_) {
    // column maxima, then the fused kernel
    cudaMemsetAsync(x_cmax(), 0, (size_t)k_ * 8, s);
    cudaMemsetAsync(p_cmax(), 0, (size_t)k_ * 8, s);
    sl::launch_colmax_rowmajor(X, n_, k_, x_cmax(), ctl, s);
    sl::launch_colmax_rowmajor(P, n_, k_, p_cmax(), ctl, s);
    const int nl = gram_fused(X, P, out, ctl, s);
    if (nl > 0) return nl + 2;
  }
  const Gram16Layout L = gram16_layout(n_pad_, slices_, ksplit_, k_);
  auto* xp = reinterpret_cast<__half*>(ws_ + L.x_planes);
  auto* pp = reinterpret_cast<__half*>(ws_ + L.p_planes);
  auto* xmax = reinterpret_cast<unsigned long long*>(ws_ + L.x_cmax);
  auto* pmax = reinterpret_cast<unsigned long long*>(ws_ + L.p_cmax);
  int* xexp = reinterpret_cast<int*>(ws_ + L.x_colexp);
  int* pexp = reinterpret_cast<int*>(ws_ + L.p_colexp);
  const int K = (int)n_pad_;
  sl::Gram16Args g;
  g.kb_total = (int)(n_pad_ / sl::kBK);
  g.ksplit = ksplit_;
  g.k = k_;
  g.part = reinterpret_cast<longlong2*>(ws_ + L.part);
  g.ctl = ctl;
  g.err = reinterpret_cast<int*>(ws_ + L.err);
  g.wait_ns = wait_ns_;
  const CUtensorMap& mx = *reinterpret_cast<const CUtensorMap*>(tmX_);
  const CUtensorMap& mp = *reinterpret_cast<const CUtensorMap*>(tmP_);
  const int rg = (int)std::min<int64_t>((2LL * k_ * k_ + 7) / 8, 152 * 8);
#define EIGREF_CALL_G16(S_)                                                                                      \
  sl::launch_slice_cols16<S_>(X, n_, k_, K, xmax, xp, xexp, ctl, s);                                           \
  sl::launch_slice_cols16<S_>(P, n_, k_, K, pmax, pp, pexp, ctl, s);                                           \
  sl::sgram16_kernel<S_><<<ksplit_, sl::kThreads, sl::kG16Smem, s>>>(mx, mp, g);                                 \
  sl::sgram16_reduce_kernel<S_><<<rg, 256, 0, s>>>(g.part, k_, ksplit_, xexp, pexp, out, ctl)
  EIGREF_SLICE_DISPATCH(slices_, EIGREF_CALL_G16)
#undef EIGREF_CALL_G16
  return 6;
}

unsigned long long* SlicedGram::x_cmax() const {
  return reinterpret_cast<unsigned long long*>(ws_ + gram16_layout(n_pad_, slices_, ksplit_, k_).x_cmax);
}

unsigned long long* SlicedGram::p_cmax() const {
  return reinterpret_cast<unsigned long long*>(ws_ + gram16_layout(n_pad_, slices_, ksplit_, k_).p_cmax);
}

void SlicedGram::colmax_x(const double* X, cudaStream_t s) {
  cudaMemsetAsync(x_cmax(), 0, (size_t)k_ * 8, s);
  sl::launch_colmax_rowmajor(X, n_, k_, x_cmax(), nullptr, s);
}

int SlicedGram::gram_ready(const double* X, const double* P, double* out, const Control* ctl, cudaStream_t s) {
  {
    const int nl = gram_fused(X, P, out, ctl, s);
    if (nl > 0) {
      // the maxima are read: clear them for the kernels that form the next ones
      cudaMemsetAsync(x_cmax(), 0, (size_t)k_ * 8, s);
      cudaMemsetAsync(p_cmax(), 0, (size_t)k_ * 8, s);
      return nl;
    }
  }
  const Gram16Layout L = gram16_layout(n_pad_, slices_, ksplit_, k_);
  auto* xp = reinterpret_cast<__half*>(ws_ + L.x_planes);
  auto* pp = reinterpret_cast<__half*>(ws_ + L.p_planes);
  int* xexp = reinterpret_cast<int*>(ws_ + L.x_colexp);
  int* pexp = reinterpret_cast<int*>(ws_ + L.p_colexp);
  const int K = (int)n_pad_;
  sl::Gram16Args g;
  g.kb_total = (int)(n_pad_ / sl::kBK);
  g.ksplit = ksplit_;
  g.k = k_;
  g.part = reinterpret_cast<longlong2*>(ws_ + L.part);
  g.ctl = ctl;
  g.err = reinterpret_cast<int*>(ws_ + L.err);
  g.wait_ns = wait_ns_;
  const CUtensorMap& mx = *reinterpret_cast<const CUtensorMap*>(tmX_);
  const CUtensorMap& mp = *reinterpret_cast<const CUtensorMap*>(tmP_);
  const int rg = (int)std::min<int64_t>((2LL * k_ * k_ + 7) / 8, 152 * 8);
  // the maxima come from the kernels that wrote X and P; once sliced, they are
  // cleared for those kernels' next run (both arrays are k entries, adjacent layout not assumed)
#define EIGREF_CALL_G16R(S_)                                                                                     \
  sl::slice_cols16_kernel<S_><<<K / 128, 256, 0, s>>>(X, n_, k_, k_, 1, K, x_cmax(), xp, xexp, ctl);            \
  sl::slice_cols16_kernel<S_><<<K / 128, 256, 0, s>>>(P, n_, k_, k_, 1, K, p_cmax(), pp, pexp, ctl);            \
  cudaMemsetAsync(x_cmax(), 0, (size_t)k_ * 8, s);                                                              \
  cudaMemsetAsync(p_cmax(), 0, (size_t)k_ * 8, s);                                                              \
  sl::sgram16_kernel<S_><<<ksplit_, sl::kThreads, sl::kG16Smem, s>>>(mx, mp, g);                                 \
  sl::sgram16_reduce_kernel<S_><<<rg, 256, 0, s>>>(g.part, k_, ksplit_, xexp, pexp, out, ctl)
  EIGREF_SLICE_DISPATCH(slices_, EIGREF_CALL_G16R)
#undef EIGREF_CALL_G16R
  return 4;
}

int SlicedGram::timed_out(cudaStream_t s) const {
  const Gram16Layout L = gram16_layout(n_pad_, slices_, ksplit_, k_);
  int v = 0;
  cudaMemcpyAsync(&v, ws_ + L.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return v;
}

double SlicedA::executed_flops() const {
  const double pairs = slices_ * (slices_ + 1) / 2.0;
  return 2.0 * (double)n_pad_ * (double)n_pad_ * (double)k_pad_ * pairs;
}

}  // namespace eigref
