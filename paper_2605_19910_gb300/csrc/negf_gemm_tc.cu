// Split-precision complex block products on the 5th-generation tensor cores.
//
// Used by the mixed-precision sweep for every block product of Alg. 1 /
// Sec. 2.3 (the multipliers, the Schur update and the downward products);
// the per-block inversions stay in FP64 (negf_inv.cu).
//
// Complex -> real.  C = A B is one real product with the real and imaginary
// parts stacked along M and K,
//
//     [Re C]   [Re A  -Im A] [Re B]
//     [Im C] = [Im A   Re A] [Im B],
//
// so 64 complex rows of C form one M = 128 tcgen05 tile.
//
// BF16 split with exact FP32 sums.  Each complex row r of A gets a power-of-two
// scale 2^e_r above all its entries, each column c of B a scale 2^e_c.  An
// entry x = 2^e_r * sum_l a_l 2^{-s(l+1)} is cut into L integer slices
// |a_l| < 2^s (s = 8 bits, or 7 when K is long) that BF16 holds exactly.
// A slice product is an integer below 2^{2s}; summed over K it stays below
// 2^24, so the FP32 accumulation in tensor memory is exact.  The products
// a_l b_m with l + m = d accumulate into TMEM accumulator d (levels
// d = 0..L-1; deeper levels are dropped), and the epilogue combines the
// levels exactly in 64-bit integers:
//     C = 2^{e_r + e_c - s(L+1)} sum_d acc_d 2^{s(L-1-d)}.
// The result carries about s*L = 32 significant bits relative to the row and
// column scales.
//
// No FP64 instruction: GB300's FP64 pipe is the scarce resource of the whole
// sweep (it runs the block inversions), so the slicing of FP64 inputs, the
// level combination, the conversion to FP64 and the additions of the
// epilogue (beta * C1, the diagonal shift E) are done with integer
// operations on the IEEE bit patterns.
//
// One CTA computes a 64 x N complex tile of one batch entry (N <= 512 / L
// TMEM columns per level); K streams through shared memory in chunks of 32
// complex columns.  Operands use the K-major, non-swizzled canonical layout
// (8-row x 16-byte core matrices).  One thread issues the MMAs; completion is
// tracked with an mbarrier whose wait is bounded.
#include <algorithm>
#include <type_traits>

#include "negf_common.cuh"
#include "negf_kernels.h"

namespace negf {

cudaError_t zinv_init();

namespace {

constexpr int TC_THREADS = 256;             // two warpgroups
constexpr int MC = 64;                       // complex rows per CTA (M = 128 real)
constexpr int CORE = 128;                    // 8 rows x 16 bytes
constexpr int LBO = CORE;                    // bytes between 16-byte K groups

// K-chunk geometry: KC complex K per chunk.  (Half-size chunks for the long
// products, to fit more CTAs per SM, measured 3-10 % slower: the extra chunk
// iterations cost more than the occupancy gained.)
template <int KC_>
struct Chunk {
  static constexpr int KC = KC_;
  static constexpr int KG = KC / 8;                  // 8-element K groups per chunk and part
  static constexpr int KR = 2 * KC;                  // real K per chunk (BF16 elements per row)
  static constexpr int SBO = (KR / 8) * CORE;        // bytes between 8-row groups
  static constexpr int A_SLICE_BYTES = 128 * KR * 2; // one slice of the A chunk
};
constexpr long long WAIT_LIMIT = 1ll << 26;  // bounded mbarrier wait
constexpr int ZERO_EXP = 0;                  // scale exponent of an all-zero row / column

struct TcCfg {
  int s;        // slice bits
  int L;        // slices (= accumulator levels)
  int n_mma;    // MMA N (complex columns per tile)
  int tmem_cols;
  int ep;       // epilogue pass width (columns)
};

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

template <class CK>
__device__ __forceinline__ uint32_t kmaj_off(int row, int kcol) {   // BF16 element
  return (uint32_t)((row >> 3) * CK::SBO + (kcol >> 3) * LBO + (row & 7) * 16 + (kcol & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// IEEE doubles are handled as 64-bit integer bit patterns throughout this
// kernel, so that no instruction of GB300's scarce FP64 pipe is issued
// (a sign flip on a double-typed value may compile to an FP64 negation).
typedef unsigned long long u64;

// e such that |x| < 2^e, from the biased exponent; zero/denormal -> very small
__device__ __forceinline__ int exp_bound(u64 u) {
  const int be = (int)((u >> 52) & 0x7FF);
  return be == 0 ? -100000 : be - 1022;
}

// |x| * 2^(frac_bits - e_scale) as an unsigned integer (truncated), |x| < 2^e_scale.
__device__ __forceinline__ u64 fixed_abs(u64 u, int e_scale, int frac_bits) {
  const int be = (int)((u >> 52) & 0x7FF);
  if (be == 0) return 0;
  const u64 m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = be - 1075 + frac_bits - e_scale;     // value = m * 2^(be-1075); sh <= frac - 53 < 0
  if (sh >= 0) return m << (sh > 10 ? 10 : sh);       // not reached for |x| < 2^e_scale
  if (sh <= -64) return 0;
  return m >> (-sh);
}

// |x| * 2^(frac_bits - e_scale) truncated, for frac_bits <= 32: the result
// fits 32 bits.  With |x| < 2^e_scale the right shift of the 53-bit mantissa
// is k = 1075 - be - frac_bits + e_scale >= 21.
__device__ __forceinline__ uint32_t fixed32(u64 u, int e_scale, int frac_bits) {
  const int be = (int)((u >> 52) & 0x7FF);
  const int k = 1075 - be - frac_bits + e_scale;
  const uint32_t lo = (uint32_t)u, hi = ((uint32_t)(u >> 32) & 0xFFFFFu) | 0x100000u;
  if (be == 0 || k >= 53) return 0u;
  return k >= 32 ? hi >> (k - 32) : __funnelshift_r(lo, hi, k);
}

// FP32 bits of the small integer in byte `bidx` of x (2^23 + byte - 2^23, exact):
// one byte permute builds 0x4B0000bb, one FP32 subtraction gives the value.
template <int BIDX>
__device__ __forceinline__ uint32_t f32_of_byte(uint32_t x) {
  return __float_as_uint(__uint_as_float(__byte_perm(x, 0x4B000000u, 0x7440u | BIDX)) - 8388608.0f);
}
__device__ __forceinline__ uint32_t f32_of_byte_rt(uint32_t x, int bidx) {
  return __float_as_uint(__uint_as_float(__byte_perm(x, 0x4B000000u, 0x7440u | (uint32_t)bidx)) - 8388608.0f);
}
// FP32 bits of the s-bit field at bit `sh` of the 64-bit value (hi:lo).
__device__ __forceinline__ uint32_t f32_of_field(uint32_t lo, uint32_t hi, int sh, uint32_t mask) {
  const uint32_t v = sh >= 32 ? hi >> (sh - 32) : __funnelshift_r(lo, hi, sh);
  return __float_as_uint(__uint_as_float((v & mask) | 0x4B000000u) - 8388608.0f);
}
// Two FP32 integers -> one word of two BF16 (their high halves), with signs.
__device__ __forceinline__ uint32_t pack_bf16x2(uint32_t f0, uint32_t f1, uint32_t signs) {
  return __byte_perm(f0, f1, 0x7632u) | signs;
}

// T += (-1)^neg * x exactly on the integer grid of unit 2^E (x: FP64 bits),
// truncating the bits of x below 2^E (below the product's own resolution).
// Returns false where the integer grid cannot hold the sum (x more than
// 2^DMAX units above the grid's range, or a non-finite x): the caller then
// adds in floating point.
template <class Acc, int DMAX>
__device__ __forceinline__ bool grid_add(Acc& T, u64 x, bool neg, int E) {
  const int be = (int)((x >> 52) & 0x7FF);
  if (be == 0) return true;                          // zero (or a negligible denormal)
  if (be == 0x7FF) return false;
  const u64 m = (x & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int d = be - 1075 - E;
  if (d > DMAX) return false;
  Acc v = d >= 0 ? ((Acc)m << d) : (d > -64 ? (Acc)(m >> (-d)) : (Acc)0);
  if (((x >> 63) != 0) != neg) v = -v;
  T += v;
  return true;
}

// Signed 64-bit integer T times 2^e2 as IEEE double bits (round to nearest even)
__device__ __forceinline__ u64 i64_scaled_bits(long long T, int e2) {
  if (T == 0) return 0ull;
  const u64 sgn = T < 0 ? 1ull : 0ull;
  u64 u = T < 0 ? (u64)(-T) : (u64)T;
  const int lz = __clzll((long long)u);
  u <<= lz;                                   // leading one at bit 63
  int e = 63 - lz + e2;
  u64 m = u >> 11;                            // 53 bits with the leading one
  const u64 rem = u & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (m & 1ull))) {
    m += 1;
    if (m >> 53) { m >>= 1; e += 1; }
  }
  const int be = e + 1023;
  if (be <= 0) return sgn << 63;
  if (be >= 2047) return (sgn << 63) | (0x7FFull << 52);
  return (sgn << 63) | ((u64)be << 52) | (m & 0xFFFFFFFFFFFFFull);
}

// Signed 128-bit integer T times 2^e2 as IEEE double bits (round to nearest even)
__device__ __forceinline__ u64 i128_scaled_bits(__int128 T, int e2) {
  if (T == 0) return 0ull;
  const u64 sgn = T < 0 ? 1ull : 0ull;
  unsigned __int128 u = T < 0 ? (unsigned __int128)(-T) : (unsigned __int128)T;
  const u64 hi = (u64)(u >> 64), lo = (u64)u;
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  u <<= lz;                                   // leading one at bit 127
  int e = 127 - lz + e2;
  u64 m = (u64)(u >> 75);                     // 53 bits with the leading one
  const unsigned __int128 rem = u & (((unsigned __int128)1 << 75) - 1);
  const unsigned __int128 half = (unsigned __int128)1 << 74;
  if (rem > half || (rem == half && (m & 1ull))) {
    m += 1;
    if (m >> 53) { m >>= 1; e += 1; }
  }
  const int be = e + 1023;
  if (be <= 0) return sgn << 63;
  if (be >= 2047) return (sgn << 63) | (0x7FFull << 52);
  return (sgn << 63) | ((u64)be << 52) | (m & 0xFFFFFFFFFFFFFull);
}

// a + b on IEEE double bit patterns with integer operations (round to nearest).
// Zeros and normals are handled, denormal results flush to zero; non-finite
// operands (never produced by the sweep) propagate as NaN.
__device__ __forceinline__ u64 add_bits(u64 ua, u64 ub) {
  const u64 ABS = 0x7FFFFFFFFFFFFFFFull;
  if ((ub & ABS) == 0) return ua;
  if ((ua & ABS) == 0) return ub;
  int ea = (int)((ua >> 52) & 0x7FF), eb = (int)((ub >> 52) & 0x7FF);
  if (ea == 0x7FF || eb == 0x7FF) return 0x7FF8000000000000ull;
  if ((ua & ABS) < (ub & ABS)) {
    u64 t = ua; ua = ub; ub = t;
    int te = ea; ea = eb; eb = te;
  }
  if (ea == 0) return ua;                     // both denormal: negligible here
  const u64 sa = ua >> 63, sb = ub >> 63;
  const u64 ma = ((ua & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 9;   // leading one at bit 61
  u64 mb = eb == 0 ? 0 : ((ub & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 9;
  const int d = ea - eb;
  if (d >= 62) mb = mb ? 1 : 0;
  else if (d > 0) mb = (mb >> d) | ((mb & ((1ull << d) - 1)) ? 1ull : 0ull);
  u64 m = (sa == sb) ? ma + mb : ma - mb;
  if (m == 0) return 0ull;
  int e = ea;
  const int lz = __clzll((long long)m);
  if (lz == 1) {                          // carry into bit 62
    m = (m >> 1) | (m & 1ull);
    e += 1;
  } else if (lz > 2) {
    m <<= (lz - 2);
    e -= (lz - 2);
  }
  const u64 rem = m & 0x1FFull;
  m >>= 9;
  if (rem > 0x100ull || (rem == 0x100ull && (m & 1ull))) {
    m += 1;
    if (m >> 53) { m >>= 1; e += 1; }
  }
  if (e <= 0) return sa << 63;
  if (e >= 2047) return (sa << 63) | (0x7FFull << 52);
  return (sa << 63) | ((u64)e << 52) | (m & 0xFFFFFFFFFFFFFull);
}

__device__ __forceinline__ u64 flip(u64 x, bool neg) { return neg ? (x ^ 0x8000000000000000ull) : x; }

__device__ __forceinline__ ulonglong2 ld_bits(const double2* p) {
  return *reinterpret_cast<const ulonglong2*>(p);
}

// element offset of op(B)(k, c): B[k][c], or B[c][k] (to be conjugated) for B^H
template <bool BC>
__device__ __forceinline__ int64_t opb_off(const ZGemm& g, int k, int c) {
  return BC ? (int64_t)c * g.ldb + k : (int64_t)k * g.ldb + c;
}

// tcgen05 shared-memory matrix descriptor: start, LBO (K), SBO (M/N), version 1, no swizzle.
template <class CK>
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((CK::SBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 accumulate
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit = WAIT_LIMIT) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
}


// exact integer value of an FP32 accumulator: every accumulator holds an
// integer (sums of integer slice products; above 2^24 FP32 values are
// integers too) of magnitude below 2^31, so the round-to-nearest conversion
// is exact; it runs on the conversion path (not the FP64 pipe), about 4x the
// rate of extracting the value from the bit pattern with integer operations
__device__ __forceinline__ long long acc_int(uint32_t bits) {
  return (long long)__float2int_rn(__uint_as_float(bits));
}

// Slices of 8 consecutive K values of one operand row (A) or column (B):
// for each slice l, 4 words of two BF16 digits with the values' signs.
// S8: 8-bit slices of a 32-bit fixed-point value (a byte permute per digit);
// otherwise s-bit fields of a 64-bit fixed-point value (a funnel shift per
// digit).
template <bool S8>
struct Digits8 {
  uint32_t lo[8], hi[8];
  uint32_t sw[4];   // BF16 sign bits of each pair of values (bits 15 and 31)
  __device__ __forceinline__ void load(const u64* v, int e_scale, int frac) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (S8) {
        lo[j] = fixed32(v[j], e_scale, frac);
        hi[j] = 0u;
      } else {
        const u64 f = fixed_abs(v[j], e_scale, frac);
        lo[j] = (uint32_t)f;
        hi[j] = (uint32_t)(f >> 32);
      }
    }
#pragma unroll
    for (int h = 0; h < 4; ++h)
      sw[h] = ((uint32_t)(v[2 * h] >> 48) & 0x8000u) | ((uint32_t)(v[2 * h + 1] >> 32) & 0x80000000u);
  }
  // digit l (0 = most significant) of all 8 values as 4 packed words
  __device__ __forceinline__ void slice(int l, int s, int L, uint32_t smask, uint32_t* out) const {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      uint32_t f0, f1;
      if (S8) {
        f0 = f32_of_byte_rt(lo[2 * h], L - 1 - l);
        f1 = f32_of_byte_rt(lo[2 * h + 1], L - 1 - l);
      } else {
        const int sh = s * (L - 1 - l);
        f0 = f32_of_field(lo[2 * h], hi[2 * h], sh, smask);
        f1 = f32_of_field(lo[2 * h + 1], hi[2 * h + 1], sh, smask);
      }
      out[h] = pack_bf16x2(f0, f1, sw[h]);
    }
  }
};

// S8: 8-bit slices of products up to 32 bits.  WIDE: products longer than
// the 64-bit level combination allows.  BC: op(B) = B^H.  Register caps
// follow the CTAs per SM that the operands' shared memory allows anyway:
// four for S8 (4 slices), three for 5-6 slices, two for WIDE (7-8).
template <bool S8, bool WIDE, bool BC>
__global__ void __launch_bounds__(TC_THREADS, S8 ? 4 : (WIDE ? 2 : 3)) zgemm_tc_kernel(ZGemm g, int tiles_n, TcCfg cfg) {
  using CK = Chunk<16>;
  using Acc = typename std::conditional<WIDE, __int128, long long>::type;
  constexpr int KC = CK::KC, KG = CK::KG, KR = CK::KR, A_SLICE_BYTES = CK::A_SLICE_BYTES;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int e_row[MC];
  __shared__ int e_col[256];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int L = cfg.L, s = cfg.s, n_mma = cfg.n_mma;
  const int tile = blockIdx.x;
  const int m0 = (tile / tiles_n) * MC;
  const int n0 = (tile % tiles_n) * n_mma;
  const int e = blockIdx.y;
  const int mt = min(MC, g.m - m0);
  const int nt = min(n_mma, g.n - n0);
  const int b_slice_bytes = n_mma * KR * 2;
  unsigned char* sA = smem;                                   // L slices of A
  unsigned char* sB = smem + (size_t)L * A_SLICE_BYTES;       // L slices of B^T

  const double2* A = g.A + (int64_t)e * g.sA;
  const double2* B = g.B + (int64_t)e * g.sB;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  // Pass 1: power-of-two scales of the rows of A (warps 0-3) and of the
  // columns of B (warps 4-7), concurrently, with eight loads in flight per
  // thread (the scan is bound by load latency, not by its arithmetic).
  for (int c = tid; c < n_mma; c += TC_THREADS) e_col[c] = -100000;
  __syncthreads();
  if (warp < 4) {
    // row tid / 2 of A, every other K from tid % 2 (two threads per row)
    const int r = tid >> 1, hh = tid & 1;
    int mx = -100000;
    if (m0 + r < g.m) {
      const double2* row = A + (int64_t)(m0 + r) * g.lda;
      for (int k0 = hh; k0 < g.k; k0 += 16) {
        ulonglong2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = k0 + 2 * u;
          v[u] = k < g.k ? ld_bits(row + k) : make_ulonglong2(0ull, 0ull);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) mx = max(mx, max(exp_bound(v[u].x), exp_bound(v[u].y)));
      }
    }
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    if (hh == 0) e_row[r] = mx < -50000 ? ZERO_EXP : mx;
  } else if (nt > 0) {
    // columns of B: thread t scans column t % nt over every (128 / nt)-th K
    // (coalesced over columns; columns t, t + 128, ... over all K when
    // nt >= 128) and publishes one running maximum per column
    const int t = tid - 128, per = nt >= 128 ? 1 : 128 / nt;
    const int kk = nt >= 128 ? 0 : t / nt;
    if (kk < per)
      for (int c = nt >= 128 ? t : t % nt; c < nt; c += 128) {
        int mx = -100000;
        for (int k0 = kk; k0 < g.k; k0 += 8 * per) {
          // op(B)(k, c) at B + k sbk + c sbc (op(B) = B^H: the strides swap;
          // the sign of the imaginary part does not matter here)
          ulonglong2 v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int k = k0 + u * per;
            v[u] = k < g.k ? ld_bits(B + opb_off<BC>(g, k, n0 + c)) : make_ulonglong2(0ull, 0ull);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) mx = max(mx, max(exp_bound(v[u].x), exp_bound(v[u].y)));
        }
        atomicMax(&e_col[c], mx);
        if (nt < 128) break;
      }
  }
  __syncthreads();
  for (int c = tid; c < n_mma; c += TC_THREADS)
    if (e_col[c] < -50000) e_col[c] = ZERO_EXP;
  __syncthreads();
  uint32_t tmem_d = 0;
  const uint32_t mb = smem_u32(&mbar);
  const int frac = s * L;
  const uint32_t smask = (1u << s) - 1u;
  bool ok = true;
  uint32_t last_parity = 0;

  const int nchunks = (g.k + KC - 1) / KC;
  // Pass 2: slices of A and of B^T, 8 consecutive K per thread item, one
  // 16-byte core-matrix row per store; A and B concurrently on the two
  // halves of the CTA (threads 0-127 slice A, 128-255 slice B).
  const int half_t = TC_THREADS / 2;
  const bool isA = tid < half_t;
  const int item0 = isA ? tid : tid - half_t;
  const int n_items = isA ? MC * KG : n_mma * KG;
  // the raw values of an item: A row r (real and imaginary parts of 8
  // consecutive K), or column c of op(B)
  auto load_item = [&](int item, int k0, u64* vre, u64* vim) {
    if (isA) {
      const int r = item / KG, kg = item % KG, gr = m0 + r;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int gk = k0 + kg * 8 + j;
        ulonglong2 v = make_ulonglong2(0ull, 0ull);
        if (gr < g.m && gk < g.k) v = ld_bits(A + (int64_t)gr * g.lda + gk);
        vre[j] = v.x;
        vim[j] = v.y;
      }
    } else {
      const int c = item % n_mma, kg = item / n_mma;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int gk = k0 + kg * 8 + j;
        ulonglong2 v = make_ulonglong2(0ull, 0ull);
        if (gk < g.k && c < nt) {   // op(B) = B^H: conj by the imaginary sign bit
          v = ld_bits(B + opb_off<BC>(g, gk, n0 + c));
          if (BC) v.y ^= 0x8000000000000000ull;
        }
        vre[j] = v.x;
        vim[j] = v.y;
      }
    }
  };
  auto slice_item = [&](int item, const u64* vre, const u64* vim, unsigned char* dst) {
    if (isA) {
      // A: row r holds [Re A | -Im A], row 64 + r holds [Im A | Re A].
      const int r = item / KG, kg = item % KG;
      Digits8<S8> dre, dim;
      dre.load(vre, e_row[r], frac);
      dim.load(vim, e_row[r], frac);
      for (int l = 0; l < L; ++l) {
        uint32_t pr[4], pi[4];
        dre.slice(l, s, L, smask, pr);
        dim.slice(l, s, L, smask, pi);
        unsigned char* base = dst + (size_t)l * A_SLICE_BYTES;
        const uint4 vr = make_uint4(pr[0], pr[1], pr[2], pr[3]);
        const uint4 vi = make_uint4(pi[0], pi[1], pi[2], pi[3]);
        const uint4 vn = make_uint4(pi[0] ^ 0x80008000u, pi[1] ^ 0x80008000u, pi[2] ^ 0x80008000u,
                                    pi[3] ^ 0x80008000u);
        *reinterpret_cast<uint4*>(base + kmaj_off<CK>(r, kg * 8)) = vr;
        *reinterpret_cast<uint4*>(base + kmaj_off<CK>(r, KC + kg * 8)) = vn;
        *reinterpret_cast<uint4*>(base + kmaj_off<CK>(MC + r, kg * 8)) = vi;
        *reinterpret_cast<uint4*>(base + kmaj_off<CK>(MC + r, KC + kg * 8)) = vr;
      }
    } else {
      // B^T (K-major): row c holds [Re B(:, c) | Im B(:, c)].
      const int c = item % n_mma, kg = item / n_mma;
      Digits8<S8> dre, dim;
      dre.load(vre, e_col[c], frac);
      dim.load(vim, e_col[c], frac);
      for (int l = 0; l < L; ++l) {
        uint32_t pr[4], pi[4];
        dre.slice(l, s, L, smask, pr);
        dim.slice(l, s, L, smask, pi);
        unsigned char* base = dst + (size_t)L * A_SLICE_BYTES + (size_t)l * b_slice_bytes;
        *reinterpret_cast<uint4*>(base + kmaj_off<CK>(c, kg * 8)) = make_uint4(pr[0], pr[1], pr[2], pr[3]);
        *reinterpret_cast<uint4*>(base + kmaj_off<CK>(c, KC + kg * 8)) = make_uint4(pi[0], pi[1], pi[2], pi[3]);
      }
    }
  };
  // The wide variants (two CTAs per SM, registers to spare) keep the first
  // item of the next chunk in flight during this chunk's MMAs (its loads are
  // issued before the barrier that hands the slices to the tensor core);
  // in the narrower variants the extra registers cost more than the latency
  // they hide.
  constexpr bool PREFETCH = WIDE;
  u64 pre_re[8], pre_im[8];
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int k0 = ch * KC;
    for (int item = item0; item < n_items; item += half_t) {
      if (PREFETCH && item == item0 && ch > 0) {
        slice_item(item, pre_re, pre_im, smem);
      } else {
        u64 vre[8], vim[8];
        load_item(item, k0, vre, vim);
        slice_item(item, vre, vim, smem);
      }
    }
    if (PREFETCH && ch + 1 < nchunks && item0 < n_items) load_item(item0, k0 + KC, pre_re, pre_im);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (ch == 0) {
      // Tensor memory is taken only now (the scales and the first chunk's
      // slices need none) and given back before the FP64 stores: with more
      // than 256 accumulator columns a CTA holds all of an SM's tensor
      // memory, and other CTAs on the SM wait in tcgen05.alloc meanwhile.
      if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base_s)), "r"(cfg.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (ch == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      tmem_d = tmem_base_s;
    }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // Descriptors advance in 16-byte units in their start-address field
      // (shared-memory addresses stay below 256 KB, the field's range).  One
      // MMA per A slice l and group of B slices m stacked along N: the
      // slices of B are consecutive rows of one K-major operand and the level
      // accumulators d = l + m consecutive TMEM columns, so up to 256 / n_mma
      // slice products go into one instruction (fewer, larger MMAs issue
      // faster from the single issuing thread).
      const uint64_t ad0 = make_desc<CK>(smem_u32(sA)), bd0 = make_desc<CK>(smem_u32(sB));
      const int per = 256 / n_mma;
#pragma unroll 1
      for (int st = 0; st < KR / 16; ++st) {
        const uint32_t koff = (uint32_t)st * 2 * LBO;       // 16 BF16 of K = two core columns
#pragma unroll 1
        for (int l = 0; l < L; ++l) {
#pragma unroll 1
          for (int mg = 0; mg < L - l; mg += per) {
            const int nm = min(per, L - l - mg);
            const uint32_t tm = tmem_d + (uint32_t)((l + mg) * n_mma);
            // the l = 0 products write every level first (d = m): overwrite at the first K step
            const uint32_t acc = (ch > 0 || st > 0 || l > 0) ? 1u : 0u;
            mma_bf16(tm, ad0 + (((uint32_t)l * A_SLICE_BYTES + koff) >> 4),
                     bd0 + (((uint32_t)mg * b_slice_bytes + koff) >> 4), make_idesc(128, nm * n_mma), acc);
          }
        }
      }
      mma_commit(mb);
    }
    __syncthreads();
    last_parity = (uint32_t)(ch & 1);
    ok = mbar_wait(mb, last_parity, g.wait_limit >= 0 ? g.wait_limit : WAIT_LIMIT);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // Epilogue in passes of EP columns (64 where the operands' shared memory
  // holds that staging, else 32).  Epilogue 1 combines each real row's level
  // accumulators into one integer T on the grid of unit 2^E,
  // E = e_row + e_col - s (L + 1); tensor memory is freed after the last
  // pass's epilogue 1; epilogue 2 adds alpha / beta1 C1 / beta2 C2 / gamma
  // dshift I on that grid and converts once to FP64 (falling back to rounded
  // FP64 additions on integer bit patterns where a term is too large for the
  // grid).
  const int EP = cfg.ep;
  Acc* stage = reinterpret_cast<Acc*>(smem);   // 128 x (EP + 1) integers (operands are dead)
  const int lds = EP + 1;                       // padded rows: conflict-free per-lane row writes
  bool tmem_live = true;
  constexpr int DMAX = WIDE ? 60 : 8;           // largest left shift of a term onto the grid
  double2* C = g.C + (int64_t)e * g.sC;
  const double2* C1 = (g.C1 && g.beta1.x != 0.0) ? g.C1 + (int64_t)e * g.sC1 : nullptr;
  const double2* C2 = (g.C2 && g.beta2.x != 0.0) ? g.C2 + (int64_t)e * g.sC2 : nullptr;
  const bool na = g.alpha.x < 0, n1 = g.beta1.x < 0, n2 = g.beta2.x < 0, ng = g.gamma.x < 0;
  const bool has_d = g.dshift && g.gamma.x != 0.0;
  ulonglong2 dsh = make_ulonglong2(0ull, 0ull);
  if (has_d) dsh = ld_bits(g.dshift + (int64_t)e * g.sD);
  if (ok) {
    const int q = warp & 3, half = warp >> 2;   // warp w reads TMEM lanes 32 (w % 4) .. + 31
    const int R = q * 32 + lane;
    for (int p0 = 0; p0 < n_mma; p0 += EP) {
      // Epilogue 1: combine the levels of this lane's real row for EP / 2 columns, 8 at a time
      const int c0 = p0 + (EP / 2) * half;
      {
#pragma unroll 1
        for (int h8 = 0; h8 < EP / 2 && c0 + h8 < n_mma; h8 += 8) {
          Acc T[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) T[i] = 0;
          for (int d = 0; d < L; ++d) {
            uint32_t v[8];
            tmem_ld8(tmem_d + ((uint32_t)(q * 32) << 16) + (uint32_t)(d * n_mma + c0 + h8), v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int sh = s * (L - 1 - d);
#pragma unroll
            for (int i = 0; i < 8; ++i) T[i] += (Acc)acc_int(v[i]) << sh;
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) stage[R * lds + (EP / 2) * half + h8 + i] = T[i];
        }
      }
      const bool last = p0 + EP >= n_mma;
      if (last) asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (last) {
        if (warp == 0)
          asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem_d), "r"(cfg.tmem_cols));
        tmem_live = false;
      }
      // Epilogue 2: the linear terms on the grid, one conversion, FP64 store;
      // EU items per thread at a time with their C1 loads issued first (the
      // phase is bound by the latency of those loads).
      const int pc = min(EP, nt - p0);
      const int items = mt * pc;
      constexpr int EU = S8 ? 2 : (WIDE ? 4 : 5);
      for (int idx0 = tid; idx0 < items; idx0 += EU * TC_THREADS) {
        ulonglong2 x1v[EU];
#pragma unroll
        for (int u = 0; u < EU; ++u) {
          const int idx = idx0 + u * TC_THREADS;
          x1v[u] = make_ulonglong2(0ull, 0ull);
          if (C1 && idx < items) x1v[u] = ld_bits(C1 + (int64_t)(m0 + idx / pc) * g.ldc1 + n0 + p0 + idx % pc);
        }
#pragma unroll
        for (int u = 0; u < EU; ++u) {
        const int idx = idx0 + u * TC_THREADS;
        if (idx >= items) break;
        const int r = idx / pc, cl = idx % pc;
        const int gr = m0 + r, gc = n0 + p0 + cl;
        const int E = e_row[r] + e_col[p0 + cl] - s * (L + 1);
        Acc tre = stage[r * lds + cl], tim = stage[(MC + r) * lds + cl];
        if (na) { tre = -tre; tim = -tim; }
        Acc xre = tre, xim = tim;
        bool grid = true;
        const ulonglong2 x1 = x1v[u];
        const ulonglong2 x2 = C2 ? ld_bits(C2 + (int64_t)gr * g.ldc2 + gc) : make_ulonglong2(0ull, 0ull);
        if (C1) grid = grid_add<Acc, DMAX>(xre, x1.x, n1, E) && grid_add<Acc, DMAX>(xim, x1.y, n1, E);
        if (C2) grid = grid && grid_add<Acc, DMAX>(xre, x2.x, n2, E) && grid_add<Acc, DMAX>(xim, x2.y, n2, E);
        const bool diag = has_d && gr == gc;
        if (diag) grid = grid && grid_add<Acc, DMAX>(xre, dsh.x, ng, E) && grid_add<Acc, DMAX>(xim, dsh.y, ng, E);
        u64 re, im;
        if (grid) {
          if (WIDE) { re = i128_scaled_bits((__int128)xre, E); im = i128_scaled_bits((__int128)xim, E); }
          else { re = i64_scaled_bits((long long)xre, E); im = i64_scaled_bits((long long)xim, E); }
        } else {   // a term too large for the grid: convert the product, then add in floating point
          if (WIDE) { re = i128_scaled_bits((__int128)tre, E); im = i128_scaled_bits((__int128)tim, E); }
          else { re = i64_scaled_bits((long long)tre, E); im = i64_scaled_bits((long long)tim, E); }
          if (C1) { re = add_bits(re, flip(x1.x, n1)); im = add_bits(im, flip(x1.y, n1)); }
          if (C2) { re = add_bits(re, flip(x2.x, n2)); im = add_bits(im, flip(x2.y, n2)); }
          if (diag) { re = add_bits(re, flip(dsh.x, ng)); im = add_bits(im, flip(dsh.y, ng)); }
        }
        *reinterpret_cast<ulonglong2*>(C + (int64_t)gr * g.ldc + gc) = make_ulonglong2(re, im);
        }
      }
      __syncthreads();
    }
  } else {
    mbar_wait(mb, last_parity);       // drain: bounded wait (default limit) for MMAs still in flight
    if (tid == 0 && g.errword) atomicOr(g.errword, ERRBIT_TIMEOUT);
  }
  if (tmem_live) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem_d), "r"(cfg.tmem_cols));
    }
  }
}

int g_tc_smem_optin = 0;

bool is_pm1(double2 z) { return z.y == 0.0 && (z.x == 1.0 || z.x == -1.0); }
bool is_pm1_or_0(double2 z) { return z.y == 0.0 && (z.x == 1.0 || z.x == -1.0 || z.x == 0.0); }

TcCfg tc_config(int n, int k, int bits, int tmem_max = 512) {
  TcCfg c;
  if (bits <= 0) bits = 32;   // a plan always passes its width (48 unless set)
  // Exact FP32 level sums: (products per level) * K_real * (2^s - 1)^2 < 2^24.
  // Products of at most 32 bits only need level 0 exact (deeper levels carry
  // weights below 2^-32); longer products need every level exact.
  const double kr = 2.0 * k;
  int best_s = 1, best_L = 1;
  for (int s = 8; s >= 2; --s) {
    const int L = (bits + s - 1) / s;
    const double per_level = bits <= 32 ? 1.0 : (double)L;
    if (per_level * kr * ((1 << s) - 1) * ((1 << s) - 1) < 16777216.0) { best_s = s; best_L = L; break; }
  }
  c.s = best_s;
  c.L = best_L;
  // TMEM columns per level: the widest N tile whose L accumulators fit the
  // allowed columns (narrower tiles let two CTAs hold tensor memory at once,
  // at the cost of slicing A once per tile)
  const int cap = std::max(16, (tmem_max / c.L) / 16 * 16);
  int nm = round_up(n < 16 ? 16 : n, 16);
  if (nm > cap) nm = cap;
  c.n_mma = nm;
  int tc = 32;
  while (tc < c.L * nm) tc <<= 1;
  c.tmem_cols = tc;
  // One 64-column epilogue pass (all of epilogue 2 after the tensor memory
  // is freed) for the 5-6 slice products, whose shared memory is raised to
  // the staging's 66.5 KB where the operands need less (three CTAs per SM
  // either way); 32-column passes for the 4-slice products (four CTAs per
  // SM) and the wide ones (128-bit staging).
  const bool wide = c.s * (c.L - 1) > 36;
  const bool s8 = c.s == 8 && c.s * c.L <= 32;
  c.ep = (c.n_mma >= 64 && !wide && !s8) ? 64 : 32;
  return c;
}

bool tc_wide(const TcCfg& c) { return c.s * (c.L - 1) > 36; }

bool tc_wide(const TcCfg& c);

size_t tc_smem_bytes(const TcCfg& c) {
  const int kr = Chunk<16>::KR;
  size_t op = (size_t)c.L * 128 * kr * 2 + (size_t)c.L * c.n_mma * kr * 2;
  size_t st = (size_t)128 * (c.ep + 1) * (tc_wide(c) ? 16 : 8);   // integer staging of one epilogue pass
  return op > st ? op : st;
}

// 8-bit slices of a 32-bit fixed-point value (byte permutes).
bool tc_s8(const TcCfg& c) { return c.s == 8 && c.s * c.L <= 32; }

}  // namespace

bool zgemm_tc_available() { return true; }

cudaError_t zgemm_tc(const ZGemm& g, cudaStream_t st) {
  if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.k <= 0) return zgemm_f64(g, st);
  if (g.opA != OP_N || g.reduce || g.k > 512 || g.bits > 56 || !is_pm1(g.alpha) ||
      (g.C1 && !is_pm1_or_0(g.beta1)) || (g.C2 && !is_pm1_or_0(g.beta2)) ||
      (g.dshift && !is_pm1_or_0(g.gamma)))
    return cudaErrorNotSupported;
  const TcCfg cfg = tc_config(g.n, g.k, g.bits, g.tc_cols > 0 ? std::min(512, g.tc_cols) : 512);
  if (cfg.L > 8) return zgemm_f64(g, st);   // too long for exact slices: the FP64 product
  const int tiles_m = (g.m + MC - 1) / MC, tiles_n = (g.n + cfg.n_mma - 1) / cfg.n_mma;
  const size_t sm = tc_smem_bytes(cfg);
  if ((int)sm > g_tc_smem_optin) return cudaErrorInvalidValue;
  dim3 grid(tiles_m * tiles_n, g.batch);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  const bool wide = tc_wide(cfg), bc = g.opB == OP_C, s8 = tc_s8(cfg);
  if (s8 && !bc) zgemm_tc_kernel<true, false, false><<<grid, TC_THREADS, sm, st>>>(g, tiles_n, cfg);
  else if (s8) zgemm_tc_kernel<true, false, true><<<grid, TC_THREADS, sm, st>>>(g, tiles_n, cfg);
  else if (!wide && !bc) zgemm_tc_kernel<false, false, false><<<grid, TC_THREADS, sm, st>>>(g, tiles_n, cfg);
  else if (!wide) zgemm_tc_kernel<false, false, true><<<grid, TC_THREADS, sm, st>>>(g, tiles_n, cfg);
  else if (!bc) zgemm_tc_kernel<false, true, false><<<grid, TC_THREADS, sm, st>>>(g, tiles_n, cfg);
  else zgemm_tc_kernel<false, true, true><<<grid, TC_THREADS, sm, st>>>(g, tiles_n, cfg);
  return cudaGetLastError();
}

double zgemm_tc_issued_flops(const ZGemm& g) {
  if (g.m <= 0 || g.n <= 0 || g.k <= 0 || g.batch <= 0) return 0.0;
  const TcCfg cfg = tc_config(g.n, g.k, g.bits, g.tc_cols > 0 ? std::min(512, g.tc_cols) : 512);
  if (cfg.L > 8) return zgemm_f64_issued_flops(g);
  const double tiles = (double)((g.m + MC - 1) / MC) * ((g.n + cfg.n_mma - 1) / cfg.n_mma);
  const double ksteps = (double)((g.k + Chunk<16>::KC - 1) / Chunk<16>::KC) * (Chunk<16>::KR / 16);
  const double pairs = cfg.L * (cfg.L + 1) / 2;
  return tiles * g.batch * ksteps * pairs * 2.0 * 128.0 * cfg.n_mma * 16.0;
}

cudaError_t kernels_init() {
  cudaError_t e = zinv_init();
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, zgemm_tc_kernel<false, true, true>);
  if (e != cudaSuccess) return e;
  const int dyn = optin - (int)fa.sharedSizeBytes - 1024;
  // all of the SM's unified L1 as shared memory: four 51 KB CTAs per SM (the
  // 64-register builds), and the same split the inversion kernel needs, so
  // the two co-reside without reconfiguring the SM
  auto setup = [&](auto kern) -> cudaError_t {
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (r != cudaSuccess) return r;
    return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
  };
  if ((e = setup(zgemm_tc_kernel<true, false, false>)) != cudaSuccess) return e;
  if ((e = setup(zgemm_tc_kernel<true, false, true>)) != cudaSuccess) return e;
  if ((e = setup(zgemm_tc_kernel<false, false, false>)) != cudaSuccess) return e;
  if ((e = setup(zgemm_tc_kernel<false, false, true>)) != cudaSuccess) return e;
  if ((e = setup(zgemm_tc_kernel<false, true, false>)) != cudaSuccess) return e;
  if ((e = setup(zgemm_tc_kernel<false, true, true>)) != cudaSuccess) return e;
  g_tc_smem_optin = dyn;
  return cudaSuccess;
}

}  // namespace negf
