// Split-precision complex block products on the 5th-generation tensor cores.
//
// Used by the mixed-precision sweep for every block product of Alg. 1 /
// Sec. 2.3 (the multipliers, the Schur update and the downward products);
// the per-block inversions stay in FP64 (negf_inv.cu).
//
// A complex product C = A B is computed as one real product on the tensor
// cores, with the real and imaginary parts stacked along M and K:
//
//     [Re C]   [Re A  -Im A] [Re B]
//     [Im C] = [Im A   Re A] [Im B]
//
// so 64 complex rows of C form one M = 128 tcgen05 tile.  Each real operand
// is split into two TF32 parts (x = hi + lo, hi = tf32(x), lo = tf32(x - hi))
// and the product is accumulated in FP32 in tensor memory as
// A_hi B_hi + A_hi B_lo + A_lo B_hi, which carries about 22 significant bits.
// The epilogue reads the accumulator with tcgen05.ld, forms the complex
// result and applies alpha / beta / the diagonal shift in FP64.
//
// One CTA computes a 64 x N complex tile (N <= 256) of one batch entry; K is
// streamed through shared memory in chunks of 32 complex columns.  Operands
// use the K-major, non-swizzled canonical layout (8-row x 16-byte core
// matrices).  One thread issues the MMAs; completion is tracked with an
// mbarrier whose wait is bounded.
#include "negf_common.cuh"
#include "negf_kernels.h"

namespace negf {

cudaError_t zinv_init();

namespace {

constexpr int TC_THREADS = 128;
constexpr int MC = 64;                // complex rows per CTA (M = 128 real)
constexpr int KC = 32;                // complex K per chunk (64 real)
constexpr int KR = 2 * KC;            // real K per chunk
constexpr int CORE_BYTES = 128;       // 8 rows x 16 bytes
constexpr int SBO = (KR / 4) * CORE_BYTES;   // bytes between 8-row groups
constexpr int LBO = CORE_BYTES;              // bytes between 16-byte K groups
constexpr int A_BYTES = 128 * KR * 4;        // one split of the A chunk
constexpr long long WAIT_LIMIT = 1ll << 26;  // bounded mbarrier wait

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// byte offset of real element (row, kcol) in a K-major non-swizzled tile
__device__ __forceinline__ uint32_t kmaj_off(int row, int kcol) {
  return (uint32_t)((row >> 3) * SBO + (kcol >> 2) * LBO + (row & 7) * 16 + (kcol & 3) * 4);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void split_tf32(double x, float& hi, float& lo) {
  hi = to_tf32((float)x);
  lo = to_tf32((float)(x - (double)hi));
}

// tcgen05 shared-memory matrix descriptor: start address, leading (K) and
// stride (M/N) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::tf32, FP32 accumulate, K-major A and B
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
      :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared memory: [A hi | A lo | B hi | B lo] operand chunks, reused as the
// FP32 staging of the accumulator in the epilogue.
__global__ void __launch_bounds__(TC_THREADS) zgemm_tc_kernel(ZGemm g, int tiles_n, int n_mma, int tmem_cols,
                                                               int* errword) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_s;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int tile = blockIdx.x;
  const int m0 = (tile / tiles_n) * MC;
  const int n0 = (tile % tiles_n) * n_mma;
  const int e = blockIdx.y;
  const int nt = min(n_mma, g.n - n0);   // valid complex columns of this tile
  const int b_bytes = n_mma * KR * 4;    // one split of the B chunk

  unsigned char* sAh = smem;
  unsigned char* sAl = smem + A_BYTES;
  unsigned char* sBh = smem + 2 * A_BYTES;
  unsigned char* sBl = smem + 2 * A_BYTES + b_bytes;

  const double2* A = g.A + (int64_t)e * g.sA;
  const double2* B = g.B + (int64_t)e * g.sB;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base_s)), "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem_d = tmem_base_s;
  const uint32_t mb = smem_u32(&mbar);
  const uint32_t idesc = make_idesc(128, n_mma);
  bool ok = true;
  uint32_t last_parity = 0;

  const int nchunks = (g.k + KC - 1) / KC;
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int k0 = ch * KC;
    // --- stage A: rows r (real part block) and 64 + r (imaginary part block)
    for (int idx = tid; idx < MC * KC; idx += TC_THREADS) {
      const int r = idx / KC, kk = idx % KC;
      const int gr = m0 + r, gk = k0 + kk;
      double2 v = make_double2(0.0, 0.0);
      if (gr < g.m && gk < g.k) v = A[(int64_t)gr * g.lda + gk];
      float rh, rl, ih, il, nih, nil;
      split_tf32(v.x, rh, rl);
      split_tf32(v.y, ih, il);
      split_tf32(-v.y, nih, nil);
      // row r: [Re A | -Im A]; row 64 + r: [Im A | Re A]
      *reinterpret_cast<float*>(sAh + kmaj_off(r, kk)) = rh;
      *reinterpret_cast<float*>(sAl + kmaj_off(r, kk)) = rl;
      *reinterpret_cast<float*>(sAh + kmaj_off(r, KC + kk)) = nih;
      *reinterpret_cast<float*>(sAl + kmaj_off(r, KC + kk)) = nil;
      *reinterpret_cast<float*>(sAh + kmaj_off(MC + r, kk)) = ih;
      *reinterpret_cast<float*>(sAl + kmaj_off(MC + r, kk)) = il;
      *reinterpret_cast<float*>(sAh + kmaj_off(MC + r, KC + kk)) = rh;
      *reinterpret_cast<float*>(sAl + kmaj_off(MC + r, KC + kk)) = rl;
    }
    // --- stage B^T (K-major): row n holds [Re B(:, n) | Im B(:, n)]
    for (int idx = tid; idx < KC * n_mma; idx += TC_THREADS) {
      const int kk = idx / n_mma, c = idx % n_mma;
      const int gk = k0 + kk, gc = n0 + c;
      double2 v = make_double2(0.0, 0.0);
      if (gk < g.k && c < nt) v = B[(int64_t)gk * g.ldb + gc];
      float rh, rl, ih, il;
      split_tf32(v.x, rh, rl);
      split_tf32(v.y, ih, il);
      *reinterpret_cast<float*>(sBh + kmaj_off(c, kk)) = rh;
      *reinterpret_cast<float*>(sBl + kmaj_off(c, kk)) = rl;
      *reinterpret_cast<float*>(sBh + kmaj_off(c, KC + kk)) = ih;
      *reinterpret_cast<float*>(sBl + kmaj_off(c, KC + kk)) = il;
    }
    // make the generic-proxy stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t aH = smem_u32(sAh), aL = smem_u32(sAl), bH = smem_u32(sBh), bL = smem_u32(sBl);
#pragma unroll 1
      for (int s = 0; s < KR / 8; ++s) {
        const uint32_t koff = (uint32_t)s * 2 * LBO;    // 8 real K = two 16-byte core columns
        const uint32_t acc0 = (ch > 0 || s > 0) ? 1u : 0u;
        mma_tf32(tmem_d, make_desc(aH + koff), make_desc(bH + koff), idesc, acc0);
        mma_tf32(tmem_d, make_desc(aH + koff), make_desc(bL + koff), idesc, 1u);
        mma_tf32(tmem_d, make_desc(aL + koff), make_desc(bH + koff), idesc, 1u);
      }
      mma_commit(mb);
    }
    __syncthreads();
    last_parity = (uint32_t)(ch & 1);
    ok = mbar_wait(mb, last_parity);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (ok) {
    // --- epilogue: TMEM lane = real row; stage FP32 rows in shared memory
    float* stage = reinterpret_cast<float*>(smem);    // 128 x n_mma floats
    const int row = warp * 32 + (tid & 31);
    for (int c0 = 0; c0 < n_mma; c0 += 16) {
      float v[16];
      tmem_ld16(tmem_d + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) stage[row * n_mma + c0 + i] = v[i];
    }
  } else {
    // give the MMAs still in flight a second bounded wait before TMEM is freed
    mbar_wait(mb, last_parity);
    if (tid == 0 && errword) atomicOr(errword, ERRBIT_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem_d), "r"(tmem_cols));
  }
  if (!ok) return;

  const float* stage = reinterpret_cast<const float*>(smem);
  double2* C = g.C + (int64_t)e * g.sC;
  const double2* C1 = g.C1 ? g.C1 + (int64_t)e * g.sC1 : nullptr;
  const double2* C2 = g.C2 ? g.C2 + (int64_t)e * g.sC2 : nullptr;
  double2 dsh = make_double2(0.0, 0.0);
  if (g.dshift) dsh = cmul(g.gamma, g.dshift[(int64_t)e * g.sD]);
  const int mt = min(MC, g.m - m0);
  for (int idx = tid; idx < mt * nt; idx += TC_THREADS) {
    const int r = idx / nt, c = idx % nt;
    const int gr = m0 + r, gc = n0 + c;
    double2 acc = make_double2((double)stage[r * n_mma + c], (double)stage[(MC + r) * n_mma + c]);
    double2 v = cmul(acc, g.alpha);
    if (C1) {
      double2 x = cmul(g.beta1, C1[(int64_t)gr * g.ldc1 + gc]);
      v.x += x.x; v.y += x.y;
    }
    if (C2) {
      double2 x = cmul(g.beta2, C2[(int64_t)gr * g.ldc2 + gc]);
      v.x += x.x; v.y += x.y;
    }
    if (g.dshift && gr == gc) { v.x += dsh.x; v.y += dsh.y; }
    C[(int64_t)gr * g.ldc + gc] = v;
  }
}

int g_tc_smem_optin = 0;

}  // namespace

bool zgemm_tc_available() { return true; }

// Largest n per tile: 256 columns of TMEM / MMA N.
static int tc_n_tile(int n) {
  int nm = round_up(n < 16 ? 16 : n, 16);
  return nm > 256 ? 256 : nm;
}

static size_t tc_smem_bytes(int n_mma) {
  size_t op = 2 * (size_t)A_BYTES + 2 * (size_t)n_mma * KR * 4;
  size_t st = (size_t)128 * n_mma * 4;
  return op > st ? op : st;
}

cudaError_t zgemm_tc(const ZGemm& g, cudaStream_t st) {
  if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.opA != OP_N || g.opB != OP_N || g.reduce) return cudaErrorNotSupported;
  if (g.k <= 0) return zgemm_f64(g, st);   // nothing to contract: the FP64 epilogue path
  const int n_mma = tc_n_tile(g.n);
  int tmem_cols = 32;
  while (tmem_cols < n_mma) tmem_cols <<= 1;
  const int tiles_m = (g.m + MC - 1) / MC, tiles_n = (g.n + n_mma - 1) / n_mma;
  const size_t sm = tc_smem_bytes(n_mma);
  if ((int)sm > g_tc_smem_optin) return cudaErrorInvalidValue;
  dim3 grid(tiles_m * tiles_n, g.batch);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  zgemm_tc_kernel<<<grid, TC_THREADS, sm, st>>>(g, tiles_n, n_mma, tmem_cols, g.errword);
  return cudaGetLastError();
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
  e = cudaFuncGetAttributes(&fa, zgemm_tc_kernel);
  if (e != cudaSuccess) return e;
  int dyn = optin - (int)fa.sharedSizeBytes - 1024;
  e = cudaFuncSetAttribute(zgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  if (e != cudaSuccess) return e;
  g_tc_smem_optin = dyn;
  return cudaSuccess;
}

}  // namespace negf
