// Batched FP64 inversion of b x b complex blocks in shared memory.
//
// Step a3 of the sweep: t_i = S_i^{-1} (Alg. 1, the LU of B2[i,i]; here an
// explicit inverse, whose later products replace the paper's GETRS calls).
// Gauss-Jordan elimination with partial pivoting (pivot = largest
// |re| + |im| in the column, first index on ties), one CTA per block, the
// whole block resident in shared memory.  The pivot search runs in one warp
// with shuffles; the rank-1 update of each column is spread over the CTA.
#include "negf_common.cuh"
#include "negf_kernels.h"

namespace negf {

namespace {

constexpr int INV_TX = 32;
constexpr int INV_TY = 8;

__global__ void __launch_bounds__(INV_TX * INV_TY)
zinv_gj_kernel(const double2* __restrict__ S, int64_t sS, double2* __restrict__ T, int64_t sT, int b,
               int32_t* __restrict__ info, int layer1, int* __restrict__ errword) {
  extern __shared__ double2 smem[];
  const int ld = b + 1;
  double2* A = smem;                 // b x ld
  double2* f = A + b * ld;           // column multipliers
  int* perm = reinterpret_cast<int*>(f + b);
  __shared__ int s_piv;
  __shared__ double2 s_pv;
  __shared__ double2 s_akk;
  __shared__ double2 s_d;
  __shared__ int s_bad;

  const int e = blockIdx.x;
  const double2* src = S + (int64_t)e * sS;
  double2* dst = T + (int64_t)e * sT;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * INV_TX + tx;
  const int nth = INV_TX * INV_TY;

  for (int i = ty; i < b; i += INV_TY)
    for (int j = tx; j < b; j += INV_TX) A[i * ld + j] = src[(int64_t)i * b + j];
  if (tid == 0) s_bad = 0;
  __syncthreads();

  for (int k = 0; k < b; ++k) {
    // Phase 1: pivot search in column k (warp 0).
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i < b; i += 32) {
        double v = cabs1(A[i * ld + k]);
        if (v != v) v = INFINITY;   // a NaN becomes the pivot and is reported
        if (v > best) { best = v; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        double ob = __shfl_down_sync(0xffffffffu, best, off);
        int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        s_piv = bi;
        perm[k] = bi;
        s_pv = A[bi * ld + k];
        s_akk = A[k * ld + k];
        double2 pv = s_pv;
        bool finite = isfinite(pv.x) && isfinite(pv.y);
        bool zero = (pv.x == 0.0 && pv.y == 0.0);
        s_d = crecip(pv);   // once per column: FP64 division is a multi-instruction sequence
        if ((!finite || zero) && !s_bad) {
          s_bad = 1;
          atomicOr(errword, finite ? ERRBIT_SINGULAR : ERRBIT_NONFINITE);
          if (info[e] == 0) info[e] = layer1;
        }
      }
    }
    __syncthreads();
    const int p = s_piv;
    const double2 d = s_d;
    // Phase 2: swap rows k and p, scale the new row k by 1/pivot, and keep the
    // multipliers f_i (column k after the swap) for i != k.
    for (int j = tid; j < b; j += nth) {
      double2 ak = A[k * ld + j];
      double2 ap = A[p * ld + j];
      A[p * ld + j] = ak;
      A[k * ld + j] = (j == k) ? d : cmul(ap, d);
    }
    for (int i = tid; i < b; i += nth) {
      if (i != k) f[i] = (i == p) ? s_akk : A[i * ld + k];
    }
    __syncthreads();
    // Phase 3: rank-1 update of every row but k.
    for (int j = tx; j < b; j += INV_TX) {
      const double2 akj = A[k * ld + j];
      for (int i = ty; i < b; i += INV_TY) {
        if (i == k) continue;
        double2 a = (j == k) ? make_double2(0.0, 0.0) : A[i * ld + j];
        A[i * ld + j] = cfnms(a, f[i], akj);
      }
    }
    __syncthreads();
  }
  // Undo the row interchanges: the in-place result is (P S)^{-1} = S^{-1} P^T,
  // so swap columns back in reverse order (each thread owns whole rows).
  for (int i = tid; i < b; i += nth) {
    for (int k = b - 1; k >= 0; --k) {
      int p = perm[k];
      if (p != k) {
        double2 t0 = A[i * ld + k];
        A[i * ld + k] = A[i * ld + p];
        A[i * ld + p] = t0;
      }
    }
  }
  __syncthreads();
  for (int i = ty; i < b; i += INV_TY)
    for (int j = tx; j < b; j += INV_TX) dst[(int64_t)i * b + j] = A[i * ld + j];
}

size_t inv_smem_bytes(int b) {
  return (size_t)b * (b + 1) * sizeof(double2) + (size_t)b * sizeof(double2) + (size_t)b * sizeof(int);
}

}  // namespace

static size_t g_inv_dyn_max = 0;   // dynamic shared memory opt-in of the kernel

cudaError_t zinv_init() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, zinv_gj_kernel);
  if (e != cudaSuccess) return e;
  size_t dyn = (size_t)optin - fa.sharedSizeBytes;
  e = cudaFuncSetAttribute(zinv_gj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  g_inv_dyn_max = dyn;
  return cudaSuccess;
}

int zinv_max_block() {
  size_t lim = g_inv_dyn_max ? g_inv_dyn_max : (size_t)227 * 1024 - 1024;
  int b = 1;
  while (inv_smem_bytes(b + 1) <= lim) ++b;
  return b;
}

cudaError_t zinv_f64(const double2* S, int64_t sS, double2* T, int64_t sT, int b, int batch,
                     int32_t* info, int layer1, int* errword, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  size_t sm = inv_smem_bytes(b);
  if (sm > g_inv_dyn_max) return cudaErrorInvalidValue;
  zinv_gj_kernel<<<batch, dim3(INV_TX, INV_TY), sm, st>>>(S, sS, T, sT, b, info, layer1, errword);
  return cudaGetLastError();
}

}  // namespace negf
