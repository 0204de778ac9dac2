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
  double2* f = A + b * ld;           // column k of the current state (multipliers)
  double2* rs = f + b;               // the pivot row scaled by 1 / pivot (new row k)
  double2* rk = rs + b;              // the old row k (moves to row p)
  int* perm = reinterpret_cast<int*>(rk + b);
  __shared__ int s_piv;
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
    // Phase 1 (warp 0): pivot of column k (largest |re| + |im| among rows
    // >= k, first index on ties), one reciprocal, and the stashes the update
    // reads: column k, the scaled pivot row and the old row k.
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = tid; i < b; i += 32) {
        const double2 a = A[i * ld + k];
        f[i] = a;
        if (i < k) continue;
        double v = cabs1(a);
        if (v != v) v = INFINITY;   // a NaN becomes the pivot and is reported
        if (v > best) { best = v; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        perm[k] = bi;
        s_piv = bi;
        const double2 pv = A[bi * ld + k];
        const bool finite = isfinite(pv.x) && isfinite(pv.y);
        const bool zero = (pv.x == 0.0 && pv.y == 0.0);
        s_d = crecip(pv);   // once per column: FP64 division is a multi-instruction sequence
        if ((!finite || zero) && !s_bad) {
          s_bad = 1;
          atomicOr(errword, finite ? ERRBIT_SINGULAR : ERRBIT_NONFINITE);
          if (info[e] == 0) info[e] = layer1;
        }
      }
      __syncwarp();
      const int p = s_piv;
      const double2 d = s_d;
      for (int j = tid; j < b; j += 32) {
        rs[j] = (j == k) ? d : cmul(A[p * ld + j], d);
        rk[j] = A[k * ld + j];
      }
    }
    __syncthreads();
    // Phase 2: the Gauss-Jordan step with rows k and p exchanged, from the
    // stashes only (each thread rewrites its own elements): new row k = rs;
    // the row that lands at p (old row k) and every other row i lose
    // (multiplier) x rs, the multiplier of row p being the old A_kk; column k
    // of those rows becomes -(multiplier) x rs_k.
    const int p = s_piv;
    for (int j = tx; j < b; j += INV_TX) {
      const double2 rsj = rs[j];
      for (int i = ty; i < b; i += INV_TY) {
        if (i == k) {
          A[k * ld + j] = rsj;
          continue;
        }
        double2 a, fi;
        if (i == p) { a = rk[j]; fi = f[k]; }
        else { a = A[i * ld + j]; fi = f[i]; }
        if (j == k) a = make_double2(0.0, 0.0);
        A[i * ld + j] = cfnms(a, fi, rsj);
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
  return (size_t)b * (b + 1) * sizeof(double2) + 3 * (size_t)b * sizeof(double2) + (size_t)b * sizeof(int);
}

}  // namespace

static size_t g_inv_dyn_max = 0;   // dynamic shared memory opt-in of the kernel
static int g_sms = 0;               // SMs of the device

cudaError_t zinv_cluster_init();
int zinv_cluster_max_block();

cudaError_t zinv_init() {
  {
    cudaError_t ce = zinv_cluster_init();
    if (ce != cudaSuccess) return ce;
  }
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, zinv_gj_kernel);
  if (e != cudaSuccess) return e;
  size_t dyn = (size_t)optin - fa.sharedSizeBytes;
  e = cudaFuncSetAttribute(zinv_gj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(zinv_gj_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  g_inv_dyn_max = dyn;
  return cudaSuccess;
}

int zinv_max_block() { return zinv_cluster_max_block(); }

cudaError_t zinv_f64_cluster(const double2* S, int64_t sS, double2* T, int64_t sT, int b, int batch, int32_t* info,
                             int layer1, int* errword, cudaStream_t st);

cudaError_t zinv_f64(const double2* S, int64_t sS, double2* T, int64_t sT, int b, int batch,
                     int32_t* info, int layer1, int* errword, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  size_t sm = inv_smem_bytes(b);
  // blocks too large for one CTA, and launches too small to fill the GPU
  // (few energies: a lone 64 x 64 inversion takes ~250 us of one SM's FP64
  // unit) go to the 2-CTA cluster kernel, which splits each block's rows
  // over two SMs
  if (sm > g_inv_dyn_max || (b >= 48 && g_sms > 0 && 2 * batch <= g_sms))
    return zinv_f64_cluster(S, sS, T, sT, b, batch, info, layer1, errword, st);
  zinv_gj_kernel<<<batch, dim3(INV_TX, INV_TY), sm, st>>>(S, sS, T, sT, b, info, layer1, errword);
  return cudaGetLastError();
}

}  // namespace negf

// ---------------------------------------------------------------------------
// Blocks too large for one CTA's shared memory (b up to 160 complex128 =
// 400 KB): a cluster of two CTAs on two SMs, each holding half of the rows.
// Per column: each CTA searches its rows for a pivot candidate, a cluster
// barrier publishes the candidates, both CTAs read them (and the old rows k
// and p) through distributed shared memory, a second barrier ends the reads,
// then each CTA swaps / scales its own rows and applies the rank-1 update to
// them.  Both CTAs take identical pivot decisions, so the column
// interchanges are undone locally at the end.
// ---------------------------------------------------------------------------
#include <cooperative_groups.h>

namespace negf {
namespace {

namespace cg = cooperative_groups;

constexpr int CL_THREADS = 256;

struct PivCand {
  double val;
  int row;
};

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(CL_THREADS)
zinv_gj_cluster_kernel(const double2* __restrict__ S, int64_t sS, double2* __restrict__ T, int64_t sT, int b,
                       int32_t* __restrict__ info, int layer1, int* __restrict__ errword) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int e = blockIdx.x >> 1;
  const int h0 = (b + 1) / 2;
  const int r0 = rank == 0 ? 0 : h0;                 // first global row of this CTA
  const int nr = rank == 0 ? h0 : b - h0;            // rows held here
  const int ld = b + 1;

  extern __shared__ double2 smem[];
  double2* A = smem;                                  // nr x ld (local rows)
  double2* rowk = A + (size_t)h0 * ld;               // old row k
  double2* rowp = rowk + b;                          // old row p
  double2* frow = rowp + b;                          // new (scaled) row k
  double2* fcol = frow + b;                          // multipliers of the local rows
  int* perm = reinterpret_cast<int*>(fcol + h0);
  __shared__ PivCand cand;
  __shared__ int s_bad;

  const double2* src = S + (int64_t)e * sS;
  double2* dst = T + (int64_t)e * sT;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < nr * b; idx += CL_THREADS) {
    const int i = idx / b, j = idx - (idx / b) * b;
    A[i * ld + j] = src[(int64_t)(r0 + i) * b + j];
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();

  for (int k = 0; k < b; ++k) {
    // (a) local pivot candidate among rows >= k held here
    if (tid < 32) {
      double best = -1.0;
      int bi = -1;
      for (int li = tid; li < nr; li += 32) {
        const int gi = r0 + li;
        if (gi < k) continue;
        double v = cabs1(A[li * ld + k]);
        if (v != v) v = INFINITY;
        if (v > best || (v == best && gi < bi)) { best = v; bi = gi; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) { best = ob; bi = oi; }
      }
      if (tid == 0) { cand.val = best; cand.row = bi; }
    }
    cluster.sync();                                   // candidates published
    // (b) the pivot row p: larger candidate, lower row on ties (same on both CTAs)
    const PivCand* other = cluster.map_shared_rank(&cand, rank ^ 1);
    PivCand c0 = rank == 0 ? cand : *other, c1 = rank == 0 ? *other : cand;
    int p;
    if (c1.row < 0) p = c0.row;
    else if (c0.row < 0) p = c1.row;
    else p = (c1.val > c0.val) ? c1.row : c0.row;
    if (p < 0) p = k;                                  // unreachable for b >= 1
    // old rows k and p, from whichever CTA holds them
    {
      const int ok = k < h0 ? 0 : 1, op = p < h0 ? 0 : 1;
      const double2* Ak = cluster.map_shared_rank(A, ok) + (size_t)(k - (ok ? h0 : 0)) * ld;
      const double2* Ap = cluster.map_shared_rank(A, op) + (size_t)(p - (op ? h0 : 0)) * ld;
      for (int j = tid; j < b; j += CL_THREADS) {
        rowk[j] = Ak[j];
        rowp[j] = Ap[j];
      }
    }
    cluster.sync();                                   // all remote reads done
    const double2 pv = rowp[k];
    if (tid == 0) {
      perm[k] = p;                                    // identical decision on both CTAs
      const bool finite = isfinite(pv.x) && isfinite(pv.y);
      const bool zero = (pv.x == 0.0 && pv.y == 0.0);
      if ((!finite || zero) && !s_bad && rank == 0) {
        s_bad = 1;
        atomicOr(errword, finite ? ERRBIT_SINGULAR : ERRBIT_NONFINITE);
        if (info[e] == 0) info[e] = layer1;
      }
    }
    const double2 d = crecip(pv);
    for (int j = tid; j < b; j += CL_THREADS) frow[j] = (j == k) ? d : cmul(rowp[j], d);
    __syncthreads();
    // (c) swap / scale the local rows and keep the multipliers
    if (k >= r0 && k < r0 + nr)
      for (int j = tid; j < b; j += CL_THREADS) A[(k - r0) * ld + j] = frow[j];
    if (p != k && p >= r0 && p < r0 + nr)
      for (int j = tid; j < b; j += CL_THREADS) A[(p - r0) * ld + j] = rowk[j];
    __syncthreads();
    for (int li = tid; li < nr; li += CL_THREADS) {
      const int gi = r0 + li;
      fcol[li] = (gi == k) ? make_double2(0.0, 0.0) : A[li * ld + k];
    }
    __syncthreads();
    // (d) rank-1 update of the local rows (all but k)
    for (int j = tid & 31; j < b; j += 32) {
      const double2 akj = frow[j];
      for (int li = tid >> 5; li < nr; li += CL_THREADS / 32) {
        if (r0 + li == k) continue;
        const double2 a = (j == k) ? make_double2(0.0, 0.0) : A[li * ld + j];
        A[li * ld + j] = cfnms(a, fcol[li], akj);
      }
    }
    __syncthreads();
  }
  __syncthreads();
  for (int li = tid; li < nr; li += CL_THREADS)
    for (int k = b - 1; k >= 0; --k) {
      const int p = perm[k];
      if (p != k) {
        const double2 t0 = A[li * ld + k];
        A[li * ld + k] = A[li * ld + p];
        A[li * ld + p] = t0;
      }
    }
  __syncthreads();
  for (int idx = tid; idx < nr * b; idx += CL_THREADS) {
    const int i = idx / b, j = idx - (idx / b) * b;
    dst[(int64_t)(r0 + i) * b + j] = A[i * ld + j];
  }
  cluster.sync();                                     // keep smem alive for remote readers
}

size_t cluster_smem_bytes(int b) {
  const int h0 = (b + 1) / 2;
  return (size_t)h0 * (b + 1) * sizeof(double2) + 3 * (size_t)b * sizeof(double2) + (size_t)h0 * sizeof(double2) +
         (size_t)b * sizeof(int);
}

size_t g_cl_dyn_max = 0;

}  // namespace

cudaError_t zinv_cluster_init() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, zinv_gj_cluster_kernel);
  if (e != cudaSuccess) return e;
  const size_t dyn = (size_t)optin - fa.sharedSizeBytes;
  e = cudaFuncSetAttribute(zinv_gj_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(zinv_gj_cluster_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  g_cl_dyn_max = dyn;
  return cudaSuccess;
}

int zinv_cluster_max_block() {
  const size_t lim = g_cl_dyn_max ? g_cl_dyn_max : (size_t)227 * 1024 - 1024;
  int b = 1;
  while (cluster_smem_bytes(b + 1) <= lim) ++b;
  return b;
}

cudaError_t zinv_f64_cluster(const double2* S, int64_t sS, double2* T, int64_t sT, int b, int batch, int32_t* info,
                             int layer1, int* errword, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  const size_t sm = cluster_smem_bytes(b);
  if (sm > g_cl_dyn_max) return cudaErrorInvalidValue;
  zinv_gj_cluster_kernel<<<2 * batch, CL_THREADS, sm, st>>>(S, sS, T, sT, b, info, layer1, errword);
  return cudaGetLastError();
}

}  // namespace negf
