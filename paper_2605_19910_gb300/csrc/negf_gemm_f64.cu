// Batched complex FP64 block products on the FP64 tensor path.
//
// The sweep's products (Alg. 1: B1[i,i+1], B1[i+1,i], the Schur update and
// the three downward products; Sec. 2.3 for the n-diagonal window) are
// dense b x b complex contractions batched over energies.  Each CTA computes
// a 32 x 32 tile of one C[e]; the four warps each own a 16 x 16 sub-tile made
// of 2 x 2 DMMA m8n8k4 tiles per real component.  A complex product takes
// three real DMMAs per k-step (the 3M / Gauss form):
//     T1 = Re A Re B,  T2 = Im A Im B,  T3 = (Re A + Im A)(Re B + Im B),
//     Re C = T1 - T2,  Im C = T3 - T1 - T2,
// three quarters of the four-product form's FP64 tensor work; the operand sums
// are formed once per staged element.  Operands are staged through shared
// memory as separate real / imaginary / sum planes so that the DMMA fragments
// load with one 8-byte access per lane.
#include "negf_common.cuh"
#include "negf_kernels.h"

namespace negf {

namespace {

constexpr int BM = 32, BN = 32, BK = 16;
constexpr int LDA_S = BK + 4;   // conflict-free A fragment loads
constexpr int LDB_S = BN + 8;   // conflict-free B fragment loads
constexpr int NTHREADS = 128;

__device__ __forceinline__ void dmma884(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
}

__device__ __forceinline__ double2 cscale(double2 a, double2 s) { return cmul(a, s); }

// Loads the BM x BK tile of op(A) (rows m0.., cols k0..) into planar smem
// (real, imaginary, real + imaginary).
__device__ __forceinline__ void load_a_tile(const double2* __restrict__ A, int lda, int opA, int m, int k,
                                            int m0, int k0, double wgt, double* Ar, double* Ai, double* As,
                                            int tid) {
  for (int idx = tid; idx < BM * BK; idx += NTHREADS) {
    int r, c;
    if (opA == OP_N) { r = idx / BK; c = idx % BK; } else { c = idx / BM; r = idx % BM; }
    int gr = m0 + r, gc = k0 + c;
    double2 v = make_double2(0.0, 0.0);
    if (gr < m && gc < k) {
      if (opA == OP_N) v = A[(int64_t)gr * lda + gc];
      else { v = A[(int64_t)gc * lda + gr]; v.y = -v.y; }
    }
    if (wgt != 1.0) { v.x *= wgt; v.y *= wgt; }
    Ar[r * LDA_S + c] = v.x;
    Ai[r * LDA_S + c] = v.y;
    As[r * LDA_S + c] = v.x + v.y;
  }
}

// Loads the BK x BN tile of op(B) (rows k0.., cols n0..) into planar smem.
__device__ __forceinline__ void load_b_tile(const double2* __restrict__ B, int ldb, int opB, int k, int n,
                                            int k0, int n0, double* Br, double* Bi, double* Bs, int tid) {
  for (int idx = tid; idx < BK * BN; idx += NTHREADS) {
    int r, c;
    if (opB == OP_N) { r = idx / BN; c = idx % BN; } else { c = idx / BK; r = idx % BK; }
    int gr = k0 + r, gc = n0 + c;
    double2 v = make_double2(0.0, 0.0);
    if (gr < k && gc < n) {
      if (opB == OP_N) v = B[(int64_t)gr * ldb + gc];
      else { v = B[(int64_t)gc * ldb + gr]; v.y = -v.y; }
    }
    Br[r * LDB_S + c] = v.x;
    Bi[r * LDB_S + c] = v.y;
    Bs[r * LDB_S + c] = v.x + v.y;
  }
}

__global__ void __launch_bounds__(NTHREADS) zgemm_f64_kernel(ZGemm g, int tiles_n) {
  __shared__ double Ar[BM * LDA_S], Ai[BM * LDA_S], As[BM * LDA_S];
  __shared__ double Br[BK * LDB_S], Bi[BK * LDB_S], Bs[BK * LDB_S];

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, tq = lane & 3;   // DMMA groupID / threadID_in_group
  const int wm = warp >> 1, wn = warp & 1;
  const int tile = blockIdx.x;
  const int m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN;

  double t1[2][2][2], t2[2][2][2], t3[2][2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int i = 0; i < 2; ++i) t1[a][c][i] = t2[a][c][i] = t3[a][c][i] = 0.0;

  const int e_first = g.reduce ? 0 : blockIdx.y;
  const int e_last = g.reduce ? g.batch : blockIdx.y + 1;
  for (int e = e_first; e < e_last; ++e) {
    const double2* A = g.A + (int64_t)e * g.sA;
    const double2* B = g.B + (int64_t)e * g.sB;
    const double wgt = g.weight ? g.weight[e] : 1.0;   // per-batch real weight on A
    if (wgt == 0.0 && g.reduce) continue;
    for (int k0 = 0; k0 < g.k; k0 += BK) {
      load_a_tile(A, g.lda, g.opA, g.m, g.k, m0, k0, wgt, Ar, Ai, As, tid);
      load_b_tile(B, g.ldb, g.opB, g.k, g.n, k0, n0, Br, Bi, Bs, tid);
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; kk += 4) {
        double are[2], aim[2], asum[2], bre[2], bim[2], bsum[2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          int r = wm * 16 + a * 8 + gq;
          are[a] = Ar[r * LDA_S + kk + tq];
          aim[a] = Ai[r * LDA_S + kk + tq];
          asum[a] = As[r * LDA_S + kk + tq];
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          int col = wn * 16 + c * 8 + gq;
          bre[c] = Br[(kk + tq) * LDB_S + col];
          bim[c] = Bi[(kk + tq) * LDB_S + col];
          bsum[c] = Bs[(kk + tq) * LDB_S + col];
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            dmma884(t1[a][c][0], t1[a][c][1], are[a], bre[c]);
            dmma884(t2[a][c][0], t2[a][c][1], aim[a], bim[c]);
            dmma884(t3[a][c][0], t3[a][c][1], asum[a], bsum[c]);
          }
      }
      __syncthreads();
    }
  }

  const int eo = g.reduce ? 0 : blockIdx.y;
  double2* C = g.C + (int64_t)eo * g.sC;
  const double2* C1 = g.C1 ? g.C1 + (int64_t)eo * g.sC1 : nullptr;
  const double2* C2 = g.C2 ? g.C2 + (int64_t)eo * g.sC2 : nullptr;
  double2 dsh = make_double2(0.0, 0.0);
  if (g.dshift) dsh = cmul(g.gamma, g.dshift[(int64_t)eo * g.sD]);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        int row = m0 + wm * 16 + a * 8 + gq;
        int col = n0 + wn * 16 + c * 8 + 2 * tq + i;
        if (row < g.m && col < g.n) {
          const double re = t1[a][c][i] - t2[a][c][i];
          const double im = t3[a][c][i] - t1[a][c][i] - t2[a][c][i];
          double2 v = cscale(make_double2(re, im), g.alpha);
          if (C1) {
            double2 x = cmul(g.beta1, C1[(int64_t)row * g.ldc1 + col]);
            v.x += x.x; v.y += x.y;
          }
          if (C2) {
            double2 x = cmul(g.beta2, C2[(int64_t)row * g.ldc2 + col]);
            v.x += x.x; v.y += x.y;
          }
          if (g.dshift && row == col) { v.x += dsh.x; v.y += dsh.y; }
          C[(int64_t)row * g.ldc + col] = v;
        }
      }
}

}  // namespace

cudaError_t zgemm_f64(const ZGemm& g, cudaStream_t st) {
  if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return cudaSuccess;
  const int tiles_m = (g.m + BM - 1) / BM, tiles_n = (g.n + BN - 1) / BN;
  dim3 grid(tiles_m * tiles_n, g.reduce ? 1 : g.batch);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  zgemm_f64_kernel<<<grid, NTHREADS, 0, st>>>(g, tiles_n);
  return cudaGetLastError();
}

double zgemm_f64_issued_flops(const ZGemm& g) {
  if (g.m <= 0 || g.n <= 0 || g.k <= 0 || g.batch <= 0) return 0.0;
  return 6.0 * g.m * (double)g.n * g.k * g.batch;
}

}  // namespace negf
