// Internal launch interface of the libnegf.so kernels (host side, C++).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace negf {

// Operand access mode of a batched block product.
enum Op : int { OP_N = 0, OP_C = 1 /* conjugate transpose */ };

// One batched complex product over a batch of energies:
//   C[e] = alpha * op(A[e]) op(B[e]) + beta1 * C1[e] + beta2 * C2[e]
//          + gamma * dshift[e] * I
// Every operand X[e] lives at X + e * sX (sX = 0 shares one block across the
// batch); blocks are row-major with leading dimension ldX.  C1/C2/dshift may
// be null.  With weight != null, op(A[e]) is scaled by the real weight[e].
// With reduce != 0 the batch is summed into one C:
//   C = alpha * sum_e weight[e] * op(A[e]) op(B[e]) + beta1 * C1.
struct ZGemm {
  int m = 0, n = 0, k = 0;
  const double2* A = nullptr; int64_t sA = 0; int lda = 0; int opA = OP_N;
  const double2* B = nullptr; int64_t sB = 0; int ldb = 0; int opB = OP_N;
  double2* C = nullptr; int64_t sC = 0; int ldc = 0;
  const double2* C1 = nullptr; int64_t sC1 = 0; int ldc1 = 0;
  const double2* C2 = nullptr; int64_t sC2 = 0; int ldc2 = 0;
  const double2* dshift = nullptr; int64_t sD = 1;
  double2 alpha = {1.0, 0.0}, beta1 = {0.0, 0.0}, beta2 = {0.0, 0.0}, gamma = {0.0, 0.0};
  const double* weight = nullptr;
  int* errword = nullptr;   // device error word for bounded-wait timeouts (tensor-core path)
  int bits = 0;             // tensor-core path: significant bits of the product (0 = 32; up to 56)
  long long wait_limit = -1;  // tensor-core path: polls of the MMA-completion wait (< 0: the default)
  int tc_cols = 0;          // tensor-core path: most TMEM columns of one CTA (0 = 512; sets the N tile)
  int batch = 1;
  int reduce = 0;
};

// FP64 product on the FP64 tensor path (mma.sync m8n8k4 f64).
cudaError_t zgemm_f64(const ZGemm& g, cudaStream_t st);
// Product from exact BF16 slices on the 5th-generation tensor cores
// (g.bits significant bits, up to 56).
cudaError_t zgemm_tc(const ZGemm& g, cudaStream_t st);
bool zgemm_tc_available();
// Flops the units execute for one call, for the profiler (the method counts
// 8 m n k per complex product): zgemm_f64 issues three real products per
// complex one (3M form), 6 m n k; zgemm_tc issues L (L + 1) / 2 BF16 slice
// products per 16-deep real K step over whole tiles of 128 real rows and its
// N tile (padding included), or the FP64 count where it hands over to
// zgemm_f64.
double zgemm_f64_issued_flops(const ZGemm& g);
double zgemm_tc_issued_flops(const ZGemm& g);

// One-time kernel attributes (shared-memory opt-in); call outside capture.
cudaError_t kernels_init();

// Batched in-place-capable FP64 inversion T[e] = S[e]^{-1} (b x b, row-major,
// contiguous) by Gauss-Jordan elimination with partial pivoting.  On an
// exactly zero or non-finite pivot: info[e] = layer1 if it was 0, and the
// error word gets ERRBIT_SINGULAR / ERRBIT_NONFINITE.
cudaError_t zinv_f64(const double2* S, int64_t sS, double2* T, int64_t sT, int b, int batch,
                     int32_t* info, int layer1, int* errword, cudaStream_t st);
int zinv_max_block();

// D[e] = s_e * I - H - extra[e]  with s_e = E[e] (b x b, extra may be null).
cudaError_t assemble_diag(const double2* H, const double2* E, const double2* extra, int64_t sExtra,
                          double2* D, int64_t sD, int b, int batch, cudaStream_t st);

// Strided batched block copy: dst[e] = src[e] (rows x cols, row-major, ld = cols).
cudaError_t copy_blocks(const double2* src, int64_t sSrc, double2* dst, int64_t sDst, int64_t elems,
                        int batch, cudaStream_t st);

// Strided 2-D block copy / update over a batch:
//   dst[e](r, c) = (acc ? dst[e](r, c) : 0) + scale * src[e](r, c)
// src[e] = src + e * sSrc (sSrc = 0 broadcasts), row-major with leading
// dimensions ldSrc / ldDst.
cudaError_t copy2d(const double2* src, int64_t sSrc, int ldSrc, double2* dst, int64_t sDst, int ldDst,
                   int rows, int cols, double scale, int acc, int batch, cudaStream_t st);

// Conjugate-transposed copy / update: dst[e](r, c) = (acc ? dst[e](r, c) : 0)
// + scale * conj(src[e](c, r)), dst rows x cols, src cols x rows.
cudaError_t copy2d_ct(const double2* src, int64_t sSrc, int ldSrc, double2* dst, int64_t sDst, int ldDst,
                      int rows, int cols, double scale, int acc, int batch, cudaStream_t st);

// dst[e] = zeros(rows x cols) with ones at (i, off + i) (cols_mode) or
// (off + i, i) (rows mode), i = 0 .. nid-1.
cudaError_t set_eye(double2* dst, int64_t sDst, int ld, int rows, int cols, int off, int nid, int rows_mode,
                    int batch, cudaStream_t st);

// dst[e](i, i) += scale * s[e] for i < n (s: per-energy complex scalars, stride sS).
cudaError_t add_diag(double2* dst, int64_t sDst, int ld, int n, const double2* s, int64_t sS, double scale,
                     int batch, cudaStream_t st);

// dst[e] += scale * E[e] * src[e]  (rows x cols, leading dimension ld, FP64).
cudaError_t axpy_scalar(double2* dst, int64_t sDst, const double2* src, int64_t sSrc, const double2* E,
                        double scale, int rows, int cols, int ld, int batch, cudaStream_t st);

// dst[e] = c0 x0[e] + c1 x1[e] + c2 x2[e] + c3 x3[e] over n contiguous elements
// (x_k[e] = x_k + e * s_k; null sources are skipped; dst may alias none of them).
cudaError_t lincomb(double2* dst, int64_t sDst, int64_t n, int batch, const double2* x0, int64_t s0, double c0,
                    const double2* x1, int64_t s1, double c1, const double2* x2, int64_t s2, double c2,
                    const double2* x3, int64_t s3, double c3, cudaStream_t st);

// Block copies between a block n-diagonal band and the band of its fused
// block tridiagonal form over a batch (map: 7 int64 per block, see
// negf_misc.cu); dir 0: original -> fused, 1: fused -> original.
cudaError_t band_remap(const double2* src, int64_t sSrc, double2* dst, int64_t sDst, const int64_t* map, int nblk,
                       int batch, int dir, cudaStream_t st);

// info[e] from a fused sub-plan's (super-layer -> its first layer) for e < n,
// and the sub-plan's error word folded into err (and cleared).
cudaError_t fold_fused_status(int32_t* info, const int32_t* sub_info, int n, int w, int* err, int* sub_err,
                              cudaStream_t st);

// D[e] = I (b x b).
cudaError_t set_identity(double2* D, int64_t sD, int b, int batch, cudaStream_t st);

// Gam[e] = i (Sig[e] - Sig[e]^H)   (b x b).
cudaError_t gamma_from_sigma(const double2* sig, int64_t sSig, double2* gam, int64_t sGam, int b,
                             int batch, cudaStream_t st);

// T[e] (+)= scale * Re sum_ij P[e]_ij Q[e]_ji  for P rows x cols, Q cols x rows.
cudaError_t trace_prod(const double2* P, int64_t sP, const double2* Q, int64_t sQ, int rows, int cols,
                       double* T, int batch, double scale, int accumulate, cudaStream_t st);

// dst(r, c) = (acc ? dst(r, c) : 0) + scale * sum_e w[e] S_e(r, c) over nE
// energies, S_e = src[e] (ct = 0) or src[e]^H (ct = 1); w nullable (= 1).
cudaError_t reduce_energies(const double2* src, int64_t sSrc, int ldSrc, int nE, const double* w, double2* dst,
                            int ldDst, int rows, int cols, double2 scale, int acc, int ct, cudaStream_t st);

// out[e] (+)= sum |A[e]_k|^2 over n contiguous elements.
cudaError_t frob2(const double2* A, int64_t sA, int64_t n, double* out, int batch, int accumulate, cudaStream_t st);

// out[e] = sum |A[e]_k - B[e]_k|^2 over n contiguous elements.
cudaError_t frob2_diff(const double2* A, int64_t sA, const double2* B, int64_t sB, int64_t n, double* out, int batch,
                       cudaStream_t st);

// out[e] = sqrt(out[e] * scale).
cudaError_t sqrt_scale(double* out, int n, double scale, cudaStream_t st);

}  // namespace negf
