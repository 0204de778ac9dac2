// Small element-wise kernels of the sweep: assembling the diagonal blocks of
// M = E I - H - Sigma (Sec. 2), strided block copies, Gamma = i(Sigma -
// Sigma^H) and the trace reduction of the transmission.
#include <algorithm>

#include "negf_common.cuh"
#include "negf_kernels.h"

namespace negf {

namespace {

__global__ void assemble_diag_kernel(const double2* __restrict__ H, const double2* __restrict__ E,
                                     const double2* __restrict__ extra, int64_t sExtra,
                                     double2* __restrict__ D, int64_t sD, int b) {
  const int e = blockIdx.y;
  const double2 en = E[e];
  const int64_t n = (int64_t)b * b;
  double2* d = D + (int64_t)e * sD;
  const double2* x = extra ? extra + (int64_t)e * sExtra : nullptr;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(idx / b), c = (int)(idx - (int64_t)r * b);
    double2 h = H[idx];
    double2 v = make_double2(-h.x, -h.y);
    if (r == c) { v.x += en.x; v.y += en.y; }
    if (x) { v.x -= x[idx].x; v.y -= x[idx].y; }
    d[idx] = v;
  }
}

__global__ void copy_blocks_kernel(const double2* __restrict__ src, int64_t sSrc, double2* __restrict__ dst,
                                   int64_t sDst, int64_t elems) {
  const int e = blockIdx.y;
  const double2* s = src + (int64_t)e * sSrc;
  double2* d = dst + (int64_t)e * sDst;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < elems;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}

__global__ void gamma_kernel(const double2* __restrict__ sig, int64_t sSig, double2* __restrict__ gam,
                             int64_t sGam, int b) {
  const int e = blockIdx.y;
  const double2* s = sig + (int64_t)e * sSig;
  double2* g = gam + (int64_t)e * sGam;
  const int64_t n = (int64_t)b * b;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(idx / b), c = (int)(idx - (int64_t)r * b);
    double2 a = s[idx];
    double2 t = s[(int64_t)c * b + r];   // (Sigma^H)_{rc} = conj(Sigma_{cr})
    // i * (a - conj(t)) = i * ((a.x - t.x) + i (a.y + t.y))
    g[idx] = make_double2(-(a.y + t.y), a.x - t.x);
  }
}

// One CTA per energy: T[e] = scale * Re sum_ij P_ij Q_ji.
__global__ void trace_prod_kernel(const double2* __restrict__ P, int64_t sP, const double2* __restrict__ Q,
                                  int64_t sQ, int rows, int cols, double* __restrict__ T, double scale,
                                  int accumulate) {
  const int e = blockIdx.x;
  const double2* p = P + (int64_t)e * sP;
  const double2* q = Q + (int64_t)e * sQ;
  double acc = 0.0;
  const int64_t n = (int64_t)rows * cols;
  for (int64_t idx = threadIdx.x; idx < n; idx += blockDim.x) {
    int i = (int)(idx / cols), j = (int)(idx - (int64_t)i * cols);
    double2 a = p[idx];
    double2 c = q[(int64_t)j * rows + i];
    acc = fma(a.x, c.x, acc);
    acc = fma(-a.y, c.y, acc);
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    acc = lane < nw ? red[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) T[e] = (accumulate ? T[e] : 0.0) + scale * acc;
  }
}

// dst(r, c) = (acc ? dst(r, c) : 0) + scale * sum_e w[e] * S_e(r, c), with
// S_e = src[e] (ct = 0) or src[e]^H (ct = 1: element (c, r), conjugated).
// Threads run along the output's contiguous index; each sums its element
// over the energies (reads coalesced per energy).
__global__ void reduce_energies_kernel(const double2* __restrict__ src, int64_t sSrc, int ldSrc, int nE,
                                       const double* __restrict__ w, double2* __restrict__ dst, int ldDst,
                                       int rows, int cols, double2 scale, int acc, int ct) {
  const int64_t n = (int64_t)rows * cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / cols), c = (int)(idx - (int64_t)r * cols);
    const int64_t o = ct ? (int64_t)c * ldSrc + r : (int64_t)r * ldSrc + c;
    double sx = 0.0, sy = 0.0;
    for (int e = 0; e < nE; ++e) {
      const double we = w ? w[e] : 1.0;
      if (we == 0.0) continue;
      const double2 v = src[(int64_t)e * sSrc + o];
      sx = fma(we, v.x, sx);
      sy = fma(we, ct ? -v.y : v.y, sy);
    }
    double2 out = acc ? dst[(int64_t)r * ldDst + c] : make_double2(0.0, 0.0);
    out.x += scale.x * sx - scale.y * sy;
    out.y += scale.x * sy + scale.y * sx;
    dst[(int64_t)r * ldDst + c] = out;
  }
}

__global__ void frob2_kernel(const double2* __restrict__ A, int64_t sA, int64_t n, double* __restrict__ out,
                             int accumulate, const double2* __restrict__ Bm = nullptr, int64_t sB = 0) {
  const int e = blockIdx.x;
  const double2* a = A + (int64_t)e * sA;
  const double2* bb = Bm ? Bm + (int64_t)e * sB : nullptr;
  double acc = 0.0;
  for (int64_t idx = threadIdx.x; idx < n; idx += blockDim.x) {
    double2 v = a[idx];
    if (bb) { const double2 u = bb[idx]; v.x -= u.x; v.y -= u.y; }
    acc = fma(v.x, v.x, acc);
    acc = fma(v.y, v.y, acc);
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    acc = lane < nw ? red[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) out[e] = (accumulate ? out[e] : 0.0) + acc;
  }
}

__global__ void sqrt_scale_kernel(double* __restrict__ out, int n, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = sqrt(out[i] * scale);
}

__global__ void set_identity_kernel(double2* __restrict__ D, int64_t sD, int b) {
  const int e = blockIdx.y;
  double2* d = D + (int64_t)e * sD;
  const int64_t n = (int64_t)b * b;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(idx / b), c = (int)(idx - (int64_t)r * b);
    d[idx] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
}

// dst(r, c) = (acc ? dst(r, c) : 0) + scale * conj(src(c, r))
__global__ void copy2d_ct_kernel(const double2* __restrict__ src, int64_t sSrc, int ldSrc, double2* __restrict__ dst,
                                 int64_t sDst, int ldDst, int rows, int cols, double scale, int acc) {
  const int e = blockIdx.y;
  const double2* sp = src + (int64_t)e * sSrc;
  double2* dp = dst + (int64_t)e * sDst;
  const int64_t n = (int64_t)rows * cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / cols), c = (int)(idx - (int64_t)r * cols);
    const double2 v = sp[(int64_t)c * ldSrc + r];
    double2 o = acc ? dp[(int64_t)r * ldDst + c] : make_double2(0.0, 0.0);
    o.x = fma(scale, v.x, o.x);
    o.y = fma(-scale, v.y, o.y);
    dp[(int64_t)r * ldDst + c] = o;
  }
}

__global__ void copy2d_kernel(const double2* __restrict__ src, int64_t sSrc, int ldSrc, double2* __restrict__ dst,
                              int64_t sDst, int ldDst, int rows, int cols, double scale, int acc) {
  const int e = blockIdx.y;
  const double2* sp = src + (int64_t)e * sSrc;
  double2* dp = dst + (int64_t)e * sDst;
  const int64_t n = (int64_t)rows * cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / cols), c = (int)(idx - (int64_t)r * cols);
    const double2 v = sp[(int64_t)r * ldSrc + c];
    double2 o = acc ? dp[(int64_t)r * ldDst + c] : make_double2(0.0, 0.0);
    o.x = fma(scale, v.x, o.x);
    o.y = fma(scale, v.y, o.y);
    dp[(int64_t)r * ldDst + c] = o;
  }
}

__global__ void set_eye_kernel(double2* __restrict__ dst, int64_t sDst, int ld, int rows, int cols, int off,
                               int nid, int rows_mode) {
  const int e = blockIdx.y;
  double2* dp = dst + (int64_t)e * sDst;
  const int64_t n = (int64_t)rows * cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / cols), c = (int)(idx - (int64_t)r * cols);
    const int i = rows_mode ? r - off : c - off;
    const int j = rows_mode ? c : r;
    const bool one = (i >= 0 && i < nid && i == j);
    dp[(int64_t)r * ld + c] = make_double2(one ? 1.0 : 0.0, 0.0);
  }
}

__global__ void add_diag_kernel(double2* __restrict__ dst, int64_t sDst, int ld, int n, const double2* __restrict__ sv,
                                int64_t sS, double scale) {
  const int e = blockIdx.y;
  double2* dp = dst + (int64_t)e * sDst;
  const double2 v = sv ? sv[(int64_t)e * sS] : make_double2(1.0, 0.0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double2 o = dp[(int64_t)i * ld + i];
    o.x = fma(scale, v.x, o.x);
    o.y = fma(scale, v.y, o.y);
    dp[(int64_t)i * ld + i] = o;
  }
}

__global__ void axpy_scalar_kernel(double2* __restrict__ dst, int64_t sDst, const double2* __restrict__ src,
                                   int64_t sSrc, const double2* __restrict__ E, double scale, int rows, int cols,
                                   int ld) {
  const int e = blockIdx.y;
  double2* d = dst + (int64_t)e * sDst;
  const double2* x = src + (int64_t)e * sSrc;
  const double2 z = make_double2(scale * E[e].x, scale * E[e].y);
  const int64_t n = (int64_t)rows * cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / cols), c = (int)(idx - (int64_t)r * cols);
    const double2 v = x[(int64_t)r * ld + c];
    double2 o = d[(int64_t)r * ld + c];
    o.x = fma(z.x, v.x, fma(-z.y, v.y, o.x));
    o.y = fma(z.x, v.y, fma(z.y, v.x, o.y));
    d[(int64_t)r * ld + c] = o;
  }
}

// dst[e] = sum_k c_k src_k[e] over n contiguous elements (null sources skipped).
struct Lincomb4 {
  const double2* src[4];
  int64_t s[4];
  double c[4];
};

__global__ void lincomb_kernel(Lincomb4 lc, double2* __restrict__ dst, int64_t sDst, int64_t n) {
  const int e = blockIdx.y;
  double2* dp = dst + (int64_t)e * sDst;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double2 o = make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (!lc.src[k]) continue;
      const double2 v = lc.src[k][(int64_t)e * lc.s[k] + idx];
      o.x = fma(lc.c[k], v.x, o.x);
      o.y = fma(lc.c[k], v.y, o.y);
    }
    dp[idx] = o;
  }
}

inline int grid_x_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > 1024 ? 1024 : g));
}

}  // namespace

cudaError_t assemble_diag(const double2* H, const double2* E, const double2* extra, int64_t sExtra,
                          double2* D, int64_t sD, int b, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  dim3 grid(grid_x_for((int64_t)b * b, 256), batch);
  assemble_diag_kernel<<<grid, 256, 0, st>>>(H, E, extra, sExtra, D, sD, b);
  return cudaGetLastError();
}

cudaError_t copy_blocks(const double2* src, int64_t sSrc, double2* dst, int64_t sDst, int64_t elems,
                        int batch, cudaStream_t st) {
  if (batch <= 0 || elems <= 0) return cudaSuccess;
  dim3 grid(grid_x_for(elems, 256), batch);
  copy_blocks_kernel<<<grid, 256, 0, st>>>(src, sSrc, dst, sDst, elems);
  return cudaGetLastError();
}

// Block copies between the band of a block n-diagonal chain and the band of
// its fused block tridiagonal form (Sec. 2.3, block fusing).  map holds 7
// entries per block: offset in the original band, rows, columns, offset of
// the super-block in the fused band, its leading dimension, and the block's
// row / column inside it.  dir 0: original -> fused, dir 1: fused -> original.
__global__ void band_remap_kernel(const double2* __restrict__ src, int64_t sSrc, double2* __restrict__ dst,
                                  int64_t sDst, const int64_t* __restrict__ map, int dir) {
  const int64_t* m = map + 7 * (int64_t)blockIdx.x;
  const int64_t oo = m[0], fo = m[3];
  const int r = (int)m[1], c = (int)m[2], fld = (int)m[4], r0 = (int)m[5], c0 = (int)m[6];
  const double2* sp = src + (int64_t)blockIdx.y * sSrc;
  double2* dp = dst + (int64_t)blockIdx.y * sDst;
  for (int idx = threadIdx.x; idx < r * c; idx += blockDim.x) {
    const int i = idx / c, j = idx - i * c;
    const int64_t oi = oo + idx, fi = fo + (int64_t)(r0 + i) * fld + c0 + j;
    if (dir == 0) dp[fi] = sp[oi];
    else dp[oi] = sp[fi];
  }
}

// info[e] = the first layer of the failing w-layer group (sub_info[e] is the
// failing super-layer, 1-based; 0 = none), and the sub-plan's error word
// folded into the plan's (and cleared).
__global__ void fold_fused_status_kernel(int32_t* __restrict__ info, const int32_t* __restrict__ sub_info, int n,
                                         int w, int* err, int* sub_err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int v = sub_info[i];
    info[i] = v > 0 ? (v - 1) * w + 1 : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int word = *sub_err;
    if (word) {
      atomicOr(err, word);
      *sub_err = 0;
    }
  }
}

cudaError_t copy2d(const double2* src, int64_t sSrc, int ldSrc, double2* dst, int64_t sDst, int ldDst,
                   int rows, int cols, double scale, int acc, int batch, cudaStream_t st) {
  if (batch <= 0 || rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid(grid_x_for((int64_t)rows * cols, 256), batch);
  copy2d_kernel<<<grid, 256, 0, st>>>(src, sSrc, ldSrc, dst, sDst, ldDst, rows, cols, scale, acc);
  return cudaGetLastError();
}

cudaError_t copy2d_ct(const double2* src, int64_t sSrc, int ldSrc, double2* dst, int64_t sDst, int ldDst,
                   int rows, int cols, double scale, int acc, int batch, cudaStream_t st) {
  if (batch <= 0 || rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid(grid_x_for((int64_t)rows * cols, 256), batch);
  copy2d_ct_kernel<<<grid, 256, 0, st>>>(src, sSrc, ldSrc, dst, sDst, ldDst, rows, cols, scale, acc);
  return cudaGetLastError();
}

cudaError_t set_eye(double2* dst, int64_t sDst, int ld, int rows, int cols, int off, int nid, int rows_mode,
                    int batch, cudaStream_t st) {
  if (batch <= 0 || rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid(grid_x_for((int64_t)rows * cols, 256), batch);
  set_eye_kernel<<<grid, 256, 0, st>>>(dst, sDst, ld, rows, cols, off, nid, rows_mode);
  return cudaGetLastError();
}

cudaError_t add_diag(double2* dst, int64_t sDst, int ld, int n, const double2* s, int64_t sS, double scale,
                     int batch, cudaStream_t st) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  dim3 grid(grid_x_for(n, 128), batch);
  add_diag_kernel<<<grid, 128, 0, st>>>(dst, sDst, ld, n, s, sS, scale);
  return cudaGetLastError();
}

cudaError_t axpy_scalar(double2* dst, int64_t sDst, const double2* src, int64_t sSrc, const double2* E,
                        double scale, int rows, int cols, int ld, int batch, cudaStream_t st) {
  if (batch <= 0 || rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid(grid_x_for((int64_t)rows * cols, 256), batch);
  axpy_scalar_kernel<<<grid, 256, 0, st>>>(dst, sDst, src, sSrc, E, scale, rows, cols, ld);
  return cudaGetLastError();
}

cudaError_t lincomb(double2* dst, int64_t sDst, int64_t n, int batch, const double2* x0, int64_t s0, double c0,
                    const double2* x1, int64_t s1, double c1, const double2* x2, int64_t s2, double c2,
                    const double2* x3, int64_t s3, double c3, cudaStream_t st) {
  if (batch <= 0 || n <= 0) return cudaSuccess;
  Lincomb4 lc{{x0, x1, x2, x3}, {s0, s1, s2, s3}, {c0, c1, c2, c3}};
  dim3 grid(grid_x_for(n, 256), batch);
  lincomb_kernel<<<grid, 256, 0, st>>>(lc, dst, sDst, n);
  return cudaGetLastError();
}

cudaError_t set_identity(double2* D, int64_t sD, int b, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  dim3 grid(grid_x_for((int64_t)b * b, 256), batch);
  set_identity_kernel<<<grid, 256, 0, st>>>(D, sD, b);
  return cudaGetLastError();
}

cudaError_t gamma_from_sigma(const double2* sig, int64_t sSig, double2* gam, int64_t sGam, int b,
                             int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  dim3 grid(grid_x_for((int64_t)b * b, 256), batch);
  gamma_kernel<<<grid, 256, 0, st>>>(sig, sSig, gam, sGam, b);
  return cudaGetLastError();
}

cudaError_t trace_prod(const double2* P, int64_t sP, const double2* Q, int64_t sQ, int rows, int cols,
                       double* T, int batch, double scale, int accumulate, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  trace_prod_kernel<<<batch, 256, 0, st>>>(P, sP, Q, sQ, rows, cols, T, scale, accumulate);
  return cudaGetLastError();
}

cudaError_t reduce_energies(const double2* src, int64_t sSrc, int ldSrc, int nE, const double* w, double2* dst,
                            int ldDst, int rows, int cols, double2 scale, int acc, int ct, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const int64_t n = (int64_t)rows * cols;
  reduce_energies_kernel<<<(int)std::min<int64_t>((n + 127) / 128, 4096), 128, 0, st>>>(
      src, sSrc, ldSrc, nE, w, dst, ldDst, rows, cols, scale, acc, ct);
  return cudaGetLastError();
}

cudaError_t frob2(const double2* A, int64_t sA, int64_t n, double* out, int batch, int accumulate, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  frob2_kernel<<<batch, 256, 0, st>>>(A, sA, n, out, accumulate);
  return cudaGetLastError();
}

cudaError_t frob2_diff(const double2* A, int64_t sA, const double2* B, int64_t sB, int64_t n, double* out, int batch,
                       cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  frob2_kernel<<<batch, 256, 0, st>>>(A, sA, n, out, 0, B, sB);
  return cudaGetLastError();
}

cudaError_t sqrt_scale(double* out, int n, double scale, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  sqrt_scale_kernel<<<(n + 255) / 256, 256, 0, st>>>(out, n, scale);
  return cudaGetLastError();
}


cudaError_t band_remap(const double2* src, int64_t sSrc, double2* dst, int64_t sDst, const int64_t* map, int nblk,
                       int batch, int dir, cudaStream_t st) {
  if (nblk <= 0 || batch <= 0) return cudaSuccess;
  for (int b0 = 0; b0 < batch; b0 += 65535) {   // grid.y limit
    const int nb = batch - b0 < 65535 ? batch - b0 : 65535;
    band_remap_kernel<<<dim3(nblk, nb), 256, 0, st>>>(src + (int64_t)b0 * sSrc, sSrc, dst + (int64_t)b0 * sDst, sDst,
                                                     map, dir);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t fold_fused_status(int32_t* info, const int32_t* sub_info, int n, int w, int* err, int* sub_err,
                              cudaStream_t st) {
  const int blocks = n > 0 ? (n + 255) / 256 : 1;
  fold_fused_status_kernel<<<blocks < 1024 ? blocks : 1024, 256, 0, st>>>(info, sub_info, n, w, err, sub_err);
  return cudaGetLastError();
}

}  // namespace negf
