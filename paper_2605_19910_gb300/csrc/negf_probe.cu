// FP64 peak probes: the rates the roofline of the FP64 kernels is taken
// against, measured on the device the library runs on.
//
// The per-block inversion (negf_inv.cu) is scalar FP64 FMA arithmetic and
// the FP64 block product (negf_gemm_f64.cu) runs on the FP64 MMA path
// (mma.sync m8n8k4 f64).  Each probe keeps every FP64 unit of the GPU busy
// with independent dependency chains of that one instruction kind (eight
// accumulators per thread or warp, no memory traffic in the loop) and reports
// the issued flops over the kernel's CUDA-event time.
#include "../../include/negf.h"
#include "negf_common.cuh"
#include "negf_kernels.h"

namespace negf {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

// a <- a x + y on eight independent chains; x, y are runtime values close to
// 1 and 0 so the chains stay finite for any iteration count.
__global__ void __launch_bounds__(PROBE_THREADS) dfma_probe_kernel(double x, double y, int iters, double* sink) {
  double a[PROBE_CHAINS];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = fma(a[j], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) s += a[j];
  if (s == 12345.678 && sink) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the loop alive
}

__device__ __forceinline__ void dmma884_acc(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
}

// D <- A B + D on eight independent m8n8k4 accumulators per warp.
__global__ void __launch_bounds__(PROBE_THREADS) dmma_probe_kernel(double x, double y, int iters, double* sink) {
  double c[PROBE_CHAINS][2];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) c[j][0] = c[j][1] = 0.0;
  const double a = x * (1.0 + 1e-6 * (threadIdx.x & 31)), b = y;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) dmma884_acc(c[j][0], c[j][1], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) s += c[j][0] + c[j][1];
  if (s == 12345.678 && sink) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Even warps run the DFMA chains, odd warps the DMMA chains, with equal flops
// per warp (8x the DFMA trips): whether the two instruction kinds share one
// FP64 unit (about the single-kind rate) or run side by side (about twice).
__global__ void __launch_bounds__(PROBE_THREADS) both_probe_kernel(double x, double y, int iters, double* sink) {
  double s = 0.0;
  if (((threadIdx.x >> 5) & 1) == 0) {
    double a[PROBE_CHAINS];
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
    for (int it = 0; it < 8 * iters; ++it) {
#pragma unroll
      for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = fma(a[j], x, y);
    }
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) s += a[j];
  } else {
    double c[PROBE_CHAINS][2];
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) c[j][0] = c[j][1] = 0.0;
    const double a = x * (1.0 + 1e-6 * (threadIdx.x & 31)), b = y;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int j = 0; j < PROBE_CHAINS; ++j) dmma884_acc(c[j][0], c[j][1], a, b);
    }
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) s += c[j][0] + c[j][1];
  }
  if (s == 12345.678 && sink) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace negf

extern "C" negf_status negf_fp64_peak(int32_t kind, int32_t iters, double* tflops, double* ms_out, void* cuda_stream) {
  if (kind < NEGF_PEAK_DFMA || kind > NEGF_PEAK_BOTH || iters < 1 || !tflops) return NEGF_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return NEGF_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // four 256-thread CTAs per SM: enough warps to keep each FP64 unit fed
  const int blocks = sms * 4;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return NEGF_ERR_CUDA;
  cudaError_t e = cudaEventRecord(a, st);
  if (e == cudaSuccess) {
    if (kind == NEGF_PEAK_DFMA)
      negf::dfma_probe_kernel<<<blocks, negf::PROBE_THREADS, 0, st>>>(0.999999, 1e-7, iters, nullptr);
    else if (kind == NEGF_PEAK_DMMA)
      negf::dmma_probe_kernel<<<blocks, negf::PROBE_THREADS, 0, st>>>(0.999999, 1e-7, iters, nullptr);
    else
      negf::both_probe_kernel<<<blocks, negf::PROBE_THREADS, 0, st>>>(0.999999, 1e-7, iters, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return NEGF_ERR_CUDA;
  const double threads = (double)blocks * negf::PROBE_THREADS;
  // DFMA: 2 flops per lane and chain per iteration; DMMA m8n8k4: 2*8*8*4 =
  // 512 flops per warp instruction, i.e. 16 per lane, per chain and iteration;
  // both: half the warps each, 16 flops per lane and chain per trip either way
  const double per = kind == NEGF_PEAK_DFMA ? 2.0 : 16.0;
  const double flops = per * negf::PROBE_CHAINS * (double)iters * threads;
  *tflops = flops / ((double)t * 1e-3) / 1e12;
  if (ms_out) *ms_out = t;
  return NEGF_OK;
}
