// Device-side helpers shared by the kernels of libnegf.so.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace negf {

// Device error word bits (folded by negf_sync into a negf_status).
enum : int { ERRBIT_SINGULAR = 1, ERRBIT_NONFINITE = 2, ERRBIT_TIMEOUT = 4 };

struct cplx { double re, im; };

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a - f * x
__device__ __forceinline__ double2 cfnms(double2 a, double2 f, double2 x) {
  a.x = fma(-f.x, x.x, a.x);
  a.x = fma(f.y, x.y, a.x);
  a.y = fma(-f.x, x.y, a.y);
  a.y = fma(-f.y, x.x, a.y);
  return a;
}
// Reciprocal of a complex number by Smith's scaled division (R. L. Smith,
// "Algorithm 116: Complex division", CACM 5(8), 1962), which avoids
// overflow in |z|^2.
__device__ __forceinline__ double2 crecip(double2 z) {
  if (fabs(z.x) >= fabs(z.y)) {
    double r = z.y / z.x;
    double den = z.x + z.y * r;
    return make_double2(1.0 / den, -r / den);
  } else {
    double r = z.x / z.y;
    double den = z.x * r + z.y;
    return make_double2(r / den, -1.0 / den);
  }
}
__device__ __forceinline__ double cabs1(double2 z) { return fabs(z.x) + fabs(z.y); }

}  // namespace negf
