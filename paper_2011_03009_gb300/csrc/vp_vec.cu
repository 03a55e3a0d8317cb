// Field-level vector operations (complex64 arrays on the device) used by the
// full-cascade fixed-point driver and the volume-integral-equation solver, and the
// source term of the full cascade with conjugate products (Eq. 2.5).
#include <cuda_runtime.h>

#include "vp.h"
#include "vp_internal.cuh"

namespace vp {
namespace {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

int vec_grid(long long n) {
  long long b = (n + 255) / 256;
  const long long cap = 152LL * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// out = a x + b y (y may be null: out = a x)
// (no __restrict__: out may alias x or y; each element is read before it is written)
__global__ void axpby_kernel(long long n, float2 a, const float2* x, float2 b, const float2* y, float2* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float2 v = cmulf(a, x[i]);
    if (y) {
      const float2 w = cmulf(b, y[i]);
      v.x += w.x;
      v.y += w.y;
    }
    out[i] = v;
  }
}

// out = x * y (pointwise)
__global__ void mul_kernel(long long n, const float2* x, const float2* y, float2* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = cmulf(x[i], y[i]);
}

// acc[0] + i acc[1] += sum (conj(x) if conj_x else x) * y, FP64 accumulation
__global__ void __launch_bounds__(256) dot_kernel(long long n, const float2* __restrict__ x,
                                                  const float2* __restrict__ y, int conj_x, double* __restrict__ acc) {
  __shared__ double part[2][8];
  double re = 0.0, im = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 a = x[i], b = y[i];
    const double ax = a.x, ay = conj_x ? -(double)a.y : (double)a.y;
    re += ax * b.x - ay * b.y;
    im += ax * b.y + ay * b.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    part[0][threadIdx.x >> 5] = re;
    part[1][threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      re += part[0][w];
      im += part[1][w];
    }
    atomicAdd(&acc[0], re);
    atomicAdd(&acc[1], im);
  }
}

// Eq. 2.5 source of harmonic n from p_1..p_nh:
//   f = C_n [ sum_{m=1}^{n-1} p_m p_{n-m} + 2 sum_{m=n+1}^{nh} p_m conj(p_{m-n}) ]
struct FieldPtrs { const float2* p[kMaxLower]; };

__global__ void source_full_kernel(FieldPtrs fp, int n, int nh, float cn, float2* __restrict__ out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int m = 1; m < n; ++m) {
      const float2 v = cmulf(__ldg(&fp.p[m - 1][i]), __ldg(&fp.p[n - m - 1][i]));
      acc.x += v.x;
      acc.y += v.y;
    }
    for (int m = n + 1; m <= nh; ++m) {
      const float2 b = __ldg(&fp.p[m - n - 1][i]);
      const float2 v = cmulf(__ldg(&fp.p[m - 1][i]), make_float2(b.x, -b.y));
      acc.x += 2.f * v.x;
      acc.y += 2.f * v.y;
    }
    out[i] = make_float2(cn * acc.x, cn * acc.y);
  }
}

}  // namespace

cudaError_t launch_axpby(long long n, float2 a, const float2* x, float2 b, const float2* y, float2* out,
                         cudaStream_t s) {
  axpby_kernel<<<vec_grid(n), 256, 0, s>>>(n, a, x, b, y, out);
  return cudaGetLastError();
}

cudaError_t launch_mul(long long n, const float2* x, const float2* y, float2* out, cudaStream_t s) {
  mul_kernel<<<vec_grid(n), 256, 0, s>>>(n, x, y, out);
  return cudaGetLastError();
}

cudaError_t launch_dot(long long n, const float2* x, const float2* y, int conj_x, double* acc, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  dot_kernel<<<vec_grid(n), 256, 0, s>>>(n, x, y, conj_x, acc);
  return cudaGetLastError();
}

cudaError_t launch_source_full(const float2* const* fields, int n, int nh, float cn, float2* out, long long count,
                               cudaStream_t s) {
  FieldPtrs fp;
  for (int i = 0; i < kMaxLower; ++i) fp.p[i] = i < nh ? fields[i] : nullptr;
  source_full_kernel<<<vec_grid(count), 256, 0, s>>>(fp, n, nh, cn, out, count);
  return cudaGetLastError();
}

}  // namespace vp
