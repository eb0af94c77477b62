// Stream-like particle update for calibration: the particle-only benchmark of
// the paper's memory-throughput experiment (Section 6, "Memory throughput").
// Per time step every particle position is advanced by one explicit Euler
// step, reflected at the walls of the unit box, and written back in place;
// no grid, no reordering.  It bounds what any particle step can reach on the
// same memory system.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/pic.h"
#include "launch.hpp"

namespace pic {
namespace {

// One step for every particle: y = x + v dt; y < 0 -> -y, y > 1 -> 2 - y,
// with the velocity component negated on reflection.  Structure of arrays
// x[a][n], v[a][n]; grid-stride over particles.
template <typename T, int D>
__global__ void k_stream_step(T *__restrict__ x, T *__restrict__ v, int64_t n, T dt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const T xi = x[a * n + p], vi = v[a * n + p];
      T y = xi + vi * dt;
      if (y < (T)0) {
        y = -y;
        v[a * n + p] = -vi;
      } else if (y > (T)1) {
        y = (T)2 - y;
        v[a * n + p] = -vi;
      }
      x[a * n + p] = y;
    }
  }
}

template <typename T> struct Vec16;
template <> struct Vec16<float> { using V = float4; static constexpr int K = 4; };
template <> struct Vec16<double> { using V = double2; static constexpr int K = 2; };

template <typename T>
__device__ __forceinline__ void reflect(T &y, T &v, bool &flip) {
  flip = false;
  if (y < (T)0) {
    y = -y;
    v = -v;
    flip = true;
  } else if (y > (T)1) {
    y = (T)2 - y;
    v = -v;
    flip = true;
  }
}

// The same step, 16 bytes per thread and row at a time (rows 16-byte aligned:
// n a multiple of the vector width); the same arithmetic per element.
template <typename T, int D>
__global__ void k_stream_step16(T *__restrict__ x, T *__restrict__ v, int64_t n, T dt) {
  using VT = typename Vec16<T>::V;
  constexpr int K = Vec16<T>::K;
  const int64_t nv = n / K, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      VT *xp = reinterpret_cast<VT *>(x + a * n) + i;
      VT *vp = reinterpret_cast<VT *>(v + a * n) + i;
      VT xv = *xp, vv = *vp;
      T *xe = reinterpret_cast<T *>(&xv), *ve = reinterpret_cast<T *>(&vv);
      bool any = false;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        T y = xe[k] + ve[k] * dt;
        bool f;
        reflect(y, ve[k], f);
        any |= f;
        xe[k] = y;
      }
      *xp = xv;
      if (any) *vp = vv;
    }
  }
}

template <typename T>
void launch_stream(int d, T *x, T *v, int64_t n, T dt, cudaStream_t s, int sms) {
  const int threads = 512;
  const bool vec = n % Vec16<T>::K == 0 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)v & 15) == 0;
  const int64_t work = vec ? n / Vec16<T>::K : n;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, (int64_t)sms * 4));
  if (vec) {
    if (d == 3) k_stream_step16<T, 3><<<grid, threads, 0, s>>>(x, v, n, dt);
    else k_stream_step16<T, 2><<<grid, threads, 0, s>>>(x, v, n, dt);
  } else {
    if (d == 3) k_stream_step<T, 3><<<grid, threads, 0, s>>>(x, v, n, dt);
    else k_stream_step<T, 2><<<grid, threads, 0, s>>>(x, v, n, dt);
  }
  count_launches(1);
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" int pic_stream_step(int32_t d, int32_t precision, void *x, void *v, int64_t n, double dt, int32_t steps,
                               void *stream) {
  if ((d != 2 && d != 3) || (precision != PIC_FP64 && precision != PIC_FP32_SPLIT) || n < 0 || steps < 0 ||
      (n > 0 && (!x || !v)))
    return PIC_EINVAL;
  if (n == 0 || steps == 0) return PIC_OK;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PIC_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int32_t k = 0; k < steps; ++k) {
    if (precision == PIC_FP64) launch_stream<double>(d, (double *)x, (double *)v, n, dt, s, sms);
    else launch_stream<float>(d, (float *)x, (float *)v, n, (float)dt, s, sms);
  }
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
