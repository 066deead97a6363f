// Vector kernels of the Lanczos method on the SQH matvec (lowest eigenvalues of H(t) and the
// gap above the ground state along the path, Sec. IV.B): block inner products with FP64
// accumulation in a fixed order, block updates w -= sum_i c_i v_i, and scaling by a device
// scalar.  Basis vectors are rows of one array with leading dimension `ld` elements.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "aqc_internal.h"

namespace aqc {

namespace {

template <typename R>
struct C2of;
template <>
struct C2of<float> {
  using T = float2;
};
template <>
struct C2of<double> {
  using T = double2;
};

constexpr int kLzThreads = 256;

// partials[(i * G + block) * 2 + {0,1}] = sum over the block's elements of conj(v_i) w
template <typename R>
__global__ void __launch_bounds__(kLzThreads) k_dotc_multi(const typename C2of<R>::T* __restrict__ V, uint64_t ld,
                                                           const typename C2of<R>::T* __restrict__ w, uint64_t N,
                                                           double* partials) {
  using C2 = typename C2of<R>::T;
  const uint32_t i = blockIdx.y, G = gridDim.x;
  const C2* v = V + (uint64_t)i * ld;
  double re = 0.0, im = 0.0;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < N; e += (uint64_t)G * blockDim.x) {
    const C2 a = v[e], b = w[e];
    re += (double)a.x * (double)b.x + (double)a.y * (double)b.y;
    im += (double)a.x * (double)b.y - (double)a.y * (double)b.x;
  }
  __shared__ double s_re[kLzThreads / 32], s_im[kLzThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_re[warp] = re;
    s_im[warp] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < kLzThreads / 32; k++) {
      a += s_re[k];
      b += s_im[k];
    }
    partials[((uint64_t)i * G + blockIdx.x) * 2] = a;
    partials[((uint64_t)i * G + blockIdx.x) * 2 + 1] = b;
  }
}

// out[2i], out[2i+1] = sum over blocks (in block order) of partials of vector i; optionally
// accumulates into acc (acc[2i..] += out)
__global__ void k_dot_finish(const double* __restrict__ partials, uint32_t G, uint32_t m, double* out, double* acc) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double a = 0.0, b = 0.0;
  for (uint32_t k = 0; k < G; k++) {
    a += partials[((uint64_t)i * G + k) * 2];
    b += partials[((uint64_t)i * G + k) * 2 + 1];
  }
  out[2 * i] = a;
  out[2 * i + 1] = b;
  if (acc) {
    acc[2 * i] += a;
    acc[2 * i + 1] += b;
  }
}

// w -= sum_i c_i v_i  (c complex, FP64, on the device)
template <typename R>
__global__ void __launch_bounds__(kLzThreads) k_sub_multi(typename C2of<R>::T* __restrict__ w,
                                                          const typename C2of<R>::T* __restrict__ V, uint64_t ld,
                                                          uint32_t m, const double* __restrict__ c, uint64_t N) {
  using C2 = typename C2of<R>::T;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < N; e += (uint64_t)gridDim.x * blockDim.x) {
    double re = (double)w[e].x, im = (double)w[e].y;
    for (uint32_t i = 0; i < m; i++) {
      const C2 v = V[(uint64_t)i * ld + e];
      const double cr = c[2 * i], ci = c[2 * i + 1];
      re -= cr * (double)v.x - ci * (double)v.y;
      im -= cr * (double)v.y + ci * (double)v.x;
    }
    w[e] = C2{(R)re, (R)im};
  }
}

// v = w / sqrt(nrm2[0])
template <typename R>
__global__ void __launch_bounds__(kLzThreads) k_scale_to(typename C2of<R>::T* __restrict__ v,
                                                         const typename C2of<R>::T* __restrict__ w, uint64_t N,
                                                         const double* __restrict__ nrm2) {
  using C2 = typename C2of<R>::T;
  const double s = 1.0 / sqrt(nrm2[0]);
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < N; e += (uint64_t)gridDim.x * blockDim.x) {
    const C2 a = w[e];
    v[e] = C2{(R)((double)a.x * s), (R)((double)a.y * s)};
  }
}

int lz_grid(uint64_t N) {
  uint64_t g = (N + 4095) / 4096;
  if (g > 256) g = 256;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

uint32_t lanczos_dot_blocks(uint64_t N) { return (uint32_t)lz_grid(N); }

cudaError_t launch_dotc_multi(int prec, const void* V, uint64_t ld, uint32_t m, const void* w, uint64_t N,
                              double* partials, double* out, double* acc, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  const dim3 grid((unsigned)lz_grid(N), m);
  if (prec == 0)
    k_dotc_multi<double><<<grid, kLzThreads, 0, s>>>((const double2*)V, ld, (const double2*)w, N, partials);
  else
    k_dotc_multi<float><<<grid, kLzThreads, 0, s>>>((const float2*)V, ld, (const float2*)w, N, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_dot_finish<<<(m + 127) / 128, 128, 0, s>>>(partials, grid.x, m, out, acc);
  return cudaGetLastError();
}

cudaError_t launch_sub_multi(int prec, void* w, const void* V, uint64_t ld, uint32_t m, const double* c, uint64_t N,
                             cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  const int grid = (int)((N + kLzThreads - 1) / kLzThreads < 4096 ? (N + kLzThreads - 1) / kLzThreads : 4096);
  if (prec == 0)
    k_sub_multi<double><<<grid, kLzThreads, 0, s>>>((double2*)w, (const double2*)V, ld, m, c, N);
  else
    k_sub_multi<float><<<grid, kLzThreads, 0, s>>>((float2*)w, (const float2*)V, ld, m, c, N);
  return cudaGetLastError();
}

cudaError_t launch_scale_to(int prec, void* v, const void* w, uint64_t N, const double* nrm2, cudaStream_t s) {
  const int grid = (int)((N + kLzThreads - 1) / kLzThreads < 4096 ? (N + kLzThreads - 1) / kLzThreads : 4096);
  if (prec == 0)
    k_scale_to<double><<<grid, kLzThreads, 0, s>>>((double2*)v, (const double2*)w, N, nrm2);
  else
    k_scale_to<float><<<grid, kLzThreads, 0, s>>>((float2*)v, (const float2*)w, N, nrm2);
  return cudaGetLastError();
}

}  // namespace aqc
