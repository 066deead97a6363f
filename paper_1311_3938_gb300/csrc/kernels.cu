// CUDA kernels of the hot path (sm_103a).
//
//  k_apply<R, MODE>: one tile of the state per CTA.  The tile is the sub-hypercube of the
//    2^n index space spanned by the layout's tile bits [0,c) and [h,h+w) (Layout); the CTA
//    stages the source vector's tile in shared memory, so every Pauli product whose flip
//    mask lies inside the tile bits is a shared-memory gather (Sec. I.A: each product maps
//    |z> to one basis state z^x with a phase).  Diagonal parts (Z strings, clause penalties
//    of Eq. hci / Eq. sat) are computed from the index, never stored.  Products no layout
//    holds ("remote") are gathered from global memory.  The epilogue depends on MODE:
//    partial sum, fused PEC step (Sec. I.B), Runge-Kutta stage, derivative, or energy.
//  Reductions accumulate in FP64 per thread -> warp -> CTA -> last-CTA sum in fixed order,
//  so results are bitwise reproducible.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "aqc_internal.h"

namespace aqc {

template <typename R>
struct Cplx;
template <>
struct Cplx<float> {
  using T = float2;
};
template <>
struct Cplx<double> {
  using T = double2;
};

template <typename R>
struct SFlip {
  uint32_t lx, x, zm, cplx;  // cplx: coefficient has an imaginary part (odd number of Y)
  R cr, ci;                  // effective coefficient coef * w_group * i^ipow
};

template <typename R>
struct SZ {
  uint32_t zm;
  uint32_t pad;
  R c;
};

__device__ __forceinline__ uint32_t tile_base(const Layout& L, uint32_t b) {
  const uint32_t gap = (uint32_t)(L.h - L.c);
  const uint32_t lowpart = b & ((1u << gap) - 1u);
  const uint32_t hipart = gap >= 32 ? 0u : (b >> gap);
  return (lowpart << L.c) | (hipart << (L.h + L.w));
}

__device__ __forceinline__ uint32_t tile_z(const Layout& L, uint32_t j, uint32_t zb) {
  const uint32_t cm = (1u << L.c) - 1u;
  return zb | (j & cm) | ((j >> L.c) << L.h);
}

// warp + CTA reduction of K doubles in fixed order; result valid in thread 0
template <int K>
__device__ __forceinline__ void cta_reduce(double (&v)[K], double* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; k++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; k++) s_red[warp * K + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; k++) {
      double a = 0.0;
      for (int w = 0; w < nw; w++) a += s_red[w * K + k];
      v[k] = a;
    }
  }
}

// Per-CTA partials -> last CTA sums them in CTA order.  Returns true in thread 0 of the last
// CTA, with the totals in v.
template <int K>
__device__ bool grid_reduce(double (&v)[K], double* partials, unsigned* counter, double* s_red) {
  __shared__ bool s_last;
  cta_reduce<K>(v, s_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; k++) partials[(size_t)blockIdx.x * K + k] = v[k];
    __threadfence();
    unsigned ticket = atomicAdd(counter, 1u);
    s_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double a[K];
#pragma unroll
  for (int k = 0; k < K; k++) a[k] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < K; k++) a[k] += __ldcg(&partials[(size_t)b * K + k]);
  }
  cta_reduce<K>(a, s_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = a[k];
    *counter = 0u;
    return true;
  }
  return false;
}

template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_apply(const ApplyParams P) {
  using C2 = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double s_red[8 * 3];

  const Layout L = P.L;
  const uint32_t tsize = 1u << L.t;
  const DevTables* tab = P.tab;
  const int fb = tab->flip_begin[P.layout_index];
  const int nloc = tab->flip_begin[P.layout_index + 1] - fb;
  const int rb = tab->flip_begin[tab->n_layouts];
  const int nrem = P.with_remote ? tab->n_remote : 0;
  const int nz = P.with_diag ? tab->n_z : 0;

  C2* s_p = reinterpret_cast<C2*>(smem);
  SFlip<R>* s_f = reinterpret_cast<SFlip<R>*>(smem + (size_t)tsize * sizeof(C2));
  SZ<R>* s_z = reinterpret_cast<SZ<R>*>(s_f + nloc + nrem);

  // effective coefficients for this evaluation time
  for (int k = threadIdx.x; k < nloc + nrem; k += blockDim.x) {
    const DevFlip d = tab->flips[k < nloc ? fb + k : rb + (k - nloc)];
    const double c = d.coef * P.w[d.group];
    double cr = 0.0, ci = 0.0;
    switch (d.ipow & 3) {
      case 0: cr = c; break;
      case 1: ci = c; break;
      case 2: cr = -c; break;
      default: ci = -c; break;
    }
    SFlip<R> f;
    f.lx = d.lx;
    f.x = d.x;
    f.zm = d.zm;
    f.cplx = (d.ipow & 1);
    f.cr = (R)cr;
    f.ci = (R)ci;
    s_f[k] = f;
  }
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    SZ<R> e;
    e.zm = tab->z[k].zm;
    e.pad = 0;
    e.c = (R)(tab->z[k].coef * P.w[tab->z[k].group]);
    s_z[k] = e;
  }
  R dconst = (R)0;
  if (P.with_diag) dconst = (R)(tab->ident[0] * P.w[0] + tab->ident[1] * P.w[1] + tab->ident[2] * P.w[2]);
  const int ncls = P.with_diag ? tab->n_classes : 0;

  const uint32_t zb = tile_base(L, blockIdx.x);
  const C2* __restrict__ src = reinterpret_cast<const C2*>(P.src);
  for (uint32_t j = threadIdx.x; j < tsize; j += blockDim.x) s_p[j] = src[tile_z(L, j, zb)];
  __syncthreads();

  double red[2] = {0.0, 0.0};
  const R h = (R)P.h;
  for (uint32_t j = threadIdx.x; j < tsize; j += blockDim.x) {
    const uint32_t z = tile_z(L, j, zb);
    const C2 pv = s_p[j];
    R ar = (R)0, ai = (R)0;
    if (P.qin) {
      const C2 q = reinterpret_cast<const C2*>(P.qin)[z];
      ar = q.x;
      ai = q.y;
    }
    if (P.with_diag) {
      R d = dconst;
      for (int k = 0; k < nz; k++) {
        const SZ<R> e = s_z[k];
        d += (__popc(e.zm & z) & 1) ? -e.c : e.c;
      }
      for (int c = 0; c < ncls; c++) {
        const DevClass cl = tab->classes[c];
        int cnt = 0;
        if (cl.pen == 0) {
          for (int k = cl.begin; k < cl.end; k++) cnt += (__popc(tab->clause_mask[k] & z) != 1);
        } else {
          for (int k = cl.begin; k < cl.end; k++) {
            const int o = 1 - __popc(tab->clause_mask[k] & z);
            cnt += o * o;
          }
        }
        d += (R)(cl.scale * P.w[cl.group]) * (R)cnt;
      }
      ar += d * pv.x;
      ai += d * pv.y;
    }
    for (int k = 0; k < nloc + nrem; k++) {
      const SFlip<R> f = s_f[k];
      C2 v;
      if (k < nloc) {
        v = s_p[j ^ f.lx];
      } else {
        v = src[z ^ f.x];
      }
      R cr = f.cr, ci = f.ci;
      if (f.zm && (__popc(f.zm & (z ^ f.x)) & 1)) {
        cr = -cr;
        ci = -ci;
      }
      if (f.cplx) {
        ar += cr * v.x - ci * v.y;
        ai += cr * v.y + ci * v.x;
      } else {
        ar += cr * v.x;
        ai += cr * v.y;
      }
    }

    if (MODE == MODE_PARTIAL) {
      reinterpret_cast<C2*>(P.qout)[z] = C2{ar, ai};
    } else if (MODE == MODE_DERIV) {
      reinterpret_cast<C2*>(P.fout)[z] = C2{ai, -ar};  // -i (ar + i ai)
    } else if (MODE == MODE_ENERGY) {
      red[0] += (double)pv.x * (double)ar + (double)pv.y * (double)ai;
      red[1] += (double)pv.x * (double)ai - (double)pv.y * (double)ar;
    } else if (MODE == MODE_STEP) {
      // f_{n+1} = -i H p_{n+1};  corrector y_{n+1};  predictor p_{n+2}  (Sec. I.B)
      const C2 fn = C2{ai, -ar};
      C2* yv = reinterpret_cast<C2*>(P.y);
      const C2 y0 = yv[z];
      const C2 a = reinterpret_cast<const C2*>(P.f0)[z];
      const C2 b = reinterpret_cast<const C2*>(P.f1)[z];
      const C2 c = reinterpret_cast<const C2*>(P.f2)[z];
      const R h24 = h / (R)24;
      C2 yn, pn;
      yn.x = y0.x + h24 * ((R)9 * fn.x + (R)19 * a.x - (R)5 * b.x + c.x);
      yn.y = y0.y + h24 * ((R)9 * fn.y + (R)19 * a.y - (R)5 * b.y + c.y);
      pn.x = yn.x + h24 * ((R)55 * fn.x - (R)59 * a.x + (R)37 * b.x - (R)9 * c.x);
      pn.y = yn.y + h24 * ((R)55 * fn.y - (R)59 * a.y + (R)37 * b.y - (R)9 * c.y);
      yv[z] = yn;
      reinterpret_cast<C2*>(P.fout)[z] = fn;
      reinterpret_cast<C2*>(P.pout)[z] = pn;
      const double dx = (double)yn.x - (double)pv.x, dy = (double)yn.y - (double)pv.y;
      red[0] += (double)yn.x * (double)yn.x + (double)yn.y * (double)yn.y;
      red[1] += dx * dx + dy * dy;
    } else if (MODE == MODE_RK4) {
      const C2 k = C2{ai, -ar};
      C2* yv = reinterpret_cast<C2*>(P.y);
      C2* acc = reinterpret_cast<C2*>(P.acc);
      C2* ys = reinterpret_cast<C2*>(P.pout);
      const C2 y0 = yv[z];
      if (P.stage == 1) {
        reinterpret_cast<C2*>(P.fout)[z] = k;
        acc[z] = k;
        const R hh = (R)0.5 * h;
        ys[z] = C2{y0.x + hh * k.x, y0.y + hh * k.y};
      } else if (P.stage == 2 || P.stage == 3) {
        C2 a = acc[z];
        a.x += (R)2 * k.x;
        a.y += (R)2 * k.y;
        acc[z] = a;
        const R hh = P.stage == 2 ? (R)0.5 * h : h;
        ys[z] = C2{y0.x + hh * k.x, y0.y + hh * k.y};
      } else {
        C2 a = acc[z];
        a.x += k.x;
        a.y += k.y;
        const R h6 = h / (R)6;
        yv[z] = C2{y0.x + h6 * a.x, y0.y + h6 * a.y};
      }
    }
  }

  if (MODE == MODE_STEP || MODE == MODE_ENERGY) {
    if (grid_reduce<2>(red, P.partials, P.counter, s_red)) {
      if (MODE == MODE_STEP) {
        P.slots[kSlotNorm2] = red[0];
        const double e = (19.0 / 270.0) * sqrt(red[1]);
        P.slots[kSlotLastErr] = e;
        if (!(e <= P.slots[kSlotMaxErr])) P.slots[kSlotMaxErr] = e;  // NaN propagates
      } else {
        P.slots[kSlotDot] = red[0];
        P.slots[kSlotDotIm] = red[1];
      }
    }
  }
}

size_t apply_smem_bytes(int prec, int t, int n_local_flips, int n_remote, int n_z) {
  const size_t amp = prec == 0 ? 16 : 8;
  const size_t fl = prec == 0 ? sizeof(SFlip<double>) : sizeof(SFlip<float>);
  const size_t zz = prec == 0 ? sizeof(SZ<double>) : sizeof(SZ<float>);
  return ((size_t)1 << t) * amp + (size_t)(n_local_flips + n_remote) * fl + (size_t)n_z * zz + 16;
}

template <typename R, int MODE>
static cudaError_t launch_one(const ApplyParams& p, int grid, int smem, cudaStream_t s) {
  static int configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_apply<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  k_apply<R, MODE><<<grid, 256, smem, s>>>(p);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_prec(const ApplyParams& p, int grid, int smem, cudaStream_t s) {
  switch (p.mode) {
    case MODE_PARTIAL: return launch_one<R, MODE_PARTIAL>(p, grid, smem, s);
    case MODE_STEP: return launch_one<R, MODE_STEP>(p, grid, smem, s);
    case MODE_RK4: return launch_one<R, MODE_RK4>(p, grid, smem, s);
    case MODE_DERIV: return launch_one<R, MODE_DERIV>(p, grid, smem, s);
    case MODE_ENERGY: return launch_one<R, MODE_ENERGY>(p, grid, smem, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_apply(int prec, const ApplyParams& p, int grid, int smem, cudaStream_t s) {
  return prec == 0 ? launch_prec<double>(p, grid, smem, s) : launch_prec<float>(p, grid, smem, s);
}

// ---- pointwise kernels ------------------------------------------------------------------
template <typename R>
__global__ void k_init(typename Cplx<R>::T* y, uint64_t N, int kind, uint64_t basis) {
  using C2 = typename Cplx<R>::T;
  const R u = (R)(1.0 / sqrt((double)N));
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    if (kind == 0)
      y[i] = C2{u, (R)0};
    else
      y[i] = C2{(R)(i == basis ? 1 : 0), (R)0};
  }
}

cudaError_t launch_init(int prec, void* y, uint64_t N, int kind, uint64_t basis, cudaStream_t s) {
  const int grid = (int)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
  if (prec == 0)
    k_init<double><<<grid, 256, 0, s>>>((double2*)y, N, kind, basis);
  else
    k_init<float><<<grid, 256, 0, s>>>((float2*)y, N, kind, basis);
  return cudaGetLastError();
}

// p_{n+1} = y_n + h/24 (55 f_n - 59 f_{n-1} + 37 f_{n-2} - 9 f_{n-3})   (AB4 predictor)
template <typename R>
__global__ void k_predict(typename Cplx<R>::T* p, const typename Cplx<R>::T* y, const typename Cplx<R>::T* f3,
                          const typename Cplx<R>::T* f2, const typename Cplx<R>::T* f1,
                          const typename Cplx<R>::T* f0, R h, uint64_t N) {
  using C2 = typename Cplx<R>::T;
  const R h24 = h / (R)24;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    const C2 a = f3[i], b = f2[i], c = f1[i], d = f0[i], yy = y[i];
    C2 r;
    r.x = yy.x + h24 * ((R)55 * a.x - (R)59 * b.x + (R)37 * c.x - (R)9 * d.x);
    r.y = yy.y + h24 * ((R)55 * a.y - (R)59 * b.y + (R)37 * c.y - (R)9 * d.y);
    p[i] = r;
  }
}

cudaError_t launch_predict(int prec, void* p, const void* y, const void* f3, const void* f2, const void* f1,
                           const void* f0, double h, uint64_t N, cudaStream_t s) {
  const int grid = (int)((N + 255) / 256 < 8192 ? (N + 255) / 256 : 8192);
  if (prec == 0)
    k_predict<double><<<grid, 256, 0, s>>>((double2*)p, (const double2*)y, (const double2*)f3, (const double2*)f2,
                                           (const double2*)f1, (const double2*)f0, h, N);
  else
    k_predict<float><<<grid, 256, 0, s>>>((float2*)p, (const float2*)y, (const float2*)f3, (const float2*)f2,
                                          (const float2*)f1, (const float2*)f0, (float)h, N);
  return cudaGetLastError();
}

int reduce_grid(uint64_t N) {
  uint64_t g = (N + 2047) / 2048;
  if (g > 1216) g = 1216;
  if (g < 1) g = 1;
  return (int)g;
}

// ||a||^2 (what = 0) with FP64 accumulation, fixed grid for a given N
template <typename R>
__global__ void __launch_bounds__(256) k_norm2(const typename Cplx<R>::T* a, uint64_t N, double* partials,
                                               unsigned* counter, double* slots) {
  using C2 = typename Cplx<R>::T;
  __shared__ double s_red[8];
  double v[1] = {0.0};
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    const C2 x = a[i];
    v[0] += (double)x.x * (double)x.x + (double)x.y * (double)x.y;
  }
  if (grid_reduce<1>(v, partials, counter, s_red)) slots[kSlotNorm2] = v[0];
}

cudaError_t launch_reduce(int prec, int what, const void* a, uint64_t N, double* partials, unsigned* counter,
                          double* slots, int grid, cudaStream_t s) {
  (void)what;
  if (prec == 0)
    k_norm2<double><<<grid, 256, 0, s>>>((const double2*)a, N, partials, counter, slots);
  else
    k_norm2<float><<<grid, 256, 0, s>>>((const float2*)a, N, partials, counter, slots);
  return cudaGetLastError();
}

template <typename R>
__global__ void k_fidelity(const typename Cplx<R>::T* a, uint64_t w, double* slots) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double x = (double)a[w].x, y = (double)a[w].y;
    slots[kSlotDot] = x * x + y * y;
  }
}

cudaError_t launch_fidelity(int prec, const void* a, uint64_t w, double* slots, cudaStream_t s) {
  if (prec == 0)
    k_fidelity<double><<<1, 32, 0, s>>>((const double2*)a, w, slots);
  else
    k_fidelity<float><<<1, 32, 0, s>>>((const float2*)a, w, slots);
  return cudaGetLastError();
}

}  // namespace aqc
