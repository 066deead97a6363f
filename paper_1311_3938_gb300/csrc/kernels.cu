// CUDA kernels of the hot path (sm_103a).
//
//  k_apply<R, MODE>: one tile of the state per CTA.  The tile is the sub-hypercube of the
//    2^n index space spanned by the layout's tile bits [0,c) and [h,h+w) (Layout); the CTA
//    stages the source vector's tile in shared memory, so every Pauli product whose flip
//    mask lies inside the tile bits is a shared-memory gather (Sec. I.A: each product maps
//    |z> to one basis state z^x with a phase).  Each thread keeps kV points in registers and
//    runs the term loop outside the point loop, so a term's mask and coefficient are read
//    once per kV points.  Diagonal parts (Z strings, clause penalties of Eq. hci / Eq. sat)
//    come from the index; the clause counts of one clause class are cached as one byte per
//    index (k_diag_codes, computed once per Hamiltonian).  Products no layout holds
//    ("remote") are gathered from global memory.  The epilogue depends on MODE: partial sum,
//    fused PEC step (Sec. I.B), Runge-Kutta stage, derivative, or energy.
//  Reductions accumulate in FP64 per thread -> warp -> CTA -> last-CTA sum in fixed order,
//  so results are bitwise reproducible.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "aqc_internal.h"

namespace cg = cooperative_groups;

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
  uint32_t lx, x, zm, zm2;
  R cr, ci;    // effective coefficient coef * w_group * i^ipow
  R cr2, ci2;  // the companion product's (0 if none)
};

// X-string product with a real coefficient: the hot case (driver and XX terms)
template <typename R>
struct PFlip;
template <>
struct PFlip<float> {
  uint32_t lx;
  float c;
};
template <>
struct PFlip<double> {
  uint32_t lx;
  uint32_t pad;
  double c;
};

template <typename R>
struct SZ {
  uint32_t zm;
  uint32_t pad;
  R c;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// dynamic shared memory map of k_apply: [tile][clause bytes][plain flips][general flips][Z strings][reduction]
template <typename R>
struct SmemMap {
  size_t code, pf, gf, zs, red, total;
  __host__ __device__ SmemMap(uint32_t tsize, int np, int ng, int nz) {
    using C2 = typename Cplx<R>::T;
    code = align16((size_t)tsize * sizeof(C2));  // the tile's clause bytes
    pf = align16(code + (size_t)tsize);
    gf = align16(pf + (size_t)np * sizeof(PFlip<R>));
    zs = align16(gf + (size_t)ng * sizeof(SFlip<R>));
    red = align16(zs + (size_t)nz * sizeof(SZ<R>));
    total = red + 8 * 2 * sizeof(double) + 16;
  }
};

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
// CTA, with the totals in v.  s_red holds >= 8*K doubles plus one int flag after them.
template <int K>
__device__ bool grid_reduce(double (&v)[K], double* partials, unsigned* counter, double* s_red) {
  int* s_last = reinterpret_cast<int*>(s_red + 8 * K);
  cta_reduce<K>(v, s_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; k++) partials[(size_t)blockIdx.x * K + k] = v[k];
    __threadfence();
    unsigned ticket = atomicAdd(counter, 1u);
    *s_last = (ticket == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!*s_last) return false;
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

// Clause-by-clause sequence (Eq. kpath) on segment k: sum over clauses j <= k of the sequence
// of pen_j(z), weighted wdone for j < k and wact for j = k.
template <typename R>
__device__ __forceinline__ R clause_sum_step(const DevTables* __restrict__ tab, const DevClass& cl, uint32_t z, int k,
                                             R wdone, R wact) {
  const int m = cl.end - cl.begin;
  const int kk = k < m ? k : m;
  R sum = (R)0;
  for (int j = 1; j <= kk; j++) {
    const int ones = __popc(tab->clause_mask[cl.begin + j - 1] & z);
    const R pen = cl.pen == 0 ? (R)(ones != 1) : (R)((1 - ones) * (1 - ones));
    sum += (j < k ? wdone : wact) * pen;
  }
  return sum;
}

__device__ __forceinline__ int clause_range_count(const DevTables* __restrict__ tab, int pen, int b, int e, uint32_t z) {
  int cnt = 0;
  if (pen == 0) {
    for (int k = b; k < e; k++) cnt += (__popc(tab->clause_mask[k] & z) != 1);
  } else {
    for (int k = b; k < e; k++) {
      const int o = 1 - __popc(tab->clause_mask[k] & z);
      cnt += o * o;
    }
  }
  return cnt;
}

template <typename R>
__device__ __forceinline__ R clause_count(const DevTables* __restrict__ tab, const DevClass& cl, uint32_t z) {
  return (R)clause_range_count(tab, cl.pen, cl.begin, cl.end, z);
}

constexpr int kThreads = 256;

// 16-byte global -> shared copies that do not pass through registers (many in flight per thread)
__device__ __forceinline__ void cp_async16(void* smem_ptr, const void* gptr) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_ptr);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gptr) : "memory");
}
// The same with an L2 eviction-priority policy (createpolicy)
__device__ __forceinline__ void cp_async16_pol(void* smem_ptr, const void* gptr, uint64_t pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_ptr);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gptr), "l"(pol)
               : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
// 16-byte global load / store with an L2 policy (loads bypass L1)
__device__ __forceinline__ float4 ldg16_pol(const void* a, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;\n"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(a), "l"(pol)
               : "memory");
  return v;
}
__device__ __forceinline__ void stg16_pol(void* a, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(a), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
}
// Drop a 128-byte L2 line without writing it back (its contents become undefined).  `dep` is a
// value loaded from the line: the discard issues only after that load has returned.
__device__ __forceinline__ void discard_l2(const void* a, float dep) {
  asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(a), "f"(dep) : "memory");
}
__device__ __forceinline__ void discard_l2(const void* a, double dep) {
  asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(a), "d"(dep) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Everything one tile pass needs, built per CTA from a single-instance launch (ApplyParams) or
// from one batch member (BatchInst).
template <typename R>
struct TileCtx {
  using C2 = typename Cplx<R>::T;
  Layout L;
  uint32_t tsize, tmask;
  int np, npf, nh, ngl, ng, nz, ncls, tcls, stage;
  int hc[3];  // ends of hop classes 0..2 (DevTables::hop_class_end)
  R dconst, wtab, h;
  // h/24 of the PEC corrector and predictor as a sum hi + lo of two state-precision numbers
  // (lo = 0 in FP64): every PEC step scales its increment by h/24, so a step size rounded once
  // to FP32 would be a time-scale error of up to 2^-24 that accumulates over the whole run
  R h24, h24lo;
  int step_k;          // clause-by-clause segment (0: none active)
  R step_wdone, step_wact;
  const DevTables* tab;
  const uint8_t* dcode;
  double w0, w1, w2;
  const C2 *src, *qin, *f0, *f1, *f2;
  C2 *qout, *y, *yout, *fout, *pout, *acc;
  C2* ylo;  // STEP, FP32: low part of y (compensated corrector), nullable
  C2* s_p;
  uint8_t* s_code;
  PFlip<R>* s_pf;
  SFlip<R>* s_gf;
  SZ<R>* s_z;
  double* s_red;
  uint64_t pol_keep, pol_drop;  // L2 policies (evict_last / evict_first) of hinted tile passes
};

// h/24 split into the state precision: hi = h/24 rounded, lo = the rounding residual (FP32 only)
template <typename R>
__device__ __forceinline__ void set_h24(TileCtx<R>& T, double h) {
  const double e = h / 24.0;
  T.h24 = (R)e;
  T.h24lo = sizeof(R) == 8 ? (R)0 : (R)(e - (double)T.h24);
}

__device__ __forceinline__ double pick3(double a, double b, double c, int g) { return g == 0 ? a : (g == 1 ? b : c); }

// Effective coefficients of layout li at weights (w0, w1, w2) into shared memory (once per CTA).
template <typename R>
__device__ __forceinline__ void load_coefficients(TileCtx<R>& T, const DevTables* __restrict__ tab, const Layout& L,
                                                  int li, bool with_diag, bool with_remote, const uint8_t* dcode,
                                                  double w0, double w1, double w2, unsigned char* smem,
                                                  unsigned char* tables = nullptr) {
  T.L = L;
  T.tsize = 1u << (L.t - L.cb);  // indices held by this CTA
  T.tmask = T.tsize - 1u;
  T.tab = tab;
  T.w0 = w0;
  T.w1 = w1;
  T.w2 = w2;
  const int fb = tab->flip_begin[li];
  T.np = tab->plain_count[li];
  T.npf = tab->plain_fast[li];
  T.nh = tab->hop_count[li];
  T.hc[0] = tab->hop_class_end[li][0];
  T.hc[1] = tab->hop_class_end[li][1];
  T.hc[2] = tab->hop_class_end[li][2];
  T.ngl = tab->flip_begin[li + 1] - fb - T.np;
  const int rb = tab->flip_begin[tab->n_layouts];
  const int nrem = with_remote ? tab->n_remote : 0;
  T.ng = T.ngl + nrem;
  T.nz = with_diag ? tab->n_z : 0;
  const SmemMap<R> map(T.tsize, T.np, T.ng, T.nz);
  T.s_p = reinterpret_cast<typename TileCtx<R>::C2*>(smem);
  T.s_code = smem + map.code;
  // coefficient tables after the tile, or in a region of their own (a second layout's tables
  // in a kernel that runs tiles of two layouts)
  unsigned char* tb = tables ? tables - map.pf : smem;
  T.s_pf = reinterpret_cast<PFlip<R>*>(tb + map.pf);
  T.s_gf = reinterpret_cast<SFlip<R>*>(tb + map.gf);
  T.s_z = reinterpret_cast<SZ<R>*>(tb + map.zs);
  T.s_red = reinterpret_cast<double*>(tb + map.red);
  for (int k = threadIdx.x; k < T.np; k += blockDim.x) {
    const DevFlip d = tab->flips[fb + k];
    PFlip<R> f;
    f.lx = d.lx;
    f.c = (R)(d.coef * pick3(w0, w1, w2, d.group));
    T.s_pf[k] = f;
  }
  for (int k = threadIdx.x; k < T.ng; k += blockDim.x) {
    const DevFlip d = tab->flips[k < T.ngl ? fb + T.np + k : rb + (k - T.ngl)];
    // c * i^ipow as (re, im)
    auto phased = [](double c, int ipow, double& cr, double& ci) {
      cr = ci = 0.0;
      switch (ipow & 3) {
        case 0: cr = c; break;
        case 1: ci = c; break;
        case 2: cr = -c; break;
        default: ci = -c; break;
      }
    };
    double cr, ci, cr2 = 0.0, ci2 = 0.0;
    phased(d.coef * pick3(w0, w1, w2, d.group), d.ipow, cr, ci);
    if (d.has2) phased(d.coef2 * pick3(w0, w1, w2, d.group2), d.ipow2, cr2, ci2);
    SFlip<R> f;
    f.lx = k < T.ngl ? d.lx : 0u;
    f.x = d.x;
    f.zm = d.zm;
    f.zm2 = d.has2 ? d.zm2 : 0u;
    f.cr = (R)cr;
    f.ci = (R)ci;
    f.cr2 = (R)cr2;
    f.ci2 = (R)ci2;
    T.s_gf[k] = f;
  }
  for (int k = threadIdx.x; k < T.nz; k += blockDim.x) {
    SZ<R> e;
    e.zm = tab->z[k].zm;
    e.pad = 0;
    e.c = (R)(tab->z[k].coef * pick3(w0, w1, w2, tab->z[k].group));
    T.s_z[k] = e;
  }
  T.dconst = (R)0;
  T.wtab = (R)0;
  T.tcls = -1;
  T.ncls = 0;
  T.dcode = nullptr;
  if (with_diag) {
    T.dconst = (R)(tab->ident[0] * w0 + tab->ident[1] * w1 + tab->ident[2] * w2);
    T.ncls = tab->n_classes;
    if (dcode && tab->table_class >= 0) {
      T.tcls = tab->table_class;
      T.dcode = dcode;
      T.wtab = (R)(tab->classes[T.tcls].scale * pick3(w0, w1, w2, tab->classes[T.tcls].group));
    }
  }
}

// Points of one thread: two "halves" of H consecutive tile indices (16 bytes each: H = 2
// complex64 or 1 complex128), the second half HB = 32 H indices after the first.  Lanes of a warp
// take consecutive halves, so every global and shared access of a warp is 512 contiguous bytes
// (coalesced, bank-conflict free) and moves as 16-byte vectors.  Products flipping only the bits
// inside a half (tile bit 0 for complex64) or the half bit (tile bit log2 HB) are register
// permutations; every other product is one 16-byte shared-memory load per half.
template <typename R>
struct Blk;
template <>
struct Blk<float> {
  static constexpr int H = 2;
};
template <>
struct Blk<double> {
  static constexpr int H = 1;
};

template <typename C2, int H>
__device__ __forceinline__ void ld16(const C2* __restrict__ a, uint32_t i, C2 (&v)[H]) {
  const float4 x = *reinterpret_cast<const float4*>(a + i);
  const C2* xs = reinterpret_cast<const C2*>(&x);
#pragma unroll
  for (int q = 0; q < H; q++) v[q] = xs[q];
}

// the same through L2 only: partial sums written by other CTAs of the same launch
template <typename C2, int H>
__device__ __forceinline__ void ld16cg(const C2* __restrict__ a, uint32_t i, C2 (&v)[H]) {
  const float4 x = __ldcg(reinterpret_cast<const float4*>(a + i));
  const C2* xs = reinterpret_cast<const C2*>(&x);
#pragma unroll
  for (int q = 0; q < H; q++) v[q] = xs[q];
}

template <typename C2, int H>
__device__ __forceinline__ void st16(C2* __restrict__ a, uint32_t i, const C2* v) {
  float4 x;
  C2* xs = reinterpret_cast<C2*>(&x);
#pragma unroll
  for (int q = 0; q < H; q++) xs[q] = v[q];
  *reinterpret_cast<float4*>(a + i) = x;
}

// Global 16-byte accesses of a tile pass.  HINT 0: plain; otherwise with an L2 policy.
template <typename C2, int H, int HINT>
__device__ __forceinline__ void gld16(const C2* __restrict__ a, uint32_t i, C2 (&v)[H], uint64_t pol) {
  if (HINT) {
    const float4 x = ldg16_pol(a + i, pol);
    const C2* xs = reinterpret_cast<const C2*>(&x);
#pragma unroll
    for (int q = 0; q < H; q++) v[q] = xs[q];
  } else {
    ld16<C2, H>(a, i, v);
  }
}
template <typename C2, int H, int HINT>
__device__ __forceinline__ void gst16(C2* __restrict__ a, uint32_t i, const C2* v, uint64_t pol) {
  if (HINT) {
    float4 x;
    C2* xs = reinterpret_cast<C2*>(&x);
#pragma unroll
    for (int q = 0; q < H; q++) xs[q] = v[q];
    stg16_pol(a + i, x, pol);
  } else {
    st16<C2, H>(a, i, v);
  }
}

// One tile: stage the source tile in shared memory, then for every point of the tile compute
// acc = q + diagonal + products, and run the mode epilogue.  rt0/rt1 collect the reduction
// partials of this thread in the state precision.
template <bool CL>
__device__ __forceinline__ void tile_sync() {
  if (CL)
    cg::this_cluster().sync();
  else
    __syncthreads();
}

// Shared memory of CTA `rank` of this cluster (this CTA's own for rank == own rank).
template <typename C2>
__device__ __forceinline__ const C2* cluster_smem(const C2* s, uint32_t rank) {
  return cg::this_cluster().map_shared_rank(s, rank);
}

// hi + lo + inc with the sum of hi and inc taken exactly (two-sum) and folded into lo; returns
// the new hi and leaves the new lo in `lo` (|lo| <= half an ulp of hi)
__device__ __forceinline__ float comp_add(float hi, float& lo, float inc) {
  const float s = hi + inc;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (inc - bp);
  const float l = lo + e;
  const float h = s + l;
  lo = l - (h - s);
  return h;
}
__device__ __forceinline__ double comp_add(double hi, double& lo, double inc) { return hi + inc; }

// HINT (L2 eviction priorities, full tiles only): 0 none; 1 a partial-sum pass whose source
// tile and output are read again soon (kept), 2 a pass whose accesses are all last uses
// (evicted first).  HOPCLS: the hop loop by hop class (one loop per class, compile-time
// register swaps and parities); off in the batched kernel, whose register budget it exceeds.
template <typename R, int MODE, bool CL, int HINT = 0, bool HOPCLS = true, bool COMP = false>
__device__ __forceinline__ void process_tile(const TileCtx<R>& T, uint32_t zb, uint32_t rank, R& rt0, R& rt1) {
  using C2 = typename Cplx<R>::T;
  constexpr int H = Blk<R>::H;
  constexpr int G = 2 * H;
  constexpr uint32_t HM = H - 1;
  constexpr uint32_t HB = 32 * H;
  constexpr bool kNeedY = (MODE == MODE_STEP || MODE == MODE_RK4);
  constexpr bool kNeedF = (MODE == MODE_STEP);
  constexpr bool kComp = (COMP && MODE == MODE_STEP && sizeof(R) == 4);  // FP32 corrector carries y's low part
  const C2 zero2 = C2{(R)0, (R)0};
  const Layout L = T.L;
  const uint32_t tsize = T.tsize, tmask = T.tmask;
  const C2* __restrict__ src = T.src;
  C2* s_p = T.s_p;

  // stage the source tile with asynchronous 16-byte copies: a pair of consecutive indices for
  // complex64 (tile bit 0 is global bit 0), one index for complex128.  In a cluster this CTA
  // stages the indices whose top tile bits equal its rank.
  tile_sync<CL>();  // readers of the previous tile (or of the coefficients' writers) are done
  const uint32_t pbits = (uint32_t)(L.t - L.cb);
  const uint32_t jbase = CL ? (rank << pbits) : 0u;
  const bool code_smem = T.tcls >= 0 && L.c >= 4 && tsize >= 16;
  {
    constexpr uint32_t per16 = 16 / sizeof(C2);  // indices per 16-byte granule
    const uint32_t granules = tsize / per16;
    for (uint32_t g = threadIdx.x; g < granules; g += blockDim.x) {
      const uint32_t j = g * per16;
      if (HINT)
        cp_async16_pol(s_p + j, src + tile_z(L, jbase | j, zb), HINT == 1 ? T.pol_keep : T.pol_drop);
      else
        cp_async16(s_p + j, src + tile_z(L, jbase | j, zb));
    }
    if (code_smem) {  // the clause bytes of the tile, 16 contiguous indices per copy
      for (uint32_t g = threadIdx.x; g < (tsize >> 4); g += blockDim.x) {
        const uint32_t j = g << 4;
        if (HINT)
          cp_async16_pol(T.s_code + j, T.dcode + tile_z(L, jbase | j, zb), T.pol_drop);
        else
          cp_async16(T.s_code + j, T.dcode + tile_z(L, jbase | j, zb));
      }
    }
    cp_async_wait_all();
  }
  tile_sync<CL>();  // every part of the tile is staged

  const bool full = tsize >= 2 * HB;  // every state with more than 6 (complex64) / 5 qubits
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // the partial sum q and the clause bytes of a block are fetched one iteration ahead (software
  // pipelining), so their latency overlaps the previous block's work
  C2 pq[G];
  uint32_t pc[G];
  auto fetch_qc = [&](uint32_t itn) {
    if (!full || itn * 2 * HB >= tsize) return;
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const uint32_t zk = tile_z(L, jbase | ((itn * 2 * HB + k * HB + lane * H) & tmask), zb);
      if (T.qin) {
        C2 t[H];
        if (HINT)
          gld16<C2, H, HINT>(T.qin, zk, t, T.pol_drop);
        else
          ld16cg<C2, H>(T.qin, zk, t);
#pragma unroll
        for (int q = 0; q < H; q++) pq[k * H + q] = t[q];
      }
      if (T.tcls >= 0 && !code_smem) {
        if (H == 2) {
          const uint32_t w2 = *reinterpret_cast<const uint16_t*>(T.dcode + zk);
          pc[k * H] = w2 & 0xffu;
          pc[k * H + (H - 1)] = (w2 >> 8) & 0xffu;
        } else {
          pc[k * H] = T.dcode[zk];
        }
      }
    }
  };
  fetch_qc(warp);
  for (uint32_t it = warp; it * 2 * HB < tsize; it += nwarps) {
    uint32_t jh[2], zh[2];
    jh[0] = (it * 2 * HB + lane * H) & tmask;
    jh[1] = (it * 2 * HB + HB + lane * H) & tmask;
    bool ok[G];
    uint32_t z[G];
#pragma unroll
    for (int k = 0; k < 2; k++) {
      zh[k] = tile_z(L, jbase | jh[k], zb);
#pragma unroll
      for (int q = 0; q < H; q++) {
        const uint32_t jj = it * 2 * HB + k * HB + lane * H + q;
        ok[k * H + q] = jj < tsize;
        z[k * H + q] = full ? zh[k] + q : tile_z(L, jbase | (jj & tmask), zb);
      }
    }
    // 1. pointwise global loads first; they complete while the shared-memory gathers run
    C2 qv[G], y0[G], a[G], b[G], c[G];
    C2 yl[G];  // low part of y (compensated FP32 corrector, COMP)
    if (kComp) {
#pragma unroll
      for (int g = 0; g < G; g++) yl[g] = zero2;
    }
    uint32_t code[G];
    if (full) {
#pragma unroll
      for (int g = 0; g < G; g++) {
        qv[g] = pq[g];
        code[g] = pc[g];
      }
      if (code_smem) {
#pragma unroll
        for (int k = 0; k < 2; k++)
#pragma unroll
          for (int q = 0; q < H; q++) code[k * H + q] = T.s_code[jh[k] + q];
      }
      fetch_qc(it + nwarps);
#pragma unroll
      for (int k = 0; k < 2; k++) {
        C2 t[H];
        if (kNeedY) {
          gld16<C2, H, HINT>(T.y, zh[k], t, T.pol_drop);
#pragma unroll
          for (int q = 0; q < H; q++) y0[k * H + q] = t[q];
        }
        if (kComp) {
          gld16<C2, H, HINT>(T.ylo, zh[k], t, T.pol_drop);
#pragma unroll
          for (int q = 0; q < H; q++) yl[k * H + q] = t[q];
        }
        if (kNeedF) {
          gld16<C2, H, HINT>(T.f0, zh[k], t, T.pol_drop);
#pragma unroll
          for (int q = 0; q < H; q++) a[k * H + q] = t[q];
          gld16<C2, H, HINT>(T.f1, zh[k], t, T.pol_drop);
#pragma unroll
          for (int q = 0; q < H; q++) b[k * H + q] = t[q];
          gld16<C2, H, HINT>(T.f2, zh[k], t, T.pol_drop);
#pragma unroll
          for (int q = 0; q < H; q++) c[k * H + q] = t[q];
        } else if (MODE == MODE_RK4) {
          if (T.stage > 1) {
            ld16<C2, H>(T.acc, zh[k], t);
#pragma unroll
            for (int q = 0; q < H; q++) a[k * H + q] = t[q];
          }
        }
      }
    } else {
#pragma unroll
      for (int g = 0; g < G; g++) {
        qv[g] = (T.qin && ok[g]) ? __ldcg(T.qin + z[g]) : zero2;
        if (kNeedY) y0[g] = ok[g] ? T.y[z[g]] : zero2;
        if (kComp) yl[g] = ok[g] ? T.ylo[z[g]] : zero2;
        if (kNeedF) {
          a[g] = ok[g] ? T.f0[z[g]] : zero2;
          b[g] = ok[g] ? T.f1[z[g]] : zero2;
          c[g] = ok[g] ? T.f2[z[g]] : zero2;
        } else if (MODE == MODE_RK4) {
          a[g] = (ok[g] && T.stage > 1) ? T.acc[z[g]] : zero2;
        }
        code[g] = (T.tcls >= 0 && ok[g]) ? (uint32_t)T.dcode[z[g]] : 0u;
      }
    }
    if (!T.qin) {
#pragma unroll
      for (int g = 0; g < G; g++) qv[g] = zero2;
    }
    // own values of the source
    C2 own[G];
    if (full) {
      C2 t0[H], t1[H];
      ld16<C2, H>(s_p, jh[0], t0);
      ld16<C2, H>(s_p, jh[1], t1);
#pragma unroll
      for (int q = 0; q < H; q++) {
        own[q] = t0[q];
        own[H + q] = t1[q];
      }
    } else {
#pragma unroll
      for (int k = 0; k < 2; k++)
#pragma unroll
        for (int q = 0; q < H; q++) own[k * H + q] = s_p[(jh[k] + q) & tmask];
    }

    // partner values u[g] = s(tile index of point g XOR lx); selects instead of runtime
    // indexing keep everything in registers
    auto gather = [&](uint32_t lx, C2 (&u)[G]) {
      const uint32_t rk = lx >> pbits;  // cluster bits of the flip: partner CTA rank ^ rk
      const uint32_t hi = lx & tmask & ~(HM | HB);
      const bool mh = (lx & HM) != 0, sw = (lx & HB) != 0;
      C2 part[G];
      if (hi == 0 && rk == 0) {
#pragma unroll
        for (int q = 0; q < H; q++) {
          part[q] = sw ? own[H + q] : own[q];
          part[H + q] = sw ? own[q] : own[H + q];
        }
      } else {
        const C2* sp = (CL && rk) ? cluster_smem(s_p, rank ^ rk) : s_p;
        const uint32_t j0 = (sw ? jh[1] : jh[0]) ^ hi, j1 = (sw ? jh[0] : jh[1]) ^ hi;
        if (full) {
          C2 t0[H], t1[H];
          ld16<C2, H>(sp, j0, t0);
          ld16<C2, H>(sp, j1, t1);
#pragma unroll
          for (int q = 0; q < H; q++) {
            part[q] = t0[q];
            part[H + q] = t1[q];
          }
        } else {
#pragma unroll
          for (int q = 0; q < H; q++) {
            part[q] = sp[(j0 + q) & tmask];
            part[H + q] = sp[(j1 + q) & tmask];
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 2; k++) {
        if (H == 2) {
          u[k * H] = mh ? part[k * H + (H - 1)] : part[k * H];
          u[k * H + (H - 1)] = mh ? part[k * H] : part[k * H + (H - 1)];
        } else {
          u[k * H] = part[k * H];
        }
      }
    };

    // 2. X strings with real coefficients.  In FP64 (bound by the FP64 pipe) the accumulators
    //    start from the partial sum of the earlier layouts, one add per component fewer; in FP32
    //    (bound by HBM) the partial sum is added last
    constexpr bool kFp64 = sizeof(R) == 8;
    R ar[G], ai[G];
#pragma unroll
    for (int g = 0; g < G; g++) {
      ar[g] = kFp64 ? qv[g].x : (R)0;
      ai[g] = kFp64 ? qv[g].y : (R)0;
    }
    // products flipping no register-held bit: one 16-byte shared load per half, no selects
    if (full) {
      for (int kk = 0; kk < T.npf; kk++) {
        const PFlip<R> f = T.s_pf[kk];
        const uint32_t rk = f.lx >> pbits, lxl = f.lx & tmask;
        const C2* sp = (CL && rk) ? cluster_smem(s_p, rank ^ rk) : s_p;
        C2 t0[H], t1[H];
        ld16<C2, H>(sp, jh[0] ^ lxl, t0);
        ld16<C2, H>(sp, jh[1] ^ lxl, t1);
#pragma unroll
        for (int q = 0; q < H; q++) {
          ar[q] += f.c * t0[q].x;
          ai[q] += f.c * t0[q].y;
          ar[H + q] += f.c * t1[q].x;
          ai[H + q] += f.c * t1[q].y;
        }
      }
    }
    for (int kk = full ? T.npf : 0; kk < T.np; kk++) {
      const PFlip<R> f = T.s_pf[kk];
      C2 u[G];
      gather(f.lx, u);
#pragma unroll
      for (int g = 0; g < G; g++) {
        ar[g] += f.c * u[g].x;
        ai[g] += f.c * u[g].y;
      }
    }
    // 3a. hops X_iX_j + Y_iY_j: 2c psi(z ^ x) where the two bits of z differ (companion
    //     coefficient c2 = -c after the i^2 phase, so cr - cr2 = 2c).  The thread's points
    //     differ only in the register-held tile bits (pair bit HM, half bit HB), so within a hop
    //     class (which of those bits the hop flips) the partners' register order and the points'
    //     parities relative to point 0 are known at compile time: one parity per hop and thread,
    //     and the coefficient is one of two values per point.
    auto hop_class = [&](auto mh_tag, auto sw_tag, int k0, int k1) {
      constexpr bool MH = decltype(mh_tag)::value, SW = decltype(sw_tag)::value;
      for (int kk = k0; kk < k1; kk++) {
        const SFlip<R> f = T.s_gf[kk];
        const uint32_t hi = f.lx & tmask & ~(HM | HB);
        C2 u[G];
        if (hi == 0u) {  // the hop flips register-held bits only: partners are own points
#pragma unroll
          for (int k = 0; k < 2; k++)
#pragma unroll
            for (int q = 0; q < H; q++) u[k * H + q] = own[(k ^ (SW ? 1 : 0)) * H + (q ^ (MH ? 1 : 0))];
        } else {
          C2 t0[H], t1[H];
          ld16<C2, H>(s_p, (SW ? jh[1] : jh[0]) ^ hi, t0);
          ld16<C2, H>(s_p, (SW ? jh[0] : jh[1]) ^ hi, t1);
#pragma unroll
          for (int q = 0; q < H; q++) {
            u[q] = t0[q ^ (MH ? 1 : 0)];
            u[H + q] = t1[q ^ (MH ? 1 : 0)];
          }
        }
        const bool p0 = (__popc(f.x & z[0]) & 1) != 0;
        const R c2 = f.cr - f.cr2;
        const R cA = p0 ? c2 : (R)0, cB = p0 ? (R)0 : c2;  // parity of point 0, its opposite
#pragma unroll
        for (int k = 0; k < 2; k++)
#pragma unroll
          for (int q = 0; q < H; q++) {
            const int g = k * H + q;
            const R c = ((MH && q) != (SW && k)) ? cB : cA;
            ar[g] += c * u[g].x;
            ai[g] += c * u[g].y;
          }
      }
    };
    if (HOPCLS && full && !CL) {
      hop_class(std::false_type{}, std::false_type{}, 0, T.hc[0]);
      if (H == 2) hop_class(std::true_type{}, std::false_type{}, T.hc[0], T.hc[1]);
      hop_class(std::false_type{}, std::true_type{}, T.hc[1], T.hc[2]);
      if (H == 2) hop_class(std::true_type{}, std::true_type{}, T.hc[2], T.nh);
    } else {
      for (int kk = 0; kk < T.nh; kk++) {
        const SFlip<R> f = T.s_gf[kk];
        C2 u[G];
        gather(f.lx, u);
        const R c2 = f.cr - f.cr2;
#pragma unroll
        for (int g = 0; g < G; g++) {
          const R c = (__popc(f.x & z[g]) & 1) ? c2 : (R)0;
          ar[g] += c * u[g].x;
          ai[g] += c * u[g].y;
        }
      }
    }
    // 3b. general products (Y/Z phases, complex coefficients) and remote products
    for (int kk = T.nh; kk < T.ng; kk++) {
      const SFlip<R> f = T.s_gf[kk];
      C2 u[G];
      if (kk < T.ngl) {
        gather(f.lx, u);
      } else {
#pragma unroll
        for (int g = 0; g < G; g++) u[g] = ok[g] ? src[z[g] ^ f.x] : zero2;
      }
#pragma unroll
      for (int g = 0; g < G; g++) {
        const uint32_t zsrc = z[g] ^ f.x;
        R cr = f.cr, ci = f.ci;
        if (__popc(f.zm & zsrc) & 1) {
          cr = -cr;
          ci = -ci;
        }
        // companion product of the same flip: its phase adds to the coefficient (exact
        // cancellation where the two phases are opposite)
        if (__popc(f.zm2 & zsrc) & 1) {
          cr -= f.cr2;
          ci -= f.ci2;
        } else {
          cr += f.cr2;
          ci += f.ci2;
        }
        ar[g] += cr * u[g].x - ci * u[g].y;
        ai[g] += cr * u[g].y + ci * u[g].x;
      }
    }
    // 4. diagonal and partial sum of the earlier layouts
    const bool with_diag = (T.nz > 0 || T.ncls > 0 || T.dconst != (R)0);
#pragma unroll
    for (int g = 0; g < G; g++) {
      if (with_diag) {
        R d = T.dconst;
        if (T.tcls >= 0) d += T.wtab * (R)code[g];
        for (int cc = 0; cc < T.ncls; cc++) {
          if (cc == T.tcls) continue;
          const DevClass cl = T.tab->classes[cc];
          // a derived class: the cached count of the table class minus its few missing clauses
          // (the same integer as counting every clause)
          const R cnt = cl.stepwise ? clause_sum_step<R>(T.tab, cl, z[g], T.step_k, T.step_wdone, T.step_wact)
                        : (cl.derived && T.tcls >= 0)
                            ? (R)((int)code[g] - clause_range_count(T.tab, cl.pen, cl.dbegin, cl.dend, z[g]))
                            : clause_count<R>(T.tab, cl, z[g]);
          d += (R)(cl.scale * pick3(T.w0, T.w1, T.w2, cl.group)) * cnt;
        }
        for (int k = 0; k < T.nz; k++) {
          const SZ<R> e = T.s_z[k];
          d += (__popc(e.zm & z[g]) & 1) ? -e.c : e.c;
        }
        ar[g] += d * own[g].x;
        ai[g] += d * own[g].y;
      }
      if (!kFp64) {
        ar[g] += qv[g].x;
        ai[g] += qv[g].y;
      }
    }
    // HINT 2: the partial sum is dead after this read; drop its L2 lines instead of writing
    // them back (one lane per 128-byte line: eight lanes of 16 bytes)
    if (HINT == 2 && full && T.qin && (lane & 7u) == 0u) {
#pragma unroll
      for (int k = 0; k < 2; k++) discard_l2(T.qin + zh[k], qv[k * H].x);
    }
    // 5. epilogue
    const R h = T.h;
    // corrector and predictor weights h/24 * (9, 19, -5, 1) and h/24 * (55, -59, 37, -9); in
    // FP64 applied as chains of fused multiply-adds (fewer FP64 instructions)
    const R h24 = kFp64 ? h / (R)24 : T.h24;
    const R h24lo = T.h24lo;
    const R c9 = (R)9 * h24, c19 = (R)19 * h24, c5 = (R)5 * h24;
    const R p55 = (R)55 * h24, p59 = (R)59 * h24, p37 = (R)37 * h24, p9 = (R)9 * h24;
    C2 o1[G], o2[G], o3[G];
#pragma unroll
    for (int g = 0; g < G; g++) {
      if (MODE == MODE_PARTIAL) {
        o1[g] = C2{ar[g], ai[g]};
      } else if (MODE == MODE_DERIV) {
        o1[g] = C2{ai[g], -ar[g]};  // -i (ar + i ai)
      } else if (MODE == MODE_ENERGY) {
        if (ok[g]) {
          rt0 += own[g].x * ar[g] + own[g].y * ai[g];
          rt1 += own[g].x * ai[g] - own[g].y * ar[g];
        }
      } else if (MODE == MODE_STEP) {
        // f_{n+1} = -i H p_{n+1};  corrector y_{n+1};  predictor p_{n+2}  (Sec. I.B)
        const C2 fn = C2{ai[g], -ar[g]};
        C2 yn, pn;
        if (kFp64) {
          yn.x = fma(c9, fn.x, fma(c19, a[g].x, fma(-c5, b[g].x, fma(h24, c[g].x, y0[g].x))));
          yn.y = fma(c9, fn.y, fma(c19, a[g].y, fma(-c5, b[g].y, fma(h24, c[g].y, y0[g].y))));
          pn.x = fma(p55, fn.x, fma(-p59, a[g].x, fma(p37, b[g].x, fma(-p9, c[g].x, yn.x))));
          pn.y = fma(p55, fn.y, fma(-p59, a[g].y, fma(p37, b[g].y, fma(-p9, c[g].y, yn.y))));
        } else {
          // the weighted sums times (hi + lo): h24 * S + h24lo * S with one rounding of the sum
          const R scx = (R)9 * fn.x + (R)19 * a[g].x - (R)5 * b[g].x + c[g].x;
          const R scy = (R)9 * fn.y + (R)19 * a[g].y - (R)5 * b[g].y + c[g].y;
          const R ix = fma(h24, scx, h24lo * scx), iy = fma(h24, scy, h24lo * scy);
          if (kComp) {
            // compensated: (y + y_lo) + increment as an exact two-sum, renormalised, so the
            // rounding of y does not accumulate over the run
            yn.x = comp_add(y0[g].x, yl[g].x, ix);
            yn.y = comp_add(y0[g].y, yl[g].y, iy);
          } else {
            yn.x = y0[g].x + ix;
            yn.y = y0[g].y + iy;
          }
          const R spx = (R)55 * fn.x - (R)59 * a[g].x + (R)37 * b[g].x - (R)9 * c[g].x;
          const R spy = (R)55 * fn.y - (R)59 * a[g].y + (R)37 * b[g].y - (R)9 * c[g].y;
          pn.x = yn.x + fma(h24, spx, h24lo * spx);
          pn.y = yn.y + fma(h24, spy, h24lo * spy);
        }
        o1[g] = yn;
        o2[g] = fn;
        o3[g] = pn;
        if (ok[g]) {
          const R dx = yn.x - own[g].x, dy = yn.y - own[g].y;
          rt0 += yn.x * yn.x + yn.y * yn.y;
          rt1 += dx * dx + dy * dy;
        }
      } else if (MODE == MODE_RK4) {
        const C2 k = C2{ai[g], -ar[g]};
        if (T.stage == 1) {
          o1[g] = k;  // history f_n
          o2[g] = k;  // accumulator
          const R hh = (R)0.5 * h;
          o3[g] = C2{y0[g].x + hh * k.x, y0[g].y + hh * k.y};
        } else if (T.stage == 2 || T.stage == 3) {
          C2 s2 = a[g];
          s2.x += (R)2 * k.x;
          s2.y += (R)2 * k.y;
          o2[g] = s2;
          const R hh = T.stage == 2 ? (R)0.5 * h : h;
          o3[g] = C2{y0[g].x + hh * k.x, y0[g].y + hh * k.y};
        } else {
          C2 s2 = a[g];
          s2.x += k.x;
          s2.y += k.y;
          const R h6 = h / (R)6;
          o1[g] = C2{y0[g].x + h6 * s2.x, y0[g].y + h6 * s2.y};
        }
      }
    }
    // stores
    if (MODE == MODE_ENERGY) continue;
    C2* d1 = MODE == MODE_PARTIAL ? T.qout : (MODE == MODE_DERIV ? T.fout : (MODE == MODE_STEP ? T.yout : nullptr));
    C2* d2 = MODE == MODE_STEP ? T.fout : nullptr;
    C2* d3 = MODE == MODE_STEP ? T.pout : nullptr;
    C2* d4 = kComp ? T.ylo : nullptr;
    if (MODE == MODE_RK4) {
      d1 = T.stage == 1 ? T.fout : (T.stage == 4 ? T.y : nullptr);
      d2 = T.stage <= 3 ? T.acc : nullptr;
      d3 = T.stage <= 3 ? T.pout : nullptr;
    }
    if (full) {
#pragma unroll
      for (int k = 0; k < 2; k++) {
        const uint64_t pol = HINT == 1 ? T.pol_keep : T.pol_drop;
        if (d1) gst16<C2, H, HINT>(d1, zh[k], o1 + k * H, pol);
        if (d2) gst16<C2, H, HINT>(d2, zh[k], o2 + k * H, pol);
        if (d3) gst16<C2, H, HINT>(d3, zh[k], o3 + k * H, pol);
        if (kComp && d4) gst16<C2, H, HINT>(d4, zh[k], yl + k * H, pol);
      }
    } else {
#pragma unroll
      for (int g = 0; g < G; g++) {
        if (!ok[g]) continue;
        if (d1) d1[z[g]] = o1[g];
        if (d2) d2[z[g]] = o2[g];
        if (d3) d3[z[g]] = o3[g];
        if (kComp && d4) d4[z[g]] = yl[g];
      }
    }
  }
}

template <typename R, int MODE, bool CL, bool COMP = false, bool TURN = false>
__global__ void __launch_bounds__(kThreads, (MODE == MODE_PARTIAL && sizeof(R) == 4 && !CL) ? 3 : 2)
    k_apply(const ApplyParams P) {
  using C2 = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  TileCtx<R> T;
  const double w0 = P.wdev ? P.wdev[0] : P.w[0], w1 = P.wdev ? P.wdev[1] : P.w[1], w2 = P.wdev ? P.wdev[2] : P.w[2];
  load_coefficients<R>(T, P.tab, P.L, P.layout_index, P.with_diag != 0, P.with_remote != 0, P.dcode, w0, w1, w2, smem);
  T.stage = P.stage;
  T.h = (R)P.h;
  set_h24(T, P.h);
  T.step_k = P.step_k;
  T.step_wdone = (R)P.step_wdone;
  T.step_wact = (R)P.step_wact;
  T.src = reinterpret_cast<const C2*>(P.src);
  T.qin = reinterpret_cast<const C2*>(P.qin);
  T.qout = reinterpret_cast<C2*>(P.qout);
  T.y = reinterpret_cast<C2*>(P.y);
  T.yout = reinterpret_cast<C2*>(P.yout ? P.yout : P.y);
  T.f0 = reinterpret_cast<const C2*>(P.f0);
  T.f1 = reinterpret_cast<const C2*>(P.f1);
  T.f2 = reinterpret_cast<const C2*>(P.f2);
  T.fout = reinterpret_cast<C2*>(P.fout);
  T.pout = reinterpret_cast<C2*>(P.pout);
  T.acc = reinterpret_cast<C2*>(P.acc);
  T.ylo = reinterpret_cast<C2*>(P.ylo);
  // TURN: the same layout's products (no diagonal, no remote products) at the next weights,
  // applied to the new predictor once a tile's step is done; tables after T's
  TileCtx<R> T2;
  if (TURN) {
    const SmemMap<R> mapA(T.tsize, T.np, T.ng, T.nz);
    const double v0 = P.wdev ? P.wdev[3] : P.w2[0], v1 = P.wdev ? P.wdev[4] : P.w2[1],
                 v2 = P.wdev ? P.wdev[5] : P.w2[2];
    load_coefficients<R>(T2, P.tab, P.L, P.layout_index, false, false, nullptr, v0, v1, v2, smem, smem + mapA.total);
    T2.stage = 0;
    T2.h = (R)P.h;
    set_h24(T2, P.h);
    T2.step_k = 0;
    T2.step_wdone = T2.step_wact = (R)0;
    T2.src = reinterpret_cast<const C2*>(P.pout);
    T2.qin = nullptr;
    T2.qout = reinterpret_cast<C2*>(P.qout);
    T2.y = T2.yout = T2.fout = T2.pout = T2.acc = T2.ylo = nullptr;
    T2.f0 = T2.f1 = T2.f2 = nullptr;
  }

  // reductions: per-thread partials over one tile in the state precision (a few dozen
  // points), promoted to FP64 once per tile; FP64 across tiles, CTAs and the grid
  double red[2] = {0.0, 0.0};
  // persistent CTAs (or clusters): one prologue and one reduction per CTA, tiles taken
  // round-robin
  uint32_t rank = 0, first = blockIdx.x, stride = gridDim.x;
  if (CL) {
    cg::cluster_group cl = cg::this_cluster();
    rank = cl.block_rank();
    first = blockIdx.x / cl.num_blocks();
    stride = gridDim.x / cl.num_blocks();
  }
  for (uint32_t tile = first; tile < P.ntiles; tile += stride) {
    R rt0 = (R)0, rt1 = (R)0;
    process_tile<R, MODE, CL, 0, true, COMP>(T, tile_base(T.L, tile), rank, rt0, rt1);
    red[0] += (double)rt0;
    red[1] += (double)rt1;
    if (TURN) {  // the tile's p_{n+2} was just stored by this CTA: restaged from L2
      R u0 = (R)0, u1 = (R)0;
      process_tile<R, MODE_PARTIAL, false>(T2, tile_base(T.L, tile), 0u, u0, u1);
    }
  }
  if (CL) cg::this_cluster().sync();  // no CTA leaves while others may read its shared memory

  if (MODE == MODE_STEP || MODE == MODE_ENERGY) {
    if (grid_reduce<2>(red, P.partials, P.counter, T.s_red)) {
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

// ---- slab-ordered step (last partial layout + fused step) ---------------------------------
// bits of v deposited, lowest first, into the set bits of mask
__device__ __forceinline__ uint32_t deposit_bits(uint32_t v, uint32_t mask) {
  uint32_t r = 0u;
  for (uint32_t m = mask; m != 0u && v != 0u; m &= m - 1u, v >>= 1) {
    if (v & 1u) r |= m & (0u - m);
  }
  return r;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Work item -> (is the fused step, slab), see SlabParams.
__device__ __forceinline__ void slab_item(const SlabParams& S, uint32_t block, bool& is_step, uint32_t& slab) {
  const uint32_t D = S.lookahead, NS = S.n_slabs;
  if (block < D) {
    is_step = false;
    slab = block;
  } else if (block < D + 2u * (NS - D)) {
    const uint32_t v = (block - D) >> 1;
    is_step = ((block - D) & 1u) != 0u;
    slab = is_step ? v : D + v;
  } else {
    is_step = true;
    slab = NS - D + (block - D - 2u * (NS - D));
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads, 2) k_slab(const SlabParams S) {
  using C2 = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_item;
  TileCtx<R> TS, TP;
  const ApplyParams& A = S.step;
  const ApplyParams& B = S.part;
  load_coefficients<R>(TS, A.tab, A.L, A.layout_index, A.with_diag != 0, A.with_remote != 0, A.dcode, A.w[0], A.w[1],
                       A.w[2], smem);
  const SmemMap<R> mapA(TS.tsize, TS.np, TS.ng, TS.nz);
  load_coefficients<R>(TP, B.tab, B.L, B.layout_index, B.with_diag != 0, B.with_remote != 0, B.dcode, B.w[0], B.w[1],
                       B.w[2], smem, smem + mapA.total);
  TS.stage = TP.stage = 0;
  TS.h = TP.h = (R)A.h;
  set_h24(TS, A.h);
  set_h24(TP, A.h);
  TS.step_k = A.step_k;
  TS.step_wdone = (R)A.step_wdone;
  TS.step_wact = (R)A.step_wact;
  TP.step_k = 0;
  TP.step_wdone = TP.step_wact = (R)0;
  TS.src = TP.src = reinterpret_cast<const C2*>(A.src);
  TS.qin = reinterpret_cast<const C2*>(A.qin);
  TS.y = reinterpret_cast<C2*>(A.y);
  TS.yout = reinterpret_cast<C2*>(A.yout ? A.yout : A.y);
  TS.f0 = reinterpret_cast<const C2*>(A.f0);
  TS.f1 = reinterpret_cast<const C2*>(A.f1);
  TS.f2 = reinterpret_cast<const C2*>(A.f2);
  TS.fout = reinterpret_cast<C2*>(A.fout);
  TS.pout = reinterpret_cast<C2*>(A.pout);
  TS.qout = nullptr;
  TS.acc = nullptr;
  TS.ylo = TP.ylo = nullptr;  // the slab order is not used under y compensation
  TP.qin = reinterpret_cast<const C2*>(B.qin);
  TP.qout = reinterpret_cast<C2*>(B.qout);
  TP.y = TP.yout = nullptr;
  TP.f0 = TP.f1 = TP.f2 = nullptr;
  TP.fout = TP.pout = TP.acc = nullptr;
  TS.pol_keep = TP.pol_keep = policy_evict_last();
  TS.pol_drop = TP.pol_drop = policy_evict_first();

  double red[2] = {0.0, 0.0};
  for (;;) {
    __syncthreads();  // s_item of the previous item has been read by every thread
    if (threadIdx.x == 0) s_item = atomicAdd(S.queue, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= S.n_items) break;
    bool is_step;
    uint32_t slab;
    slab_item(S, item / S.tiles, is_step, slab);
    const uint32_t j = item % S.tiles;
    const uint32_t zs = deposit_bits(slab, S.slab_mask);
    R rt0 = (R)0, rt1 = (R)0;
    if (!is_step) {
      process_tile<R, MODE_PARTIAL, false, 1>(TP, zs | deposit_bits(j, S.free_part), 0u, rt0, rt1);
      __syncthreads();  // every thread's stores of this tile are issued
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(S.done + slab, 1u);
      }
    } else {
      if (threadIdx.x == 0) {
        // every partial tile of this slab was handed out earlier to a running CTA, so the wait
        // ends; the poll limit only guards against a fault elsewhere
        uint32_t polls = 0;
        while (ld_acquire(S.done + slab) < S.tiles) {
          if (++polls > S.spin_limit) {
            A.slots[kSlotFault] = 1.0;
            break;
          }
          __nanosleep(64);
        }
      }
      __syncthreads();
      process_tile<R, MODE_STEP, false, 2>(TS, zs | deposit_bits(j, S.free_step), 0u, rt0, rt1);
      red[0] += (double)rt0;
      red[1] += (double)rt1;
    }
  }
  if (grid_reduce<2>(red, A.partials, A.counter, TS.s_red)) {
    A.slots[kSlotNorm2] = red[0];
    const double e = (19.0 / 270.0) * sqrt(red[1]);
    A.slots[kSlotLastErr] = e;
    if (!(e <= A.slots[kSlotMaxErr])) A.slots[kSlotMaxErr] = e;
    // every other CTA has left its item loop: reset the work counters for the next launch
    *S.queue = 0u;
    for (uint32_t k = 0; k < S.n_slabs; k++) S.done[k] = 0u;
  }
}

// ---- batched stepping -----------------------------------------------------------------
// Schedule weights on the device (same expression as the host side).
__device__ __forceinline__ double batch_weight(const BatchInst& I, double s, int g) {
  return ((I.poly[g][3] * s + I.poly[g][2]) * s + I.poly[g][1]) * s + I.poly[g][0];
}

// One PEC grid step of many independent states per launch.  Each CTA takes one work item
// (member, tile) of layout level `level`; a member whose integration is finished is skipped.
// Level > 0: partial sums into the member's q; level 0: the fused PEC step (as k_apply
// MODE_STEP), with per-member reductions summed by the member's last CTA, which then advances
// the member's step counter.
template <typename R, int NT>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 2 : 1) k_batch(BatchLaunch B) {
  using C2 = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const BatchItem it = B.items[blockIdx.x];
  BatchInst* I = B.insts + it.inst;
  const int64_t n = I->step;
  if (n >= I->nsteps) return;  // finished member: uniform for the whole CTA
  const int level = B.level;
  const int nl = I->nl;
  const double tau = (double)(n + 1) * I->h / I->T;
  const double s = I->s_kind == 1 ? tau * tau * (3.0 - 2.0 * tau) : tau;
  TileCtx<R> T;
  const bool first = (level == nl - 1);  // first layout pass of this member's evaluation
  load_coefficients<R>(T, I->tab, I->layouts[level], level, level == diag_level(nl), first, I->dcode,
                       batch_weight(*I, s, 0), batch_weight(*I, s, 1), batch_weight(*I, s, 2), smem);
  T.stage = 0;
  T.h = (R)I->h;
  set_h24(T, I->h);
  T.step_k = 0;  // clause-by-clause sequences are not batched
  T.step_wdone = T.step_wact = (R)0;
  C2* const* v = reinterpret_cast<C2* const*>(I->vec);
  T.src = v[kVecP];
  T.qin = first ? nullptr : v[kVecQ];
  T.qout = v[kVecQ];
  T.y = T.yout = v[kVecY];
  T.f0 = v[kVecF0 + (int)(n & 3)];
  T.f1 = v[kVecF0 + (int)((n - 1) & 3)];
  T.f2 = v[kVecF0 + (int)((n - 2) & 3)];
  T.fout = v[kVecF0 + (int)((n + 1) & 3)];
  T.pout = v[kVecP];
  T.acc = nullptr;
  T.ylo = nullptr;  // members run the plain corrector (aqc_batch_add refuses y compensation)
  R rt0 = (R)0, rt1 = (R)0;
  if (level > 0) {
    process_tile<R, MODE_PARTIAL, false, 0, false>(T, tile_base(T.L, it.tile), 0u, rt0, rt1);
    return;
  }
  process_tile<R, MODE_STEP, false, 0, false>(T, tile_base(T.L, it.tile), 0u, rt0, rt1);
  double red[2] = {(double)rt0, (double)rt1};
  cta_reduce<2>(red, T.s_red);
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    B.partials[2 * (size_t)blockIdx.x] = red[0];
    B.partials[2 * (size_t)blockIdx.x + 1] = red[1];
    __threadfence();
    const unsigned ticket = atomicAdd(&I->ticket, 1u);
    s_last = (ticket == I->item_end - I->item_begin - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double acc[2] = {0.0, 0.0};
  for (uint32_t k = I->item_begin + threadIdx.x; k < I->item_end; k += blockDim.x) {
    acc[0] += __ldcg(&B.partials[2 * (size_t)k]);
    acc[1] += __ldcg(&B.partials[2 * (size_t)k + 1]);
  }
  cta_reduce<2>(acc, T.s_red);
  if (threadIdx.x == 0) {
    I->norm2 = acc[0];
    const double e = (19.0 / 270.0) * sqrt(acc[1]);
    I->last_err = e;
    if (!(e <= I->max_err)) I->max_err = e;
    I->ticket = 0u;
    I->step = n + 1;
  }
}

size_t apply_smem_bytes(int prec, int t, int n_plain, int n_general, int n_z) {
  const uint32_t tsize = 1u << t;
  return prec == 0 ? SmemMap<double>(tsize, n_plain, n_general, n_z).total
                   : SmemMap<float>(tsize, n_plain, n_general, n_z).total;
}

// Persistent grid: (resident CTAs per SM for this smem size) x SMs, at most one CTA per tile;
// for cluster layouts, the number of clusters that can be resident at once (x cluster size).
template <typename R, int MODE, bool CL, bool COMP, bool TURN>
static cudaError_t grid_for(uint32_t ntiles, int smem, cudaStream_t s, int* grid) {
  static int configured = 0, cached_smem = -1, cached_dev = -1, cached_g = 0;
  auto kern = k_apply<R, MODE, CL, COMP, TURN>;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!(dev == cached_dev && smem == cached_smem)) {
    int g = 0;
    if (CL) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 1u << kClusterBits;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(1u << kClusterBits);
      cfg.blockDim = dim3(kThreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
      if (e != cudaSuccess) return e;
      g = (nclusters < 1 ? 1 : nclusters) << kClusterBits;
    } else {
      int sms = 0, per = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem);
      if (e != cudaSuccess) return e;
      g = sms * (per < 1 ? 1 : per);
    }
    cached_dev = dev;
    cached_smem = smem;
    cached_g = g;
  }
  uint64_t g = (uint64_t)cached_g;
  if (g > (uint64_t)kMaxApplyGrid) g = kMaxApplyGrid;
  if (CL) {
    const uint64_t tiles_ctas = (uint64_t)ntiles << kClusterBits;
    if (g > tiles_ctas) g = tiles_ctas;
    g &= ~(uint64_t)((1u << kClusterBits) - 1u);
  } else if (g > ntiles) {
    g = ntiles;
  }
  *grid = (int)g;
  return cudaSuccess;
}

template <typename R, int MODE, bool CL, bool COMP = false, bool TURN = false>
static cudaError_t launch_one(const ApplyParams& p, int smem, cudaStream_t s) {
  int grid = 0;
  cudaError_t e = grid_for<R, MODE, CL, COMP, TURN>(p.ntiles, smem, s, &grid);
  if (e != cudaSuccess) return e;
  if (p.max_grid > 0 && grid > p.max_grid) {  // whole clusters, at least one
    const int unit = CL ? (1 << kClusterBits) : 1;
    grid = p.max_grid / unit * unit;
    if (grid < unit) grid = unit;
  }
  if (CL) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1u << kClusterBits;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_apply<R, MODE, CL, COMP, TURN>, p);
    if (e != cudaSuccess) return e;
  } else {
    k_apply<R, MODE, CL, COMP, TURN><<<grid, kThreads, smem, s>>>(p);
  }
  return cudaGetLastError();
}

template <typename R, bool CL>
static cudaError_t launch_prec(const ApplyParams& p, int smem, cudaStream_t s) {
  switch (p.mode) {
    case MODE_PARTIAL: return launch_one<R, MODE_PARTIAL, CL>(p, smem, s);
    case MODE_STEP:
      // the compensated corrector (complex64) and the turn of layouts (per-CTA tiles) are
      // instantiations of their own
      if constexpr (!CL) {
        if constexpr (sizeof(R) == 4) {
          if (p.ylo) return p.turn ? launch_one<R, MODE_STEP, CL, true, true>(p, smem, s)
                                   : launch_one<R, MODE_STEP, CL, true, false>(p, smem, s);
        } else {
          if (p.ylo) return cudaErrorInvalidValue;
        }
        if (p.turn) return launch_one<R, MODE_STEP, CL, false, true>(p, smem, s);
      } else {
        if (p.ylo || p.turn) return cudaErrorInvalidValue;
      }
      return launch_one<R, MODE_STEP, CL>(p, smem, s);
    case MODE_RK4: return launch_one<R, MODE_RK4, CL>(p, smem, s);
    case MODE_DERIV: return launch_one<R, MODE_DERIV, CL>(p, smem, s);
    case MODE_ENERGY: return launch_one<R, MODE_ENERGY, CL>(p, smem, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_apply(int prec, const ApplyParams& p, int smem, cudaStream_t s) {
  if (p.L.cb > 0) {
    if (p.L.cb != kClusterBits || prec != 1) return cudaErrorInvalidValue;  // complex64 clusters only
    return launch_prec<float, true>(p, smem, s);
  }
  return prec == 0 ? launch_prec<double, false>(p, smem, s) : launch_prec<float, false>(p, smem, s);
}

size_t table_smem_bytes(int prec, int t, int n_plain, int n_general, int n_z) {
  const uint32_t tsize = 1u << t;
  if (prec == 0) {
    const SmemMap<double> m(tsize, n_plain, n_general, n_z);
    return m.total - m.pf;
  }
  const SmemMap<float> m(tsize, n_plain, n_general, n_z);
  return m.total - m.pf;
}

template <typename R>
static cudaError_t launch_slab_t(const SlabParams& p, int smem, cudaStream_t s) {
  static int configured = 0, cached_smem = -1, cached_dev = -1, cached_g = 0;
  auto kern = k_slab<R>;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!(dev == cached_dev && smem == cached_smem)) {
    int sms = 0, per = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    cached_dev = dev;
    cached_smem = smem;
    cached_g = sms * (per < 1 ? 1 : per);
  }
  int g = cached_g > kMaxApplyGrid ? kMaxApplyGrid : cached_g;
  if ((uint32_t)g > p.n_items) g = (int)p.n_items;
  kern<<<g, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_slab(int prec, const SlabParams& p, int smem, cudaStream_t s) {
  if (p.part.L.cb != 0 || p.step.L.cb != 0 || p.n_slabs == 0 || p.n_slabs > (uint32_t)kMaxSlabs || p.tiles == 0 ||
      p.lookahead == 0 || p.lookahead > p.n_slabs)
    return cudaErrorInvalidValue;
  return prec == 0 ? launch_slab_t<double>(p, smem, s) : launch_slab_t<float>(p, smem, s);
}

template <typename R, int NT>
static cudaError_t launch_batch_t(const BatchLaunch& b, int nitems, int smem, cudaStream_t s) {
  static int configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_batch<R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  k_batch<R, NT><<<nitems, NT, smem, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_batch(int prec, int threads, const BatchLaunch& b, int nitems, int smem, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (prec == 0) {
    return threads == 128 ? launch_batch_t<double, 128>(b, nitems, smem, s) : launch_batch_t<double, 256>(b, nitems, smem, s);
  }
  return threads == 128 ? launch_batch_t<float, 128>(b, nitems, smem, s) : launch_batch_t<float, 256>(b, nitems, smem, s);
}

// per-index clause counts of one class (computed once per Hamiltonian)
__global__ void k_diag_codes(uint8_t* out, uint64_t N, const DevTables* tab, int cls) {
  const DevClass cl = tab->classes[cls];
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (uint8_t)clause_count<float>(tab, cl, (uint32_t)i);
}

cudaError_t launch_diag_codes(uint8_t* out, uint64_t N, const DevTables* tab, int cls, cudaStream_t s) {
  const int grid = (int)((N + 255) / 256 < 8192 ? (N + 255) / 256 : 8192);
  k_diag_codes<<<grid, 256, 0, s>>>(out, N, tab, cls);
  return cudaGetLastError();
}

// ---- pointwise kernels ------------------------------------------------------------------
// kind 0: uniform 1/sqrt(N) (|S>, Sec. II.A.1); 1: |basis>; 2: Dicke state of Hamming weight
// `basis` (Eq. initstate), amplitude `amp` = C(n, basis)^(-1/2) on every index of that weight
template <typename R>
__global__ void k_init(typename Cplx<R>::T* y, uint64_t N, int kind, uint64_t basis, double amp) {
  using C2 = typename Cplx<R>::T;
  const R u = (R)(1.0 / sqrt((double)N));
  const R a = (R)amp;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    if (kind == 0)
      y[i] = C2{u, (R)0};
    else if (kind == 1)
      y[i] = C2{(R)(i == basis ? 1 : 0), (R)0};
    else
      y[i] = C2{(uint64_t)__popcll(i) == basis ? a : (R)0, (R)0};
  }
}

cudaError_t launch_init(int prec, void* y, uint64_t N, int kind, uint64_t basis, double amp, cudaStream_t s) {
  const int grid = (int)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
  if (prec == 0)
    k_init<double><<<grid, 256, 0, s>>>((double2*)y, N, kind, basis, amp);
  else
    k_init<float><<<grid, 256, 0, s>>>((float2*)y, N, kind, basis, amp);
  return cudaGetLastError();
}

// dst[z] = src[M(z)] for a permutation M of the index bits, M(z) = OR_b tab[b][byte b of z]
// (qubit relabelling: the state lives in the library's bit order, callers see qubit order)
template <typename R>
__global__ void k_permute_bits(typename Cplx<R>::T* __restrict__ dst, const typename Cplx<R>::T* __restrict__ src,
                               uint64_t N, const uint32_t* __restrict__ tab) {
  __shared__ uint32_t s_tab[4 * 256];
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) s_tab[i] = tab[i];
  __syncthreads();
  for (uint64_t z = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; z < N; z += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t zz = (uint32_t)z;
    const uint32_t m = s_tab[zz & 255u] | s_tab[256 + ((zz >> 8) & 255u)] | s_tab[512 + ((zz >> 16) & 255u)] |
                       s_tab[768 + (zz >> 24)];
    dst[z] = src[m];
  }
}

cudaError_t launch_permute(int prec, void* dst, const void* src, uint64_t N, const uint32_t* tab, cudaStream_t s) {
  const int grid = (int)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
  if (prec == 0)
    k_permute_bits<double><<<grid, 256, 0, s>>>((double2*)dst, (const double2*)src, N, tab);
  else
    k_permute_bits<float><<<grid, 256, 0, s>>>((float2*)dst, (const float2*)src, N, tab);
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

// ---- bounded wait (the give-up path of the library's inter-CTA and copy waits) -------------
// One thread polls `flag` (acquire loads, ~1 us apart) until it is nonzero or `polls` polls have
// passed; giving up sets slots[kSlotFault], as the TMA and slab waits do.
__global__ void k_wait_flag(const unsigned* flag, int64_t polls, double* slots) {
  if (threadIdx.x != 0) return;
  for (int64_t i = 0; i < polls; i++) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(flag) : "memory");
    if (v != 0u) return;
    __nanosleep(1000);
  }
  slots[kSlotFault] = 1.0;
}

cudaError_t launch_wait_flag(const unsigned* flag, int64_t polls, double* slots, cudaStream_t s) {
  k_wait_flag<<<1, 32, 0, s>>>(flag, polls, slots);
  return cudaGetLastError();
}

// ---- FP64 FMA throughput (the denominator of the complex128 step's ALU roofline) -------
__device__ double g_fma_sink;

// kFmaChains independent FMA chains per thread (enough to cover the FP64 pipe's latency); the
// result is stored only if it takes a value it never takes, so the chains stay live
constexpr int kFmaChains = 8;
__global__ void __launch_bounds__(256) k_fma64(int iters, double m, double c) {
  double a[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; k++) a[k] = 1.0 + 1e-3 * k + 1e-9 * threadIdx.x;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kFmaChains; k++) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kFmaChains; k++) s += a[k];
  if (s == -1.0) g_fma_sink = s;
}

cudaError_t launch_fma64(int blocks, int iters, cudaStream_t s) {
  k_fma64<<<blocks, 256, 0, s>>>(iters, 0.999999999, 1e-12);
  return cudaGetLastError();
}

int64_t fma64_count(int blocks, int iters) { return (int64_t)blocks * 256 * kFmaChains * iters; }

struct GraphWeights {
  double w[kGraphStepWeights * kMaxGraphSteps];
};

__global__ void k_set_weights(double* dst, const GraphWeights W, int count) {
  const int i = (int)threadIdx.x;
  if (i < count) dst[i] = W.w[i];
}

cudaError_t launch_set_weights(double* dst, const double* w, int count, cudaStream_t s) {
  if (count < 0 || count > kGraphStepWeights * kMaxGraphSteps) return cudaErrorInvalidValue;
  GraphWeights W;
  for (int i = 0; i < count; i++) W.w[i] = w[i];
  for (int i = count; i < kGraphStepWeights * kMaxGraphSteps; i++) W.w[i] = 0.0;
  k_set_weights<<<1, kGraphStepWeights * kMaxGraphSteps, 0, s>>>(dst, W, count);
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
  __shared__ double s_red[8 + 2];
  double v[1] = {0.0};
  R part = (R)0;  // state-precision partial over 16 elements, then FP64
  int cnt = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
    const C2 x = a[i];
    part += x.x * x.x + x.y * x.y;
    if (++cnt == 16) {
      v[0] += (double)part;
      part = (R)0;
      cnt = 0;
    }
  }
  v[0] += (double)part;
  if (grid_reduce<1>(v, partials, counter, s_red)) slots[kSlotNorm2] = v[0];
}

// sum of squares of the 16 bytes at index j: two complex64 or one complex128 amplitude
template <typename R>
struct Sq16;
template <>
struct Sq16<float> {
  static __device__ __forceinline__ float of(const void* base, uint64_t j) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(base) + j);
    return (v.x * v.x + v.y * v.y) + (v.z * v.z + v.w * v.w);
  }
};
template <>
struct Sq16<double> {
  static __device__ __forceinline__ double of(const void* base, uint64_t j) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(base) + j);
    return v.x * v.x + v.y * v.y;
  }
};

// ||a||^2 of a 16-byte-aligned vector: 16-byte loads, four in flight per thread, the state-
// precision sum of each group of four promoted to FP64; the same fixed grid as k_norm2
template <typename R>
__global__ void __launch_bounds__(256) k_norm2_v(const void* a, uint64_t N, double* partials, unsigned* counter,
                                                 double* slots) {
  using C2 = typename Cplx<R>::T;
  constexpr uint64_t A = 16 / sizeof(C2);  // amplitudes per 16-byte load
  __shared__ double s_red[8 + 2];
  double v[1] = {0.0};
  const uint64_t nv = N / A, stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (; j + 3 * stride < nv; j += 4 * stride) {
    const R q0 = Sq16<R>::of(a, j), q1 = Sq16<R>::of(a, j + stride);
    const R q2 = Sq16<R>::of(a, j + 2 * stride), q3 = Sq16<R>::of(a, j + 3 * stride);
    v[0] += (double)((q0 + q1) + (q2 + q3));
  }
  R part = (R)0;
  for (; j < nv; j += stride) part += Sq16<R>::of(a, j);
  if (A == 2 && (N & 1) && blockIdx.x == 0 && threadIdx.x == 0) {  // odd length: the last amplitude
    const C2 x = reinterpret_cast<const C2*>(a)[N - 1];
    part += x.x * x.x + x.y * x.y;
  }
  v[0] += (double)part;
  if (grid_reduce<1>(v, partials, counter, s_red)) slots[kSlotNorm2] = v[0];
}

cudaError_t launch_reduce(int prec, int what, const void* a, uint64_t N, double* partials, unsigned* counter,
                          double* slots, int grid, cudaStream_t s) {
  (void)what;
  const bool aligned = (((uintptr_t)a) & 15u) == 0;  // else one 8-byte (complex64) load per amplitude
  if (prec == 0)
    k_norm2_v<double><<<grid, 256, 0, s>>>(a, N, partials, counter, slots);  // complex128 is 16-byte aligned
  else if (aligned)
    k_norm2_v<float><<<grid, 256, 0, s>>>(a, N, partials, counter, slots);
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
