// Partial-sum pass over a strided tile layout whose products are all X strings with real
// coefficients (the driver term of Eq. Hix and the XX couplings of the nonlinear path) or hops
// X_iX_j + Y_iY_j (Eq. Hixy), complex64 only:
//   q_out(z) = q_in(z) + sum_k c_k [hop_k: bits i_k, j_k of z differ] psi(z ^ x_k)
// for every z of the tile (gather form of the per-qubit action, Sec. I.A).
//
// GB300 structure: one CTA of 512 threads per SM, persistent over tiles.  The 64 KiB source
// tile (2^13 amplitudes) is brought into shared memory by one TMA tensor copy
// (cp.async.bulk.tensor, 4-D map: chunk, gap bits, tile rows, top bits) into one of two buffers,
// completion tracked by an mbarrier, so the next tile streams in while this one is computed.
// Each thread holds 16 amplitudes in registers: pairs (tile bit 0) at 8 positions spanning tile
// bits 6..8.  Products flipping only bits 6..8 are register permutations; all others read one
// 16-byte shared-memory vector per pair, at one base address plus immediate offsets.  The
// partial sum streams through registers: loaded before the tile wait, stored after the flips.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "aqc_internal.h"

namespace aqc {

namespace {

constexpr int kXThreads = 512;
constexpr uint32_t kXTileBytes = (1u << kXTileBits) * 8u;  // complex64 tile
constexpr uint32_t kXRegMask = 0x1c0u;                        // tile bits 6..8: register positions
constexpr uint32_t kXWaitPolls = 1u << 24;                     // mbarrier polls before giving up

struct XFlip {
  uint32_t lx;
  float c;
  uint32_t par;  // hops: the flip mask, whose bits must differ in z; 0 for X strings
  uint32_t pad;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0u;
}

// bounded wait for phase `phase` of the mbarrier; false if it did not complete
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (uint32_t i = 0; i < kXWaitPolls; i++)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1, int c2,
                                            int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fma4(float4& a, float c, const float4& g) {
  a.x = fmaf(c, g.x, a.x);
  a.y = fmaf(c, g.y, a.y);
  a.z = fmaf(c, g.z, a.z);
  a.w = fmaf(c, g.w, a.w);
}

__device__ __forceinline__ float4 swap_pair(const float4& g) { return make_float4(g.z, g.w, g.x, g.y); }

// products flipping register positions only: acc[r] += c * own[r ^ RB]
template <int RB>
__device__ __forceinline__ void reg_flip(float c, const float4 (&own)[8], float4 (&acc)[8]) {
#pragma unroll
  for (int r = 0; r < 8; r++) fma4(acc[r], c, own[r ^ RB]);
}

// other products: acc[r] += c * tile[(jw ^ sx) | ((r ^ RB) << 6)], row = tile + (jw ^ (sx & ~1)) * 8;
// SW: the flip includes the pair bit (tile bit 0), so the two amplitudes of a pair trade places
template <int RB, bool SW>
__device__ __forceinline__ void smem_flip(float c, const unsigned char* row, float4 (&acc)[8]) {
#pragma unroll
  for (int r = 0; r < 8; r++) {
    const float4 g = *reinterpret_cast<const float4*>(row + ((r ^ RB) << 9));
    fma4(acc[r], c, SW ? swap_pair(g) : g);
  }
}

// hops: 2c at output amplitudes whose two flipped bits differ, else 0.  The flip's register
// bits (RB: local bits 6..8, the pair index r) and its pair bit (SW: local bit 0) fix the
// parity of every amplitude of the thread relative to its first one: pair r's first amplitude
// differs by parity(r & RB), its second by that ^ SW.  cA is the coefficient at the parity of
// the thread's first amplitude, cB at the opposite parity, so no per-amplitude parity is left.
template <int R_, int RB>
__device__ __forceinline__ constexpr bool pair_parity() {
  return (((R_ & RB) ^ ((R_ & RB) >> 1) ^ ((R_ & RB) >> 2)) & 1) != 0;
}
template <int RB, bool SW, int R_>
__device__ __forceinline__ void hop_pair(float cA, float cB, const float4& g, float4& a) {
  constexpr bool p = pair_parity<R_, RB>();
  const float c0 = p ? cB : cA, c1 = (p != SW) ? cB : cA;
  a.x = fmaf(c0, g.x, a.x);
  a.y = fmaf(c0, g.y, a.y);
  a.z = fmaf(c1, g.z, a.z);
  a.w = fmaf(c1, g.w, a.w);
}
template <int RB, bool SW>
__device__ __forceinline__ void smem_hop(float cA, float cB, const unsigned char* row, float4 (&acc)[8]) {
  auto one = [&](auto r_tag) {
    constexpr int r = decltype(r_tag)::value;
    const float4 g = *reinterpret_cast<const float4*>(row + ((r ^ RB) << 9));
    hop_pair<RB, SW, r>(cA, cB, SW ? swap_pair(g) : g, acc[r]);
  };
  one(std::integral_constant<int, 0>{});
  one(std::integral_constant<int, 1>{});
  one(std::integral_constant<int, 2>{});
  one(std::integral_constant<int, 3>{});
  one(std::integral_constant<int, 4>{});
  one(std::integral_constant<int, 5>{});
  one(std::integral_constant<int, 6>{});
  one(std::integral_constant<int, 7>{});
}
template <int RB>
__device__ __forceinline__ void reg_hop(float cA, float cB, const float4 (&own)[8], float4 (&acc)[8]) {
  auto one = [&](auto r_tag) {
    constexpr int r = decltype(r_tag)::value;
    hop_pair<RB, false, r>(cA, cB, own[r ^ RB], acc[r]);
  };
  one(std::integral_constant<int, 0>{});
  one(std::integral_constant<int, 1>{});
  one(std::integral_constant<int, 2>{});
  one(std::integral_constant<int, 3>{});
  one(std::integral_constant<int, 4>{});
  one(std::integral_constant<int, 5>{});
  one(std::integral_constant<int, 6>{});
  one(std::integral_constant<int, 7>{});
}

__device__ __forceinline__ double weight_of(const XPartialParams& P, int g) {
  if (P.wdev) return P.wdev[g];
  return g == 0 ? P.w[0] : (g == 1 ? P.w[1] : P.w[2]);
}

__global__ void __launch_bounds__(kXThreads, 1) k_partial_x(const __grid_constant__ XPartialParams P) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // [pad to 1 KiB][tile buffer 0][tile buffer 1][flips][2 mbarriers]
  unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  unsigned char* const buf0 = base;
  unsigned char* const buf1 = base + kXTileBytes;
  const DevTables* tab = P.tab;
  const int fb = tab->flip_begin[P.layout_index];
  const int np = tab->plain_count[P.layout_index] + tab->hop_count[P.layout_index];  // X strings, then hops
  const int npl = tab->plain_count[P.layout_index];
  XFlip* s_f = reinterpret_cast<XFlip*>(base + 2 * kXTileBytes);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(base + 2 * kXTileBytes + ((np * sizeof(XFlip) + 15) & ~(size_t)15));
  const uint32_t bar0 = smem_addr(s_bar), bar1 = smem_addr(s_bar + 1);
  const uint32_t tid = threadIdx.x;
  for (int k = tid; k < np; k += blockDim.x) {
    const DevFlip d = tab->flips[fb + k];
    const bool hop = k >= npl;  // X_iX_j + Y_iY_j: 2c where the bits differ
    s_f[k] = XFlip{d.lx, (float)((hop ? 2.0 : 1.0) * d.coef * weight_of(P, d.group)), hop ? d.x : 0u, 0u};
  }
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  const Layout L = P.L;
  const uint32_t gap = (uint32_t)(L.h - L.c);
  const uint32_t lane = tid & 31u, warp = tid >> 5;
  const uint32_t jw = (warp << 9) | (lane << 1);  // tile position of this thread's first pair
  uint32_t zoff[8];                                 // index offsets of the thread's 8 pairs
#pragma unroll
  for (int r = 0; r < 8; r++) zoff[r] = tile_z(L, jw | ((uint32_t)r << 6), 0u);

  const uint32_t first = blockIdx.x, stride = gridDim.x, ntiles = P.ntiles;
  auto issue = [&](uint32_t tile, int b) {  // thread 0: TMA copy of a tile into buffer b
    const int x1 = (int)(tile & ((1u << gap) - 1u)), x3 = (int)(tile >> gap);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    const uint32_t bb = b ? bar1 : bar0;
    mbar_expect_tx(bb, kXTileBytes);
    if (P.tma_rank == 5)
      tma_load_5d(smem_addr(b ? buf1 : buf0), &P.tmap, bb, 0, 0, x1, 0, x3);
    else
      tma_load_4d(smem_addr(b ? buf1 : buf0), &P.tmap, bb, 0, x1, 0, x3);
  };
  if (tid == 0) {
    if (first < ntiles) issue(first, 0);
    if (first + stride < ntiles) issue(first + stride, 1);
  }
  const float2* __restrict__ qin = reinterpret_cast<const float2*>(P.qin);
  float2* __restrict__ qout = reinterpret_cast<float2*>(P.qout);
  uint32_t k = 0;
  for (uint32_t tile = first; tile < ntiles; tile += stride, k++) {
    const int b = (int)(k & 1u);
    const uint32_t zb = tile_base(L, tile);
    const uint32_t zj = zb | zoff[0];  // index of the thread's first amplitude
    float4 acc[8];
    if (qin) {
#pragma unroll
      for (int r = 0; r < 8; r++) acc[r] = __ldcg(reinterpret_cast<const float4*>(qin + (zb + zoff[r])));
    } else {
#pragma unroll
      for (int r = 0; r < 8; r++) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const bool ok = mbar_wait(b ? bar1 : bar0, (k >> 1) & 1u);
    if (__syncthreads_or(!ok)) {  // uniform: a copy that never completed (not expected)
      if (tid == 0) P.slots[kSlotFault] = 1.0;
      break;
    }
    const unsigned char* t = b ? buf1 : buf0;
    float4 own[8];
#pragma unroll
    for (int r = 0; r < 8; r++) own[r] = *reinterpret_cast<const float4*>(t + ((jw | ((uint32_t)r << 6)) << 3));
    for (int kk = 0; kk < np; kk++) {
      const XFlip f = s_f[kk];
      const uint32_t rb = (f.lx & kXRegMask) >> 6, sx = f.lx & ~kXRegMask;
      if (f.par) {  // hop: one parity per thread (its first amplitude), the rest is fixed by RB, SW
        const bool pb = (__popc(zj & f.par) & 1u) != 0u;
        const float cA = pb ? f.c : 0.f, cB = pb ? 0.f : f.c;
        if (sx == 0u) {
          switch (rb) {
            case 1: reg_hop<1>(cA, cB, own, acc); break;
            case 2: reg_hop<2>(cA, cB, own, acc); break;
            case 3: reg_hop<3>(cA, cB, own, acc); break;
            case 4: reg_hop<4>(cA, cB, own, acc); break;
            case 5: reg_hop<5>(cA, cB, own, acc); break;
            case 6: reg_hop<6>(cA, cB, own, acc); break;
            default: reg_hop<7>(cA, cB, own, acc); break;
          }
        } else {
          const unsigned char* row = t + ((jw ^ (sx & ~1u)) << 3);
          const bool sw = (sx & 1u) != 0u;
          switch (rb | (sw ? 8u : 0u)) {
            case 0: smem_hop<0, false>(cA, cB, row, acc); break;
            case 1: smem_hop<1, false>(cA, cB, row, acc); break;
            case 2: smem_hop<2, false>(cA, cB, row, acc); break;
            case 3: smem_hop<3, false>(cA, cB, row, acc); break;
            case 4: smem_hop<4, false>(cA, cB, row, acc); break;
            case 5: smem_hop<5, false>(cA, cB, row, acc); break;
            case 6: smem_hop<6, false>(cA, cB, row, acc); break;
            case 7: smem_hop<7, false>(cA, cB, row, acc); break;
            case 8: smem_hop<0, true>(cA, cB, row, acc); break;
            case 9: smem_hop<1, true>(cA, cB, row, acc); break;
            case 10: smem_hop<2, true>(cA, cB, row, acc); break;
            case 11: smem_hop<3, true>(cA, cB, row, acc); break;
            case 12: smem_hop<4, true>(cA, cB, row, acc); break;
            case 13: smem_hop<5, true>(cA, cB, row, acc); break;
            case 14: smem_hop<6, true>(cA, cB, row, acc); break;
            default: smem_hop<7, true>(cA, cB, row, acc); break;
          }
        }
        continue;
      }
      if (sx == 0u) {
        switch (rb) {
          case 1: reg_flip<1>(f.c, own, acc); break;
          case 2: reg_flip<2>(f.c, own, acc); break;
          case 3: reg_flip<3>(f.c, own, acc); break;
          case 4: reg_flip<4>(f.c, own, acc); break;
          case 5: reg_flip<5>(f.c, own, acc); break;
          case 6: reg_flip<6>(f.c, own, acc); break;
          default: reg_flip<7>(f.c, own, acc); break;
        }
      } else {
        const unsigned char* row = t + ((jw ^ (sx & ~1u)) << 3);
        const bool sw = (sx & 1u) != 0u;
        switch (rb | (sw ? 8u : 0u)) {
          case 0: smem_flip<0, false>(f.c, row, acc); break;
          case 1: smem_flip<1, false>(f.c, row, acc); break;
          case 2: smem_flip<2, false>(f.c, row, acc); break;
          case 3: smem_flip<3, false>(f.c, row, acc); break;
          case 4: smem_flip<4, false>(f.c, row, acc); break;
          case 5: smem_flip<5, false>(f.c, row, acc); break;
          case 6: smem_flip<6, false>(f.c, row, acc); break;
          case 7: smem_flip<7, false>(f.c, row, acc); break;
          case 8: smem_flip<0, true>(f.c, row, acc); break;
          case 9: smem_flip<1, true>(f.c, row, acc); break;
          case 10: smem_flip<2, true>(f.c, row, acc); break;
          case 11: smem_flip<3, true>(f.c, row, acc); break;
          case 12: smem_flip<4, true>(f.c, row, acc); break;
          case 13: smem_flip<5, true>(f.c, row, acc); break;
          case 14: smem_flip<6, true>(f.c, row, acc); break;
          default: smem_flip<7, true>(f.c, row, acc); break;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 8; r++) *reinterpret_cast<float4*>(qout + (zb + zoff[r])) = acc[r];
    __syncthreads();  // every read of buffer b is done: it can take the tile after next
    if (tid == 0 && tile + 2 * stride < ntiles) issue(tile + 2 * stride, b);
  }
  // A CTA that gave up at tile k leaves only after the copies issued for tiles k and k + 1 have
  // landed (bounded); after a normal end no copy is outstanding.
  if (tid == 0) {
    for (uint32_t kq = k; kq < k + 2u; kq++)
      if (first + kq * stride < ntiles) (void)mbar_wait((kq & 1u) ? bar1 : bar0, (kq >> 1) & 1u);
  }
  __syncthreads();
}

}  // namespace

bool xpartial_layout_ok(const Layout& L) {
  // TMA box: the chunk as 2^(c+1) floats (one box row up to c = 7, else 256 x 2^(c-7)), 2^w <= 256
  // rows; a strided tile of 2^13 amplitudes
  return L.cb == 0 && L.t == kXTileBits && L.c >= 1 && L.c <= 12 && L.w >= 1 && L.w <= 8 && L.h > L.c;
}

size_t xpartial_smem_bytes(int n_flips) {
  return 1024 + 2 * (size_t)kXTileBytes + (((size_t)n_flips * sizeof(XFlip) + 15) & ~(size_t)15) + 16;
}

cudaError_t launch_partial_x(const XPartialParams& p, int smem, cudaStream_t s) {
  static int configured = 0, cached_dev = -1, cached_smem = -1, cached_g = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_partial_x, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!(dev == cached_dev && smem == cached_smem)) {
    int sms = 0, per = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_partial_x, kXThreads, smem);
    if (e != cudaSuccess) return e;
    cached_dev = dev;
    cached_smem = smem;
    cached_g = sms * (per < 1 ? 1 : per);
  }
  int g = cached_g;
  if (p.max_grid > 0 && g > p.max_grid) g = p.max_grid;
  if ((uint32_t)g > p.ntiles) g = (int)p.ntiles;
  k_partial_x<<<g, kXThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace aqc
