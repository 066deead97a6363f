// C ABI (include/aqc.h): context, SQH term packing, layouts, schedule, step rule and the
// integrator driver (RK4 start-up, then one fused PEC kernel chain per step).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/aqc.h"
#include "aqc_internal.h"

using namespace aqc;

namespace {

enum { V_Y = 0, V_P = 1, V_Q = 2, V_F0 = 3, V_ACC = 7, V_COUNT = 8 };

struct TermH {
  uint32_t x, zm;
  double coef;
  int group;
};
struct ClauseH {
  uint32_t mask;
  int group, pen;
  double scale;
  int stepwise;  // member of the clause-by-clause sequence (Eq. kpath)
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int tile_bits_max(int prec) { return prec == AQC_C128 ? 12 : 13; }
int chunk_bits(int prec) { return prec == AQC_C128 ? 4 : 5; }  // 256-byte contiguous chunks

// Cluster tiles (opt-in with tile_bits = 16; complex64, 22 <= n <= 28): 2^16 indices over 8
// CTAs, so two layouts hold every bit: [0,16) and [0, 32-n) + [16, n) (chunks of at least 16
// amplitudes = 128 bytes).  On GB300 at n = 28 this is slower than three per-CTA layouts (the
// 128-byte-chunk pass and the cluster barriers cost more than the saved pass), so it is not
// the default.
constexpr int kClusterTileBits = 16;
bool cluster_layouts_apply(int n, int prec, int tile_bits) {
  return prec == AQC_C64 && tile_bits == kClusterTileBits && n >= 22 && n <= 28;
}

std::vector<Layout> layouts_for(int n, int prec, int tile_bits, bool allow_clusters) {
  std::vector<Layout> ls;
  if (allow_clusters && cluster_layouts_apply(n, prec, tile_bits)) {
    const int T = tile_bits_max(prec) + kClusterBits;  // 16
    ls.push_back(Layout{T, T, 0, T, kClusterBits});
    ls.push_back(Layout{2 * T - n, T, n - T, T, kClusterBits});
    return ls;
  }
  const int tmax = (tile_bits > 0 && tile_bits <= tile_bits_max(prec)) ? tile_bits : tile_bits_max(prec);
  const int cc = chunk_bits(prec);
  if (n <= tmax) {
    ls.push_back(Layout{n, n, 0, n});
    return ls;
  }
  // every layout gets full-size tiles; when fewer high bits than a full strided layout holds
  // are left, the last layout takes a longer contiguous run instead (fewer rows per tile, so
  // fewer memory pages per tile), or overlaps its predecessor if that run would not fit
  ls.push_back(Layout{tmax, tmax, 0, tmax});
  const int w = tmax - cc;
  int start = tmax;
  while (start < n) {
    const int left = n - start;
    if (left >= w) {
      ls.push_back(Layout{cc, start, w, cc + w});
      start += w;
    } else if (tmax - left <= start) {
      ls.push_back(Layout{tmax - left, start, left, tmax});
      start = n;
    } else {
      ls.push_back(Layout{cc, n - w, w, cc + w});
      start = n;
    }
  }
  return ls;
}


struct WsPlan {
  size_t off_tab, off_slots, off_counter, off_sync, off_perm, off_wdev, off_partials, off_dcode, off_vec, vec_bytes, total;
  size_t partial_doubles;
};

WsPlan plan_workspace(int n, int prec, unsigned flags = 0) {
  WsPlan w;
  const size_t amp = prec == AQC_C128 ? 16 : 8;
  w.off_tab = 0;
  w.off_slots = align_up(sizeof(DevTables), 256);
  w.off_counter = w.off_slots + 256;
  w.off_sync = w.off_counter + 256;  // slab work counter + per-slab counters
  w.off_perm = w.off_sync + align_up((1 + kMaxSlabs) * sizeof(unsigned), 256);  // bit-permutation tables
  w.off_wdev = w.off_perm + 4 * 256 * sizeof(uint32_t);  // weights of graph-replayed steps
  w.off_partials = w.off_wdev + align_up((size_t)kGraphStepWeights * kMaxGraphSteps * sizeof(double), 256);
  // k_apply grids are persistent (at most kMaxApplyGrid CTAs); k_norm2 uses reduce_grid()
  size_t g = std::max((size_t)kMaxApplyGrid, (size_t)reduce_grid((uint64_t)1 << n));
  w.partial_doubles = 3 * g;
  w.off_dcode = align_up(w.off_partials + w.partial_doubles * sizeof(double), 256);
  w.off_vec = align_up(w.off_dcode + ((size_t)1 << n), 256);
  w.vec_bytes = align_up(((size_t)1 << n) * amp, 256);
  // AQC_WS_STEP_CONTROL: one more vector, the state at the start of a segment of constant step
  w.total = w.off_vec + (V_COUNT + ((flags & AQC_WS_STEP_CONTROL) ? 1 : 0)) * w.vec_bytes;
  return w;
}

thread_local std::string g_create_error;

}  // namespace

struct aqc_ctx {
  int device = 0, prec = 0, n = 0;
  uint64_t N = 0;
  size_t amp = 0;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  WsPlan wp;
  void* vec[V_COUNT];
  DevTables* d_tab = nullptr;
  double* d_slots = nullptr;
  unsigned* d_counter = nullptr;
  unsigned* d_sync = nullptr;
  uint32_t* d_perm = nullptr;
  double* d_partials = nullptr;
  uint8_t* d_dcode = nullptr;
  DevTables* h_tab = nullptr;

  std::vector<TermH> terms;
  std::vector<ClauseH> clauses;
  bool dirty = true;
  std::vector<Layout> layouts;
  std::vector<int> nplain, ngeneral;  // local X-string / general products per layout
  std::vector<int> nhop;              // of the general ones, the hops (leading)
  std::vector<char> xpartial;        // layout l's partial pass can run as k_partial_x
  int n_remote = 0, n_z = 0;
  int table_class = -1;
  int step_class = -1, step_m = 0;  // clause-by-clause sequence (class index, length)
  double eval_s = 0.0;              // path parameter s of the evaluation being issued

  bool have_sched = false;
  int s_kind = 0;
  double T = 0;
  double poly[3][4];
  int64_t nsteps_req = 0;
  double kappa = 0.1;
  int tile_bits = 0;  // 0: the precision's default
  int slab_req = 0;   // slab bits: 0 off (default), -1 automatic, k > 0 at most k
  int relabel = 1;    // choose the qubit -> index-bit order that keeps flips inside layouts
  std::vector<int> perm;  // perm[q] = index bit of qubit q in the library's vectors
  bool permuted = false;  // perm is not the identity
  SlabParams slab;    // slab-ordered last passes of a PEC step (slab.n_slabs == 0: off)
  bool in_batch = false;  // batch members use per-CTA tiles only

  // staged host transfers (aqc_transfer_attach): caller-owned staging vectors, library-owned
  // copy streams; in_free / out_free mark when the context stream has consumed / the output
  // copy stream has drained the staging vector
  void* stage_in = nullptr;
  void* stage_out = nullptr;
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t ev_in_ready = nullptr, ev_in_free = nullptr, ev_out_ready = nullptr, ev_out_free = nullptr;
  bool stage_pending = false;  // a staged vector waits for aqc_set_initial_state(AQC_INIT_STAGED)

  bool have_state = false;
  bool hist_ready = false;
  // The run is a sequence of segments of constant step h: the current one starts at seg_t0 and
  // has seg_m steps; `step` is the step index inside it (it selects the RK4 start-up for
  // step < 3 and the derivative ring slot).  The fixed-step grid is one segment from t = 0.
  int64_t step = 0, nsteps = 0, evals = 0;
  double h = 0;
  double seg_t0 = 0.0;
  int64_t seg_m = 0;
  int64_t steps_done = 0;   // accepted grid steps since the initial state, all segments
  bool at_end = false;      // the last step of the run landed on T
  // step-size control (aqc_set_integrator with adaptive = 1)
  int adaptive = 0;
  double tol = 0.0;
  int grow_after = 16;
  int small_run = 0;        // accepted PEC steps in a row with an estimate <= tol ||y|| / 32
  int64_t rejects = 0;
  double max_err_acc = 0.0; // max estimate over accepted PEC steps
  double hmin = 0.0;
  void* vec_save = nullptr; // the workspace's extra vector (AQC_WS_STEP_CONTROL): the state at the
                            // start of the current segment, or the low part of y under ycomp
  int ycomp = 0;            // compensated complex64 corrector (aqc_set_y_compensation)
  int64_t seg_done0 = 0;    // accepted steps before the current segment
  std::vector<aqc_segment> segs;
  int64_t launches = 0;  // kernel launches issued (monotone counter)

  // CUDA-graph replay of K PEC steps (fixed-step grid, no slab order, no clause-by-clause
  // sequence): captured once on a private stream, replayed on `stream` after the host has
  // written the K steps' weights to d_wdev
  int graph_req = -1;             // 0 off, -1 automatic, K > 0 (a multiple of 4, <= kMaxGraphSteps)
  int grid_limit = 0;             // > 0: CTAs per layout-pass launch at most (aqc_set_grid_limit)
  // turn of layouts (aqc_set_layout_turns): the fused step alternates between layouts 0 and 1
  // and leaves its layout's products of p_{n+2} in q, so the next step skips that pass
  int turn_req = 0;               // 0 off (default), 1 or -1: on where it applies
  int q_ready = -1;               // layout whose products of the current p are already in q, or -1
  double* d_wdev = nullptr;       // 3 K weights of the replayed steps
  const double* cur_wdev = nullptr;  // set while a capture is issuing step j: d_wdev + 3 j
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  struct GraphKey {
    int K = 0, phase = 0, q_ready = -1;
    double h = 0.0;
    int64_t tables = -1;
    uint32_t n_slabs = 0;
    void* vec[V_COUNT] = {};
  } gkey;
  int64_t g_launches = 0;         // kernel launches in one replay
  int g_q_ready_end = -1;         // q_ready after one replay
  int64_t graph_replays = 0;
  int64_t tables_version = 0;     // bumped by every table build

  std::string err;
};

#define FAIL(ctx, code, ...)                                     \
  do {                                                           \
    char buf_[512];                                              \
    snprintf(buf_, sizeof(buf_), __VA_ARGS__);                   \
    (ctx)->err = buf_;                                           \
    return (code);                                               \
  } while (0)

#define CUDA_TRY(ctx, expr)                                                                  \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) FAIL(ctx, AQC_E_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

uint32_t layout_mask(const Layout& L) {
  uint32_t m = L.c >= 32 ? 0xffffffffu : ((1u << L.c) - 1u);
  if (L.w > 0) m |= ((1u << L.w) - 1u) << L.h;
  return m;
}

uint32_t compress_mask(const Layout& L, uint32_t x) {
  uint32_t r = 0;
  for (int g = 0; g < 32; g++) {
    if (!((x >> g) & 1u)) continue;
    if (g < L.c)
      r |= 1u << g;
    else
      r |= 1u << (L.c + (g - L.h));
  }
  return r;
}

void plan_layouts(aqc_ctx* c) { c->layouts = layouts_for(c->n, c->prec, c->tile_bits, !c->in_batch); }

// ---- qubit relabelling ----------------------------------------------------------------------
// The library may store qubit q at index bit perm[q] (a relabelling of the tensor factors of
// Eq. ztensor): a product whose flip mask spans two layouts is gathered from global memory once
// per evaluation, and most such products can be moved inside one layout by relabelling.  All
// entry points take and return qubit-order data; only the device vectors are in bit order.
uint64_t map_bits(const std::vector<int>& perm, uint64_t z) {
  uint64_t r = 0;
  for (size_t q = 0; q < perm.size(); q++)
    if ((z >> q) & 1u) r |= (uint64_t)1 << perm[q];
  return r;
}

uint64_t phys_index(const aqc_ctx* c, uint64_t z) { return c->permuted ? map_bits(c->perm, z) : z; }

// dst[z] = src[M(z)], M(z) = map_bits(m, z)
int permute_gather(aqc_ctx* c, void* dst, const void* src, const std::vector<int>& m) {
  uint32_t tab[4 * 256];
  for (int b = 0; b < 4; b++)
    for (int v = 0; v < 256; v++) {
      uint32_t r = 0;
      for (int i = 0; i < 8; i++) {
        const int q = 8 * b + i;
        if (((v >> i) & 1) && q < c->n) r |= 1u << m[q];
      }
      tab[256 * b + v] = r;
    }
  CUDA_TRY(c, cudaMemcpyAsync(c->d_perm, tab, sizeof(tab), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, launch_permute(c->prec, dst, src, c->N, c->d_perm, c->stream));
  c->launches++;
  return AQC_OK;
}

std::vector<int> inverse_perm(const std::vector<int>& p) {
  std::vector<int> r(p.size());
  for (size_t q = 0; q < p.size(); q++) r[p[q]] = (int)q;
  return r;
}

// qubit order -> library order: dst[p] = src[perm^-1(p)]
int to_library_order(aqc_ctx* c, void* dst, const void* src) { return permute_gather(c, dst, src, inverse_perm(c->perm)); }
// library order -> qubit order: dst[z] = src[perm(z)]
int to_qubit_order(aqc_ctx* c, void* dst, const void* src) { return permute_gather(c, dst, src, c->perm); }

// Order that minimises the products (weighted by how many share a flip mask) that no layout
// holds: deterministic local search over transpositions, kept only if strictly better than the
// identity.
std::vector<int> choose_order(const aqc_ctx* c) {
  std::vector<int> id(c->n);
  for (int q = 0; q < c->n; q++) id[q] = q;
  if (!c->relabel || c->layouts.size() < 2) return id;
  std::vector<std::pair<uint32_t, int>> masks;  // distinct multi-bit flip masks with counts
  for (const TermH& th : c->terms) {
    if (__builtin_popcount(th.x) < 2) continue;
    bool found = false;
    for (auto& m : masks)
      if (m.first == th.x) {
        m.second++;
        found = true;
      }
    if (!found) masks.push_back({th.x, 1});
  }
  if (masks.empty()) return id;
  std::vector<uint32_t> lm;
  for (const Layout& L : c->layouts) lm.push_back(layout_mask(L));
  auto cost = [&](const std::vector<int>& p) {
    int k = 0;
    for (const auto& m : masks) {
      const uint32_t x = (uint32_t)map_bits(p, m.first);
      bool held = false;
      for (uint32_t l : lm) held = held || (x & ~l) == 0;
      if (!held) k += m.second;
    }
    return k;
  };
  const int c0 = cost(id);
  if (c0 == 0) return id;
  std::vector<int> cur = id, best = id;
  int ccur = c0, cbest = c0;
  uint64_t st = 0x9E3779B97F4A7C15ull;  // SplitMix64 stream
  auto next = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (int it = 0; it < 20000 && cbest > 0; it++) {
    const int a = (int)(next() % (uint64_t)c->n), b = (int)(next() % (uint64_t)c->n);
    if (a == b) continue;
    std::swap(cur[a], cur[b]);
    const int cn = cost(cur);
    if (cn <= ccur || (next() & 63u) == 0u) {
      ccur = cn;
      if (cn < cbest) {
        cbest = cn;
        best = cur;
      }
    } else {
      std::swap(cur[a], cur[b]);
    }
  }
  return cbest < c0 ? best : id;
}

int popcount32(uint32_t v) { return __builtin_popcount(v); }

// Slab order for the last two passes of a PEC step (SlabParams): needs three or more layouts
// (one full partial pass carries the products no layout holds and reads nothing another slab
// rewrites) and index bits outside layout 0 and the last layout.  "Automatic" selects it for
// complex64 states larger than L2 (the step is HBM-bound there), with slabs of 2^20 indices;
// the highest free bits are fixed, so a slab is made of the longest contiguous runs.  Off by
// default: on GB300 at 28 qubits the single launch moves 10% fewer bytes than the separate
// passes but runs slower (two CTAs per SM for both item kinds, more load latency exposed).
void plan_slabs(aqc_ctx* c) {
  memset(&c->slab, 0, sizeof(c->slab));
  const int nl = (int)c->layouts.size();
  if (c->slab_req == 0 || c->in_batch || nl < 3) return;
  for (const Layout& L : c->layouts)
    if (L.cb != 0) return;
  const uint32_t all = c->n >= 32 ? 0xffffffffu : ((1u << c->n) - 1u);
  const uint32_t avail = all & ~layout_mask(c->layouts[0]) & ~layout_mask(c->layouts[nl - 1]);
  int want;
  if (c->slab_req > 0) {
    want = c->slab_req;
  } else {
    if (c->prec != AQC_C64 || c->N * c->amp < ((uint64_t)64 << 20)) return;
    want = c->n - 20;
  }
  want = std::min(want, std::min(popcount32(avail), 11));
  if (want <= 0) return;
  uint32_t mask = 0;
  for (int b = 31, got = 0; b >= 0 && got < want; b--) {
    if ((avail >> b) & 1u) {
      mask |= 1u << b;
      got++;
    }
  }
  SlabParams& S = c->slab;
  S.slab_mask = mask;
  S.free_part = all & ~layout_mask(c->layouts[nl - 1]) & ~mask;
  S.free_step = all & ~layout_mask(c->layouts[0]) & ~mask;
  S.n_slabs = 1u << want;
  S.tiles = 1u << popcount32(S.free_step);
  if (popcount32(S.free_part) != popcount32(S.free_step)) {  // layouts of unequal tile size
    memset(&c->slab, 0, sizeof(c->slab));
    return;
  }
  S.lookahead = std::min<uint32_t>(2u, S.n_slabs);
  S.n_items = 2u * S.n_slabs * S.tiles;
  S.spin_limit = 1u << 22;
  S.queue = c->d_sync;
  S.done = c->d_sync + 1;
}

int build_tables(aqc_ctx* c) {
  c->tables_version++;
  c->q_ready = -1;
  plan_layouts(c);
  DevTables* t = c->h_tab;
  memset(t, 0, sizeof(DevTables));
  const int nl = (int)c->layouts.size();
  if (nl > kMaxLayouts) FAIL(c, AQC_E_UNSUPPORTED, "too many layouts (%d)", nl);
  t->n_layouts = nl;
  std::vector<std::vector<DevFlip>> per(nl + 1);
  int nz = 0;
  // qubit order of the library's vectors; a state already set moves to the new order
  {
    std::vector<int> np = choose_order(c);
    std::vector<int> old = c->perm.empty() ? std::vector<int>() : c->perm;
    if (old.empty()) {
      old.resize(c->n);
      for (int q = 0; q < c->n; q++) old[q] = q;
    }
    if (np != old && c->have_state) {
      // new[p] = old[old_perm(new_perm^-1(p))]
      const std::vector<int> inv = inverse_perm(np);
      std::vector<int> m(c->n);
      for (int p = 0; p < c->n; p++) m[p] = old[inv[p]];
      void* live[] = {c->vec[V_Y], c->vec[V_P], c->vec[V_F0], c->vec[V_F0 + 1], c->vec[V_F0 + 2],
                      c->vec[V_F0 + 3], c->vec_save};
      for (void* v : live) {
        if (!v) continue;
        int rc = permute_gather(c, c->vec[V_ACC], v, m);
        if (rc) return rc;
        CUDA_TRY(c, cudaMemcpyAsync(v, c->vec[V_ACC], (size_t)c->N * c->amp, cudaMemcpyDeviceToDevice, c->stream));
      }
    }
    c->perm = np;
    c->permuted = false;
    for (int q = 0; q < c->n; q++) c->permuted = c->permuted || np[q] != q;
  }
  for (const TermH& th0 : c->terms) {
    TermH th = th0;
    th.x = (uint32_t)phys_index(c, th0.x);
    th.zm = (uint32_t)phys_index(c, th0.zm);
    if (th.x == 0) {
      if (th.zm == 0) {
        t->ident[th.group] += th.coef;
      } else {
        if (nz >= kMaxZ) FAIL(c, AQC_E_UNSUPPORTED, "more than %d diagonal Pauli products", kMaxZ);
        t->z[nz].zm = th.zm;
        t->z[nz].group = th.group;
        t->z[nz].coef = th.coef;
        nz++;
      }
      continue;
    }
    DevFlip f;
    memset(&f, 0, sizeof(f));
    f.x = th.x;
    f.zm = th.zm;
    f.group = th.group;
    f.ipow = __builtin_popcount(th.x & th.zm) & 3;
    f.coef = th.coef;
    int where = nl;
    for (int l = 0; l < nl; l++) {
      if ((th.x & ~layout_mask(c->layouts[l])) == 0) {
        where = l;
        break;
      }
    }
    f.lx = where < nl ? compress_mask(c->layouts[where], th.x) : 0u;
    // a second product with the same flip mask shares the first one's gather
    bool merged = false;
    for (DevFlip& e : per[where]) {
      if (e.x == f.x && !e.has2) {
        e.has2 = 1;
        e.zm2 = f.zm;
        e.group2 = f.group;
        e.ipow2 = f.ipow;
        e.coef2 = f.coef;
        merged = true;
        break;
      }
    }
    if (!merged) per[where].push_back(f);
  }
  int pos = 0;
  c->nplain.assign(nl, 0);
  c->ngeneral.assign(nl, 0);
  c->nhop.assign(nl, 0);
  c->xpartial.assign(nl, 0);
  for (int l = 0; l <= nl; l++) {
    t->flip_begin[l] = pos;
    if (pos + (int)per[l].size() > kMaxFlips) FAIL(c, AQC_E_UNSUPPORTED, "more than %d off-diagonal products", kMaxFlips);
    // X strings with real coefficients first (the kernel's fast loops: those flipping no
    // register-held tile bit, then the others), then general products
    int np = 0, nfast = 0;
    if (l < nl) {
      const uint32_t regbits = c->prec == AQC_C128 ? kRegBitsC128 : kRegBitsC64;
      for (const DevFlip& f : per[l])
        if (f.zm == 0 && !f.has2 && (f.lx & regbits) == 0) t->flips[pos + np++] = f;
      nfast = np;
      for (const DevFlip& f : per[l])
        if (f.zm == 0 && !f.has2 && (f.lx & regbits) != 0) t->flips[pos + np++] = f;
    }
    // general range: hops first (the kernels' hop loop), then the other general products
    auto is_hop = [](const DevFlip& f) {
      return f.has2 && f.zm == 0 && f.zm2 == f.x && (f.ipow2 & 3) == 2 && f.group2 == f.group &&
             f.coef2 == f.coef && __builtin_popcount(f.x) == 2;
    };
    int k = np, nh = 0;
    if (l < nl) {
      // hops by class: which of the register-held tile bits (the pair bit of complex64 and the
      // half bit) each flips, so that the kernels' hop loops know both at compile time
      const uint32_t pair_bit = c->prec == AQC_C128 ? 0u : 1u, half_bit = c->prec == AQC_C128 ? 32u : 64u;
      auto hop_class = [&](const DevFlip& f) {
        return ((f.lx & pair_bit) ? 1 : 0) | ((f.lx & half_bit) ? 2 : 0);
      };
      for (int cls = 0; cls < 4; cls++) {
        for (const DevFlip& f : per[l])
          if (is_hop(f) && hop_class(f) == cls) t->flips[pos + k++] = f;
        if (cls < 3) t->hop_class_end[l][cls] = k - np;
      }
      nh = k - np;
      for (const DevFlip& f : per[l])
        if ((f.zm != 0 || f.has2) && !is_hop(f)) t->flips[pos + k++] = f;
    } else {
      for (const DevFlip& f : per[l]) t->flips[pos + k++] = f;
    }
    t->hop_count[l] = nh;
    t->plain_count[l] = np;
    t->plain_fast[l] = nfast;
    if (l < nl) {
      c->nplain[l] = np;
      c->ngeneral[l] = (int)per[l].size() - np;
      c->nhop[l] = nh;
    }
    if (l > 0 && l < nl) {  // X strings and hops only: the TMA-fed partial kernel
      const bool ok = c->prec == AQC_C64 && xpartial_layout_ok(c->layouts[l]) && c->ngeneral[l] == nh &&
                      xpartial_smem_bytes(np + nh) <= 227 * 1024;
      c->xpartial[l] = ok ? 1 : 0;
    }
    pos += (int)per[l].size();
  }
  t->flip_begin[nl + 1] = pos;
  t->n_remote = (int)per[nl].size();
  c->n_remote = t->n_remote;
  t->n_z = nz;
  c->n_z = nz;
  // clause classes (group, penalty, scale), clauses sorted by class in first-seen order
  std::vector<ClauseH> cl = c->clauses;
  std::vector<int> cls_of(cl.size());
  std::vector<DevClass> classes;
  for (size_t i = 0; i < cl.size(); i++) {
    int k = -1;
    for (size_t j = 0; j < classes.size(); j++)
      if (classes[j].group == cl[i].group && classes[j].pen == cl[i].pen && classes[j].scale == cl[i].scale &&
          classes[j].stepwise == cl[i].stepwise)
        k = (int)j;
    if (k < 0) {
      if ((int)classes.size() >= kMaxClasses) FAIL(c, AQC_E_UNSUPPORTED, "more than %d clause classes", kMaxClasses);
      DevClass dc;
      memset(&dc, 0, sizeof(dc));
      dc.group = cl[i].group;
      dc.pen = cl[i].pen;
      dc.scale = cl[i].scale;
      dc.stepwise = cl[i].stepwise;
      classes.push_back(dc);
      k = (int)classes.size() - 1;
    }
    cls_of[i] = k;
  }
  if ((int)cl.size() > kMaxClauses) FAIL(c, AQC_E_UNSUPPORTED, "more than %d clauses", kMaxClauses);
  int cp = 0;
  for (size_t k = 0; k < classes.size(); k++) {
    classes[k].begin = cp;
    for (size_t i = 0; i < cl.size(); i++)
      if (cls_of[i] == (int)k) t->clause_mask[cp++] = (uint32_t)phys_index(c, cl[i].mask);
    classes[k].end = cp;
    t->classes[k] = classes[k];
  }
  t->n_classes = (int)classes.size();
  // cache the counts of the first fixed-weight clause class as one byte per index when they fit
  t->table_class = -1;
  c->step_class = -1;
  for (size_t k = 0; k < classes.size(); k++) {
    if (classes[k].stepwise) {
      c->step_class = (int)k;
      continue;
    }
    if (t->table_class >= 0) continue;
    const int cnt = classes[k].end - classes[k].begin;
    const int maxv = classes[k].pen == AQC_PEN_SQUARED ? 4 * cnt : cnt;
    if (maxv <= 255) t->table_class = (int)k;
  }
  // a class whose clauses are the table class's minus a few (the catalyst H_{m-1} of Eq. nlpath
  // beside H_f) counts as the cached byte minus those few clauses
  if (t->table_class >= 0) {
    const DevClass& B = classes[t->table_class];
    int dp = cp;
    for (size_t k = 0; k < classes.size(); k++) {
      DevClass& C = classes[k];
      if ((int)k == t->table_class || C.stepwise || C.pen != B.pen) continue;
      std::vector<uint32_t> rest(t->clause_mask + B.begin, t->clause_mask + B.end);
      bool sub = true;
      for (int i = C.begin; i < C.end && sub; i++) {
        auto it = std::find(rest.begin(), rest.end(), t->clause_mask[i]);
        if (it == rest.end())
          sub = false;
        else
          rest.erase(it);
      }
      if (!sub || (int)rest.size() > kMaxDerivedDiff || (int)rest.size() >= C.end - C.begin) continue;
      if (dp + (int)rest.size() > kMaxClauses) break;
      C.derived = 1;
      C.dbegin = dp;
      for (uint32_t m : rest) t->clause_mask[dp++] = m;
      C.dend = dp;
      t->classes[k] = C;
    }
  }
  c->step_m = c->step_class >= 0 ? classes[c->step_class].end - classes[c->step_class].begin : 0;
  c->table_class = t->table_class;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_tab, t, sizeof(DevTables), cudaMemcpyHostToDevice, c->stream));
  if (t->table_class >= 0) {
    CUDA_TRY(c, launch_diag_codes(c->d_dcode, c->N, c->d_tab, t->table_class, c->stream));
    c->launches++;
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  plan_slabs(c);
  c->dirty = false;
  return AQC_OK;
}

double sched_s(const aqc_ctx* c, double t) {
  const double tau = t / c->T;
  return c->s_kind == AQC_S_SMOOTHSTEP ? tau * tau * (3.0 - 2.0 * tau) : tau;
}

// Group weights at time t; also records s(t) for the clause-by-clause coefficients.
void sched_weights(aqc_ctx* c, double t, double w[3]) {
  const double s = sched_s(c, t);
  c->eval_s = s;
  for (int g = 0; g < 3; g++) w[g] = ((c->poly[g][3] * s + c->poly[g][2]) * s + c->poly[g][1]) * s + c->poly[g][0];
}

double group_bound(const aqc_ctx* c, int g) {
  double b = 0.0;
  for (const TermH& t : c->terms)
    if (t.group == g) b += fabs(t.coef);
  for (const ClauseH& k : c->clauses)
    if (k.group == g) b += fabs(k.scale) * (k.pen == AQC_PEN_SQUARED ? 4.0 : 1.0);
  return b;
}

int64_t rule_steps(const aqc_ctx* c) {
  double b[3];
  for (int g = 0; g < 3; g++) b[g] = group_bound(c, g);
  double lam = 0.0;
  for (int i = 0; i <= 1024; i++) {
    const double s = i / 1024.0;
    double v = 0.0;
    for (int g = 0; g < 3; g++) {
      const double wg = ((c->poly[g][3] * s + c->poly[g][2]) * s + c->poly[g][1]) * s + c->poly[g][0];
      v += fabs(wg) * b[g];
    }
    lam = std::max(lam, v);
  }
  const double n = ceil(c->T * lam / c->kappa);
  return std::max<int64_t>(4, (int64_t)n);
}

// The driver's tensor-map encoder, looked up once through the runtime (no link to libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// A complex64 vector of 2^n amplitudes as a float tensor whose box is one tile of layout L:
// 4-D (2^(c+1) floats of the contiguous chunk, 2^(h-c) gap positions, 2^w tile rows, top bits)
// while the chunk fits one box row (c <= 7), else 5-D with the chunk as 256 x 2^(c-7) floats.
// Returns the rank, or 0 if no map can be made.
int encode_tile_map(CUtensorMap* m, const void* v, int n, const Layout& L) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || ((uintptr_t)v & 15u)) return 0;
  const cuuint32_t es[5] = {1u, 1u, 1u, 1u, 1u};
  if (L.c <= 7) {
    const cuuint64_t dims[4] = {(cuuint64_t)2 << L.c, (cuuint64_t)1 << (L.h - L.c), (cuuint64_t)1 << L.w,
                                (cuuint64_t)1 << (n - L.h - L.w)};
    const cuuint64_t strides[3] = {(cuuint64_t)8 << L.c, (cuuint64_t)8 << L.h, (cuuint64_t)8 << (L.h + L.w)};
    const cuuint32_t box[4] = {(cuuint32_t)2 << L.c, 1u, (cuuint32_t)1 << L.w, 1u};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(v), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS ? 4 : 0;
  }
  const cuuint64_t dims[5] = {256u, (cuuint64_t)1 << (L.c - 7), (cuuint64_t)1 << (L.h - L.c), (cuuint64_t)1 << L.w,
                              (cuuint64_t)1 << (n - L.h - L.w)};
  const cuuint64_t strides[4] = {1024u, (cuuint64_t)8 << L.c, (cuuint64_t)8 << L.h, (cuuint64_t)8 << (L.h + L.w)};
  const cuuint32_t box[5] = {256u, (cuuint32_t)1 << (L.c - 7), 1u, (cuuint32_t)1 << L.w, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(v), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS ? 5 : 0;
}

// Coefficients of the clause-by-clause sequence at s (Eq. kpath): on segment k (s_k in [0, 1)),
// clauses j < k weigh 1 (1 - s_k on the last segment, where H_m = 0), clause k weighs s_k (0 on
// the last segment), later clauses 0; step_k = 0 outside [0, 1).
void set_step_fields(const aqc_ctx* c, ApplyParams* p) {
  p->step_k = 0;
  p->step_wdone = p->step_wact = 0.0;
  const int m = c->step_m;
  const double s = c->eval_s;
  if (c->step_class < 0 || m < 1 || !(s >= 0.0 && s < 1.0)) return;
  int k = (int)floor((double)m * s) + 1;
  if (k > m) k = m;
  const double sk = (double)m * s - (double)k + 1.0;
  if (!(sk >= 0.0 && sk < 1.0)) return;
  p->step_k = k;
  p->step_wdone = k <= m - 1 ? 1.0 : 1.0 - sk;
  p->step_wact = k <= m - 1 ? sk : 0.0;
}

ApplyParams base_params(aqc_ctx* c) {
  ApplyParams p;
  memset(&p, 0, sizeof(p));
  set_step_fields(c, &p);
  p.tab = c->d_tab;
  p.n = c->n;
  p.partials = c->d_partials;
  p.counter = c->d_counter;
  p.max_grid = c->grid_limit;
  p.slots = c->d_slots;
  return p;
}

// One evaluation of H(t) src over all layouts.  The strided layouts run first as partial sums
// (the first one also adds the products no layout holds); the contiguous layout 0 runs last
// with the mode epilogue, so the kernel touching the most vectors has the smallest page
// footprint per tile.  The diagonal is added by layout 0 (see diag_level).
// With top >= 0, only the partial passes of layouts top .. 1 run (the first of them adds the
// products no layout holds); the caller finishes the evaluation.
int evaluate(aqc_ctx* c, const double w[3], const void* src, ApplyParams fin, void* partial_out, int top = -1) {
  c->q_ready = -1;  // the passes below overwrite q
  const int nl = (int)c->layouts.size();
  const int hi = top >= 0 ? top : nl - 1, lo = top >= 0 ? 1 : 0;
  for (int l = hi; l >= lo; l--) {
    const bool first = (l == hi), last = (l == 0), diag = (l == diag_level(nl));
    ApplyParams p = last ? fin : base_params(c);
    p.L = c->layouts[l];
    p.layout_index = l;
    p.with_diag = diag;
    p.with_remote = first;
    for (int g = 0; g < 3; g++) p.w[g] = w[g];
    p.src = src;
    p.wdev = c->cur_wdev;
    p.qin = first ? nullptr : c->vec[V_Q];
    if (!last) {
      p.mode = MODE_PARTIAL;
      p.qout = c->vec[V_Q];
    } else if (fin.mode == MODE_PARTIAL) {
      p.qout = partial_out;
    }
    p.dcode = (diag && c->table_class >= 0) ? c->d_dcode : nullptr;
    p.ntiles = 1u << (c->n - p.L.t);
    // X-string-only strided layouts: TMA-fed partial kernel
    if (!last && !diag && c->xpartial[l] && !(first && c->n_remote > 0)) {
      XPartialParams x;
      memset(&x, 0, sizeof(x));
      x.tma_rank = encode_tile_map(&x.tmap, src, c->n, p.L);
      if (x.tma_rank) {
        x.tab = c->d_tab;
        x.L = p.L;
        x.layout_index = l;
        for (int g = 0; g < 3; g++) x.w[g] = w[g];
        x.wdev = c->cur_wdev;
        x.max_grid = c->grid_limit;
        x.qin = p.qin;
        x.qout = p.qout;
        x.ntiles = p.ntiles;
        x.slots = c->d_slots;
        CUDA_TRY(c, launch_partial_x(x, (int)xpartial_smem_bytes(c->nplain[l] + c->nhop[l]), c->stream));
        c->launches++;
        continue;
      }
    }
    const size_t smem = apply_smem_bytes(c->prec, p.L.t - p.L.cb, c->nplain[l],
                                         c->ngeneral[l] + (first ? c->n_remote : 0), diag ? c->n_z : 0);
    if (smem > 227 * 1024) FAIL(c, AQC_E_UNSUPPORTED, "shared memory %zu bytes too large", smem);
    CUDA_TRY(c, launch_apply(c->prec, p, (int)smem, c->stream));
    c->launches++;
  }
  return AQC_OK;
}

int ensure_ready(aqc_ctx* c) {
  if (!c->have_sched) FAIL(c, AQC_E_STATE, "no schedule set");
  if (c->dirty) {
    int rc = build_tables(c);
    if (rc) return rc;
  }
  return AQC_OK;
}

int rk4_step(aqc_ctx* c) {
  const double t = c->seg_t0 + (double)c->step * c->h, hh = c->h;
  double w[3];
  for (int stage = 1; stage <= 4; stage++) {
    const double ts = stage == 1 ? t : (stage == 4 ? t + hh : t + 0.5 * hh);
    sched_weights(c, ts, w);
    ApplyParams fin = base_params(c);
    fin.mode = MODE_RK4;
    fin.stage = stage;
    fin.h = hh;
    fin.y = c->vec[V_Y];
    fin.acc = c->vec[V_ACC];
    fin.pout = c->vec[V_P];
    fin.fout = c->vec[V_F0 + (int)(c->step & 3)];
    int rc = evaluate(c, w, stage == 1 ? c->vec[V_Y] : c->vec[V_P], fin, nullptr);
    if (rc) return rc;
    c->evals++;
  }
  return AQC_OK;  // the caller counts the step (count_step)
}

int start_history(aqc_ctx* c) {
  // f_3 = -i H(t_3) y_3, then p_4 from the AB4 predictor
  double w[3];
  sched_weights(c, c->seg_t0 + 3.0 * c->h, w);
  ApplyParams fin = base_params(c);
  fin.mode = MODE_DERIV;
  fin.fout = c->vec[V_F0 + 3];
  int rc = evaluate(c, w, c->vec[V_Y], fin, nullptr);
  if (rc) return rc;
  c->evals++;
  CUDA_TRY(c, launch_predict(c->prec, c->vec[V_P], c->vec[V_Y], c->vec[V_F0 + 3], c->vec[V_F0 + 2],
                             c->vec[V_F0 + 1], c->vec[V_F0 + 0], c->h, c->N, c->stream));
  c->launches++;
  if (c->ycomp)  // the PEC steps' low part of y starts at zero
    CUDA_TRY(c, cudaMemsetAsync(c->vec_save, 0, (size_t)c->N * c->amp, c->stream));
  c->hist_ready = true;
  return AQC_OK;
}

// Slab order: layouts nl-2 .. 1 as full partial passes (the first adds the products no layout
// holds), then one k_slab launch for layout nl-1 (partial) and layout 0 (fused step).
int pec_step_slabs(aqc_ctx* c, const double w[3], const ApplyParams& fin) {
  const int nl = (int)c->layouts.size();
  ApplyParams stub = base_params(c);
  stub.mode = MODE_PARTIAL;
  stub.qout = c->vec[V_Q];
  int rc = evaluate(c, w, c->vec[V_P], stub, c->vec[V_Q], nl - 2);
  if (rc) return rc;
  SlabParams S = c->slab;
  const int lp = nl - 1;
  S.part = base_params(c);
  S.part.L = c->layouts[lp];
  S.part.layout_index = lp;
  S.part.mode = MODE_PARTIAL;
  S.part.src = c->vec[V_P];
  S.part.qin = c->vec[V_Q];
  S.part.qout = c->vec[V_Q];
  S.step = fin;
  S.step.L = c->layouts[0];
  S.step.layout_index = 0;
  S.step.with_diag = (0 == diag_level(nl));
  S.step.with_remote = 0;
  S.step.src = c->vec[V_P];
  S.step.qin = c->vec[V_Q];
  S.step.dcode = (S.step.with_diag && c->table_class >= 0) ? c->d_dcode : nullptr;
  for (int g = 0; g < 3; g++) S.part.w[g] = S.step.w[g] = w[g];
  S.part.h = S.step.h = c->h;
  const int t = c->layouts[0].t;
  const size_t smem = apply_smem_bytes(c->prec, t, c->nplain[0], c->ngeneral[0], S.step.with_diag ? c->n_z : 0) +
                      table_smem_bytes(c->prec, t, c->nplain[lp], c->ngeneral[lp], 0);
  if (smem > 227 * 1024) FAIL(c, AQC_E_UNSUPPORTED, "shared memory %zu bytes too large", smem);
  CUDA_TRY(c, launch_slab(c->prec, S, (int)smem, c->stream));
  c->launches++;
  return AQC_OK;
}

// The turn of layouts applies where every pass is a per-CTA tile pass of a fixed-step grid and
// the products no layout holds (gathered from all of p) can stay in a partial pass.
bool turn_applies(const aqc_ctx* c) {
  const int nl = (int)c->layouts.size();
  if (c->turn_req == 0 || c->adaptive || c->in_batch || c->slab.n_slabs || c->step_class >= 0 || nl < 2) return false;
  for (const Layout& L : c->layouts)
    if (L.cb > 0) return false;
  return nl >= 3 || c->n_remote == 0;
}

// One PEC step with the turn of layouts (Sec. I.B step; the layout order is this library's):
// q holds layout Xp's products of p_{n+1} (Xp = q_ready, or -1); the layouts other than Xp and
// the fused layout Xc add theirs as partial passes (the first one also the products no layout
// holds); the fused step on Xc completes f_{n+1}, corrects y, predicts p_{n+2} and leaves Xc's
// products of p_{n+2} at the next weights in q.  Xc alternates between layouts 0 and 1.
int pec_step_turn(aqc_ctx* c, const ApplyParams& fin0, const double w[3]) {
  const int nl = (int)c->layouts.size();
  const int Xp = c->q_ready, Xc = Xp == 0 ? 1 : 0;
  double w2[3];
  sched_weights(c, c->seg_t0 + (double)(c->step + 2) * c->h, w2);
  bool any = false;
  for (int l = nl - 1; l >= 0; l--) {
    if (l == Xp || l == Xc) continue;
    const bool first = !any;
    ApplyParams p = base_params(c);
    p.mode = MODE_PARTIAL;
    p.L = c->layouts[l];
    p.layout_index = l;
    p.with_diag = 0;
    p.with_remote = first;
    for (int g = 0; g < 3; g++) p.w[g] = w[g];
    p.wdev = c->cur_wdev;
    p.src = c->vec[V_P];
    p.qin = (first && Xp < 0) ? nullptr : c->vec[V_Q];
    p.qout = c->vec[V_Q];
    p.ntiles = 1u << (c->n - p.L.t);
    any = true;
    if (c->xpartial[l] && !(first && c->n_remote > 0)) {
      XPartialParams x;
      memset(&x, 0, sizeof(x));
      x.tma_rank = encode_tile_map(&x.tmap, p.src, c->n, p.L);
      if (x.tma_rank) {
        x.tab = c->d_tab;
        x.L = p.L;
        x.layout_index = l;
        for (int g = 0; g < 3; g++) x.w[g] = w[g];
        x.wdev = c->cur_wdev;
        x.max_grid = c->grid_limit;
        x.qin = p.qin;
        x.qout = p.qout;
        x.ntiles = p.ntiles;
        x.slots = c->d_slots;
        CUDA_TRY(c, launch_partial_x(x, (int)xpartial_smem_bytes(c->nplain[l] + c->nhop[l]), c->stream));
        c->launches++;
        continue;
      }
    }
    const size_t smem = apply_smem_bytes(c->prec, p.L.t, c->nplain[l], c->ngeneral[l] + (first ? c->n_remote : 0), 0);
    if (smem > 227 * 1024) FAIL(c, AQC_E_UNSUPPORTED, "shared memory %zu bytes too large", smem);
    CUDA_TRY(c, launch_apply(c->prec, p, (int)smem, c->stream));
    c->launches++;
  }
  ApplyParams f = fin0;
  f.L = c->layouts[Xc];
  f.layout_index = Xc;
  f.with_diag = 1;
  f.with_remote = !any;  // only when no partial pass ran, i.e. with no products no layout holds
  for (int g = 0; g < 3; g++) {
    f.w[g] = w[g];
    f.w2[g] = w2[g];
  }
  f.wdev = c->cur_wdev;
  f.turn = 1;
  f.src = c->vec[V_P];
  f.qin = (!any && Xp < 0) ? nullptr : c->vec[V_Q];
  f.qout = c->vec[V_Q];
  f.dcode = c->table_class >= 0 ? c->d_dcode : nullptr;
  f.ntiles = 1u << (c->n - f.L.t);
  const size_t smem = apply_smem_bytes(c->prec, f.L.t, c->nplain[Xc], c->ngeneral[Xc] + (any ? 0 : c->n_remote), c->n_z) +
                      table_smem_bytes(c->prec, f.L.t, c->nplain[Xc], c->ngeneral[Xc], 0);
  if (smem > 227 * 1024) FAIL(c, AQC_E_UNSUPPORTED, "shared memory %zu bytes too large", smem);
  CUDA_TRY(c, launch_apply(c->prec, f, (int)smem, c->stream));
  c->launches++;
  c->q_ready = Xc;
  return AQC_OK;
}

int pec_step(aqc_ctx* c) {
  const int64_t n = c->step;
  double w[3];
  sched_weights(c, c->seg_t0 + (double)(n + 1) * c->h, w);
  ApplyParams fin = base_params(c);
  fin.mode = MODE_STEP;
  fin.h = c->h;
  fin.y = c->vec[V_Y];
  fin.f0 = c->vec[V_F0 + (int)(n & 3)];
  fin.f1 = c->vec[V_F0 + (int)((n - 1) & 3)];
  fin.f2 = c->vec[V_F0 + (int)((n - 2) & 3)];
  fin.fout = c->vec[V_F0 + (int)((n + 1) & 3)];
  fin.pout = c->vec[V_P];
  // under step-size control y_{n+1} goes to the scratch vector, so a rejected step keeps y_n
  fin.yout = c->adaptive ? c->vec[V_ACC] : nullptr;
  fin.ylo = c->ycomp ? c->vec_save : nullptr;
  int rc;
  if (turn_applies(c))
    rc = pec_step_turn(c, fin, w);
  else
    rc = (c->slab.n_slabs && !c->ycomp) ? pec_step_slabs(c, w, fin) : evaluate(c, w, c->vec[V_P], fin, nullptr);
  if (rc) return rc;
  c->evals++;
  return AQC_OK;  // the caller counts the step (count_step) or decides on it (control_step)
}

// m = ceil(R / hp) steps of h = R / m for a segment of length R, a ratio a hair above an integer
// (the rounding of hp = R / N) counted as that integer
int64_t segment_steps(double R, double hp) {
  const double q = ceil((R / hp) * (1.0 - 1e-12));
  return q < 1.0 ? 1 : (int64_t)q;
}

// A new segment of constant step from t0 with proposed step hp (it lands on T).
int begin_segment(aqc_ctx* c, double t0, double hp, int64_t m_given = 0) {
  if (!(hp >= c->hmin)) FAIL(c, AQC_E_NUMERIC, "step size %.3e fell below the minimum %.3e", hp, c->hmin);
  const double R = c->T - t0;
  c->seg_m = m_given > 0 ? m_given : segment_steps(R, hp);
  c->h = m_given > 0 ? c->T / (double)m_given : R / (double)c->seg_m;
  c->seg_t0 = t0;
  c->step = 0;
  c->hist_ready = false;
  c->q_ready = -1;
  c->small_run = 0;
  c->seg_done0 = c->steps_done;
  if (c->adaptive)  // kept until the segment's first PEC step is accepted
    CUDA_TRY(c, cudaMemcpyAsync(c->vec_save, c->vec[V_Y], (size_t)c->N * c->amp, cudaMemcpyDeviceToDevice,
                                c->stream));
  aqc_segment sg;
  memset(&sg, 0, sizeof(sg));
  sg.t0 = t0;
  sg.h = c->h;
  sg.end = AQC_SEG_RUNNING;
  c->segs.push_back(sg);
  return AQC_OK;
}

// The first segment after an initial state: the grid of n_steps (or the step rule), h = T / N.
int plan_first_segment(aqc_ctx* c) {
  if (c->nsteps != 0) return AQC_OK;
  c->nsteps = c->nsteps_req > 0 ? c->nsteps_req : rule_steps(c);
  c->hmin = (c->T / (double)c->nsteps) * 0x1p-30;
  c->segs.clear();
  return begin_segment(c, 0.0, c->T / (double)c->nsteps, c->nsteps);
}

// One accepted grid step of the current segment.
void count_step(aqc_ctx* c) {
  c->step++;
  c->steps_done++;
  c->segs.back().steps++;
  if (c->step >= c->seg_m) {
    c->at_end = true;
    c->segs.back().end = AQC_SEG_AT_T;
  }
}

// Step-size control after a PEC step whose y_{n+1} sits in the scratch vector: accept (the
// scratch becomes y) if (19/270)||y_{n+1} - p_{n+1}|| <= tol ||y_{n+1}||, else restart from this
// step's start with h/2; after grow_after small estimates in a row, restart with 2h.
int control_step(aqc_ctx* c) {
  double sl[kSlotCount];
  CUDA_TRY(c, cudaMemcpyAsync(sl, c->d_slots, sizeof(sl), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const double e = sl[kSlotLastErr], y2 = sl[kSlotNorm2];
  if (sl[kSlotFault] != 0.0) FAIL(c, AQC_E_TIMEOUT, "a kernel gave up waiting (a tile copy or a slab's partial sums)");
  if (!std::isfinite(e) || !std::isfinite(y2)) FAIL(c, AQC_E_NUMERIC, "non-finite error estimate or norm");
  const double lim = c->tol * sqrt(y2);
  if (!(e <= lim)) {
    c->rejects++;
    c->segs.back().end = AQC_SEG_REJECTED;
    if (c->step == 3) {  // the segment's first PEC step also judged its RK4 start-up: redo it all
      std::swap(c->vec[V_Y], c->vec_save);
      c->steps_done = c->seg_done0;
      c->segs.back().steps = 0;
      return begin_segment(c, c->seg_t0, 0.5 * c->h);
    }
    return begin_segment(c, c->seg_t0 + (double)c->step * c->h, 0.5 * c->h);
  }
  std::swap(c->vec[V_Y], c->vec[V_ACC]);
  if (e > c->max_err_acc) c->max_err_acc = e;
  count_step(c);
  if (c->at_end) return AQC_OK;
  c->small_run = e <= lim / 32.0 ? c->small_run + 1 : 0;
  if (c->grow_after > 0 && c->small_run >= c->grow_after) {
    c->segs.back().end = AQC_SEG_GREW;
    return begin_segment(c, c->seg_t0 + (double)c->step * c->h, 2.0 * c->h);
  }
  return AQC_OK;
}

// ---- CUDA-graph replay of PEC steps ---------------------------------------------------------
// A replay covers K consecutive PEC steps starting at a step index of the captured phase
// (index mod 4 selects the derivative ring slots).  Everything a captured launch bakes in -- the
// vectors, h, the tables' layouts and shapes -- is in the key; the weights are not: the host
// computes them (sched_weights, the expression the eager steps use, so both give the same
// bits) and writes them to d_wdev ahead of each replay.

int graph_k(const aqc_ctx* c) {
  if (c->adaptive || c->in_batch || c->slab.n_slabs || c->step_class >= 0) return 0;
  if (c->graph_req < 0) return c->n <= 20 ? 16 : 0;  // launch-bound sizes
  return c->graph_req;
}

aqc_ctx::GraphKey graph_key(const aqc_ctx* c, int K) {
  aqc_ctx::GraphKey k;
  k.K = K;
  k.phase = (int)(c->step & 3);
  k.q_ready = c->q_ready;
  k.h = c->h;
  k.tables = c->tables_version;
  k.n_slabs = c->slab.n_slabs;
  for (int v = 0; v < V_COUNT; v++) k.vec[v] = c->vec[v];
  return k;
}

bool same_key(const aqc_ctx::GraphKey& a, const aqc_ctx::GraphKey& b) {
  if (a.K != b.K || a.phase != b.phase || a.q_ready != b.q_ready || memcmp(&a.h, &b.h, sizeof(double)) != 0 ||
      a.tables != b.tables ||
      a.n_slabs != b.n_slabs)
    return false;
  for (int v = 0; v < V_COUNT; v++)
    if (a.vec[v] != b.vec[v]) return false;
  return true;
}

void drop_step_graph(aqc_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->gkey = aqc_ctx::GraphKey();
}

// Capture K PEC steps from the current step on the private stream; host counters are left as
// they were (the replay advances them).
int capture_steps(aqc_ctx* c, int K) {
  drop_step_graph(c);
  if (!c->cap_stream) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  const int64_t step0 = c->step, evals0 = c->evals, launches0 = c->launches;
  const int q_ready0 = c->q_ready;
  cudaStream_t user = c->stream;
  c->stream = c->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  int rc = AQC_OK;
  if (e == cudaSuccess) {
    for (int j = 0; j < K && rc == AQC_OK; j++) {
      c->cur_wdev = c->d_wdev + kGraphStepWeights * j;
      rc = pec_step(c);
      c->step++;
    }
    c->cur_wdev = nullptr;
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e_end = e == cudaSuccess ? cudaStreamEndCapture(c->cap_stream, &graph) : e;
  c->stream = user;
  c->g_launches = c->launches - launches0;
  c->g_q_ready_end = c->q_ready;
  c->step = step0;
  c->evals = evals0;
  c->launches = launches0;
  c->q_ready = q_ready0;
  if (rc != AQC_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess || e_end != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    FAIL(c, AQC_E_CUDA, "capture of %d PEC steps: %s", K, cudaGetErrorString(e != cudaSuccess ? e : e_end));
  }
  e = cudaGraphInstantiate(&c->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    c->gexec = nullptr;
    FAIL(c, AQC_E_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  c->gkey = graph_key(c, K);  // the key of the state the replays start from
  return AQC_OK;
}

// K PEC steps of the fixed-step grid as one graph replay (the caller checked that K steps
// remain in the segment and in the call's step budget).
int pec_steps_graph(aqc_ctx* c, int K) {
  if (!c->gexec || !same_key(graph_key(c, K), c->gkey)) {
    int rc = capture_steps(c, K);
    if (rc) return rc;
  }
  double wb[kGraphStepWeights * kMaxGraphSteps];
  for (int j = 0; j < K; j++) {
    sched_weights(c, c->seg_t0 + (double)(c->step + j + 2) * c->h, wb + kGraphStepWeights * j + 3);
    sched_weights(c, c->seg_t0 + (double)(c->step + j + 1) * c->h, wb + kGraphStepWeights * j);
  }
  CUDA_TRY(c, launch_set_weights(c->d_wdev, wb, kGraphStepWeights * K, c->stream));
  CUDA_TRY(c, cudaGraphLaunch(c->gexec, c->stream));
  c->launches += 1 + c->g_launches;
  c->evals += K;
  c->graph_replays++;
  c->q_ready = c->g_q_ready_end;
  for (int j = 0; j < K; j++) count_step(c);
  return AQC_OK;
}

int read_slot(aqc_ctx* c, int slot, double* out) {
  CUDA_TRY(c, cudaMemcpyAsync(out, c->d_slots + slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return AQC_OK;
}

}  // namespace


// ---------------------------------------------------------------------------------------
// Batches: many contexts stepped together by k_batch, K PEC steps per CUDA-graph replay.
// ---------------------------------------------------------------------------------------
struct aqc_batch {
  int device = 0, prec = 0, max_members = 0;
  int64_t max_items = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char* ws = nullptr;
  BatchInst* d_insts = nullptr;
  BatchItem* d_items[kMaxLayouts] = {nullptr};
  double* d_partials = nullptr;
  std::vector<aqc_ctx*> members;   // slot -> context (nullptr = free)
  std::vector<int64_t> step_at_add;
  std::vector<BatchInst> h_insts;  // host copy (refreshed by poll / rebuild)
  int nitems[kMaxLayouts] = {0};
  int smem[kMaxLayouts] = {0};
  int nlevels = 0;
  bool dirty = true;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  int threads = 256, steps_per_round = 16;
  int64_t launches = 0;
  std::string err;
};

namespace {

struct BatchPlan {
  size_t off_insts, off_items, off_partials, total;
};

BatchPlan plan_batch(int max_members, int64_t max_items) {
  BatchPlan b;
  b.off_insts = 0;
  b.off_items = align_up((size_t)max_members * sizeof(BatchInst), 256);
  b.off_partials = align_up(b.off_items + (size_t)kMaxLayouts * (size_t)max_items * sizeof(BatchItem), 256);
  b.total = align_up(b.off_partials + (size_t)max_items * 2 * sizeof(double), 256);
  return b;
}

#define BFAIL(b, code, ...)                    \
  do {                                         \
    char buf_[512];                            \
    snprintf(buf_, sizeof(buf_), __VA_ARGS__); \
    (b)->err = buf_;                           \
    return (code);                             \
  } while (0)

#define BCUDA(b, expr)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) BFAIL(b, AQC_E_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

void fill_inst(const aqc_ctx* c, BatchInst* I) {
  memset(I, 0, sizeof(*I));
  I->tab = c->d_tab;
  I->dcode = c->table_class >= 0 ? c->d_dcode : nullptr;
  for (int v = 0; v < kVecCount; v++) I->vec[v] = c->vec[v];
  I->nl = (int)c->layouts.size();
  for (int l = 0; l < I->nl; l++) I->layouts[l] = c->layouts[l];
  I->s_kind = c->s_kind;
  I->T = c->T;
  I->h = c->h;
  for (int g = 0; g < 3; g++)
    for (int k = 0; k < 4; k++) I->poly[g][k] = c->poly[g][k];
  I->step = c->step;
  I->nsteps = c->nsteps;
}

int batch_pull(aqc_batch* b) {
  if (b->max_members == 0) return AQC_OK;
  BCUDA(b, cudaMemcpyAsync(b->h_insts.data(), b->d_insts, sizeof(BatchInst) * b->max_members, cudaMemcpyDeviceToHost,
                           b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  return AQC_OK;
}

void drop_graph(aqc_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
}

// work lists + per-level shared memory + one captured graph of K batched grid steps
int batch_rebuild(aqc_batch* b) {
  int rc = batch_pull(b);
  if (rc) return rc;
  std::vector<BatchItem> items[kMaxLayouts];
  int smem[kMaxLayouts] = {0};
  int nlev = 0;
  for (int slot = 0; slot < b->max_members; slot++) {
    aqc_ctx* c = b->members[slot];
    if (!c) continue;
    BatchInst& I = b->h_insts[slot];
    const int nl = (int)c->layouts.size();
    nlev = std::max(nlev, nl);
    for (int l = 0; l < nl; l++) {
      const uint32_t ntiles = 1u << (c->n - c->layouts[l].t);
      if (l == 0) I.item_begin = (uint32_t)items[0].size();
      for (uint32_t t = 0; t < ntiles; t++) items[l].push_back(BatchItem{(uint32_t)slot, t});
      if (l == 0) I.item_end = (uint32_t)items[0].size();
      const bool first = (l == nl - 1), diag = (l == diag_level(nl));
      const size_t sm = apply_smem_bytes(c->prec, c->layouts[l].t, c->nplain[l],
                                         c->ngeneral[l] + (first ? c->n_remote : 0), diag ? c->n_z : 0);
      if (sm > 227 * 1024) BFAIL(b, AQC_E_UNSUPPORTED, "shared memory %zu bytes too large", sm);
      smem[l] = std::max(smem[l], (int)sm);
    }
    I.ticket = 0;
  }
  for (int l = 0; l < nlev; l++) {
    if ((int64_t)items[l].size() > b->max_items) BFAIL(b, AQC_E_NOMEM, "batch needs %zu work items > max_items", items[l].size());
    if (!items[l].empty())
      BCUDA(b, cudaMemcpyAsync(b->d_items[l], items[l].data(), items[l].size() * sizeof(BatchItem),
                               cudaMemcpyHostToDevice, b->stream));
    b->nitems[l] = (int)items[l].size();
    b->smem[l] = smem[l];
  }
  for (int l = nlev; l < kMaxLayouts; l++) b->nitems[l] = 0;
  b->nlevels = nlev;
  BCUDA(b, cudaMemcpyAsync(b->d_insts, b->h_insts.data(), sizeof(BatchInst) * b->max_members, cudaMemcpyHostToDevice,
                           b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  drop_graph(b);
  if (nlev > 0) {
    BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < b->steps_per_round && e == cudaSuccess; k++) {
      for (int l = nlev - 1; l >= 0 && e == cudaSuccess; l--) {
        BatchLaunch bl;
        bl.items = b->d_items[l];
        bl.insts = b->d_insts;
        bl.partials = b->d_partials;
        bl.level = l;
        e = launch_batch(b->prec, b->threads, bl, b->nitems[l], b->smem[l], b->stream);
      }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      BFAIL(b, AQC_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    b->graph = g;
    BCUDA(b, cudaGraphInstantiate(&b->gexec, g, 0));
  }
  b->dirty = false;
  return AQC_OK;
}

}  // namespace

namespace aqc {
void set_global_error(const char* msg) { g_create_error = msg; }
}  // namespace aqc

namespace {

// Wait for and destroy the copy streams and events of the staged transfers.
void release_transfers(aqc_ctx* c) {
  if (c->copy_in) cudaStreamSynchronize(c->copy_in);
  if (c->copy_out) cudaStreamSynchronize(c->copy_out);
  cudaEvent_t* evs[4] = {&c->ev_in_ready, &c->ev_in_free, &c->ev_out_ready, &c->ev_out_free};
  for (cudaEvent_t* e : evs) {
    if (*e) cudaEventDestroy(*e);
    *e = nullptr;
  }
  if (c->copy_in) cudaStreamDestroy(c->copy_in);
  if (c->copy_out) cudaStreamDestroy(c->copy_out);
  c->copy_in = c->copy_out = nullptr;
  c->stage_in = c->stage_out = nullptr;
  c->stage_pending = false;
}

}  // namespace

extern "C" {

size_t aqc_workspace_bytes_ex(int n_qubits, int precision, unsigned flags) {
  if (n_qubits < 1 || n_qubits > kMaxN) return 0;
  if (precision != AQC_C128 && precision != AQC_C64) return 0;
  if (flags & ~(unsigned)AQC_WS_STEP_CONTROL) return 0;
  return plan_workspace(n_qubits, precision, flags).total;
}

size_t aqc_workspace_bytes(int n_qubits, int precision) { return aqc_workspace_bytes_ex(n_qubits, precision, 0); }

int aqc_create(aqc_ctx** out, int device, int precision, int n_qubits, void* workspace, size_t workspace_bytes,
               void* cuda_stream) {
  if (!out) {
    g_create_error = "out is NULL";
    return AQC_E_INVAL;
  }
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > kMaxN || (precision != AQC_C128 && precision != AQC_C64)) {
    g_create_error = "n_qubits must be in [1, 31] and precision AQC_C128 or AQC_C64";
    return AQC_E_INVAL;
  }
  const WsPlan wp = plan_workspace(n_qubits, precision);
  if (!workspace || workspace_bytes < wp.total) {
    g_create_error = "workspace missing or smaller than aqc_workspace_bytes()";
    return AQC_E_NOMEM;
  }
  if (((uintptr_t)workspace) & 255u) {
    g_create_error = "workspace must be 256-byte aligned";
    return AQC_E_INVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    g_create_error = "no such CUDA device";
    return AQC_E_CUDA;
  }
  aqc_ctx* c = new (std::nothrow) aqc_ctx();
  if (!c) {
    g_create_error = "host allocation failed";
    return AQC_E_NOMEM;
  }
  c->h_tab = new (std::nothrow) DevTables();
  if (!c->h_tab) {
    delete c;
    g_create_error = "host allocation failed";
    return AQC_E_NOMEM;
  }
  c->device = device;
  c->prec = precision;
  c->n = n_qubits;
  c->N = (uint64_t)1 << n_qubits;
  c->amp = precision == AQC_C128 ? 16 : 8;
  c->stream = (cudaStream_t)cuda_stream;
  c->ws = (char*)workspace;
  c->wp = wp;
  c->d_tab = (DevTables*)(c->ws + wp.off_tab);
  c->d_slots = (double*)(c->ws + wp.off_slots);
  c->d_counter = (unsigned*)(c->ws + wp.off_counter);
  c->d_sync = (unsigned*)(c->ws + wp.off_sync);
  c->d_perm = (uint32_t*)(c->ws + wp.off_perm);
  c->d_partials = (double*)(c->ws + wp.off_partials);
  c->d_wdev = (double*)(c->ws + wp.off_wdev);
  c->d_dcode = (uint8_t*)(c->ws + wp.off_dcode);
  for (int v = 0; v < V_COUNT; v++) c->vec[v] = c->ws + wp.off_vec + (size_t)v * wp.vec_bytes;
  if (workspace_bytes >= plan_workspace(n_qubits, precision, AQC_WS_STEP_CONTROL).total)
    c->vec_save = c->ws + wp.off_vec + (size_t)V_COUNT * wp.vec_bytes;
  for (int g = 0; g < 3; g++)
    for (int k = 0; k < 4; k++) c->poly[g][k] = 0.0;
  DeviceGuard dg(device);
  if (cudaMemsetAsync(c->ws + wp.off_slots, 0, wp.off_partials - wp.off_slots, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    g_create_error = "cudaMemsetAsync on the workspace failed";
    delete c->h_tab;
    delete c;
    return AQC_E_CUDA;
  }
  *out = c;
  return AQC_OK;
}

void aqc_destroy(aqc_ctx* ctx) {
  if (!ctx) return;
  {
    DeviceGuard dg(ctx->device);
    release_transfers(ctx);
    drop_step_graph(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  }
  delete ctx->h_tab;
  delete ctx;
}

int aqc_set_stream(aqc_ctx* ctx, void* cuda_stream) {
  if (!ctx) return AQC_E_INVAL;
  ctx->stream = (cudaStream_t)cuda_stream;
  return AQC_OK;
}

int aqc_load_terms(aqc_ctx* ctx, int group, size_t n_terms, const uint64_t* xmask, const uint64_t* zmask,
                   const double* coef) {
  if (!ctx) return AQC_E_INVAL;
  if (group < 0 || group > 2) FAIL(ctx, AQC_E_INVAL, "group must be 0, 1 or 2");
  if (n_terms && (!xmask || !zmask || !coef)) FAIL(ctx, AQC_E_INVAL, "NULL term array");
  const uint64_t lim = ctx->N;
  for (size_t k = 0; k < n_terms; k++) {
    if (xmask[k] >= lim || zmask[k] >= lim) FAIL(ctx, AQC_E_INVAL, "term %zu: mask >= 2^n", k);
    if (!isfinite(coef[k])) FAIL(ctx, AQC_E_INVAL, "term %zu: non-finite coefficient", k);
  }
  for (size_t k = 0; k < n_terms; k++) ctx->terms.push_back(TermH{(uint32_t)xmask[k], (uint32_t)zmask[k], coef[k], group});
  ctx->dirty = true;
  return AQC_OK;
}

int aqc_load_clauses(aqc_ctx* ctx, int group, size_t m, const int32_t* bits, int penalty, double scale) {
  if (!ctx) return AQC_E_INVAL;
  if (group < 0 || group > 2) FAIL(ctx, AQC_E_INVAL, "group must be 0, 1 or 2");
  const int stepwise = (penalty & AQC_CLAUSE_STEPWISE) ? 1 : 0;
  penalty &= ~AQC_CLAUSE_STEPWISE;
  if (penalty != AQC_PEN_INDICATOR && penalty != AQC_PEN_SQUARED) FAIL(ctx, AQC_E_INVAL, "bad penalty kind");
  if (stepwise) {
    for (const ClauseH& c : ctx->clauses)
      if (c.stepwise) FAIL(ctx, AQC_E_INVAL, "the context already holds a clause-by-clause sequence");
    if (m == 0) FAIL(ctx, AQC_E_INVAL, "empty clause-by-clause sequence");
  }
  if (!isfinite(scale)) FAIL(ctx, AQC_E_INVAL, "non-finite scale");
  if (m && !bits) FAIL(ctx, AQC_E_INVAL, "NULL clause array");
  for (size_t k = 0; k < m; k++) {
    const int a = bits[3 * k], b = bits[3 * k + 1], d = bits[3 * k + 2];
    if (a < 0 || b < 0 || d < 0 || a >= ctx->n || b >= ctx->n || d >= ctx->n || a == b || b == d || a == d)
      FAIL(ctx, AQC_E_INVAL, "clause %zu: bits must be distinct and < n", k);
  }
  for (size_t k = 0; k < m; k++) {
    const uint32_t mask = (1u << bits[3 * k]) | (1u << bits[3 * k + 1]) | (1u << bits[3 * k + 2]);
    ctx->clauses.push_back(ClauseH{mask, group, penalty, scale, stepwise});
  }
  ctx->dirty = true;
  return AQC_OK;
}

int aqc_clear_hamiltonian(aqc_ctx* ctx) {
  if (!ctx) return AQC_E_INVAL;
  ctx->terms.clear();
  ctx->clauses.clear();
  ctx->dirty = true;
  return AQC_OK;
}

int aqc_set_schedule(aqc_ctx* ctx, int s_kind, double T, const double coefA[4], const double coefB[4],
                     const double coefC[4]) {
  if (!ctx) return AQC_E_INVAL;
  if (s_kind != AQC_S_LINEAR && s_kind != AQC_S_SMOOTHSTEP) FAIL(ctx, AQC_E_INVAL, "bad s_kind");
  if (!(T > 0.0) || !isfinite(T)) FAIL(ctx, AQC_E_INVAL, "T must be positive and finite");
  const double* cs[3] = {coefA, coefB, coefC};
  for (int g = 0; g < 3; g++)
    for (int k = 0; k < 4; k++) {
      const double v = cs[g] ? cs[g][k] : 0.0;
      if (!isfinite(v)) FAIL(ctx, AQC_E_INVAL, "non-finite schedule coefficient");
      ctx->poly[g][k] = v;
    }
  ctx->s_kind = s_kind;
  ctx->T = T;
  ctx->have_sched = true;
  ctx->have_state = false;  // a new schedule restarts the integration
  return AQC_OK;
}

int aqc_set_tile_bits(aqc_ctx* ctx, int tile_bits) {
  if (!ctx) return AQC_E_INVAL;
  const int lo = chunk_bits(ctx->prec) + 1, hi = tile_bits_max(ctx->prec);
  const bool cluster = ctx->prec == AQC_C64 && tile_bits == kClusterTileBits;
  if (tile_bits != 0 && !cluster && (tile_bits < lo || tile_bits > hi))
    FAIL(ctx, AQC_E_INVAL, "tile_bits must be 0, in [%d, %d], or 16 (complex64 cluster tiles)", lo, hi);
  ctx->tile_bits = tile_bits;
  ctx->dirty = true;
  ctx->have_state = false;
  return AQC_OK;
}

int aqc_set_relabel(aqc_ctx* ctx, int enable) {
  if (!ctx) return AQC_E_INVAL;
  ctx->relabel = enable ? 1 : 0;
  ctx->dirty = true;  // a state already set moves to the new order at the next table build
  return AQC_OK;
}

int aqc_set_graph_steps(aqc_ctx* ctx, int k_steps) {
  if (!ctx) return AQC_E_INVAL;
  if (!(k_steps == -1 || k_steps == 0 || (k_steps >= 4 && k_steps <= kMaxGraphSteps && k_steps % 4 == 0)))
    FAIL(ctx, AQC_E_INVAL, "k_steps must be -1, 0 or a multiple of 4 in [4, %d]", kMaxGraphSteps);
  ctx->graph_req = k_steps;
  DeviceGuard dg(ctx->device);
  drop_step_graph(ctx);
  return AQC_OK;
}

int aqc_measure_fp64_fma(int device, void* cuda_stream, int iters, double* tflops_out, double* ms_out) {
  if (!tflops_out || iters < 1 || iters > (1 << 24)) {
    g_create_error = "tflops_out must be non-NULL and iters in [1, 2^24]";
    return AQC_E_INVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    g_create_error = "no such CUDA device";
    return AQC_E_CUDA;
  }
  DeviceGuard dg(device);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    g_create_error = "cudaDeviceGetAttribute failed";
    return AQC_E_CUDA;
  }
  const int blocks = 4 * sms;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch_fma64(blocks, iters / 8 + 1, s);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = launch_fma64(blocks, iters, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || !(ms > 0.f)) {
    g_create_error = std::string("FP64 FMA timing: ") + cudaGetErrorString(e);
    return AQC_E_CUDA;
  }
  *tflops_out = 2.0 * (double)fma64_count(blocks, iters) / ((double)ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return AQC_OK;
}

int aqc_set_y_compensation(aqc_ctx* ctx, int enable) {
  if (!ctx) return AQC_E_INVAL;
  if (enable) {
    if (ctx->prec != AQC_C64) FAIL(ctx, AQC_E_UNSUPPORTED, "y compensation is for complex64 states");
    if (!ctx->vec_save)
      FAIL(ctx, AQC_E_NOMEM, "y compensation needs the workspace's extra vector (AQC_WS_Y_COMPENSATION)");
    if (ctx->adaptive) FAIL(ctx, AQC_E_UNSUPPORTED, "y compensation and step-size control are exclusive");
  }
  ctx->ycomp = enable ? 1 : 0;
  ctx->have_state = false;  // the integrator restarts from a new initial state
  DeviceGuard dg(ctx->device);
  drop_step_graph(ctx);
  return AQC_OK;
}

int aqc_wait_selftest(aqc_ctx* ctx, int64_t polls) {
  if (!ctx) return AQC_E_INVAL;
  if (polls < 1 || polls > 10000000) FAIL(ctx, AQC_E_INVAL, "polls must be in [1, 10^7]");
  DeviceGuard dg(ctx->device);
  unsigned* flag = reinterpret_cast<unsigned*>(ctx->d_slots + kSlotWaitFlag);
  CUDA_TRY(ctx, cudaMemsetAsync(flag, 0, sizeof(double), ctx->stream));
  CUDA_TRY(ctx, launch_wait_flag(flag, polls, ctx->d_slots, ctx->stream));
  ctx->launches++;
  double fault = 0.0;
  CUDA_TRY(ctx, cudaMemcpyAsync(&fault, ctx->d_slots + kSlotFault, sizeof(double), cudaMemcpyDeviceToHost,
                                ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (fault != 0.0) {
    const double zero = 0.0;
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_slots + kSlotFault, &zero, sizeof(double), cudaMemcpyHostToDevice,
                                  ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    FAIL(ctx, AQC_E_TIMEOUT, "the wait gave up after %lld polls (self-test: nothing sets its flag)",
         (long long)polls);
  }
  return AQC_OK;
}

int aqc_set_layout_turns(aqc_ctx* ctx, int mode) {
  if (!ctx) return AQC_E_INVAL;
  if (mode < -1 || mode > 1) FAIL(ctx, AQC_E_INVAL, "mode must be -1, 0 or 1");
  ctx->turn_req = mode;
  ctx->q_ready = -1;
  DeviceGuard dg(ctx->device);
  drop_step_graph(ctx);
  return AQC_OK;
}

int aqc_set_grid_limit(aqc_ctx* ctx, int max_ctas) {
  if (!ctx) return AQC_E_INVAL;
  if (max_ctas < 0) FAIL(ctx, AQC_E_INVAL, "max_ctas must be >= 0");
  ctx->grid_limit = max_ctas;
  DeviceGuard dg(ctx->device);
  drop_step_graph(ctx);  // captured launches carry the grid size
  return AQC_OK;
}

int aqc_get_graph_replays(const aqc_ctx* ctx, int64_t* out) {
  if (!ctx || !out) return AQC_E_INVAL;
  *out = ctx->graph_replays;
  return AQC_OK;
}

int aqc_set_slab_bits(aqc_ctx* ctx, int slab_bits) {
  if (!ctx) return AQC_E_INVAL;
  if (slab_bits < -1 || slab_bits > 11) FAIL(ctx, AQC_E_INVAL, "slab_bits must be -1, 0 or 1..11");
  ctx->slab_req = slab_bits;
  if (!ctx->dirty) plan_slabs(ctx);
  return AQC_OK;
}

int aqc_set_integrator(aqc_ctx* ctx, int64_t n_steps, double kappa, int adaptive, double tol) {
  if (!ctx) return AQC_E_INVAL;
  if (n_steps < 0) FAIL(ctx, AQC_E_INVAL, "n_steps must be >= 0");
  if (kappa < 0.0 || !isfinite(kappa)) FAIL(ctx, AQC_E_INVAL, "kappa must be >= 0");
  if (adaptive != 0 && adaptive != 1) FAIL(ctx, AQC_E_INVAL, "adaptive must be 0 or 1");
  if (adaptive && !(tol > 0.0 && isfinite(tol))) FAIL(ctx, AQC_E_INVAL, "tol must be positive and finite");
  if (adaptive && ctx->in_batch) FAIL(ctx, AQC_E_STATE, "a batch member cannot take step-size control");
  if (adaptive && ctx->ycomp) FAIL(ctx, AQC_E_UNSUPPORTED, "step-size control and y compensation are exclusive");
  if (adaptive && !ctx->vec_save)
    FAIL(ctx, AQC_E_NOMEM, "the workspace has no room for step-size control (aqc_workspace_bytes_ex with "
                           "AQC_WS_STEP_CONTROL)");
  ctx->nsteps_req = n_steps;
  ctx->kappa = kappa > 0.0 ? kappa : 0.1;
  ctx->adaptive = adaptive;
  ctx->tol = adaptive ? tol : 0.0;
  ctx->have_state = false;
  return AQC_OK;
}

int aqc_set_step_growth(aqc_ctx* ctx, int grow_after) {
  if (!ctx) return AQC_E_INVAL;
  if (grow_after < 0) FAIL(ctx, AQC_E_INVAL, "grow_after must be >= 0");
  ctx->grow_after = grow_after;
  return AQC_OK;
}

int aqc_get_grid(aqc_ctx* ctx, int64_t* n_steps, double* h) {
  if (!ctx) return AQC_E_INVAL;
  if (!ctx->have_sched) FAIL(ctx, AQC_E_STATE, "no schedule set");
  const int64_t N = ctx->nsteps > 0 ? ctx->nsteps : (ctx->nsteps_req > 0 ? ctx->nsteps_req : rule_steps(ctx));
  // (under step-size control: the initial grid, whose step the first segment takes)
  if (n_steps) *n_steps = N;
  if (h) *h = ctx->T / (double)N;
  return AQC_OK;
}

int aqc_set_initial_state(aqc_ctx* ctx, int kind, uint64_t basis, const void* user) {
  if (!ctx) return AQC_E_INVAL;
  DeviceGuard dg(ctx->device);
  if (ctx->dirty) {  // the qubit order of the vectors must be known
    ctx->have_state = false;
    int rc = build_tables(ctx);
    if (rc) return rc;
  }
  void* y = ctx->vec[V_Y];
  const size_t bytes = (size_t)ctx->N * ctx->amp;
  switch (kind) {
    case AQC_INIT_UNIFORM:
      CUDA_TRY(ctx, launch_init(ctx->prec, y, ctx->N, 0, 0, 0.0, ctx->stream));
      ctx->launches++;
      break;
    case AQC_INIT_BASIS:
      if (basis >= ctx->N) FAIL(ctx, AQC_E_INVAL, "basis index >= 2^n");
      CUDA_TRY(ctx, launch_init(ctx->prec, y, ctx->N, 1, phys_index(ctx, basis), 0.0, ctx->stream));
      ctx->launches++;
      break;
    case AQC_INIT_DICKE: {
      if (basis > (uint64_t)ctx->n) FAIL(ctx, AQC_E_INVAL, "Hamming weight %llu > n", (unsigned long long)basis);
      double binom = 1.0;  // C(n, k), exact in FP64 for n <= 31
      for (uint64_t i = 1; i <= basis; i++) binom = binom * (double)(ctx->n - basis + i) / (double)i;
      CUDA_TRY(ctx, launch_init(ctx->prec, y, ctx->N, 2, basis, 1.0 / sqrt(binom), ctx->stream));
      ctx->launches++;
      break;
    }
    case AQC_INIT_USER_HOST:
      if (!user) FAIL(ctx, AQC_E_INVAL, "user vector is NULL");
      CUDA_TRY(ctx, cudaMemcpyAsync(ctx->permuted ? ctx->vec[V_ACC] : y, user, bytes, cudaMemcpyHostToDevice,
                                    ctx->stream));
      if (ctx->permuted) {
        int rc = to_library_order(ctx, y, ctx->vec[V_ACC]);
        if (rc) return rc;
      }
      break;
    case AQC_INIT_STAGED:
      if (!ctx->stage_pending) FAIL(ctx, AQC_E_STATE, "no staged initial state (aqc_stage_initial_state)");
      CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_in_ready, 0));
      if (ctx->permuted) {
        int rc = to_library_order(ctx, y, ctx->stage_in);
        if (rc) return rc;
      } else {
        CUDA_TRY(ctx, cudaMemcpyAsync(y, ctx->stage_in, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      }
      CUDA_TRY(ctx, cudaEventRecord(ctx->ev_in_free, ctx->stream));
      ctx->stage_pending = false;
      break;
    case AQC_INIT_USER_DEVICE:
      if (!user) FAIL(ctx, AQC_E_INVAL, "user vector is NULL");
      if (ctx->permuted) {
        int rc = to_library_order(ctx, y, user);
        if (rc) return rc;
      } else {
        CUDA_TRY(ctx, cudaMemcpyAsync(y, user, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      }
      break;
    default:
      FAIL(ctx, AQC_E_INVAL, "bad initial-state kind");
  }
  CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_slots, 0, kSlotCount * sizeof(double), ctx->stream));
  ctx->step = 0;
  ctx->evals = 0;
  ctx->nsteps = 0;
  ctx->hist_ready = false;
  ctx->q_ready = -1;
  ctx->steps_done = 0;
  ctx->at_end = false;
  ctx->rejects = 0;
  ctx->max_err_acc = 0.0;
  ctx->seg_t0 = 0.0;
  ctx->seg_m = 0;
  ctx->segs.clear();
  ctx->have_state = true;
  return AQC_OK;
}

int aqc_propagate(aqc_ctx* ctx, int64_t max_steps, aqc_stats* stats) {
  if (!ctx) return AQC_E_INVAL;
  if (!ctx->have_state) FAIL(ctx, AQC_E_STATE, "no initial state (or schedule/integrator changed since)");
  DeviceGuard dg(ctx->device);
  int rc = ensure_ready(ctx);
  if (rc) return rc;
  rc = plan_first_segment(ctx);
  if (rc) return rc;
  const int64_t target = max_steps < 0 ? INT64_MAX : ctx->steps_done + max_steps;
  const int64_t launches0 = ctx->launches;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (stats) {
    CUDA_TRY(ctx, cudaEventCreate(&e0));
    CUDA_TRY(ctx, cudaEventCreate(&e1));
    CUDA_TRY(ctx, cudaEventRecord(e0, ctx->stream));
  }
  while (!ctx->at_end && ctx->steps_done < target) {
    if (ctx->step < 3) {
      rc = rk4_step(ctx);
      if (!rc) count_step(ctx);
    } else {
      if (!ctx->hist_ready) {
        rc = start_history(ctx);
        if (rc) break;
      }
      const int K = graph_k(ctx);
      if (K > 0 && ctx->seg_m - ctx->step >= K && target - ctx->steps_done >= K) {
        rc = pec_steps_graph(ctx, K);
        if (rc) break;
        continue;
      }
      rc = pec_step(ctx);
      if (!rc) {
        if (ctx->adaptive)
          rc = control_step(ctx);
        else
          count_step(ctx);
      }
    }
    if (rc) break;
  }
  if (stats) {
    cudaEventRecord(e1, ctx->stream);
    if (!rc) {
      memset(stats, 0, sizeof(*stats));
      stats->steps_done = ctx->steps_done;
      stats->n_steps = ctx->adaptive ? ctx->steps_done + (ctx->seg_m - ctx->step) : ctx->nsteps;
      stats->evaluations = ctx->evals;
      stats->h = ctx->h;
      stats->t = ctx->seg_t0 + (double)ctx->step * ctx->h;
      stats->launches = ctx->launches - launches0;
      stats->rejects = ctx->rejects;
      stats->segments = (int64_t)ctx->segs.size();
      cudaError_t e = launch_reduce(ctx->prec, 0, ctx->vec[V_Y], ctx->N, ctx->d_partials, ctx->d_counter,
                                    ctx->d_slots, reduce_grid(ctx->N), ctx->stream);
      ctx->launches++;
      double sl[kSlotCount];
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl, ctx->d_slots, sizeof(sl), cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        ctx->err = std::string("stats readback: ") + cudaGetErrorString(e);
        rc = AQC_E_CUDA;
      } else {
        stats->norm2 = sl[kSlotNorm2];
        stats->max_err_est = ctx->adaptive ? ctx->max_err_acc : sl[kSlotMaxErr];
        stats->last_err_est = sl[kSlotLastErr];
        stats->elapsed_ms = ms;
        if (sl[kSlotFault] != 0.0) {
          ctx->err = "a kernel gave up waiting (a tile copy or a slab's partial sums); results are invalid";
          rc = AQC_E_TIMEOUT;
          const double zero = 0.0;
          cudaMemcpyAsync(ctx->d_slots + kSlotFault, &zero, sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
          cudaStreamSynchronize(ctx->stream);
        } else if (!isfinite(sl[kSlotNorm2])) {
          ctx->err = "non-finite state norm";
          rc = AQC_E_NUMERIC;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  return rc;
}

int aqc_get_segments(aqc_ctx* ctx, aqc_segment* out, int64_t max_out, int64_t* count) {
  if (!ctx) return AQC_E_INVAL;
  if (max_out < 0 || (max_out > 0 && !out)) FAIL(ctx, AQC_E_INVAL, "out is NULL or max_out < 0");
  const int64_t n = (int64_t)ctx->segs.size();
  for (int64_t i = 0; i < n && i < max_out; i++) out[i] = ctx->segs[(size_t)i];
  if (count) *count = n;
  return AQC_OK;
}

int aqc_get_state(aqc_ctx* ctx, void* dst, int dst_on_device) {
  if (!ctx) return AQC_E_INVAL;
  if (!dst) FAIL(ctx, AQC_E_INVAL, "dst is NULL");
  DeviceGuard dg(ctx->device);
  const void* src = ctx->vec[V_Y];
  if (ctx->permuted) {  // back to qubit order: on the device directly, or via the scratch vector
    int rc = to_qubit_order(ctx, dst_on_device ? dst : ctx->vec[V_ACC], ctx->vec[V_Y]);
    if (rc) return rc;
    src = ctx->vec[V_ACC];
  }
  if (!(ctx->permuted && dst_on_device))
    CUDA_TRY(ctx, cudaMemcpyAsync(dst, src, (size_t)ctx->N * ctx->amp,
                                  dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return AQC_OK;
}

int aqc_transfer_attach(aqc_ctx* ctx, void* stage_in, void* stage_out) {
  if (!ctx) return AQC_E_INVAL;
  if (!stage_in || !stage_out) FAIL(ctx, AQC_E_INVAL, "staging vector is NULL");
  if ((((uintptr_t)stage_in) | ((uintptr_t)stage_out)) & 255u) FAIL(ctx, AQC_E_INVAL, "staging vectors must be 256-byte aligned");
  const size_t bytes = (size_t)ctx->N * ctx->amp;
  const char *a = (const char*)stage_in, *b = (const char*)stage_out;
  if (a < b + bytes && b < a + bytes) FAIL(ctx, AQC_E_INVAL, "staging vectors overlap");
  const char *w0 = ctx->ws, *w1 = ctx->ws + ctx->wp.total;
  if ((a < w1 && w0 < a + bytes) || (b < w1 && w0 < b + bytes)) FAIL(ctx, AQC_E_INVAL, "staging vector overlaps the workspace");
  DeviceGuard dg(ctx->device);
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // nothing of the context still reads the old vectors
  release_transfers(ctx);
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking);
  cudaEvent_t* evs[4] = {&ctx->ev_in_ready, &ctx->ev_in_free, &ctx->ev_out_ready, &ctx->ev_out_free};
  for (cudaEvent_t* ev : evs)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    release_transfers(ctx);
    FAIL(ctx, AQC_E_CUDA, "copy stream / event creation: %s", cudaGetErrorString(e));
  }
  // never-recorded events count as complete: the first stage and fetch wait for nothing
  ctx->stage_in = stage_in;
  ctx->stage_out = stage_out;
  return AQC_OK;
}

int aqc_stage_initial_state(aqc_ctx* ctx, const void* host_src) {
  if (!ctx) return AQC_E_INVAL;
  if (!host_src) FAIL(ctx, AQC_E_INVAL, "host_src is NULL");
  if (!ctx->stage_in) FAIL(ctx, AQC_E_STATE, "no staging vectors (aqc_transfer_attach)");
  DeviceGuard dg(ctx->device);
  CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->copy_in, ctx->ev_in_free, 0));
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->stage_in, host_src, (size_t)ctx->N * ctx->amp, cudaMemcpyHostToDevice,
                                ctx->copy_in));
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev_in_ready, ctx->copy_in));
  ctx->stage_pending = true;
  return AQC_OK;
}

int aqc_fetch_state(aqc_ctx* ctx, void* host_dst) {
  if (!ctx) return AQC_E_INVAL;
  if (!host_dst) FAIL(ctx, AQC_E_INVAL, "host_dst is NULL");
  if (!ctx->stage_out) FAIL(ctx, AQC_E_STATE, "no staging vectors (aqc_transfer_attach)");
  DeviceGuard dg(ctx->device);
  const size_t bytes = (size_t)ctx->N * ctx->amp;
  CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_out_free, 0));
  if (ctx->permuted) {
    int rc = to_qubit_order(ctx, ctx->stage_out, ctx->vec[V_Y]);
    if (rc) return rc;
  } else {
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->stage_out, ctx->vec[V_Y], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev_out_ready, ctx->stream));
  CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->copy_out, ctx->ev_out_ready, 0));
  CUDA_TRY(ctx, cudaMemcpyAsync(host_dst, ctx->stage_out, bytes, cudaMemcpyDeviceToHost, ctx->copy_out));
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev_out_free, ctx->copy_out));
  return AQC_OK;
}

int aqc_transfer_wait(aqc_ctx* ctx) {
  if (!ctx) return AQC_E_INVAL;
  if (!ctx->stage_in) return AQC_OK;
  DeviceGuard dg(ctx->device);
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->copy_in));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->copy_out));
  return AQC_OK;
}

int aqc_fidelity(aqc_ctx* ctx, uint64_t w, double* out) {
  if (!ctx || !out) return AQC_E_INVAL;
  if (w >= ctx->N) FAIL(ctx, AQC_E_INVAL, "w >= 2^n");
  DeviceGuard dg(ctx->device);
  CUDA_TRY(ctx, launch_fidelity(ctx->prec, ctx->vec[V_Y], phys_index(ctx, w), ctx->d_slots, ctx->stream));
  ctx->launches++;
  return read_slot(ctx, kSlotDot, out);
}

int aqc_energy(aqc_ctx* ctx, int group_mask, double t, double* out) {
  if (!ctx || !out) return AQC_E_INVAL;
  if (group_mask < 1 || group_mask > 7) FAIL(ctx, AQC_E_INVAL, "group_mask must be in 1..7");
  if (!std::isfinite(t)) FAIL(ctx, AQC_E_INVAL, "t must be finite");
  DeviceGuard dg(ctx->device);
  if (ctx->dirty) {
    int rc = build_tables(ctx);
    if (rc) return rc;
  }
  double w[3] = {0.0, 0.0, 0.0};
  if (t >= 0.0) {
    if (!ctx->have_sched) FAIL(ctx, AQC_E_STATE, "no schedule set");
    sched_weights(ctx, t, w);  // also sets s(t) for a clause-by-clause sequence
    for (int g = 0; g < 3; g++)
      if (!((group_mask >> g) & 1)) w[g] = 0.0;
  } else {
    for (int g = 0; g < 3; g++) w[g] = ((group_mask >> g) & 1) ? 1.0 : 0.0;
    if (ctx->T > 0.0) ctx->eval_s = sched_s(ctx, ctx->seg_t0 + (double)ctx->step * ctx->h);  // s now
  }
  ApplyParams fin = base_params(ctx);
  fin.mode = MODE_ENERGY;
  int rc = evaluate(ctx, w, ctx->vec[V_Y], fin, nullptr);
  if (rc) return rc;
  return read_slot(ctx, kSlotDot, out);
}

int aqc_norm2(aqc_ctx* ctx, double* out) {
  if (!ctx || !out) return AQC_E_INVAL;
  DeviceGuard dg(ctx->device);
  CUDA_TRY(ctx, launch_reduce(ctx->prec, 0, ctx->vec[V_Y], ctx->N, ctx->d_partials, ctx->d_counter, ctx->d_slots,
                              reduce_grid(ctx->N), ctx->stream));
  ctx->launches++;
  return read_slot(ctx, kSlotNorm2, out);
}

// ---- Lanczos (spectrum along the path) ----------------------------------------------------
namespace {

// eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm sequence of the LDL^T pivots)
int sturm_below(const double* a, const double* b, int k, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < k; i++) {
    d = (a[i] - x) - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) cnt++;
  }
  return cnt;
}

// j-th smallest eigenvalue (0-based) by bisection inside the Gershgorin interval
double tridiag_eig(const double* a, const double* b, int k, int j) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; i++) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < k - 1 ? fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200; it++) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;  // interval at the resolution of doubles
    if (sturm_below(a, b, k, mid) > j)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Eigenvector of the symmetric tridiagonal (a, b) for the eigenvalue lam: inverse iteration with
// a row-pivoted LU of (T - lam I) (three sweeps from a fixed start), normalised, sign chosen so
// that s[0] >= 0.
void tridiag_eigvec(const double* a, const double* b, int k, double lam, double* s) {
  if (k == 1) {
    s[0] = 1.0;
    return;
  }
  std::vector<double> dd(k), du(k, 0.0), du2(k, 0.0), mult(k, 0.0);
  std::vector<char> piv(k, 0);
  double scale = 0.0;
  for (int i = 0; i < k; i++) scale = std::max(scale, fabs(a[i] - lam) + (i < k - 1 ? fabs(b[i]) : 0.0));
  const double tiny = std::max(scale, 1e-300) * 1e-18;
  for (int i = 0; i < k; i++) dd[i] = a[i] - lam;
  for (int i = 0; i < k - 1; i++) du[i] = b[i];
  for (int i = 0; i < k - 1; i++) {
    const double dl = b[i];
    if (fabs(dd[i]) >= fabs(dl)) {
      if (dd[i] == 0.0) dd[i] = tiny;
      mult[i] = dl / dd[i];
      dd[i + 1] -= mult[i] * du[i];
    } else {  // rows i and i+1 trade places
      piv[i] = 1;
      mult[i] = dd[i] / dl;
      dd[i] = dl;
      const double tmp = dd[i + 1];
      dd[i + 1] = du[i] - mult[i] * tmp;
      if (i < k - 2) {
        du2[i] = du[i + 1];
        du[i + 1] = -mult[i] * du2[i];
      }
      du[i] = tmp;
    }
  }
  if (dd[k - 1] == 0.0) dd[k - 1] = tiny;
  for (int i = 0; i < k; i++) s[i] = 1.0 + 0.01 * (double)(i % 7);
  for (int sweep = 0; sweep < 3; sweep++) {
    for (int i = 0; i < k - 1; i++) {
      if (!piv[i]) {
        s[i + 1] -= mult[i] * s[i];
      } else {
        const double t = s[i];
        s[i] = s[i + 1];
        s[i + 1] = t - mult[i] * s[i];
      }
    }
    s[k - 1] /= dd[k - 1];
    s[k - 2] = (s[k - 2] - du[k - 2] * s[k - 1]) / dd[k - 2];
    for (int i = k - 3; i >= 0; i--) s[i] = (s[i] - du[i] * s[i + 1] - du2[i] * s[i + 2]) / dd[i];
    double nrm = 0.0;
    for (int i = 0; i < k; i++) nrm += s[i] * s[i];
    nrm = sqrt(nrm);
    for (int i = 0; i < k; i++) s[i] /= nrm;
  }
  if (s[0] < 0.0)
    for (int i = 0; i < k; i++) s[i] = -s[i];
}

struct LzPlan {
  size_t ld_bytes, off_partials, off_coef, off_h, off_scal, total;
  uint32_t G;
};

LzPlan lanczos_plan(int n, int prec, int max_iter) {
  LzPlan p;
  const uint64_t N = (uint64_t)1 << n;
  const size_t amp = prec == AQC_C128 ? 16 : 8;
  p.ld_bytes = align_up(N * amp, 256);
  const size_t m = (size_t)max_iter + 1;
  p.G = lanczos_dot_blocks(N);
  p.off_partials = m * p.ld_bytes;
  p.off_coef = align_up(p.off_partials + m * p.G * 2 * sizeof(double), 256);
  p.off_h = align_up(p.off_coef + m * 2 * sizeof(double), 256);
  p.off_scal = align_up(p.off_h + m * 2 * sizeof(double), 256);
  p.total = p.off_scal + 256;
  return p;
}

}  // namespace

int aqc_hpsi(aqc_ctx* ctx, double t, const void* psi, void* out) {
  if (!ctx) return AQC_E_INVAL;
  if (!psi || !out || psi == out) FAIL(ctx, AQC_E_INVAL, "psi and out must be distinct device pointers");
  if (!ctx->have_sched) FAIL(ctx, AQC_E_STATE, "no schedule set");
  DeviceGuard dg(ctx->device);
  if (ctx->dirty) {
    int rc = build_tables(ctx);
    if (rc) return rc;
  }
  double w[3];
  sched_weights(ctx, t, w);
  ApplyParams fin = base_params(ctx);
  fin.mode = MODE_PARTIAL;
  if (!ctx->permuted) return evaluate(ctx, w, psi, fin, out);
  // qubit order in and out: psi -> scratch (library order) -> H psi into out -> qubit order
  int rc = to_library_order(ctx, ctx->vec[V_ACC], psi);
  if (!rc) rc = evaluate(ctx, w, ctx->vec[V_ACC], fin, out);
  if (!rc) rc = to_qubit_order(ctx, ctx->vec[V_ACC], out);
  if (rc) return rc;
  CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->vec[V_ACC], (size_t)ctx->N * ctx->amp, cudaMemcpyDeviceToDevice,
                                ctx->stream));
  return AQC_OK;
}


size_t aqc_batch_workspace_bytes(int max_members, int64_t max_items) {
  if (max_members < 1 || max_members > 65536 || max_items < 1 || max_items > ((int64_t)1 << 28)) return 0;
  return plan_batch(max_members, max_items).total;
}

int aqc_batch_create(aqc_batch** out, int device, int precision, int max_members, int64_t max_items, void* workspace,
                     size_t workspace_bytes, void* cuda_stream) {
  if (!out) return AQC_E_INVAL;
  *out = nullptr;
  if (precision != AQC_C128 && precision != AQC_C64) {
    g_create_error = "precision must be AQC_C128 or AQC_C64";
    return AQC_E_INVAL;
  }
  const size_t need = aqc_batch_workspace_bytes(max_members, max_items);
  if (need == 0) {
    g_create_error = "max_members must be in [1, 65536] and max_items in [1, 2^28]";
    return AQC_E_INVAL;
  }
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255u)) {
    g_create_error = "batch workspace missing, unaligned or smaller than aqc_batch_workspace_bytes()";
    return AQC_E_NOMEM;
  }
  aqc_batch* b = new (std::nothrow) aqc_batch();
  if (!b) return AQC_E_NOMEM;
  b->device = device;
  b->prec = precision;
  b->max_members = max_members;
  b->max_items = max_items;
  b->ws = (char*)workspace;
  const BatchPlan bp = plan_batch(max_members, max_items);
  b->d_insts = (BatchInst*)(b->ws + bp.off_insts);
  for (int l = 0; l < kMaxLayouts; l++)
    b->d_items[l] = (BatchItem*)(b->ws + bp.off_items + (size_t)l * (size_t)max_items * sizeof(BatchItem));
  b->d_partials = (double*)(b->ws + bp.off_partials);
  b->members.assign(max_members, nullptr);
  b->step_at_add.assign(max_members, 0);
  b->h_insts.assign(max_members, BatchInst());
  memset(b->h_insts.data(), 0, sizeof(BatchInst) * max_members);
  DeviceGuard dg(device);
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      g_create_error = "cudaStreamCreateWithFlags failed";
      return AQC_E_CUDA;
    }
    b->own_stream = true;
  }
  if (cudaMemsetAsync(b->d_insts, 0, sizeof(BatchInst) * max_members, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess) {
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    g_create_error = "cudaMemsetAsync on the batch workspace failed";
    return AQC_E_CUDA;
  }
  *out = b;
  return AQC_OK;
}

void aqc_batch_destroy(aqc_batch* b) {
  if (!b) return;
  DeviceGuard dg(b->device);
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

int aqc_batch_set_shape(aqc_batch* b, int threads, int steps_per_round) {
  if (!b) return AQC_E_INVAL;
  if (threads != 128 && threads != 256) BFAIL(b, AQC_E_INVAL, "threads must be 128 or 256");
  if (steps_per_round < 1 || steps_per_round > 4096) BFAIL(b, AQC_E_INVAL, "steps_per_round must be in [1, 4096]");
  b->threads = threads;
  b->steps_per_round = steps_per_round;
  b->dirty = true;
  return AQC_OK;
}

int aqc_batch_add(aqc_batch* b, aqc_ctx* c, int* slot_out) {
  if (!b || !c) return AQC_E_INVAL;
  if (c->device != b->device || c->prec != b->prec) BFAIL(b, AQC_E_INVAL, "context device/precision differ from the batch");
  if (!c->have_state) BFAIL(b, AQC_E_STATE, "context has no initial state");
  for (const ClauseH& k : c->clauses)
    if (k.stepwise) BFAIL(b, AQC_E_UNSUPPORTED, "clause-by-clause sequences are not batched");
  if (c->adaptive) BFAIL(b, AQC_E_UNSUPPORTED, "contexts under step-size control are not batched");
  if (c->ycomp) BFAIL(b, AQC_E_UNSUPPORTED, "contexts under y compensation are not batched");
  for (aqc_ctx* m : b->members)
    if (m == c) BFAIL(b, AQC_E_INVAL, "context is already a member");
  int slot = -1;
  for (int i = 0; i < b->max_members; i++)
    if (!b->members[i]) {
      slot = i;
      break;
    }
  if (slot < 0) BFAIL(b, AQC_E_NOMEM, "batch is full (%d members)", b->max_members);
  DeviceGuard dg(b->device);
  if (!c->in_batch) {
    c->in_batch = true;  // per-CTA tiles for the batched kernel
    c->dirty = true;
  }
  int rc = ensure_ready(c);
  if (rc) {
    c->in_batch = false;
    c->dirty = true;
    BFAIL(b, rc, "member: %s", c->err.c_str());
  }
  rc = plan_first_segment(c);
  if (rc) {
    c->in_batch = false;
    c->dirty = true;
    BFAIL(b, rc, "member: %s", c->err.c_str());
  }
  // start-up on the batch stream: RK4 steps, f_3 and the first predictor (after the
  // context's own queued work, e.g. its initial state)
  BCUDA(b, cudaStreamSynchronize(c->stream));
  cudaStream_t saved = c->stream;
  c->stream = b->stream;
  while (rc == 0 && c->step < 3 && c->step < c->nsteps) {
    rc = rk4_step(c);
    if (!rc) count_step(c);
  }
  if (rc == 0 && c->step >= 3 && c->step < c->nsteps && !c->hist_ready) rc = start_history(c);
  c->stream = saved;
  if (rc) BFAIL(b, rc, "member start-up: %s", c->err.c_str());
  rc = batch_pull(b);
  if (rc) return rc;
  fill_inst(c, &b->h_insts[slot]);
  BCUDA(b, cudaMemcpyAsync(b->d_insts + slot, &b->h_insts[slot], sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  b->members[slot] = c;
  b->step_at_add[slot] = c->step;
  b->dirty = true;
  if (slot_out) *slot_out = slot;
  return AQC_OK;
}

int aqc_batch_remove(aqc_batch* b, int slot) {
  if (!b) return AQC_E_INVAL;
  if (slot < 0 || slot >= b->max_members || !b->members[slot]) BFAIL(b, AQC_E_INVAL, "no member in slot %d", slot);
  DeviceGuard dg(b->device);
  int rc = batch_pull(b);
  if (rc) return rc;
  aqc_ctx* c = b->members[slot];
  const BatchInst& I = b->h_insts[slot];
  c->evals += I.step - b->step_at_add[slot];
  c->step = I.step;
  c->steps_done = I.step;  // one segment from t = 0 (batch members run the fixed-step grid)
  if (!c->segs.empty()) c->segs.back().steps = I.step;
  if (c->step >= c->seg_m) {
    c->at_end = true;
    if (!c->segs.empty()) c->segs.back().end = AQC_SEG_AT_T;
  }
  if (c->step >= 3) c->hist_ready = true;
  // carry the member's reductions into the context's result slots
  double sl[3] = {I.norm2, I.max_err, I.last_err};
  if (I.step > b->step_at_add[slot]) {
    cudaMemcpyAsync(c->d_slots + kSlotNorm2, &sl[0], sizeof(double), cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(c->d_slots + kSlotMaxErr, &sl[1], sizeof(double), cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(c->d_slots + kSlotLastErr, &sl[2], sizeof(double), cudaMemcpyHostToDevice, b->stream);
    BCUDA(b, cudaStreamSynchronize(b->stream));
  }
  b->members[slot] = nullptr;
  c->in_batch = false;
  c->dirty = true;
  memset(&b->h_insts[slot], 0, sizeof(BatchInst));
  BCUDA(b, cudaMemcpyAsync(b->d_insts + slot, &b->h_insts[slot], sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  b->dirty = true;
  return AQC_OK;
}

int aqc_batch_run(aqc_batch* b, int64_t rounds) {
  if (!b) return AQC_E_INVAL;
  if (rounds < 0) BFAIL(b, AQC_E_INVAL, "rounds must be >= 0");
  DeviceGuard dg(b->device);
  if (b->dirty) {
    int rc = batch_rebuild(b);
    if (rc) return rc;
  }
  if (!b->gexec) return AQC_OK;
  int per = 0;
  for (int l = 0; l < b->nlevels; l++) per += b->nitems[l] > 0 ? 1 : 0;
  for (int64_t r = 0; r < rounds; r++) {
    BCUDA(b, cudaGraphLaunch(b->gexec, b->stream));
    b->launches += (int64_t)per * b->steps_per_round;
  }
  return AQC_OK;
}

int aqc_batch_poll(aqc_batch* b, int64_t* steps_done, int* active_out, int64_t* launches_out) {
  if (!b) return AQC_E_INVAL;
  DeviceGuard dg(b->device);
  int rc = batch_pull(b);
  if (rc) return rc;
  int active = 0;
  for (int i = 0; i < b->max_members; i++) {
    const aqc_ctx* c = b->members[i];
    if (steps_done) steps_done[i] = c ? b->h_insts[i].step : -1;
    if (c && b->h_insts[i].step < b->h_insts[i].nsteps) active++;
  }
  if (active_out) *active_out = active;
  if (launches_out) *launches_out = b->launches;
  return AQC_OK;
}

const char* aqc_batch_last_error(const aqc_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

int aqc_launch_count(const aqc_ctx* ctx, int64_t* out) {
  if (!ctx || !out) return AQC_E_INVAL;
  *out = ctx->launches;
  return AQC_OK;
}

const char* aqc_last_error(const aqc_ctx* ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

const char* aqc_version(void) { return "aqc-gb300 0.1.0 (sm_103a)"; }



size_t aqc_lanczos_workspace_bytes(int n_qubits, int precision, int max_iter) {
  if (n_qubits < 1 || n_qubits > kMaxN || (precision != AQC_C128 && precision != AQC_C64) || max_iter < 1 ||
      max_iter > 4096)
    return 0;
  return lanczos_plan(n_qubits, precision, max_iter).total;
}

int aqc_tridiag_eigvec(int k, const double* a, const double* b, double lam, double* out) {
  if (k < 1 || !a || (k > 1 && !b) || !out || !std::isfinite(lam)) return AQC_E_INVAL;
  tridiag_eigvec(a, b, k, lam, out);
  return AQC_OK;
}

int aqc_tridiag_eigvals(int k, const double* a, const double* b, int n_eig, double* out) {
  if (k < 1 || !a || (k > 1 && !b) || n_eig < 1 || n_eig > k || !out) return AQC_E_INVAL;
  for (int j = 0; j < n_eig; j++) out[j] = tridiag_eig(a, b, k, j);
  return AQC_OK;
}

int aqc_lanczos(aqc_ctx* ctx, double t, const void* start, void* work, size_t work_bytes, int max_iter, int n_eig,
                double tol, double* eig, double* conv, int* iters_out) {
  if (!ctx) return AQC_E_INVAL;
  if (!start || !work || !eig) FAIL(ctx, AQC_E_INVAL, "start, work and eig must be non-NULL");
  if (max_iter < 1 || max_iter > 4096 || n_eig < 1 || n_eig > max_iter || !(tol >= 0.0))
    FAIL(ctx, AQC_E_INVAL, "need 1 <= n_eig <= max_iter <= 4096 and tol >= 0");
  const LzPlan P = lanczos_plan(ctx->n, ctx->prec, max_iter);
  if (work_bytes < P.total) FAIL(ctx, AQC_E_NOMEM, "work has %zu bytes, %zu needed", work_bytes, P.total);
  if (((uintptr_t)work & 255u) || ((uintptr_t)start & 15u)) FAIL(ctx, AQC_E_INVAL, "work must be 256-byte aligned");
  if (!ctx->have_sched) FAIL(ctx, AQC_E_STATE, "no schedule set");
  DeviceGuard dg(ctx->device);
  if (ctx->dirty) {
    int rc = build_tables(ctx);
    if (rc) return rc;
  }
  double w[3];
  sched_weights(ctx, t, w);
  char* base = (char*)work;
  const uint64_t ld = P.ld_bytes / ctx->amp;  // elements between basis vectors
  auto V = [&](int i) { return (void*)(base + (size_t)i * P.ld_bytes); };
  double* partials = (double*)(base + P.off_partials);
  double* coef = (double*)(base + P.off_coef);
  double* h = (double*)(base + P.off_h);
  double* scal = (double*)(base + P.off_scal);
  cudaStream_t s = ctx->stream;
  const uint64_t N = ctx->N;
  // v_0 = start / ||start||
  if (ctx->permuted) {
    int rc = to_library_order(ctx, V(0), start);
    if (rc) return rc;
  } else {
    CUDA_TRY(ctx, cudaMemcpyAsync(V(0), start, N * ctx->amp, cudaMemcpyDeviceToDevice, s));
  }
  CUDA_TRY(ctx, launch_dotc_multi(ctx->prec, V(0), ld, 1, V(0), N, partials, scal, nullptr, s));
  CUDA_TRY(ctx, launch_scale_to(ctx->prec, V(0), V(0), N, scal, s));
  ctx->launches += 3;
  std::vector<double> alpha, beta, prev(n_eig, 0.0), cur(n_eig, 0.0), chg(n_eig, INFINITY);
  int iters = 0;
  bool have_prev = false;
  for (int j = 0; j < max_iter; j++) {
    void* wv = V(j + 1);
    ApplyParams fin = base_params(ctx);
    fin.mode = MODE_PARTIAL;
    int rc = evaluate(ctx, w, V(j), fin, wv);
    if (rc) return rc;
    CUDA_TRY(ctx, cudaMemsetAsync(h, 0, (size_t)(j + 1) * 2 * sizeof(double), s));
    for (int pass = 0; pass < 2; pass++) {  // classical Gram-Schmidt, twice
      CUDA_TRY(ctx, launch_dotc_multi(ctx->prec, V(0), ld, (uint32_t)(j + 1), wv, N, partials, coef, h, s));
      CUDA_TRY(ctx, launch_sub_multi(ctx->prec, wv, V(0), ld, (uint32_t)(j + 1), coef, N, s));
      ctx->launches += 3;
    }
    CUDA_TRY(ctx, launch_dotc_multi(ctx->prec, wv, ld, 1, wv, N, partials, scal, nullptr, s));
    ctx->launches += 2;
    double hj[2], nrm2[2];
    CUDA_TRY(ctx, cudaMemcpyAsync(hj, h + 2 * j, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(ctx, cudaMemcpyAsync(nrm2, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (!std::isfinite(hj[0]) || !std::isfinite(nrm2[0])) FAIL(ctx, AQC_E_NUMERIC, "non-finite Lanczos coefficient");
    alpha.push_back(hj[0]);
    const double bj = sqrt(std::max(nrm2[0], 0.0));
    iters = j + 1;
    const bool invariant = bj <= 1e-13 * std::max(1.0, fabs(hj[0]));
    const int m = std::min(n_eig, iters);
    const bool check = invariant || iters == max_iter || iters % 8 == 0;
    if (check && iters >= n_eig) {
      for (int e = 0; e < m; e++) cur[e] = tridiag_eig(alpha.data(), beta.data(), iters, e);
      bool done = have_prev;
      for (int e = 0; e < m; e++) {
        chg[e] = have_prev ? fabs(cur[e] - prev[e]) : INFINITY;
        done = done && chg[e] <= tol * std::max(1.0, fabs(cur[e]));
      }
      prev = cur;
      have_prev = true;
      if (done || invariant) break;
    }
    if (invariant) break;
    beta.push_back(bj);
    CUDA_TRY(ctx, launch_scale_to(ctx->prec, wv, wv, N, scal, s));
    ctx->launches++;
  }
  CUDA_TRY(ctx, cudaStreamSynchronize(s));  // the caller's work buffer is free on return
  const int m = std::min(n_eig, iters);
  for (int e = 0; e < n_eig; e++) {
    eig[e] = e < m ? tridiag_eig(alpha.data(), beta.data(), iters, e) : NAN;
    if (conv) conv[e] = e < m ? chg[e] : NAN;
  }
  if (iters_out) *iters_out = iters;
  return AQC_OK;
}

int aqc_lanczos_ground(aqc_ctx* ctx, double t, const void* start, void* work, size_t work_bytes, int max_iter,
                       double tol, double* theta_out, double* resid_out, void* ground_out, int* iters_out) {
  if (!ctx) return AQC_E_INVAL;
  if (!start || !work || !theta_out || !ground_out) FAIL(ctx, AQC_E_INVAL, "start, work, theta and ground_out must be non-NULL");
  if (max_iter < 1 || max_iter > 4096 || !(tol >= 0.0)) FAIL(ctx, AQC_E_INVAL, "need 1 <= max_iter <= 4096 and tol >= 0");
  const LzPlan P = lanczos_plan(ctx->n, ctx->prec, max_iter);
  if (work_bytes < P.total) FAIL(ctx, AQC_E_NOMEM, "work has %zu bytes, %zu needed", work_bytes, P.total);
  if (((uintptr_t)work & 255u) || ((uintptr_t)start & 15u) || ((uintptr_t)ground_out & 15u))
    FAIL(ctx, AQC_E_INVAL, "work must be 256-byte aligned, start and ground_out 16-byte aligned");
  if (!ctx->have_sched) FAIL(ctx, AQC_E_STATE, "no schedule set");
  DeviceGuard dg(ctx->device);
  if (ctx->dirty) {
    int rc = build_tables(ctx);
    if (rc) return rc;
  }
  double w[3];
  sched_weights(ctx, t, w);
  char* base = (char*)work;
  const uint64_t ld = P.ld_bytes / ctx->amp;
  auto V = [&](int i) { return (void*)(base + (size_t)i * P.ld_bytes); };
  double* partials = (double*)(base + P.off_partials);
  double* coef = (double*)(base + P.off_coef);
  double* h = (double*)(base + P.off_h);
  double* scal = (double*)(base + P.off_scal);
  cudaStream_t s = ctx->stream;
  const uint64_t N = ctx->N;
  const size_t bytes = (size_t)N * ctx->amp;
  if (ctx->permuted) {
    int rc = to_library_order(ctx, V(0), start);
    if (rc) return rc;
  } else {
    CUDA_TRY(ctx, cudaMemcpyAsync(V(0), start, bytes, cudaMemcpyDeviceToDevice, s));
  }
  CUDA_TRY(ctx, launch_dotc_multi(ctx->prec, V(0), ld, 1, V(0), N, partials, scal, nullptr, s));
  CUDA_TRY(ctx, launch_scale_to(ctx->prec, V(0), V(0), N, scal, s));
  ctx->launches += 3;
  std::vector<double> alpha, beta, sv;
  int iters = 0;
  double theta = 0.0;
  for (int j = 0; j < max_iter; j++) {
    void* wv = V(j + 1);
    ApplyParams fin = base_params(ctx);
    fin.mode = MODE_PARTIAL;
    int rc = evaluate(ctx, w, V(j), fin, wv);
    if (rc) return rc;
    CUDA_TRY(ctx, cudaMemsetAsync(h, 0, (size_t)(j + 1) * 2 * sizeof(double), s));
    for (int pass = 0; pass < 2; pass++) {  // classical Gram-Schmidt, twice
      CUDA_TRY(ctx, launch_dotc_multi(ctx->prec, V(0), ld, (uint32_t)(j + 1), wv, N, partials, coef, h, s));
      CUDA_TRY(ctx, launch_sub_multi(ctx->prec, wv, V(0), ld, (uint32_t)(j + 1), coef, N, s));
      ctx->launches += 3;
    }
    CUDA_TRY(ctx, launch_dotc_multi(ctx->prec, wv, ld, 1, wv, N, partials, scal, nullptr, s));
    ctx->launches += 2;
    double hj[2], nrm2[2];
    CUDA_TRY(ctx, cudaMemcpyAsync(hj, h + 2 * j, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(ctx, cudaMemcpyAsync(nrm2, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (!std::isfinite(hj[0]) || !std::isfinite(nrm2[0])) FAIL(ctx, AQC_E_NUMERIC, "non-finite Lanczos coefficient");
    alpha.push_back(hj[0]);
    const double bj = sqrt(std::max(nrm2[0], 0.0));
    iters = j + 1;
    const bool invariant = bj <= 1e-13 * std::max(1.0, fabs(hj[0]));
    if (invariant || iters == max_iter || iters % 4 == 0) {
      // Ritz residual of the lowest pair: ||H x - theta x|| = beta_j |s_last|
      theta = tridiag_eig(alpha.data(), beta.data(), iters, 0);
      sv.assign(iters, 0.0);
      tridiag_eigvec(alpha.data(), beta.data(), iters, theta, sv.data());
      if (invariant || bj * fabs(sv[iters - 1]) <= tol * std::max(1.0, fabs(theta)) || iters == max_iter) break;
    }
    beta.push_back(bj);
    CUDA_TRY(ctx, launch_scale_to(ctx->prec, wv, wv, N, scal, s));
    ctx->launches++;
  }
  // x = sum_i s_i v_i into V(iters) (free: the last, unnormalised residual), then unit norm
  void* x = V(iters);
  std::vector<double> c(2 * (size_t)iters, 0.0);
  for (int i = 0; i < iters; i++) c[2 * (size_t)i] = -sv[i];
  CUDA_TRY(ctx, cudaMemcpyAsync(coef, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  CUDA_TRY(ctx, cudaMemsetAsync(x, 0, bytes, s));
  CUDA_TRY(ctx, launch_sub_multi(ctx->prec, x, V(0), ld, (uint32_t)iters, coef, N, s));
  CUDA_TRY(ctx, launch_dotc_multi(ctx->prec, x, ld, 1, x, N, partials, scal, nullptr, s));
  CUDA_TRY(ctx, launch_scale_to(ctx->prec, x, x, N, scal, s));
  ctx->launches += 4;
  // residual ||H x - theta x|| with one more matvec (into the scratch vector)
  {
    ApplyParams fin = base_params(ctx);
    fin.mode = MODE_PARTIAL;
    int rc = evaluate(ctx, w, x, fin, ctx->vec[V_ACC]);
    if (rc) return rc;
    const double th[2] = {theta, 0.0};
    CUDA_TRY(ctx, cudaMemcpyAsync(coef, th, sizeof(th), cudaMemcpyHostToDevice, s));
    CUDA_TRY(ctx, launch_sub_multi(ctx->prec, ctx->vec[V_ACC], x, ld, 1, coef, N, s));
    CUDA_TRY(ctx, launch_dotc_multi(ctx->prec, ctx->vec[V_ACC], ld, 1, ctx->vec[V_ACC], N, partials, scal, nullptr, s));
    ctx->launches += 3;
    double r2[2];
    CUDA_TRY(ctx, cudaMemcpyAsync(r2, scal, sizeof(r2), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (resid_out) *resid_out = sqrt(std::max(r2[0], 0.0));
  }
  if (ctx->permuted) {
    int rc = to_qubit_order(ctx, ground_out, x);
    if (rc) return rc;
  } else {
    CUDA_TRY(ctx, cudaMemcpyAsync(ground_out, x, bytes, cudaMemcpyDeviceToDevice, s));
  }
  CUDA_TRY(ctx, cudaStreamSynchronize(s));
  *theta_out = theta;
  if (iters_out) *iters_out = iters;
  return AQC_OK;
}

}  // extern "C"
