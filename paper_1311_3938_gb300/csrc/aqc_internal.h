// Internal declarations shared by the host driver (api.cu) and the kernels (kernels.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace aqc {

constexpr int kMaxFlips = 2048;   // off-diagonal Pauli products over all layouts
constexpr int kMaxZ = 1024;       // diagonal Pauli products (Z strings)
constexpr int kMaxClauses = 1024; // EC3 clauses
constexpr int kMaxClasses = 8;    // (group, penalty kind, scale) classes of clauses
constexpr int kMaxLayouts = 8;
constexpr int kMaxN = 31;
constexpr int kMaxApplyGrid = 4096;  // persistent k_apply grids never exceed this many CTAs

// One off-diagonal Pauli product in gather form: (P psi)(z) = i^ipow (-1)^{|zm & (z^x)|} psi(z^x),
// optionally with a companion product of the same flip mask x (zm2, ipow2, group2, coef2) that
// shares the gather: X_iX_j + Y_iY_j of Eq. Hixy is one entry whose coefficient is exactly
// 2c or 0 per source index, so Hamming-weight sectors stay exactly separate.
struct DevFlip {
  uint32_t x;      // global flip mask
  uint32_t lx;     // the same mask in tile-local bits of its layout (0 for remote terms)
  uint32_t zm;     // Z/Y positions (sign from the source index z^x)
  uint32_t zm2;    // companion's Z/Y positions
  int32_t group;   // weight slot A/B/C
  int32_t ipow;    // |x & zm| mod 4 (Y = i X Z)
  int32_t group2, ipow2;
  int32_t has2;    // a companion product is present
  int32_t pad;
  double coef;
  double coef2;
};

struct DevZ {      // diagonal product coef (-1)^{|zm & z|}
  uint32_t zm;
  int32_t group;
  double coef;
};

struct DevClass {  // clauses [begin, end) share group, penalty and scale
  int32_t group;
  int32_t pen;     // 0 indicator [k != 1], 1 squared (1-k)^2
  int32_t begin, end;
  int32_t stepwise;  // the clause-by-clause sequence h_1..h_m (Eq. kpath), in order
  int32_t derived;   // 1: the clauses are those of the byte-table class minus clause_mask[dbegin, dend)
  int32_t dbegin, dend;
  double scale;
};
constexpr int kMaxDerivedDiff = 8;  // clauses a derived class may lack

// Tile layout: tile bits are [0, c) and [h, h + w); t = c + w; remaining bits index tiles.
// cb > 0: the tile belongs to a cluster of 2^cb CTAs; the top cb tile bits select the CTA, each
// CTA holds 2^(t - cb) indices in its shared memory, and the others read it through
// distributed shared memory.
struct Layout {
  int c, h, w, t;
  int cb;
};
constexpr int kClusterBits = 3;  // 8 CTAs per cluster

// First index of tile b: b's low h-c bits go to index bits [c, h), the rest above h+w.
__host__ __device__ __forceinline__ uint32_t tile_base(const Layout& L, uint32_t b) {
  const uint32_t gap = (uint32_t)(L.h - L.c);
  const uint32_t lowpart = b & ((1u << gap) - 1u);
  const uint32_t hipart = gap >= 32 ? 0u : (b >> gap);
  return (lowpart << L.c) | (hipart << (L.h + L.w));
}

// Index of tile position j (tile bits: [0,c) then [h,h+w)) in the tile starting at zb.
__host__ __device__ __forceinline__ uint32_t tile_z(const Layout& L, uint32_t j, uint32_t zb) {
  const uint32_t cm = (1u << L.c) - 1u;
  return zb | (j & cm) | ((j >> L.c) << L.h);
}

struct DevTables {
  int n_layouts;
  int n_remote;                     // flips no layout holds, gathered from global memory
  int flip_begin[kMaxLayouts + 2];  // layout l: [flip_begin[l], flip_begin[l+1]); remote after
  int plain_count[kMaxLayouts + 2]; // leading X-string products (zm = 0, real) of each range
  int plain_fast[kMaxLayouts + 2];  // of those, the leading ones that flip no register-held tile bit
  int hop_count[kMaxLayouts + 2];   // leading entries of the general range that are hops:
                                    // X_iX_j + Y_iY_j with one real coefficient c, i.e.
                                    // 2c psi(z ^ x) where bits i, j of z differ, else 0
  int hop_class_end[kMaxLayouts + 2][3];  // hops sorted by the register-held tile bits they
                                    // flip (class 0: neither, 1: the pair bit, 2: the half
                                    // bit, 3: both); ends of classes 0..2 within the hops'
                                    // range, class 3 ends at hop_count
  int n_z;
  int n_classes;
  int table_class;                  // clause class whose counts are in the per-index byte table, or -1
  int pad;
  double ident[3];                  // identity prefactors per group (energy shifts m^(0))
  DevClass classes[kMaxClasses];
  uint32_t clause_mask[kMaxClauses];
  DevZ z[kMaxZ];
  DevFlip flips[kMaxFlips];
};

enum Mode : int {
  MODE_PARTIAL = 0,  // qout = qin + [diag + remote] + local flips
  MODE_STEP = 1,     // f_{n+1} = -i(...); PEC corrector + next predictor + reductions
  MODE_RK4 = 2,      // RK4 stage (stage 1..4)
  MODE_DERIV = 3,    // fout = -i(...)
  MODE_ENERGY = 4,   // reduce Re <src| (...) >
};

struct ApplyParams {
  const DevTables* tab;
  int n;
  uint32_t ntiles;   // 2^(n - L.t); CTAs loop over tiles blockIdx.x, blockIdx.x + gridDim.x, ...
  Layout L;
  int layout_index;
  int with_diag;
  int with_remote;
  int mode;
  int stage;         // RK4 stage 1..4
  double w[3];       // group weights A, B, C at the evaluation time
  const double* wdev; // nullable: read the weights from this device array instead of w (steps
                      // replayed from a CUDA graph, whose weights the host writes before a replay)
  int max_grid;       // > 0: at most this many CTAs (the kernels are persistent over tiles)
  int turn;           // STEP: also apply this layout's products, at the weights w2 (wdev[3..5]
                      // when wdev is set), to the new predictor p_{n+2}; the sum goes to qout
  double w2[3];
  double h;
  const uint8_t* dcode; // per-index clause counts of class table_class (nullable)
  const void* src;   // vector the Hamiltonian acts on
  const void* qin;   // partial sum from earlier layouts (nullable)
  void* qout;        // PARTIAL: output partial sum
  void* y;           // STEP: y_n -> y_{n+1};  RK4: y (stage 4 writes y)
  void* yout;        // STEP: where y_{n+1} goes (nullptr: in place over y, the fixed-step grid;
                     // a second vector under step-size control, so a rejected step keeps y_n)
  const void* f0;    // STEP: f_n
  const void* f1;    // STEP: f_{n-1}
  const void* f2;    // STEP: f_{n-2}
  void* fout;        // STEP: f_{n+1};  DERIV: f;  RK4 stage 1: history f_n
  void* pout;        // STEP: p_{n+2};  RK4: stage input for the next stage (ys)
  void* acc;         // RK4 accumulator
  void* ylo;         // STEP, complex64: low part of y (compensated corrector; nullable)
  int step_k;        // clause-by-clause segment k (0: no clause of the sequence active)
  double step_wdone; // coefficient of clauses j < k of the sequence
  double step_wact;  // coefficient of clause k
  double* partials;  // per-CTA reduction partials (3 doubles per CTA)
  unsigned* counter; // last-CTA ticket (reset to 0 by the last CTA)
  double* slots;     // results: see kSlot*
};

// One PEC step's last two layout passes over slabs of the index space (kernel k_slab).  A slab
// fixes the bits of slab_mask, bits that neither layout holds, so each slab is a union of
// whole tiles of both layouts.  Work items run in the order P(0..D-1), then P(D+v), S(v) for
// v = 0.., then the last S: P(s) = every tile of slab s of the partial layout (partial sum into
// q), S(s) = every tile of slab s of layout 0 (the fused step); S(s) waits for P(s).  The q and
// p of a slab are read again by S(s) shortly after P(s) wrote or read them, while they are still
// in L2, so a step moves two vectors less from HBM than separate layout passes.
struct SlabParams {
  ApplyParams part;     // MODE_PARTIAL on the slab layout (src = p, qin = qout = q)
  ApplyParams step;     // MODE_STEP on layout 0
  uint32_t slab_mask;   // index bits fixed by a slab
  uint32_t free_part;   // bits that number the partial layout's tiles within a slab
  uint32_t free_step;   // the same for layout 0
  uint32_t n_slabs;     // 2^popcount(slab_mask)
  uint32_t tiles;       // tiles per slab (both layouts)
  uint32_t lookahead;   // D, 1 <= D <= n_slabs
  uint32_t n_items;     // 2 * n_slabs * tiles
  uint32_t spin_limit;  // polls before a wait gives up (sets slots[kSlotFault])
  unsigned* queue;      // next work item (reset to 0 by the last CTA)
  unsigned* done;       // finished partial tiles per slab (reset to 0 by the last CTA)
};
constexpr int kMaxSlabs = 2048;

// Partial-sum pass of a strided layout holding only X strings with real coefficients
// (complex64, kernel k_partial_x): the source tile arrives by TMA through `tmap`.
constexpr int kXTileBits = 13;
struct XPartialParams {
  CUtensorMap tmap;      // source as a 4-D float tensor (chunk, gap bits, tile rows, top bits),
                         // 5-D when the chunk exceeds one box row (chunk split in two dims)
  int tma_rank;          // 4 or 5
  const DevTables* tab;
  Layout L;
  int layout_index;
  double w[3];
  const double* wdev;    // nullable: weights from device memory (as ApplyParams::wdev)
  int max_grid;          // > 0: at most this many CTAs
  const void* qin;       // nullable
  void* qout;
  uint32_t ntiles;
  double* slots;         // kSlotFault is set if a tile copy never completes
};

// vectors of a state (workspace order)
constexpr int kVecY = 0, kVecP = 1, kVecQ = 2, kVecF0 = 3, kVecAcc = 7, kVecCount = 8;

// One member of a batch: everything its PEC steps need, read by the batched kernel on the device.
struct BatchInst {
  const DevTables* tab;
  const uint8_t* dcode;  // nullable
  void* vec[kVecCount];
  Layout layouts[kMaxLayouts];
  int nl;
  int s_kind;
  double T, h;
  double poly[3][4];
  int64_t step;    // next PEC step n (computes f_{n+1}); advanced by the member's last CTA
  int64_t nsteps;
  uint32_t item_begin, item_end;  // the member's items in the level-0 work list
  unsigned ticket;
  int pad;
  double norm2, max_err, last_err;
};

struct BatchItem {
  uint32_t inst;
  uint32_t tile;
};

struct BatchLaunch {
  const BatchItem* items;
  BatchInst* insts;
  double* partials;  // two doubles per level-0 item
  int level;
};

// Which layout pass of an evaluation adds the diagonal: layout 0, the last pass (the fused step
// kernel in a propagation, memory-bound with issue slots to spare; its clause bytes are staged
// in shared memory with the tile).  The first pass (the highest layout) adds the products no
// layout holds.
__host__ __device__ inline int diag_level(int n_layouts) {
  (void)n_layouts;
  return 0;
}

// Tile bits a thread holds in registers (see process_tile): bit 0 and bit 6 for complex64 (two
// halves of two amplitudes, 64 indices apart), bit 5 for complex128 (two single amplitudes).
constexpr uint32_t kRegBitsC64 = 0x41u;
constexpr uint32_t kRegBitsC128 = 0x20u;

// result slots (doubles) in the workspace
constexpr int kSlotNorm2 = 0;
constexpr int kSlotMaxErr = 1;
constexpr int kSlotLastErr = 2;
constexpr int kSlotDot = 3;
constexpr int kSlotDotIm = 4;
constexpr int kSlotFault = 5;  // nonzero: an inter-CTA wait gave up (results of that step are invalid)
constexpr int kSlotCount = 8;

// PEC steps per CUDA-graph replay of a lone context: at most this many; the weights of each
// replayed step come from a device array of kGraphStepWeights doubles per step
// (ApplyParams::wdev: the weights at t_{n+1}, then at t_{n+2} for the turn of layouts)
constexpr int kMaxGraphSteps = 64;
constexpr int kGraphStepWeights = 6;

cudaError_t launch_apply(int prec, const ApplyParams& p, int smem_bytes, cudaStream_t s);
int apply_grid(int prec, int mode, uint32_t ntiles, int smem_bytes);
size_t apply_smem_bytes(int prec, int t, int n_plain, int n_general, int n_z);
size_t table_smem_bytes(int prec, int t, int n_plain, int n_general, int n_z);
cudaError_t launch_slab(int prec, const SlabParams& p, int smem_bytes, cudaStream_t s);
bool xpartial_layout_ok(const Layout& L);
size_t xpartial_smem_bytes(int n_flips);
cudaError_t launch_partial_x(const XPartialParams& p, int smem_bytes, cudaStream_t s);
uint32_t lanczos_dot_blocks(uint64_t N);
cudaError_t launch_dotc_multi(int prec, const void* V, uint64_t ld, uint32_t m, const void* w, uint64_t N,
                              double* partials, double* out, double* acc, cudaStream_t s);
cudaError_t launch_sub_multi(int prec, void* w, const void* V, uint64_t ld, uint32_t m, const double* c, uint64_t N,
                             cudaStream_t s);
cudaError_t launch_scale_to(int prec, void* v, const void* w, uint64_t N, const double* nrm2, cudaStream_t s);
cudaError_t launch_diag_codes(uint8_t* out, uint64_t N, const DevTables* tab, int cls, cudaStream_t s);
cudaError_t launch_init(int prec, void* y, uint64_t N, int kind, uint64_t basis, double amp, cudaStream_t s);
cudaError_t launch_permute(int prec, void* dst, const void* src, uint64_t N, const uint32_t* tab, cudaStream_t s);
cudaError_t launch_predict(int prec, void* p, const void* y, const void* f3, const void* f2, const void* f1,
                           const void* f0, double h, uint64_t N, cudaStream_t s);
cudaError_t launch_reduce(int prec, int what, const void* a, uint64_t N, double* partials, unsigned* counter,
                          double* slots, int grid, cudaStream_t s);
cudaError_t launch_fidelity(int prec, const void* a, uint64_t w, double* slots, cudaStream_t s);
// dst[0 .. count) = w[0 .. count), count <= kGraphStepWeights kMaxGraphSteps, the values passed
// as kernel arguments (no host buffer outlives the call)
cudaError_t launch_set_weights(double* dst, const double* w, int count, cudaStream_t s);
// k_fma64: `blocks` CTAs of 256 threads, each thread `iters` rounds of independent FP64 FMAs;
// fma64_count gives the FMAs one launch performs
cudaError_t launch_fma64(int blocks, int iters, cudaStream_t s);
// k_wait_flag: one thread waits for *flag != 0 for at most `polls` polls (~1 us each); giving
// up sets slots[kSlotFault]
cudaError_t launch_wait_flag(const unsigned* flag, int64_t polls, double* slots, cudaStream_t s);
constexpr int kSlotWaitFlag = 6;  // a slot whose bits serve as the self-test's flag (never set)
int64_t fma64_count(int blocks, int iters);
int reduce_grid(uint64_t N);
cudaError_t launch_batch(int prec, int threads, const BatchLaunch& b, int nitems, int smem, cudaStream_t s);

}  // namespace aqc
