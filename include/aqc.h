/*
 * aqc.h -- C ABI of the GB300 adiabatic-evolution hot path (libaqc.so).
 *
 * The library integrates the time-dependent Schroedinger equation i d/dt psi = H(t) psi
 * (hbar = 1; Eq. schroedinger of arXiv:1311.3938) for a 2^n-amplitude state, where
 *     H(t) = A(s) H_A + B(s) H_B + C(s) H_C                     (Eq. aqc, Eq. nlpath)
 * and each group H_g is stored in the paper's Sparse Quantum Hamiltonian form
 * (Sec. I.A, Eq. SQH-Hamiltonian): a list of Pauli products with real prefactors, plus
 * Exact-Cover-3 clause penalties (Eq. hci, Eq. sat).  The integrator is a fourth-order
 * predictor-corrector with one H|psi> per step (Sec. I.B): Adams-Bashforth-4 predictor,
 * Adams-Moulton-4 corrector in PEC mode, fixed step h = T/N or step-size control on the
 * corrector's Milne estimate, started by three classical Runge-Kutta-4 steps.  All arithmetic
 * runs in CUDA kernels for sm_103a.
 *
 * Conventions (all entry points)
 *   - Return value: AQC_OK (0) or a negative AQC_E_* code; the context keeps a message
 *     readable with aqc_last_error().  Errors leave the context usable unless stated.
 *   - Basis index z: bit (q-1) of z is qubit q (Eq. ztensor and the formula after it).
 *   - State vectors: interleaved complex, (re, im) per amplitude, 2^n amplitudes; complex128
 *     (16 bytes/amplitude) for AQC_C128 or complex64 (8 bytes/amplitude) for AQC_C64.
 *   - Host arrays passed in are copied; the caller keeps ownership.
 *   - Device memory: the library allocates none.  The caller passes one device workspace
 *     of at least aqc_workspace_bytes() bytes at aqc_create(); it must stay valid until
 *     aqc_destroy().  All vectors, tables and reduction slots live in it.
 *   - Stream: all device work of a context is ordered on the stream given at creation (or
 *     aqc_set_stream()).  Functions that return host values synchronise that stream; the
 *     others only enqueue work.
 *   - Sizes: 1 <= n <= 31; masks must be < 2^n; clause bits distinct and < n.
 */
#ifndef AQC_H
#define AQC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- codes ------------------------------------------------------------------------- */
#define AQC_OK 0
#define AQC_E_INVAL (-1)        /* bad argument (size, mask, pointer, enum)              */
#define AQC_E_NOMEM (-2)        /* workspace too small / host allocation failed           */
#define AQC_E_CUDA (-3)         /* a CUDA runtime call failed (message has the CUDA text) */
#define AQC_E_NUMERIC (-4)      /* non-finite value detected in a reduction               */
#define AQC_E_STATE (-5)        /* call out of order (e.g. propagate before a schedule)   */
#define AQC_E_UNSUPPORTED (-6)  /* a term no layout can hold, or a size beyond the limits */
#define AQC_E_TIMEOUT (-7)      /* a bounded wait inside a kernel gave up (a tile copy that
                                   never landed, a partial sum that never came): that call's
                                   results are invalid; the context stays usable            */

#define AQC_C128 0 /* complex128 state, FP64 arithmetic                                   */
#define AQC_C64 1  /* complex64 state, FP32 arithmetic, FP64 reductions                   */

#define AQC_GRP_A 0 /* weight A(s), e.g. the initial Hamiltonian H_i                     */
#define AQC_GRP_B 1 /* weight B(s), e.g. the final Hamiltonian H_f                       */
#define AQC_GRP_C 2 /* weight C(s), e.g. a third path Hamiltonian                        */

#define AQC_PEN_INDICATOR 0 /* penalty [k != 1], k = number of 1-bits of the clause      */
#define AQC_PEN_SQUARED 1   /* penalty (1 - k)^2 (Eq. hci)                               */

#define AQC_S_LINEAR 0     /* s = t/T (Eq. aqc)                                          */
#define AQC_S_SMOOTHSTEP 1 /* s = 3 tau^2 - 2 tau^3, tau = t/T                           */

#define AQC_INIT_UNIFORM 0     /* |S> = 2^{-n/2} sum_z |z> (Sec. II.A.1)                  */
#define AQC_INIT_BASIS 1       /* |basis>                                                 */
#define AQC_INIT_USER_HOST 2   /* copy of a host vector (state precision, interleaved)   */
#define AQC_INIT_USER_DEVICE 3 /* copy of a device vector (state precision, interleaved) */
#define AQC_INIT_DICKE 4       /* C(n,k)^{-1/2} sum_{|u|=k} |u>, k = `basis` (Eq. initstate)  */
#define AQC_INIT_STAGED 5      /* the vector of the last aqc_stage_initial_state              */

typedef struct aqc_ctx aqc_ctx;

typedef struct {
  int64_t steps_done;  /* accepted grid steps since the initial state was set            */
  int64_t n_steps;     /* N of the grid h = T/N (step-size control: steps_done plus the
                          steps left in the current segment)                             */
  int64_t evaluations; /* H|psi> evaluations so far (rejected steps included)            */
  double t;            /* current time                                                   */
  double h;            /* current step size                                              */
  double norm2;        /* ||psi||^2 after the call (FP64 reduction)                      */
  double max_err_est;  /* max over accepted PEC steps of (19/270) ||y_{n+1} - p_{n+1}||  */
  double last_err_est; /* the same for the last PEC step                                 */
  double elapsed_ms;   /* device time of the call (CUDA events on the context stream)    */
  int64_t launches;    /* kernel launches this call issued                               */
  int64_t rejects;     /* PEC steps rejected by the step-size control since the initial state */
  int64_t segments;    /* segments of constant step begun since the initial state         */
} aqc_stats;

/* One segment of constant step size of a run (aqc_get_segments). */
#define AQC_SEG_RUNNING 0  /* the current segment                                           */
#define AQC_SEG_AT_T 1     /* its last step landed on T                                     */
#define AQC_SEG_REJECTED 2 /* a PEC step was rejected: the next segment starts there, h/2    */
#define AQC_SEG_GREW 3     /* small estimates: the next segment starts here with 2h          */
typedef struct {
  double t0;     /* start time                                                              */
  double h;      /* step size                                                               */
  int64_t steps; /* accepted grid steps                                                     */
  int32_t end;   /* AQC_SEG_*                                                               */
  int32_t pad;
} aqc_segment;

/* ---- lifetime ---------------------------------------------------------------------- */

/* Bytes of device workspace a context for (n_qubits, precision) needs: eight state-sized
 * vectors (y, p, q, four derivative slots f, one Runge-Kutta accumulator) plus tables and
 * reduction slots.  Returns 0 for unsupported arguments. */
size_t aqc_workspace_bytes(int n_qubits, int precision);

/* The same with options: AQC_WS_STEP_CONTROL adds one state-sized vector, which step-size
 * control (aqc_set_integrator with adaptive = 1) uses for the state at the start of a segment of
 * constant step, and y compensation (aqc_set_y_compensation) for the low part of y; the two are
 * exclusive, so AQC_WS_Y_COMPENSATION names the same vector.  Returns 0 for unsupported
 * arguments or unknown flags. */
#define AQC_WS_STEP_CONTROL 1u
#define AQC_WS_Y_COMPENSATION AQC_WS_STEP_CONTROL
size_t aqc_workspace_bytes_ex(int n_qubits, int precision, unsigned flags);

/* Create a context on `device` for n_qubits with state precision AQC_C128 or AQC_C64.
 * `workspace` is a caller-owned device pointer (256-byte aligned) of at least
 * aqc_workspace_bytes() bytes; `cuda_stream` is a cudaStream_t (NULL = legacy default).
 * On success *out receives the context. */
int aqc_create(aqc_ctx **out, int device, int precision, int n_qubits, void *workspace, size_t workspace_bytes,
               void *cuda_stream);

/* Release the host-side context (the workspace and staging vectors stay the caller's); waits
 * for pending staged copies and destroys the copy streams of aqc_transfer_attach.  NULL is
 * ignored. */
void aqc_destroy(aqc_ctx *ctx);

/* Order all later work of the context on `cuda_stream`. */
int aqc_set_stream(aqc_ctx *ctx, void *cuda_stream);

/* ---- Hamiltonian (Sec. I.A, Eq. SQH-Hamiltonian) ------------------------------------ */

/* Append n_terms Pauli products to group `group`: term k is
 *     coef[k] * prod_q P_q,  P_q = X if only xmask bit q set, Z if only zmask bit q set,
 *                                  Y if both set, identity otherwise,
 * so Y = i X Z per qubit.  xmask = zmask = 0 is the identity (energy shift m^(0)). */
int aqc_load_terms(aqc_ctx *ctx, int group, size_t n_terms, const uint64_t *xmask, const uint64_t *zmask,
                   const double *coef);

/* Append m Exact-Cover-3 clauses (Eq. 1clause) to group `group`: bits[3k..3k+2] are the
 * 0-based bits of clause k (distinct, < n); its diagonal energy on |z> is
 * scale * pen(#ones), pen per `penalty` (AQC_PEN_*; Eq. hci for AQC_PEN_SQUARED).
 * penalty | AQC_CLAUSE_STEPWISE makes the m clauses, in the given order, the sequence
 * h_1..h_m of the clause-by-clause term H_d(s) of Eq. kpath: clause j is further multiplied by
 * its coefficient in sum_k [(1 - s_k) H_{k-1} + s_k H_k] [0 <= s_k < 1], s_k = m s - k + 1,
 * H_k = h_1 + ... + h_k, H_0 = H_m = 0 (use a group weight of 1 for Eq. cbc).  One such
 * sequence per context; contexts holding one cannot join a batch. */
#define AQC_CLAUSE_STEPWISE 0x100
int aqc_load_clauses(aqc_ctx *ctx, int group, size_t m, const int32_t *bits, int penalty, double scale);

/* Remove all terms and clauses of all groups. */
int aqc_clear_hamiltonian(aqc_ctx *ctx);

/* ---- path schedule (Eq. aqc, Eq. nlpath) --------------------------------------------- */

/* Runtime T > 0 and weights A, B, C as cubics in s: w_g(s) = sum_k coef_g[k] s^k, with
 * s(t) per s_kind (AQC_S_*).  Straight line: A = {1,-1,0,0}, B = {0,1,0,0}, C = 0. */
int aqc_set_schedule(aqc_ctx *ctx, int s_kind, double T, const double coefA[4], const double coefB[4],
                     const double coefC[4]);

/* ---- integrator (Sec. I.B) ----------------------------------------------------------- */

/* Step grid.  n_steps > 0 sets N; n_steps == 0 applies the step rule
 * N = max(4, ceil(T * Lambda / kappa)), Lambda = max over s in [0,1] (1025-point grid) of
 * sum_g |w_g(s)| * ||H_g||_1 (sum of |prefactors| + max clause penalties), with kappa > 0
 * (0 selects 0.1; the PEC scheme is stable on the imaginary axis up to about 0.22).
 * adaptive = 0: the fixed-step grid h = T/N (tol ignored).
 * adaptive = 1: step-size control on the Milne estimate of Sec. I.B's predictor-corrector (the
 * paper states no control rule; this is the library's).  The run is a sequence of segments of
 * constant step h that each start with up to three RK4 steps; the first segment has the grid
 * step T/N.  A PEC step is accepted if (19/270) ||y_{n+1} - p_{n+1}|| <= tol ||y_{n+1}||; a
 * rejected step is discarded and a new segment starts at that step's start with h' = h/2.
 * After grow_after (aqc_set_step_growth, default 16) accepted PEC steps in a row with an
 * estimate <= tol ||y|| / 32, a new segment starts with h' = 2h.  A segment from t0 with
 * proposed step h' takes m = ceil((T - t0) / h') steps of (T - t0) / m, so the run lands on T.
 * The first PEC step of a segment also judges the RK4 start-up that built its history: if it
 * is rejected, the whole segment is redone from its own start with h/2.  Needs a workspace of
 * aqc_workspace_bytes_ex(n, precision, AQC_WS_STEP_CONTROL) bytes (else AQC_E_NOMEM).
 * Each PEC step reads two numbers back to the host (one synchronisation per step).  A step
 * below 2^-30 T/N fails with AQC_E_NUMERIC.  tol must be positive for adaptive = 1.  Resets
 * the integration (a new initial state is needed).  A context under step-size control cannot
 * join a batch. */
int aqc_set_integrator(aqc_ctx *ctx, int64_t n_steps, double kappa, int adaptive, double tol);

/* Consecutive small-estimate PEC steps before the step grows (0 = never grows). */
int aqc_set_step_growth(aqc_ctx *ctx, int grow_after);

/* The segments of constant step of the run so far (since the last initial state), in order:
 * up to max_out entries into out[], their total number into *count (may be NULL).  The fixed-
 * step grid is one segment. */
int aqc_get_segments(aqc_ctx *ctx, aqc_segment *out, int64_t max_out, int64_t *count);

/* The step grid the next (or current) propagation uses: N and h = T/N (step rule above). */
int aqc_get_grid(aqc_ctx *ctx, int64_t *n_steps, double *h);

/* Tile size of the shared-memory tiles (2^tile_bits amplitudes per CTA tile; 0 = default:
 * 13 for AQC_C64, 12 for AQC_C128; allowed 6..13 / 5..12).  Smaller tiles give more CTAs for
 * small states but more layout passes for large ones.  For AQC_C64 states of 22..28 qubits,
 * 16 selects cluster tiles: 2^16 amplitudes spread over a cluster of 8 CTAs that read each
 * other's shared memory, so two layout passes cover every bit (per-CTA tiles need three).
 * Batch members always use per-CTA tiles.  Resets the integrator. */
int aqc_set_tile_bits(aqc_ctx *ctx, int tile_bits);

/* Qubit relabelling (enable = 1, the default): when products flip several qubits, the library
 * may store qubit q at another index bit so that as many products as possible lie inside one
 * tile layout (a product no layout holds costs one extra state-vector read per evaluation).
 * Transparent to callers: every entry point takes and returns qubit-order indices and vectors
 * (Eq. ztensor); only the context's device vectors are reordered.  0 keeps the identity order.
 * A state already set is reordered when the tables are next built. */
int aqc_set_relabel(aqc_ctx *ctx, int enable);

/* Slab order of a PEC step (one PEC step = the one H*psi evaluation of Sec. I.B plus the
 * corrector/predictor update).  With three or more layouts, the last partial-sum pass and the
 * fused step kernel run as one launch over slabs of the index space (fixed values of up to
 * `slab_bits` index bits that neither layout holds): each slab's partial sum is consumed by
 * the step while it is still in L2, so a step moves two state vectors less through HBM.
 * 0 (default) = off, -1 = automatic (AQC_C64 states of 64 MiB or more, slabs of 2^20
 * amplitudes), 1..11 = at most that many slab bits.  On GB300 the slab launch moves about 10%
 * fewer bytes per step at 28 qubits but runs slower than the separate passes, hence off.  Results equal those of the layer order up
 * to the rounding of the partial sums' summation order.  The step's CTAs wait for the partial
 * tiles of their slab with a bounded poll; a wait that gives up (only possible after a fault
 * elsewhere) makes the next aqc_propagate with stats return AQC_E_TIMEOUT.  Does not reset the
 * integrator. */
int aqc_set_slab_bits(aqc_ctx *ctx, int slab_bits);

/* CUDA-graph replay of the PEC steps of Sec. I.B on the fixed-step grid: K consecutive steps
 * (all their layout passes) are captured once into a graph on a library-owned stream and
 * replayed on the context stream, K steps per host call, which removes the per-launch host
 * cost that dominates small states.  Before each replay one small kernel writes the K steps'
 * schedule weights, computed on the host by the same expression as the step-by-step path, into
 * the workspace; results are bit-identical to k_steps = 0.  k_steps: 0 = off, -1 = automatic
 * (default: K = 16 for n <= 20, off above), or a multiple of 4 in [4, 64].  The graph is
 * recaptured when the tables, the step size or the vectors change, and is not used under
 * step-size control, the slab order or a clause-by-clause sequence (those steps run one by
 * one).  Grid steps that remain after the last whole replay run one by one.  AQC_E_INVAL for
 * other k_steps; a failed capture returns AQC_E_CUDA from aqc_propagate. */
int aqc_set_graph_steps(aqc_ctx *ctx, int k_steps);

/* Turn of layouts for the PEC steps of Sec. I.B (this library's pass order): the fused step
 * kernel alternates between tile layouts 0 and 1 and, besides completing f_{n+1} = -i H p_{n+1},
 * the corrector and the predictor p_{n+2}, applies its own layout's products at the next step's
 * weights to p_{n+2} (restaged from L2 right after it is written), leaving that partial sum for
 * the next step, which then skips one partial pass: (3k + 4) N b per step instead of
 * (3k + 5) N b for k >= 2 layouts.  Applies on the fixed-step grid with per-CTA tiles, outside
 * batches, the slab order and clause-by-clause sequences, and when the products no layout holds
 * can stay in a partial pass (k >= 3, or none of them).  mode: 0 off (the default: on GB300 the
 * turned step measured slower, 4.71 against 4.37 ms at 28 qubits in complex64), 1 or -1 on where
 * it applies.  Results equal those of the plain pass order up to the order in which the
 * layouts' sums are added.  AQC_E_INVAL for other modes. */
int aqc_set_layout_turns(aqc_ctx *ctx, int mode);

/* Compensated corrector for complex64 states (reading of the FP32 state, Sec. I.B): each PEC
 * step adds its increment h/24 (9 f_{n+1} + 19 f_n - 5 f_{n-1} + f_{n-2}) to y as an exact
 * two-sum and keeps the rounding in a second complex64 vector (the workspace's extra vector,
 * AQC_WS_Y_COMPENSATION), folded into the next step's sum.  The FP32 rounding of y then no
 * longer accumulates over the run (about sqrt(steps) x 2^-24 without it); the step moves two
 * more vectors (9 N b instead of 7 N b of algorithmic bytes).  The state, norms, fidelity and
 * energy use y (within half an FP32 ulp of y + low part).  enable: 0 off (default) or 1; resets
 * the integrator (set the initial state again).  AQC_E_UNSUPPORTED for complex128 or under
 * step-size control, AQC_E_NOMEM without the extra vector. */
int aqc_set_y_compensation(aqc_ctx *ctx, int enable);

/* At most max_ctas CTAs for each layout pass of this context's evaluations (0 = no limit,
 * the default: every SM).  The pass kernels are persistent over tiles, so a smaller grid only
 * takes longer; results are unchanged (the state bit for bit, FP64 reductions up to their
 * summation order).  A serving loop gives a large state that runs beside a batch of small ones
 * part of the GPU, so that the batch's launches find SMs free instead of waiting for the large
 * state's kernels to end.  AQC_E_INVAL for max_ctas < 0. */
int aqc_set_grid_limit(aqc_ctx *ctx, int max_ctas);

/* Graph replays (aqc_set_graph_steps) the context has issued since creation. */
int aqc_get_graph_replays(const aqc_ctx *ctx, int64_t *out);

/* Set psi(0) and reset the integrator to t = 0.  kind = AQC_INIT_*; `basis` is the index for
 * AQC_INIT_BASIS and the Hamming weight k (0..n) for AQC_INIT_DICKE (the balanced superposition
 * of all basis states with k one-bits, the ground state of Eq. Hixyz in that sector);
 * `user` points to 2^n interleaved amplitudes in the state precision (host or device memory
 * per the kind).  AQC_INIT_STAGED takes the vector of the last aqc_stage_initial_state (the
 * context stream waits for its copy; none pending: AQC_E_STATE).  Out-of-range index or
 * weight: AQC_E_INVAL. */
int aqc_set_initial_state(aqc_ctx *ctx, int kind, uint64_t basis, const void *user);

/* Advance by up to max_steps grid steps (max_steps < 0: to t = T).  The first three steps
 * are RK4, the rest PEC.  Fills *stats if non-NULL (then synchronises the stream). */
int aqc_propagate(aqc_ctx *ctx, int64_t max_steps, aqc_stats *stats);

/* ---- results (Sec. II.B) ------------------------------------------------------------- */

/* Copy psi to dst (2^n interleaved amplitudes in the state precision); dst is device
 * memory if dst_on_device, else host memory (pinned memory recommended). */
int aqc_get_state(aqc_ctx *ctx, void *dst, int dst_on_device);

/* ---- staged host transfers ------------------------------------------------------------
 * Copy-engine transfers that overlap the integrator: the next instance's psi(0) travels to
 * the device, and the last instance's final psi (Sec. II.B's result) back to the host, while
 * the context stream integrates.  The caller owns two device staging vectors of 2^n
 * amplitudes each in the state precision (256-byte aligned, outside the workspace); the
 * library owns two copy streams and the events that order them against the context stream.  Host buffers should be pinned:
 * from pageable memory the copies are correct but do not overlap. */

/* Attach the staging vectors (device pointers, each 2^n amplitudes; distinct) and create the
 * copy streams.  Calling it again replaces the vectors after all pending copies finished.
 * NULL or misaligned vectors: AQC_E_INVAL; a failed stream or event creation: AQC_E_CUDA. */
int aqc_transfer_attach(aqc_ctx *ctx, void *stage_in, void *stage_out);

/* Enqueue the copy of 2^n host amplitudes (qubit order, state precision) into the input
 * staging vector, on the input copy stream, after the previous staged vector was consumed by
 * aqc_set_initial_state(AQC_INIT_STAGED).  Returns at once; `host_src` must stay unchanged
 * until aqc_transfer_wait returns or the context stream has passed the consuming
 * aqc_set_initial_state.  No aqc_transfer_attach: AQC_E_STATE. */
int aqc_stage_initial_state(aqc_ctx *ctx, const void *host_src);

/* Enqueue on the context stream the copy of psi (qubit order) into the output staging vector,
 * after the previous fetch left it, then on the output copy stream its copy into 2^n host
 * amplitudes at `host_dst`.  Returns at once; `host_dst` holds psi once aqc_transfer_wait
 * returns.  No aqc_transfer_attach: AQC_E_STATE. */
int aqc_fetch_state(aqc_ctx *ctx, void *host_dst);

/* Block the host until every staged copy and fetch issued so far has completed. */
int aqc_transfer_wait(aqc_ctx *ctx);

/* |<w|psi>|^2, the success probability P_1 of the solution w (Sec. II.B). */
int aqc_fidelity(aqc_ctx *ctx, uint64_t w, double *out);

/* <psi| sum_{g in group_mask} w_g H_g |psi>, not divided by ||psi||^2: bit g of group_mask
 * (1..7) selects group g (1 << AQC_GRP_B alone: the final energy E(T) of Sec. II.B when group B
 * holds H_f).  t >= 0: w_g = the group weight at time t, so group_mask = 7 gives <H(t)>;
 * t = AQC_UNIT_WEIGHTS (any t < 0): w_g = 1 for every selected group.  A clause-by-clause
 * sequence (Eq. kpath) takes its coefficients at t (at the current time for unit weights). */
#define AQC_UNIT_WEIGHTS (-1.0)
int aqc_energy(aqc_ctx *ctx, int group_mask, double t, double *out);

/* ||psi||^2 (FP64 accumulation). */
int aqc_norm2(aqc_ctx *ctx, double *out);

/* out = H(t) psi for caller-owned device vectors psi, out (state precision, 2^n amplitudes,
 * distinct, not inside the workspace).  Uses the workspace vector q as scratch, so it
 * must not overlap a propagation of the same context (same stream ordering suffices).
 * This is the stand-alone SQH matvec of Sec. I.A. */
int aqc_hpsi(aqc_ctx *ctx, double t, const void *psi, void *out);

/* ---- batches: many states stepped per launch ---------------------------------------- */
/* A batch steps many contexts of one device and precision together: each batched launch
 * processes (member, tile) work items of all members, so small states share the GPU, and K
 * PEC grid steps (Sec. I.B) are captured once in a CUDA graph and replayed.  Every member
 * keeps its own Hamiltonian, schedule, step grid and state; its arithmetic is the same as in
 * aqc_propagate, so a member's result does not depend on the other members.  While a context
 * is a member it must not be used directly; aqc_batch_remove hands it back (its step count,
 * ||psi||^2 and error estimates updated) for aqc_fidelity / aqc_energy / aqc_get_state. */
typedef struct aqc_batch aqc_batch;

/* Workspace bytes for a batch of up to max_members members and max_items work items per
 * layout level (a member contributes 2^(n - tile_bits) items per level).  0 if invalid. */
size_t aqc_batch_workspace_bytes(int max_members, int64_t max_items);

/* Create a batch; `workspace` is caller-owned device memory (256-byte aligned) of at least
 * aqc_batch_workspace_bytes() bytes; cuda_stream NULL makes the batch create its own stream. */
int aqc_batch_create(aqc_batch **out, int device, int precision, int max_members, int64_t max_items, void *workspace,
                     size_t workspace_bytes, void *cuda_stream);
void aqc_batch_destroy(aqc_batch *b);

/* Launch shape: threads per CTA (128 or 256) and PEC steps per graph replay (1..4096). */
int aqc_batch_set_shape(aqc_batch *b, int threads, int steps_per_round);

/* Add a context that has a Hamiltonian, a schedule and an initial state; its RK4 start-up
 * runs now on the batch stream.  *slot_out receives its slot.  Members run the fixed-step grid
 * with the plain corrector: a context under step-size control or y compensation, or with a
 * clause-by-clause sequence, is refused (AQC_E_UNSUPPORTED); a full batch gives AQC_E_NOMEM. */
int aqc_batch_add(aqc_batch *b, aqc_ctx *ctx, int *slot_out);

/* Remove the member in `slot` and hand its context back. */
int aqc_batch_remove(aqc_batch *b, int slot);

/* Enqueue `rounds` graph replays: every member advances by up to rounds * steps_per_round
 * grid steps and stops at its own t = T.  Asynchronous. */
int aqc_batch_run(aqc_batch *b, int64_t rounds);

/* Synchronise the batch stream; steps_done[slot] (array of max_members, may be NULL) gets each
 * member's completed grid steps (-1 for a free slot), *active_out the members not yet at T,
 * *launches_out the kernel launches issued so far. */
int aqc_batch_poll(aqc_batch *b, int64_t *steps_done, int *active_out, int64_t *launches_out);

/* Message of the last error of b (or of the last failed aqc_batch_create if b is NULL). */
const char *aqc_batch_last_error(const aqc_batch *b);

/* ---- spectrum along the path (Sec. IV.B: gap above the ground state) ------------------ */

/* Bytes of the caller-owned device memory aqc_lanczos needs for max_iter iterations: the
 * Krylov basis (max_iter + 1 state vectors) plus reduction scratch; 0 for bad arguments. */
size_t aqc_lanczos_workspace_bytes(int n_qubits, int precision, int max_iter);

/* Lowest eigenvalues of H(t) by the Lanczos method with full reorthogonalisation (classical
 * Gram-Schmidt twice per step, FP64 inner products) on the SQH matvec of aqc_hpsi.  The Krylov
 * space starts from the caller's device vector `start` (2^n amplitudes, state precision, need
 * not be normalised): for a Hamiltonian that conserves the Hamming weight (Eq. Sigmaz), a start
 * inside one sector (AQC_INIT_DICKE state) gives that sector's spectrum.  Each distinct
 * eigenvalue reachable from `start` appears once.  `work` (device, work_bytes >=
 * aqc_lanczos_workspace_bytes) is scratch.  Stops after max_iter steps, on an invariant
 * subspace, or when the n_eig lowest Ritz values moved by at most tol * max(1, |value|) over the
 * last 8 steps.  Writes the n_eig lowest Ritz values in ascending order to eig[] and their last
 * change to conv[] (host arrays of n_eig doubles; conv may be NULL) and the steps taken to
 * *iters_out (may be NULL).  Uses the context's partial-sum vector (not during a propagation
 * call); synchronises the context stream. */
int aqc_lanczos(aqc_ctx *ctx, double t, const void *start, void *work, size_t work_bytes, int max_iter, int n_eig,
                double tol, double *eig, double *conv, int *iters_out);

/* The lowest eigenpair (theta, x) of H(t) reachable from `start`, by the Lanczos iteration of
 * aqc_lanczos run until the Ritz residual beta_k |s_k| (from the recurrence, checked every 4
 * steps) is at most tol * max(1, |theta|), the Krylov space is invariant, or max_iter steps.  For a
 * Hamiltonian that conserves the Hamming weight and a start inside one weight sector, x is that
 * sector's ground state: the initial state of the XY algorithm is the ground state of Eq. Hixy in
 * the solution's sector (Sec. II.A).  x (unit norm, qubit order, state precision, phase chosen so
 * that <start|x> > 0) goes to the caller's device vector ground_out (2^n amplitudes, 16-byte
 * aligned); *theta_out gets theta, *resid_out (may be NULL) the residual ||H x - theta x|| of
 * the returned x, computed with one more H*x, *iters_out (may be NULL) the steps taken.  `work`
 * as for aqc_lanczos (aqc_lanczos_workspace_bytes).  Uses the context's partial-sum and scratch
 * vectors (not during a propagation call); synchronises the context stream. */
int aqc_lanczos_ground(aqc_ctx *ctx, double t, const void *start, void *work, size_t work_bytes, int max_iter,
                       double tol, double *theta_out, double *resid_out, void *ground_out, int *iters_out);

/* Host helper (no device work): the unit eigenvector, first entry >= 0, of the symmetric
 * tridiagonal matrix (a[0..k), b[0..k-1)) for its eigenvalue lam (inverse iteration with a
 * row-pivoted LU of T - lam I, three sweeps); the Ritz coefficients of aqc_lanczos_ground. */
int aqc_tridiag_eigvec(int k, const double *a, const double *b, double lam, double *out);

/* Host helper (no device work): the n_eig lowest eigenvalues, ascending, of the symmetric
 * tridiagonal matrix with diagonal a[0..k) and off-diagonal b[0..k-1), by Sturm-sequence
 * bisection to full double precision. */
int aqc_tridiag_eigvals(int k, const double *a, const double *b, int n_eig, double *out);

/* ---- entry point that allocates nothing ---------------------------------------------- */

/* Bytes of the library's static device scratch used by aqc_norm2_noalloc (per device). */
#define AQC_NOALLOC_SCRATCH_BYTES 16384

/* ||psi||^2 (FP64 accumulation) of a caller-owned device vector psi of n_amplitudes
 * interleaved amplitudes in `precision` (AQC_C128 or AQC_C64), written to the host double *out.
 * The paper has no counterpart: this is a service for callers that may not allocate device
 * memory -- code running inside another framework's memory pool or allocator, plugins whose
 * host application owns all GPU memory, or work issued where cudaMalloc is not allowed.  It
 * needs no context and no workspace and calls no allocating routine: its reduction scratch is a
 * static device array of AQC_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library
 * holds until exit.  It runs on the calling thread's current device (psi must live there) and
 * on `cuda_stream`, and synchronises that stream.  The first call on a device looks up the
 * scratch address once; make that first call before any stream capture.  All calls on a
 * device share the scratch, so calls that overlap on the GPU (different streams or threads
 * without ordering) race and give wrong results.  n_amplitudes must be in [1, 2^31] and psi
 * aligned to its amplitude size (16 bytes for AQC_C128, 8 for AQC_C64); other sizes and
 * pointers are rejected with AQC_E_INVAL; errors are described by aqc_last_error(NULL). */
int aqc_norm2_noalloc(int precision, const void *psi, uint64_t n_amplitudes, void *cuda_stream, double *out);

/* ---- measurement ---------------------------------------------------------------------- */

/* The FP64 FMA rate of `device` in TFLOP/s (2 flops per FMA), the denominator of the
 * complex128 PEC step's ALU roofline: one warm-up launch, then one timed launch (CUDA events on
 * `cuda_stream`) of 4 CTAs of 256 threads per SM, each thread running 8 independent FMA chains
 * for `iters` rounds.  Synchronises the stream; *ms_out (nullable) receives the timed launch's
 * duration.  iters in [1, 2^24], else AQC_E_INVAL; errors are described by
 * aqc_last_error(NULL).  The paper has no counterpart. */
int aqc_measure_fp64_fma(int device, void *cuda_stream, int iters, double *tflops_out, double *ms_out);

/* Self-test of the bounded waits (the paper has no counterpart): the library's kernels that wait
 * on other CTAs or on tensor copies poll a bounded number of times and, on giving up, set a fault
 * slot that the next aqc_propagate with stats reports as AQC_E_TIMEOUT.  This call runs that
 * give-up path on purpose, without any fault: one thread waits for a workspace flag that nothing
 * sets, for `polls` polls of about 1 us, records the give-up, and the host returns AQC_E_TIMEOUT
 * and clears the slot, so the context stays usable.  polls in [1, 10^7] (else AQC_E_INVAL).
 * Synchronises the context stream. */
int aqc_wait_selftest(aqc_ctx *ctx, int64_t polls);

/* Total kernel launches the context has issued since creation (monotone counter). */
int aqc_launch_count(const aqc_ctx *ctx, int64_t *out);

/* Message of the last error of ctx (or, for ctx == NULL, of the last failed aqc_create,
 * aqc_norm2_noalloc or aqc_measure_fp64_fma on the calling thread). */
const char *aqc_last_error(const aqc_ctx *ctx);

/* Library version string. */
const char *aqc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AQC_H */
