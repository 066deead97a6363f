/*
 * Plain FP64 CPU oracle for the adiabatic-evolution hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the package's smoke check and the bench's CPU
 * baseline leg may load this code.  It shares no source with the CUDA path and is written
 * for obviousness, not speed: loops follow the paper's definitions one term at a time.
 *
 * What it computes:
 *   - SQH matvec (Sec. I.A, Eq. SQH-Hamiltonian and the paragraph after Eq. ising):
 *     H|psi> is the sum over stored Pauli products acting on each basis state |z>.  Each
 *     product is applied to |z> one qubit at a time (sigma^x flips bit, sigma^z gives a
 *     sign, sigma^y = both with a factor i) and the result is scattered into the output.
 *     Clause penalties of Exact Cover 3 (Eq. hci, Eq. sat) are diagonal in |z>.
 *   - Time-dependent coefficients (Sec. I.A last paragraph; Eq. aqc, Eq. nlpath):
 *     H(t) = sum_g w_g(s(t)) H_g with w_g a cubic polynomial in s; clauses marked as a
 *     clause-by-clause sequence (Eq. cbc, Eq. kpath) get in addition their coefficient in
 *     H_d(s), evaluated from the definition term by term.
 *   - Integration of i d/dt psi = H(t) psi (Eq. schroedinger, hbar = 1) with a fourth-order
 *     predictor-corrector that evaluates H|psi> once per step (Sec. I.B): Adams-Bashforth-4
 *     predictor, Adams-Moulton-4 corrector, PEC mode, fixed step h = T/N, started with three
 *     classical Runge-Kutta-4 steps.
 * Pins: tests/test_oracle_pins.py (dense Kronecker matrices, exact exponentials, closed
 * forms, convergence order, a library ODE solver), tests/test_oracle_xy_pins.py and
 * tests/test_oracle_cbc_pins.py; tests/test_oracle_mutations.py plants mistakes in a copy of
 * this file and checks that a pin catches each.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- Hamiltonian in SQH form ------------------------------------------------------- */
typedef struct {
  int n;                       /* qubits; basis index z has bit (q-1) = z_q (Eq. ztensor) */
  int nterms;                  /* Pauli products m * sigma...sigma (Eq. SQH-Hamiltonian)   */
  const uint64_t *xmask;       /* qubits carrying sigma^x or sigma^y                       */
  const uint64_t *zmask;       /* qubits carrying sigma^z or sigma^y                       */
  const double *coef;          /* real prefactor m_l^(j)                                   */
  const int *term_group;       /* which time-dependent weight multiplies the term (0..2)  */
  int nclauses;                /* EC3 clauses (Eq. 1clause)                                */
  const int *clause_bits;      /* 3 per clause, 0-based bits                               */
  const int *clause_group;
  const int *clause_penalty;   /* 0: [k != 1] (indicator), 1: (1-k)^2 (Eq. hci)            */
  const double *clause_scale;  /* Omega                                                    */
  const int *clause_step;      /* 0, or j >= 1: clause h_j of the clause-by-clause sequence */
  int step_m;                  /* m: length of that sequence (Eq. kpath)                    */
} or_ham;

/* ---- schedule: s(t) and the three group weights ------------------------------------ */
typedef struct {
  int s_kind;        /* 0: s = t/T (Eq. aqc); 1: s = 3 tau^2 - 2 tau^3, tau = t/T */
  double T;
  double poly[3][4]; /* w_g(s) = sum_k poly[g][k] s^k */
} or_sched;

/* w[0..2]: group weights at t; w[3]: the path parameter s(t) */
void or_weights(const or_sched *sc, double t, double w[4]) {
  double tau = t / sc->T;
  double s = tau;
  if (sc->s_kind == 1) s = 3.0 * tau * tau - 2.0 * tau * tau * tau;
  w[3] = s;
  for (int g = 0; g < 3; g++) {
    double v = 0.0, sk = 1.0;
    for (int k = 0; k < 4; k++) {
      v += sc->poly[g][k] * sk;
      sk *= s;
    }
    w[g] = v;
  }
}

/* single-qubit action on |b>: returns new bit and multiplies (re,im) by the matrix entry */
static int pauli_on_bit(int xq, int zq, int b, double *re, double *im) {
  double r = *re, i = *im;
  if (xq && zq) {              /* sigma^y |b> = i (-1)^b |1-b> */
    double sign = b ? -1.0 : 1.0;
    *re = -i * sign;
    *im = r * sign;
    return 1 - b;
  }
  if (xq) return 1 - b;        /* sigma^x |b> = |1-b> */
  if (zq) {                    /* sigma^z |b> = (-1)^b |b> */
    if (b) { *re = -r; *im = -i; }
    return b;
  }
  return b;
}

/* ---- threaded scatter helper ------------------------------------------------------- */
typedef struct {
  const or_ham *H;
  const double *w;
  const double *psi;
  double *out;
  uint64_t lo, hi;
  pthread_barrier_t *bar;
} or_job;

static double clause_penalty(int kind, int k) {
  if (kind == 1) return (double)((1 - k) * (1 - k));
  return k == 1 ? 0.0 : 1.0;
}

/* Coefficient of clause h_j (1-based) in Eq. kpath:
 *   H_d(s) = sum_{k=1}^{m} [(1 - s_k) H_{k-1} + s_k H_k] Theta(s_k) Theta(1 - s_k),
 *   s_k = m s - k + 1,  H_k = h_1 + ... + h_k (1 <= k <= m-1),  H_0 = H_m = 0.
 * Theta(s_k) Theta(1 - s_k) is read as s_k in [0, 1), so every s lies in one segment: the sum
 * has one nonzero term.  Near a segment end the rounded s_k of two neighbouring segments can
 * both land in [0, 1); the first (lowest k) is the segment s lies in. */
static double kpath_coef(int j, int m, double s) {
  for (int k = 1; k <= m; k++) {
    double sk = (double)m * s - (double)k + 1.0;
    if (!(sk >= 0.0 && sk < 1.0)) continue;
    int in_prev = (k - 1 >= 1) && (k - 1 <= m - 1) && (j <= k - 1); /* h_j is part of H_{k-1} */
    int in_cur = (k <= m - 1) && (j <= k);                           /* h_j is part of H_k */
    return (1.0 - sk) * (double)in_prev + sk * (double)in_cur;
  }
  return 0.0;
}

/* weight of clause k of H at the weights w (w[3] = s) */
static double clause_weight(const or_ham *H, const double *w, int k) {
  double g = w[H->clause_group[k]] * H->clause_scale[k];
  if (H->clause_step && H->clause_step[k] > 0) g *= kpath_coef(H->clause_step[k], H->step_m, w[3]);
  return g;
}

static void *scatter_worker(void *arg) {
  or_job *jb = (or_job *)arg;
  const or_ham *H = jb->H;
  /* one term at a time: |z> -> product of single-qubit operations, added at the image */
  for (int t = 0; t < H->nterms; t++) {
    double c = jb->w[H->term_group[t]] * H->coef[t];
    if (c != 0.0) {
      /* the qubits the product acts on, lowest first (identity elsewhere) */
      const uint64_t act = H->xmask[t] | H->zmask[t];
      for (uint64_t z = jb->lo; z < jb->hi; z++) {
        double re = jb->psi[2 * z], im = jb->psi[2 * z + 1];
        uint64_t zout = z;
        for (uint64_t rest = act; rest != 0; rest &= rest - 1) {
          int q = __builtin_ctzll(rest);
          int xq = (int)((H->xmask[t] >> q) & 1u);
          int zq = (int)((H->zmask[t] >> q) & 1u);
          int b = (int)((z >> q) & 1u);
          int nb = pauli_on_bit(xq, zq, b, &re, &im);
          zout = (zout & ~(1ull << q)) | ((uint64_t)nb << q);
        }
        jb->out[2 * zout] += c * re;
        jb->out[2 * zout + 1] += c * im;
      }
    }
    if (jb->bar) pthread_barrier_wait(jb->bar);
  }
  /* clause penalties are diagonal: (1 - #ones)^2 or [#ones != 1] on |z> (Eq. hci, Eq. sat) */
  for (uint64_t z = jb->lo; z < jb->hi; z++) {
    double d = 0.0;
    for (int k = 0; k < H->nclauses; k++) {
      const int *cb = H->clause_bits + 3 * k;
      int ones = (int)((z >> cb[0]) & 1u) + (int)((z >> cb[1]) & 1u) + (int)((z >> cb[2]) & 1u);
      d += clause_weight(H, jb->w, k) * clause_penalty(H->clause_penalty[k], ones);
    }
    jb->out[2 * z] += d * jb->psi[2 * z];
    jb->out[2 * z + 1] += d * jb->psi[2 * z + 1];
  }
  return NULL;
}

/* out = sum_g w_g H_g psi; psi and out are interleaved (re, im), length 2*2^n */
int or_hpsi(const or_ham *H, const double w[4], const double *psi, double *out, int nthreads) {
  uint64_t N = 1ull << H->n;
  memset(out, 0, sizeof(double) * 2 * N);
  if (nthreads < 1) nthreads = 1;
  if ((uint64_t)nthreads > N) nthreads = (int)N;
  if (nthreads == 1) {
    or_job jb = {H, w, psi, out, 0, N, NULL};
    scatter_worker(&jb);
    return 0;
  }
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
  or_job *jobs = (or_job *)malloc(sizeof(or_job) * nthreads);
  pthread_barrier_t bar;
  if (!th || !jobs || pthread_barrier_init(&bar, NULL, (unsigned)nthreads) != 0) {
    free(th);
    free(jobs);
    return -1;
  }
  for (int i = 0; i < nthreads; i++) {
    jobs[i].H = H; jobs[i].w = w; jobs[i].psi = psi; jobs[i].out = out;
    jobs[i].lo = N * (uint64_t)i / (uint64_t)nthreads;
    jobs[i].hi = N * (uint64_t)(i + 1) / (uint64_t)nthreads;
    jobs[i].bar = &bar;
  }
  for (int i = 1; i < nthreads; i++) pthread_create(&th[i], NULL, scatter_worker, &jobs[i]);
  scatter_worker(&jobs[0]);
  for (int i = 1; i < nthreads; i++) pthread_join(th[i], NULL);
  pthread_barrier_destroy(&bar);
  free(th);
  free(jobs);
  return 0;
}

/* Selected outputs (H psi)(z) for z in zs[0..nz): for every stored product, the one basis state
 * z' whose image under the product is |z> (z' = z xor xmask) contributes coef * (the product's
 * matrix element <z|P|z'>) * psi[z'], the element being built qubit by qubit as in the scatter
 * loop; clause penalties add their diagonal value at z.  Used to check single outputs of very
 * large states. */
int or_hpsi_at(const or_ham *H, const double w[4], const double *psi, int64_t nz, const uint64_t *zs, double *out) {
  for (int64_t k = 0; k < nz; k++) {
    const uint64_t z = zs[k];
    double acc_re = 0.0, acc_im = 0.0;
    for (int t = 0; t < H->nterms; t++) {
      double c = w[H->term_group[t]] * H->coef[t];
      if (c == 0.0) continue;
      uint64_t zsrc = z ^ H->xmask[t];
      double re = psi[2 * zsrc], im = psi[2 * zsrc + 1];
      uint64_t zimg = zsrc;
      for (uint64_t rest = H->xmask[t] | H->zmask[t]; rest != 0; rest &= rest - 1) {
        int q = __builtin_ctzll(rest); /* the qubits the product acts on, lowest first */
        int xq = (int)((H->xmask[t] >> q) & 1u);
        int zq = (int)((H->zmask[t] >> q) & 1u);
        int b = (int)((zsrc >> q) & 1u);
        int nb = pauli_on_bit(xq, zq, b, &re, &im);
        zimg = (zimg & ~(1ull << q)) | ((uint64_t)nb << q);
      }
      if (zimg != z) return -3; /* cannot happen: the image of z^x under P is z */
      acc_re += c * re;
      acc_im += c * im;
    }
    double d = 0.0;
    for (int j = 0; j < H->nclauses; j++) {
      const int *cb = H->clause_bits + 3 * j;
      int ones = (int)((z >> cb[0]) & 1u) + (int)((z >> cb[1]) & 1u) + (int)((z >> cb[2]) & 1u);
      d += clause_weight(H, w, j) * clause_penalty(H->clause_penalty[j], ones);
    }
    out[2 * k] = acc_re + d * psi[2 * z];
    out[2 * k + 1] = acc_im + d * psi[2 * z + 1];
  }
  return 0;
}

/* f = -i H(t) y   (Eq. schroedinger with hbar = 1) */
static int deriv(const or_ham *H, const or_sched *sc, double t, const double *y, double *f, double *tmp,
                 uint64_t N, int nthreads) {
  double w[4];
  or_weights(sc, t, w);
  if (or_hpsi(H, w, y, tmp, nthreads) != 0) return -1;
  for (uint64_t z = 0; z < N; z++) {
    /* -i (a + ib) = b - ia */
    f[2 * z] = tmp[2 * z + 1];
    f[2 * z + 1] = -tmp[2 * z];
  }
  return 0;
}

typedef struct {
  int64_t steps_done;
  int64_t evaluations;       /* H|psi> evaluations */
  double max_err_est;        /* max over PEC steps of (19/270) ||y_{n+1} - p_{n+1}|| */
  double last_err_est;
  double t_end;
} or_stats;

/*
 * Propagate psi (in/out, interleaved) from t = 0 over `max_steps` of the nsteps-step grid
 * h = T/nsteps (max_steps < 0: all nsteps, ending at t = T exactly).
 *   steps 1..3 (or fewer): classical RK4 (start-up; the paper does not say how the
 *     multistep history is started)
 *   steps 4..: PEC with
 *     p_{n+1} = y_n + h/24 (55 f_n - 59 f_{n-1} + 37 f_{n-2} - 9 f_{n-3})      (predict)
 *     f_{n+1} = -i H(t_{n+1}) p_{n+1}                                           (evaluate)
 *     y_{n+1} = y_n + h/24 (9 f_{n+1} + 19 f_n - 5 f_{n-1} + f_{n-2})           (correct)
 */
int or_propagate(const or_ham *H, const or_sched *sc, int64_t nsteps, int64_t max_steps, double *psi,
                 or_stats *st, int nthreads) {
  uint64_t N = 1ull << H->n;
  size_t bytes = sizeof(double) * 2 * N;
  if (nsteps < 1) return -2;
  if (max_steps < 0 || max_steps > nsteps) max_steps = nsteps;
  double h = sc->T / (double)nsteps;
  double *f[4], *tmp = (double *)malloc(bytes), *ys = (double *)malloc(bytes), *k = (double *)malloc(bytes),
         *acc = (double *)malloc(bytes), *p = (double *)malloc(bytes);
  for (int i = 0; i < 4; i++) f[i] = (double *)malloc(bytes);
  int bad = !tmp || !ys || !k || !acc || !p;
  for (int i = 0; i < 4; i++) bad |= !f[i];
  memset(st, 0, sizeof(*st));
  if (bad) goto fail;

  int64_t nrk = max_steps < 3 ? max_steps : 3;
  /* ---- RK4 start-up ---- */
  for (int64_t n = 0; n < nrk; n++) {
    double t = (double)n * h;
    /* k1 = f(t, y); also the history value f_n */
    if (deriv(H, sc, t, psi, f[n], tmp, N, nthreads)) goto fail;
    st->evaluations++;
    for (uint64_t i = 0; i < 2 * N; i++) acc[i] = f[n][i];
    /* k2 */
    for (uint64_t i = 0; i < 2 * N; i++) ys[i] = psi[i] + 0.5 * h * f[n][i];
    if (deriv(H, sc, t + 0.5 * h, ys, k, tmp, N, nthreads)) goto fail;
    st->evaluations++;
    for (uint64_t i = 0; i < 2 * N; i++) acc[i] += 2.0 * k[i];
    /* k3 */
    for (uint64_t i = 0; i < 2 * N; i++) ys[i] = psi[i] + 0.5 * h * k[i];
    if (deriv(H, sc, t + 0.5 * h, ys, k, tmp, N, nthreads)) goto fail;
    st->evaluations++;
    for (uint64_t i = 0; i < 2 * N; i++) acc[i] += 2.0 * k[i];
    /* k4 */
    for (uint64_t i = 0; i < 2 * N; i++) ys[i] = psi[i] + h * k[i];
    if (deriv(H, sc, t + h, ys, k, tmp, N, nthreads)) goto fail;
    st->evaluations++;
    for (uint64_t i = 0; i < 2 * N; i++) acc[i] += k[i];
    for (uint64_t i = 0; i < 2 * N; i++) psi[i] += (h / 6.0) * acc[i];
    st->steps_done++;
  }
  if (max_steps > 3) {
    /* history f_3 = f(t_3, y_3) */
    if (deriv(H, sc, 3.0 * h, psi, f[3], tmp, N, nthreads)) goto fail;
    st->evaluations++;
    /* f[(n)&3] holds f_n */
    for (int64_t n = 3; n < max_steps; n++) {
      const double *fn = f[n & 3], *fn1 = f[(n - 1) & 3], *fn2 = f[(n - 2) & 3], *fn3 = f[(n - 3) & 3];
      for (uint64_t i = 0; i < 2 * N; i++)
        p[i] = psi[i] + (h / 24.0) * (55.0 * fn[i] - 59.0 * fn1[i] + 37.0 * fn2[i] - 9.0 * fn3[i]);
      double *fnew = f[(n + 1) & 3]; /* overwrites f_{n-3}, no longer needed */
      if (deriv(H, sc, (double)(n + 1) * h, p, fnew, tmp, N, nthreads)) goto fail;
      st->evaluations++;
      double e2 = 0.0;
      for (uint64_t i = 0; i < 2 * N; i++) {
        double ynew = psi[i] + (h / 24.0) * (9.0 * fnew[i] + 19.0 * fn[i] - 5.0 * fn1[i] + fn2[i]);
        e2 += (ynew - p[i]) * (ynew - p[i]);
        psi[i] = ynew;
      }
      double est = (19.0 / 270.0) * sqrt(e2);
      st->last_err_est = est;
      if (est > st->max_err_est) st->max_err_est = est;
      st->steps_done++;
    }
  }
  st->t_end = (double)st->steps_done * h;
  free(tmp); free(ys); free(k); free(acc); free(p);
  for (int i = 0; i < 4; i++) free(f[i]);
  return 0;
fail:
  free(tmp); free(ys); free(k); free(acc); free(p);
  for (int i = 0; i < 4; i++) free(f[i]);
  return -1;
}

/* ---- adaptive step size (the paper states no step control; reading: Milne estimate) ----
 * The integration is a sequence of segments of constant step h.  A segment starting at t0 with
 * a proposed step hp takes m = ceil((T - t0) / hp) steps of h = (T - t0) / m, so that the last
 * step of the run lands on T; step k of the segment starts at t0 + k h.  Each segment begins
 * with up to three classical RK4 steps (accepted without an estimate), then f_3 and PEC steps as
 * in or_propagate.  A PEC step is accepted if its Milne estimate e = (19/270) ||y_{n+1} - p_{n+1}||
 * is at most tol ||y_{n+1}||.  A rejected step is discarded and a new segment starts with
 * hp = h/2: at the step's start, or, for the first PEC step of a segment (whose estimate also
 * judges the RK4 start-up that built its history), at the segment's own start, the RK4 steps
 * discarded with it.  After `grow_after` (> 0) accepted PEC steps in a row with
 * e <= tol ||y_{n+1}|| / 32, a new segment starts at the current time with hp = 2h.  A proposed
 * step below hmin fails the run (-4). */
typedef struct {
  double t0, h;
  int64_t steps; /* accepted grid steps of the segment */
  int32_t end;   /* 0 running, 1 reached T, 2 a PEC step was rejected, 3 the step grew */
  int32_t pad;
} or_segment;

typedef struct {
  int64_t steps_done;   /* accepted grid steps (RK4 and PEC) */
  int64_t evaluations;  /* H|psi> evaluations, rejected steps included */
  int64_t rejects;      /* rejected PEC steps */
  int64_t segments;     /* segments begun */
  int64_t pec_attempts; /* PEC steps tried (accepted and rejected) */
  double max_err_est;   /* max of e over accepted PEC steps */
  double t_end;
} or_astats;

/* m = ceil(R / hp), with R / hp a hair above an integer (rounding of hp = R / N) counted as
 * that integer, so a proposed step of exactly R / N gives N steps */
static int64_t segment_steps(double R, double hp) {
  double q = ceil((R / hp) * (1.0 - 1e-12));
  return q < 1.0 ? 1 : (int64_t)q;
}

/* ratio_log (may be NULL): e / (tol ||y_{n+1}||) of every PEC attempt, up to ratio_cap entries */
int or_propagate_adaptive(const or_ham *H, const or_sched *sc, double h0, double tol, int grow_after, double hmin,
                          int64_t max_steps, double *psi, or_astats *st, or_segment *log, int64_t log_cap,
                          double *ratio_log, int64_t ratio_cap, int nthreads) {
  uint64_t N = 1ull << H->n;
  size_t bytes = sizeof(double) * 2 * N;
  if (!(h0 > 0.0) || !(tol > 0.0) || !(hmin > 0.0)) return -2;
  double *f[4], *tmp = (double *)malloc(bytes), *ys = (double *)malloc(bytes), *k = (double *)malloc(bytes),
         *acc = (double *)malloc(bytes), *p = (double *)malloc(bytes), *ynew = (double *)malloc(bytes),
         *yseg = (double *)malloc(bytes); /* the state at the segment's start */
  for (int i = 0; i < 4; i++) f[i] = (double *)malloc(bytes);
  int bad = !tmp || !ys || !k || !acc || !p || !ynew || !yseg, rc = 0;
  for (int i = 0; i < 4; i++) bad |= !f[i];
  memset(st, 0, sizeof(*st));
  if (bad) { rc = -1; goto out; }

  double t0 = 0.0, hp = h0, h = 0.0;
  int64_t m = 0, kk = 0; /* steps in the segment, index of the next step */
  int small_run = 0, restart = 1, have_hist = 0;
  int64_t cur = -1;      /* log entry of the current segment */
  int64_t seg_done = 0;  /* accepted steps before the current segment */
  while (max_steps < 0 || st->steps_done < max_steps) {
    if (restart) {
      if (hp < hmin) { rc = -4; break; }
      double R = sc->T - t0;
      m = segment_steps(R, hp);
      h = R / (double)m;
      kk = 0;
      small_run = 0;
      have_hist = 0;
      restart = 0;
      memcpy(yseg, psi, bytes);
      seg_done = st->steps_done;
      st->segments++;
      cur = st->segments - 1;
      if (cur < log_cap) {
        log[cur].t0 = t0; log[cur].h = h; log[cur].steps = 0; log[cur].end = 0; log[cur].pad = 0;
      }
    }
    if (kk >= m) break;
    double t = t0 + (double)kk * h;
    if (kk < 3) {
      /* classical RK4 step; k1 is the history value f_kk */
      if (deriv(H, sc, t, psi, f[kk], tmp, N, nthreads)) { rc = -1; break; }
      for (uint64_t i = 0; i < 2 * N; i++) acc[i] = f[kk][i];
      for (uint64_t i = 0; i < 2 * N; i++) ys[i] = psi[i] + 0.5 * h * f[kk][i];
      if (deriv(H, sc, t + 0.5 * h, ys, k, tmp, N, nthreads)) { rc = -1; break; }
      for (uint64_t i = 0; i < 2 * N; i++) acc[i] += 2.0 * k[i];
      for (uint64_t i = 0; i < 2 * N; i++) ys[i] = psi[i] + 0.5 * h * k[i];
      if (deriv(H, sc, t + 0.5 * h, ys, k, tmp, N, nthreads)) { rc = -1; break; }
      for (uint64_t i = 0; i < 2 * N; i++) acc[i] += 2.0 * k[i];
      for (uint64_t i = 0; i < 2 * N; i++) ys[i] = psi[i] + h * k[i];
      if (deriv(H, sc, t + h, ys, k, tmp, N, nthreads)) { rc = -1; break; }
      for (uint64_t i = 0; i < 2 * N; i++) acc[i] += k[i];
      for (uint64_t i = 0; i < 2 * N; i++) psi[i] += (h / 6.0) * acc[i];
      st->evaluations += 4;
      st->steps_done++;
      kk++;
      if (cur < log_cap) log[cur].steps++;
      if (kk == m && cur < log_cap) log[cur].end = 1;
      continue;
    }
    if (!have_hist) { /* f_3 = f(t_3, y_3) */
      if (deriv(H, sc, t, psi, f[3], tmp, N, nthreads)) { rc = -1; break; }
      st->evaluations++;
      have_hist = 1;
    }
    const double *fn = f[kk & 3], *fn1 = f[(kk - 1) & 3], *fn2 = f[(kk - 2) & 3], *fn3 = f[(kk - 3) & 3];
    for (uint64_t i = 0; i < 2 * N; i++)
      p[i] = psi[i] + (h / 24.0) * (55.0 * fn[i] - 59.0 * fn1[i] + 37.0 * fn2[i] - 9.0 * fn3[i]);
    double *fnew = f[(kk + 1) & 3];
    if (deriv(H, sc, t0 + (double)(kk + 1) * h, p, fnew, tmp, N, nthreads)) { rc = -1; break; }
    st->evaluations++;
    double e2 = 0.0, y2 = 0.0;
    for (uint64_t i = 0; i < 2 * N; i++) {
      ynew[i] = psi[i] + (h / 24.0) * (9.0 * fnew[i] + 19.0 * fn[i] - 5.0 * fn1[i] + fn2[i]);
      e2 += (ynew[i] - p[i]) * (ynew[i] - p[i]);
      y2 += ynew[i] * ynew[i];
    }
    double est = (19.0 / 270.0) * sqrt(e2), lim = tol * sqrt(y2);
    if (ratio_log && st->pec_attempts < ratio_cap) ratio_log[st->pec_attempts] = est / lim;
    st->pec_attempts++;
    if (!(est <= lim)) { /* reject: a new segment with half the step */
      st->rejects++;
      if (cur < log_cap) log[cur].end = 2;
      if (kk == 3) { /* the first PEC step: the segment's start-up goes too */
        memcpy(psi, yseg, bytes);
        st->steps_done = seg_done;
        if (cur < log_cap) log[cur].steps = 0;
      } else {
        t0 = t;
      }
      hp = 0.5 * h;
      restart = 1;
      continue;
    }
    memcpy(psi, ynew, bytes);
    if (est > st->max_err_est) st->max_err_est = est;
    st->steps_done++;
    kk++;
    if (cur < log_cap) log[cur].steps++;
    if (kk == m) {
      if (cur < log_cap) log[cur].end = 1;
      continue;
    }
    small_run = est <= lim / 32.0 ? small_run + 1 : 0;
    if (grow_after > 0 && small_run >= grow_after) { /* the step grows: new segment from here */
      if (cur < log_cap) log[cur].end = 3;
      t0 = t0 + (double)kk * h;
      hp = 2.0 * h;
      restart = 1;
    }
  }
  st->t_end = (kk >= m && m > 0) ? t0 + (double)m * h : t0 + (double)kk * h;
out:
  free(tmp); free(ys); free(k); free(acc); free(p); free(ynew); free(yseg);
  for (int i = 0; i < 4; i++) free(f[i]);
  return rc;
}
