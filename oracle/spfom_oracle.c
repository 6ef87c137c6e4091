/*
 * spfom_oracle.c -- plain FP64 CPU oracle of the SPFOM iteration.
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the package smoke check and the
 * benchmark's CPU-baseline leg call this code; the CUDA library never does and
 * shares no source with it. Everything is single-threaded, written in the order
 * of the paper's definitions, with fixed summation orders, and compiled without
 * floating-point contraction so that it gives the same bits on every host.
 *
 * Notation (products j, resources i, segments l), with the paper's letters in
 * brackets: margin m_j = r_j - sum_i a_ij y_i  [r_j - eta_j], sales x_lj
 * [y_ij], no-purchase x_l0 [y_i0], duals y_i [eta_j], nominal attraction v_lj
 * [w_ij], shadow attraction w_lj [v_ij], no-purchase attraction v_l0 [w_i0].
 *
 * Sources:
 *   Section 3 (choice probability pi' of the generalized attraction model);
 *   Section 3.2 (sales-based LP, eqs. sales-based_obj .. sales-based_4);
 *   Section 4.1 (Lagrangian minimax entro_obj .. entro_cons_4, inner problem
 *     z_i, Algorithm 1 FAST-INNER, Lemma 1, golden-section search over y_i0,
 *     projected dual ascent, Algorithm 2 SPFOM);
 *   Section 4.2 (regularised dual step, eq. stronglycvxupdate);
 *   Section 4.3 (Algorithm 3, parallel SPFOM: many sampled customers per step);
 *   Section 5.2 (resource incidence, eq. new_NRM_1).
 * Averaging, the KKT residual and restarts are not in the paper (its Remark in
 * Section 4.2 notes that SPFOM forms no residuals); they are the solver's own
 * additions and are marked as such below.
 *
 * Parity pins (the tests check these against independent definitions):
 *   orc_margins, orc_segment_solve  -- brute force over all assortments with
 *       the closed-form choice probability, and LP strong duality (HiGHS);
 *   orc_sweep (sales / consumption)  -- finite differences of the dual
 *       function, whose gradient is c - A s (Danskin);
 *   orc_fast_inner, orc_segment_golden -- agree with orc_segment_solve as the
 *       golden-section tolerance shrinks (Lemma 1);
 *   orc_run dual step + averaging     -- convergence to the LP optimum on tiny
 *       instances; y >= 0; y stays 0 when capacities do not bind;
 *   orc_evaluate (KKT residual and restart rules; the paper defines neither,
 *       so the definition below is the solver's own) -- pinned by a
 *       hand-worked three-segment instance whose dual function is known in
 *       closed form: the residuals, the objective pair, every restart
 *       trigger (progress, epoch length at its boundary), the mu halving, the
 *       tau decay and both bounds of the tau-balance clamp.
 *   orc_recover (Lemma recover, Section 4.4) -- the recovered assortment
 *       probabilities reproduce the sales through the closed-form choice
 *       probabilities, sum to one, and turn the SBLP optimum (HiGHS) into a
 *       CBLP solution with the CBLP optimum's revenue (HiGHS on the
 *       enumerated CBLP).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int32_t n, m;
  int64_t L;
  const double* r;        /* [n] prices */
  const double* c;        /* [m] capacities */
  const int32_t* a_ptr;   /* [n+1] product j uses resources a_idx[a_ptr[j] .. a_ptr[j+1]) */
  const int32_t* a_idx;   /* [nnzA] */
  const double* a_val;    /* [nnzA] or NULL (all ones) */
  const int64_t* seg_ptr; /* [L+1] */
  const int32_t* seg_prod;/* [nnz] */
  const double* v;        /* [nnz] nominal attraction */
  const double* w;        /* [nnz] shadow attraction, NULL = MNL */
  const double* lam;      /* [L] arrival rate */
  const double* v0;       /* [L] no-purchase attraction */
} orc_instance;

typedef struct {
  double tau;           /* step size; <= 0 selects tau0 * mean(r) / mean(c) */
  double tau0;
  double mu;            /* regulariser of eq. stronglycvxupdate; 0 = Algorithm 2 step */
  double batch_frac;    /* p: each segment is solved with probability p; >= 1 = all */
  uint64_t seed;
  int64_t eval_every;   /* KKT evaluation period (solver addition); <= 0 = never */
  double restart_beta;  /* restart when KKT(avg) <= beta * KKT(anchor) (solver addition) */
  double restart_artificial; /* or when the epoch holds >= this fraction of all iterations */
  double restart_tau_decay;  /* tau <- tau * decay at each restart (1 = constant step) */
  double restart_tau_balance;/* > 0: restarts forced by the epoch length also scale tau by
                                clamp(sqrt(pinf / gap), b, 1 / b) (solver addition) */
  double kkt_tol;
} orc_params;

typedef struct {
  /* caller-owned arrays */
  double* y;       /* [m] current dual iterate */
  double* sum_y;   /* [m] sum of the duals at which the epoch's responses were taken */
  double* sum_g;   /* [m] sum of the epoch's consumption vectors */
  double* s;       /* [n] product sales of the last iteration */
  double* g;       /* [m] resource consumption of the last iteration */
  double* x_cur;   /* [nnz] current response of every segment (batch_frac < 1 only) */
  double* sum_x;   /* [nnz] epoch sum of every segment's response (solver addition), or NULL */
  /* scalars */
  double sum_P;
  int64_t count;   /* iterations in the current restart epoch */
  int64_t t;       /* iterations done */
  int64_t restarts;
  double mu_cur;
  double tau_used;
  double kkt_anchor;
  double z_sum;    /* sum_l z_l at the last iteration's dual point (full batch) */
  double P;        /* revenue r^T s of the last iteration */
  double dual_iter;/* c^T y + sum_l z_l at the last iteration's dual point (full batch) */
  double kkt, pinf, gap, dual_avg, primal_avg;
  int64_t evals;
  int32_t converged;
} orc_state;

/* ---------------------------------------------------------------- a1 ---- */
/* Margins m_j = r_j - sum_i a_ij y_i: the objective coefficient of the inner
 * problem z_i in Section 4.1 (r_j - eta_j) with the incidence of eq.
 * new_NRM_1. The inner sum runs in stored order. */
void orc_margins(const orc_instance* I, const double* y, double* marg) {
  for (int32_t j = 0; j < I->n; ++j) {
    double acc = 0.0;
    for (int32_t p = I->a_ptr[j]; p < I->a_ptr[j + 1]; ++p) {
      double a = I->a_val ? I->a_val[p] : 1.0;
      acc += a * y[I->a_idx[p]];
    }
    marg[j] = I->r[j] - acc;
  }
}

/* ---------------------------------------------------------------- a2 ---- */
/* Effective attractions of the generalized attraction model (Section 3, pi'):
 * with S offered, the denominator is v_0 + sum_{k in S} v_k + sum_{k in C\S} w_k
 * = vt_0 + sum_{k in S} vt_k with vt_k = v_k - w_k, vt_0 = v_0 + sum_{k in C} w_k. */
static double seg_vt0(const orc_instance* I, int64_t l) {
  double vt0 = I->v0[l];
  if (I->w)
    for (int64_t p = I->seg_ptr[l]; p < I->seg_ptr[l + 1]; ++p) vt0 += I->w[p];
  return vt0;
}
static double item_vt(const orc_instance* I, int64_t p) { return I->w ? I->v[p] - I->w[p] : I->v[p]; }

/* Key of item p: revenue per unit of the balance budget, m v / vt (+inf when
 * vt = 0). For MNL it is the margin, the order of Algorithm 1. */
static double item_key(const orc_instance* I, int64_t p, double mj) {
  double vt = item_vt(I, p);
  if (vt == 0.0) return INFINITY;
  return (mj * I->v[p]) / vt;
}

/* Sort positions pos[0..k) by key descending, ties by position ascending. */
static void sort_desc(int64_t* pos, double* key, int k) {
  for (int a = 1; a < k; ++a) {
    int64_t pp = pos[a];
    double kk = key[a];
    int b = a - 1;
    while (b >= 0 && (key[b] < kk || (key[b] == kk && pos[b] > pp))) {
      key[b + 1] = key[b];
      pos[b + 1] = pos[b];
      --b;
    }
    key[b + 1] = kk;
    pos[b + 1] = pp;
  }
}

#define ORC_KMAX 4096

/* Exact best response of segment l at margins marg (the inner problem z_i of
 * Section 4.1 in its GAM form). Every vertex of the segment's feasible set is
 * an assortment point x_j = lam v_j / (vt_0 + sum_{k in S} vt_k), j in S, so
 * z_l = lam * max_S N(S)/D(S) with N(S) = sum_S m v and D(S) = vt_0 + sum_S vt.
 * The maximiser is a prefix of the items with m_j > 0 sorted by key m v / vt
 * (the greedy order of Lemma 1): scan the prefixes, keep the first best one.
 * Writes x (length K, CSR order), returns z_l and the prefix length. */
double orc_segment_solve(const orc_instance* I, int64_t l, const double* marg, double* x, int32_t* kstar_out) {
  int64_t b = I->seg_ptr[l], e = I->seg_ptr[l + 1];
  int K = (int)(e - b);
  int64_t pos[ORC_KMAX];
  double key[ORC_KMAX];
  int nc = 0;
  for (int64_t p = b; p < e; ++p) {
    if (x) x[p - b] = 0.0;
    double mj = marg[I->seg_prod[p]];
    if (mj > 0.0 && nc < ORC_KMAX) {
      pos[nc] = p;
      key[nc] = item_key(I, p, mj);
      ++nc;
    }
  }
  sort_desc(pos, key, nc);
  double vt0 = seg_vt0(I, l);
  double N = 0.0, D = vt0, bestR = 0.0, bestD = vt0;
  int kstar = 0;
  for (int k = 0; k < nc; ++k) {
    int64_t p = pos[k];
    N += marg[I->seg_prod[p]] * I->v[p];
    D += item_vt(I, p);
    double R = N / D;
    if (R > bestR) {
      bestR = R;
      bestD = D;
      kstar = k + 1;
    }
  }
  double lam = I->lam[l];
  if (x)
    for (int k = 0; k < kstar; ++k) x[pos[k] - b] = lam * I->v[pos[k]] / bestD;
  if (kstar_out) *kstar_out = kstar;
  (void)K;
  return lam * bestR;
}

/* Algorithm 1 (FAST-INNER) in GAM form for a fixed no-purchase level, given as
 * u = x_l0 / vt_0. The balance leaves the budget lam - vt_0 u to spread over the
 * items, item j costing vt_j / v_j per unit of sales and capped at v_j u by the
 * scaling constraint; items are filled greedily in descending key order until
 * the budget is spent, continuing into non-positive margins while budget is
 * left (the budget starts at lam - x_l0, our reading of the initialisation).
 * Returns sum_j m_j x_j; x (CSR order) may be NULL. */
double orc_fast_inner(const orc_instance* I, int64_t l, const double* marg, double u, double* x) {
  int64_t b = I->seg_ptr[l], e = I->seg_ptr[l + 1];
  int64_t pos[ORC_KMAX];
  double key[ORC_KMAX];
  int k = 0;
  for (int64_t p = b; p < e && k < ORC_KMAX; ++p) {
    if (x) x[p - b] = 0.0;
    double mj = marg[I->seg_prod[p]];
    double vt = item_vt(I, p);
    if (vt == 0.0 && !(mj > 0.0)) continue; /* costs no budget, earns nothing: leave at 0 */
    pos[k] = p;
    key[k] = (vt == 0.0) ? INFINITY : (mj * I->v[p]) / vt;
    ++k;
  }
  sort_desc(pos, key, k);
  double budget = I->lam[l] - seg_vt0(I, l) * u;
  double val = 0.0;
  for (int t = 0; t < k; ++t) {
    int64_t p = pos[t];
    double vt = item_vt(I, p), vv = I->v[p], cap = vv * u, xj;
    if (vt == 0.0) {
      xj = cap;
    } else {
      if (!(budget > 0.0)) break;
      double need = budget * vv / vt;
      xj = need < cap ? need : cap;
      budget -= xj * vt / vv;
    }
    if (x) x[p - b] = xj;
    val += marg[I->seg_prod[p]] * xj;
  }
  return val;
}

/* Golden-section search of Section 4.1 over the no-purchase level, run on u =
 * x_l0 / vt_0 in [lam / (vt_0 + sum_{m_j>0} vt_j), lam / vt_0] (the optimal
 * assortment holds only positive margins, so the optimum lies in this range).
 * z(u) is concave (an LP value with u in the right-hand side). Stops when the
 * bracket is below eps * (upper end); returns the best value evaluated. */
double orc_segment_golden(const orc_instance* I, int64_t l, const double* marg, double eps) {
  int64_t b = I->seg_ptr[l], e = I->seg_ptr[l + 1];
  double vt0 = seg_vt0(I, l), sum_pos = 0.0;
  for (int64_t p = b; p < e; ++p)
    if (marg[I->seg_prod[p]] > 0.0) sum_pos += item_vt(I, p);
  double lam = I->lam[l];
  double lo = lam / (vt0 + sum_pos), hi = lam / vt0;
  const double phi = 0.6180339887498949; /* (sqrt(5) - 1) / 2 */
  double a = lo, bb = hi;
  double x1 = bb - phi * (bb - a), x2 = a + phi * (bb - a);
  double f1 = orc_fast_inner(I, l, marg, x1, NULL), f2 = orc_fast_inner(I, l, marg, x2, NULL);
  double best = orc_fast_inner(I, l, marg, lo, NULL);
  double fh = orc_fast_inner(I, l, marg, hi, NULL);
  if (fh > best) best = fh;
  for (int it = 0; it < 400 && (bb - a) > eps * hi; ++it) {
    if (f1 < f2) {
      a = x1; x1 = x2; f1 = f2;
      x2 = a + phi * (bb - a);
      f2 = orc_fast_inner(I, l, marg, x2, NULL);
    } else {
      bb = x2; x2 = x1; f2 = f1;
      x1 = bb - phi * (bb - a);
      f1 = orc_fast_inner(I, l, marg, x1, NULL);
    }
    if (f1 > best) best = f1;
    if (f2 > best) best = f2;
  }
  return best;
}

/* ---------------------------------------------------------------- a3 ---- */
/* Product sales s_j = sum_l x_lj (ascending l, then CSR position), resource
 * consumption g_i = sum_j a_ij s_j (ascending j, then stored order) and revenue
 * P = r^T s (ascending j): the aggregate sum_i y_ij of the dual step of
 * Algorithm 2, pushed through the incidence of eq. new_NRM_1. */
static void aggregate(const orc_instance* I, const double* s, double* g, double* P) {
  for (int32_t i = 0; i < I->m; ++i) g[i] = 0.0;
  double rev = 0.0;
  for (int32_t j = 0; j < I->n; ++j) {
    for (int32_t p = I->a_ptr[j]; p < I->a_ptr[j + 1]; ++p) {
      double a = I->a_val ? I->a_val[p] : 1.0;
      g[I->a_idx[p]] += a * s[j];
    }
    rev += I->r[j] * s[j];
  }
  *P = rev;
}

/* Full best-response sweep at dual point y: every segment's response, the
 * sales, consumption, revenue and sum_l z_l. Any of the outputs may be NULL. */
void orc_sweep(const orc_instance* I, const double* y, double* s_out, double* g_out, double* P_out,
               double* zsum_out, double* z_seg_out) {
  double* marg = (double*)malloc(sizeof(double) * (size_t)(I->n > 0 ? I->n : 1));
  double* s = (double*)calloc((size_t)(I->n > 0 ? I->n : 1), sizeof(double));
  double xbuf[ORC_KMAX];
  orc_margins(I, y, marg);
  double zsum = 0.0;
  for (int64_t l = 0; l < I->L; ++l) {
    double z = orc_segment_solve(I, l, marg, xbuf, NULL);
    if (z_seg_out) z_seg_out[l] = z;
    zsum += z;
    for (int64_t p = I->seg_ptr[l]; p < I->seg_ptr[l + 1]; ++p) s[I->seg_prod[p]] += xbuf[p - I->seg_ptr[l]];
  }
  if (s_out) memcpy(s_out, s, sizeof(double) * (size_t)I->n);
  if (g_out || P_out) {
    double* g = (double*)malloc(sizeof(double) * (size_t)(I->m > 0 ? I->m : 1));
    double P;
    aggregate(I, s, g, &P);
    if (g_out) memcpy(g_out, g, sizeof(double) * (size_t)I->m);
    if (P_out) *P_out = P;
    free(g);
  }
  if (zsum_out) *zsum_out = zsum;
  free(s);
  free(marg);
}

/* Dual function of the Lagrangian minimax (eq. entro_obj with the inner
 * maximisation done): Dual(y) = c^T y + sum_l z_l(y). Terms with y_i = 0 are
 * skipped so that non-binding capacities given as huge numbers contribute 0. */
double orc_dual(const orc_instance* I, const double* y) {
  double zsum = 0.0, cy = 0.0;
  orc_sweep(I, y, NULL, NULL, NULL, &zsum, NULL);
  for (int32_t i = 0; i < I->m; ++i)
    if (y[i] != 0.0) cy += I->c[i] * y[i];
  return cy + zsum;
}

/* ---------------------------------------------------------------- a7 ---- */
/* SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014) applied to
 * seed ^ (t << 32) ^ l: segment l is solved at iteration t when the hash is
 * below p * 2^64 (Bernoulli(p) sampling, so E[S_t] = p I as in the proof of
 * Theorem 1). */
static uint64_t splitmix64(uint64_t key) {
  uint64_t z = key + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
uint64_t orc_sample_hash(uint64_t seed, int64_t t, int64_t l) {
  return splitmix64(seed ^ ((uint64_t)t << 32) ^ (uint64_t)l);
}
static int sampled(const orc_params* P, int64_t t, int64_t l) {
  if (P->batch_frac >= 1.0) return 1;
  uint64_t thr = (uint64_t)ldexp(P->batch_frac, 64);
  return orc_sample_hash(P->seed, t, l) < thr;
}

double orc_default_tau(const orc_instance* I, double tau0) {
  double sr = 0.0, sc = 0.0;
  for (int32_t j = 0; j < I->n; ++j) sr += I->r[j];
  for (int32_t i = 0; i < I->m; ++i) sc += I->c[i];
  double mr = I->n > 0 ? sr / I->n : 0.0, mc = I->m > 0 ? sc / I->m : 0.0;
  if (!(mc > 0.0) || !(mr > 0.0)) return tau0;
  return tau0 * mr / mc;
}

void orc_state_init(const orc_instance* I, const orc_params* P, orc_state* S) {
  for (int32_t i = 0; i < I->m; ++i) {
    S->sum_y[i] = 0.0;
    S->sum_g[i] = 0.0;
    S->g[i] = 0.0;
  }
  for (int32_t j = 0; j < I->n; ++j) S->s[j] = 0.0;
  if (S->x_cur)
    for (int64_t p = 0; p < I->seg_ptr[I->L]; ++p) S->x_cur[p] = 0.0;
  S->sum_P = 0.0;
  S->count = 0;
  S->t = 0;
  S->restarts = 0;
  S->mu_cur = P->mu;
  S->tau_used = P->tau > 0.0 ? P->tau : orc_default_tau(I, P->tau0);
  S->kkt_anchor = INFINITY;
  S->z_sum = S->P = S->dual_iter = NAN;
  S->kkt = S->pinf = S->gap = S->dual_avg = S->primal_avg = NAN;
  S->evals = 0;
  S->converged = 0;
}

/* KKT residual of the averaged pair (solver addition, in the spirit of the
 * PDLP residuals the Remark of Section 4.2 contrasts SPFOM with):
 *   pinf = ||(gbar - c)_+||_2 / (1 + ||c||_2),
 *   gap  = |Dual(ybar) - Pbar| / (1 + |Dual(ybar)| + |Pbar|),  KKT = max(pinf, gap).
 * Restart (solver addition): when KKT <= beta * KKT at the last restart, or the
 * epoch holds at least restart_artificial of all iterations: y <- ybar, the
 * epoch sums are cleared, mu is halved (mu continuation, Theorem 1) and tau is
 * multiplied by restart_tau_decay (a restarted subgradient schedule); a restart
 * forced by the epoch length (no progress) also multiplies tau by
 * clamp(sqrt(pinf / gap), b, 1 / b) when restart_tau_balance = b > 0. */
void orc_evaluate(const orc_instance* I, const orc_params* P, orc_state* S) {
  int32_t m = I->m;
  double* ybar = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double cnt = (double)S->count;
  double pinf2 = 0.0, c2 = 0.0;
  for (int32_t i = 0; i < m; ++i) {
    ybar[i] = S->sum_y[i] / cnt;
    double gbar = S->sum_g[i] / cnt;
    double over = gbar - I->c[i];
    if (over > 0.0) pinf2 += over * over;
    c2 += I->c[i] * I->c[i];
  }
  double Pbar = S->sum_P / cnt;
  double D = orc_dual(I, ybar);
  S->pinf = sqrt(pinf2) / (1.0 + sqrt(c2));
  S->gap = fabs(D - Pbar) / (1.0 + fabs(D) + fabs(Pbar));
  S->kkt = S->pinf > S->gap ? S->pinf : S->gap;
  S->dual_avg = D;
  S->primal_avg = Pbar;
  S->evals += 1;
  S->converged = S->kkt <= P->kkt_tol;
  int progress = S->kkt <= P->restart_beta * S->kkt_anchor;
  if (!S->converged && (progress || (double)S->count >= P->restart_artificial * (double)S->t)) {
    for (int32_t i = 0; i < m; ++i) {
      S->y[i] = ybar[i];
      S->sum_y[i] = 0.0;
      S->sum_g[i] = 0.0;
    }
    S->sum_P = 0.0;
    S->count = 0;
    S->kkt_anchor = S->kkt;
    if (S->mu_cur > 0.0) S->mu_cur *= 0.5;
    S->tau_used *= P->restart_tau_decay;
    if (!progress && P->restart_tau_balance > 0.0) {
      /* a constant step leaves a duality gap of order tau; when the epoch
       * rule (not progress) forces the restart, move tau towards the step
       * that balances the gap against the infeasibility */
      double b = P->restart_tau_balance, f = 1.0;
      if (S->pinf > 0.0 && S->gap > 0.0) f = sqrt(S->pinf / S->gap);
      if (f < b) f = b;
      if (f > 1.0 / b) f = 1.0 / b;
      S->tau_used *= f;
    }
    S->restarts += 1;
  }
  free(ybar);
}

/* ------------------------------------------------------------ a1..a6 ---- */
/* One SPFOM iteration (Algorithm 2; Algorithm 3 with every worker's batch
 * together), from y = y^{t-1}:
 *   a1 margins at y;  a7 draw the segments to solve;
 *   a2 each drawn segment's exact best response (unsampled segments keep their
 *      previous response, so the aggregate runs over all segments as in the
 *      dual step of Algorithm 2);
 *   a3 s = sum_l x_l, g = A s, P = r^T s;
 *   a4 y_i <- max(0, (1 - tau mu) y_i - tau (c_i - g_i))   (eq. stronglycvxupdate;
 *      mu = 0 gives the step of Algorithm 2);
 *   a5 epoch sums: sum_y += y^{t-1}, sum_g += g, sum_P += P (solver addition);
 *   a6 every eval_every iterations, KKT of the averages and the restart test. */
/* One segment of iteration t: its response (solved if drawn, else the stale
 * one), added to the product sales s_acc and, with sum_x, to the epoch sums;
 * returns z_l when solved (0 otherwise). */
static double segment_step(const orc_instance* I, const orc_params* P, orc_state* S, int64_t l, int64_t t,
                           int full, const double* marg, double* xbuf, double* s_acc) {
  int64_t b = I->seg_ptr[l], e = I->seg_ptr[l + 1];
  double z = 0.0;
  if (full || sampled(P, t, l)) {
    z = orc_segment_solve(I, l, marg, xbuf, NULL);
    if (!full)
      for (int64_t p = b; p < e; ++p) S->x_cur[p] = xbuf[p - b];
  }
  for (int64_t p = b; p < e; ++p) s_acc[I->seg_prod[p]] += full ? xbuf[p - b] : S->x_cur[p];
  if (S->sum_x) /* the first iteration of an epoch starts the sums afresh */
    for (int64_t p = b; p < e; ++p) {
      double x = full ? xbuf[p - b] : S->x_cur[p];
      S->sum_x[p] = S->count == 0 ? x : S->sum_x[p] + x;
    }
  return z;
}

int orc_run(const orc_instance* I, const orc_params* P, orc_state* S, int64_t iters) {
  int32_t n = I->n, m = I->m;
  double* marg = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* yprev = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double xbuf[ORC_KMAX];
  int full = P->batch_frac >= 1.0;
  if (!full && !S->x_cur) {
    free(marg);
    free(yprev);
    return 1;
  }
  for (int64_t it = 0; it < iters; ++it) {
    if (S->converged) break;
    int64_t t = S->t + 1;
    memcpy(yprev, S->y, sizeof(double) * (size_t)m);
    orc_margins(I, S->y, marg);
    double zsum = 0.0;
    for (int32_t j = 0; j < n; ++j) S->s[j] = 0.0;
#ifdef _OPENMP
    /* Timing build only (liboracle_omp.so): segments split over the host's
     * cores, per-thread sales summed in thread order afterwards -- a
     * different summation order, so never used for parity. */
    {
      int nt = omp_get_max_threads();
      double* sl = (double*)calloc((size_t)nt * (size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel reduction(+ : zsum)
      {
        double xb[ORC_KMAX];
        double* my = sl + (size_t)omp_get_thread_num() * (size_t)(n > 0 ? n : 1);
#pragma omp for schedule(static)
        for (int64_t l = 0; l < I->L; ++l) zsum += segment_step(I, P, S, l, t, full, marg, xb, my);
      }
      for (int k = 0; k < nt; ++k)
        for (int32_t j = 0; j < n; ++j) S->s[j] += sl[(size_t)k * (size_t)n + j];
      free(sl);
    }
#else
    for (int64_t l = 0; l < I->L; ++l) zsum += segment_step(I, P, S, l, t, full, marg, xbuf, S->s);
#endif
    double Pv;
    aggregate(I, S->s, S->g, &Pv);
    double cy = 0.0;
    for (int32_t i = 0; i < m; ++i)
      if (yprev[i] != 0.0) cy += I->c[i] * yprev[i];
    S->z_sum = full ? zsum : NAN;
    S->dual_iter = full ? cy + zsum : NAN;
    S->P = Pv;
    double tau = S->tau_used, shrink = 1.0 - tau * S->mu_cur;
    for (int32_t i = 0; i < m; ++i) {
      double yi = shrink * yprev[i] - tau * (I->c[i] - S->g[i]);
      S->y[i] = yi > 0.0 ? yi : 0.0;
    }
    for (int32_t i = 0; i < m; ++i) {
      S->sum_y[i] += yprev[i];
      S->sum_g[i] += S->g[i];
    }
    S->sum_P += Pv;
    S->count += 1;
    S->t = t;
    if (P->eval_every > 0 && t % P->eval_every == 0) orc_evaluate(I, P, S);
  }
  free(marg);
  free(yprev);
  return 0;
}

/* ------------------------------------------------------------ f4 -------- */
/* Assortment probabilities from sales (Lemma recover, Section 4.4), GAM form
 * in build letters. For segment l with sales x_k (k in C_l, CSR order):
 *   u_k = x_k / v_k, the no-purchase sales x_0 = lam - sum_k (vt_k / v_k) x_k
 *   (the balance row), u_0 = x_0 / vt_0;
 *   rank the products by u descending (ties: lower CSR position first):
 *   u_(1) >= ... >= u_(K), u_(K+1) = 0; D_r = vt_0 + sum_{q <= r} vt_(q);
 *   alpha_0 = (u_0 - u_(1)) vt_0 / lam            (the empty assortment),
 *   alpha_r = (u_(r) - u_(r+1)) D_r / lam, r = 1..K (the top-r products).
 * Since the choice probability of product j in the top-r set is v_j / D_r,
 * lam sum_{r >= rank(j)} alpha_r v_j / D_r = v_j u_(rank j) = x_j (the sum
 * telescopes), and sum_r alpha_r = (x_0 + sum_k (vt_k / v_k) x_k) / lam = 1;
 * SBLP feasibility (x >= 0, x_k / v_k <= x_0 / vt_0) makes every alpha >= 0.
 * The paper sorts by y_ij / w_ij and sums the attractions of S_il = {0..l}
 * (no-purchase included): the same construction with its letters.
 * Output: alpha[seg_ptr[l] + l + r] for r = 0..K; order[seg_ptr[l] + r - 1] =
 * CSR position (within the segment) of the rank-r product. A segment with
 * lam = 0 gets alpha_0 = 1 and zeros. */
void orc_recover(const orc_instance* I, const double* x, double* alpha, int32_t* order) {
  int32_t pos[ORC_KMAX];
  double u[ORC_KMAX];
  for (int64_t l = 0; l < I->L; ++l) {
    int64_t b = I->seg_ptr[l];
    int K = (int)(I->seg_ptr[l + 1] - b);
    double lam = I->lam[l], vt0 = I->v0[l], bal = 0.0;
    for (int k = 0; k < K; ++k) {
      double w = I->w ? I->w[b + k] : 0.0;
      vt0 += w;
    }
    for (int k = 0; k < K; ++k) {
      double v = I->v[b + k], vt = v - (I->w ? I->w[b + k] : 0.0);
      u[k] = x[b + k] / v;
      bal += (vt / v) * x[b + k];
      pos[k] = k;
    }
    /* insertion sort of positions by u descending, stable */
    for (int a = 1; a < K; ++a) {
      int p = pos[a];
      int q = a - 1;
      while (q >= 0 && u[pos[q]] < u[p]) {
        pos[q + 1] = pos[q];
        --q;
      }
      pos[q + 1] = p;
    }
    double* al = alpha + b + l;
    if (!(lam > 0.0)) {
      al[0] = 1.0;
      for (int r = 1; r <= K; ++r) al[r] = 0.0;
    } else {
      double u0 = (lam - bal) / vt0;
      al[0] = ((u0 - (K > 0 ? u[pos[0]] : 0.0)) * vt0) / lam;
      double D = vt0;
      for (int r = 1; r <= K; ++r) {
        int p = pos[r - 1];
        double vt = I->v[b + p] - (I->w ? I->w[b + p] : 0.0);
        D += vt;
        double next = r < K ? u[pos[r]] : 0.0;
        al[r] = ((u[p] - next) * D) / lam;
      }
    }
    if (order)
      for (int r = 0; r < K; ++r) order[b + r] = pos[r];
  }
}
