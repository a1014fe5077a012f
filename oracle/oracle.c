/*
 * FP64 CPU oracle for batched MIMO tree-search detection (arXiv 2002.09561).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product path.  It shares
 * no code with the CUDA library.  Each function names the passage of the
 * paper it writes out; the conventions the paper leaves open are listed in
 * oracle.h.  Plain loops, no blocking or reordering beyond what the paper's
 * definitions state; one OpenMP loop over independent received vectors.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_P 16
#define ORC_MAX_Q 64 /* complex-tree children (64-QAM) */

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Sec. III-A: s_i belongs to a finite alphabet.  Square QAM with unit mean
 * energy: per real dimension the P-PAM levels (2k-(P-1))*alpha with
 * 2*alpha^2*(P^2-1)/3 = 1, i.e. alpha = sqrt(3 / (2 (Q-1))). */
int orc_pam_levels(int qam, double* levels) {
  int P = 0;
  for (int p = 2; p <= ORC_MAX_P; ++p)
    if (p * p == qam) P = p;
  if (P < 2) return -1;
  const double alpha = sqrt(3.0 / (2.0 * (qam - 1)));
  for (int k = 0; k < P; ++k) levels[k] = (2.0 * k - (P - 1)) * alpha;
  return P;
}

/* Real-valued form of y = Hs + n (Eq. 1), interleaved: complex entry
 * h = a + ib becomes [[a, -b], [b, a]]; y_j becomes (Re y_j, Im y_j). */
void orc_real_decompose(int N, int M, const double* H, const double* y, double* Hr, double* yr) {
  const int n = 2 * M;
  for (int r = 0; r < N; ++r) {
    for (int c = 0; c < M; ++c) {
      const double a = H[(r * M + c) * 2 + 0];
      const double b = H[(r * M + c) * 2 + 1];
      Hr[(2 * r) * n + 2 * c] = a;
      Hr[(2 * r) * n + 2 * c + 1] = -b;
      Hr[(2 * r + 1) * n + 2 * c] = b;
      Hr[(2 * r + 1) * n + 2 * c + 1] = a;
    }
    if (y && yr) {
      yr[2 * r] = y[2 * r];
      yr[2 * r + 1] = y[2 * r + 1];
    }
  }
}

/* Sec. III-B: H = QR, ybar = Q^T y, keep the upper n x n block of R.
 * Householder reflections; the sign of each row is then fixed so that the
 * diagonal of R is positive (flipping row k of R, entry k of ybar and
 * column k of Q together leaves QR and Q^T y consistent). */
int orc_qr(int m, int n, const double* A, const double* y, double* Q_out, double* R_out,
           double* ybar_out) {
  double* W = (double*)malloc(sizeof(double) * m * n);
  double* V = (double*)calloc((size_t)m * n, sizeof(double)); /* column k holds v_k */
  double* beta = (double*)calloc(n, sizeof(double));
  double* yy = (double*)malloc(sizeof(double) * m);
  memcpy(W, A, sizeof(double) * m * n);
  if (y) memcpy(yy, y, sizeof(double) * m);
  else memset(yy, 0, sizeof(double) * m);
  int singular = 0;

  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int i = k; i < m; ++i) s += W[i * n + k] * W[i * n + k];
    const double sigma = sqrt(s);
    if (sigma == 0.0) {
      singular = 1;
      continue;
    }
    const double alpha = (W[k * n + k] >= 0.0) ? -sigma : sigma;
    double vv = 0.0;
    for (int i = k; i < m; ++i) {
      double v = W[i * n + k];
      if (i == k) v -= alpha;
      V[i * n + k] = v;
      vv += v * v;
    }
    beta[k] = 2.0 / vv;
    for (int j = k; j < n; ++j) {
      double t = 0.0;
      for (int i = k; i < m; ++i) t += V[i * n + k] * W[i * n + j];
      t *= beta[k];
      for (int i = k; i < m; ++i) W[i * n + j] -= t * V[i * n + k];
    }
    double t = 0.0;
    for (int i = k; i < m; ++i) t += V[i * n + k] * yy[i];
    t *= beta[k];
    for (int i = k; i < m; ++i) yy[i] -= t * V[i * n + k];
  }

  double* sgn = (double*)malloc(sizeof(double) * n);
  for (int k = 0; k < n; ++k) sgn[k] = (W[k * n + k] < 0.0) ? -1.0 : 1.0;
  if (R_out) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) R_out[i * n + j] = (j >= i) ? sgn[i] * W[i * n + j] : 0.0;
  }
  if (ybar_out)
    for (int i = 0; i < n; ++i) ybar_out[i] = sgn[i] * yy[i];
  if (Q_out) {
    /* Q e_j = H_0 H_1 ... H_{n-1} e_j, then the sign fix on column j */
    double* e = (double*)malloc(sizeof(double) * m);
    for (int j = 0; j < n; ++j) {
      memset(e, 0, sizeof(double) * m);
      e[j] = 1.0;
      for (int k = n - 1; k >= 0; --k) {
        if (beta[k] == 0.0) continue;
        double t = 0.0;
        for (int i = k; i < m; ++i) t += V[i * n + k] * e[i];
        t *= beta[k];
        for (int i = k; i < m; ++i) e[i] -= t * V[i * n + k];
      }
      for (int i = 0; i < m; ++i) Q_out[i * n + j] = sgn[j] * e[i];
    }
    free(e);
  }
  free(sgn);
  free(W);
  free(V);
  free(beta);
  free(yy);
  return singular;
}

/* The objective of Sec. III-B written out: ||ybar - R x||^2. */
double orc_metric(int n, const double* R, const double* ybar, const double* levels, const int* k) {
  double m = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = ybar[i];
    for (int j = i; j < n; ++j) r -= R[i * n + j] * levels[k[j]];
    m += r * r;
  }
  return m;
}

/* Eq. 2: exhaustive ML over all qam^M vectors of the complex system. */
void orc_ml_bruteforce(int N, int M, int qam, const double* H, const double* y, uint8_t* sym_out,
                       double* d1, double* d2) {
  double lev[ORC_MAX_P];
  const int P = orc_pam_levels(qam, lev);
  int* q = (int*)calloc(M, sizeof(int));
  double best = INFINITY, second = INFINITY;
  for (;;) {
    double dist = 0.0;
    for (int r = 0; r < N; ++r) {
      double er = y[2 * r], ei = y[2 * r + 1];
      for (int c = 0; c < M; ++c) {
        const double hr = H[(r * M + c) * 2], hi = H[(r * M + c) * 2 + 1];
        const double sr = lev[q[c] / P], si = lev[q[c] % P];
        er -= hr * sr - hi * si;
        ei -= hr * si + hi * sr;
      }
      dist += er * er + ei * ei;
    }
    if (dist < best) {
      second = best;
      best = dist;
      for (int c = 0; c < M; ++c) sym_out[c] = (uint8_t)q[c];
    } else if (dist < second) {
      second = dist;
    }
    int c = 0;
    while (c < M && ++q[c] == qam) q[c++] = 0;
    if (c == M) break;
  }
  free(q);
  if (d1) *d1 = best;
  if (d2) *d2 = second;
}

/* ------------------------------------------------------------------------- */
/* Depth-first search (Algorithm 1 with the Best-FS list discipline, Sec.   */
/* IV-A) shared by the sphere decoder and the hybrid's master.              */
/* ------------------------------------------------------------------------- */

typedef struct {
  int n, P;
  const double *R, *yb, *lev;
  double r2;        /* squared radius: best leaf so far (or the initial one) */
  double r2b;       /* second-best leaf, used for pruning when two_best is set */
  int two_best;
  int order;
  uint64_t rng;
  long long budget;
  int budget_hit;
  int found;
  int* x;    /* current path, x[i] = PAM index of row i */
  int* best; /* best leaf */
  orc_stats* st;
  /* hybrid only */
  int K, d;
  double min_gap;
  int *kb_cur, *kb_nxt;
  double *kb_ped, *kb_ped2;
  void* kb_cand;
} dfs_ctx;

static uint64_t splitmix64_next(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Eq. 4 / Eq. inc: the interference of the fixed rows on row i,
 * c_i = ybar_i - sum_{j>i} R_ij x_j; the child with value a then adds
 * (c_i - R_ii a)^2 to its parent's partial distance. */
static double row_residual(int n, const double* R, const double* yb, const double* lev, const int* x,
                           int i) {
  double c = yb[i];
  for (int j = i + 1; j < n; ++j) c -= R[i * n + j] * lev[x[j]];
  return c;
}

/* Visiting order of the children: Best-FS sorts them by partial distance
 * (Sec. IV-A; equal distances keep the lower PAM index first). */
static void child_order(dfs_ctx* s, const double* ped, int* ord) {
  const int P = s->P;
  for (int k = 0; k < P; ++k) ord[k] = k;
  if (s->order == ORC_ORDER_SE || s->order == ORC_ORDER_REVERSED) {
    for (int a = 1; a < P; ++a) {
      int v = ord[a], b = a - 1;
      while (b >= 0 && ped[ord[b]] > ped[v]) {
        ord[b + 1] = ord[b];
        --b;
      }
      ord[b + 1] = v;
    }
    if (s->order == ORC_ORDER_REVERSED)
      for (int a = 0; a < P / 2; ++a) {
        int t = ord[a];
        ord[a] = ord[P - 1 - a];
        ord[P - 1 - a] = t;
      }
  } else if (s->order == ORC_ORDER_RANDOM) {
    for (int a = P - 1; a > 0; --a) {
      int b = (int)(splitmix64_next(&s->rng) % (uint64_t)(a + 1));
      int t = ord[a];
      ord[a] = ord[b];
      ord[b] = t;
    }
  }
}

/* Algorithm 1, leaf branch: a complete solution inside the sphere replaces
 * the radius, r^2 = E(s) (Sec. III-B, pruning). */
static void sd_leaf(dfs_ctx* s, double ped) {
  s->st->leaves++;
  s->found = 1;
  if (!s->two_best || ped < s->r2) {
    if (s->two_best) s->r2b = s->r2;
    s->r2 = ped;
    memcpy(s->best, s->x, sizeof(int) * s->n);
  } else {
    s->r2b = ped;
  }
}

/* Algorithm 1 body for the node whose rows n-1..i+1 are fixed (partial
 * distance ped_parent): branch over row i, evaluate every successor
 * incrementally, prune those with E >= r^2, recurse into the others in the
 * chosen order. */
static void sd_visit(dfs_ctx* s, int i, double ped_parent) {
  if (s->budget > 0 && s->st->nodes >= s->budget) {
    s->budget_hit = 1;
    return;
  }
  s->st->nodes++;
  const int n = s->n, P = s->P;
  const double c = row_residual(n, s->R, s->yb, s->lev, s->x, i);
  double ped[ORC_MAX_P] = {0};
  int ord[ORC_MAX_P] = {0};
  for (int k = 0; k < P; ++k) {
    const double dlt = c - s->R[i * n + i] * s->lev[k];
    ped[k] = ped_parent + dlt * dlt;
    s->st->peds++;
  }
  child_order(s, ped, ord);
  for (int t = 0; t < P; ++t) {
    const int k = ord[t];
    const double bound = s->two_best ? s->r2b : s->r2;
    if (!(ped[k] < bound)) continue; /* pruned */
    s->x[i] = k;
    if (i == 0) sd_leaf(s, ped[k]);
    else sd_visit(s, i - 1, ped[k]);
    if (s->budget_hit) return;
  }
}

int orc_sd(int n, int P, const double* R, const double* ybar, const double* levels, double r2_init,
           long long budget, int order, uint64_t seed, int two_best, int* k_out, double* d1,
           double* d2, orc_stats* st) {
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  if (!(r2_init > 0.0)) return -1;
  int* x = (int*)calloc(n, sizeof(int));
  int* best = (int*)calloc(n, sizeof(int));
  int status = ORC_V_OK;
  double r2 = r2_init;
  dfs_ctx s;
  for (;;) {
    memset(&s, 0, sizeof(s));
    s.n = n;
    s.P = P;
    s.R = R;
    s.yb = ybar;
    s.lev = levels;
    s.r2 = r2;
    s.r2b = r2;
    s.two_best = two_best;
    s.order = order;
    s.rng = seed;
    s.budget = budget;
    s.x = x;
    s.best = best;
    s.st = st;
    sd_visit(&s, n - 1, 0.0);
    if (s.found || s.budget_hit) break;
    /* empty sphere: double the radius and search again */
    r2 *= 2.0; /* empty sphere: double the radius r^2 (Sec. III-B names r^2 the radius) */
    st->restarts++;
    status = ORC_V_EMPTY_RETRIED;
    if (!(r2 < 1e300)) break;
  }
  if (s.budget_hit) status = ORC_V_BUDGET_EXCEEDED;
  if (s.found) {
    memcpy(k_out, best, sizeof(int) * n);
    if (d1) *d1 = s.r2;
    if (d2) *d2 = two_best ? s.r2b : INFINITY;
  } else {
    memset(k_out, 0, sizeof(int) * n);
    if (d1) *d1 = INFINITY;
    if (d2) *d2 = INFINITY;
  }
  free(x);
  free(best);
  return status;
}

/* ------------------------------------------------------------------------- */
/* K-best (Sec. VI): breadth-first, keep the K best nodes of every level.   */
/* ------------------------------------------------------------------------- */

typedef struct {
  double ped;
  int parent; /* rank of the parent in the previous level's sorted list */
  int k;      /* PAM index of the child */
} kb_cand;

static int kb_cmp(const void* a, const void* b) {
  const kb_cand* x = (const kb_cand*)a;
  const kb_cand* y = (const kb_cand*)b;
  if (x->ped < y->ped) return -1;
  if (x->ped > y->ped) return 1;
  if (x->parent != y->parent) return x->parent < y->parent ? -1 : 1;
  return (x->k > y->k) - (x->k < y->k);
}

static double rel_gap(double lo, double hi) {
  if (hi > 0.0) return (hi - lo) / hi;
  return (hi == lo) ? 0.0 : 1.0;
}

/* One K-best run over rows top..0, starting from a single node whose rows
 * above `top` are fixed in prefix[] with partial distance ped0.  Candidates
 * with PED >= r2 are dropped; the K smallest by (PED, parent rank, child)
 * survive.  Returns the number of final leaves (0 = empty); the best leaf
 * goes to out_path / out_ped. */
static int kbest_run(int n, int P, const double* R, const double* yb, const double* lev, int K,
                     double r2, int top, const int* prefix, double ped0, int* cur, int* nxt,
                     double* ped_cur, double* ped_nxt, kb_cand* cand, int* out_path,
                     double* out_ped, double* min_gap, orc_stats* st) {
  int S = 1;
  memcpy(cur, prefix, sizeof(int) * n);
  ped_cur[0] = ped0;
  for (int i = top; i >= 0; --i) {
    int C = 0;
    for (int p = 0; p < S; ++p) {
      st->nodes++;
      const double c = row_residual(n, R, yb, lev, cur + (size_t)p * n, i);
      for (int k = 0; k < P; ++k) {
        const double dlt = c - R[i * n + i] * lev[k];
        const double pd = ped_cur[p] + dlt * dlt;
        st->peds++;
        if (pd < r2) {
          cand[C].ped = pd;
          cand[C].parent = p;
          cand[C].k = k;
          ++C;
        }
      }
    }
    if (C == 0) return 0;
    qsort(cand, C, sizeof(kb_cand), kb_cmp);
    const int keep = C < K ? C : K;
    if (C > K && min_gap) {
      const double g = rel_gap(cand[K - 1].ped, cand[K].ped);
      if (g < *min_gap) *min_gap = g;
    }
    for (int t = 0; t < keep; ++t) {
      memcpy(nxt + (size_t)t * n, cur + (size_t)cand[t].parent * n, sizeof(int) * n);
      nxt[(size_t)t * n + i] = cand[t].k;
      ped_nxt[t] = cand[t].ped;
    }
    int* ti = cur;
    cur = nxt;
    nxt = ti;
    double* td = ped_cur;
    ped_cur = ped_nxt;
    ped_nxt = td;
    S = keep;
  }
  if (S > 1 && min_gap) {
    const double g = rel_gap(ped_cur[0], ped_cur[1]);
    if (g < *min_gap) *min_gap = g;
  }
  memcpy(out_path, cur, sizeof(int) * n);
  *out_ped = ped_cur[0];
  return S;
}

int orc_kbest(int n, int P, const double* R, const double* ybar, const double* levels, int K,
              double r2, int* k_out, double* d1, double* min_gap, orc_stats* st) {
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  if (K < 1 || !(r2 > 0.0)) return -1;
  int* cur = (int*)calloc((size_t)K * P * n, sizeof(int));
  int* nxt = (int*)calloc((size_t)K * P * n, sizeof(int));
  double* pc = (double*)calloc((size_t)K * P, sizeof(double));
  double* pn = (double*)calloc((size_t)K * P, sizeof(double));
  kb_cand* cand = (kb_cand*)malloc(sizeof(kb_cand) * (size_t)K * P);
  int* prefix = (int*)calloc(n, sizeof(int));
  double gap = 1.0, ped = INFINITY;
  int status = ORC_V_OK;
  for (;;) {
    gap = 1.0;
    int S = kbest_run(n, P, R, ybar, levels, K, r2, n - 1, prefix, 0.0, cur, nxt, pc, pn, cand,
                      k_out, &ped, &gap, st);
    if (S > 0) break;
    r2 *= 2.0; /* empty sphere: double the radius r^2 */
    st->restarts++;
    status = ORC_V_EMPTY_RETRIED;
    if (!(r2 < 1e300)) {
      memset(k_out, 0, sizeof(int) * n);
      break;
    }
  }
  if (d1) *d1 = ped;
  if (min_gap) *min_gap = gap;
  free(cur);
  free(nxt);
  free(pc);
  free(pn);
  free(cand);
  free(prefix);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Hybrid SD-K-best (Sec. VI): a Best-FS SD master over the top d rows; each */
/* node it reaches at depth d is handed to a K-best worker that finishes the */
/* remaining rows with the radius current at hand-off and shrinks it with   */
/* its best leaf.                                                           */
/* ------------------------------------------------------------------------- */

static void hybrid_handoff(dfs_ctx* s, int top, double ped) {
  int* leaf = (int*)malloc(sizeof(int) * s->n);
  double lp = INFINITY;
  int S = kbest_run(s->n, s->P, s->R, s->yb, s->lev, s->K, s->r2, top, s->x, ped, s->kb_cur,
                    s->kb_nxt, s->kb_ped, s->kb_ped2, (kb_cand*)s->kb_cand, leaf, &lp, &s->min_gap,
                    s->st);
  if (S > 0 && lp < s->r2) {
    s->st->leaves++;
    s->found = 1;
    s->r2 = lp;
    memcpy(s->best, leaf, sizeof(int) * s->n);
  }
  free(leaf);
}

static void hybrid_visit(dfs_ctx* s, int i, double ped_parent) {
  s->st->nodes++;
  const int n = s->n, P = s->P;
  const double c = row_residual(n, s->R, s->yb, s->lev, s->x, i);
  double ped[ORC_MAX_P] = {0};
  int ord[ORC_MAX_P] = {0};
  for (int k = 0; k < P; ++k) {
    const double dlt = c - s->R[i * n + i] * s->lev[k];
    ped[k] = ped_parent + dlt * dlt;
    s->st->peds++;
  }
  child_order(s, ped, ord);
  for (int t = 0; t < P; ++t) {
    const int k = ord[t];
    if (!(ped[k] < s->r2)) continue;
    s->x[i] = k;
    if (i == 0) sd_leaf(s, ped[k]);                     /* d = n: the master reaches leaves */
    else if (i == n - s->d) hybrid_handoff(s, i - 1, ped[k]); /* depth d reached */
    else hybrid_visit(s, i - 1, ped[k]);
  }
}

int orc_hybrid(int n, int P, const double* R, const double* ybar, const double* levels, int K,
               int d, double r2_init, int order, uint64_t seed, int* k_out, double* d1,
               double* min_gap, orc_stats* st) {
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  if (K < 1 || d < 0 || !(r2_init > 0.0)) return -1;
  if (d > n) d = n;
  int* x = (int*)calloc(n, sizeof(int));
  int* best = (int*)calloc(n, sizeof(int));
  int* cur = (int*)calloc((size_t)K * P * n, sizeof(int));
  int* nxt = (int*)calloc((size_t)K * P * n, sizeof(int));
  double* pc = (double*)calloc((size_t)K * P, sizeof(double));
  double* pn = (double*)calloc((size_t)K * P, sizeof(double));
  kb_cand* cand = (kb_cand*)malloc(sizeof(kb_cand) * (size_t)K * P);
  int status = ORC_V_OK;
  double r2 = r2_init;
  dfs_ctx s;
  for (;;) {
    memset(&s, 0, sizeof(s));
    s.n = n;
    s.P = P;
    s.R = R;
    s.yb = ybar;
    s.lev = levels;
    s.r2 = r2;
    s.r2b = r2;
    s.order = order;
    s.rng = seed;
    s.x = x;
    s.best = best;
    s.st = st;
    s.K = K;
    s.d = d;
    s.min_gap = 1.0;
    s.kb_cur = cur;
    s.kb_nxt = nxt;
    s.kb_ped = pc;
    s.kb_ped2 = pn;
    s.kb_cand = cand;
    if (d == 0) hybrid_handoff(&s, n - 1, 0.0);
    else hybrid_visit(&s, n - 1, 0.0);
    if (s.found) break;
    r2 *= 2.0; /* empty sphere: double the radius r^2 (Sec. III-B names r^2 the radius) */
    st->restarts++;
    status = ORC_V_EMPTY_RETRIED;
    if (!(r2 < 1e300)) break;
  }
  if (s.found) {
    memcpy(k_out, best, sizeof(int) * n);
    if (d1) *d1 = s.r2;
  } else {
    memset(k_out, 0, sizeof(int) * n);
    if (d1) *d1 = INFINITY;
  }
  if (min_gap) *min_gap = s.min_gap;
  free(x);
  free(best);
  free(cur);
  free(nxt);
  free(pc);
  free(pn);
  free(cand);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Complex tree: level j = real rows 2j+1 (Im) and 2j (Re) taken together.   */
/* ------------------------------------------------------------------------- */

/* Partial distances of the Q children of the node whose rows above 2j+1 are
 * fixed in x: row 2j+1 takes k_im, then row 2j (whose residual now includes
 * x[2j+1]) takes k_re.  Leaves x[2j], x[2j+1] modified. */
static void complex_children(int n, int P, const double* R, const double* yb, const double* lev, int* x, int j,
                             double ped_parent, double* ped) {
  const int r1 = 2 * j + 1, r0 = 2 * j;
  const double c1 = row_residual(n, R, yb, lev, x, r1);
  for (int q = 0; q < P * P; ++q) {
    const int k_re = q / P, k_im = q % P;
    const double d1v = c1 - R[r1 * n + r1] * lev[k_im];
    x[r1] = k_im;
    const double c0 = row_residual(n, R, yb, lev, x, r0);
    const double d0v = c0 - R[r0 * n + r0] * lev[k_re];
    ped[q] = ped_parent + d1v * d1v + d0v * d0v;
  }
}

static void sdc_visit(dfs_ctx* s, int j, double ped_parent) {
  if (s->budget > 0 && s->st->nodes >= s->budget) {
    s->budget_hit = 1;
    return;
  }
  s->st->nodes++;
  const int P = s->P, Q = P * P;
  double ped[ORC_MAX_Q];
  int ord[ORC_MAX_Q];
  complex_children(s->n, P, s->R, s->yb, s->lev, s->x, j, ped_parent, ped);
  s->st->peds += Q;
  /* increasing partial distance, ties to the lower q (stable insertion sort) */
  for (int q = 0; q < Q; ++q) {
    int b = q - 1;
    while (b >= 0 && ped[ord[b]] > ped[q]) {
      ord[b + 1] = ord[b];
      --b;
    }
    ord[b + 1] = q;
  }
  for (int t = 0; t < Q; ++t) {
    const int q = ord[t];
    const double bound = s->two_best ? s->r2b : s->r2;
    if (!(ped[q] < bound)) continue;
    s->x[2 * j + 1] = q % P;
    s->x[2 * j] = q / P;
    if (j == 0) sd_leaf(s, ped[q]);
    else sdc_visit(s, j - 1, ped[q]);
    if (s->budget_hit) return;
  }
}

int orc_sd_complex(int n, int P, const double* R, const double* ybar, const double* levels, double r2_init,
                   long long budget, int two_best, int* k_out, double* d1, double* d2, orc_stats* st) {
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  if (!(r2_init > 0.0) || (n & 1) || P * P > ORC_MAX_Q) return -1;
  int* x = (int*)calloc(n, sizeof(int));
  int* best = (int*)calloc(n, sizeof(int));
  int status = ORC_V_OK;
  double r2 = r2_init;
  dfs_ctx s;
  for (;;) {
    memset(&s, 0, sizeof(s));
    s.n = n;
    s.P = P;
    s.R = R;
    s.yb = ybar;
    s.lev = levels;
    s.r2 = r2;
    s.r2b = r2;
    s.two_best = two_best;
    s.budget = budget;
    s.x = x;
    s.best = best;
    s.st = st;
    sdc_visit(&s, n / 2 - 1, 0.0);
    if (s.found || s.budget_hit) break;
    r2 *= 2.0; /* empty sphere: double the radius r^2 and search again */
    st->restarts++;
    status = ORC_V_EMPTY_RETRIED;
    if (!(r2 < 1e300)) break;
  }
  if (s.budget_hit) status = ORC_V_BUDGET_EXCEEDED;
  if (s.found) {
    memcpy(k_out, best, sizeof(int) * n);
    if (d1) *d1 = s.r2;
    if (d2) *d2 = two_best ? s.r2b : INFINITY;
  } else {
    memset(k_out, 0, sizeof(int) * n);
    if (d1) *d1 = INFINITY;
    if (d2) *d2 = INFINITY;
  }
  free(x);
  free(best);
  return status;
}

/* K-best over complex levels; kb_cand.k holds the child's q. */
static int kbest_run_complex(int n, int P, const double* R, const double* yb, const double* lev, int K,
                             double r2, int* cur, int* nxt, double* ped_cur, double* ped_nxt, kb_cand* cand,
                             int* out_path, double* out_ped, double* min_gap, orc_stats* st) {
  const int Q = P * P;
  int S = 1;
  double ped[ORC_MAX_Q];
  memset(cur, 0, sizeof(int) * n);
  ped_cur[0] = 0.0;
  for (int j = n / 2 - 1; j >= 0; --j) {
    int C = 0;
    for (int p = 0; p < S; ++p) {
      st->nodes++;
      complex_children(n, P, R, yb, lev, cur + (size_t)p * n, j, ped_cur[p], ped);
      st->peds += Q;
      for (int q = 0; q < Q; ++q) {
        if (ped[q] < r2) {
          cand[C].ped = ped[q];
          cand[C].parent = p;
          cand[C].k = q;
          ++C;
        }
      }
    }
    if (C == 0) return 0;
    qsort(cand, C, sizeof(kb_cand), kb_cmp);
    const int keep = C < K ? C : K;
    if (C > K && min_gap) {
      const double g = rel_gap(cand[K - 1].ped, cand[K].ped);
      if (g < *min_gap) *min_gap = g;
    }
    for (int t = 0; t < keep; ++t) {
      memcpy(nxt + (size_t)t * n, cur + (size_t)cand[t].parent * n, sizeof(int) * n);
      nxt[(size_t)t * n + 2 * j + 1] = cand[t].k % P;
      nxt[(size_t)t * n + 2 * j] = cand[t].k / P;
      ped_nxt[t] = cand[t].ped;
    }
    int* ti = cur;
    cur = nxt;
    nxt = ti;
    double* td = ped_cur;
    ped_cur = ped_nxt;
    ped_nxt = td;
    S = keep;
  }
  if (S > 1 && min_gap) {
    const double g = rel_gap(ped_cur[0], ped_cur[1]);
    if (g < *min_gap) *min_gap = g;
  }
  memcpy(out_path, cur, sizeof(int) * n);
  *out_ped = ped_cur[0];
  return S;
}

int orc_kbest_complex(int n, int P, const double* R, const double* ybar, const double* levels, int K,
                      double r2, int* k_out, double* d1, double* min_gap, orc_stats* st) {
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  if (K < 1 || !(r2 > 0.0) || (n & 1) || P * P > ORC_MAX_Q) return -1;
  const size_t cap = (size_t)K * P * P;
  int* cur = (int*)calloc(cap * n, sizeof(int));
  int* nxt = (int*)calloc(cap * n, sizeof(int));
  double* pc = (double*)calloc(cap, sizeof(double));
  double* pn = (double*)calloc(cap, sizeof(double));
  kb_cand* cand = (kb_cand*)malloc(sizeof(kb_cand) * cap);
  double gap = 1.0, ped = INFINITY;
  int status = ORC_V_OK;
  for (;;) {
    gap = 1.0;
    const int S = kbest_run_complex(n, P, R, ybar, levels, K, r2, cur, nxt, pc, pn, cand, k_out, &ped, &gap, st);
    if (S > 0) break;
    r2 *= 2.0; /* empty sphere: double the radius r^2 */
    st->restarts++;
    status = ORC_V_EMPTY_RETRIED;
    if (!(r2 < 1e300)) {
      memset(k_out, 0, sizeof(int) * n);
      break;
    }
  }
  if (d1) *d1 = ped;
  if (min_gap) *min_gap = gap;
  free(cur);
  free(nxt);
  free(pc);
  free(pn);
  free(cand);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Batch drivers                                                             */
/* ------------------------------------------------------------------------- */

int orc_qr_batch(int B, int N, int M, const double* H, const double* y, double* R, double* ybar,
                 int nthreads) {
  if (B < 0 || N < M || M < 1) return -1;
  const int n = 2 * M, m = 2 * N;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
  {
    double* Hr = (double*)malloc(sizeof(double) * m * n);
    double* yr = (double*)malloc(sizeof(double) * m);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
    for (int b = 0; b < B; ++b) {
      orc_real_decompose(N, M, H + (size_t)b * N * M * 2, y + (size_t)b * N * 2, Hr, yr);
      orc_qr(m, n, Hr, yr, NULL, R + (size_t)b * n * n, ybar + (size_t)b * n);
    }
    free(Hr);
    free(yr);
  }
  return 0;
}

int orc_detect_batch(int algo, int B, int N, int M, int qam, const double* H, const double* y,
                     const double* noise_var, double radius, int K, int depth, long long budget,
                     int order, int want_gap, uint8_t* sym, double* metric, int* status,
                     long long* stats, double* gap, int nthreads) {
  double lev[ORC_MAX_P];
  const int P = orc_pam_levels(qam, lev);
  if (P < 0 || B < 0 || N < M || M < 1) return -1;
  if ((algo == ORC_KBEST || algo == ORC_HYBRID || algo == ORC_KBEST_COMPLEX) && K < 1) return -1;
  if (algo < ORC_SD || algo > ORC_KBEST_COMPLEX) return -1;
  const int n = 2 * M, m = 2 * N;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
  {
    double* Hr = (double*)malloc(sizeof(double) * m * n);
    double* yr = (double*)malloc(sizeof(double) * m);
    double* R = (double*)malloc(sizeof(double) * n * n);
    double* yb = (double*)malloc(sizeof(double) * n);
    int* k = (int*)malloc(sizeof(int) * n);
    int* k2 = (int*)malloc(sizeof(int) * n);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; ++b) {
      const double* Hb = H + (size_t)b * N * M * 2;
      const double* yv = y + (size_t)b * N * 2;
      orc_real_decompose(N, M, Hb, yv, Hr, yr);
      orc_qr(m, n, Hr, yr, NULL, R, yb);
      double r2 = radius;
      if (radius < 0.0) r2 = (double)N * M * noise_var[b]; /* Sec. III-B radius */
      orc_stats st;
      memset(&st, 0, sizeof(st));
      double d1 = INFINITY, d2 = INFINITY, g = 1.0;
      int vs = ORC_V_OK;
      if (algo == ORC_SD) {
        vs = orc_sd(n, P, R, yb, lev, r2, budget, order, (uint64_t)b, 0, k, &d1, NULL, &st);
        if (want_gap) {
          orc_stats st2;
          orc_sd(n, P, R, yb, lev, r2, budget, order, (uint64_t)b, 1, k2, NULL, &d2, &st2);
          g = rel_gap(d1, d2);
        }
      } else if (algo == ORC_SD_COMPLEX) {
        vs = orc_sd_complex(n, P, R, yb, lev, r2, budget, 0, k, &d1, NULL, &st);
        if (want_gap) {
          orc_stats st2;
          orc_sd_complex(n, P, R, yb, lev, r2, budget, 1, k2, NULL, &d2, &st2);
          g = rel_gap(d1, d2);
        }
      } else if (algo == ORC_KBEST_COMPLEX) {
        vs = orc_kbest_complex(n, P, R, yb, lev, K, r2, k, &d1, &g, &st);
      } else if (algo == ORC_KBEST) {
        vs = orc_kbest(n, P, R, yb, lev, K, r2, k, &d1, &g, &st);
      } else if (algo == ORC_HYBRID) {
        vs = orc_hybrid(n, P, R, yb, lev, K, depth, r2, order, (uint64_t)b, k, &d1, &g, &st);
      } else {
        uint8_t q[64];
        double e1, e2;
        orc_ml_bruteforce(N, M, qam, Hb, yv, q, &e1, &e2);
        for (int j = 0; j < M; ++j) {
          k[2 * j] = q[j] / P;
          k[2 * j + 1] = q[j] % P;
        }
        /* ||y - Hs||^2 and ||ybar - Rs||^2 differ by a constant (Sec. III-B) */
        const double offset = e1 - orc_metric(n, R, yb, lev, k);
        g = rel_gap(e1 - offset, e2 - offset);
      }
      if (sym)
        for (int j = 0; j < M; ++j) sym[(size_t)b * M + j] = (uint8_t)(k[2 * j] * P + k[2 * j + 1]);
      if (metric) metric[b] = orc_metric(n, R, yb, lev, k);
      if (status) status[b] = vs;
      if (stats) {
        stats[(size_t)b * 4 + 0] = st.nodes;
        stats[(size_t)b * 4 + 1] = st.peds;
        stats[(size_t)b * 4 + 2] = st.restarts;
        stats[(size_t)b * 4 + 3] = st.leaves;
      }
      if (gap) gap[b] = g;
    }
    free(Hr);
    free(yr);
    free(R);
    free(yb);
    free(k);
    free(k2);
  }
  return 0;
}

/* BER/SER accounting: Gray code per PAM dimension of q = k_re*P + k_im. */
void orc_count_errors(int B, int M, int qam, const uint8_t* sym_hat, const uint8_t* sym_true,
                      long long* out) {
  int P = 0;
  for (int p = 2; p <= ORC_MAX_P; ++p)
    if (p * p == qam) P = p;
  long long be = 0, se = 0;
  for (long long t = 0; t < (long long)B * M; ++t) {
    const int a = sym_hat[t], b = sym_true[t];
    if (a != b) ++se;
    const int ga_re = (a / P) ^ ((a / P) >> 1), gb_re = (b / P) ^ ((b / P) >> 1);
    const int ga_im = (a % P) ^ ((a % P) >> 1), gb_im = (b % P) ^ ((b % P) >> 1);
    int x = (ga_re ^ gb_re) | ((ga_im ^ gb_im) << 8);
    while (x) {
      be += x & 1;
      x >>= 1;
    }
  }
  out[0] = be;
  out[1] = se;
}
