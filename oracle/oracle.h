/*
 * FP64 CPU oracle for batched MIMO tree-search detection.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that
 * the CUDA detectors are checked against.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * path (the CUDA library and its Python binding) never calls into it.  It
 * shares no code, header or table with the CUDA sources.
 *
 * Everything is double precision and written to follow the paper
 * ("Performance/Complexity Trade-offs of the Sphere Decoder Algorithm for
 * Massive MIMO Systems", arXiv 2002.09561) step by step:
 *   system model        y = H s + n                      Sec. III-A, Eq. 1
 *   ML detection        argmin ||y - H s||^2             Sec. III-A, Eq. 2
 *   QR preprocessing    ||y - Hs||^2 = ||ybar - R s||^2  Sec. III-B
 *   level decomposition sum_k g_k                        Sec. III-B, Eq. 4
 *   sphere decoder      select / branch / evaluate / prune, Algorithm 1
 *   Best-FS ordering    children sorted by PD             Sec. IV-A
 *   incremental PD      E(P_i) = E(P) + new terms        Sec. IV-C, Eq. inc
 *   K-best              keep the K best per level        Sec. VI
 *   hybrid SD-K-best    SD master hands nodes to K-best  Sec. VI
 *
 * Conventions fixed where the paper is silent:
 *   - unit-energy square QAM, PAM levels (2k-(P-1))*alpha per dimension,
 *     complex index q = k_re*P + k_im, Gray bits per dimension;
 *   - real-valued tree over the interleaved decomposition: real index 2j is
 *     Re(s_j), 2j+1 is Im(s_j); complex entry h becomes [[Re,-Im],[Im,Re]];
 *   - rows are expanded top row first (i = n-1 ... 0), survival is PED < r^2;
 *   - ties in child order go to the lower PAM index; K-best ties go to
 *     (PED, parent rank, child index);
 *   - noise variance sigma^2 per complex receive entry, read from the
 *     paper's radius formula r^2 = N M 10^(-SNR/10) (Sec. III-B) as
 *     sigma^2 = 10^(-SNR/10) for unit-energy symbols.  Parity unpinned (SNR
 *     convention): the paper's ML error-rate curves (Sec. VII-B) agree with
 *     it in shape only, 5.5 dB apart; the functions below take sigma^2 (or
 *     r^2) as an input and are pinned independently of it.
 */
#ifndef MIMO_ORACLE_H
#define MIMO_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SD = 0, ORC_KBEST = 1, ORC_HYBRID = 2, ORC_ML = 3, ORC_SD_COMPLEX = 4, ORC_KBEST_COMPLEX = 5 };
/* child visiting order of the depth-first part (SD and the hybrid master) */
enum { ORC_ORDER_SE = 0, ORC_ORDER_NATURAL = 1, ORC_ORDER_REVERSED = 2, ORC_ORDER_RANDOM = 3 };
/* per-vector outcome */
enum { ORC_V_OK = 0, ORC_V_EMPTY_RETRIED = 1, ORC_V_BUDGET_EXCEEDED = 2 };

/* PAM levels of the unit-energy square QAM with `qam` points; returns P or -1. */
int orc_pam_levels(int qam, double* levels);

/* Interleaved real decomposition of a complex N x M system (H row-major,
 * (re,im) pairs) into Hr (2N x 2M, row-major) and yr (2N).  yr may be NULL. */
void orc_real_decompose(int N, int M, const double* H, const double* y, double* Hr, double* yr);

/* Householder QR of the m x n real matrix A (row-major, m >= n) with a
 * positive diagonal.  R_out: n x n row-major (lower part zero).
 * ybar_out: first n entries of Q^T y (y may be NULL).  Q_out: m x n thin Q,
 * row-major, or NULL.  Returns 0, or 1 if a column is exactly dependent. */
int orc_qr(int m, int n, const double* A, const double* y, double* Q_out, double* R_out,
           double* ybar_out);

/* ||ybar - R x||^2 with x[i] = levels[k[i]]. */
double orc_metric(int n, const double* R, const double* ybar, const double* levels, const int* k);

/* Exact ML by enumerating all qam^M complex vectors on the original system
 * (Eq. 2).  sym_out: M complex indices.  d1/d2: best and second-best
 * ||y - H s||^2. */
void orc_ml_bruteforce(int N, int M, int qam, const double* H, const double* y, uint8_t* sym_out,
                       double* d1, double* d2);

typedef struct {
  long long nodes;     /* branched nodes, root included */
  long long peds;      /* children whose PED was evaluated */
  long long restarts;  /* empty-sphere radius doublings */
  long long leaves;    /* leaves that shrank the radius */
} orc_stats;

/* Schnorr-Euchner (Best-FS) depth-first sphere decoder on (R, ybar).
 * r2_init: initial squared radius (INFINITY allowed).  budget: cap on
 * branched nodes (0 = none).  order: ORC_ORDER_*; seed for RANDOM.
 * two_best: prune against the second-best leaf so that d2 is exact.
 * k_out: n PAM indices.  Returns ORC_V_*. */
int orc_sd(int n, int P, const double* R, const double* ybar, const double* levels, double r2_init,
           long long budget, int order, uint64_t seed, int two_best, int* k_out, double* d1,
           double* d2, orc_stats* st);

/* K-best on (R, ybar) with squared radius r2 (INFINITY = plain K-best).
 * min_gap: smallest relative gap at a K / K+1 selection boundary or between
 * the two best final leaves (1.0 if none).  Returns ORC_V_* (EMPTY when no
 * candidate survives; the caller doubles the radius). */
int orc_kbest(int n, int P, const double* R, const double* ybar, const double* levels, int K,
              double r2, int* k_out, double* d1, double* min_gap, orc_stats* st);

/* Hybrid SD-K-best: Best-FS SD over the top d rows with a running radius;
 * every prefix inside the sphere is finished by K-best(K) over the remaining
 * rows with the radius current at hand-off.  order: visiting order of the
 * prefixes (the result does not depend on it). */
int orc_hybrid(int n, int P, const double* R, const double* ybar, const double* levels, int K,
               int d, double r2_init, int order, uint64_t seed, int* k_out, double* d1,
               double* min_gap, orc_stats* st);

/* Complex-tree searches: one tree level per complex antenna with the Q = P^2
 * symbols of the QAM alphabet as children (the tree of Sec. III-B, which the
 * paper's node counts refer to).  On the interleaved real (R, ybar) above,
 * complex level j is the pair of real rows 2j+1 (imaginary part) and 2j
 * (real part): child q = k_re * P + k_im has the partial distance of the
 * real path that fixes row 2j+1 to k_im and then row 2j to k_re (Eq. inc
 * applied twice), so a complex node is the real tree grouped two levels at
 * a time.  Children are visited / selected in increasing partial distance,
 * ties to the lower q (K-best: key (distance, parent rank, q)).  n = 2M must
 * be even; nodes count complex-level branchings, peds count children. */
int orc_sd_complex(int n, int P, const double* R, const double* ybar, const double* levels, double r2_init,
                   long long budget, int two_best, int* k_out, double* d1, double* d2, orc_stats* st);
int orc_kbest_complex(int n, int P, const double* R, const double* ybar, const double* levels, int K,
                      double r2, int* k_out, double* d1, double* min_gap, orc_stats* st);

/* Batch driver over B independent received vectors (complex H [B][N][M][2],
 * y [B][N][2], noise_var [B]).  radius_mode: r2 >= 0 uses that value,
 * INFINITY none, negative = the paper's r^2 = N*M*sigma^2.
 * Outputs: sym [B][M], metric [B] (||ybar - R s||^2), status [B],
 * stats [B][4] (nodes, peds, restarts, leaves), gap [B] (d2-d1)/d2 for SD
 * and ML, min_gap for K-best and hybrid.  Any output may be NULL.
 * nthreads <= 0 uses all cores.  Returns 0 or -1 on bad arguments. */
int orc_detect_batch(int algo, int B, int N, int M, int qam, const double* H, const double* y,
                     const double* noise_var, double radius, int K, int depth, long long budget,
                     int order, int want_gap, uint8_t* sym, double* metric, int* status,
                     long long* stats, double* gap, int nthreads);

/* QR of a batch: R [B][n][n] row-major and ybar [B][n] (n = 2M). */
int orc_qr_batch(int B, int N, int M, const double* H, const double* y, double* R, double* ybar,
                 int nthreads);

/* Bit and symbol errors of detected vs transmitted complex indices, with
 * the Gray map per PAM dimension.  out[0] = bit errors, out[1] = symbol
 * errors. */
void orc_count_errors(int B, int M, int qam, const uint8_t* sym_hat, const uint8_t* sym_true,
                      long long* out);

int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
