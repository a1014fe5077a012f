/*
 * mimo_detect.h -- C ABI of the GB300 (sm_103a) batched MIMO tree-search
 * detectors: sphere decoding, K-best and the hybrid SD / K-best of
 * "Performance/Complexity Trade-offs of the Sphere Decoder Algorithm for
 * Massive MIMO Systems" (arXiv 2002.09561).
 *
 * Problem (Sec. III-A, Eq. 1): for each of `batch` independent received
 * vectors, y = H s + n with H an n_rx x n_tx complex channel, s a vector of
 * n_tx symbols from a unit-energy square QAM alphabet and n white noise of
 * variance noise_var per complex entry.  Every detector first reduces the
 * problem by a QR factorisation (Sec. III-B) and then searches the tree of
 * Eq. 4 over the real-valued, interleaved decomposition (real index 2j is
 * Re s_j, 2j+1 is Im s_j; rows are expanded from the last one, 2 n_tx - 1,
 * down to 0).
 *
 * Memory.  Unless a call sets MDX_HOST_BUFFERS in mdx_params.flags, every
 * array argument is a DEVICE pointer on the context's device, owned by the
 * caller; the library never frees caller memory and never keeps a caller
 * pointer beyond the call.  With MDX_HOST_BUFFERS, the same arguments are
 * host pointers (pinned memory gives asynchronous copies); the library
 * stages them through buffers it allocated in mdx_create (the inputs are
 * copied in chunks on a stream of the context's own, after the work already
 * queued on `stream`, and the QR of each chunk starts as soon as that chunk
 * is in) and returns after the results are back in host memory.
 *
 * Layouts (all row-major, C order):
 *   H          double [batch][n_rx][n_tx][2]   (re, im) pairs
 *   y          double [batch][n_rx][2]
 *   noise_var  double [batch]                  sigma^2 per complex entry
 *   sym_out    uint8  [batch][n_tx]            complex index q = k_re*P + k_im,
 *                                              P = sqrt(qam), PAM level
 *                                              (2k-(P-1))*sqrt(3/(2(qam-1)))
 *   metric_out double [batch]                  ||ybar - R s_hat||^2 in FP64
 *   vstatus    int32  [batch]                  MDX_V_* per vector
 *   stats      int64  [batch][5]               nodes branched, partial distances
 *                                              evaluated, radius doublings,
 *                                              leaves re-scored in FP64, and the
 *                                              algorithmic FP32 flops of the search,
 *                                              sum over branched nodes at row i of
 *                                              2 (n-1-i) + 4 P; may be NULL
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  Device-pointer calls only enqueue work and return; a
 * CUDA error raised by an earlier asynchronous launch is reported by the
 * next call as MDX_ECUDA.  A context is not thread-safe: one host thread
 * (or external serialisation) per context.
 *
 * Errors.  Every entry point validates its arguments before enqueuing
 * anything and returns MDX_EINVAL (bad pointer, size or parameter),
 * MDX_EUNSUPPORTED (a size beyond what the context was created for or the
 * kernels support) or MDX_ECUDA; on any error nothing has been written to
 * the outputs.  mdx_strerror() names a status; mdx_last_error() returns a
 * one-line description of the last failure of this context.
 */
#ifndef MIMO_DETECT_H
#define MIMO_DETECT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdx_ctx mdx_ctx;

typedef enum {
  MDX_OK = 0,
  MDX_EINVAL = -1,
  MDX_EUNSUPPORTED = -2,
  MDX_ENOMEM = -3,
  MDX_ECUDA = -4
} mdx_status;

/* Per-vector outcome written to vstatus. */
enum {
  MDX_V_OK = 0,              /* searched to completion */
  MDX_V_EMPTY_RETRIED = 1,   /* the initial sphere held no leaf; the radius was doubled
                                (r^2 <- 2 r^2) until one did; the answer is still exact
                                for detect_sd */
  MDX_V_BUDGET_EXCEEDED = 2, /* node_budget ran out; best leaf found so far (or the
                                first leaf reached) is returned */
  MDX_V_SINGULAR = 3         /* R has a zero diagonal entry; outputs are zero */
};

/* mdx_params.flags */
enum {
  MDX_HOST_BUFFERS = 1 << 0, /* array arguments are host pointers (see Memory) */
  MDX_NO_RESCORE = 1 << 1,   /* skip the FP64 re-scoring of the final leaf candidates;
                                metric_out is then the FP32 partial distance */
  MDX_LEARNED_RADIUS = 1 << 2, /* initial radius from the context's MLP (mdx_mlp_load) */
  MDX_SEQUENTIAL_SEARCH = 1 << 3, /* detect_sd: one warp searches each vector's whole tree
                                     (no subtree splitting between warps), so visited-node
                                     counts are those of the sequential search */
  MDX_COMPLEX_TREE = 1 << 6,      /* detect_sd / detect_kbest: search the complex tree of
                                     Sec. III-B (one level per complex antenna, the QAM
                                     alphabet's qam points as children; on the interleaved
                                     real R a level is the real rows 2j+1 and 2j, i.e. the
                                     real tree grouped two levels at a time).  Children in
                                     increasing partial distance, ties to the lower index
                                     q; K-best keeps K per complex level.  stats count
                                     complex-level nodes and qam children per node.
                                     detect_sd runs it one warp per vector (no splitting). */
  MDX_LINEAR_MMSE = 1 << 8,       /* detect_linear: MMSE instead of zero forcing */
  MDX_ORDER_NATURAL = 1 << 7,     /* detect_sd: visit children in natural index order instead
                                     of Schnorr-Euchner order (the unsorted depth-first
                                     search of Sec. IV-A, a control); one warp per vector */
  MDX_LEARNED_ORDER = 1 << 5      /* detect_sd: the MLP's per-row child ranking (mdx_mlp_load)
                                     proposes the first leaf x^ (the top-ranked PAM index
                                     of every real row, ties to the lower index); the
                                     search treats x^ as its first descent, i.e. the
                                     initial r^2 is capped at ||ybar - R x^||^2 (FP32)
                                     x (1 + 2^-16).  Exactness is unchanged: x^ is a
                                     lattice point, so the cap is at least d_ML. */
};

/* Largest sizes the kernels support. */
#define MDX_MAX_TX 100   /* n_tx (real tree depth 2*n_tx <= 200) */
#define MDX_MAX_RX 128
#define MDX_MAX_K 256

typedef struct {
  int n_rx;              /* N >= n_tx */
  int n_tx;              /* M, 1 <= M <= MDX_MAX_TX */
  int qam;               /* 4, 16 or 64 */
  double init_radius_sq; /* initial squared radius r^2 of the sphere (Sec. III-B):
                            INFINITY = no radius; < 0 = the paper's r^2 = N M sigma^2
                            (per vector, from noise_var); > 0 = this value */
  int K;                 /* survivors kept per level, 1 <= K <= MDX_MAX_K
                            (detect_kbest, detect_hybrid) */
  int hybrid_depth;      /* real rows explored by the hybrid's SD master (Sec. VI),
                            0..min(2 n_tx, 12) with sqrt(qam)^depth <= 4096 */
  long long node_budget; /* per-vector budget of branched nodes (detect_sd,
                            detect_hybrid); 0 = none.  detect_sd: an exact cap
                            (a budgeted search keeps each vector's tree in one
                            worker, without subtree splitting); detect_hybrid:
                            the vector stops once a finished prefix run brings
                            its count to the budget, so the runs in flight may
                            pass it */
  int flags;             /* MDX_* flags above */
} mdx_params;

/* Context: selects `device`, allocates the workspace for up to max_batch
 * vectors of at most max_n_rx x max_n_tx (QR outputs, candidate buffers and
 * host-staging buffers).  No later call allocates device memory.
 * Returns MDX_ENOMEM if the workspace does not fit. */
mdx_status mdx_create(mdx_ctx** ctx, int device, int max_batch, int max_n_rx, int max_n_tx);
mdx_status mdx_destroy(mdx_ctx* ctx);
const char* mdx_strerror(mdx_status s);
const char* mdx_last_error(const mdx_ctx* ctx);
/* Bytes of device workspace this context holds. */
size_t mdx_workspace_bytes(const mdx_ctx* ctx);

/* QR preprocessing alone (Sec. III-B): H = Q R with a real positive diagonal,
 * ybar = Q^H y, both returned in the real interleaved form of size n = 2 n_tx.
 *   R_out    double [batch][n][n], row-major, zero below the diagonal
 *   ybar_out double [batch][n]
 * Computed in FP64 (complex Householder reflections). */
mdx_status mdx_qr(mdx_ctx* ctx, int batch, int n_rx, int n_tx, const double* H, const double* y,
                  double* R_out, double* ybar_out, int flags, void* stream);

/* Exact sphere decoder (Sec. III-B, Algorithm 1) with the Best-FS /
 * Schnorr-Euchner order (Sec. IV-A) and incremental partial distances
 * (Sec. IV-C, Eq. inc): depth-first, children visited in increasing partial
 * distance, a child is pruned when its partial distance is >= r^2, and every
 * leaf reached shrinks r^2 to its distance.  Partial distances are FP32 with
 * a small pruning slack; the final leaf candidates are re-scored in FP64, so
 * the answer is the maximum-likelihood point of Eq. 2 (up to FP64 ties).
 * Uses p->init_radius_sq, p->node_budget, p->flags. */
mdx_status detect_sd(mdx_ctx* ctx, const mdx_params* p, int batch, const double* H,
                     const double* y, const double* noise_var, uint8_t* sym_out,
                     double* metric_out, int32_t* vstatus, int64_t* stats, void* stream);

/* K-best (Sec. VI): breadth-first; at every row all children of the
 * surviving nodes are evaluated and the K with the smallest partial distance
 * (among those inside the radius, if one is given) survive; the best final
 * leaf is returned.  FP32 partial distances, FP64 re-scoring of the final
 * candidates.  Uses p->K, p->init_radius_sq, p->flags. */
mdx_status detect_kbest(mdx_ctx* ctx, const mdx_params* p, int batch, const double* H,
                        const double* y, const double* noise_var, uint8_t* sym_out,
                        double* metric_out, int32_t* vstatus, int64_t* stats, void* stream);

/* Hybrid SD / K-best (Sec. VI): a Best-FS sphere decoder explores the top
 * p->hybrid_depth rows; every node it reaches at that depth inside the
 * current sphere is finished by a K-best(p->K) worker that prunes with the
 * shared, shrinking radius, stops when all its survivors leave the sphere and
 * shrinks the radius with its best leaf.  The result equals the best K-best
 * leaf over all depth-d prefixes inside the initial sphere, independent of the
 * order in which workers take them.  Uses p->K, p->hybrid_depth,
 * p->init_radius_sq, p->node_budget, p->flags. */
mdx_status detect_hybrid(mdx_ctx* ctx, const mdx_params* p, int batch, const double* H,
                         const double* y, const double* noise_var, uint8_t* sym_out,
                         double* metric_out, int32_t* vstatus, int64_t* stats, void* stream);
/* Linear detection, the controls of Sec. III-A: zero forcing
 * x = H^+ y = R^-1 ybar (back substitution on the FP64 QR), or with
 * MDX_LINEAR_MMSE in p->flags, x = (H^H H + sigma^2 I)^-1 H^H y
 * (regularised normal equations, Cholesky; needs noise_var; n_tx <= 32).
 * Every real component is sliced to the nearest PAM level (clipped); the
 * outputs are as for detect_sd (metric ||ybar - R x^||^2 in FP64, stats
 * zero except rescored = 1).  K, radius, depth and budget are ignored. */
mdx_status detect_linear(mdx_ctx* ctx, const mdx_params* p, int batch, const double* H, const double* y,
                         const double* noise_var, uint8_t* sym_out, double* metric_out, int32_t* vstatus,
                         int64_t* stats, void* stream);

/* ---------------------------------------------------------------------------
 * Uneven batches: one call detects many requests that differ in antennas,
 * modulation, detector and K.  (The paper detects one system at a time; this
 * is the batching layer around its detectors.)  Request r reads H at
 * H + reqs[r].h_offset (double [n_rx][n_tx][2]), y at y + reqs[r].y_offset
 * (double [n_rx][2]) and noise_var[r], and writes sym_out + reqs[r].sym_offset
 * (uint8 [n_tx]), metric_out[r], vstatus[r], stats[r][5].  `reqs` is a HOST
 * array; every other pointer is device memory.  The QR runs per (n_rx, n_tx)
 * class; the search is one persistent kernel whose warps take requests from a
 * global counter, heaviest classes first: exact SD (Algorithm 1, one warp per
 * request, node_budget honoured; real or complex tree) or K-best (Sec. VI,
 * tournament selection),
 * with R and the search state in a per-warp shared-memory slice, or in a
 * per-warp global-memory slot for requests too large for the slice.  The slice
 * size and warps per CTA come from the context's tuning table
 * (mdx_autotune_mixed) or a default.  With MDX_GRAPH in flags the launch
 * sequence is captured into a CUDA graph on the first call and replayed by
 * later calls with the same request table and pointers (the table must not
 * change between such calls).
 * Limits: n_tx <= MDX_MAX_TX, K <= MDX_MAX_K, nreq <= the context's max_batch
 * and the sum of per-request QR outputs within the workspace. */
enum {
  MDX_ALGO_SD = 0,
  MDX_ALGO_KBEST = 1,
  MDX_ALGO_SD_COMPLEX = 2, /* complex-tree SD, as MDX_COMPLEX_TREE */
  MDX_ALGO_SD_NATURAL = 3  /* natural-order SD, as MDX_ORDER_NATURAL */
};
enum { MDX_GRAPH = 1 << 4 };
typedef struct {
  int n_rx, n_tx, qam;
  int algo;               /* MDX_ALGO_SD or MDX_ALGO_KBEST */
  int K;                  /* K-best survivors */
  int pad;
  double init_radius_sq;  /* as in mdx_params */
  long long node_budget;  /* exact SD: cap on branched nodes, 0 = none */
  long long h_offset;     /* in doubles */
  long long y_offset;     /* in doubles */
  long long sym_offset;   /* in symbols */
} mdx_request;
mdx_status detect_mixed(mdx_ctx* ctx, int nreq, const mdx_request* reqs, const double* H, const double* y,
                        const double* noise_var, uint8_t* sym_out, double* metric_out, int32_t* vstatus,
                        int64_t* stats, int flags, void* stream);
/* Tune the persistent kernel for a request table: times detect_mixed on the
 * given (device) inputs for each candidate (warps per CTA, shared-memory
 * slice) and keeps the fastest in the context; results[0..2] = chosen warps,
 * slice bytes, milliseconds.  Outputs are overwritten during tuning. */
mdx_status mdx_autotune_mixed(mdx_ctx* ctx, int nreq, const mdx_request* reqs, const double* H, const double* y,
                              const double* noise_var, uint8_t* sym_out, double* metric_out, int32_t* vstatus,
                              double* results, void* stream);

/* Bit and symbol errors of detected against transmitted indices (the error
 * rates plotted in Sec. VII), with a Gray code per PAM dimension of
 * q = k_re*P + k_im.  counts_out int64[2] = {bit errors, symbol errors},
 * overwritten (not accumulated). */
mdx_status mdx_count_errors(mdx_ctx* ctx, int batch, int n_tx, int qam, const uint8_t* sym_hat,
                            const uint8_t* sym_true, int64_t* counts_out, int flags,
                            void* stream);

/* ---------------------------------------------------------------------------
 * Learned initial radius (the paper has no learned component; its radius is
 * the fixed r^2 = N M sigma^2 of Sec. III-B).  A multilayer perceptron with
 * two hidden layers of 256 ReLU units reads, per received vector,
 *   x = [R upper triangle in column-packed order (entry (r, c), r <= c, at
 *        c (c + 1) / 2 + r), ybar, SNR_dB / 30]  (zero-padded to d_in)
 * and outputs o (d_out values, zero-padded): o[0] predicts
 * log(d_ML / sigma^2), trained with a pinball loss at the 0.9 quantile so
 * that the radius r^2 = sigma^2 exp(o[0]) usually contains the ML point;
 * o[1 + r P + k] are logits that real row r of the ML point has PAM index k
 * (cross-entropy, weight 0.2).  Weights are BF16, accumulation FP32, on the
 * tensor cores (tcgen05); FP32 master weights and Adam moments are kept on
 * the device.  detect_sd with MDX_LEARNED_RADIUS starts from the predicted
 * radius and doubles it on an empty sphere, so its answer is unchanged;
 * with MDX_LEARNED_ORDER the logits' top-ranked leaf caps that radius.
 * Parameter vector (FP32, this order): W1 [256][d_in], b1 [256],
 * W2 [256][256], b2 [256], W3 [d_out][256], b3 [d_out].
 * Models are for square systems n_rx = n_tx.  Above n_tx = 32 the input is a
 * summary of the system instead (d_in = round_up(n + 3, 64), d_out = 128):
 * [log R_ii (n), log(d_B / sigma^2) / 10 with d_B the distance of the
 * Babai point, log(||ybar||^2 / (n sigma^2)) / 10, SNR_dB / 30]; such a
 * model has the radius head only (trained on any detector's answer metric,
 * e.g. the hybrid's) and serves MDX_LEARNED_RADIUS in detect_sd and
 * detect_hybrid (whose answer is likewise unchanged: a radius below the
 * answer's distance empties the sphere and is doubled). */
size_t mdx_mlp_param_count(int n_tx, int qam);
mdx_status mdx_mlp_dims(int n_tx, int qam, int* d_in, int* d_out);
/* Create (or replace) the context's model for n_tx x n_tx, qam, with a
 * training workspace for batches of up to max_train_batch vectors, weights
 * drawn He-uniform from `seed`.  Allocates device memory (model, moments,
 * activations for max(max_batch, max_train_batch) rows). */
mdx_status mdx_mlp_init(mdx_ctx* ctx, int n_tx, int qam, int max_train_batch, unsigned long long seed);
/* Copy the FP32 parameter vector from / to HOST memory (count values). */
mdx_status mdx_mlp_set_params(mdx_ctx* ctx, const float* params, size_t count);
mdx_status mdx_mlp_get_params(mdx_ctx* ctx, float* params, size_t count);
/* QR + features + forward pass for `batch` vectors (device pointers, layouts
 * as for detect_*): out float [batch][d_out]; feat_out float [batch][d_in]
 * (the features before BF16 rounding) or NULL. */
mdx_status mdx_mlp_predict(mdx_ctx* ctx, const mdx_params* p, int batch, const double* H, const double* y,
                           const double* noise_var, float* out, float* feat_out, void* stream);
/* One training step on `batch` vectors with their targets (ml_sym
 * uint8 [batch][n_tx] and ml_metric double [batch], as returned by
 * detect_sd; ml_sym may be NULL for a summary model, whose target is the
 * metric alone): forward, loss, backward on the tensor cores; if `update`,
 * one Adam step with learning rate lr (beta 0.9 / 0.999).  grad_out float
 * [param_count] receives the gradient and loss_out float [2] the batch's
 * (pinball, cross-entropy) losses; both device pointers or NULL. */
mdx_status mdx_mlp_train_step(mdx_ctx* ctx, const mdx_params* p, int batch, const double* H, const double* y,
                              const double* noise_var, const uint8_t* ml_sym, const double* ml_metric, float lr,
                              int update, float* grad_out, float* loss_out, void* stream);
/* Waits for the device and reports whether a bounded wait inside a model
 * kernel expired (*err_out != 0). */
mdx_status mdx_mlp_error(mdx_ctx* ctx, int* err_out);

/* K-best detection for callers that may not allocate device memory.
 * (The paper has no counterpart; this is a deployment variant of
 * detect_kbest.)  Some callers cannot allocate once they are running: a
 * real-time receiver that fixes its memory at start-up, or a process whose
 * device memory is held by another allocator.  They cannot create an
 * mdx_ctx, which allocates its workspace.  This entry point takes no
 * context and allocates nothing: it computes exactly what detect_kbest
 * computes (same kernels, same outputs), on the current device, with its
 * scratch (QR outputs, flags, work counter) in one static device array of
 * MDX_NOALLOC_SCRATCH_BYTES that the library reserves on every GPU it is
 * loaded on until the process exits.
 *   - Device pointers only; arguments as for detect_kbest.  The flags
 *     detect_kbest rejects (MDX_LEARNED_RADIUS, MDX_LEARNED_ORDER,
 *     MDX_ORDER_NATURAL) and MDX_HOST_BUFFERS return MDX_EUNSUPPORTED, as do
 *     K and sizes whose shared memory detect_kbest would refuse.
 *   - A batch whose scratch exceeds the array returns MDX_EUNSUPPORTED
 *     (about 6.7 KB per vector at 16x16, 243 KB at 100x100).
 *   - All calls share the array and it keeps the last call's contents; the
 *     call clears what must start at zero itself.  Calls whose work
 *     overlaps on the GPU (other streams, other host threads) race:
 *     serialise them on one stream.
 *   - The first call on each device looks up the array's address with that
 *     device current; make that first call before any stream capture.  The
 *     address is kept until the process exits: resetting the device
 *     (cudaDeviceReset) between calls is not supported.
 * Errors are reported by the return value only (there is no context). */
#define MDX_NOALLOC_SCRATCH_BYTES (16u << 20)
mdx_status detect_kbest_noalloc(const mdx_params* p, int batch, const double* H, const double* y,
                                const double* noise_var, uint8_t* sym_out, double* metric_out,
                                int32_t* vstatus, int64_t* stats, void* stream);

/* Kernel timing for benchmarks.  While enabled, every call records CUDA
 * events on its stream around the QR kernel and the search kernel (up to
 * 1024 calls are kept; with MDX_HOST_BUFFERS the QR interval includes the
 * wait for the staged inputs).  mdx_profile_read waits for those events, writes
 * ms_out[0] = summed QR time, ms_out[1] = summed search time (milliseconds),
 * ms_out[2] = number of calls recorded, ms_out[3] = the error word of the
 * last detect_sd launch (non-zero if a bounded wait inside it expired),
 * ms_out[4..7] = that launch's subtree-splitting counters (checks that saw
 * idle warps, checks that donated, tasks donated, checks with no level to
 * split), and clears the record.  ms_out must hold 8 doubles.  Not part of
 * the detection path; enable = 0 turns it off. */
mdx_status mdx_profile(mdx_ctx* ctx, int enable);
mdx_status mdx_profile_read(mdx_ctx* ctx, double* ms_out);

/* Arithmetic-throughput probes for roofline denominators (not part of the
 * detection path; the paper has none).  Runs three short kernels on
 * `device` (about 40 ms in all, on `stream`, synchronously) filling every SM:
 *   out[0] = FP32 FMA throughput, TFLOP/s (8 independent FFMA chains per
 *            thread; the unit of the tree searches' partial distances),
 *   out[1] = FP64 FMA throughput, TFLOP/s (8 DFMA chains per thread; the
 *            QR's panel),
 *   out[2] = FP64 mma.sync m8n8k4 throughput, TFLOP/s, with the A and B
 *            operand values changed before every MMA (the QR's trailing
 *            updates),
 *   out[3] = milliseconds the three timed launches took.
 * An FMA counts as 2 flops.  Allocates and frees a small device buffer.
 * Returns MDX_EINVAL for a bad device or NULL out, MDX_ECUDA on a CUDA error. */
mdx_status mdx_measure_peaks(int device, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
