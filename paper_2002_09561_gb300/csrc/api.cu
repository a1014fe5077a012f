// C ABI of libmdx (include/mimo_detect.h): context and workspace, argument
// checks, host staging, and the launch sequence QR -> search -> FP64
// re-scoring of every detect_* call.  Also the Gray-coded error counter.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "mdx_internal.cuh"

struct mdx_ctx {
  int device = 0;
  int num_sms = 0;
  int max_batch = 0, max_rx = 0, max_tx = 0;
  size_t bytes = 0;
  // QR outputs and search scratch
  double* R64 = nullptr;
  double* yb64 = nullptr;
  float* R32 = nullptr;
  float* yb32 = nullptr;
  int* singular = nullptr;
  unsigned int* counter = nullptr;
  unsigned long long* counts = nullptr;
  // sphere-decoder task queue
  void* sd_shared = nullptr;
  void* sd_queue = nullptr;
  unsigned char* sd_vstate = nullptr;
  int* sd_order = nullptr;
  unsigned long long sd_epoch = 0;
  // learned radius model (mdx_mlp_init), null until created
  mdx::MlpState* mlp = nullptr;
  // staging for MDX_HOST_BUFFERS
  double* sH = nullptr;
  double* sy = nullptr;
  double* snv = nullptr;
  uint8_t* ssym = nullptr;
  uint8_t* ssym2 = nullptr;
  double* smet = nullptr;
  int32_t* svst = nullptr;
  int64_t* sstats = nullptr;
  // host inputs are copied on this stream in up to kHostChunks chunks, each
  // followed by an event the QR of that chunk waits for (see run_detect)
  static constexpr int kHostChunks = 8;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_free = nullptr;
  cudaEvent_t ev_chunk[kHostChunks] = {};
  // uneven batches (detect_mixed): the uploaded request table and its device
  // descriptors [MixedReq x n | order x n | QR ids x n], the QR class runs
  // (n_rx, n_tx, first id, count), per-warp global state slots, the tuning
  // (warps per CTA, shared-memory slice per warp, placement per request
  // class) and the captured graph with the arguments it was captured for
  std::vector<mdx_request> mx_table;
  unsigned long long mx_gen = 0;  // bumped whenever descriptors or tuning change
  unsigned char* mx_dev = nullptr;
  size_t mx_dev_bytes = 0;
  unsigned char* mx_pinned = nullptr;
  size_t mx_pinned_bytes = 0;
  std::vector<int> mx_qr;  // 4 ints per class run
  int mx_maxK = 0;
  size_t mx_gslot = 16;
  unsigned char* mx_scratch = nullptr;
  size_t mx_scratch_bytes = 0;
  int mx_W = 8, mx_slice = 12288;
  std::vector<std::pair<unsigned long long, int>> mx_modes;  // class key -> MIX_* bits
  cudaGraphExec_t mx_graph = nullptr;
  std::vector<const void*> mx_graph_key;
  // optional kernel timing (mdx_profile)
  static constexpr int kProfSlots = 1024;
  bool prof = false;
  int prof_n = 0;
  cudaEvent_t prof_ev[kProfSlots][3] = {};
  char err[320] = {0};
};

namespace {

using namespace mdx;

mdx_status fail(mdx_ctx* c, mdx_status s, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

mdx_status cuda_fail(mdx_ctx* c, cudaError_t e, const char* where) {
  return fail(c, MDX_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Switches to the context's device for the lifetime of the guard.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int pam_of(int qam) {
  switch (qam) {
    case 4: return 2;
    case 16: return 4;
    case 64: return 8;
    default: return -1;
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// True when p is memory the device can address (device or managed memory).
bool is_device_ptr(const void* p, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == device;
}

template <typename T>
cudaError_t alloc(mdx_ctx* c, T** p, size_t count) {
  const size_t b = sizeof(T) * (count ? count : 1);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), b);
  if (e == cudaSuccess) c->bytes += b;
  return e;
}

void free_all(mdx_ctx* c) {
  if (c->mlp) {
    mlp_free(c->mlp);
    c->mlp = nullptr;
  }
  for (int i = 0; i < mdx_ctx::kProfSlots; ++i)
    for (int k = 0; k < 3; ++k)
      if (c->prof_ev[i][k]) cudaEventDestroy(c->prof_ev[i][k]);
  void* ptrs[] = {c->R64, c->yb64, c->R32,  c->yb32, c->singular, c->counter,  c->counts,
                  c->sH,  c->sy,   c->snv,  c->ssym, c->ssym2,    c->smet,     c->svst,
                  c->sstats, c->sd_shared, c->sd_queue, c->sd_vstate, c->sd_order};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->mx_graph) cudaGraphExecDestroy(c->mx_graph);
  if (c->mx_dev) cudaFree(c->mx_dev);
  if (c->mx_scratch) cudaFree(c->mx_scratch);
  if (c->mx_pinned) cudaFreeHost(c->mx_pinned);
  for (cudaEvent_t ev : c->ev_chunk)
    if (ev) cudaEventDestroy(ev);
  if (c->ev_free) cudaEventDestroy(c->ev_free);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
}

enum Algo { ALGO_SD = 0, ALGO_KBEST = 1, ALGO_HYBRID = 2, ALGO_LINEAR = 3 };

// Task-queue slots of the sphere decoder (tasks exist only while warps are idle).
constexpr unsigned int kSdQueueSlots = 1u << 16;

mdx_status run_detect(int algo, mdx_ctx* c, const mdx_params* p, int batch, const double* H,
                      const double* y, const double* nv, uint8_t* sym, double* met, int32_t* vst,
                      int64_t* stats, void* stream) {
  if (!c) return MDX_EINVAL;
  if (!p) return fail(c, MDX_EINVAL, "params is NULL");
  if (batch < 0) return fail(c, MDX_EINVAL, "batch %d < 0", batch);
  if (batch == 0) return MDX_OK;
  if (batch > c->max_batch)
    return fail(c, MDX_EUNSUPPORTED, "batch %d > context max_batch %d", batch, c->max_batch);
  const int M = p->n_tx, N = p->n_rx, P = pam_of(p->qam);
  if (M < 1 || N < M) return fail(c, MDX_EINVAL, "need n_rx >= n_tx >= 1 (got %d, %d)", N, M);
  if (M > c->max_tx || N > c->max_rx)
    return fail(c, MDX_EUNSUPPORTED, "%dx%d exceeds the context's %dx%d", N, M, c->max_rx, c->max_tx);
  if (P < 0) return fail(c, MDX_EINVAL, "qam %d not in {4, 16, 64}", p->qam);
  const int n = 2 * M;
  const double r0 = p->init_radius_sq;
  if (isnan(r0) || r0 == 0.0) return fail(c, MDX_EINVAL, "init_radius_sq must be > 0, < 0 or INFINITY");
  int radius_mode = isinf(r0) ? (r0 > 0 ? RADIUS_NONE : RADIUS_PAPER) : (r0 < 0 ? RADIUS_PAPER : RADIUS_VALUE);
  const bool learned = (p->flags & MDX_LEARNED_RADIUS) != 0;
  const bool order = (p->flags & MDX_LEARNED_ORDER) != 0;
  if (learned || order) {
    if (algo != ALGO_SD && !(algo == ALGO_HYBRID && !order))
      return fail(c, MDX_EUNSUPPORTED, "MDX_LEARNED_RADIUS applies to detect_sd and detect_hybrid, "
                                      "MDX_LEARNED_ORDER to detect_sd");
    if (!c->mlp || mlp_ntx(c->mlp) != M || mlp_qam(c->mlp) != p->qam || N != M)
      return fail(c, MDX_EUNSUPPORTED, "the learned radius / order needs a model for this %dx%d %d-QAM (mdx_mlp_init)",
                  N, M, p->qam);
    if (!nv) return fail(c, MDX_EINVAL, "noise_var needed for the learned radius / order (network input)");
    if (order && mlp_reduced(c->mlp))
      return fail(c, MDX_EUNSUPPORTED, "MDX_LEARNED_ORDER needs a model with the ordering head (n_tx <= %d)",
                  kFullFeaturesMaxTx);
  }
  if (p->node_budget < 0) return fail(c, MDX_EINVAL, "node_budget < 0");
  const bool mmse = (p->flags & MDX_LINEAR_MMSE) != 0;
  if (algo == ALGO_LINEAR) {
    if (mmse && !nv) return fail(c, MDX_EINVAL, "noise_var needed for MMSE");
    if ((mmse && M > 32) || linear_smem_bytes(n, mmse) > 227 * 1024)
      return fail(c, MDX_EUNSUPPORTED, "MMSE supports n_tx <= 32 (got %d)", M);
  }
  if (algo != ALGO_SD && algo != ALGO_LINEAR) {
    if (p->K < 1 || p->K > MDX_MAX_K) return fail(c, MDX_EINVAL, "K %d not in 1..%d", p->K, MDX_MAX_K);
  }
  const bool complex_tree = (p->flags & MDX_COMPLEX_TREE) != 0;
  const bool natural = (p->flags & MDX_ORDER_NATURAL) != 0;
  if (complex_tree && algo == ALGO_HYBRID) return fail(c, MDX_EUNSUPPORTED, "MDX_COMPLEX_TREE applies to SD and K-best");
  if (natural && (algo != ALGO_SD || complex_tree))
    return fail(c, MDX_EUNSUPPORTED, "MDX_ORDER_NATURAL applies to detect_sd on the real tree");
  if (algo == ALGO_HYBRID) {
    const int d = p->hybrid_depth;
    if (d < 0 || d > n || d > 12) return fail(c, MDX_EINVAL, "hybrid_depth %d not in 0..min(n, 12)", d);
    long long np = 1;
    for (int l = 0; l < d; ++l) np *= P;
    if (np > 4096) return fail(c, MDX_EUNSUPPORTED, "P^depth = %lld > 4096 prefixes", np);
  }
  if (algo == ALGO_KBEST && kbest_smem_bytes(n, p->K, P, complex_tree) > 227 * 1024)
    return fail(c, MDX_EUNSUPPORTED, "K=%d at n=%d, P=%d needs more than 227 KB of shared memory", p->K,
                n, P);
  if (algo == ALGO_HYBRID && hybrid_smem_bytes(n, p->K, P, p->hybrid_depth) == (size_t)-1)
    return fail(c, MDX_EUNSUPPORTED, "hybrid K=%d at n=%d, P=%d, depth %d does not fit in shared memory", p->K, n,
                P, p->hybrid_depth);
  const bool host = (p->flags & MDX_HOST_BUFFERS) != 0;
  if (!H || !y || !sym || !met || !vst) return fail(c, MDX_EINVAL, "NULL input or output pointer");
  if (radius_mode == RADIUS_PAPER && !nv) return fail(c, MDX_EINVAL, "noise_var needed for the paper radius");
  if (!host) {
    if (!aligned16(H) || !aligned16(y)) return fail(c, MDX_EINVAL, "H and y must be 16-byte aligned");
    const void* ptrs[] = {H, y, sym, met, vst};
    for (const void* q : ptrs)
      if (!is_device_ptr(q, c->device))
        return fail(c, MDX_EINVAL, "pointer %p is not device memory of device %d", q, c->device);
    if (nv && !is_device_ptr(nv, c->device)) return fail(c, MDX_EINVAL, "noise_var is not device memory");
    if (stats && !is_device_ptr(stats, c->device)) return fail(c, MDX_EINVAL, "stats is not device memory");
  }

  DeviceGuard g(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "earlier asynchronous error");

  const double* dH = H;
  const double* dy = y;
  const double* dnv = nv;
  uint8_t* dsym = sym;
  double* dmet = met;
  int32_t* dvst = vst;
  int64_t* dstats = stats;
  // Host inputs: copied on the context's copy stream in chunks of at least
  // 32 MB, each chunk's QR waiting on the caller's stream for that chunk
  // only, so that the copy of chunk j + 1 overlaps the QR of chunk j.  The
  // copy stream first waits for everything already queued on the caller's
  // stream (an earlier call may still read the staging buffers).
  const size_t h_bytes = sizeof(double) * 2 * (size_t)batch * N * M;
  const int chunks = host ? (int)std::min<size_t>(mdx_ctx::kHostChunks,
                                                  std::max<size_t>(1, h_bytes / ((size_t)32 << 20)))
                          : 1;
  auto chunk_begin = [&](int j) { return (int)((long long)batch * j / chunks); };
  if (host) {
    cudaStream_t cs = c->copy_stream;
    e = cudaEventRecord(c->ev_free, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, c->ev_free, 0);
    if (e == cudaSuccess && nv)
      e = cudaMemcpyAsync(c->snv, nv, sizeof(double) * batch, cudaMemcpyHostToDevice, cs);
    for (int j = 0; j < chunks && e == cudaSuccess; ++j) {
      const size_t b0 = (size_t)chunk_begin(j), nb = (size_t)chunk_begin(j + 1) - b0;
      e = cudaMemcpyAsync(c->sH + b0 * 2 * N * M, H + b0 * 2 * N * M, sizeof(double) * 2 * nb * N * M,
                          cudaMemcpyHostToDevice, cs);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->sy + b0 * 2 * N, y + b0 * 2 * N, sizeof(double) * 2 * nb * N, cudaMemcpyHostToDevice,
                            cs);
      if (e == cudaSuccess) e = cudaEventRecord(c->ev_chunk[j], cs);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device staging");
    dH = c->sH;
    dy = c->sy;
    dnv = nv ? c->snv : nullptr;
    dsym = c->ssym;
    dmet = c->smet;
    dvst = c->svst;
    dstats = stats ? c->sstats : nullptr;
  }

  cudaEvent_t* ev = nullptr;
  if (c->prof && c->prof_n < mdx_ctx::kProfSlots) {
    ev = c->prof_ev[c->prof_n++];
    cudaEventRecord(ev[0], s);
  }
  for (int j = 0; j < chunks; ++j) {
    const int b0 = chunk_begin(j), nb = chunk_begin(j + 1) - b0;
    if (host) {
      e = cudaStreamWaitEvent(s, c->ev_chunk[j], 0);
      if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device staging");
    }
    QrOut q{c->R64 + (size_t)b0 * tri_stride64(n), c->yb64 + (size_t)b0 * vec_stride64(n),
            c->R32 + (size_t)b0 * tri_stride32(n), c->yb32 + (size_t)b0 * vec_stride32(n),
            nullptr, nullptr, c->singular + b0};
    e = launch_qr(nb, N, M, dH + (size_t)b0 * 2 * N * M, dy + (size_t)b0 * 2 * N, q, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "QR launch");
  }

  if (learned || order) {
    // radius proposed by the network (r^2 = sigma^2 exp(o_0)) and/or capped by
    // the distance of its top-ranked leaf
    const int rows = round_up(batch, 128);
    e = mlp_features(c->mlp, batch, rows, c->R32, c->yb32, dnv, false, nullptr, s);
    if (e == cudaSuccess) e = mlp_forward(c->mlp, rows, false, s);
    if (e == cudaSuccess)
      e = mlp_radius(c->mlp, batch, dnv, learned, order, radius_mode, r0, N, c->R32, c->yb32, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "learned radius");
    radius_mode = RADIUS_PER_VECTOR;
  }
  SearchArgs a{};
  a.batch = batch;
  a.n = n;
  a.P = P;
  a.n_rx = N;
  a.n_tx = M;
  a.alpha64 = sqrt(3.0 / (2.0 * (p->qam - 1)));
  a.alpha = (float)a.alpha64;
  a.R32 = c->R32;
  a.yb32 = c->yb32;
  a.R64 = c->R64;
  a.yb64 = c->yb64;
  a.singular = c->singular;
  a.noise_var = dnv;
  a.r2_vec = (learned || order) ? mlp_r2(c->mlp) : nullptr;
  a.radius_mode = radius_mode;
  a.radius_value = r0;
  a.K = p->K;
  a.depth = p->hybrid_depth;
  a.budget = p->node_budget;
  a.flags = p->flags;
  a.work_counter = c->counter;
  a.sym_out = dsym;
  a.metric_out = dmet;
  a.vstatus = dvst;
  a.stats = dstats;
  e = cudaMemsetAsync(c->counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return cuda_fail(c, e, "work counter reset");
  if (algo == ALGO_SD && (complex_tree || natural)) {
    // complex-tree or natural-order SD: the persistent warp-per-vector kernel on a uniform batch
    const int malgo = complex_tree ? MIX_ALGO_SD_COMPLEX : MIX_ALGO_SD_NATURAL;
    MixedArgs m{};
    m.nreq = batch;
    m.uniform.n_rx = N;
    m.uniform.n_tx = M;
    m.uniform.n = n;
    m.uniform.P = P;
    m.uniform.algo = malgo;
    m.uniform.mode = mixed_greedy_mode(malgo, n, 0, P, c->mx_slice);
    m.uniform.radius_mode = radius_mode;
    m.uniform.radius_value = r0;
    m.uniform.alpha = a.alpha;
    m.uniform.alpha64 = a.alpha64;
    m.uniform.budget = p->node_budget;
    m.r2_vec = a.r2_vec;
    m.R32 = c->R32;
    m.yb32 = c->yb32;
    m.R64 = c->R64;
    m.yb64 = c->yb64;
    m.singular = c->singular;
    m.noise_var = dnv;
    m.counter = c->counter;
    m.slice_bytes = c->mx_slice;
    m.flags = p->flags;
    m.sym_out = dsym;
    m.metric_out = dmet;
    m.vstatus = dvst;
    m.stats = dstats;
    m.gslot_bytes = (m.uniform.mode & MIX_STATE_SMEM) ? 16 : mixed_state_bytes(malgo, n, 0, P);
    const int warps = mixed_resident_warps(c->mx_W, c->mx_slice, 0, c->num_sms);
    if (warps < 1) return fail(c, MDX_EUNSUPPORTED, "no launch configuration fits this size");
    const size_t sbytes = (size_t)warps * m.gslot_bytes;
    if (c->mx_scratch_bytes < sbytes) {
      // per-warp search state, allocated once on first use and kept
      if (c->mx_graph) {
        cudaGraphExecDestroy(c->mx_graph);
        c->mx_graph = nullptr;
      }
      cudaStreamSynchronize(s);
      if (c->mx_scratch) cudaFree(c->mx_scratch);
      c->mx_scratch = nullptr;
      c->mx_scratch_bytes = 0;
      e = cudaMalloc(reinterpret_cast<void**>(&c->mx_scratch), sbytes);
      if (e != cudaSuccess) return fail(c, MDX_ENOMEM, "%zu bytes of per-warp search state", sbytes);
      c->mx_scratch_bytes = sbytes;
    }
    m.gscratch = c->mx_scratch;
    if (ev) cudaEventRecord(ev[1], s);
    e = launch_mixed(m, c->mx_W, 0, c->num_sms, s);
  } else if (algo == ALGO_SD) {
    if (ev) cudaEventRecord(ev[1], s);
    SdWorkspace w{c->sd_shared, c->sd_queue, kSdQueueSlots, c->sd_vstate, ++c->sd_epoch, c->sd_order};
    e = launch_sd(a, w, c->num_sms, s);
  }
  else if (algo == ALGO_KBEST) {
    if (ev) cudaEventRecord(ev[1], s);
    e = launch_kbest(a, c->num_sms, s);
  } else if (algo == ALGO_LINEAR) {
    if (ev) cudaEventRecord(ev[1], s);
    e = launch_linear(a, mmse, c->num_sms, s);
  } else {
    if (ev) cudaEventRecord(ev[1], s);
    e = launch_hybrid(a, c->num_sms, s);
  }
  if (e == cudaErrorInvalidConfiguration)
    return fail(c, MDX_EUNSUPPORTED, "no launch configuration fits this size");
  if (e != cudaSuccess) return cuda_fail(c, e, "search launch");
  if (ev) cudaEventRecord(ev[2], s);

  if (host) {
    e = cudaMemcpyAsync(sym, c->ssym, (size_t)batch * M, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(met, c->smet, sizeof(double) * batch, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vst, c->svst, sizeof(int32_t) * batch, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && stats)
      e = cudaMemcpyAsync(stats, c->sstats, sizeof(int64_t) * kStats * (size_t)batch, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host results");
  }
  return MDX_OK;
}

// ---------------------------------------------------------------------------
// Uneven batches.

unsigned long long class_key(const mdx_request& q) {
  return (unsigned long long)q.n_rx | ((unsigned long long)q.n_tx << 8) | ((unsigned long long)q.qam << 16) |
         ((unsigned long long)q.algo << 24) | ((unsigned long long)(q.algo == MDX_ALGO_KBEST ? q.K : 0) << 32);
}

bool mode_fits(int mode, int algo, int n, int K, int slice) {
  size_t need = 0;
  if (mode & MIX_STAGE_R) need += mixed_stage_bytes(n);
  if (mode & MIX_STATE_SMEM) need += mixed_state_bytes(algo, n, K, 0);
  return need <= (size_t)slice;
}

// Most shared-memory use that fits: everything, else the state, else R.
int greedy_mode(int algo, int n, int K, int slice) { return mixed_greedy_mode(algo, n, K, 0, slice); }

int mode_for(const mdx_ctx* c, const mdx_request& q) {
  const int n = 2 * q.n_tx;
  const unsigned long long k = class_key(q);
  for (const auto& e : c->mx_modes)
    if (e.first == k && mode_fits(e.second, q.algo, n, q.K, c->mx_slice)) return e.second;
  return greedy_mode(q.algo, n, q.K, c->mx_slice);
}

mdx_status check_request(mdx_ctx* c, int r, const mdx_request& q) {
  if (q.n_tx < 1 || q.n_rx < q.n_tx)
    return fail(c, MDX_EINVAL, "request %d: need n_rx >= n_tx >= 1 (got %d, %d)", r, q.n_rx, q.n_tx);
  if (q.n_tx > c->max_tx || q.n_rx > c->max_rx)
    return fail(c, MDX_EUNSUPPORTED, "request %d: %dx%d exceeds the context's %dx%d", r, q.n_rx, q.n_tx, c->max_rx,
                c->max_tx);
  if (pam_of(q.qam) < 0) return fail(c, MDX_EINVAL, "request %d: qam %d not in {4, 16, 64}", r, q.qam);
  if (q.algo != MDX_ALGO_SD && q.algo != MDX_ALGO_KBEST && q.algo != MDX_ALGO_SD_COMPLEX &&
      q.algo != MDX_ALGO_SD_NATURAL)
    return fail(c, MDX_EINVAL, "request %d: algo %d is not an MDX_ALGO_* detector", r, q.algo);
  if (q.algo == MDX_ALGO_KBEST && (q.K < 1 || q.K > MDX_MAX_K))
    return fail(c, MDX_EINVAL, "request %d: K %d not in 1..%d", r, q.K, MDX_MAX_K);
  if (isnan(q.init_radius_sq) || q.init_radius_sq == 0.0)
    return fail(c, MDX_EINVAL, "request %d: init_radius_sq must be > 0, < 0 or INFINITY", r);
  if (q.node_budget < 0) return fail(c, MDX_EINVAL, "request %d: node_budget < 0", r);
  if (q.h_offset < 0 || q.y_offset < 0 || q.sym_offset < 0 || (q.h_offset & 1) || (q.y_offset & 1))
    return fail(c, MDX_EINVAL, "request %d: offsets must be >= 0, h_offset and y_offset even", r);
  return MDX_OK;
}

bool same_table(const mdx_ctx* c, int nreq, const mdx_request* reqs) {
  return (int)c->mx_table.size() == nreq && nreq > 0 &&
         memcmp(c->mx_table.data(), reqs, sizeof(mdx_request) * (size_t)nreq) == 0;
}

// Builds the device descriptors of a request table (placement from the
// current tuning), the heaviest-first order and the QR class runs, uploads
// them, and sizes the per-warp global state slots.  Skipped when the table
// and the tuning are those of the last upload.
mdx_status mixed_upload(mdx_ctx* c, int nreq, const mdx_request* reqs, cudaStream_t s) {
  if (same_table(c, nreq, reqs)) return MDX_OK;
  std::vector<MixedReq> d((size_t)nreq);
  long long roff = 0, yoff = 0;
  int maxK = 0;
  size_t gslot = 16;
  std::vector<std::pair<double, int>> cost((size_t)nreq);
  for (int r = 0; r < nreq; ++r) {
    const mdx_request& q = reqs[r];
    MixedReq& m = d[r];
    memset(&m, 0, sizeof(m));
    m.n_rx = q.n_rx;
    m.n_tx = q.n_tx;
    m.n = 2 * q.n_tx;
    m.P = pam_of(q.qam);
    m.algo = q.algo;
    m.K = q.algo == MDX_ALGO_KBEST ? q.K : 0;
    m.mode = mode_for(c, q);
    const double r0 = q.init_radius_sq;
    m.radius_mode = isinf(r0) ? (r0 > 0 ? RADIUS_NONE : RADIUS_PAPER) : (r0 < 0 ? RADIUS_PAPER : RADIUS_VALUE);
    m.radius_value = r0;
    m.alpha64 = sqrt(3.0 / (2.0 * (q.qam - 1)));
    m.alpha = (float)m.alpha64;
    m.budget = q.algo != MDX_ALGO_KBEST ? q.node_budget : 0;
    m.h_off = q.h_offset;
    m.yin_off = q.y_offset;
    m.sym_off = q.sym_offset;
    m.r_off = roff;
    m.y_off = yoff;
    m.r_off64 = roff;
    m.y_off64 = yoff;
    roff += tri_stride32(m.n);
    yoff += vec_stride32(m.n);
    if (m.K > maxK) maxK = m.K;
    if (!(m.mode & MIX_STATE_SMEM)) gslot = std::max(gslot, mixed_state_bytes(m.algo, m.n, m.K, m.P));
    // a cost proxy for the order: the exact SD's tree grows fastest with n
    const double n = m.n;
    cost[r].first = (m.algo != MDX_ALGO_KBEST) ? n * n * n * m.P : n * m.K * (n + 8.0 * m.P);
    cost[r].second = r;
  }
  std::stable_sort(cost.begin(), cost.end(),
                   [](const std::pair<double, int>& a, const std::pair<double, int>& b) { return a.first > b.first; });
  // QR runs: requests grouped by (n_rx, n_tx)
  std::vector<int> ids((size_t)nreq);
  for (int r = 0; r < nreq; ++r) ids[r] = r;
  std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) {
    return std::make_pair(reqs[a].n_rx, reqs[a].n_tx) < std::make_pair(reqs[b].n_rx, reqs[b].n_tx);
  });
  std::vector<int> runs;
  for (int t = 0; t < nreq; ++t) {
    const mdx_request& q = reqs[ids[t]];
    if (runs.empty() || runs[runs.size() - 4] != q.n_rx || runs[runs.size() - 3] != q.n_tx) {
      runs.push_back(q.n_rx);
      runs.push_back(q.n_tx);
      runs.push_back(t);
      runs.push_back(0);
    }
    runs.back() += 1;
  }
  const size_t bytes = sizeof(MixedReq) * (size_t)nreq + 2 * sizeof(int) * (size_t)nreq;
  cudaError_t e = cudaSuccess;
  if (c->mx_pinned_bytes < bytes) {
    if (c->mx_pinned) cudaFreeHost(c->mx_pinned);
    c->mx_pinned = nullptr;
    c->mx_pinned_bytes = 0;
    e = cudaMallocHost(reinterpret_cast<void**>(&c->mx_pinned), bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "pinned descriptor buffer");
    c->mx_pinned_bytes = bytes;
  }
  if (c->mx_dev_bytes < bytes) {
    if (c->mx_graph) {
      cudaGraphExecDestroy(c->mx_graph);
      c->mx_graph = nullptr;
    }
    if (c->mx_dev) cudaFree(c->mx_dev);
    c->mx_dev = nullptr;
    c->mx_dev_bytes = 0;
    e = cudaMalloc(reinterpret_cast<void**>(&c->mx_dev), bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "descriptor buffer");
    c->mx_dev_bytes = bytes;
  }
  memcpy(c->mx_pinned, d.data(), sizeof(MixedReq) * (size_t)nreq);
  int* ord = reinterpret_cast<int*>(c->mx_pinned + sizeof(MixedReq) * (size_t)nreq);
  for (int t = 0; t < nreq; ++t) ord[t] = cost[t].second;
  memcpy(ord + nreq, ids.data(), sizeof(int) * (size_t)nreq);
  // the stream may still be reading the previous descriptors: upload in order on it
  e = cudaMemcpyAsync(c->mx_dev, c->mx_pinned, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "descriptor upload");
  // per-warp global state slots for the requests whose state is not in shared memory
  const int warps = mixed_resident_warps(c->mx_W, c->mx_slice, maxK, c->num_sms);
  if (warps < 1) return fail(c, MDX_EUNSUPPORTED, "no launch of %d warps x %d bytes fits", c->mx_W, c->mx_slice);
  const size_t sbytes = (size_t)warps * gslot;
  if (c->mx_scratch_bytes < sbytes) {
    if (c->mx_graph) {
      cudaGraphExecDestroy(c->mx_graph);
      c->mx_graph = nullptr;
    }
    if (c->mx_scratch) cudaFree(c->mx_scratch);
    c->mx_scratch = nullptr;
    c->mx_scratch_bytes = 0;
    e = cudaMalloc(reinterpret_cast<void**>(&c->mx_scratch), sbytes);
    if (e != cudaSuccess) return fail(c, MDX_ENOMEM, "%zu bytes of per-warp search state", sbytes);
    c->mx_scratch_bytes = sbytes;
  }
  c->mx_table.assign(reqs, reqs + nreq);
  c->mx_qr = runs;
  c->mx_maxK = maxK;
  c->mx_gslot = gslot;
  ++c->mx_gen;
  return MDX_OK;
}

// The launch sequence of one uneven batch: counter reset, QR per class, search.
cudaError_t mixed_launches(mdx_ctx* c, int nreq, const double* dH, const double* dy, const double* dnv,
                           uint8_t* dsym, double* dmet, int32_t* dvst, int64_t* dstats, int flags, cudaStream_t s,
                           cudaEvent_t* ev) {
  const MixedReq* dreqs = reinterpret_cast<const MixedReq*>(c->mx_dev);
  const int* dorder = reinterpret_cast<const int*>(c->mx_dev + sizeof(MixedReq) * (size_t)nreq);
  const int* dids = dorder + nreq;
  if (ev) cudaEventRecord(ev[0], s);
  QrOut q{c->R64, c->yb64, c->R32, c->yb32, nullptr, nullptr, c->singular};
  for (size_t k = 0; k + 3 < c->mx_qr.size(); k += 4) {
    const cudaError_t e = launch_qr_gather(c->mx_qr[k + 3], c->mx_qr[k], c->mx_qr[k + 1], dids + c->mx_qr[k + 2],
                                           dreqs, dH, dy, q, s);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemsetAsync(c->counter, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[1], s);
  MixedArgs a{};
  a.nreq = nreq;
  a.reqs = dreqs;
  a.order = dorder;
  a.R32 = c->R32;
  a.yb32 = c->yb32;
  a.R64 = c->R64;
  a.yb64 = c->yb64;
  a.singular = c->singular;
  a.noise_var = dnv;
  a.counter = c->counter;
  a.gscratch = c->mx_scratch;
  a.gslot_bytes = c->mx_gslot;
  a.slice_bytes = c->mx_slice;
  a.flags = flags;
  a.sym_out = dsym;
  a.metric_out = dmet;
  a.vstatus = dvst;
  a.stats = dstats;
  e = launch_mixed(a, c->mx_W, c->mx_maxK, c->num_sms, s);
  if (ev && e == cudaSuccess) cudaEventRecord(ev[2], s);
  return e;
}

mdx_status run_mixed(mdx_ctx* c, int nreq, const mdx_request* reqs, const double* H, const double* y,
                     const double* nv, uint8_t* sym, double* met, int32_t* vst, int64_t* stats, int flags,
                     void* stream) {
  if (!c) return MDX_EINVAL;
  if (nreq < 0) return fail(c, MDX_EINVAL, "nreq %d < 0", nreq);
  if (nreq == 0) return MDX_OK;
  if (!reqs) return fail(c, MDX_EINVAL, "request table is NULL");
  if (nreq > c->max_batch)
    return fail(c, MDX_EUNSUPPORTED, "nreq %d > context max_batch %d", nreq, c->max_batch);
  if (!H || !y || !sym || !met || !vst) return fail(c, MDX_EINVAL, "NULL input or output pointer");
  const bool host = (flags & MDX_HOST_BUFFERS) != 0;
  long long h_end = 0, y_end = 0, s_end = 0;
  bool need_nv = false;
  if (!same_table(c, nreq, reqs)) {
    for (int r = 0; r < nreq; ++r) {
      const mdx_status st = check_request(c, r, reqs[r]);
      if (st != MDX_OK) return st;
    }
  }
  for (int r = 0; r < nreq; ++r) {
    const mdx_request& q = reqs[r];
    h_end = std::max(h_end, q.h_offset + 2LL * q.n_rx * q.n_tx);
    y_end = std::max(y_end, q.y_offset + 2LL * q.n_rx);
    s_end = std::max(s_end, q.sym_offset + (long long)q.n_tx);
    need_nv |= (q.init_radius_sq < 0.0);
  }
  if (need_nv && !nv) return fail(c, MDX_EINVAL, "noise_var needed for the paper radius");
  if (host) {
    if (h_end > 2LL * c->max_batch * c->max_rx * c->max_tx || y_end > 2LL * c->max_batch * c->max_rx ||
        s_end > (long long)c->max_batch * c->max_tx)
      return fail(c, MDX_EUNSUPPORTED, "host buffers larger than the context's staging");
  } else {
    if (!aligned16(H) || !aligned16(y)) return fail(c, MDX_EINVAL, "H and y must be 16-byte aligned");
    const void* ptrs[] = {H, y, sym, met, vst};
    for (const void* q : ptrs)
      if (!is_device_ptr(q, c->device))
        return fail(c, MDX_EINVAL, "pointer %p is not device memory of device %d", q, c->device);
    if (nv && !is_device_ptr(nv, c->device)) return fail(c, MDX_EINVAL, "noise_var is not device memory");
    if (stats && !is_device_ptr(stats, c->device)) return fail(c, MDX_EINVAL, "stats is not device memory");
  }
  DeviceGuard g(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "earlier asynchronous error");
  mdx_status st = mixed_upload(c, nreq, reqs, s);
  if (st != MDX_OK) return st;

  const double* dH = H;
  const double* dy = y;
  const double* dnv = nv;
  uint8_t* dsym = sym;
  double* dmet = met;
  int32_t* dvst = vst;
  int64_t* dstats = stats;
  if (host) {
    e = cudaMemcpyAsync(c->sH, H, sizeof(double) * (size_t)h_end, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->sy, y, sizeof(double) * (size_t)y_end, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nv) e = cudaMemcpyAsync(c->snv, nv, sizeof(double) * nreq, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device staging");
    dH = c->sH;
    dy = c->sy;
    dnv = nv ? c->snv : nullptr;
    dsym = c->ssym;
    dmet = c->smet;
    dvst = c->svst;
    dstats = stats ? c->sstats : nullptr;
  }
  if (flags & MDX_GRAPH) {
    const std::vector<const void*> key = {reinterpret_cast<const void*>(c->mx_gen), dH, dy, dnv, dsym, dmet, dvst,
                                          dstats, reinterpret_cast<const void*>((uintptr_t)(flags & ~MDX_HOST_BUFFERS))};
    if (!c->mx_graph || c->mx_graph_key != key) {
      if (c->mx_graph) cudaGraphExecDestroy(c->mx_graph);
      c->mx_graph = nullptr;
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(c, e, "graph capture (use a non-default stream)");
      const cudaError_t le = mixed_launches(c, nreq, dH, dy, dnv, dsym, dmet, dvst, dstats, flags, s, nullptr);
      e = cudaStreamEndCapture(s, &graph);
      if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (le == cudaErrorInvalidConfiguration)
          return fail(c, MDX_EUNSUPPORTED, "no launch configuration fits this size");
        return cuda_fail(c, le, "captured launches");
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
      e = cudaGraphInstantiate(&c->mx_graph, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        c->mx_graph = nullptr;
        return cuda_fail(c, e, "graph instantiation");
      }
      c->mx_graph_key = key;
    }
    e = cudaGraphLaunch(c->mx_graph, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
  } else {
    cudaEvent_t* ev = nullptr;
    if (c->prof && c->prof_n < mdx_ctx::kProfSlots) ev = c->prof_ev[c->prof_n++];
    e = mixed_launches(c, nreq, dH, dy, dnv, dsym, dmet, dvst, dstats, flags, s, ev);
    if (e == cudaErrorInvalidConfiguration) return fail(c, MDX_EUNSUPPORTED, "no launch configuration fits this size");
    if (e != cudaSuccess) return cuda_fail(c, e, "uneven-batch launches");
  }
  if (host) {
    e = cudaMemcpyAsync(sym, c->ssym, (size_t)s_end, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(met, c->smet, sizeof(double) * nreq, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vst, c->svst, sizeof(int32_t) * nreq, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && stats)
      e = cudaMemcpyAsync(stats, c->sstats, sizeof(int64_t) * kStats * (size_t)nreq, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host results");
  }
  return MDX_OK;
}

// Milliseconds of one detect_mixed call (after one untimed call).
mdx_status time_mixed(mdx_ctx* c, int nreq, const mdx_request* reqs, const double* H, const double* y,
                      const double* nv, uint8_t* sym, double* met, int32_t* vst, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(c, MDX_ECUDA, "event creation");
  mdx_status st = run_mixed(c, nreq, reqs, H, y, nv, sym, met, vst, nullptr, 0, s);
  if (st == MDX_OK) {
    cudaEventRecord(e0, s);
    st = run_mixed(c, nreq, reqs, H, y, nv, sym, met, vst, nullptr, 0, s);
    cudaEventRecord(e1, s);
  }
  if (st == MDX_OK) {
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) st = cuda_fail(c, e, "tuning run");
    else cudaEventElapsedTime(ms, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

void set_tuning(mdx_ctx* c, int W, int slice, const std::vector<std::pair<unsigned long long, int>>& modes) {
  c->mx_W = W;
  c->mx_slice = slice;
  c->mx_modes = modes;
  c->mx_table.clear();  // descriptors are rebuilt with the new placement
}

mdx_status run_autotune(mdx_ctx* c, int nreq, const mdx_request* reqs, const double* H, const double* y,
                        const double* nv, uint8_t* sym, double* met, int32_t* vst, double* results, void* stream) {
  if (!c) return MDX_EINVAL;
  if (nreq < 1 || !reqs) return fail(c, MDX_EINVAL, "autotuning needs a non-empty request table");
  for (int r = 0; r < nreq; ++r) {
    const mdx_status st = check_request(c, r, reqs[r]);
    if (st != MDX_OK) return st;
  }
  DeviceGuard g(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // 1. warps per CTA and slice size, every class on its greedy placement
  struct Shape {
    int W, S;
  };
  const Shape shapes[] = {{4, 0},     {4, 16384},  {4, 49152}, {8, 0},    {8, 6144},  {8, 12288},
                          {8, 24576}, {16, 0},     {16, 3072}, {16, 6144}, {16, 12288}};
  int bestW = c->mx_W, bestS = c->mx_slice;
  float best = INFINITY;
  for (const Shape& sh : shapes) {
    set_tuning(c, sh.W, sh.S, {});
    if (mixed_resident_warps(sh.W, sh.S, MDX_MAX_K, c->num_sms) < 1) continue;
    float ms = INFINITY;
    const mdx_status st = time_mixed(c, nreq, reqs, H, y, nv, sym, met, vst, s, &ms);
    if (st != MDX_OK) return st;
    if (ms < best) {
      best = ms;
      bestW = sh.W;
      bestS = sh.S;
    }
  }
  // 2. placement per request class, each class timed alone
  std::vector<unsigned long long> keys;
  for (int r = 0; r < nreq; ++r)
    if (std::find(keys.begin(), keys.end(), class_key(reqs[r])) == keys.end()) keys.push_back(class_key(reqs[r]));
  std::vector<std::pair<unsigned long long, int>> modes;
  for (unsigned long long k : keys) {
    std::vector<mdx_request> sub;
    for (int r = 0; r < nreq; ++r)
      if (class_key(reqs[r]) == k) sub.push_back(reqs[r]);
    const mdx_request& q0 = sub[0];
    const int n = 2 * q0.n_tx;
    const int greedy = greedy_mode(q0.algo, n, q0.K, bestS);
    int win = greedy;
    float win_ms = INFINITY;
    for (int m : {greedy, 0, (int)MIX_STAGE_R, (int)MIX_STATE_SMEM, (int)(MIX_STAGE_R | MIX_STATE_SMEM)}) {
      if (!mode_fits(m, q0.algo, n, q0.K, bestS) || (m == greedy && win_ms < INFINITY)) continue;
      std::vector<std::pair<unsigned long long, int>> trial = modes;
      trial.push_back({k, m});
      set_tuning(c, bestW, bestS, trial);
      float ms = INFINITY;
      const mdx_status st = time_mixed(c, (int)sub.size(), sub.data(), H, y, nv, sym, met, vst, s, &ms);
      if (st != MDX_OK) return st;
      // keep the greedy placement unless another is clearly faster
      if (m == greedy) win_ms = ms;
      else if (ms < 0.97f * win_ms) {
        win = m;
        win_ms = ms;
      }
    }
    modes.push_back({k, win});
  }
  // 3. the whole table with the chosen placements; keep them only if not slower
  set_tuning(c, bestW, bestS, modes);
  float ms = INFINITY;
  mdx_status st = time_mixed(c, nreq, reqs, H, y, nv, sym, met, vst, s, &ms);
  if (st != MDX_OK) return st;
  if (!(ms <= best)) {
    set_tuning(c, bestW, bestS, {});
    ms = best;
  }
  if (results) {
    results[0] = bestW;
    results[1] = bestS;
    results[2] = ms;
  }
  return MDX_OK;
}

// Gray-coded bit errors and symbol errors, one thread per symbol.
__global__ void count_errors_kernel(long long total, int P, const uint8_t* __restrict__ a,
                                    const uint8_t* __restrict__ b, unsigned long long* counts) {
  unsigned long long be = 0, se = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int x = a[t], z = b[t];
    se += (x != z);
    const int xr = x / P, xi = x % P, zr = z / P, zi = z % P;
    be += __popc((xr ^ (xr >> 1)) ^ (zr ^ (zr >> 1))) + __popc((xi ^ (xi >> 1)) ^ (zi ^ (zi >> 1)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    be += __shfl_xor_sync(0xffffffffu, be, o);
    se += __shfl_xor_sync(0xffffffffu, se, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&counts[0], be);
    atomicAdd(&counts[1], se);
  }
}

}  // namespace

namespace mdx {
cudaError_t launch_count_errors(int batch, int n_tx, int qam, const uint8_t* a, const uint8_t* b,
                                unsigned long long* counts, cudaStream_t s) {
  const long long total = (long long)batch * n_tx;
  int grid = (int)((total + 255) / 256);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  count_errors_kernel<<<grid, 256, 0, s>>>(total, pam_of(qam), a, b, counts);
  return cudaGetLastError();
}
}  // namespace mdx

extern "C" {

const char* mdx_strerror(mdx_status s) {
  switch (s) {
    case MDX_OK: return "ok";
    case MDX_EINVAL: return "invalid argument";
    case MDX_EUNSUPPORTED: return "unsupported size or parameter";
    case MDX_ENOMEM: return "out of device memory";
    case MDX_ECUDA: return "CUDA error";
  }
  return "unknown status";
}

const char* mdx_last_error(const mdx_ctx* ctx) { return ctx ? ctx->err : "no context"; }

size_t mdx_workspace_bytes(const mdx_ctx* ctx) { return ctx ? ctx->bytes : 0; }

mdx_status mdx_create(mdx_ctx** out, int device, int max_batch, int max_n_rx, int max_n_tx) {
  if (!out) return MDX_EINVAL;
  *out = nullptr;
  if (max_batch < 1 || max_n_tx < 1 || max_n_rx < max_n_tx || max_n_tx > MDX_MAX_TX ||
      max_n_rx > MDX_MAX_RX)
    return MDX_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MDX_EINVAL;
  }
  mdx_ctx* c = new mdx_ctx();
  c->device = device;
  c->max_batch = max_batch;
  c->max_rx = max_n_rx;
  c->max_tx = max_n_tx;
  DeviceGuard g(device);
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  const size_t B = (size_t)max_batch;
  const int n = 2 * max_n_tx;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  // FP64 buffers sized with the FP32 strides (multiples of 4 elements), so that
  // an uneven batch of up to max_batch requests also fits
  chk(alloc(c, &c->R64, B * tri_stride32(n)));
  chk(alloc(c, &c->yb64, B * vec_stride32(n)));
  chk(alloc(c, &c->R32, B * tri_stride32(n)));
  chk(alloc(c, &c->yb32, B * vec_stride32(n)));
  chk(alloc(c, &c->singular, B));
  chk(alloc(c, &c->counter, 4));
  chk(alloc(c, &c->counts, 2));
  chk(alloc(c, &c->sH, B * max_n_rx * max_n_tx * 2));
  chk(alloc(c, &c->sy, B * max_n_rx * 2));
  chk(alloc(c, &c->snv, B));
  chk(alloc(c, &c->ssym, B * max_n_tx));
  chk(alloc(c, &c->ssym2, B * max_n_tx));
  chk(alloc(c, &c->smet, B));
  chk(alloc(c, &c->svst, B));
  chk(alloc(c, &c->sstats, B * kStats));
  chk(alloc(c, reinterpret_cast<unsigned char**>(&c->sd_shared), sd_shared_bytes()));
  chk(alloc(c, reinterpret_cast<unsigned char**>(&c->sd_queue), sd_task_bytes() * kSdQueueSlots));
  chk(alloc(c, &c->sd_vstate, B * sd_vec_state_bytes(n)));
  chk(alloc(c, &c->sd_order, sd_order_ints(max_batch)));
  chk(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  chk(cudaEventCreateWithFlags(&c->ev_free, cudaEventDisableTiming));
  for (cudaEvent_t& ev : c->ev_chunk) chk(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return MDX_ENOMEM;
  }
  // task slots are published by sequence numbers that never equal zero
  if (cudaMemset(c->sd_queue, 0, sd_task_bytes() * kSdQueueSlots) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return MDX_ECUDA;
  }
  *out = c;
  return MDX_OK;
}

mdx_status mdx_destroy(mdx_ctx* ctx) {
  if (!ctx) return MDX_EINVAL;
  DeviceGuard g(ctx->device);
  free_all(ctx);
  delete ctx;
  return MDX_OK;
}

mdx_status mdx_qr(mdx_ctx* c, int batch, int n_rx, int n_tx, const double* H, const double* y,
                  double* R_out, double* ybar_out, int flags, void* stream) {
  if (!c) return MDX_EINVAL;
  if (flags & MDX_HOST_BUFFERS) return fail(c, MDX_EUNSUPPORTED, "mdx_qr takes device pointers only");
  if (batch < 0) return fail(c, MDX_EINVAL, "batch < 0");
  if (batch == 0) return MDX_OK;
  if (n_tx < 1 || n_rx < n_tx) return fail(c, MDX_EINVAL, "need n_rx >= n_tx >= 1");
  if (n_tx > MDX_MAX_TX || n_rx > MDX_MAX_RX) return fail(c, MDX_EUNSUPPORTED, "size beyond %dx%d", MDX_MAX_RX, MDX_MAX_TX);
  if (!H || !y || !R_out || !ybar_out) return fail(c, MDX_EINVAL, "NULL pointer");
  if (!aligned16(H) || !aligned16(y)) return fail(c, MDX_EINVAL, "H and y must be 16-byte aligned");
  const void* ptrs[] = {H, y, R_out, ybar_out};
  for (const void* q : ptrs)
    if (!is_device_ptr(q, c->device)) return fail(c, MDX_EINVAL, "pointer %p is not device memory", q);
  DeviceGuard g(c->device);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "earlier asynchronous error");
  QrOut q{nullptr, nullptr, nullptr, nullptr, R_out, ybar_out, nullptr};
  e = launch_qr(batch, n_rx, n_tx, H, y, q, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "QR launch");
  return MDX_OK;
}

mdx_status detect_sd(mdx_ctx* ctx, const mdx_params* p, int batch, const double* H, const double* y,
                     const double* noise_var, uint8_t* sym_out, double* metric_out, int32_t* vstatus,
                     int64_t* stats, void* stream) {
  return run_detect(ALGO_SD, ctx, p, batch, H, y, noise_var, sym_out, metric_out, vstatus, stats, stream);
}

mdx_status detect_kbest(mdx_ctx* ctx, const mdx_params* p, int batch, const double* H,
                        const double* y, const double* noise_var, uint8_t* sym_out,
                        double* metric_out, int32_t* vstatus, int64_t* stats, void* stream) {
  return run_detect(ALGO_KBEST, ctx, p, batch, H, y, noise_var, sym_out, metric_out, vstatus, stats,
                    stream);
}

mdx_status detect_hybrid(mdx_ctx* ctx, const mdx_params* p, int batch, const double* H,
                         const double* y, const double* noise_var, uint8_t* sym_out,
                         double* metric_out, int32_t* vstatus, int64_t* stats, void* stream) {
  return run_detect(ALGO_HYBRID, ctx, p, batch, H, y, noise_var, sym_out, metric_out, vstatus, stats,
                    stream);
}

mdx_status detect_linear(mdx_ctx* ctx, const mdx_params* p, int batch, const double* H, const double* y,
                         const double* noise_var, uint8_t* sym_out, double* metric_out, int32_t* vstatus,
                         int64_t* stats, void* stream) {
  return run_detect(ALGO_LINEAR, ctx, p, batch, H, y, noise_var, sym_out, metric_out, vstatus, stats, stream);
}

mdx_status detect_mixed(mdx_ctx* ctx, int nreq, const mdx_request* reqs, const double* H, const double* y,
                        const double* noise_var, uint8_t* sym_out, double* metric_out, int32_t* vstatus,
                        int64_t* stats, int flags, void* stream) {
  return run_mixed(ctx, nreq, reqs, H, y, noise_var, sym_out, metric_out, vstatus, stats, flags, stream);
}

mdx_status mdx_autotune_mixed(mdx_ctx* ctx, int nreq, const mdx_request* reqs, const double* H, const double* y,
                              const double* noise_var, uint8_t* sym_out, double* metric_out, int32_t* vstatus,
                              double* results, void* stream) {
  return run_autotune(ctx, nreq, reqs, H, y, noise_var, sym_out, metric_out, vstatus, results, stream);
}

mdx_status mdx_count_errors(mdx_ctx* c, int batch, int n_tx, int qam, const uint8_t* sym_hat,
                            const uint8_t* sym_true, int64_t* counts_out, int flags, void* stream) {
  if (!c) return MDX_EINVAL;
  if (batch < 0 || n_tx < 1) return fail(c, MDX_EINVAL, "bad batch or n_tx");
  if (pam_of(qam) < 0) return fail(c, MDX_EINVAL, "qam %d not in {4, 16, 64}", qam);
  if (!sym_hat || !sym_true || !counts_out) return fail(c, MDX_EINVAL, "NULL pointer");
  const bool host = (flags & MDX_HOST_BUFFERS) != 0;
  if (host && ((size_t)batch > (size_t)c->max_batch || n_tx > c->max_tx))
    return fail(c, MDX_EUNSUPPORTED, "batch beyond the staging buffers");
  if (!host) {
    const void* ptrs[] = {sym_hat, sym_true, counts_out};
    for (const void* q : ptrs)
      if (!is_device_ptr(q, c->device)) return fail(c, MDX_EINVAL, "pointer %p is not device memory", q);
  }
  DeviceGuard g(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "earlier asynchronous error");
  const uint8_t* a = sym_hat;
  const uint8_t* b = sym_true;
  if (host) {
    e = cudaMemcpyAsync(c->ssym, sym_hat, (size_t)batch * n_tx, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ssym2, sym_true, (size_t)batch * n_tx, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "staging");
    a = c->ssym;
    b = c->ssym2;
  }
  e = cudaMemsetAsync(c->counts, 0, 2 * sizeof(unsigned long long), s);
  if (e == cudaSuccess && batch > 0) e = launch_count_errors(batch, n_tx, qam, a, b, c->counts, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(counts_out, c->counts, 2 * sizeof(int64_t),
                        host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && host) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "error count");
  return MDX_OK;
}

size_t mdx_mlp_param_count(int n_tx, int qam) {
  if (n_tx < 1 || n_tx > MDX_MAX_TX || pam_of(qam) < 0) return 0;
  return (size_t)mlp_count(n_tx, qam);
}

mdx_status mdx_mlp_dims(int n_tx, int qam, int* d_in, int* d_out) {
  if (n_tx < 1 || n_tx > MDX_MAX_TX || pam_of(qam) < 0 || !d_in || !d_out) return MDX_EINVAL;
  mlp_dims(n_tx, qam, d_in, d_out);
  return MDX_OK;
}

mdx_status mdx_mlp_init(mdx_ctx* c, int n_tx, int qam, int max_train_batch, unsigned long long seed) {
  if (!c) return MDX_EINVAL;
  if (n_tx < 1 || n_tx > c->max_tx || pam_of(qam) < 0)
    return fail(c, MDX_EINVAL, "model size n_tx %d, qam %d not within the context", n_tx, qam);
  if (max_train_batch < 0) return fail(c, MDX_EINVAL, "max_train_batch < 0");
  DeviceGuard g(c->device);
  if (c->mlp) {
    mlp_free(c->mlp);
    c->mlp = nullptr;
  }
  const int cap = max_train_batch > c->max_batch ? max_train_batch : c->max_batch;
  MlpState* m = nullptr;
  cudaError_t e = mlp_alloc(&m, n_tx, qam, cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MDX_ENOMEM, "model workspace: %s", cudaGetErrorString(e));
  }
  c->mlp = m;
  // He-uniform weights from a SplitMix64 stream; zero biases except the radius
  // head, which starts at log(n_tx) (the mean of d_ML / sigma^2 is about n_tx)
  int D0, DO;
  mlp_dims(n_tx, qam, &D0, &DO);
  const int n = 2 * n_tx, P = pam_of(qam);
  const bool reduced = n_tx > kFullFeaturesMaxTx;
  const int din = reduced ? n + 3 : n * (n + 1) / 2 + n + 1, dout = reduced ? 1 : 1 + n * P;
  const long long cnt = mlp_count(n_tx, qam);
  float* h = new float[cnt]();
  uint64_t st = seed * 0x9E3779B97F4A7C15ull + 0x5DEECE66Dull;
  auto uni = [&]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  };
  const int H = 256;
  size_t o = 0;
  const double a1 = sqrt(6.0 / din), a2 = sqrt(6.0 / H), a3 = 0.1 * sqrt(6.0 / H);
  for (int r = 0; r < H; ++r)
    for (int k = 0; k < D0; ++k) h[o++] = k < din ? (float)(a1 * uni()) : 0.0f;
  o += H;  // b1
  for (int r = 0; r < H; ++r)
    for (int k = 0; k < H; ++k) h[o++] = (float)(a2 * uni());
  o += H;  // b2
  for (int r = 0; r < DO; ++r)
    for (int k = 0; k < H; ++k) h[o++] = r < dout ? (float)(a3 * uni()) : 0.0f;
  h[o] = (float)log((double)n_tx);  // b3[0]
  e = cudaMemcpy(mlp_params(m), h, sizeof(float) * cnt, cudaMemcpyHostToDevice);
  delete[] h;
  if (e == cudaSuccess) e = mlp_pack(m, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "model init");
  c->bytes += mlp_bytes(m);
  return MDX_OK;
}

mdx_status mdx_mlp_set_params(mdx_ctx* c, const float* host, size_t count) {
  if (!c || !host) return MDX_EINVAL;
  if (!c->mlp) return fail(c, MDX_EUNSUPPORTED, "no model (mdx_mlp_init)");
  if (count != (size_t)mlp_count(mlp_ntx(c->mlp), mlp_qam(c->mlp))) return fail(c, MDX_EINVAL, "parameter count");
  DeviceGuard g(c->device);
  cudaError_t e = cudaMemcpy(mlp_params(c->mlp), host, sizeof(float) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = mlp_pack(c->mlp, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "set params");
  return MDX_OK;
}

mdx_status mdx_mlp_get_params(mdx_ctx* c, float* host, size_t count) {
  if (!c || !host) return MDX_EINVAL;
  if (!c->mlp) return fail(c, MDX_EUNSUPPORTED, "no model (mdx_mlp_init)");
  if (count != (size_t)mlp_count(mlp_ntx(c->mlp), mlp_qam(c->mlp))) return fail(c, MDX_EINVAL, "parameter count");
  DeviceGuard g(c->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(host, mlp_params(c->mlp), sizeof(float) * count, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "get params");
  return MDX_OK;
}

// QR + features for a batch of device inputs; returns rows (padded batch) or <0.
static mdx_status mlp_prepare(mdx_ctx* c, const mdx_params* p, int batch, const double* H, const double* y,
                              const double* nv, bool train, float* feat_out, cudaStream_t s, int* rows_out) {
  if (!c) return MDX_EINVAL;
  if (!p) return fail(c, MDX_EINVAL, "params is NULL");
  if (!c->mlp) return fail(c, MDX_EUNSUPPORTED, "no model (mdx_mlp_init)");
  if (p->flags & MDX_HOST_BUFFERS) return fail(c, MDX_EUNSUPPORTED, "device pointers only");
  if (batch < 1 || batch > mlp_cap(c->mlp) || batch > c->max_batch)
    return fail(c, MDX_EUNSUPPORTED, "batch %d outside 1..%d", batch, c->max_batch);
  if (p->n_tx != mlp_ntx(c->mlp) || p->n_rx != p->n_tx || p->qam != mlp_qam(c->mlp))
    return fail(c, MDX_EINVAL, "the model was built for %dx%d %d-QAM", mlp_ntx(c->mlp), mlp_ntx(c->mlp),
                mlp_qam(c->mlp));
  if (!H || !y || !nv) return fail(c, MDX_EINVAL, "NULL input");
  if (!aligned16(H) || !aligned16(y)) return fail(c, MDX_EINVAL, "H and y must be 16-byte aligned");
  const void* ptrs[] = {H, y, nv};
  for (const void* q : ptrs)
    if (!is_device_ptr(q, c->device)) return fail(c, MDX_EINVAL, "pointer %p is not device memory", q);
  const int rows = round_up(batch, 128);
  QrOut q{c->R64, c->yb64, c->R32, c->yb32, nullptr, nullptr, c->singular};
  cudaError_t e = launch_qr(batch, p->n_rx, p->n_tx, H, y, q, s);
  if (e == cudaSuccess) e = mlp_features(c->mlp, batch, rows, c->R32, c->yb32, nv, train, feat_out, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "features");
  *rows_out = rows;
  return MDX_OK;
}

mdx_status mdx_mlp_predict(mdx_ctx* c, const mdx_params* p, int batch, const double* H, const double* y,
                           const double* nv, float* out, float* feat_out, void* stream) {
  if (!c) return MDX_EINVAL;
  if (!out) return fail(c, MDX_EINVAL, "NULL output");
  DeviceGuard g(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rows = 0;
  mdx_status st = mlp_prepare(c, p, batch, H, y, nv, false, feat_out, s, &rows);
  if (st != MDX_OK) return st;
  cudaError_t e = mlp_forward(c->mlp, rows, false, s);
  int D0, DO;
  mlp_dims(p->n_tx, p->qam, &D0, &DO);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, mlp_outputs(c->mlp), sizeof(float) * DO * (size_t)batch, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "forward");
  return MDX_OK;
}

mdx_status mdx_mlp_train_step(mdx_ctx* c, const mdx_params* p, int batch, const double* H, const double* y,
                              const double* nv, const uint8_t* ml_sym, const double* ml_metric, float lr,
                              int update, float* grad_out, float* loss_out, void* stream) {
  if (!c) return MDX_EINVAL;
  if (!c->mlp) return fail(c, MDX_EUNSUPPORTED, "no model (mdx_mlp_init)");
  const bool need_sym = !mlp_reduced(c->mlp);
  if (!ml_metric || (need_sym && !ml_sym)) return fail(c, MDX_EINVAL, "NULL targets");
  if ((ml_sym && !is_device_ptr(ml_sym, c->device)) || !is_device_ptr(ml_metric, c->device))
    return fail(c, MDX_EINVAL, "targets must be device memory");
  if (!(lr >= 0.0f)) return fail(c, MDX_EINVAL, "learning rate");
  DeviceGuard g(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rows = 0;
  mdx_status st = mlp_prepare(c, p, batch, H, y, nv, true, nullptr, s, &rows);
  if (st != MDX_OK) return st;
  cudaError_t e = mlp_forward(c->mlp, rows, true, s);
  if (e == cudaSuccess) e = mlp_backward(c->mlp, batch, rows, ml_metric, nv, ml_sym, s);
  if (e == cudaSuccess && grad_out)
    e = cudaMemcpyAsync(grad_out, mlp_grads(c->mlp), sizeof(float) * mlp_count(p->n_tx, p->qam),
                        cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && loss_out)
    e = cudaMemcpyAsync(loss_out, mlp_loss(c->mlp), 2 * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && update) e = mlp_adam(c->mlp, lr, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "train step");
  return MDX_OK;
}

mdx_status mdx_mlp_error(mdx_ctx* c, int* err_out) {
  if (!c || !err_out) return MDX_EINVAL;
  if (!c->mlp) {
    *err_out = 0;
    return MDX_OK;
  }
  DeviceGuard g(c->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(err_out, mlp_err(c->mlp), sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "model error word");
  return MDX_OK;
}

mdx_status mdx_profile(mdx_ctx* c, int enable) {
  if (!c) return MDX_EINVAL;
  DeviceGuard g(c->device);
  if (enable && !c->prof_ev[0][0]) {
    for (int i = 0; i < mdx_ctx::kProfSlots; ++i)
      for (int k = 0; k < 3; ++k) {
        cudaError_t e = cudaEventCreate(&c->prof_ev[i][k]);
        if (e != cudaSuccess) return cuda_fail(c, e, "event create");
      }
  }
  c->prof = enable != 0;
  c->prof_n = 0;
  return MDX_OK;
}

mdx_status mdx_profile_read(mdx_ctx* c, double* ms_out) {
  if (!c || !ms_out) return MDX_EINVAL;
  DeviceGuard g(c->device);
  double qr = 0.0, search = 0.0;
  for (int i = 0; i < c->prof_n; ++i) {
    cudaError_t e = cudaEventSynchronize(c->prof_ev[i][2]);
    if (e != cudaSuccess) return cuda_fail(c, e, "event sync");
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, c->prof_ev[i][0], c->prof_ev[i][1]);
    cudaEventElapsedTime(&b, c->prof_ev[i][1], c->prof_ev[i][2]);
    qr += a;
    search += b;
  }
  int err = 0;
  unsigned int cnt[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpy(&err, static_cast<char*>(c->sd_shared) + sd_error_offset(), sizeof(int),
                             cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(cnt, static_cast<char*>(c->sd_shared) + sd_counters_offset(), sizeof(cnt),
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "error word");
  for (int k = 0; k < 4; ++k) ms_out[4 + k] = cnt[k];
  ms_out[0] = qr;
  ms_out[1] = search;
  ms_out[2] = c->prof_n;
  ms_out[3] = err;
  c->prof_n = 0;
  return MDX_OK;
}

}  // extern "C"
