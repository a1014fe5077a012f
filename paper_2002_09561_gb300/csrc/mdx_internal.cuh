// Internal declarations shared by the CUDA translation units of libmdx.
// Device-side data layout (per received vector b, real dimension n = 2 n_tx):
//   R (upper triangular, n x n) is stored column-packed: column c holds rows
//   0..c contiguously at offset c (c + 1) / 2, so the entries a row update
//   needs (column c, rows below the current level) are contiguous and the
//   diagonal R_cc sits at the end of its column.  The per-vector stride is
//   rounded up to 16 bytes (tri_stride32 / tri_stride64).
//   ybar has n entries per vector (stride n rounded up to 16 bytes).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mimo_detect.h"

#define MDX_MAX_N (2 * MDX_MAX_TX)

namespace mdx {

__host__ __device__ __forceinline__ int col_off(int c) { return c * (c + 1) / 2; }
__host__ __device__ __forceinline__ int tri(int n) { return n * (n + 1) / 2; }
__host__ __device__ __forceinline__ int round_up(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ __forceinline__ int tri_stride32(int n) { return round_up(tri(n), 4); }
__host__ __device__ __forceinline__ int tri_stride64(int n) { return round_up(tri(n), 2); }
__host__ __device__ __forceinline__ int vec_stride32(int n) { return round_up(n, 4); }
__host__ __device__ __forceinline__ int vec_stride64(int n) { return round_up(n, 2); }

// Per-vector statistics slots (nodes, peds, restarts, rescored, flops).
constexpr int kStats = 5;

// Radius modes derived from mdx_params.init_radius_sq.
enum { RADIUS_NONE = 0, RADIUS_PAPER = 1, RADIUS_VALUE = 2, RADIUS_PER_VECTOR = 3 };

// Outputs of the QR kernel (any pointer may be null).
struct QrOut {
  double* R64;      // column-packed, stride tri_stride64(n)
  double* yb64;     // stride vec_stride64(n)
  float* R32;       // column-packed, stride tri_stride32(n)
  float* yb32;      // stride vec_stride32(n)
  double* Rdense;   // [n][n] row-major (mdx_qr)
  double* ybdense;  // [n]
  int* singular;    // [batch] 1 if a diagonal entry of R is zero
};

// Everything the search kernels read and write for one launch.
struct SearchArgs {
  int batch, n, P, n_rx, n_tx;
  float alpha;    // PAM spacing factor sqrt(3 / (2 (qam - 1)))
  double alpha64;
  const float* R32;
  const float* yb32;
  const double* R64;
  const double* yb64;
  const int* singular;
  const double* noise_var;
  const float* r2_vec;  // per-vector initial r^2 (RADIUS_PER_VECTOR), else null
  int radius_mode;
  double radius_value;
  int K;
  int depth;           // hybrid master depth
  long long budget;    // per-vector branched-node cap, 0 = none
  int flags;
  unsigned int* work_counter;  // dynamic vector queue (zeroed before launch)
  uint8_t* sym_out;
  double* metric_out;
  int32_t* vstatus;
  int64_t* stats;
};

cudaError_t launch_qr(int batch, int n_rx, int n_tx, const double* H, const double* y, QrOut out,
                      cudaStream_t s);

// One request of an uneven batch as the device sees it (built by the host
// from mdx_request).  R and ybar of request r live at r_off / y_off (elements)
// in the R32/R64 and yb32/yb64 workspaces; both offsets are multiples of 4.
struct MixedReq {
  int n_rx, n_tx, n, P;
  int algo, K;
  int mode;         // MIX_* placement bits chosen by the tuner
  int radius_mode;  // RADIUS_NONE / RADIUS_PAPER / RADIUS_VALUE
  float alpha;
  float pad0;
  double alpha64;
  double radius_value;
  long long budget;
  long long h_off, yin_off;  // H and y of the request (doubles)
  long long sym_off;
  long long r_off, y_off;      // FP32 R / ybar (elements)
  long long r_off64, y_off64;  // FP64 R / ybar (elements)
};
// placement of a request's data: R and ybar staged in the warp's shared-memory
// slice, and the search state (SD stacks / K-best survivors) in the slice;
// otherwise each is read from / kept in global memory
enum { MIX_STAGE_R = 1, MIX_STATE_SMEM = 2 };
// detector of a request (MDX_ALGO_SD / MDX_ALGO_KBEST, or the complex-tree SD)
enum { MIX_ALGO_SD_COMPLEX = 2, MIX_ALGO_SD_NATURAL = 3 };

cudaError_t launch_qr_gather(int count, int n_rx, int n_tx, const int* ids, const MixedReq* reqs,
                             const double* H, const double* y, QrOut out, cudaStream_t s);

struct MixedArgs {
  int nreq;
  const MixedReq* reqs;  // null: a uniform batch described by `uniform` (request r = vector r)
  const int* order;      // requests in the order warps take them (null: table order)
  MixedReq uniform;      // uniform batch: the fields shared by every vector, offsets zero
  const float* r2_vec;   // uniform batch with RADIUS_PER_VECTOR: initial r^2 per vector
  const float* R32;
  const float* yb32;
  const double* R64;
  const double* yb64;
  const int* singular;
  const double* noise_var;
  unsigned int* counter;
  unsigned char* gscratch;  // per-warp global state slots
  size_t gslot_bytes;
  int slice_bytes;          // shared memory per warp
  int flags;
  uint8_t* sym_out;
  double* metric_out;
  int32_t* vstatus;
  int64_t* stats;
};
// Bytes of a request's staged R + ybar and of its search state.
size_t mixed_stage_bytes(int n);
size_t mixed_state_bytes(int algo, int n, int K, int P);
// Warps a launch with this shape keeps resident (for sizing gscratch).
int mixed_resident_warps(int warps_per_cta, int slice_bytes, int max_K, int num_sms);
cudaError_t launch_mixed(const MixedArgs& a, int warps_per_cta, int max_K, int num_sms, cudaStream_t s);
// Placement of a uniform batch's vectors for a slice size (MIX_* bits).
int mixed_greedy_mode(int algo, int n, int K, int P, int slice_bytes);
// Global workspace of the sphere decoder's task queue (see sd.cu).
struct SdWorkspace {
  void* shared;          // sd_shared_bytes()
  void* queue;           // qcap task records of sd_task_bytes()
  unsigned int qcap;     // power of two
  unsigned char* vstate; // batch x sd_vec_state_bytes(n)
  unsigned long long epoch;  // distinct per launch on this workspace
  int* order;            // batch ints + sd_order_scratch_ints(): the fresh-vector order
};
size_t sd_order_ints(int max_batch);
size_t sd_shared_bytes();
size_t sd_error_offset();
size_t sd_counters_offset();
size_t sd_task_bytes();
size_t sd_vec_state_bytes(int n);
cudaError_t launch_sd(const SearchArgs& a, const SdWorkspace& w, int num_sms, cudaStream_t s);
cudaError_t launch_kbest(const SearchArgs& a, int num_sms, cudaStream_t s);
// Shared memory of the K-best kernel for (n, K, P, key capacity).
size_t kbest_smem_bytes(int n, int K, int P, bool complex_tree);
cudaError_t launch_hybrid(const SearchArgs& a, int num_sms, cudaStream_t s);
// Linear detectors (linear.cu): ZF or MMSE on the QR workspace.
size_t linear_smem_bytes(int n, bool mmse);
cudaError_t launch_linear(const SearchArgs& a, bool mmse, int num_sms, cudaStream_t s);
// Shared memory the hybrid needs for (n, K, P, depth), or (size_t)-1 if it does not fit.
size_t hybrid_smem_bytes(int n, int K, int P, int depth);
// Learned radius model (mlp.cu).  Systems with n_tx <= kFullFeaturesMaxTx use
// the full features (R's upper triangle, ybar, SNR) and both heads; larger
// ones summary features and the radius head only.
constexpr int kFullFeaturesMaxTx = 32;
struct MlpState;
void mlp_dims(int n_tx, int qam, int* D0, int* DO);
long long mlp_count(int n_tx, int qam);
cudaError_t mlp_alloc(MlpState** out, int n_tx, int qam, int cap);
void mlp_free(MlpState* s);
cudaError_t mlp_pack(MlpState* s, cudaStream_t st);
cudaError_t mlp_features(MlpState* s, int batch, int rows, const float* R32, const float* yb32, const double* nv,
                         bool train, float* F, cudaStream_t st);
cudaError_t mlp_forward(MlpState* s, int rows, bool train, cudaStream_t st);
cudaError_t mlp_backward(MlpState* s, int batch, int rows, const double* ml_metric, const double* nv,
                         const uint8_t* ml_sym, cudaStream_t st);
cudaError_t mlp_adam(MlpState* s, float lr, cudaStream_t st);
// Per-vector initial r^2 into mlp_r2(): learned (sigma^2 exp(o_0)) or the base
// radius (RADIUS_* mode), capped by the top-ranked leaf's distance if order.
cudaError_t mlp_radius(MlpState* s, int batch, const double* nv, bool learned, bool order, int base_mode,
                       double base_value, int n_rx, const float* R32, const float* yb32, cudaStream_t st);
// accessors (the struct is private to mlp.cu)
float* mlp_params(MlpState* s);
float* mlp_grads(MlpState* s);
float* mlp_outputs(MlpState* s);
float* mlp_r2(MlpState* s);
float* mlp_loss(MlpState* s);
int* mlp_err(MlpState* s);
int mlp_cap(MlpState* s);
int mlp_ntx(MlpState* s);
int mlp_qam(MlpState* s);
bool mlp_reduced(MlpState* s);
size_t mlp_bytes(MlpState* s);

cudaError_t launch_count_errors(int batch, int n_tx, int qam, const uint8_t* a, const uint8_t* b,
                                unsigned long long* counts, cudaStream_t s);

// ---------------------------------------------------------------------------------------
// Device helpers shared by the search kernels.

// FP32 rounding unit.
constexpr float kU32 = 5.9604645e-8f;

// Bound under which an FP32 partial distance may still belong to a point
// whose exact distance is below r2.  E is the per-vector error scale
// u * sqrt(sum_i ((n - i + 1) T_i)^2) with T_i = |ybar_i| + a_max sum_j |R_ij|:
// the absolute error of an FP32 partial distance D is at most about
// 2 sqrt(D) E + 2 n u D (first-order bound of the FMA chains).
__device__ __forceinline__ float prune_bound(float r2, float E, int n) {
  if (!(r2 < INFINITY)) return INFINITY;
  return r2 + 4.0f * sqrtf(r2) * E + 4.0f * (float)n * kU32 * r2;
}

// Warp-wide minimum of 64-bit keys (every lane gets it): the high words are
// reduced first, then the low words of the lanes holding that high word; two
// single-instruction 32-bit reductions instead of five shuffle rounds.
__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long key) {
  const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
  const unsigned mhi = __reduce_min_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_min_sync(0xffffffffu, hi == mhi ? lo : 0xffffffffu);
  return ((unsigned long long)mhi << 32) | mlo;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace mdx

namespace mdx {

// ||ybar - R x||^2 in FP64 for the PAM-index path x (n <= 224), computed by
// the calling warp (all 32 lanes) column by column: lane l accumulates the
// residual of rows l, l+32, ...  Every lane returns the same value.  Lane k < P
// holds the FP64 level (2k - (P-1)) alpha, fetched per column by a shuffle
// (an FP64 conversion and product per column would occupy the FP64 unit).
__device__ __forceinline__ double rescore_fp64_warp(int n, int P, double alpha64,
                                                     const double* __restrict__ R64,
                                                     const double* __restrict__ y64,
                                                     const uint8_t* x, int lane) {
  double rr[7];
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    const int r = lane + 32 * t;
    rr[t] = (r < n) ? y64[r] : 0.0;
  }
  const double lv = (double)(2 * (lane < P ? lane : 0) - (P - 1)) * alpha64;
  for (int j = 0; j < n; ++j) {
    const double xj = __shfl_sync(0xffffffffu, lv, (int)x[j]);
    const double* col = R64 + col_off(j);
#pragma unroll
    for (int t = 0; t < 7; ++t) {
      const int r = lane + 32 * t;
      if (r <= j) rr[t] = fma(-col[r], xj, rr[t]);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < 7; ++t) s = fma(rr[t], rr[t], s);
  return __shfl_sync(0xffffffffu, warp_sum(s), 0);
}

// FP32 error scale E of one vector (see prune_bound), computed by one warp
// from the FP32 R (column-packed, shared memory) and ybar.
__device__ __forceinline__ float error_scale_warp(int n, int P, float alpha, const float* Rc,
                                                  const float* yb, int lane) {
  const float amax = alpha * (float)(P - 1);
  float e2 = 0.0f;
  for (int r = lane; r < n; r += 32) {
    float T = fabsf(yb[r]);
    for (int j = r; j < n; ++j) T += amax * fabsf(Rc[col_off(j) + r]);
    const float w = (float)(n - r + 1) * T;
    e2 += w * w;
  }
  return __shfl_sync(0xffffffffu, sqrtf(warp_sum(e2)) * kU32, 0);
}

__host__ __device__ __forceinline__ int pow2ceil(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace mdx
