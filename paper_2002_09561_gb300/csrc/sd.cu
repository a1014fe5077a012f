// Exact sphere decoder (Sec. III-B, Algorithm 1) with Best-FS /
// Schnorr-Euchner child order (Sec. IV-A) and incremental partial distances
// (Sec. IV-C, Eq. inc), one warp per received vector.
//
// Mapping.  Lane l owns the rows r = l + 32 t (t < ROWS).  For the node at
// level i (rows n-1..i+1 fixed) the residual of every lower row,
//   z_r = ybar_r - sum_{j > i} R_rj x_j   (r <= i),
// sits in a shared-memory stack zs[level i][r]; descending into child x_i = a
// costs one FMA per row below (z_r -= R_ri a), and the interference of row i
// is simply c_i = z_i.  Each partial distance is built by one FMA chain in a
// fixed order (j = n-1 down to i+1), so FP32 results do not depend on the
// warp's reduction shape.  The control state of the current level (parent
// partial distance, c_i, zig-zag pointers) is warp-uniform and lives in
// registers; it is pushed to shared memory on descent and popped on
// backtrack.
//
// Children are visited in increasing (c_i - R_ii a_k)^2 by a zig-zag around
// u_i = c_i / (R_ii alpha) in PAM-index space, ties to the lower index; a
// child whose partial distance reaches the pruning bound ends the level (all
// later children are farther).  A leaf inside the bound shrinks the radius
// and is recorded in a small candidate list; at the end the candidates within
// FP32 error of the best are re-scored in FP64 against the FP64 R and ybar.
// Vectors are taken from a global counter, so a warp that finishes an easy
// vector immediately starts the next one.
#include "mdx_internal.cuh"

namespace mdx {
namespace {

constexpr int kWarps = 4;  // warps per CTA
constexpr int kCand = 8;   // leaf candidates kept per vector

__host__ __device__ inline int path_pad(int n) { return round_up(n, 16); }

// Shared-memory bytes per warp for real dimension n, a multiple of 16 so that
// every warp's region (staged with 16-byte vector stores) starts aligned.
__host__ __device__ inline size_t sd_warp_bytes(int n) {
  const size_t b = sizeof(float) * (2 * (size_t)tri_stride32(n) + 4 * (size_t)n + kCand) +
                   sizeof(int) * (size_t)n + (size_t)path_pad(n) * (1 + kCand);
  return (b + 15) / 16 * 16;
}

template <int ROWS>
__global__ void __launch_bounds__(kWarps * 32) sd_kernel(SearchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.n, P = a.P;
  (void)kWarps;
  const int ts = tri_stride32(n);
  unsigned char* base = smem + warp * sd_warp_bytes(n);
  float* Rc = reinterpret_cast<float*>(base);  // column-packed R (FP32)
  float* zs = Rc + ts;                          // residual stack, level i at col_off(i)
  float* lv_ped = zs + ts;                      // per level: parent partial distance
  float* lv_c = lv_ped + n;                     // c_i
  float* lv_u = lv_c + n;                       // u_i
  float* lv_rinv = lv_u + n;                    // 1 / (2 alpha R_ii)
  float* cand_ped = lv_rinv + n;                // kCand
  int* lv_lohi = reinterpret_cast<int*>(cand_ped + kCand);
  uint8_t* xs = reinterpret_cast<uint8_t*>(lv_lohi + n);  // current path
  uint8_t* cand_x = xs + path_pad(n);                       // kCand paths
  const int pp = path_pad(n);
  const float alpha = a.alpha;
  const float uoff = 0.5f * (float)(P - 1);
  const float amax = alpha * (float)(P - 1);

  for (;;) {
    int v = 0;
    if (lane == 0) v = (int)atomicAdd(a.work_counter, 1u);
    v = __shfl_sync(0xffffffffu, v, 0);
    if (v >= a.batch) break;

    if (a.singular && a.singular[v]) {
      for (int j = lane; j < a.n_tx; j += 32) a.sym_out[(size_t)v * a.n_tx + j] = 0;
      if (lane == 0) {
        a.metric_out[v] = 0.0;
        a.vstatus[v] = MDX_V_SINGULAR;
        if (a.stats)
          for (int q = 0; q < kStats; ++q) a.stats[(size_t)v * kStats + q] = 0;
      }
      continue;
    }

    // stage R (FP32) and the top residual level (= ybar)
    const float4* src = reinterpret_cast<const float4*>(a.R32 + (size_t)v * ts);
    for (int t = lane; t < ts / 4; t += 32) reinterpret_cast<float4*>(Rc)[t] = src[t];
    const float* yb = a.yb32 + (size_t)v * vec_stride32(n);
    for (int r = lane; r < n; r += 32) zs[col_off(n - 1) + r] = yb[r];
    __syncwarp();
    for (int r = lane; r < n; r += 32) lv_rinv[r] = 0.5f / (alpha * Rc[col_off(r) + r]);

    // FP32 error scale of this vector (see prune_bound)
    float e2 = 0.0f;
#pragma unroll
    for (int t = 0; t < ROWS; ++t) {
      const int r = lane + 32 * t;
      if (r < n) {
        float T = fabsf(yb[r]);
        for (int j = r; j < n; ++j) T += amax * fabsf(Rc[col_off(j) + r]);
        const float w = (float)(n - r + 1) * T;
        e2 += w * w;
      }
    }
    // broadcast so that every lane takes identical pruning decisions
    const float E = __shfl_sync(0xffffffffu, sqrtf(warp_sum(e2)) * kU32, 0);

    float r2;
    if (a.radius_mode == RADIUS_NONE) r2 = INFINITY;
    else if (a.radius_mode == RADIUS_PAPER) r2 = (float)((double)a.n_rx * a.n_tx * a.noise_var[v]);
    else if (a.radius_mode == RADIUS_PER_VECTOR) r2 = a.r2_vec[v];
    else r2 = (float)a.radius_value;
    if (!(r2 > 0.0f)) r2 = INFINITY;  // zero or NaN radius: search without one

    long long nodes = 0, peds = 0, restarts = 0, flops = 0;
    int ncand = 0;
    bool budget_hit = false;
    float best = INFINITY;
    __syncwarp();

    for (;;) {  // radius-doubling loop
      float bnd = prune_bound(r2, E, n);
      int i = n - 1;
      float ped_par = 0.0f;
      float c = zs[col_off(n - 1) + n - 1];
      float rii = Rc[col_off(n - 1) + n - 1];
      float u = fmaf(c, lv_rinv[n - 1], uoff);
      int lo = min(max((int)ceilf(u - 0.5f), 0), P - 1);
      int hi = lo + 1;
      nodes += 1;
      for (;;) {
        // next child of the node at level i in Schnorr-Euchner order
        int k = -1;
        if (lo >= 0 || hi < P) {
          if (hi >= P || (lo >= 0 && fabsf(u - (float)lo) <= fabsf((float)hi - u))) k = lo--;
          else k = hi++;
        }
        float ped = INFINITY;
        if (k >= 0) {
          const float d = fmaf(-rii, (float)(2 * k - (P - 1)) * alpha, c);
          ped = fmaf(d, d, ped_par);
          ++peds;
        }
        if (k < 0 || !(ped < bnd)) {
          if (i == n - 1) break;  // root exhausted
          ++i;                    // backtrack: pop level i
          ped_par = lv_ped[i];
          c = lv_c[i];
          u = lv_u[i];
          const int lh = lv_lohi[i];
          lo = (lh & 0xffff) - 1;
          hi = lh >> 16;
          rii = Rc[col_off(i) + i];
          continue;
        }
        if (i == 0) {
          // leaf inside the sphere: record it, shrink the radius (Alg. 1)
          if (lane == 0) xs[0] = (uint8_t)k;
          __syncwarp();
          int slot = -1;
          if (ncand < kCand) {
            slot = ncand++;
          } else {
            float worst = -1.0f;
            for (int q = 0; q < kCand; ++q)
              if (cand_ped[q] > worst) {
                worst = cand_ped[q];
                slot = q;
              }
            if (!(ped < worst)) slot = -1;
          }
          if (slot >= 0) {
            for (int r = lane; r < n; r += 32) cand_x[slot * pp + r] = xs[r];
            if (lane == 0) cand_ped[slot] = ped;
          }
          __syncwarp();
          if (ped < best) best = ped;
          if (ped < r2) {
            r2 = ped;
            bnd = prune_bound(r2, E, n);
          }
          continue;
        }
        if (a.budget > 0 && nodes >= a.budget) {
          budget_hit = true;
          break;
        }
        // descend into child k: push level i, update the residuals of the rows below
        const float av = (float)(2 * k - (P - 1)) * alpha;
        if (lane == 0) {
          lv_ped[i] = ped_par;
          lv_c[i] = c;
          lv_u[i] = u;
          lv_lohi[i] = (lo + 1) | (hi << 16);
          xs[i] = (uint8_t)k;
        }
        const float* zin = zs + col_off(i);
        float* zout = zs + col_off(i - 1);
        const float* rc = Rc + col_off(i);
#pragma unroll
        for (int t = 0; t < ROWS; ++t) {
          const int r = lane + 32 * t;
          if (r < i) zout[r] = fmaf(-rc[r], av, zin[r]);
        }
        __syncwarp();
        --i;
        ped_par = ped;
        c = zout[i];
        rii = Rc[col_off(i) + i];
        u = fmaf(c, lv_rinv[i], uoff);
        lo = min(max((int)ceilf(u - 0.5f), 0), P - 1);
        hi = lo + 1;
        ++nodes;
        flops += 2 * (n - 1 - i) + 4 * P;
      }
      if (ncand > 0 || budget_hit || !(r2 < INFINITY) || restarts >= 64) break;
      r2 *= 4.0f;  // empty sphere: double the radius and search again
      ++restarts;
    }

    // FP64 re-scoring of the candidates within FP32 error of the best
    const double* R64 = a.R64 + (size_t)v * tri_stride64(n);
    const double* y64 = a.yb64 + (size_t)v * vec_stride64(n);
    const float keep = prune_bound(best, E, n);
    const double alpha64 = a.alpha64;
    int win = -1;
    double win_m = INFINITY;
    long long rescored = 0;
    for (int q = 0; q < ncand; ++q) {
      if (!(cand_ped[q] <= keep)) continue;
      double m;
      if (a.flags & MDX_NO_RESCORE) {
        m = (double)cand_ped[q];
      } else {
        double rr[ROWS];
#pragma unroll
        for (int t = 0; t < ROWS; ++t) {
          const int r = lane + 32 * t;
          rr[t] = (r < n) ? y64[r] : 0.0;
        }
        for (int j = 0; j < n; ++j) {
          const double xj = (double)(2 * (int)cand_x[q * pp + j] - (P - 1)) * alpha64;
          const double* col = R64 + col_off(j);
#pragma unroll
          for (int t = 0; t < ROWS; ++t) {
            const int r = lane + 32 * t;
            if (r <= j) rr[t] = fma(-col[r], xj, rr[t]);
          }
        }
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < ROWS; ++t) s = fma(rr[t], rr[t], s);
        m = __shfl_sync(0xffffffffu, warp_sum(s), 0);
        ++rescored;
      }
      bool better = m < win_m;
      if (!better && m == win_m && win >= 0) {
        // tie: lexicographically smaller index vector, top row first
        for (int j = n - 1; j >= 0; --j) {
          const int x1 = cand_x[q * pp + j], x2 = cand_x[win * pp + j];
          if (x1 != x2) {
            better = x1 < x2;
            break;
          }
        }
      }
      if (better) {
        win = q;
        win_m = m;
      }
    }

    for (int j = lane; j < a.n_tx; j += 32) {
      uint8_t s = 0;
      if (win >= 0) s = (uint8_t)(cand_x[win * pp + 2 * j] * P + cand_x[win * pp + 2 * j + 1]);
      a.sym_out[(size_t)v * a.n_tx + j] = s;
    }
    if (lane == 0) {
      a.metric_out[v] = (win >= 0) ? win_m : (double)INFINITY;
      a.vstatus[v] = budget_hit ? MDX_V_BUDGET_EXCEEDED : (restarts > 0 ? MDX_V_EMPTY_RETRIED : MDX_V_OK);
      if (a.stats) {
        a.stats[(size_t)v * kStats + 0] = nodes;
        a.stats[(size_t)v * kStats + 1] = peds;
        a.stats[(size_t)v * kStats + 2] = restarts;
        a.stats[(size_t)v * kStats + 3] = rescored;
        a.stats[(size_t)v * kStats + 4] = flops;
      }
    }
    __syncwarp();
  }
}

template <int ROWS>
cudaError_t launch_rows(const SearchArgs& a, int num_sms, cudaStream_t s) {
  // as many warps per CTA (up to kWarps) as fit in 200 KB of shared memory
  int wpc = (int)((200u * 1024u) / sd_warp_bytes(a.n));
  if (wpc > kWarps) wpc = kWarps;
  if (wpc < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = sd_warp_bytes(a.n) * wpc;
  cudaError_t e = cudaFuncSetAttribute(sd_kernel<ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sd_kernel<ROWS>, wpc * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = per_sm * num_sms;
  const int need = (a.batch + wpc - 1) / wpc;
  if (grid > need) grid = need;
  sd_kernel<ROWS><<<grid, wpc * 32, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sd(const SearchArgs& a, int num_sms, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  if (a.n <= 32) return launch_rows<1>(a, num_sms, s);
  if (a.n <= 64) return launch_rows<2>(a, num_sms, s);
  if (a.n <= 128) return launch_rows<4>(a, num_sms, s);
  return launch_rows<7>(a, num_sms, s);
}

}  // namespace mdx
