// Linear detectors, the controls the paper compares the tree searches with
// (Sec. III-A): zero forcing, x = H^+ y = R^-1 ybar (back substitution on the
// QR workspace), and MMSE, x = (H^H H + sigma^2 I)^-1 H^H y =
// (R^T R + sigma^2 I)^-1 R^T ybar on the real interleaved form (Cholesky
// factorisation and two triangular solves).  Both in FP64, one warp per
// vector, lanes over rows; every real component is then sliced to the nearest
// PAM level (clipped to the grid) and the metric ||ybar - R x^||^2 is
// evaluated in FP64 like the searches' final leaves.
#include "mdx_internal.cuh"

namespace mdx {
namespace {

constexpr int kLinWarps = 4;

__host__ __device__ inline size_t lin_warp_bytes(int n, bool mmse) {
  size_t b = sizeof(double) * (size_t)round_up(n, 2) + (size_t)round_up(n, 16);  // x, sliced path
  if (mmse) b += sizeof(double) * ((size_t)n * n + (size_t)round_up(n, 2));       // G (row-major), rhs
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ uint8_t slice_level(double x, double alpha64, int P) {
  const double u = 0.5 * (x / alpha64 + (double)(P - 1));
  double k = floor(u + 0.5);
  k = k < 0.0 ? 0.0 : (k > (double)(P - 1) ? (double)(P - 1) : k);
  return (uint8_t)k;
}

// Back substitution R x = rhs (R column-packed upper triangular, FP64).
// rhs in x on entry, the solution on return; lanes own rows.
__device__ void back_substitute(int n, const double* R, double* x, int lane) {
  for (int i = n - 1; i >= 0; --i) {
    __syncwarp();
    const double xi = x[i] / R[col_off(i) + i];
    __syncwarp();
    const double* col = R + col_off(i);
    for (int r = lane; r < i; r += 32) x[r] = fma(-col[r], xi, x[r]);
    if (lane == 0) x[i] = xi;
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kLinWarps * 32) linear_kernel(SearchArgs a, int mmse) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.n, P = a.P;
  unsigned char* base = smem + (size_t)warp * lin_warp_bytes(n, mmse != 0);
  double* x = reinterpret_cast<double*>(base);
  uint8_t* path = reinterpret_cast<uint8_t*>(x + round_up(n, 2));
  double* G = reinterpret_cast<double*>(path + round_up(n, 16));  // MMSE only
  double* rhs = G + (size_t)n * n;
  const int gw = blockIdx.x * kLinWarps + warp, nw = gridDim.x * kLinWarps;
  for (int v = gw; v < a.batch; v += nw) {
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
    const double* R = a.R64 + (size_t)v * tri_stride64(n);
    const double* yb = a.yb64 + (size_t)v * vec_stride64(n);
    if (!mmse) {
      for (int r = lane; r < n; r += 32) x[r] = yb[r];
      back_substitute(n, R, x, lane);
    } else {
      const double s2 = a.noise_var[v];
      // G = R^T R + sigma^2 I (lower triangle), rhs = R^T ybar
      for (int e = lane; e < n * n; e += 32) {
        const int i = e / n, j = e % n;
        if (j > i) continue;
        const double* ci = R + col_off(i);
        const double* cj = R + col_off(j);
        double g = (i == j) ? s2 : 0.0;
        for (int k = 0; k <= j; ++k) g = fma(ci[k], cj[k], g);
        G[e] = g;
      }
      for (int i = lane; i < n; i += 32) {
        const double* ci = R + col_off(i);
        double b = 0.0;
        for (int k = 0; k <= i; ++k) b = fma(ci[k], yb[k], b);
        rhs[i] = b;
      }
      __syncwarp();
      // Cholesky G = L L^T in place (lower triangle), column by column
      for (int k = 0; k < n; ++k) {
        const double d = sqrt(G[k * n + k]);
        __syncwarp();
        for (int i = k + 1 + lane; i < n; i += 32) G[i * n + k] /= d;
        if (lane == 0) G[k * n + k] = d;
        __syncwarp();
        for (int e = lane; e < (n - k - 1) * (n - k - 1); e += 32) {
          const int i = k + 1 + e / (n - k - 1), j = k + 1 + e % (n - k - 1);
          if (j <= i) G[i * n + j] = fma(-G[i * n + k], G[j * n + k], G[i * n + j]);
        }
        __syncwarp();
      }
      // L z = rhs, then L^T x = z
      for (int i = 0; i < n; ++i) {
        const double zi = rhs[i] / G[i * n + i];
        __syncwarp();
        for (int r = i + 1 + lane; r < n; r += 32) rhs[r] = fma(-G[r * n + i], zi, rhs[r]);
        if (lane == 0) rhs[i] = zi;
        __syncwarp();
      }
      for (int i = n - 1; i >= 0; --i) {
        const double xi = rhs[i] / G[i * n + i];
        __syncwarp();
        for (int r = lane; r < i; r += 32) rhs[r] = fma(-G[i * n + r], xi, rhs[r]);
        if (lane == 0) rhs[i] = xi;
        __syncwarp();
      }
      for (int r = lane; r < n; r += 32) x[r] = rhs[r];
      __syncwarp();
    }
    for (int r = lane; r < n; r += 32) path[r] = slice_level(x[r], a.alpha64, P);
    __syncwarp();
    const double m = rescore_fp64_warp(n, P, a.alpha64, R, yb, path, lane);
    for (int j = lane; j < a.n_tx; j += 32)
      a.sym_out[(size_t)v * a.n_tx + j] = (uint8_t)(path[2 * j] * P + path[2 * j + 1]);
    if (lane == 0) {
      a.metric_out[v] = m;
      a.vstatus[v] = MDX_V_OK;
      if (a.stats) {
        int64_t* s = a.stats + (size_t)v * kStats;
        s[0] = 0;
        s[1] = 0;
        s[2] = 0;
        s[3] = 1;
        s[4] = 0;
      }
    }
    __syncwarp();
  }
}

}  // namespace

size_t linear_smem_bytes(int n, bool mmse) { return lin_warp_bytes(n, mmse) * kLinWarps; }

cudaError_t launch_linear(const SearchArgs& a, bool mmse, int num_sms, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  const size_t smem = linear_smem_bytes(a.n, mmse);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(linear_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, linear_kernel, kLinWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)per_sm * num_sms;
  const long long need = (a.batch + kLinWarps - 1) / kLinWarps;
  if (grid > need) grid = need;
  linear_kernel<<<(int)grid, kLinWarps * 32, smem, s>>>(a, mmse ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace mdx
