// Batched FP64 QR preprocessing (Sec. III-B): H = QR with a real positive
// diagonal and ybar = Q^H y, by complex Householder reflections applied to the
// augmented matrix [H | y] held in shared memory.  One CTA per matrix; the
// CTA's lanes are split into column workers of LPC lanes each (LPC = 16 for
// n_rx <= 16, else 32): worker 0 forms the reflector of column k, then every
// worker applies it to its share of the remaining columns.  The complex R is
// written out in the real interleaved form (entry r_ab -> [[Re,-Im],[Im,Re]])
// that the tree search uses.
#include "mdx_internal.cuh"

namespace mdx {
namespace {

template <int LPC>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int o = LPC / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Output bases of one matrix (any pointer may be null).
struct QrDst {
  double* R64;
  double* yb64;
  float* R32;
  float* yb32;
  double* Rdense;
  double* ybdense;
  int* singular;
};

// Factorises one [H | y] (N x M complex, row-major; y of N) with the calling CTA.
template <int LPC>
__device__ void qr_one(int N, int M, const double2* __restrict__ Hb, const double2* __restrict__ yb,
                       const QrDst& out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* A = reinterpret_cast<double2*>(smem_raw);  // column-major, (M+1) columns of N
  double2* alpha = A + (size_t)(M + 1) * N;           // R_kk before the phase fix
  double* tau = reinterpret_cast<double*>(alpha + M);
  int* sing = reinterpret_cast<int*>(tau + M);

  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const int lane_g = tid % LPC;  // lane within the column worker
  const int worker = tid / LPC;
  const int nworkers = nthr / LPC;

  // load [H | y] (global row-major complex) into column-major smem
  for (int t = tid; t < N * M; t += nthr) {
    const int r = t / M, c = t % M;
    A[(size_t)c * N + r] = Hb[t];
  }
  for (int r = tid; r < N; r += nthr) A[(size_t)M * N + r] = yb[r];
  if (tid == 0) *sing = 0;
  __syncthreads();

  for (int k = 0; k < M; ++k) {
    double2* col = A + (size_t)k * N;
    if (tid < 32) {
      // warp 0 forms the reflector; with LPC = 16 both half-warps compute the
      // same sums, so full-warp shuffles stay uniform
      double s = 0.0;
      for (int i = k + lane_g; i < N; i += LPC) s += col[i].x * col[i].x + col[i].y * col[i].y;
      s = group_sum<LPC>(s);
      const double sigma = sqrt(s);
      const double2 x0 = col[k];
      const double ax0 = hypot(x0.x, x0.y);
      double2 al;
      double t = 0.0;
      if (sigma == 0.0) {
        al = make_double2(0.0, 0.0);
      } else {
        // alpha = -e^{i arg x0} sigma keeps v_0 = x0 - alpha free of cancellation
        const double2 ph = (ax0 > 0.0) ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
        al = make_double2(-ph.x * sigma, -ph.y * sigma);
        t = 1.0 / (sigma * (sigma + ax0));  // 2 / ||v||^2
      }
      __syncwarp();
      if (tid == 0) {
        alpha[k] = al;
        tau[k] = t;
        if (sigma == 0.0) *sing = 1;
        col[k] = make_double2(x0.x - al.x, x0.y - al.y);  // v_0; v_i = col[i] for i > k
      }
    }
    __syncthreads();
    const double t = tau[k];
    if (t != 0.0) {
      // every lane of a warp runs the same number of iterations (shuffles inside)
      for (int base = k + 1; base <= M; base += nworkers) {
        const int j = base + worker;
        const bool act = j <= M;
        double2* cj = A + (size_t)(act ? j : M) * N;
        double wr = 0.0, wi = 0.0;  // w = v^H a_j
        if (act) {
          for (int i = k + lane_g; i < N; i += LPC) {
            const double2 v = col[i], a = cj[i];
            wr += v.x * a.x + v.y * a.y;
            wi += v.x * a.y - v.y * a.x;
          }
        }
        wr = group_sum<LPC>(wr) * t;
        wi = group_sum<LPC>(wi) * t;
        if (act) {
          for (int i = k + lane_g; i < N; i += LPC) {
            const double2 v = col[i];
            double2 a = cj[i];
            a.x -= v.x * wr - v.y * wi;
            a.y -= v.x * wi + v.y * wr;
            cj[i] = a;
          }
        }
      }
    }
    __syncthreads();
  }

  // phase fix: row k of R and ybar_k times conj(alpha_k / |alpha_k|), R_kk = |alpha_k|
  const int n = 2 * M;
  const int nb = M * (M + 1) / 2;  // complex entries (a, c) with a <= c
  for (int t = tid; t < nb; t += nthr) {
    // unrank t -> (a, c), a <= c, column-major over c
    int c = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (c * (c + 1) / 2 > t) --c;
    while ((c + 1) * (c + 2) / 2 <= t) ++c;
    const int a = t - c * (c + 1) / 2;
    const double2 al = alpha[a];
    const double aa = hypot(al.x, al.y);
    const double2 ph = (aa > 0.0) ? make_double2(al.x / aa, al.y / aa) : make_double2(1.0, 0.0);
    double re, im;
    if (a == c) {
      re = aa;
      im = 0.0;
    } else {
      const double2 r = A[(size_t)c * N + a];
      re = r.x * ph.x + r.y * ph.y;  // r * conj(ph)
      im = r.y * ph.x - r.x * ph.y;
    }
    const int r0 = 2 * a, c0 = 2 * c;
    // the 2x2 block [[re, -im], [im, re]] at rows r0..r0+1, columns c0..c0+1
    const double vals[4] = {re, -im, im, re};
    const int rows[4] = {r0, r0, r0 + 1, r0 + 1};
    const int cols[4] = {c0, c0 + 1, c0, c0 + 1};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int rr = rows[e], cc = cols[e];
      if (rr > cc) continue;  // below the diagonal (only in diagonal blocks)
      const double v = vals[e];
      if (out.R64) out.R64[col_off(cc) + rr] = v;
      if (out.R32) out.R32[col_off(cc) + rr] = (float)v;
      if (out.Rdense) out.Rdense[(size_t)rr * n + cc] = v;
    }
  }
  if (out.Rdense) {
    // zero the rest of the lower triangle
    for (int t = tid; t < n * n; t += nthr) {
      const int rr = t / n, cc = t % n;
      if (rr > cc) out.Rdense[t] = 0.0;
    }
  }
  for (int a = tid; a < M; a += nthr) {
    const double2 al = alpha[a];
    const double aa = hypot(al.x, al.y);
    const double2 ph = (aa > 0.0) ? make_double2(al.x / aa, al.y / aa) : make_double2(1.0, 0.0);
    const double2 r = A[(size_t)M * N + a];
    const double re = r.x * ph.x + r.y * ph.y, im = r.y * ph.x - r.x * ph.y;
    if (out.yb64) {
      out.yb64[2 * a] = re;
      out.yb64[2 * a + 1] = im;
    }
    if (out.yb32) {
      out.yb32[2 * a] = (float)re;
      out.yb32[2 * a + 1] = (float)im;
    }
    if (out.ybdense) {
      out.ybdense[2 * a] = re;
      out.ybdense[2 * a + 1] = im;
    }
  }
  if (out.singular && tid == 0) *out.singular = *sing;
}

template <int LPC>
__global__ void qr_kernel(int batch, int N, int M, const double* __restrict__ H,
                          const double* __restrict__ y, QrOut out) {
  const int b = blockIdx.x;
  if (b >= batch) return;
  const int n = 2 * M;
  QrDst d;
  d.R64 = out.R64 ? out.R64 + (size_t)b * tri_stride64(n) : nullptr;
  d.yb64 = out.yb64 ? out.yb64 + (size_t)b * vec_stride64(n) : nullptr;
  d.R32 = out.R32 ? out.R32 + (size_t)b * tri_stride32(n) : nullptr;
  d.yb32 = out.yb32 ? out.yb32 + (size_t)b * vec_stride32(n) : nullptr;
  d.Rdense = out.Rdense ? out.Rdense + (size_t)b * n * n : nullptr;
  d.ybdense = out.ybdense ? out.ybdense + (size_t)b * n : nullptr;
  d.singular = out.singular ? out.singular + b : nullptr;
  qr_one<LPC>(N, M, reinterpret_cast<const double2*>(H) + (size_t)b * N * M,
              reinterpret_cast<const double2*>(y) + (size_t)b * N, d);
}

// One CTA per listed request of an uneven batch (all of one n_rx x n_tx);
// inputs and outputs at the request's own offsets.
template <int LPC>
__global__ void qr_gather_kernel(int count, const int* __restrict__ ids, const MixedReq* __restrict__ reqs,
                                 const double* __restrict__ H, const double* __restrict__ y, QrOut out) {
  if ((int)blockIdx.x >= count) return;
  const int r = ids[blockIdx.x];
  const MixedReq q = reqs[r];
  QrDst d{out.R64 + q.r_off, out.yb64 + q.y_off, out.R32 + q.r_off, out.yb32 + q.y_off, nullptr, nullptr,
          out.singular + r};
  qr_one<LPC>(q.n_rx, q.n_tx, reinterpret_cast<const double2*>(H + q.h_off),
              reinterpret_cast<const double2*>(y + q.yin_off), d);
}

size_t qr_smem(int n_rx, int n_tx) {
  return sizeof(double2) * ((size_t)(n_tx + 1) * n_rx + n_tx) + sizeof(double) * n_tx + sizeof(int) * 4;
}

}  // namespace

cudaError_t launch_qr_gather(int count, int n_rx, int n_tx, const int* ids, const MixedReq* reqs,
                             const double* H, const double* y, QrOut out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = qr_smem(n_rx, n_tx);
  if (n_rx <= 16) {
    cudaFuncSetAttribute(qr_gather_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    qr_gather_kernel<16><<<count, 32, smem, s>>>(count, ids, reqs, H, y, out);
  } else {
    const int threads = n_tx <= 32 ? 128 : 256;
    cudaFuncSetAttribute(qr_gather_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    qr_gather_kernel<32><<<count, threads, smem, s>>>(count, ids, reqs, H, y, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_qr(int batch, int n_rx, int n_tx, const double* H, const double* y, QrOut out,
                      cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  const size_t smem = qr_smem(n_rx, n_tx);
  if (n_rx <= 16) {
    // two 16-lane workers per warp
    cudaFuncSetAttribute(qr_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    qr_kernel<16><<<batch, 32, smem, s>>>(batch, n_rx, n_tx, H, y, out);
  } else {
    const int threads = n_tx <= 32 ? 128 : 256;
    cudaFuncSetAttribute(qr_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    qr_kernel<32><<<batch, threads, smem, s>>>(batch, n_rx, n_tx, H, y, out);
  }
  return cudaGetLastError();
}

}  // namespace mdx
