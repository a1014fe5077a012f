// Batched FP64 QR preprocessing (Sec. III-B): H = QR with a real positive
// diagonal and ybar = Q^H y, by complex Householder reflections applied to the
// augmented matrix [H | y].  Three forms: up to 32 receive antennas, several
// matrices per warp held in registers (qr_small_kernel, below); beyond that one
// CTA per matrix in shared memory, either with column workers of 32 lanes
// (qr_kernel: worker 0 forms the reflector of column k, then every worker
// applies it to its share of the remaining columns) or, from 48 transmit
// antennas, blocked with FP64 MMA trailing updates (qr_dmma_kernel).  The
// complex R is written out in the real interleaved form (entry r_ab ->
// [[Re,-Im],[Im,Re]]) that the tree search uses.
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

// Phase fix and output of a factorised [R | ybar]: row k of R and ybar_k are
// multiplied by conj(alpha_k / |alpha_k|) so that R_kk = |alpha_k| > 0; R is
// written in the real interleaved form (entry r_ab -> [[Re,-Im],[Im,Re]]).
// getA(c, r) returns the complex entry of column c, row r (r < c for R, the
// ybar column is c = M).
// alpha and tau are overwritten: alpha_k by its phase alpha_k / |alpha_k|
// (1 if zero) and tau_k by |alpha_k|.
template <typename GetA>
__device__ void qr_writeout(int M, GetA getA, double2* alpha, double* tau, const QrDst& out) {
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  for (int a = tid; a < M; a += nthr) {
    const double2 al = alpha[a];
    const double aa = hypot(al.x, al.y);
    alpha[a] = (aa > 0.0) ? make_double2(al.x / aa, al.y / aa) : make_double2(1.0, 0.0);
    tau[a] = aa;
  }
  __syncthreads();
  const int n = 2 * M;
  const int nb = M * (M + 1) / 2;  // complex entries (a, c) with a <= c
  for (int t = tid; t < nb; t += nthr) {
    // unrank t -> (a, c), a <= c, column-major over c
    int c = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);  // exact after the corrections below
    while (c * (c + 1) / 2 > t) --c;
    while ((c + 1) * (c + 2) / 2 <= t) ++c;
    const int a = t - c * (c + 1) / 2;
    const double2 ph = alpha[a];
    const double aa = tau[a];
    double re, im;
    if (a == c) {
      re = aa;
      im = 0.0;
    } else {
      const double2 r = getA(c, a);
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
    const double2 ph = alpha[a];
    const double2 r = getA(M, a);
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
}

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

  qr_writeout(M, [&](int c, int r) { return A[(size_t)c * N + r]; }, alpha, tau, out);
  if (out.singular && tid == 0) *out.singular = *sing;
}

// ---------------------------------------------------------------------------
// Blocked Householder QR with the trailing updates on the FP64 tensor cores.
//
// Measured on this GPU: an m8n8k4 FP64 MMA occupies a scheduler's FP64 unit
// for about 585 cycles (256 FMA) and an FP64 FMA instruction for about 75
// (32 FMA), so the MMA path is not faster per FMA; it wins (for n_tx >= 48)
// because the block update needs no cross-lane reductions, and loses to
// qr_one on small matrices, where the panel dominates.
//
// Same reflectors as qr_one (H_k = I - tau_k v_k v_k^H, tau_k real), taken in
// panels of 8 columns.  On this GPU an FP64 instruction of one warp occupies
// its scheduler's FP64 unit for tens of cycles, so the level-2 panel is
// spread over four warps, one per scheduler, each holding 32 rows of the
// panel in registers (lane = row); column sums are warp reductions plus one
// exchange through shared memory.  The panel also builds Y = V T, the
// compact-WY form H_k ... H_{k+7} = I - V T V^H (Y_j = tau_j (v_j -
// Y[:, 0:j] (V[:, 0:j]^H v_j)), T_jj = tau_j), so that the columns right of
// the panel are updated as A_t <- A_t - V (Y^H A_t) in two FP64 MMA steps
// (mma.sync m8n8k4 .f64; complex products as four real ones), 8 columns per
// warp task.  Matrices live in shared memory as separate real and imaginary
// planes, column-major with a column stride of N8 + 4 doubles (N8 = N
// rounded up to 8), zero-padded to N8 rows and C8 = round_up(M + 1, 8)
// columns, so the MMA tiles need no masks; the padding stays zero.

constexpr int kQrdWarps = 8;  // per CTA where one matrix fills the SM's shared memory, else 4 (two CTAs per SM)
constexpr int kPanelWarps = 4;
constexpr int kTileStride = 12;                     // doubles per column of a warp's 8 x 8 tile
constexpr int kTileDoubles = 2 * 8 * kTileStride;  // one W tile: real plane, then imaginary plane

// Shared memory of one matrix: A = [H | y] as real and imaginary planes; two
// Y = V T buffers (the panel being applied and the one being factored); the
// W tiles of the trailing update; panel reduction scratch; alpha, tau.  V is
// not stored separately: below the diagonal of its panel columns A holds it.
struct QrdLayout {
  int N8, C8, S;
  size_t off_are, off_aim, off_y[2], off_tile, off_red, off_alpha, off_tau, off_sing, bytes;
  __host__ __device__ void init(int N, int M) {
    N8 = round_up(N, 8);
    C8 = round_up(M + 1, 8);
    S = N8 + 4;
    size_t o = 0;
    auto take = [&](size_t bytes) {
      const size_t at = o;
      o += (bytes + 15) / 16 * 16;
      return at;
    };
    off_are = take(sizeof(double) * (size_t)C8 * S);
    off_aim = take(sizeof(double) * (size_t)C8 * S);
    off_y[0] = take(sizeof(double) * 16 * (size_t)S);  // Y re: 8 columns of stride S, then Y im
    off_y[1] = take(sizeof(double) * 16 * (size_t)S);
    off_tile = take(sizeof(double) * kTileDoubles * (C8 / 8));
    off_red = take(sizeof(double) * (8 + 2 * 16 * kPanelWarps));
    off_alpha = take(sizeof(double2) * (size_t)M);
    off_tau = take(sizeof(double) * (size_t)M);
    off_sing = take(16);
    bytes = o;
  }
};

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// Sign flip on the integer pipe: an FP64 negation would occupy the FP64 unit,
// which the MMAs around it share.
__device__ __forceinline__ double ineg(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void panel_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kPanelWarps * 32)); }
__device__ __forceinline__ void update_sync(int threads) { asm volatile("bar.sync 2, %0;" ::"r"(threads)); }

// Conversions between a positive normal double in [1e-30, 1e30] and a float
// estimate of it, done on the integer pipe (rebias the exponent, keep the top
// 23 fraction bits): an FP64 conversion would occupy the FP64 unit.
__device__ __forceinline__ float f32_estimate(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = ((hi >> 20) & 0x7ffu) - 1023u + 127u;
  return __uint_as_float((e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
__device__ __forceinline__ double f64_of(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = ((b >> 23) & 0xffu) - 127u + 1023u;
  return __hiloint2double((int)((e << 20) | ((b & 0x7fffffu) >> 3)), (int)((b & 7u) << 29));
}

// 1 / sqrt(x) for a positive x: a single-precision estimate y0 (relative
// error below 2^-21) refined by one third-order step of the binomial series
// (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + O(e^3), e = 1 - x y0^2 (error below
// 2^-60 before rounding).
__device__ __forceinline__ double rsqrt64(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  const double y = f64_of(rsqrtf(f32_estimate(x)));
  const double e = fma(-(x * y), y, 1.0);
  return fma(y, e * fma(0.375, e, 0.5), y);
}
// 1 / d for a positive d: single-precision estimate refined by one
// third-order step of 1 / (1 - e) = 1 + e + e^2 + O(e^3), e = 1 - d y0.
__device__ __forceinline__ double rcp64(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / d;
  const double y = f64_of(__frcp_rn(f32_estimate(d)));
  const double e = fma(-d, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// Sum of 16 per-lane values over the warp, scattered: on return lane l holds
// the total of value (l >> 1) & 15 (16 additions instead of 80).
__device__ __forceinline__ double reduce_scatter16(double (&v)[16], int lane) {
  double a8[8], a4[4], a2[2];
  {
    const bool h = (lane >> 4) & 1;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const double keep = h ? v[8 + m] : v[m], give = h ? v[m] : v[8 + m];
      a8[m] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
  }
  {
    const bool h = (lane >> 3) & 1;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const double keep = h ? a8[4 + m] : a8[m], give = h ? a8[m] : a8[4 + m];
      a4[m] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
  }
  {
    const bool h = (lane >> 2) & 1;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const double keep = h ? a4[2 + m] : a4[m], give = h ? a4[m] : a4[2 + m];
      a2[m] = keep + __shfl_xor_sync(0xffffffffu, give, 4);
    }
  }
  const bool h = (lane >> 1) & 1;
  const double keep = h ? a2[1] : a2[0], give = h ? a2[0] : a2[1];
  double a1 = keep + __shfl_xor_sync(0xffffffffu, give, 2);
  return a1 + __shfl_xor_sync(0xffffffffu, a1, 1);
}

// Sum of the first nlw of four per-warp partials p[0], p[stride], ...
__device__ __forceinline__ double sum_live(const double* p, int stride, int nlw) {
  if (nlw == 2) return p[0] + p[stride];
  if (nlw == 3) return (p[0] + p[stride]) + p[2 * stride];
  return (p[0] + p[stride]) + (p[2 * stride] + p[3 * stride]);
}

// Factors the panel of columns k..k+7 (bw of them are reflector columns) with
// warps 0..3, lane = row k + 32 warp + lane.  Writes the panel back (R above
// the diagonal, the reflectors' first entries on it and V below it) and
// Y = V T into Yb.  Warps without rows in the panel (32 warp >= N8 - k) skip
// every FP64 instruction; with one live warp the panel needs no shared-memory
// exchange at all.
__device__ void qrd_panel(const QrdLayout& L, int k, int bw, double* Are, double* Aim, double* Yb, double* red,
                          double2* alpha, double* tau, int* sing, int warp, int lane) {
  const int S = L.S;
  const int rr = 32 * warp + lane, r = k + rr;
  const bool live = r < L.N8;
  const int nlw = min(kPanelWarps, (L.N8 - k + 31) / 32);  // warps with rows in the panel
  const bool wlive = warp < nlw;
  if (nlw == 1 && !wlive) return;  // warp 0 factors the panel alone, without barriers
  double pr[8], pi[8], yr[8], yi[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    pr[j] = live ? Are[(size_t)(k + j) * S + r] : 0.0;
    pi[j] = live ? Aim[(size_t)(k + j) * S + r] : 0.0;
    yr[j] = 0.0;
    yi[j] = 0.0;
  }
  double* rn = red;      // [0..3] norm partials, [4..5] x0
  double* rd = red + 8;  // [warp][16] dot partials
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (j < bw) {
      const bool in_j = rr >= j;  // row in the support of v_j
      // ---- norm of the column's rows j.. and x0
      double s = 0.0, x0r, x0i;
      if (wlive) s = wsum(in_j ? fma(pr[j], pr[j], pi[j] * pi[j]) : 0.0);
      if (nlw == 1) {
        x0r = __shfl_sync(0xffffffffu, pr[j], j);
        x0i = __shfl_sync(0xffffffffu, pi[j], j);
      } else {
        if (lane == 0) rn[warp] = s;
        if (rr == j) {
          rn[4] = pr[j];
          rn[5] = pi[j];
        }
        panel_sync();
        if (wlive) s = sum_live(rn, 1, nlw);
        x0r = rn[4];
        x0i = rn[5];
      }
      // ---- alpha_j = -e^{i arg x0} sigma, tau_j = 1 / (sigma (sigma + |x0|)),
      // sigma = sqrt(s); with t = 1 / sqrt(s q), q = |x0|^2: sigma / |x0| = s t
      // and |x0| / sigma = q t, so alpha = -x0 s t and tau = 1 / (s (1 + q t))
      double alr = 0.0, ali = 0.0, tj = 0.0;
      if (wlive && s > 0.0) {
        const double q = fma(x0r, x0r, x0i * x0i);
        if (q > 0.0) {
          const double t = rsqrt64(s * q);
          const double st = s * t;
          alr = -(x0r * st);
          ali = -(x0i * st);
          tj = rcp64(s * fma(q, t, 1.0));
        } else {
          alr = -(s * rsqrt64(s));
          tj = rcp64(s);
        }
      }
      if (rr == j) {
        pr[j] = x0r - alr;
        pi[j] = x0i - ali;
      }
      if (rr == 0) {
        alpha[k + j] = make_double2(alr, ali);
        tau[k + j] = tj;
        if (!(s > 0.0)) *sing = 1;
      }
      // ---- slot m < j: z_m = v_m^H v_j; slot m >= j: w_{m+1} = v_j^H a_{m+1}
      double tot = 0.0;
      if (wlive) {
        double v[16];
#pragma unroll
        for (int m = 0; m < 7; ++m) {
          const int c = (m < j) ? m : m + 1;
          double dr, di;
          if (m < j) {  // conj(v_m) v_j
            dr = fma(pr[c], pr[j], pi[c] * pi[j]);
            di = fma(pr[c], pi[j], -pi[c] * pr[j]);
          } else {  // conj(v_j) a_c
            dr = fma(pr[j], pr[c], pi[j] * pi[c]);
            di = fma(pr[j], pi[c], -pi[j] * pr[c]);
          }
          v[2 * m] = in_j ? dr : 0.0;
          v[2 * m + 1] = in_j ? di : 0.0;
        }
        v[14] = 0.0;
        v[15] = 0.0;
        tot = reduce_scatter16(v, lane);
      }
      if (nlw > 1) {
        if ((lane & 1) == 0) rd[warp * 16 + (lane >> 1)] = tot;
        panel_sync();
        if (wlive) tot = sum_live(rd + ((lane >> 1) & 15), 16, nlw);
      }
      if (wlive) {
        double t[14];
#pragma unroll
        for (int m = 0; m < 14; ++m) t[m] = __shfl_sync(0xffffffffu, tot, 2 * m);
        // ---- Y_j = tau_j (v_j - sum_{l<j} Y_l z_l)
        {
          double ar = in_j ? pr[j] : 0.0, ai = in_j ? pi[j] : 0.0;
#pragma unroll
          for (int l = 0; l < 8; ++l) {
            if (l < j) {
              const double zr = t[2 * l], zi = t[2 * l + 1];
              ar = fma(-yr[l], zr, fma(yi[l], zi, ar));
              ai = fma(-yr[l], zi, fma(-yi[l], zr, ai));
            }
          }
          yr[j] = tj * ar;
          yi[j] = tj * ai;
        }
        // ---- apply H_j to the panel columns right of j: a_c -= (tau_j v_j) w_c
        {
          const double tvr = tj * pr[j], tvi = tj * pi[j];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if (c > j && in_j) {
              const double wr = t[2 * (c - 1)], wi = t[2 * (c - 1) + 1];
              pr[c] = fma(-tvr, wr, fma(tvi, wi, pr[c]));
              pi[c] = fma(-tvr, wi, fma(-tvi, wr, pi[c]));
            }
          }
        }
      }
    }
  }
  if (live) {
    double* Yre = Yb;
    double* Yim = Yb + 8 * S;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      Are[(size_t)(k + j) * S + r] = pr[j];
      Aim[(size_t)(k + j) * S + r] = pi[j];
      Yre[j * S + rr] = (j < bw) ? yr[j] : 0.0;
      Yim[j * S + rr] = (j < bw) ? yi[j] : 0.0;
    }
  }
}

// One warp: W = Y^H A_t for the tile of columns c0..c0+7 over rows k..N8-1,
// summed over the 8-row blocks blk0, blk0 + bstep, ... (bstep > 1 leaves a
// partial sum).  Each complex product takes three real MMAs instead of four
// (Gauss): with A1 = Yr^T Ar, A2 = Yi^T Ai and A3 = (Yr - Yi)^T (Ar + Ai),
// Re W = A1 + A2 and Im W = A3 - A1 + A2.  An MMA holds the FP64 unit about
// eight times as long as the FP64 addition that forms an operand sum, so the
// trade saves FP64 time.
__device__ void qrd_w(const QrdLayout& L, int k, int c0, const double* Are, const double* Aim, const double* Yb,
                      double* tile, int blk0, int bstep, int lane) {
  const int S = L.S, g = lane >> 2, q = lane & 3;
  const int R8 = L.N8 - k;
  // A operand (Y^H)[i][rr] -> Y[rr][i], B operand A_t[rr][c]; the two halves
  // of each block accumulate separately (six independent chains)
  double p10 = 0.0, p11 = 0.0, p20 = 0.0, p21 = 0.0, p30 = 0.0, p31 = 0.0;
  double q10 = 0.0, q11 = 0.0, q20 = 0.0, q21 = 0.0, q30 = 0.0, q31 = 0.0;
  const double* bre = Are + (size_t)(c0 + g) * S + k;
  const double* bim = Aim + (size_t)(c0 + g) * S + k;
  const double* yre = Yb + g * S;
  const double* yim = Yb + 8 * S + g * S;
  for (int ks = 8 * blk0; ks + 8 <= R8; ks += 8 * bstep) {
    {
      const double vr = yre[ks + q], vi = yim[ks + q], xr = bre[ks + q], xi = bim[ks + q];
      dmma(p10, p11, vr, xr);
      dmma(p20, p21, vi, xi);
      dmma(p30, p31, vr - vi, xr + xi);
    }
    {
      const double vr = yre[ks + 4 + q], vi = yim[ks + 4 + q], xr = bre[ks + 4 + q], xi = bim[ks + 4 + q];
      dmma(q10, q11, vr, xr);
      dmma(q20, q21, vi, xi);
      dmma(q30, q31, vr - vi, xr + xi);
    }
  }
  {
    double* tre = tile;
    double* tim = tile + 8 * kTileStride;
    const double a10 = p10 + q10, a11 = p11 + q11, a20 = p20 + q20, a21 = p21 + q21;
    const double a30 = p30 + q30, a31 = p31 + q31;
    tre[(2 * q) * kTileStride + g] = a10 + a20;
    tre[(2 * q + 1) * kTileStride + g] = a11 + a21;
    tim[(2 * q) * kTileStride + g] = (a30 - a10) + a20;
    tim[(2 * q + 1) * kTileStride + g] = (a31 - a11) + a21;
  }
}

// A_t -= V W for rows k + m0 .. k + m0 + 15 of the tile at column c0 (W from
// qrd_w in tile).  V is read from the panel's columns of A: entry (row rr,
// reflector i) is A[k + rr][k + i] for rr >= i and zero above (the updates
// only ever follow full panels of 8 reflectors).  For V W, with T1 = Vr Wr,
// T2 = Vi Wi and T3 = (Vr + Vi)(Wr + Wi): Re = T1 - T2, Im = T3 - T1 - T2.
__device__ void qrd_update(const QrdLayout& L, int k, int c0, int m0, double* Are, double* Aim, const double* tile,
                           int lane) {
  const int S = L.S, g = lane >> 2, q = lane & 3;
  const int R8 = L.N8 - k;
  const double* tre = tile;
  const double* tim = tile + 8 * kTileStride;
  // A operand V[r][i], B operand W[i][n]; two row tiles of 8
  const double w0r = tre[g * kTileStride + q], w0i = tim[g * kTileStride + q];
  const double w1r = tre[g * kTileStride + 4 + q], w1i = tim[g * kTileStride + 4 + q];
  const double w0s = w0r + w0i, w1s = w1r + w1i;
  {
    const bool two = m0 + 8 < R8;
    double* pr0 = Are + (size_t)(c0 + 2 * q) * S + k + m0 + g;
    double* pi0 = Aim + (size_t)(c0 + 2 * q) * S + k + m0 + g;
    double cr0 = pr0[0], cr1 = pr0[S], ci0 = pi0[0], ci1 = pi0[S];
    double dr0 = 0.0, dr1 = 0.0, di0 = 0.0, di1 = 0.0;
    if (two) {
      dr0 = pr0[8];
      dr1 = pr0[S + 8];
      di0 = pi0[8];
      di1 = pi0[S + 8];
    }
    double t10 = 0.0, t11 = 0.0, t20 = 0.0, t21 = 0.0, u10 = 0.0, u11 = 0.0, u20 = 0.0, u21 = 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const double wr = h ? w1r : w0r, wi = h ? w1i : w0i, ws = h ? w1s : w0s;
      const int i = 4 * h + q;
      const size_t vo = (size_t)(k + i) * S + k + m0 + g;
      const bool up = m0 + g >= i;  // below or on the diagonal of reflector i
      const double vr = up ? Are[vo] : 0.0, vi = up ? Aim[vo] : 0.0;
      dmma(t10, t11, vr, wr);
      dmma(t20, t21, vi, wi);
      dmma(ci0, ci1, ineg(vr + vi), ws);
      if (two) {
        const double ur = Are[vo + 8], ui = Aim[vo + 8];  // rows m0 + 8.. are all below the panel's diagonal
        dmma(u10, u11, ur, wr);
        dmma(u20, u21, ui, wi);
        dmma(di0, di1, ineg(ur + ui), ws);
      }
    }
    // Re -= T1 - T2, Im -= T3 - T1 - T2 (the T3 part is already in ci / di)
    pr0[0] = (cr0 - t10) + t20;
    pr0[S] = (cr1 - t11) + t21;
    pi0[0] = (ci0 + t10) + t20;
    pi0[S] = (ci1 + t11) + t21;
    if (two) {
      pr0[8] = (dr0 - u10) + u20;
      pr0[S + 8] = (dr1 - u11) + u21;
      pi0[8] = (di0 + u10) + u20;
      pi0[S + 8] = (di1 + u11) + u21;
    }
  }
}

// Factorises one [H | y] with the calling CTA.
//
// Four warps (two CTAs per SM, one matrix's panel overlapping the other's
// update): panel k, then W and A -= V W for every tile right of it, with
// barriers between.
//
// Eight warps (one matrix per SM): the schedule looks one panel ahead.
// While warps 4..7 apply panel k to the columns k+16.. (W for their tiles, a
// barrier of their own, then A -= V W in units of (tile, 16 rows)), warps
// 0..3 apply it to the next panel's columns k+8..k+15 alone (W split over the
// four warps by 8-row blocks and summed, then A -= V W) and factor panel k+8
// into the other Y buffer.  The FP64 units are shared by a panel warp and an
// update warp on each scheduler, so the panel's latency gaps fill with MMAs.
__device__ void qr_dmma_one(int N, int M, const double2* __restrict__ Hb, const double2* __restrict__ yb,
                            const QrDst& out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  QrdLayout L;
  L.init(N, M);
  double* Are = reinterpret_cast<double*>(smem_raw + L.off_are);
  double* Aim = reinterpret_cast<double*>(smem_raw + L.off_aim);
  double* const Y0 = reinterpret_cast<double*>(smem_raw + L.off_y[0]);
  double* const Y1 = reinterpret_cast<double*>(smem_raw + L.off_y[1]);
  double* red = reinterpret_cast<double*>(smem_raw + L.off_red);
  double2* alpha = reinterpret_cast<double2*>(smem_raw + L.off_alpha);
  double* tau = reinterpret_cast<double*>(smem_raw + L.off_tau);
  int* sing = reinterpret_cast<int*>(smem_raw + L.off_sing);
  double* tiles = reinterpret_cast<double*>(smem_raw + L.off_tile);
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;

  const int plane = L.C8 * L.S;
  for (int t = tid; t < plane; t += nthr) {
    Are[t] = 0.0;
    Aim[t] = 0.0;
  }
  if (tid == 0) *sing = 0;
  __syncthreads();
  for (int t = tid; t < N * M; t += nthr) {
    const int r = t / M, c = t % M;
    const double2 h = Hb[t];
    Are[(size_t)c * L.S + r] = h.x;
    Aim[(size_t)c * L.S + r] = h.y;
  }
  for (int r = tid; r < N; r += nthr) {
    const double2 v = yb[r];
    Are[(size_t)M * L.S + r] = v.x;
    Aim[(size_t)M * L.S + r] = v.y;
  }
  __syncthreads();
  if (nw == kPanelWarps) {
    for (int k = 0; k < M; k += 8) {
      qrd_panel(L, k, min(8, M - k), Are, Aim, Y0, red, alpha, tau, sing, warp, lane);
      __syncthreads();
      // W_t = Y^H A_t for every tile of 8 columns (k+8 .. M), then A_t -= V W_t
      // in units of (tile, 16 rows)
      const int ntiles = (M + 1 - (k + 8) + 7) / 8;
      const int nrb = (L.N8 - k + 15) / 16;
      for (int t = warp; t < ntiles; t += nw)
        qrd_w(L, k, k + 8 + 8 * t, Are, Aim, Y0, tiles + (size_t)t * kTileDoubles, 0, 1, lane);
      __syncthreads();
      for (int u = warp; u < ntiles * nrb; u += nw) {
        const int t = u / nrb, rb = u - t * nrb;
        qrd_update(L, k, k + 8 + 8 * t, 16 * rb, Are, Aim, tiles + (size_t)t * kTileDoubles, lane);
      }
      __syncthreads();
    }
  } else {
    if (warp < kPanelWarps) qrd_panel(L, 0, min(8, M), Are, Aim, Y0, red, alpha, tau, sing, warp, lane);
    __syncthreads();
    // tiles right of panel k exist while k + 8 <= M (column M is y); panel k is then full
    for (int k = 0, b = 0; k + 8 <= M; k += 8, b ^= 1) {
      const int kn = k + 8;
      const int ntiles = (M + 1 - kn + 7) / 8;  // tile 0 holds the next panel's columns
      const int nrb = (L.N8 - k + 15) / 16;
      const double* Yc = b ? Y1 : Y0;
      double* const Yn = b ? Y0 : Y1;
      if (warp < kPanelWarps) {
        // the next panel's Y buffer holds the four partial W until that panel writes it
        double* part = Yn;
        qrd_w(L, k, kn, Are, Aim, Yc, part + warp * kTileDoubles, warp, kPanelWarps, lane);
        panel_sync();
        {
          const int e = tid;  // 0..127: entry (plane, column, row) of the 2 x 8 x 8 tile
          const int at = (e >> 6) * 8 * kTileStride + ((e >> 3) & 7) * kTileStride + (e & 7);
          tiles[at] = (part[at] + part[kTileDoubles + at]) + (part[2 * kTileDoubles + at] + part[3 * kTileDoubles + at]);
        }
        panel_sync();
        for (int rb = warp; rb < nrb; rb += kPanelWarps) qrd_update(L, k, kn, 16 * rb, Are, Aim, tiles, lane);
        panel_sync();
        if (kn < M) qrd_panel(L, kn, min(8, M - kn), Are, Aim, Yn, red, alpha, tau, sing, warp, lane);
      } else {
        const int uw = warp - kPanelWarps, un = nw - kPanelWarps;
        for (int t = 1 + uw; t < ntiles; t += un)
          qrd_w(L, k, kn + 8 * t, Are, Aim, Yc, tiles + (size_t)t * kTileDoubles, 0, 1, lane);
        update_sync(un * 32);
        for (int u = uw; u < (ntiles - 1) * nrb; u += un) {
          const int t = 1 + u / nrb, rb = u - (t - 1) * nrb;
          qrd_update(L, k, kn + 8 * t, 16 * rb, Are, Aim, tiles + (size_t)t * kTileDoubles, lane);
        }
      }
      __syncthreads();
    }
  }
  qr_writeout(M, [&](int c, int r) { return make_double2(Are[(size_t)c * L.S + r], Aim[(size_t)c * L.S + r]); },
              alpha, tau, out);
  if (out.singular && tid == 0) *out.singular = *sing;
}

template <int WQ>
__global__ void __launch_bounds__(WQ * 32, WQ == kPanelWarps ? 2 : 1)
    qr_dmma_kernel(int batch, int N, int M, const double* __restrict__ H, const double* __restrict__ y,
                   QrOut out) {
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
  qr_dmma_one(N, M, reinterpret_cast<const double2*>(H) + (size_t)b * N * M,
              reinterpret_cast<const double2*>(y) + (size_t)b * N, d);
}

template <int WQ>
__global__ void __launch_bounds__(WQ * 32, WQ == kPanelWarps ? 2 : 1)
    qr_dmma_gather_kernel(int count, const int* __restrict__ ids, const MixedReq* __restrict__ reqs,
                          const double* __restrict__ H, const double* __restrict__ y, QrOut out) {
  if ((int)blockIdx.x >= count) return;
  const int r = ids[blockIdx.x];
  const MixedReq q = reqs[r];
  QrDst d{out.R64 + q.r_off64, out.yb64 + q.y_off64, out.R32 + q.r_off, out.yb32 + q.y_off, nullptr, nullptr,
          out.singular + r};
  qr_dmma_one(q.n_rx, q.n_tx, reinterpret_cast<const double2*>(H + q.h_off),
              reinterpret_cast<const double2*>(y + q.yin_off), d);
}

// ---------------------------------------------------------------------------
// Small systems (n_rx <= 32): the same reflectors, column by column in the
// left-looking order (column j receives reflectors 0..j-1, then forms its own),
// for 32 / L matrices per warp with L lanes per matrix (L = 2 for n_rx <= 16,
// 4 for n_rx <= 32): lane L m + h holds rows r = L q + h (q < 8) of matrix
// m's current column in registers.  An FP64
// instruction occupies its scheduler's FP64 unit for about 70 cycles however
// many lanes it serves, so here every lane does useful FMAs and a reflector
// costs one two-lane reduction, where one CTA per matrix spends most of its
// FP64 instructions on cross-lane sums and idle rows.  The reflectors v_k
// (rows k..N-1) and tau_k live in shared memory, entry-major with the warp's
// matrices innermost (consecutive lanes read consecutive 16-byte entries);
// the phases of R's rows stay in the registers of the lanes owning them.
constexpr int kQsSlots = 8;  // rows per lane (n_rx <= 8 L)

__host__ __device__ inline int qs_vo(int k, int N) { return k * N - k * (k - 1) / 2; }  // first entry of v_k
__host__ __device__ inline int qs_lanes(int N) { return N <= 16 ? 2 : 4; }
__host__ __device__ inline size_t qs_smem(int N, int M) {
  const int mats = 32 / qs_lanes(N);
  return sizeof(double2) * mats * (size_t)qs_vo(M, N) + sizeof(double) * mats * (size_t)M;
}

// One R entry z = R_kc (complex, after the phase fix) in the real interleaved
// outputs: the block [[Re, -Im], [Im, Re]] at rows 2k.., columns 2c..
__device__ __forceinline__ void qs_put(const QrDst& out, int n, int k, int c, double re, double im) {
  const double vals[4] = {re, -im, im, re};
  const int rows[4] = {2 * k, 2 * k, 2 * k + 1, 2 * k + 1};
  const int cols[4] = {2 * c, 2 * c + 1, 2 * c, 2 * c + 1};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int rr = rows[e], cc = cols[e];
    if (rr > cc) continue;
    if (out.R64) out.R64[col_off(cc) + rr] = vals[e];
    if (out.R32) out.R32[col_off(cc) + rr] = (float)vals[e];
    if (out.Rdense) out.Rdense[(size_t)rr * n + cc] = vals[e];
  }
}

// Factorises the [H | y] of this lane group (act: the group has a matrix).
// Hb: row-major N x M complex, yb: N complex.  Every lane of the warp calls
// this with the same N, M (shuffles inside).
template <int L>
__device__ void qr_small_pair(int N, int M, bool act, const double2* __restrict__ Hb,
                              const double2* __restrict__ yv, const QrDst& out, double2* V, double* Tau) {
  constexpr int kQsMats = 32 / L;
  const int lane = threadIdx.x & 31, m = lane / L, h = lane % L;
  const int n = 2 * M;
  double2 a[kQsSlots], ph[kQsSlots];
#pragma unroll
  for (int q = 0; q < kQsSlots; ++q) ph[q] = make_double2(1.0, 0.0);
  int sing = 0;
  for (int j = 0; j <= M; ++j) {
#pragma unroll
    for (int q = 0; q < kQsSlots; ++q) {
      const int r = L * q + h;
      a[q] = make_double2(0.0, 0.0);
      if (act && r < N) a[q] = (j < M) ? Hb[(size_t)r * M + j] : yv[r];
    }
    // reflectors 0 .. j-1: a <- a - v_k tau_k (v_k^H a) over rows k..N-1
    const int kend = j < M ? j : M;
    for (int k = 0; k < kend; ++k) {
      const double2* vk = V + (size_t)(qs_vo(k, N) - k) * kQsMats + m;  // entry r at vk[r * kQsMats]
      double wr = 0.0, wi = 0.0;
#pragma unroll
      for (int q = 0; q < kQsSlots; ++q) {
        const int r = L * q + h;
        if (L * q + L - 1 < k || L * q >= N) continue;  // no lane of the group has this row
        if (r >= k && r < N) {
          const double2 v = vk[(size_t)r * kQsMats];
          wr = fma(v.x, a[q].x, fma(v.y, a[q].y, wr));
          wi = fma(v.x, a[q].y, fma(-v.y, a[q].x, wi));
        }
      }
#pragma unroll
      for (int o = 1; o < L; o <<= 1) {
        wr += __shfl_xor_sync(0xffffffffu, wr, o);
        wi += __shfl_xor_sync(0xffffffffu, wi, o);
      }
      const double tk = Tau[k * kQsMats + m];
      wr *= tk;
      wi *= tk;
#pragma unroll
      for (int q = 0; q < kQsSlots; ++q) {
        const int r = L * q + h;
        if (L * q + L - 1 < k || L * q >= N) continue;
        if (r >= k && r < N) {
          const double2 v = vk[(size_t)r * kQsMats];
          a[q].x = fma(-v.x, wr, fma(v.y, wi, a[q].x));
          a[q].y = fma(-v.x, wi, fma(-v.y, wr, a[q].y));
        }
      }
    }
    if (j < M) {
      // column j of R above the diagonal: rows k < j, final now, phase-fixed
#pragma unroll
      for (int q = 0; q < kQsSlots; ++q) {
        const int r = L * q + h;
        if (act && r < j) {
          const double re = a[q].x * ph[q].x + a[q].y * ph[q].y, im = a[q].y * ph[q].x - a[q].x * ph[q].y;
          qs_put(out, n, r, j, re, im);
        }
      }
      // reflector j from rows j..N-1
      double s = 0.0;
      double2 x0 = make_double2(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < kQsSlots; ++q) {
        const int r = L * q + h;
        if (r >= j && r < N) s = fma(a[q].x, a[q].x, fma(a[q].y, a[q].y, s));
        if (r == j) x0 = a[q];
      }
#pragma unroll
      for (int o = 1; o < L; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const int h0 = j % L;
      x0.x = __shfl_sync(0xffffffffu, x0.x, (lane & ~(L - 1)) | h0);
      x0.y = __shfl_sync(0xffffffffu, x0.y, (lane & ~(L - 1)) | h0);
      double sigma = 0.0, tj = 0.0;
      double2 phr = make_double2(1.0, 0.0), al = make_double2(0.0, 0.0);
      if (s > 0.0) {
        const double rs = rsqrt64(s);
        sigma = s * rs;
        const double qq = fma(x0.x, x0.x, x0.y * x0.y);
        double ax0 = 0.0;
        double2 p0 = make_double2(1.0, 0.0);
        if (qq > 0.0) {
          const double rq = rsqrt64(qq);
          ax0 = qq * rq;
          p0 = make_double2(x0.x * rq, x0.y * rq);
        }
        // alpha = -e^{i arg x0} sigma keeps v_j = x0 - alpha free of cancellation
        al = make_double2(-p0.x * sigma, -p0.y * sigma);
        phr = make_double2(-p0.x, -p0.y);
        tj = rcp64(sigma * (sigma + ax0));
      } else {
        sing = 1;
      }
      double2* vj = V + (size_t)(qs_vo(j, N) - j) * kQsMats + m;
#pragma unroll
      for (int q = 0; q < kQsSlots; ++q) {
        const int r = L * q + h;
        if (r >= j && r < N) vj[(size_t)r * kQsMats] = (r == j) ? make_double2(x0.x - al.x, x0.y - al.y) : a[q];
        if (r == j) ph[q] = phr;
      }
      if (h == 0) Tau[j * kQsMats + m] = tj;
      if (act && h == h0) qs_put(out, n, j, j, sigma, 0.0);
    } else {
      // ybar = Q^H y: rows k < M of the y column, phase-fixed
#pragma unroll
      for (int q = 0; q < kQsSlots; ++q) {
        const int r = L * q + h;
        if (act && r < M) {
          const double re = a[q].x * ph[q].x + a[q].y * ph[q].y, im = a[q].y * ph[q].x - a[q].x * ph[q].y;
          if (out.yb64) {
            out.yb64[2 * r] = re;
            out.yb64[2 * r + 1] = im;
          }
          if (out.yb32) {
            out.yb32[2 * r] = (float)re;
            out.yb32[2 * r + 1] = (float)im;
          }
          if (out.ybdense) {
            out.ybdense[2 * r] = re;
            out.ybdense[2 * r + 1] = im;
          }
        }
      }
    }
    __syncwarp();
  }
  if (act) {
    if (out.Rdense)
      for (int t = h; t < n * n; t += L)
        if (t / n > t % n) out.Rdense[t] = 0.0;
    if (h == 0 && out.singular) *out.singular = sing;
  }
}

template <int L>
__global__ void __launch_bounds__(32) qr_small_kernel(int batch, int N, int M, const double* __restrict__ H,
                                                      const double* __restrict__ y, QrOut out) {
  constexpr int kQsMats = 32 / L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* V = reinterpret_cast<double2*>(smem_raw);
  double* Tau = reinterpret_cast<double*>(V + (size_t)kQsMats * qs_vo(M, N));
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * kQsMats + lane / L;
  const bool act = b < batch;
  const int n = 2 * M;
  const int bb = act ? b : 0;
  QrDst d;
  d.R64 = out.R64 ? out.R64 + (size_t)bb * tri_stride64(n) : nullptr;
  d.yb64 = out.yb64 ? out.yb64 + (size_t)bb * vec_stride64(n) : nullptr;
  d.R32 = out.R32 ? out.R32 + (size_t)bb * tri_stride32(n) : nullptr;
  d.yb32 = out.yb32 ? out.yb32 + (size_t)bb * vec_stride32(n) : nullptr;
  d.Rdense = out.Rdense ? out.Rdense + (size_t)bb * n * n : nullptr;
  d.ybdense = out.ybdense ? out.ybdense + (size_t)bb * n : nullptr;
  d.singular = out.singular ? out.singular + bb : nullptr;
  qr_small_pair<L>(N, M, act, reinterpret_cast<const double2*>(H) + (size_t)bb * N * M,
                reinterpret_cast<const double2*>(y) + (size_t)bb * N, d, V, Tau);
}

// Uneven batches: the listed requests (all N x M) at their own offsets.
template <int L>
__global__ void __launch_bounds__(32) qr_small_gather_kernel(int count, const int* __restrict__ ids,
                                                             const MixedReq* __restrict__ reqs,
                                                             const double* __restrict__ H,
                                                             const double* __restrict__ y, int N, int M,
                                                             QrOut out) {
  constexpr int kQsMats = 32 / L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* V = reinterpret_cast<double2*>(smem_raw);
  double* Tau = reinterpret_cast<double*>(V + (size_t)kQsMats * qs_vo(M, N));
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kQsMats + lane / L;
  const bool act = i < count;
  const MixedReq q = reqs[ids[act ? i : 0]];
  const int r = ids[act ? i : 0];
  QrDst d{out.R64 + q.r_off64, out.yb64 + q.y_off64, out.R32 + q.r_off, out.yb32 + q.y_off, nullptr, nullptr,
          out.singular + r};
  qr_small_pair<L>(N, M, act, reinterpret_cast<const double2*>(H + q.h_off),
                reinterpret_cast<const double2*>(y + q.yin_off), d, V, Tau);
}

// The tensor-core form for n_tx >= kQrdMinTx when its shared memory fits.
#ifndef MDX_QRD_MIN_TX
#define MDX_QRD_MIN_TX 48
#endif
constexpr int kQrdMinTx = MDX_QRD_MIN_TX;
size_t qrd_smem(int n_rx, int n_tx) {
  QrdLayout L;
  L.init(n_rx, n_tx);
  return L.bytes;
}
// The look-ahead keeps four partial W tiles in a free Y buffer of 16 S
// doubles, S = round_up(n_rx, 8) + 4 >= n_tx + 4.
static_assert(16 * (kQrdMinTx + 4) >= 4 * kTileDoubles, "Y buffer too small for the partial W tiles");
bool use_qrd(int n_rx, int n_tx) {
  return n_tx >= kQrdMinTx && n_rx <= 128 && qrd_smem(n_rx, n_tx) <= 227 * 1024;
}
// Four warps per CTA when two such CTAs fit in one SM's shared memory: one
// matrix's panel then overlaps the other's trailing update.
int qrd_warps(int n_rx, int n_tx) {
  return 2 * qrd_smem(n_rx, n_tx) <= 227 * 1024 ? kPanelWarps : kQrdWarps;
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
  QrDst d{out.R64 + q.r_off64, out.yb64 + q.y_off64, out.R32 + q.r_off, out.yb32 + q.y_off, nullptr, nullptr,
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
  if (use_qrd(n_rx, n_tx)) {
    const int wq = qrd_warps(n_rx, n_tx);
    const size_t sm = qrd_smem(n_rx, n_tx);
    if (wq == kPanelWarps) {
      cudaFuncSetAttribute(qr_dmma_gather_kernel<kPanelWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      qr_dmma_gather_kernel<kPanelWarps><<<count, wq * 32, sm, s>>>(count, ids, reqs, H, y, out);
    } else {
      cudaFuncSetAttribute(qr_dmma_gather_kernel<kQrdWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      qr_dmma_gather_kernel<kQrdWarps><<<count, wq * 32, sm, s>>>(count, ids, reqs, H, y, out);
    }
    return cudaGetLastError();
  }
  if (n_rx <= 32) {
    const size_t sm = qs_smem(n_rx, n_tx);
    if (n_rx <= 16) {
      cudaFuncSetAttribute(qr_small_gather_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      qr_small_gather_kernel<2><<<(count + 15) / 16, 32, sm, s>>>(count, ids, reqs, H, y, n_rx, n_tx, out);
    } else {
      cudaFuncSetAttribute(qr_small_gather_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      qr_small_gather_kernel<4><<<(count + 7) / 8, 32, sm, s>>>(count, ids, reqs, H, y, n_rx, n_tx, out);
    }
    return cudaGetLastError();
  }
  const size_t smem = qr_smem(n_rx, n_tx);
  {
    const int threads = n_tx <= 32 ? 128 : 256;
    cudaFuncSetAttribute(qr_gather_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    qr_gather_kernel<32><<<count, threads, smem, s>>>(count, ids, reqs, H, y, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_qr(int batch, int n_rx, int n_tx, const double* H, const double* y, QrOut out,
                      cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  if (use_qrd(n_rx, n_tx)) {
    const int wq = qrd_warps(n_rx, n_tx);
    const size_t sm = qrd_smem(n_rx, n_tx);
    if (wq == kPanelWarps) {
      cudaFuncSetAttribute(qr_dmma_kernel<kPanelWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      qr_dmma_kernel<kPanelWarps><<<batch, wq * 32, sm, s>>>(batch, n_rx, n_tx, H, y, out);
    } else {
      cudaFuncSetAttribute(qr_dmma_kernel<kQrdWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      qr_dmma_kernel<kQrdWarps><<<batch, wq * 32, sm, s>>>(batch, n_rx, n_tx, H, y, out);
    }
    return cudaGetLastError();
  }
  if (n_rx <= 32) {
    // 16 matrices per warp with two lanes each (n_rx <= 16), else 8 with four
    const size_t sm = qs_smem(n_rx, n_tx);
    if (n_rx <= 16) {
      cudaFuncSetAttribute(qr_small_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      qr_small_kernel<2><<<(batch + 15) / 16, 32, sm, s>>>(batch, n_rx, n_tx, H, y, out);
    } else {
      cudaFuncSetAttribute(qr_small_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      qr_small_kernel<4><<<(batch + 7) / 8, 32, sm, s>>>(batch, n_rx, n_tx, H, y, out);
    }
    return cudaGetLastError();
  }
  const size_t smem = qr_smem(n_rx, n_tx);
  {
    const int threads = n_tx <= 32 ? 128 : 256;
    cudaFuncSetAttribute(qr_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    qr_kernel<32><<<batch, threads, smem, s>>>(batch, n_rx, n_tx, H, y, out);
  }
  return cudaGetLastError();
}

}  // namespace mdx
