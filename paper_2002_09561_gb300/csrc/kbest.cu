// K-best (Sec. VI) and the hybrid SD / K-best (Sec. VI), one CTA per
// received vector, vectors taken from a global counter.
//
// K-best level step.  Thread t owns survivor t: it computes the interference
// c_i = ybar_i - sum_{j>i} R_ij x_j of its path by one FMA chain (Eq. 4,
// shared by the node's P children, Eq. inc), then the P child partial
// distances.  Each child becomes a 64-bit key (FP32 partial distance bits,
// then parent rank * P + child index), so one ascending bitonic sort over the
// level's candidates orders them by (distance, parent rank, child) and the
// first K keys are the survivors; candidates outside the pruning bound get an
// all-ones key and sort last.  The new survivors copy their parent's path
// (4-byte words; the path stride is an odd number of words so that threads
// reading their own paths hit distinct banks) and append their child.
//
// Hybrid.  The master part enumerates every depth-d prefix (rows n-1..n-d),
// keeps those inside the initial sphere and sorts them by partial distance;
// the CTA then finishes them best-first, each by a K-best run over the
// remaining rows under the current radius (a run stops as soon as all its
// survivors leave the sphere), and shrinks the radius with the run's best
// leaf.  Prefixes are taken while their own partial distance is inside the
// sphere; the first one outside ends the vector, since all later ones are
// farther.  The answer is the best K-best leaf over the prefixes inside the
// initial sphere, whatever the order, because a radius above the answer only
// removes nodes that could not lead to it.
//
// Both kernels keep the final leaves within FP32 error of the best and
// re-score them in FP64 against the FP64 R and ybar.
#include "mdx_internal.cuh"

namespace mdx {
namespace {

constexpr uint64_t kInfKey = ~0ull;
constexpr int kCandMax = 8;  // final leaves re-scored in FP64

__host__ __device__ inline int path_stride(int n) {
  int w = round_up(n, 4) / 4;
  if ((w & 1) == 0) ++w;
  return 4 * w;
}

struct KbLayout {
  int n, K, P, keys_cap, pp, ts;
  size_t off_R, off_yb, off_keys, off_xa, off_xb, off_pa, off_pb, off_cx, off_cp, off_misc, bytes;
  __host__ __device__ void init(int n_, int K_, int P_, int keys_cap_) {
    n = n_;
    K = K_;
    P = P_;
    keys_cap = keys_cap_;
    pp = path_stride(n);
    ts = tri_stride32(n);
    size_t o = 0;
    off_keys = o;
    o += sizeof(uint64_t) * keys_cap;
    off_R = o;
    o += sizeof(float) * ts;
    off_yb = o;
    o += sizeof(float) * round_up(n, 4);
    off_pa = o;
    o += sizeof(float) * round_up(K, 4);
    off_pb = o;
    o += sizeof(float) * round_up(K, 4);
    off_cp = o;
    o += sizeof(float) * kCandMax;
    off_misc = o;
    o += 64;
    off_xa = o;
    o += (size_t)pp * K;
    off_xb = o;
    o += (size_t)pp * K;
    off_cx = o;
    o += (size_t)pp * kCandMax;
    bytes = round_up((int)o, 16);
  }
};

// Ascending bitonic sort of Cs (a power of two) keys by T threads.  Thread t
// handles the pairs t, t + T, ...; for strides up to 32 a warp's pairs lie in
// its own 64 consecutive keys (when T >= Cs / 2), so a stage followed by such a
// stage needs only a warp barrier; every other transition takes the CTA barrier.
__device__ __forceinline__ void bitonic_sort(uint64_t* keys, int Cs, int tid, int T) {
  const bool warp_local = T >= (Cs >> 1);
  for (int size = 2; size <= Cs; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int p = tid; p < (Cs >> 1); p += T) {
        const int lo = ((p & ~(stride - 1)) << 1) | (p & (stride - 1));
        const int hi = lo + stride;
        const bool asc = (lo & size) == 0;
        const uint64_t x = keys[lo], y = keys[hi];
        if ((x > y) == asc) {
          keys[lo] = y;
          keys[hi] = x;
        }
      }
      // the next stage's stride: half this one, or the next size's first
      const int next = stride > 1 ? stride >> 1 : size;
      if (warp_local && stride <= 32 && next <= 32) __syncwarp();
      else __syncthreads();
    }
  }
  __syncthreads();
}

struct KbCtx {
  int n, P, K, pp, tid, T;
  float alpha;
  const float* Rc;
  const float* yb;
  uint64_t* keys;
  int* misc;  // misc[0]: valid-candidate count
};

// Runs the K-best level steps over rows top..0 from the S survivors in
// (*xcur, *pcur); on return the survivors are sorted by partial distance in
// (*xcur, *pcur) and their number is returned (0 = all left the sphere).
// r2s points to the shared squared radius (read once per level).
__device__ int kbest_levels(const KbCtx& c, int top, int S, uint8_t** xcur, uint8_t** xnxt,
                            float** pcur, float** pnxt, const float* r2s, float E,
                            long long* nodes, long long* peds, long long* flops) {
  const int n = c.n, P = c.P, K = c.K, pp = c.pp, tid = c.tid, T = c.T;
  for (int i = top; i >= 0 && S > 0; --i) {
    const float bnd = prune_bound(*r2s, E, n);
    const int SP = S * P;
    const int Cs = pow2ceil(SP < 2 ? 2 : SP);
    if (tid < S) {
      const uint8_t* xp = *xcur + (size_t)tid * pp;
      float ci = c.yb[i];
      for (int j = n - 1; j > i; --j)
        ci = fmaf(-c.Rc[col_off(j) + i], (float)(2 * (int)xp[j] - (P - 1)) * c.alpha, ci);
      const float rii = c.Rc[col_off(i) + i];
      const float p0 = (*pcur)[tid];
      for (int k = 0; k < P; ++k) {
        const float d = fmaf(-rii, (float)(2 * k - (P - 1)) * c.alpha, ci);
        const float ped = fmaf(d, d, p0);
        const unsigned id = (unsigned)(tid * P + k);
        c.keys[tid * P + k] = (ped < bnd) ? (((uint64_t)__float_as_uint(ped) << 32) | id) : kInfKey;
      }
    }
    for (int q = SP + tid; q < Cs; q += T) c.keys[q] = kInfKey;
    if (tid == 0) c.misc[0] = 0;
    __syncthreads();
    bitonic_sort(c.keys, Cs, tid, T);
    for (int q = tid; q < Cs; q += T)
      if (c.keys[q] != kInfKey && (q + 1 == Cs || c.keys[q + 1] == kInfKey)) c.misc[0] = q + 1;
    __syncthreads();
    const int valid = c.misc[0];
    const int kept = valid < K ? valid : K;
    if (tid < kept) {
      const uint64_t key = c.keys[tid];
      const unsigned id = (unsigned)(key & 0xffffffffu);
      const int par = (int)(id / (unsigned)P), k = (int)(id % (unsigned)P);
      const uint32_t* src = reinterpret_cast<const uint32_t*>(*xcur + (size_t)par * pp);
      uint32_t* dst = reinterpret_cast<uint32_t*>(*xnxt + (size_t)tid * pp);
      for (int w = 0; w < pp / 4; ++w) dst[w] = src[w];
      (*xnxt)[(size_t)tid * pp + i] = (uint8_t)k;
      (*pnxt)[tid] = __uint_as_float((unsigned)(key >> 32));
    }
    *nodes += S;
    *peds += SP;
    *flops += (long long)S * (2 * (n - 1 - i) + 4 * P);
    __syncthreads();
    uint8_t* tx = *xcur;
    *xcur = *xnxt;
    *xnxt = tx;
    float* tp = *pcur;
    *pcur = *pnxt;
    *pnxt = tp;
    S = kept;
  }
  return S;
}

// Stage R and ybar of vector v into shared memory and compute E and r2.
__device__ void stage_vector(const SearchArgs& a, int v, const KbLayout& L, unsigned char* smem,
                             float* misc_f) {
  const int tid = threadIdx.x, T = blockDim.x;
  float* Rc = reinterpret_cast<float*>(smem + L.off_R);
  float* yb = reinterpret_cast<float*>(smem + L.off_yb);
  const float4* src = reinterpret_cast<const float4*>(a.R32 + (size_t)v * L.ts);
  for (int t = tid; t < L.ts / 4; t += T) reinterpret_cast<float4*>(Rc)[t] = src[t];
  const float* ys = a.yb32 + (size_t)v * vec_stride32(a.n);
  for (int r = tid; r < a.n; r += T) yb[r] = ys[r];
  __syncthreads();
  if (tid < 32) {
    const float E = error_scale_warp(a.n, a.P, a.alpha, Rc, yb, tid);
    if (tid == 0) {
      float r2;
      if (a.radius_mode == RADIUS_NONE) r2 = INFINITY;
      else if (a.radius_mode == RADIUS_PAPER) r2 = (float)((double)a.n_rx * a.n_tx * a.noise_var[v]);
      else if (a.radius_mode == RADIUS_PER_VECTOR) r2 = a.r2_vec[v];
      else r2 = (float)a.radius_value;
      if (!(r2 > 0.0f)) r2 = INFINITY;
      misc_f[0] = E;
      misc_f[1] = r2;
    }
  }
  __syncthreads();
}

// Re-score candidate paths (cx, cped; count nc, sorted or not) in FP64 with
// warp 0, write the outputs of vector v.
__device__ void finish_vector(const SearchArgs& a, int v, const uint8_t* cx, const float* cped,
                              int nc, int pp, float E, int status, long long nodes, long long peds,
                              long long restarts, long long flops) {
  const int tid = threadIdx.x;
  if (tid >= 32) return;
  const int lane = tid, n = a.n, P = a.P;
  float best = INFINITY;
  for (int q = 0; q < nc; ++q) best = fminf(best, cped[q]);
  const float keep = prune_bound(best, E, n);
  const double* R64 = a.R64 + (size_t)v * tri_stride64(n);
  const double* y64 = a.yb64 + (size_t)v * vec_stride64(n);
  int win = -1;
  double win_m = INFINITY;
  long long rescored = 0;
  for (int q = 0; q < nc; ++q) {
    if (!(cped[q] <= keep)) continue;
    double m;
    if (a.flags & MDX_NO_RESCORE) {
      m = (double)cped[q];
    } else {
      m = rescore_fp64_warp(n, P, a.alpha64, R64, y64, cx + (size_t)q * pp, lane);
      ++rescored;
    }
    bool better = m < win_m;
    if (!better && m == win_m && win >= 0) {
      for (int j = n - 1; j >= 0; --j) {
        const int x1 = cx[(size_t)q * pp + j], x2 = cx[(size_t)win * pp + j];
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
    if (win >= 0) s = (uint8_t)(cx[(size_t)win * pp + 2 * j] * P + cx[(size_t)win * pp + 2 * j + 1]);
    a.sym_out[(size_t)v * a.n_tx + j] = s;
  }
  if (lane == 0) {
    a.metric_out[v] = (win >= 0) ? win_m : (double)INFINITY;
    a.vstatus[v] = status;
    if (a.stats) {
      a.stats[(size_t)v * kStats + 0] = nodes;
      a.stats[(size_t)v * kStats + 1] = peds;
      a.stats[(size_t)v * kStats + 2] = restarts;
      a.stats[(size_t)v * kStats + 3] = rescored;
      a.stats[(size_t)v * kStats + 4] = flops;
    }
  }
}

__device__ bool singular_vector(const SearchArgs& a, int v) {
  if (!(a.singular && a.singular[v])) return false;
  for (int j = threadIdx.x; j < a.n_tx; j += blockDim.x) a.sym_out[(size_t)v * a.n_tx + j] = 0;
  if (threadIdx.x == 0) {
    a.metric_out[v] = 0.0;
    a.vstatus[v] = MDX_V_SINGULAR;
    if (a.stats)
      for (int q = 0; q < kStats; ++q) a.stats[(size_t)v * kStats + q] = 0;
  }
  return true;
}

__global__ void kbest_kernel(SearchArgs a, KbLayout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, T = blockDim.x;
  const int n = a.n, P = a.P;
  uint64_t* keys = reinterpret_cast<uint64_t*>(smem + L.off_keys);
  int* misc = reinterpret_cast<int*>(smem + L.off_misc);
  float* misc_f = reinterpret_cast<float*>(misc + 4);
  KbCtx c{n, P, a.K, L.pp, tid, T, a.alpha, reinterpret_cast<float*>(smem + L.off_R),
          reinterpret_cast<float*>(smem + L.off_yb), keys, misc};

  for (;;) {
    if (tid == 0) misc[1] = (int)atomicAdd(a.work_counter, 1u);
    __syncthreads();
    const int v = misc[1];
    __syncthreads();
    if (v >= a.batch) break;
    if (singular_vector(a, v)) continue;
    stage_vector(a, v, L, smem, misc_f);
    const float E = misc_f[0];
    long long nodes = 0, peds = 0, restarts = 0, flops = 0;
    int S = 0;
    uint8_t *xcur = nullptr, *xnxt = nullptr;
    float *pcur = nullptr, *pnxt = nullptr;
    for (;;) {
      xcur = smem + L.off_xa;
      xnxt = smem + L.off_xb;
      pcur = reinterpret_cast<float*>(smem + L.off_pa);
      pnxt = reinterpret_cast<float*>(smem + L.off_pb);
      if (tid == 0) pcur[0] = 0.0f;
      __syncthreads();
      S = kbest_levels(c, n - 1, 1, &xcur, &xnxt, &pcur, &pnxt, &misc_f[1], E, &nodes, &peds, &flops);
      if (S > 0 || !(misc_f[1] < INFINITY) || restarts >= 64) break;
      __syncthreads();
      if (tid == 0) misc_f[1] *= 4.0f;  // empty sphere: double the radius
      ++restarts;
      __syncthreads();
    }
    const int nc = S < kCandMax ? S : kCandMax;
    finish_vector(a, v, xcur, pcur, nc, L.pp, E, restarts > 0 ? MDX_V_EMPTY_RETRIED : MDX_V_OK,
                  nodes, peds, restarts, flops);
    __syncthreads();
  }
}

__global__ void hybrid_kernel(SearchArgs a, KbLayout L, int nprefix) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, T = blockDim.x;
  const int n = a.n, P = a.P, d = a.depth;
  uint64_t* keys = reinterpret_cast<uint64_t*>(smem + L.off_keys);
  int* misc = reinterpret_cast<int*>(smem + L.off_misc);
  float* misc_f = reinterpret_cast<float*>(misc + 4);
  float* Rc = reinterpret_cast<float*>(smem + L.off_R);
  float* yb = reinterpret_cast<float*>(smem + L.off_yb);
  uint8_t* cx = smem + L.off_cx;
  float* cped = reinterpret_cast<float*>(smem + L.off_cp);
  KbCtx c{n, P, a.K, L.pp, tid, T, a.alpha, Rc, yb, keys, misc};
  // prefix keys live in the upper part of the key buffer (the levels use the lower part)
  uint64_t* pkeys = keys + (L.keys_cap - nprefix);

  for (;;) {
    if (tid == 0) misc[1] = (int)atomicAdd(a.work_counter, 1u);
    __syncthreads();
    const int v = misc[1];
    __syncthreads();
    if (v >= a.batch) break;
    if (singular_vector(a, v)) continue;
    stage_vector(a, v, L, smem, misc_f);
    const float E = misc_f[0];
    long long nodes = 0, peds = 0, restarts = 0, flops = 0;
    bool budget_hit = false;
    int ncand = 0;  // uniform copy of the candidate count
    if (tid == 0) misc[2] = 0;
    for (;;) {
      // master: all depth-d prefixes inside the current sphere, best first
      const float bnd0 = prune_bound(misc_f[1], E, n);
      int np = 1;
      for (int l = 0; l < d; ++l) np *= P;
      for (int q = tid; q < nprefix; q += T) {
        if (q >= np) {
          pkeys[q] = kInfKey;
          continue;
        }
        int rem = q;
        float ped = 0.0f;
        uint8_t xs[16];
        for (int l = 0; l < d; ++l) {
          const int i = n - 1 - l;
          xs[l] = (uint8_t)(rem % P);
          rem /= P;
          float ci = yb[i];
          for (int m = 0; m < l; ++m)
            ci = fmaf(-Rc[col_off(n - 1 - m) + i], (float)(2 * (int)xs[m] - (P - 1)) * a.alpha, ci);
          const float dd = fmaf(-Rc[col_off(i) + i], (float)(2 * (int)xs[l] - (P - 1)) * a.alpha, ci);
          ped = fmaf(dd, dd, ped);
        }
        pkeys[q] = (ped < bnd0) ? (((uint64_t)__float_as_uint(ped) << 32) | (unsigned)q) : kInfKey;
      }
      __syncthreads();
      bitonic_sort(pkeys, nprefix, tid, T);
      for (int t = 0; t < nprefix; ++t) {
        const uint64_t key = pkeys[t];
        const float pped = __uint_as_float((unsigned)(key >> 32));
        if (key == kInfKey || !(pped < prune_bound(misc_f[1], E, n))) break;
        if (a.budget > 0 && nodes >= a.budget) {
          budget_hit = true;
          break;
        }
        ++nodes;  // the master's node at depth d, handed over
        flops += 2 * (d > 0 ? d - 1 : 0) + 4 * P;
        // hand the prefix to the K-best worker (the whole CTA)
        uint8_t* xcur = smem + L.off_xa;
        uint8_t* xnxt = smem + L.off_xb;
        float* pcur = reinterpret_cast<float*>(smem + L.off_pa);
        float* pnxt = reinterpret_cast<float*>(smem + L.off_pb);
        if (tid == 0) {
          int rem = (int)(key & 0xffffffffu);
          for (int l = 0; l < d; ++l) {
            xcur[n - 1 - l] = (uint8_t)(rem % P);
            rem /= P;
          }
          pcur[0] = pped;
        }
        __syncthreads();
        const int S = kbest_levels(c, n - 1 - d, 1, &xcur, &xnxt, &pcur, &pnxt, &misc_f[1], E,
                                   &nodes, &peds, &flops);
        if (S > 0) {
          // keep this run's leaves within FP32 error of its best in the candidate list,
          // then shrink the radius with its best leaf
          const float lim = prune_bound(fminf(pcur[0], misc_f[1]), E, n);
          for (int s = 0; s < S && s < kCandMax; ++s) {
            const float ps = pcur[s];
            if (!(ps <= lim)) break;
            int slot = -1;
            if (ncand < kCandMax) {
              slot = ncand++;
            } else {
              float worst = -1.0f;
              for (int q = 0; q < kCandMax; ++q)
                if (cped[q] > worst) {
                  worst = cped[q];
                  slot = q;
                }
              if (!(ps < worst)) slot = -1;
            }
            if (slot >= 0) {
              const uint32_t* src = reinterpret_cast<const uint32_t*>(xcur + (size_t)s * L.pp);
              uint32_t* dst = reinterpret_cast<uint32_t*>(cx + (size_t)slot * L.pp);
              for (int w = tid; w < L.pp / 4; w += T) dst[w] = src[w];
              if (tid == 0) cped[slot] = ps;
            }
            __syncthreads();
          }
          if (tid == 0 && pcur[0] < misc_f[1]) misc_f[1] = pcur[0];
        }
        __syncthreads();
      }
      if (ncand > 0 || budget_hit || !(misc_f[1] < INFINITY) || restarts >= 64) break;
      __syncthreads();
      if (tid == 0) misc_f[1] *= 4.0f;
      ++restarts;
      __syncthreads();
    }
    finish_vector(a, v, cx, cped, ncand, L.pp, E,
                  budget_hit ? MDX_V_BUDGET_EXCEEDED : (restarts > 0 ? MDX_V_EMPTY_RETRIED : MDX_V_OK),
                  nodes, peds, restarts, flops);
    __syncthreads();
  }
}

int kb_threads(int K, int P) {
  int C = pow2ceil(K * P);
  int T = C / 2;
  if (T < 32) T = 32;
  if (T > 1024) T = 1024;
  return T;
}

cudaError_t launch_generic(const void* fn, const SearchArgs& a, const KbLayout& L, int T, int extra,
                           bool hybrid, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, T, L.bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = per_sm * num_sms;
  if (grid > a.batch) grid = a.batch;
  if (hybrid) hybrid_kernel<<<grid, T, L.bytes, s>>>(a, L, extra);
  else kbest_kernel<<<grid, T, L.bytes, s>>>(a, L);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_kbest(const SearchArgs& a, int num_sms, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  const int C = pow2ceil(a.K * a.P);
  KbLayout L;
  L.init(a.n, a.K, a.P, C < 2 ? 2 : C);
  if (L.bytes > 227 * 1024) return cudaErrorInvalidConfiguration;
  return launch_generic((const void*)kbest_kernel, a, L, kb_threads(a.K, a.P), 0, false, num_sms, s);
}

cudaError_t launch_hybrid(const SearchArgs& a, int num_sms, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  int np = 1;
  for (int l = 0; l < a.depth; ++l) np *= a.P;
  const int nprefix = pow2ceil(np < 2 ? 2 : np);
  const int C = pow2ceil(a.K * a.P);
  KbLayout L;
  L.init(a.n, a.K, a.P, (C < 2 ? 2 : C) + nprefix);
  if (L.bytes > 227 * 1024) return cudaErrorInvalidConfiguration;
  return launch_generic((const void*)hybrid_kernel, a, L, kb_threads(a.K, a.P), nprefix, true, num_sms,
                        s);
}

}  // namespace mdx
