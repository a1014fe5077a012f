// Warp-level K-best (Sec. VI) shared by the hybrid detector and the
// uneven-batch kernel: one warp runs the level steps of a K-best search with
// survivor paths and partial distances in a caller-provided workspace.
#pragma once

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

// Interference of row i for the survivor path xp (Eq. 4, shared by the
// node's children as in Eq. inc): ybar_i - sum_{j>i} R_ij a(x_j) as eight
// FMA chains (chain p takes j = n-1-p, n-9-p, ...; chain 0 starts from
// ybar_i), added as ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7)).  G
// consecutive lanes (1, 2, 4 or 8; this one is s = lane % G) share the
// survivor, each running the chains p = s, s + G, ...; all of them return
// the same bits, and so does every G.
template <int G>
__device__ __forceinline__ float row_interference(const float* Rc, const float* yb, const uint8_t* xp, int n,
                                                  int P, float alpha, int i, int s) {
  constexpr int M = 8 / G;
  float acc[M];
#pragma unroll
  for (int m = 0; m < M; ++m) acc[m] = (s + G * m == 0) ? yb[i] : 0.0f;
  if (M <= 2) {
    // one or two chains per lane: software-pipelined in batches of four steps,
    // the next batch's loads and level conversions issued before this batch's
    // FMAs.  A step past the chain's end is fmaf(-0, 0, acc) = acc exactly.
    constexpr int B = 4;
    float rb[B][M], ab[B][M];
    auto fetch = [&](int j0, float (&r)[B][M], float (&av)[B][M]) {
#pragma unroll
      for (int b = 0; b < B; ++b)
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int j = j0 - 8 * b - (s + G * m);
          const bool ok = j > i;
          r[b][m] = ok ? Rc[col_off(j) + i] : 0.0f;
          av[b][m] = ok ? (float)(2 * (int)xp[j] - (P - 1)) * alpha : 0.0f;
        }
    };
    int j0 = n - 1;
    fetch(j0, rb, ab);
    while (j0 > i) {
      float rn[B][M], an[B][M];
      fetch(j0 - 8 * B, rn, an);
#pragma unroll
      for (int b = 0; b < B; ++b)
#pragma unroll
        for (int m = 0; m < M; ++m) acc[m] = fmaf(-rb[b][m], ab[b][m], acc[m]);
#pragma unroll
      for (int b = 0; b < B; ++b)
#pragma unroll
        for (int m = 0; m < M; ++m) {
          rb[b][m] = rn[b][m];
          ab[b][m] = an[b][m];
        }
      j0 -= 8 * B;
    }
  } else {
    for (int j0 = n - 1; j0 > i; j0 -= 8) {
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int j = j0 - (s + G * m);
        if (j > i) acc[m] = fmaf(-Rc[col_off(j) + i], (float)(2 * (int)xp[j] - (P - 1)) * alpha, acc[m]);
      }
    }
  }
#pragma unroll
  for (int b = 1; b < 8; b <<= 1) {
    if (b < G) {
#pragma unroll
      for (int m = 0; m < M; ++m) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], b);
    } else {
      const int mb = b / G;
#pragma unroll
      for (int m = 0; m < M; ++m)
        if ((m & mb) == 0) acc[m] += acc[m + mb];
    }
  }
  return acc[0];
}

// 64-bit key helpers and one bitonic stage on a warp's 32 E register keys
// (element r * 32 + lane): strides below 32 by shuffles, larger ones inside
// the thread.
__device__ __forceinline__ uint64_t kmin(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t kmax(uint64_t a, uint64_t b) { return a < b ? b : a; }

template <int E>
__device__ __forceinline__ void run_stage(uint64_t (&key)[E], int lane, int size, int stride) {
  if (stride >= 32) {
    const int rs = stride >> 5;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      if ((r & rs) == 0) {
        const bool asc = (((r << 5) | lane) & size) == 0;
        const uint64_t a = key[r], b = key[r | rs];
        key[r] = asc ? kmin(a, b) : kmax(a, b);
        key[r | rs] = asc ? kmax(a, b) : kmin(a, b);
      }
    }
  } else {
    const bool lower = (lane & stride) == 0;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const uint64_t p = __shfl_xor_sync(0xffffffffu, key[r], stride);
      const bool asc = (((r << 5) | lane) & size) == 0;
      key[r] = (lower == asc) ? kmin(key[r], p) : kmax(key[r], p);
    }
  }
}

// Ascending bitonic sort of a warp's 32 E register keys.
template <int E>
__device__ __forceinline__ void run_sort(uint64_t (&key)[E], int lane) {
#pragma unroll
  for (int size = 2; size <= 32 * E; size <<= 1)
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) run_stage<E>(key, lane, size, stride);
}

// Key of child k of survivor t (partial distance ped, fields as below) whose
// P children sit on the aligned lanes base .. base + P - 1 of one register.
// The distance field is the running maximum of the partial distances along
// the survivor's Schnorr-Euchner order (increasing |u - k|, ties to the lower
// index), so that sorting keys (distance, parent rank, SE rank, child) orders
// and prunes the children exactly as the tournament of warp_kbest emits them:
// a survivor's stream ends at its first child outside the bound, and a child
// leaves its stream only after the ones before it.  Every lane of the warp
// must call this (shuffles inside).  SE = false gives the plain key
// (distance, parent rank, child) of the K-best of Sec. VI instead, each child
// pruned on its own distance.
template <int P, bool SE = true>
__device__ __forceinline__ uint64_t child_key(float ped, float u, int t, int k, bool act, float bnd, int lane) {
  if (!SE)
    return (act && ped < bnd) ? (((uint64_t)__float_as_uint(ped) << 32) | ((unsigned)t << 8) | (unsigned)k)
                              : kInfKey;
  const float dk = fabsf(u - (float)k);
  const int base = lane & ~(P - 1);
  float run = ped;
  int rank = 0;
#pragma unroll
  for (int k2 = 0; k2 < P; ++k2) {
    const float p2 = __shfl_sync(0xffffffffu, ped, base + k2);
    const float d2 = fabsf(u - (float)k2);
    if (d2 < dk || (d2 == dk && k2 < k)) {
      run = fmaxf(run, p2);
      ++rank;
    }
  }
  return (act && run < bnd)
             ? (((uint64_t)__float_as_uint(run) << 32) | ((unsigned)t << 8) | ((unsigned)rank << 4) | (unsigned)k)
             : kInfKey;
}

template <bool SE = true>
__device__ __forceinline__ uint64_t child_key(float ped, float u, int t, int k, int P, bool act, float bnd,
                                              int lane) {
  if (P == 8) return child_key<8, SE>(ped, u, t, k, act, bnd, lane);
  if (P == 4) return child_key<4, SE>(ped, u, t, k, act, bnd, lane);
  if (P == 2) return child_key<2, SE>(ped, u, t, k, act, bnd, lane);
  return child_key<16, SE>(ped, u, t, k, act, bnd, lane);
}

// One K-best level (row i) by one warp when the S P children fit in its lanes
// (S P <= 32, P <= 8): lanes t P .. t P + P - 1 compute survivor t's
// interference together (row_interference with G = P) and then child
// k = lane % P each; the keys of the first pow2ceil(S P) lanes (the rest are
// empty) are sorted in registers.  Writes the kept
// survivors (paths and partial distances, sorted) to xnxt / pnxt and returns
// their number.
template <int P, bool SE>
__device__ int warp_level_small_p(const float* Rc, const float* yb, int n, int K, int pp, float alpha, int i,
                                  float bnd, int S, const uint8_t* xcur, uint8_t* xnxt, const float* pcur,
                                  float* pnxt, int lane) {
  constexpr int lp = P == 8 ? 3 : (P == 4 ? 2 : 1);
  const int t = lane >> lp, k = lane & (P - 1);
  const bool act = t < S;
  const uint8_t* xp = xcur + (size_t)(act ? t : 0) * pp;
  const float c = row_interference<P>(Rc, yb, xp, n, P, alpha, i, k);
  const float rii = Rc[col_off(i) + i];
  const float rinv = 0.5f / (alpha * rii);
  const float p0 = act ? pcur[t] : 0.0f;
  const float u = fmaf(c, rinv, 0.5f * (float)(P - 1));
  const float d = fmaf(-rii, (float)(2 * k - (P - 1)) * alpha, c);
  const float ped = fmaf(d, d, p0);
  uint64_t key[1] = {child_key<P, SE>(ped, u, t, k, act, bnd, lane)};
  const int valid = __popc(__ballot_sync(0xffffffffu, key[0] != kInfKey));
  const int kept = min(K, valid);
  if (kept <= 8) {
    // few children inside the bound: take them smallest first (keys are unique)
    uint64_t mine = key[0], got = kInfKey;
    for (int s2 = 0; s2 < kept; ++s2) {
      const uint64_t m = warp_min_u64(mine);
      if (lane == s2) got = m;
      if (mine == m) mine = kInfKey;
    }
    key[0] = got;
  } else {
    // lanes from C = pow2ceil(S P) on hold only empty keys: sorting blocks of C suffices
    const int C = pow2ceil(S * P);
    for (int size = 2; size <= C; size <<= 1)
      for (int stride = size >> 1; stride > 0; stride >>= 1) run_stage<1>(key, lane, size, stride);
  }
  // slot s = lane: parent, child and partial distance (the parent's lanes hold c)
  const unsigned lo = (unsigned)key[0];
  const int ts = lane < kept ? (int)(lo >> 8) : 0, ks = (int)(lo & 15u);
  const float cs = __shfl_sync(0xffffffffu, c, (ts << lp) & 31);
  if (lane < kept) {
    const float ds = fmaf(-rii, (float)(2 * ks - (P - 1)) * alpha, cs);
    pnxt[lane] = fmaf(ds, ds, pcur[ts]);
  }
  // new paths: only the words holding rows i .. n-1 are copied (the lower rows
  // are written by the levels below before anything reads them)
  const int wpp = pp >> 2, w0 = i >> 2, sh = 8 * (i & 3);
  for (int s2 = 0; s2 < kept; ++s2) {
    const int tp = __shfl_sync(0xffffffffu, ts, s2), kp = __shfl_sync(0xffffffffu, ks, s2);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(xcur + (size_t)tp * pp);
    uint32_t* dst = reinterpret_cast<uint32_t*>(xnxt + (size_t)s2 * pp);
    for (int wd = w0 + lane; wd < wpp; wd += 32) {
      uint32_t word = src[wd];
      if (wd == w0) word = (word & ~(0xffu << sh)) | ((uint32_t)kp << sh);
      dst[wd] = word;
    }
  }
  __syncwarp();
  return kept;
}

template <bool SE = true>
__device__ int warp_level_small(const float* Rc, const float* yb, int n, int P, int K, int pp, float alpha, int i,
                                float bnd, int S, const uint8_t* xcur, uint8_t* xnxt, const float* pcur,
                                float* pnxt, int lane) {
  if (P == 8) return warp_level_small_p<8, SE>(Rc, yb, n, K, pp, alpha, i, bnd, S, xcur, xnxt, pcur, pnxt, lane);
  if (P == 4) return warp_level_small_p<4, SE>(Rc, yb, n, K, pp, alpha, i, bnd, S, xcur, xnxt, pcur, pnxt, lane);
  return warp_level_small_p<2, SE>(Rc, yb, n, K, pp, alpha, i, bnd, S, xcur, xnxt, pcur, pnxt, lane);
}

// One warp's K-best run over rows top..0 from the node (prefix path in
// *xcur[0], partial distance in (*pcur)[0]).  Selection is a tournament: the
// children of each survivor come out of its Schnorr-Euchner zig-zag in
// increasing distance, so the K best children of the level are the first K
// results of merging those sorted streams.  Lane l enumerates the children of
// survivors l, l+32, ... (SPL slots); each round a warp-wide arg-min over the
// lanes' current heads (ties to the lower parent rank) picks the next
// survivor and its lane advances that stream by one child.  The merge stops
// after K picks or when the smallest head leaves the sphere.  Returns the
// number of final survivors, sorted by partial distance in (*xcur, *pcur).
// SMALL: levels whose S P children fit in the warp's lanes take
// warp_level_small instead (the same selection, lower latency).
template <int SPL, bool SMALL = true>
__device__ int warp_kbest(const float* Rc, const float* yb, int n, int P, int K, int pp, float alpha, int top,
                          const unsigned int* r2bits, float E, uint16_t* sel, uint8_t** xcur, uint8_t** xnxt,
                          float** pcur, float** pnxt, int lane, long long* nodes, long long* flops) {
  const float uoff = 0.5f * (float)(P - 1);
  int S = 1;
  for (int i = top; i >= 0 && S > 0; --i) {
    float r2 = 0.0f;
    if (lane == 0) r2 = __uint_as_float(*(volatile const unsigned int*)r2bits);
    const float bnd = prune_bound(__shfl_sync(0xffffffffu, r2, 0), E, n);
    if (SMALL && S * P <= 32 && P <= 8) {
      // the level's children fit in the warp: the same selection without the tournament
      const int kept = warp_level_small(Rc, yb, n, P, K, pp, alpha, i, bnd, S, *xcur, *xnxt, *pcur, *pnxt, lane);
      *nodes += S;
      *flops += (long long)S * (2 * (n - 1 - i) + 4 * P);
      uint8_t* tx = *xcur;
      *xcur = *xnxt;
      *xnxt = tx;
      float* tp = *pcur;
      *pcur = *pnxt;
      *pnxt = tp;
      S = kept;
      continue;
    }
    const float rii = Rc[col_off(i) + i];
    const float rinv = 0.5f / (alpha * rii);
    float c[SPL], u[SPL], head[SPL], pp0[SPL];
    int lo[SPL], hi[SPL], kh[SPL];
#pragma unroll
    for (int t = 0; t < SPL; ++t) {
      const int sv = lane + 32 * t;
      head[t] = INFINITY;
      kh[t] = -1;
      lo[t] = -1;
      hi[t] = P;
      c[t] = 0.f;
      u[t] = 0.f;
      pp0[t] = 0.f;
      if (sv < S) {
        c[t] = row_interference<1>(Rc, yb, *xcur + (size_t)sv * pp, n, P, alpha, i, 0);
        pp0[t] = (*pcur)[sv];
        u[t] = fmaf(c[t], rinv, uoff);
        lo[t] = min(max((int)ceilf(u[t] - 0.5f), 0), P - 1);
        hi[t] = lo[t] + 1;
      }
    }
    // first child of every stream
#pragma unroll
    for (int t = 0; t < SPL; ++t) {
      if (lo[t] >= 0 || hi[t] < P) {
        const int k = (hi[t] >= P || (lo[t] >= 0 && fabsf(u[t] - (float)lo[t]) <= fabsf((float)hi[t] - u[t])))
                          ? lo[t]--
                          : hi[t]++;
        const float d = fmaf(-rii, (float)(2 * k - (P - 1)) * alpha, c[t]);
        const float pd = fmaf(d, d, pp0[t]);
        if (pd < bnd) {
          head[t] = pd;
          kh[t] = k;
        }
      }
    }
    int kept = 0;
    while (kept < K) {
      // this lane's smallest head, then the warp's (ties to the lower parent rank)
      uint64_t best = kInfKey;
#pragma unroll
      for (int t = 0; t < SPL; ++t) {
        if (kh[t] >= 0) {
          const uint64_t key = ((uint64_t)__float_as_uint(head[t]) << 32) | (unsigned)(lane + 32 * t);
          if (key < best) best = key;
        }
      }
      best = warp_min_u64(best);
      if (best == kInfKey) break;
      const int sv = (int)(best & 0xffffffffu);
      if ((sv & 31) == lane) {
        const int t = sv >> 5;
#pragma unroll
        for (int tt = 0; tt < SPL; ++tt) {
          if (tt == t) {
            sel[2 * kept] = (uint16_t)sv;
            sel[2 * kept + 1] = (uint16_t)kh[tt];
            (*pnxt)[kept] = head[tt];
            // advance this stream by one child
            kh[tt] = -1;
            head[tt] = INFINITY;
            if (lo[tt] >= 0 || hi[tt] < P) {
              const int k = (hi[tt] >= P ||
                             (lo[tt] >= 0 && fabsf(u[tt] - (float)lo[tt]) <= fabsf((float)hi[tt] - u[tt])))
                                ? lo[tt]--
                                : hi[tt]++;
              const float d = fmaf(-rii, (float)(2 * k - (P - 1)) * alpha, c[tt]);
              const float pd = fmaf(d, d, pp0[tt]);
              if (pd < bnd) {
                head[tt] = pd;
                kh[tt] = k;
              }
            }
          }
        }
      }
      ++kept;
    }
    __syncwarp();
    for (int t = lane; t < kept; t += 32) {
      const int par = sel[2 * t], k = sel[2 * t + 1];
      const uint32_t* src = reinterpret_cast<const uint32_t*>(*xcur + (size_t)par * pp);
      uint32_t* dst = reinterpret_cast<uint32_t*>(*xnxt + (size_t)t * pp);
      for (int w = 0; w < pp / 4; ++w) dst[w] = src[w];
      (*xnxt)[(size_t)t * pp + i] = (uint8_t)k;
    }
    *nodes += S;
    *flops += (long long)S * (2 * (n - 1 - i) + 4 * P);
    __syncwarp();
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

__device__ int warp_kbest_any(const float* Rc, const float* yb, int n, int P, int K, int pp, float alpha, int top,
                              const unsigned int* r2bits, float E, uint16_t* sel, uint8_t** xcur, uint8_t** xnxt,
                              float** pcur, float** pnxt, int lane, long long* nodes, long long* flops) {
  if (K <= 32)
    return warp_kbest<1>(Rc, yb, n, P, K, pp, alpha, top, r2bits, E, sel, xcur, xnxt, pcur, pnxt, lane, nodes, flops);
  if (K <= 64)
    return warp_kbest<2>(Rc, yb, n, P, K, pp, alpha, top, r2bits, E, sel, xcur, xnxt, pcur, pnxt, lane, nodes, flops);
  if (K <= 128)
    return warp_kbest<4>(Rc, yb, n, P, K, pp, alpha, top, r2bits, E, sel, xcur, xnxt, pcur, pnxt, lane, nodes, flops);
  return warp_kbest<8>(Rc, yb, n, P, K, pp, alpha, top, r2bits, E, sel, xcur, xnxt, pcur, pnxt, lane, nodes, flops);
}

}  // namespace
}  // namespace mdx
