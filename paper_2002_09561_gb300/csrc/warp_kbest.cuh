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
template <int SPL>
__device__ int warp_kbest(const float* Rc, const float* yb, int n, int P, int K, int pp, float alpha, int top,
                          const unsigned int* r2bits, float E, uint16_t* sel, uint8_t** xcur, uint8_t** xnxt,
                          float** pcur, float** pnxt, int lane, long long* nodes, long long* flops) {
  const float uoff = 0.5f * (float)(P - 1);
  int S = 1;
  for (int i = top; i >= 0 && S > 0; --i) {
    float r2 = 0.0f;
    if (lane == 0) r2 = __uint_as_float(*(volatile const unsigned int*)r2bits);
    const float bnd = prune_bound(__shfl_sync(0xffffffffu, r2, 0), E, n);
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
        const uint8_t* xp = *xcur + (size_t)sv * pp;
        // interference of row i: four independent partial sums over j > i
        float a0 = yb[i], a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int j = n - 1;
        for (; j - 3 > i; j -= 4) {
          a0 = fmaf(-Rc[col_off(j) + i], (float)(2 * (int)xp[j] - (P - 1)) * alpha, a0);
          a1 = fmaf(-Rc[col_off(j - 1) + i], (float)(2 * (int)xp[j - 1] - (P - 1)) * alpha, a1);
          a2 = fmaf(-Rc[col_off(j - 2) + i], (float)(2 * (int)xp[j - 2] - (P - 1)) * alpha, a2);
          a3 = fmaf(-Rc[col_off(j - 3) + i], (float)(2 * (int)xp[j - 3] - (P - 1)) * alpha, a3);
        }
        for (; j > i; --j) a0 = fmaf(-Rc[col_off(j) + i], (float)(2 * (int)xp[j] - (P - 1)) * alpha, a0);
        c[t] = (a0 + a1) + (a2 + a3);
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
