// Uneven batches: one persistent search kernel over requests that differ in
// antennas, modulation, detector and K (the batching layer around the
// paper's detectors; the paper runs one system at a time).
//
// Every warp of the grid takes requests from a global counter, in the order
// the host chose (heaviest classes first), and searches each one alone:
//   exact SD   Algorithm 1 with Schnorr-Euchner child order (Sec. IV-A) and
//              incremental partial distances (Eq. inc), one warp walking the
//              whole tree: lanes own rows, the residual of every row below the
//              current level sits in a stack zs[level][row], so a descent
//              costs one FMA per lower row, every lane forms the next
//              interference from row i - 1 itself, and a node whose nearest
//              child is outside the sphere is counted but not entered;
//   K-best     Sec. VI, selection of the K best children per level by a
//              warp tournament over the survivors' Schnorr-Euchner child
//              streams (warp_kbest.cuh).
// Each warp owns a slice of the CTA's shared memory and a slot of global
// memory.  Per request class the tuner decides whether R and ybar are copied
// into the slice (MIX_STAGE_R) and whether the search state (SD stacks and
// leaf candidates, or K-best survivor paths) lives in the slice
// (MIX_STATE_SMEM) or in the global slot; the kernel uses generic pointers,
// so one code path serves every placement.  Leaves within the FP32 error
// bound of the best are re-scored in FP64 against the FP64 R and ybar.
#include "mdx_internal.cuh"
#include "warp_kbest.cuh"

namespace mdx {
namespace {

constexpr int kMixCand = 8;  // SD leaf candidates kept per request

__host__ __device__ inline size_t stage_bytes(int n) {
  return sizeof(float) * ((size_t)tri_stride32(n) + round_up(n, 4));
}

__host__ __device__ inline int mix_path_pad(int n) { return round_up(n, 16); }

__host__ __device__ inline size_t sd_state_bytes(int n) {
  const size_t n4 = (size_t)round_up(n, 4);
  const size_t b = sizeof(float) * (round_up(tri(n), 4) + 5 * n4) + sizeof(int) * n4 + sizeof(float) * kMixCand +
                   (size_t)mix_path_pad(n) * (1 + kMixCand);
  return (b + 15) / 16 * 16;
}

// Complex-tree SD: residual stack, per complex level {parent distance, c of
// row 2j+1, c of row 2j before x_{2j+1}, visited-children mask low word} and
// the mask's high word, level constants {R_{2j+1,2j+1}, R_{2j,2j+1}, R_{2j,2j}},
// candidates, path.
__host__ __device__ inline size_t sdc_state_bytes(int n) {
  const size_t M = (size_t)n / 2;
  const size_t b = sizeof(float) * round_up(tri(n), 4) + 16 * M + sizeof(unsigned) * round_up((int)M, 4) +
                   16 * M + sizeof(float) * kMixCand + (size_t)mix_path_pad(n) * (1 + kMixCand);
  return (b + 15) / 16 * 16;
}

__host__ __device__ inline size_t kb_state_bytes(int n, int K) {
  const size_t b = 16 + 2 * sizeof(float) * round_up(K, 4) + 2 * sizeof(uint16_t) * round_up(K, 8) +
                   2 * (size_t)path_stride(n) * K;
  return (b + 15) / 16 * 16;
}

__device__ float initial_r2(const MixedArgs& g, const MixedReq& q, int r) {
  float r2;
  if (q.radius_mode == RADIUS_PER_VECTOR) r2 = g.r2_vec[r];
  else if (q.radius_mode == RADIUS_NONE) r2 = INFINITY;
  else if (q.radius_mode == RADIUS_PAPER) r2 = (float)((double)q.n_rx * q.n_tx * g.noise_var[r]);
  else r2 = (float)q.radius_value;
  return (r2 > 0.0f) ? r2 : INFINITY;
}

// Picks, among nc candidate paths (stride cs bytes) with FP32 distances cped,
// the one of least FP64 metric (ties: smaller index vector, top row first)
// among those within the FP32 error bound of the best; writes the request's
// outputs.  All lanes call it.
__device__ void finish_request(const MixedArgs& g, const MixedReq& q, int r, const uint8_t* cx, int cs,
                               const float* cped, int nc, float E, int status, long long nodes, long long peds,
                               long long restarts, long long flops, int lane) {
  const int n = q.n, P = q.P;
  float best = INFINITY;
  for (int k = 0; k < nc; ++k) best = fminf(best, cped[k]);
  const float keep = prune_bound(best, E, n);
  const double* R64 = g.R64 + q.r_off64;
  const double* y64 = g.yb64 + q.y_off64;
  int win = -1;
  double win_m = INFINITY;
  long long rescored = 0;
  for (int k = 0; k < nc; ++k) {
    if (!(cped[k] <= keep)) continue;
    double m;
    if (g.flags & MDX_NO_RESCORE) {
      m = (double)cped[k];
    } else {
      m = rescore_fp64_warp(n, P, q.alpha64, R64, y64, cx + (size_t)k * cs, lane);
      ++rescored;
    }
    bool better = m < win_m;
    if (!better && m == win_m && win >= 0) {
      for (int j = n - 1; j >= 0; --j) {
        const int x1 = cx[(size_t)k * cs + j], x2 = cx[(size_t)win * cs + j];
        if (x1 != x2) {
          better = x1 < x2;
          break;
        }
      }
    }
    if (better) {
      win = k;
      win_m = m;
    }
  }
  uint8_t* so = g.sym_out + q.sym_off;
  for (int j = lane; j < q.n_tx; j += 32)
    so[j] = (win >= 0) ? (uint8_t)(cx[(size_t)win * cs + 2 * j] * P + cx[(size_t)win * cs + 2 * j + 1]) : 0;
  if (lane == 0) {
    g.metric_out[r] = (win >= 0) ? win_m : (double)INFINITY;
    g.vstatus[r] = status;
    if (g.stats) {
      int64_t* s = g.stats + (size_t)r * kStats;
      s[0] = nodes;
      s[1] = peds;
      s[2] = restarts;
      s[3] = rescored;
      s[4] = flops;
    }
  }
}

// Exact SD of one request by one warp (ROWS = rows per lane, n <= 32 ROWS).
// In Schnorr-Euchner order a visited node's next sibling is evaluated with
// it; outside the sphere it finishes the level (the bound only shrinks), and
// a pop goes straight to the nearest level above with a sibling left inside
// (each level keeps that return level), so no iteration is spent climbing
// through finished levels.  NAT: children in natural index order (the
// unsorted depth-first search the paper compares against, Sec. IV-A)
// instead; a child outside the sphere then does not end its level, and pops
// go up one level at a time.
template <int ROWS, bool NAT>
__device__ void sd_request(const MixedArgs& g, const MixedReq& q, int r, const float* Rc, const float* yb,
                           unsigned char* st, float E, int lane) {
  const int n = q.n, P = q.P, n4 = round_up(n, 4);
  const float alpha = q.alpha, uoff = 0.5f * (float)(P - 1);
  float* zs = reinterpret_cast<float*>(st);
  float* lv_ped = zs + round_up(tri(n), 4);
  float* lv_c = lv_ped + n4;
  float* lv_u = lv_c + n4;
  float* lv_rii = lv_u + n4;
  float* lv_rinv = lv_rii + n4;
  int* lv_lohi = reinterpret_cast<int*>(lv_rinv + n4);
  float* cped = reinterpret_cast<float*>(lv_lohi + n4);
  uint8_t* xs = reinterpret_cast<uint8_t*>(cped + kMixCand);
  uint8_t* cx = xs + mix_path_pad(n);
  const int cs = mix_path_pad(n);

  for (int rr = lane; rr < n; rr += 32) {
    const float d = Rc[col_off(rr) + rr];
    lv_rii[rr] = d;
    lv_rinv[rr] = 0.5f / (alpha * d);
  }
  float r2_start = initial_r2(g, q, r);
  float r2 = r2_start;
  long long nodes = 0, peds = 0, flops = 0;
  int restarts = 0, ncand = 0;
  bool bh = false;
  for (;;) {
    // the root: z_r = ybar_r for every row
#pragma unroll
    for (int t = 0; t < ROWS; ++t) {
      const int rr = lane + 32 * t;
      if (rr < n) zs[col_off(n - 1) + rr] = yb[rr];
    }
    __syncwarp();
    float bnd = prune_bound(r2, E, n);
    int i = n - 1;
    // sorted order: the level a pop from level i goes to, the nearest level
    // above whose next child was inside the sphere when the path left it
    // (n: none); the levels in between have no child left to try
    int ret = n;
    float ped_par = 0.0f;
    float c = zs[col_off(i) + i];
    float rii = lv_rii[i];
    float u = fmaf(c, lv_rinv[i], uoff);
    int lo = NAT ? 0 : min(max((int)ceilf(u - 0.5f), 0), P - 1);
    int hi = NAT ? P : lo + 1;
    ++nodes;
    flops += 4 * P;
    for (;;) {
      int k = -1;
      if (NAT) {
        if (lo < P) k = lo++;
      } else if (lo >= 0 || hi < P) {
        if (hi >= P || (lo >= 0 && fabsf(u - (float)lo) <= fabsf((float)hi - u))) k = lo--;
        else k = hi++;
      }
      float ped = INFINITY;
      if (k >= 0) {
        const float d = fmaf(-rii, (float)(2 * k - (P - 1)) * alpha, c);
        ped = fmaf(d, d, ped_par);
        ++peds;
      }
      if (NAT && k >= 0 && !(ped < bnd)) continue;  // unsorted: try the next child
      // sorted order: whether the level's next child (the one a later
      // iteration would take) is outside the sphere now, evaluated with the
      // same operations; the bound only shrinks, so then it is outside then
      // and nothing at this level is left to try
      auto level_done = [&]() {
        if (lo < 0 && hi >= P) return true;
        const int k2 = (hi >= P || (lo >= 0 && fabsf(u - (float)lo) <= fabsf((float)hi - u))) ? lo : hi;
        const float d2 = fmaf(-rii, (float)(2 * k2 - (P - 1)) * alpha, c);
        if (fmaf(d2, d2, ped_par) < bnd) return false;
        ++peds;  // the evaluation that ends the level, made here
        return true;
      };
      bool up = k < 0 || !(ped < bnd);
      if (i == 0 && !up) {
        // leaf inside the sphere: keep it among the kMixCand best, shrink the radius
        int slot = -1;
        if (lane == 0) {
          xs[0] = (uint8_t)k;
          if (ncand < kMixCand) {
            slot = ncand;
          } else {
            float worst = -1.0f;
            for (int t = 0; t < kMixCand; ++t)
              if (cped[t] > worst) {
                worst = cped[t];
                slot = t;
              }
            if (!(ped < worst)) slot = -1;
          }
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        __syncwarp();
        if (slot >= 0) {
          for (int rr = lane; rr < n; rr += 32) cx[(size_t)slot * cs + rr] = xs[rr];
          if (lane == 0) cped[slot] = ped;
          if (slot == ncand) ++ncand;
        }
        __syncwarp();
        if (ped < r2) {
          r2 = ped;
          bnd = prune_bound(r2, E, n);
        }
        if (NAT || !level_done()) continue;
        up = true;
      }
      if (up) {
        if (NAT) {
          if (i == n - 1) break;  // the root is exhausted
          ++i;                    // backtrack
        } else {
          if (ret >= n) break;  // no level above has a child left
          i = ret;              // back to the nearest level with one
        }
        ped_par = lv_ped[i];
        c = lv_c[i];
        u = lv_u[i];
        rii = lv_rii[i];
        const int lh = lv_lohi[i];
        lo = (lh & 0xff) - 1;
        if (!NAT) ret = (lh >> 8) & 0xff;
        hi = lh >> 16;
        continue;
      }
      if (q.budget > 0 && nodes >= q.budget) {
        bh = true;
        break;
      }
      // descend into child k: push level i, update the residuals of the rows below
      const float av = (float)(2 * k - (P - 1)) * alpha;
      const float* zin = zs + col_off(i);
      const float* rc = Rc + col_off(i);
      // the next level's interference, computed by every lane from row i - 1
      // (the same FMA as that row's residual below; the column was written
      // before the last warp barrier), and the new level's first child, the
      // PAM index nearest u (sorted order only): outside the sphere it rules
      // out every child, so the node is counted with that one evaluation and
      // the search goes on at level i
      const float cnext = fmaf(-rc[i - 1], av, zin[i - 1]);
      const float unext = fmaf(cnext, lv_rinv[i - 1], uoff);
      const int lonext = NAT ? 0 : min(max((int)ceilf(unext - 0.5f), 0), P - 1);
      bool done_here = false;
      if (!NAT) {
        const float d1 = fmaf(-lv_rii[i - 1], (float)(2 * lonext - (P - 1)) * alpha, cnext);
        done_here = level_done();
        if (!(fmaf(d1, d1, ped) < bnd)) {
          ++nodes;
          ++peds;
          flops += 2 * (n - i) + 4 * P;
          if (!done_here) continue;
          // nothing else at this level: back to the return level
          if (ret >= n) break;
          i = ret;
          ped_par = lv_ped[i];
          c = lv_c[i];
          u = lv_u[i];
          rii = lv_rii[i];
          const int lh = lv_lohi[i];
          lo = (lh & 0xff) - 1;
          ret = (lh >> 8) & 0xff;
          hi = lh >> 16;
          continue;
        }
      }
      if (lane == 0) {
        lv_ped[i] = ped_par;
        lv_c[i] = c;
        lv_u[i] = u;
        lv_lohi[i] = (lo + 1) | (NAT ? 0 : ret << 8) | (hi << 16);
        xs[i] = (uint8_t)k;
      }
      if (!NAT && !done_here) ret = i;
      float* zout = zs + col_off(i - 1);
#pragma unroll
      for (int t = 0; t < ROWS; ++t) {
        const int rr = lane + 32 * t;
        if (rr < i) zout[rr] = fmaf(-rc[rr], av, zin[rr]);
      }
      --i;
      __syncwarp();
      c = cnext;
      ped_par = ped;
      rii = lv_rii[i];
      u = unext;
      lo = lonext;
      hi = NAT ? P : lo + 1;
      ++nodes;
      flops += 2 * (n - 1 - i) + 4 * P;
    }
    if (ncand == 0 && !bh && r2_start < INFINITY && restarts < 64) {
      // empty sphere: r^2 <- 2 r^2 and search again
      r2_start *= 2.0f;
      r2 = r2_start;
      ++restarts;
      continue;
    }
    break;
  }
  __syncwarp();
  const int status = bh ? MDX_V_BUDGET_EXCEEDED : (restarts > 0 ? MDX_V_EMPTY_RETRIED : MDX_V_OK);
  finish_request(g, q, r, cx, cs, cped, ncand, E, status, nodes, peds, restarts, flops, lane);
}

// Complex-tree exact SD of one request by one warp: one tree level per complex
// antenna j (real rows 2j+1, then 2j), Q = P^2 children.  The next child of a
// node is the unvisited one of least partial distance (ties to the lower q),
// found by a warp arg-min; a level is exhausted when that child leaves the
// sphere.  A descent updates the residuals of the rows below by both fixed
// rows; the rest (candidates, radius shrink and doubling, budget, FP64
// re-scoring) is as in sd_request.
template <int ROWS>
__device__ void sdc_request(const MixedArgs& g, const MixedReq& q, int r, const float* Rc, const float* yb,
                            unsigned char* st, float E, int lane) {
  const int n = q.n, P = q.P, Q = P * P, M = n / 2;
  const float alpha = q.alpha;
  float* zs = reinterpret_cast<float*>(st);
  float4* lv = reinterpret_cast<float4*>(zs + round_up(tri(n), 4));
  unsigned* lv_hi = reinterpret_cast<unsigned*>(lv + M);
  float4* lv_r = reinterpret_cast<float4*>(lv_hi + round_up(M, 4));
  float* cped = reinterpret_cast<float*>(lv_r + M);
  uint8_t* xs = reinterpret_cast<uint8_t*>(cped + kMixCand);
  uint8_t* cx = xs + mix_path_pad(n);
  const int cs = mix_path_pad(n);
  for (int j = lane; j < M; j += 32) {
    const int r1 = 2 * j + 1, r0 = 2 * j;
    lv_r[j] = make_float4(Rc[col_off(r1) + r1], Rc[col_off(r1) + r0], Rc[col_off(r0) + r0], 0.0f);
  }
  float r2_start = initial_r2(g, q, r);
  float r2 = r2_start;
  long long nodes = 0, peds = 0, flops = 0;
  int restarts = 0, ncand = 0;
  bool bh = false;
  for (;;) {
#pragma unroll
    for (int t = 0; t < ROWS; ++t) {
      const int rr = lane + 32 * t;
      if (rr < n) zs[col_off(n - 1) + rr] = yb[rr];
    }
    __syncwarp();
    float bnd = prune_bound(r2, E, n);
    int j = M - 1;
    float ped_par = 0.0f;
    float c1 = zs[col_off(n - 1) + n - 1], c0 = zs[col_off(n - 1) + n - 2];
    float4 rl = lv_r[j];
    unsigned long long mask = 0ull;
    ++nodes;
    peds += Q;
    flops += 10 * Q;
    for (;;) {
      // the unvisited child of least partial distance
      unsigned long long best = ~0ull;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int qq = lane + 32 * t;
        if (qq < Q && !((mask >> qq) & 1ull)) {
          const int kre = qq / P, kim = qq - kre * P;
          const float aim = (float)(2 * kim - (P - 1)) * alpha, are = (float)(2 * kre - (P - 1)) * alpha;
          const float d1 = fmaf(-rl.x, aim, c1);
          const float p1 = fmaf(d1, d1, ped_par);
          const float d0 = fmaf(-rl.z, are, fmaf(-rl.y, aim, c0));
          const float pd = fmaf(d0, d0, p1);
          const unsigned long long key = ((unsigned long long)__float_as_uint(pd) << 32) | (unsigned)qq;
          if (key < best) best = key;
        }
      }
      best = warp_min_u64(best);
      const float ped = (best == ~0ull) ? INFINITY : __uint_as_float((unsigned)(best >> 32));
      if (!(ped < bnd)) {
        if (j == M - 1) break;  // the root is exhausted
        ++j;                    // backtrack
        const float4 s4 = lv[j];
        ped_par = s4.x;
        c1 = s4.y;
        c0 = s4.z;
        mask = (unsigned long long)__float_as_uint(s4.w) | ((unsigned long long)lv_hi[j] << 32);
        rl = lv_r[j];
        continue;
      }
      const int qk = (int)(best & 0xffffffffu);
      mask |= 1ull << qk;
      const int kre = qk / P, kim = qk - kre * P;
      if (j == 0) {
        // leaf inside the sphere: keep it among the kMixCand best, shrink the radius
        int slot = -1;
        if (lane == 0) {
          xs[1] = (uint8_t)kim;
          xs[0] = (uint8_t)kre;
          if (ncand < kMixCand) {
            slot = ncand;
          } else {
            float worst = -1.0f;
            for (int t = 0; t < kMixCand; ++t)
              if (cped[t] > worst) {
                worst = cped[t];
                slot = t;
              }
            if (!(ped < worst)) slot = -1;
          }
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        __syncwarp();
        if (slot >= 0) {
          for (int rr = lane; rr < n; rr += 32) cx[(size_t)slot * cs + rr] = xs[rr];
          if (lane == 0) cped[slot] = ped;
          if (slot == ncand) ++ncand;
        }
        __syncwarp();
        if (ped < r2) {
          r2 = ped;
          bnd = prune_bound(r2, E, n);
        }
        continue;
      }
      if (q.budget > 0 && nodes >= q.budget) {
        bh = true;
        break;
      }
      // descend: push level j, update the residuals of rows 0..2j-1 by both fixed rows
      const float aim = (float)(2 * kim - (P - 1)) * alpha, are = (float)(2 * kre - (P - 1)) * alpha;
      if (lane == 0) {
        lv[j] = make_float4(ped_par, c1, c0, __uint_as_float((unsigned)mask));
        lv_hi[j] = (unsigned)(mask >> 32);
        xs[2 * j + 1] = (uint8_t)kim;
        xs[2 * j] = (uint8_t)kre;
      }
      const float* zin = zs + col_off(2 * j + 1);
      float* zout = zs + col_off(2 * j - 1);
      const float* ra = Rc + col_off(2 * j + 1);
      const float* rb = Rc + col_off(2 * j);
      float n1 = 0.0f, n0 = 0.0f;
#pragma unroll
      for (int t = 0; t < ROWS; ++t) {
        const int rr = lane + 32 * t;
        if (rr < 2 * j) {
          const float z = fmaf(-rb[rr], are, fmaf(-ra[rr], aim, zin[rr]));
          zout[rr] = z;
          if (rr == 2 * j - 1) n1 = z;
          if (rr == 2 * j - 2) n0 = z;
        }
      }
      --j;
      c1 = __shfl_sync(0xffffffffu, n1, (2 * j + 1) & 31);
      c0 = __shfl_sync(0xffffffffu, n0, (2 * j) & 31);
      __syncwarp();
      ped_par = ped;
      rl = lv_r[j];
      mask = 0ull;
      ++nodes;
      peds += Q;
      flops += 4 * (n - 2 - 2 * j) + 10 * Q;
    }
    if (ncand == 0 && !bh && r2_start < INFINITY && restarts < 64) {
      r2_start *= 2.0f;  // empty sphere: r^2 <- 2 r^2 and search again
      r2 = r2_start;
      ++restarts;
      continue;
    }
    break;
  }
  __syncwarp();
  const int status = bh ? MDX_V_BUDGET_EXCEEDED : (restarts > 0 ? MDX_V_EMPTY_RETRIED : MDX_V_OK);
  finish_request(g, q, r, cx, cs, cped, ncand, E, status, nodes, peds, restarts, flops, lane);
}

// K-best of one request by one warp (SPL survivor slots per lane, K <= 32 SPL).
template <int SPL>
__device__ void kb_request(const MixedArgs& g, const MixedReq& q, int r, const float* Rc, const float* yb,
                           unsigned char* st, float E, int lane) {
  const int n = q.n, P = q.P, K = q.K, pp = path_stride(n);
  unsigned int* r2w = reinterpret_cast<unsigned int*>(st);
  float* pa = reinterpret_cast<float*>(st + 16);
  float* pb = pa + round_up(K, 4);
  uint16_t* sel = reinterpret_cast<uint16_t*>(pb + round_up(K, 4));
  uint8_t* xa = reinterpret_cast<uint8_t*>(sel + 2 * round_up(K, 8));
  uint8_t* xb = xa + (size_t)pp * K;
  float r2 = initial_r2(g, q, r);
  long long nodes = 0, flops = 0;
  int restarts = 0, S = 0;
  uint8_t *xcur = xa, *xnxt = xb;
  float *pcur = pa, *pnxt = pb;
  for (;;) {
    xcur = xa;
    xnxt = xb;
    pcur = pa;
    pnxt = pb;
    if (lane == 0) {
      *r2w = __float_as_uint(r2);
      pa[0] = 0.0f;
    }
    __syncwarp();
    S = warp_kbest<SPL, false>(Rc, yb, n, P, K, pp, q.alpha, n - 1, r2w, E, sel, &xcur, &xnxt, &pcur, &pnxt, lane, &nodes,
                        &flops);
    __syncwarp();
    if (S > 0 || !(r2 < INFINITY) || restarts >= 64) break;
    r2 *= 2.0f;  // every survivor left the sphere: r^2 <- 2 r^2
    ++restarts;
  }
  const int nc = S < kCandMax ? S : kCandMax;
  finish_request(g, q, r, xcur, pp, pcur, nc, E, restarts > 0 ? MDX_V_EMPTY_RETRIED : MDX_V_OK, nodes,
                 nodes * P, restarts, flops, lane);
}

template <int KSPL>
__global__ void mixed_kernel(MixedArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, W = blockDim.x >> 5;
  unsigned char* slice = smem + (size_t)warp * g.slice_bytes;
  unsigned char* gslot = g.gscratch + ((size_t)blockIdx.x * W + warp) * g.gslot_bytes;
  for (;;) {
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(g.counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= (unsigned int)g.nreq) break;
    const int r = g.order ? g.order[t] : (int)t;
    MixedReq q;
    if (g.reqs) {
      q = g.reqs[r];
    } else {
      q = g.uniform;
      q.r_off = (long long)r * tri_stride32(q.n);
      q.y_off = (long long)r * vec_stride32(q.n);
      q.r_off64 = (long long)r * tri_stride64(q.n);
      q.y_off64 = (long long)r * vec_stride64(q.n);
      q.sym_off = (long long)r * q.n_tx;
    }
    if (g.singular[r]) {
      for (int j = lane; j < q.n_tx; j += 32) g.sym_out[q.sym_off + j] = 0;
      if (lane == 0) {
        g.metric_out[r] = 0.0;
        g.vstatus[r] = MDX_V_SINGULAR;
        if (g.stats)
          for (int k = 0; k < kStats; ++k) g.stats[(size_t)r * kStats + k] = 0;
      }
      continue;
    }
    const float* Rc = g.R32 + q.r_off;
    const float* yb = g.yb32 + q.y_off;
    unsigned char* st = gslot;
    if (q.mode & MIX_STAGE_R) {
      const int ts = tri_stride32(q.n);
      float* sR = reinterpret_cast<float*>(slice);
      float* sy = sR + ts;
      const float4* src = reinterpret_cast<const float4*>(Rc);
      for (int k = lane; k < ts / 4; k += 32) reinterpret_cast<float4*>(sR)[k] = src[k];
      for (int k = lane; k < q.n; k += 32) sy[k] = yb[k];
      Rc = sR;
      yb = sy;
      if (q.mode & MIX_STATE_SMEM) st = slice + stage_bytes(q.n);
    } else if (q.mode & MIX_STATE_SMEM) {
      st = slice;
    }
    __syncwarp();
    const float E = error_scale_warp(q.n, q.P, q.alpha, Rc, yb, lane);
    if (q.algo == MDX_ALGO_SD) {
      if (q.n <= 32) sd_request<1, false>(g, q, r, Rc, yb, st, E, lane);
      else if (q.n <= 64) sd_request<2, false>(g, q, r, Rc, yb, st, E, lane);
      else if (q.n <= 128) sd_request<4, false>(g, q, r, Rc, yb, st, E, lane);
      else sd_request<7, false>(g, q, r, Rc, yb, st, E, lane);
    } else if (q.algo == MIX_ALGO_SD_NATURAL) {
      if (q.n <= 32) sd_request<1, true>(g, q, r, Rc, yb, st, E, lane);
      else if (q.n <= 64) sd_request<2, true>(g, q, r, Rc, yb, st, E, lane);
      else if (q.n <= 128) sd_request<4, true>(g, q, r, Rc, yb, st, E, lane);
      else sd_request<7, true>(g, q, r, Rc, yb, st, E, lane);
    } else if (q.algo == MIX_ALGO_SD_COMPLEX) {
      if (q.n <= 32) sdc_request<1>(g, q, r, Rc, yb, st, E, lane);
      else if (q.n <= 64) sdc_request<2>(g, q, r, Rc, yb, st, E, lane);
      else if (q.n <= 128) sdc_request<4>(g, q, r, Rc, yb, st, E, lane);
      else sdc_request<7>(g, q, r, Rc, yb, st, E, lane);
    } else {
      if (q.K <= 32) kb_request<1>(g, q, r, Rc, yb, st, E, lane);
      else if (KSPL <= 2 || q.K <= 64) kb_request<2>(g, q, r, Rc, yb, st, E, lane);
      else if constexpr (KSPL > 2) {
        if (q.K <= 128) kb_request<4>(g, q, r, Rc, yb, st, E, lane);
        else kb_request<8>(g, q, r, Rc, yb, st, E, lane);
      }
    }
    __syncwarp();
  }
}

template <int KSPL>
cudaError_t prepare(int W, int slice_bytes, int num_sms, int* grid) {
  const int smem = W * slice_bytes;
  cudaError_t e = cudaFuncSetAttribute(mixed_kernel<KSPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mixed_kernel<KSPL>, W * 32, (size_t)smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = per_sm * num_sms;
  return cudaSuccess;
}

}  // namespace

size_t mixed_stage_bytes(int n) { return stage_bytes(n); }

size_t mixed_state_bytes(int algo, int n, int K, int P) {
  (void)P;
  if (algo == MDX_ALGO_SD || algo == MIX_ALGO_SD_NATURAL) return sd_state_bytes(n);
  if (algo == MIX_ALGO_SD_COMPLEX) return sdc_state_bytes(n);
  return kb_state_bytes(n, K);
}

int mixed_greedy_mode(int algo, int n, int K, int P, int slice) {
  const size_t stage = stage_bytes(n), state = mixed_state_bytes(algo, n, K, P);
  if (stage + state <= (size_t)slice) return MIX_STAGE_R | MIX_STATE_SMEM;
  if (state <= (size_t)slice) return MIX_STATE_SMEM;
  if (stage <= (size_t)slice) return MIX_STAGE_R;
  return 0;
}

int mixed_resident_warps(int W, int slice_bytes, int max_K, int num_sms) {
  int grid = 0;
  const cudaError_t e = (max_K > 64) ? prepare<8>(W, slice_bytes, num_sms, &grid)
                                     : prepare<2>(W, slice_bytes, num_sms, &grid);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return grid * W;
}

cudaError_t launch_mixed(const MixedArgs& a, int W, int max_K, int num_sms, cudaStream_t s) {
  if (a.nreq <= 0) return cudaSuccess;
  if (W < 1 || W > 32 || a.slice_bytes < 0 || (a.slice_bytes & 15)) return cudaErrorInvalidConfiguration;
  int grid = 0;
  cudaError_t e = (max_K > 64) ? prepare<8>(W, a.slice_bytes, num_sms, &grid)
                               : prepare<2>(W, a.slice_bytes, num_sms, &grid);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)W * a.slice_bytes;
  if (max_K > 64) mixed_kernel<8><<<grid, W * 32, smem, s>>>(a);
  else mixed_kernel<2><<<grid, W * 32, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mdx
