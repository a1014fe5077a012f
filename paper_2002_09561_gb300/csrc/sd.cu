// Exact sphere decoder (Sec. III-B, Algorithm 1) with Best-FS /
// Schnorr-Euchner child order (Sec. IV-A), incremental partial distances
// (Sec. IV-C, Eq. inc) and dynamic subtree splitting between warps (the
// load balancing of the paper's parallel SD, Sec. V-C, recast for a GPU).
//
// This warp-per-task kernel serves n > 32 (more than 16 transmit antennas);
// smaller systems take the group kernel of sd_group.cu, which runs the same
// search with four vectors per warp.
//
// Unit of work: a task = one tree node (rows n-1..L+1 fixed, row L to
// expand) of one vector, explored depth-first by one warp.  A vector starts
// as its root task.  Warps take work in this order: a queued task, else a
// fresh vector (heaviest first, see launch_sd), else they wait (idle).  While any warp is idle, a busy warp
// checks every kSplitEvery nodes and donates all untried children of its
// top-most open level whose next child is inside the sphere as new tasks,
// marking that level exhausted.  The only
// state the tasks of a vector share is its radius (an FP32 r^2 in global
// memory, shrunk with atomicMin) and its leaf-candidate list; a per-vector
// count of unfinished tasks tells the warp finishing the last one to
// re-score the candidates in FP64 and write the result.  Every answer is the
// one the sequential search gives: the subtrees partition the tree and
// pruning only ever uses a radius that some leaf of the vector has reached.
//
// One node step.  Lane l owns the rows r = l + 32 t (t < ROWS).  For the
// node at level i (rows n-1..i+1 fixed) the residual of every lower row,
//   z_r = ybar_r - sum_{j > i} R_rj x_j   (r <= i),
// is kept in a shared-memory stack zs[level i][r]; descending into child
// x_i = a costs one FMA per row below (z_r -= R_ri a), and every lane forms
// the interference of the next row itself from row i - 1 (read after the
// warp barrier that ends each descent); a node whose nearest child is
// outside the sphere is counted but not entered.
// Each partial distance is one FMA chain in a fixed order (j = n-1 down to
// i+1), identical whether a node is reached by descent or rebuilt from a
// task's path.  The control state of the current level is warp-uniform and
// lives in registers; it is pushed to shared memory on descent and popped on
// backtrack.  Children are visited in increasing (c_i - R_ii a_k)^2 by a
// zig-zag around u_i = c_i / (2 alpha R_ii) + (P-1)/2 in PAM-index space,
// ties to the lower index; a child reaching the pruning bound ends the level.
// A visited node's next sibling is evaluated with it: outside the sphere (the
// bound only shrinks) it ends its level at once, and a pop goes straight to
// the nearest level above with a sibling left inside, which each level keeps
// packed with its cursors.
//
// The task queue is a ring: a consumer claims an index, waits for the
// producer's sequence number, copies the record and marks the slot free; a
// producer that wraps onto a slot waits for that mark before writing.
// Every spin-wait is bounded: a claimed slot that never becomes ready, a slot
// that is never freed or a candidate lock that is never released sets the
// launch's error word and the warp moves on; an idle warp that waits too
// long simply exits (the busy warps drain the queue themselves before they
// finish).
#include "sd_common.cuh"

namespace mdx {

namespace {

// Blocks per SM the register allocation is made for: for n <= 32 the shared
// memory allows up to eight 4-warp blocks; six (80 registers, no spills)
// measured fastest for the learned-radius search, larger n allows fewer.
#ifndef MDX_SD_MIN_BLOCKS_N32
#define MDX_SD_MIN_BLOCKS_N32 6
#endif
template <int ROWS>
__global__ void __launch_bounds__(kWarpsMax * 32, ROWS == 1 ? MDX_SD_MIN_BLOCKS_N32 : (ROWS == 2 ? 3 : 1))
    sd_kernel(SdArgs g) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SearchArgs& a = g.a;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.n, P = a.P;
  // a vector's tree is split between warps unless the search is sequential or
  // has a node budget (a cap per vector, which tasks running at once could
  // only check between periodic checks)
  const bool may_split = !(a.flags & MDX_SEQUENTIAL_SEARCH) && a.budget <= 0;
  const int ts = tri_stride32(n);
  unsigned char* base = smem + warp * sd_warp_bytes(n);
  float* Rc = reinterpret_cast<float*>(base);  // column-packed R (FP32)
  float* zs = Rc + ts;                          // residual stack, level i at col_off(i)
  // per level: {parent partial distance, c_i, u_i, zig-zag cursors (lo + 1) | hi << 16
  // as bits}, pushed and popped as one 16-byte access
  float4* lv_st = reinterpret_cast<float4*>(zs + ts);
  float2* lv_r = reinterpret_cast<float2*>(lv_st + n);     // per level: {R_ii, 1 / (2 alpha R_ii)}
  uint8_t* xs = reinterpret_cast<uint8_t*>(lv_r + n);      // current path
  const float alpha = a.alpha;
  const float uoff = 0.5f * (float)(P - 1);
  int staged = -1;   // vector whose R is in shared memory
  int restart_v = -1;  // vector whose root this warp searches again (radius doubled)

  for (;;) {
    // ------------------------------------------------------------- get work
    int v = -1, top = n - 1;
    float top_ped = 0.0f;
    bool fresh = false;
    if (restart_v >= 0) {
      v = restart_v;
      restart_v = -1;
    } else {
      long long slot = -1;
      if (lane == 0) slot = queue_pop(g);
      slot = __shfl_sync(0xffffffffu, slot, 0);
      if (slot >= 0) {
        SdTask* t = g.queue + ((unsigned)slot & (g.qcap - 1));
        const unsigned long long want = (g.epoch << 32) | ((unsigned long long)slot + 1ull);
        int ok = 1;
        if (lane == 0) {
          ok = 0;
          for (int it = 0; it < (1 << 22); ++it) {
            if (*(volatile unsigned long long*)&t->seq == want) {
              ok = 1;
              break;
            }
            __nanosleep(32);
          }
          if (!ok) atomicExch(&g.sh->error, 1);
          __threadfence();
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) continue;  // a producer never published: error recorded, skip
        __threadfence();
        v = __shfl_sync(0xffffffffu, lane == 0 ? *(volatile int*)&t->v : 0, 0);
        top = __shfl_sync(0xffffffffu, lane == 0 ? *(volatile int*)&t->level : 0, 0);
        top_ped = __shfl_sync(0xffffffffu, lane == 0 ? *(volatile float*)&t->ped : 0.0f, 0);
        const bool valid = v >= 0 && v < a.batch && top >= 0 && top < n;
        if (valid)
          for (int j = top + 1 + lane; j < n; j += 32) xs[j] = ((volatile uint8_t*)t->x)[j];
        __syncwarp();
        if (lane == 0) {
          __threadfence();
          atomicExch(&t->seq, g.epoch << 32);  // copied out: the slot may be reused
        }
        if (!valid) {
          if (lane == 0) atomicExch(&g.sh->error, 2);
          continue;
        }
      } else {
        if (lane == 0) {
          v = (int)atomicAdd(&g.sh->vec_next, 1u);
          if (v < a.batch && g.order) v = g.order[v];
        }
        v = __shfl_sync(0xffffffffu, v, 0);
        if (v < a.batch) {
          fresh = true;
        } else {
          // idle: wait until a task is queued or everything is finished (a
          // search that does not split queues no task)
          int leave = may_split ? 0 : 1;
          if (lane == 0 && may_split) {
            atomicAdd(&g.sh->idle, 1);
            for (int it = 0; it < (1 << 22); ++it) {
              if (*(volatile unsigned int*)&g.sh->q_head < *(volatile unsigned int*)&g.sh->q_tail) break;
              if (*(volatile int*)&g.sh->outstanding == 0) {
                leave = 1;
                break;
              }
              __nanosleep(500);
              if (it == (1 << 22) - 1) leave = 1;
            }
            atomicSub(&g.sh->idle, 1);
          }
          leave = __shfl_sync(0xffffffffu, leave, 0);
          if (leave) break;
          continue;
        }
      }
    }
    SdVec* vs = vec_of(g, v);

    // --------------------------------------------------- stage the vector
    if (staged != v) {
      const float4* src = reinterpret_cast<const float4*>(a.R32 + (size_t)v * ts);
      for (int t = lane; t < ts / 4; t += 32) reinterpret_cast<float4*>(Rc)[t] = src[t];
      __syncwarp();
      for (int r = lane; r < n; r += 32) {
        const float rr = Rc[col_off(r) + r];
        lv_r[r] = make_float2(rr, 0.5f / (alpha * rr));
      }
      staged = v;
    }
    const float* yb = a.yb32 + (size_t)v * vec_stride32(n);

    if (fresh) {
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
      __syncwarp();
      const float E0 = error_scale_warp(n, P, alpha, Rc, yb, lane);
      float r2;
      if (a.radius_mode == RADIUS_NONE) r2 = INFINITY;
      else if (a.radius_mode == RADIUS_PAPER) r2 = (float)((double)a.n_rx * a.n_tx * a.noise_var[v]);
      else if (a.radius_mode == RADIUS_PER_VECTOR) r2 = a.r2_vec[v];
      else r2 = (float)a.radius_value;
      if (!(r2 > 0.0f)) r2 = INFINITY;
      if (lane == 0) {
        vs->r2bits = __float_as_uint(r2);
        vs->pending = 1;
        vs->lock = 0;
        vs->ncand = 0;
        vs->nodes = vs->peds = vs->flops = 0ull;
        vs->restarts = 0;
        vs->budget_hit = 0;
        vs->E = E0;
        vs->r2_start = r2;
        __threadfence();
        atomicAdd(&g.sh->outstanding, 1);
      }
      top = n - 1;
      top_ped = 0.0f;
    }
    __syncwarp();
    // values other warps may change are read by lane 0 and broadcast, so that
    // every lane of the warp takes the same decisions
    const float E = __shfl_sync(0xffffffffu, lane == 0 ? *(volatile float*)&vs->E : 0.0f, 0);

    // ------------------------------------------- residuals of the task node
    // z_r = ybar_r - sum_{j > top} R_rj x_j, r <= top, as one FMA chain from j = n-1 down
#pragma unroll
    for (int t = 0; t < ROWS; ++t) {
      const int r = lane + 32 * t;
      if (r <= top) {
        float z = yb[r];
        for (int j = n - 1; j > top; --j)
          z = fmaf(-Rc[col_off(j) + r], (float)(2 * (int)xs[j] - (P - 1)) * alpha, z);
        zs[col_off(top) + r] = z;
      }
    }
    __syncwarp();

    // -------------------------------------------------- depth-first search
    // task totals (64-bit) and the 32-bit counts since the last fold; the
    // algorithmic flops of a branched node at level l are 2 (n - 1 - l) + 4P,
    // kept as a node count and a sum of levels
    long long nodes = 0, peds = 0, flops = 0;
    int n32 = 0, p32 = 0, lsum = 0, since = 0;
    int task_nodes = 0;
    const int node_flops0 = 2 * (n - 1) + 4 * P;
#define SD_FOLD()                                            \
  do {                                                       \
    nodes += n32;                                            \
    peds += p32;                                             \
    flops += (long long)n32 * node_flops0 - 2ll * lsum;      \
    n32 = p32 = lsum = 0;                                    \
  } while (0)
    // nodes of this vector already counted by finished or committed tasks
    long long committed = 0;
    if (a.budget > 0) {
      committed = (long long)__shfl_sync(0xffffffffu, lane == 0 ? *(volatile unsigned long long*)&vs->nodes : 0ull, 0);
    }
    float r2 = __uint_as_float(
        __shfl_sync(0xffffffffu, lane == 0 ? *(volatile unsigned int*)&vs->r2bits : 0u, 0));
    float bnd = prune_bound(r2, E, n);
    bool stop = __shfl_sync(0xffffffffu, lane == 0 ? *(volatile int*)&vs->budget_hit : 0, 0) != 0;
    int i = top;
    float ped_par = top_ped;
    float c = zs[col_off(top) + top];
    const float2 rtop = lv_r[top];
    float rii = rtop.x;
    float u = fmaf(c, rtop.y, uoff);
    int lo = min(max((int)ceilf(u - 0.5f), 0), P - 1);
    int hi = lo + 1;
    // the level a pop from level i goes to: the nearest level above whose
    // next child was inside the sphere when the path left it (top + 1: none,
    // the task is done); the levels in between have no child left to try
    int ret = top + 1;
    n32 = 1;
    lsum = top;
    // Whether the level's next child in Schnorr-Euchner order (the one a
    // later iteration would take) is outside the sphere now, evaluated with
    // the same operations; the bound only shrinks, so it is outside then and
    // the level has nothing left.  The evaluation is counted here.
    auto level_done = [&]() {
      if (lo < 0 && hi >= P) return true;
      const int k2 = (hi >= P || (lo >= 0 && fabsf(u - (float)lo) <= fabsf((float)hi - u))) ? lo : hi;
      const float d2 = fmaf(-rii, (float)(2 * k2 - (P - 1)) * alpha, c);
      if (fmaf(d2, d2, ped_par) < bnd) return false;
      ++p32;
      return true;
    };
    // back to the return level (false: the task's node is exhausted)
    auto pop = [&]() {
      if (ret > top) return false;
      i = ret;
      const float4 st = lv_st[i];
      ped_par = st.x;
      c = st.y;
      u = st.z;
      rii = lv_r[i].x;
      const int lh = __float_as_int(st.w);
      lo = (lh & 0xff) - 1;
      ret = (lh >> 8) & 0xff;
      hi = lh >> 16;
      return true;
    };
    // budget left for this task's uncommitted nodes (n32 counts them)
    int left32 = 0x7fffffff;
    if (a.budget > 0) {
      const long long left = a.budget - committed;
      left32 = left < 0 ? 0 : (left > 0x7fffffffll ? 0x7fffffff : (int)left);
    }
    while (!stop) {
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
        ++p32;
      }
      if (k < 0 || !(ped < bnd)) {
        if (!pop()) break;  // the task's node is exhausted
        continue;
      }
      if (i == 0) {
        // leaf inside the sphere: record it in the vector's list, shrink the radius
        if (lane == 0) xs[0] = (uint8_t)k;
        __syncwarp();
        int slot = -1;
        if (lane == 0) {
          if (lock_acquire(&vs->lock)) {
            volatile SdVec* vv = vs;
            const int nc = vv->ncand;
            if (nc < kCand) {
              slot = nc;
              vv->ncand = nc + 1;
            } else {
              float worst = -1.0f;
              int w = -1;
              for (int q = 0; q < kCand; ++q)
                if (vv->cand_ped[q] > worst) {
                  worst = vv->cand_ped[q];
                  w = q;
                }
              if (ped < worst) slot = w;
            }
            if (slot < 0) lock_release(&vs->lock);
          } else {
            atomicExch(&g.sh->error, 1);
          }
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= 0) {
          uint8_t* dst = cand_path(vs, slot, n);
          for (int r = lane; r < n; r += 32) dst[r] = xs[r];
          __syncwarp();
          if (lane == 0) {
            vs->cand_ped[slot] = ped;
            lock_release(&vs->lock);
          }
        }
        if (lane == 0) atomicMin(&vs->r2bits, __float_as_uint(ped));
        if (ped < r2) {
          r2 = ped;
          bnd = prune_bound(r2, E, n);
        }
        if (level_done() && !pop()) break;
        continue;
      }
      if (n32 >= left32) {
        if (lane == 0) atomicExch(&vs->budget_hit, 1);
        break;
      }
      // descend into child k: push level i, update the residuals of the rows below
      const float av = (float)(2 * k - (P - 1)) * alpha;
      const float* zin = zs + col_off(i);
      const float* rc = Rc + col_off(i);
      // the next level's interference, computed by every lane from row i - 1
      // (the same FMA as that row's residual below; the column was written
      // before the last warp barrier), and the new level's first child, the
      // PAM index nearest u: outside the sphere it rules out every child, so
      // the node is counted with that one evaluation and the search goes on
      // at level i
      const float cnext = fmaf(-rc[i - 1], av, zin[i - 1]);
      const float2 rl = lv_r[i - 1];
      const float unext = fmaf(cnext, rl.y, uoff);
      const int lonext = min(max((int)ceilf(unext - 0.5f), 0), P - 1);
      const bool done_here = level_done();
      {
        const float d1 = fmaf(-rl.x, (float)(2 * lonext - (P - 1)) * alpha, cnext);
        if (!(fmaf(d1, d1, ped) < bnd)) {
          ++n32;
          ++p32;
          lsum += i - 1;
          ++task_nodes;
          if (done_here && !pop()) break;
          continue;
        }
      }
      if (lane == 0) {
        lv_st[i] = make_float4(ped_par, c, u, __int_as_float((lo + 1) | (ret << 8) | (hi << 16)));
        xs[i] = (uint8_t)k;
      }
      if (!done_here) ret = i;
      float* zout = zs + col_off(i - 1);
#pragma unroll
      for (int t = 0; t < ROWS; ++t) {
        const int r = lane + 32 * t;
        if (r < i) zout[r] = fmaf(-rc[r], av, zin[r]);
      }
      --i;
      __syncwarp();
      c = cnext;
      ped_par = ped;
      rii = rl.x;
      u = unext;
      lo = lonext;
      hi = lo + 1;
      ++n32;
      lsum += i;
      ++task_nodes;

      // periodic: radius refresh, budget, and splitting while warps are idle
      if (++since >= kSplitEvery) {
        since = 0;
        SD_FOLD();
        const float gr2 = __uint_as_float(
            __shfl_sync(0xffffffffu, lane == 0 ? *(volatile unsigned int*)&vs->r2bits : 0u, 0));
        if (gr2 < r2) {
          r2 = gr2;
          bnd = prune_bound(r2, E, n);
        }
        if (a.budget > 0) {
          unsigned long long tot = 0;
          if (lane == 0) {
            tot = atomicAdd(&vs->nodes, (unsigned long long)nodes) + (unsigned long long)nodes;
            if (tot >= (unsigned long long)a.budget) atomicExch(&vs->budget_hit, 1);
          }
          int bh = 0;
          if (lane == 0) bh = *(volatile int*)&vs->budget_hit;
          tot = __shfl_sync(0xffffffffu, tot, 0);
          bh = __shfl_sync(0xffffffffu, bh, 0);
          nodes = 0;
          committed = (long long)tot;
          if (tot >= (unsigned long long)a.budget || bh) {
            stop = true;
            break;
          }
          const long long left = a.budget - committed;
          left32 = left > 0x7fffffffll ? 0x7fffffff : (int)left;
        }
        // split only while more warps wait than tasks are queued for them
        int want = 0;
        if (may_split && task_nodes >= kSplitMinNodes && lane == 0) {
          const int idle_w = *(volatile int*)&g.sh->idle;
          const int queued = (int)(*(volatile unsigned int*)&g.sh->q_tail - *(volatile unsigned int*)&g.sh->q_head);
          want = idle_w > queued ? 1 : 0;
        }
        const int idle = __shfl_sync(0xffffffffu, want, 0);
        if (idle > 0) {
          if (lane == 0) atomicAdd(&g.sh->split_checks, 1u);
          // donate the in-sphere children of the top-most open level (at least
          // kMinSplitLevel rows deep, above the current node unless the warp is at
          // the task's root): the largest subtrees this warp would reach last.
          // Levels whose next child is outside the sphere are closed on the way
          // (their later children are farther).
          int given = 0;
          const int lmin = (i == top) ? i : i + 1;  // keep the current node unless it is the task's root
          for (int l = top; l >= lmin && l >= kMinSplitLevel && given == 0; --l) {
            int llo, lhi;
            float lc, lu, lped, lrii;
            if (l == i) {
              llo = lo;
              lhi = hi;
              lc = c;
              lu = u;
              lped = ped_par;
              lrii = rii;
            } else {
              const float4 st = lv_st[l];
              const int lh = __float_as_int(st.w);
              llo = (lh & 0xff) - 1;
              lhi = lh >> 16;
              lc = st.y;
              lu = st.z;
              lped = st.x;
              lrii = lv_r[l].x;
            }
            if (llo < 0 && lhi >= P) continue;
            // children inside the sphere, in SE order: counted first, then written
            int cnt = 0;
            {
              int a_lo = llo, a_hi = lhi;
              while (a_lo >= 0 || a_hi < P) {
                int kk;
                if (a_hi >= P || (a_lo >= 0 && fabsf(lu - (float)a_lo) <= fabsf((float)a_hi - lu))) kk = a_lo--;
                else kk = a_hi++;
                const float d = fmaf(-lrii, (float)(2 * kk - (P - 1)) * alpha, lc);
                if (!(fmaf(d, d, lped) < bnd)) break;
                ++cnt;
              }
            }
            long long base_slot = -1;
            if (cnt > 0 && lane == 0) {
              atomicAdd(&vs->pending, cnt);
              atomicAdd(&g.sh->outstanding, cnt);
              base_slot = queue_reserve(g, cnt);
              if (base_slot < 0) {
                atomicSub(&vs->pending, cnt);
                atomicSub(&g.sh->outstanding, cnt);
              } else {
                atomicAdd(&g.sh->donated, (unsigned)cnt);
              }
            }
            base_slot = __shfl_sync(0xffffffffu, base_slot, 0);
            if (cnt > 0 && base_slot < 0) break;  // queue full: keep the rest
            for (int q = 0; q < cnt; ++q) {
              int kk;
              if (lhi >= P || (llo >= 0 && fabsf(lu - (float)llo) <= fabsf((float)lhi - lu))) kk = llo--;
              else kk = lhi++;
              const float d = fmaf(-lrii, (float)(2 * kk - (P - 1)) * alpha, lc);
              const float pd = fmaf(d, d, lped);
              const unsigned long long sl = (unsigned long long)base_slot + q;
              SdTask* t = g.queue + ((unsigned)sl & (g.qcap - 1));
              int wok = 1;
              if (lane == 0) {
                wok = slot_writable(g, t, sl);
                if (!wok) {
                  // error recorded; the task is dropped (this task still holds the
                  // vector open, so its pending count cannot reach zero here)
                  atomicExch(&g.sh->error, 3);
                  atomicSub(&vs->pending, 1);
                  atomicSub(&g.sh->outstanding, 1);
                }
              }
              wok = __shfl_sync(0xffffffffu, wok, 0);
              if (!wok) continue;
              for (int j = l + 1 + lane; j < n; j += 32) t->x[j] = xs[j];
              if (lane == 0) {
                t->x[l] = (uint8_t)kk;
                t->v = v;
                t->level = l - 1;
                t->ped = pd;
              }
              __threadfence();
              __syncwarp();
              if (lane == 0) atomicExch(&t->seq, (g.epoch << 32) | (sl + 1ull));
            }
            given += cnt;
            // the donated (or out-of-sphere) children are gone from this warp's search
            if (l == i) {
              lo = -1;
              hi = P;
            } else if (lane == 0) {
              int* w = reinterpret_cast<int*>(&lv_st[l]) + 3;
              *w = (*w & 0xff00) | (P << 16);  // no child left; the return level stays
            }
            __syncwarp();
          }
          if (lane == 0) {
            if (given > 0) atomicAdd(&g.sh->splits, 1u);
            else atomicAdd(&g.sh->no_level, 1u);
          }
        }
      }
    }

    // ------------------------------------------------ task done: account
    SD_FOLD();
    if (lane == 0) {
      atomicAdd(&vs->nodes, (unsigned long long)nodes);
      atomicAdd(&vs->peds, (unsigned long long)peds);
      atomicAdd(&vs->flops, (unsigned long long)flops);
      __threadfence();
    }
    int last = 0;
    if (lane == 0) last = (atomicSub(&vs->pending, 1) == 1);
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
      __threadfence();
      volatile SdVec* vv = vs;
      const int nc = __shfl_sync(0xffffffffu, lane == 0 ? vv->ncand : 0, 0);
      const bool bh = __shfl_sync(0xffffffffu, lane == 0 ? vv->budget_hit : 0, 0) != 0;
      const float r2s = __shfl_sync(0xffffffffu, lane == 0 ? vv->r2_start : 0.0f, 0);
      const int rs = __shfl_sync(0xffffffffu, lane == 0 ? vv->restarts : 0, 0);
      if (nc == 0 && !bh && r2s < INFINITY && rs < 64) {
        // empty sphere: double the radius (r^2 <- 2 r^2) and search the root
        // again; this warp takes the new root itself (outstanding stays: the
        // new root replaces this task)
        if (lane == 0) {
          const float nr2 = 2.0f * r2s;
          vs->r2_start = nr2;
          vs->r2bits = __float_as_uint(nr2);
          vs->restarts += 1;
          vs->pending = 1;
          __threadfence();
        }
        __syncwarp();
        restart_v = v;
        continue;
      }
      // FP64 re-scoring of the candidates within FP32 error of the best
      float best = INFINITY;
      for (int q = 0; q < nc; ++q) best = fminf(best, vv->cand_ped[q]);
      const float keep = prune_bound(best, E, n);
      const double* R64 = a.R64 + (size_t)v * tri_stride64(n);
      const double* y64 = a.yb64 + (size_t)v * vec_stride64(n);
      // candidates are read through L2 (other warps wrote them) into this
      // warp's path buffer; the winner's indices are kept in registers
      int win = -1;
      double win_m = INFINITY;
      long long rescored = 0;
      uint8_t wsym[(MDX_MAX_TX + 31) / 32 * 2];
      for (int q = 0; q < nc; ++q) {
        if (!(vv->cand_ped[q] <= keep)) continue;
        const uint8_t* cx = cand_path(vs, q, n);
        __syncwarp();
        for (int r = lane; r < n; r += 32) xs[r] = __ldcg(cx + r);
        __syncwarp();
        double m;
        if (a.flags & MDX_NO_RESCORE) {
          m = (double)vv->cand_ped[q];
        } else {
          m = rescore_fp64_warp(n, P, a.alpha64, R64, y64, xs, lane);
          ++rescored;
        }
        bool better = m < win_m;
        if (!better && m == win_m && win >= 0) {
          // tie: lexicographically smaller index vector, top row first
          const uint8_t* wx = cand_path(vs, win, n);
          for (int j = n - 1; j >= 0; --j) {
            const uint8_t w1 = xs[j], w2 = __ldcg(wx + j);
            if (w1 != w2) {
              better = w1 < w2;
              break;
            }
          }
        }
        if (better) {
          win = q;
          win_m = m;
#pragma unroll
          for (int t = 0; t < (MDX_MAX_TX + 31) / 32; ++t) {
            const int j = lane + 32 * t;
            if (j < a.n_tx) {
              wsym[2 * t] = xs[2 * j];
              wsym[2 * t + 1] = xs[2 * j + 1];
            }
          }
        }
      }
#pragma unroll
      for (int t = 0; t < (MDX_MAX_TX + 31) / 32; ++t) {
        const int j = lane + 32 * t;
        if (j < a.n_tx)
          a.sym_out[(size_t)v * a.n_tx + j] = win >= 0 ? (uint8_t)(wsym[2 * t] * P + wsym[2 * t + 1]) : 0;
      }
      if (lane == 0) {
        a.metric_out[v] = (win >= 0) ? win_m : (double)INFINITY;
        a.vstatus[v] = bh ? MDX_V_BUDGET_EXCEEDED : (vv->restarts > 0 ? MDX_V_EMPTY_RETRIED : MDX_V_OK);
        if (a.stats) {
          a.stats[(size_t)v * kStats + 0] = (long long)vv->nodes;
          a.stats[(size_t)v * kStats + 1] = (long long)vv->peds;
          a.stats[(size_t)v * kStats + 2] = vv->restarts;
          a.stats[(size_t)v * kStats + 3] = rescored;
          a.stats[(size_t)v * kStats + 4] = (long long)vv->flops;
        }
      }
    }
    __syncwarp();
    if (lane == 0) atomicSub(&g.sh->outstanding, 1);
  }
}

#undef SD_FOLD

// Fresh vectors are taken heaviest first (longest-processing-time order),
// so that the searches that take longest start early and their subtrees can
// be split while the light vectors still keep every worker busy.  The cost
// proxy is the noise variance (the search grows steeply as the SNR falls),
// bucketed at a quarter octave: a counting sort by histogram, exclusive scan
// and scatter.  The order inside a bucket is arbitrary; answers do not depend
// on it.
constexpr int kOrderBuckets = 1024;

__device__ __forceinline__ int order_bucket(double nv) {
  // -log2(sigma^2) * 4, offset: ascending buckets = descending noise variance
  const float b = floorf(-log2f((float)nv) * 4.0f) + (float)(kOrderBuckets / 2);
  return (int)fminf(fmaxf(b, 0.0f), (float)(kOrderBuckets - 1));
}

__global__ void sd_order_hist(int batch, const double* __restrict__ nv, unsigned int* cnt) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < batch) atomicAdd(&cnt[order_bucket(nv[v])], 1u);
}

// exclusive scan of the kOrderBuckets counts into cnt[kOrderBuckets + b]
__global__ void __launch_bounds__(kOrderBuckets) sd_order_scan(unsigned int* cnt) {
  __shared__ unsigned int s[kOrderBuckets];
  const int t = threadIdx.x;
  const unsigned int mine = cnt[t];
  s[t] = mine;
  __syncthreads();
  for (int o = 1; o < kOrderBuckets; o <<= 1) {
    const unsigned int add = t >= o ? s[t - o] : 0u;
    __syncthreads();
    s[t] += add;
    __syncthreads();
  }
  cnt[kOrderBuckets + t] = s[t] - mine;
}

__global__ void sd_order_scatter(int batch, const double* __restrict__ nv, unsigned int* cnt, int* order) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < batch) order[atomicAdd(&cnt[kOrderBuckets + order_bucket(nv[v])], 1u)] = v;
}

template <int ROWS>
cudaError_t launch_rows(const SdArgs& g, int num_sms, cudaStream_t s) {
  // as many warps per CTA (up to kWarpsMax) as fit in 200 KB of shared memory
  int wpc = (int)((200u * 1024u) / sd_warp_bytes(g.a.n));
  if (wpc > kWarpsMax) wpc = kWarpsMax;
  if (wpc < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = sd_warp_bytes(g.a.n) * wpc;
  cudaError_t e = cudaFuncSetAttribute(sd_kernel<ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sd_kernel<ROWS>, wpc * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // a persistent grid: every warp stays until the queue and the vectors are done
  const int grid = per_sm * num_sms;
  sd_kernel<ROWS><<<grid, wpc * 32, smem, s>>>(g);
  return cudaGetLastError();
}

}  // namespace

size_t sd_vec_state_bytes(int n) { return vec_state_bytes(n); }
size_t sd_order_ints(int max_batch) { return (size_t)max_batch + 2 * kOrderBuckets; }
size_t sd_task_bytes() { return sizeof(SdTask); }
size_t sd_shared_bytes() { return sizeof(SdShared); }
size_t sd_error_offset() { return offsetof(SdShared, error); }
size_t sd_counters_offset() { return offsetof(SdShared, split_checks); }

cudaError_t launch_sd(const SearchArgs& a, const SdWorkspace& w, int num_sms, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  if (a.n > kTaskPath) return cudaErrorInvalidConfiguration;
  SdArgs g;
  g.a = a;
  g.sh = reinterpret_cast<SdShared*>(w.shared);
  g.queue = reinterpret_cast<SdTask*>(w.queue);
  g.qcap = w.qcap;
  g.vstate = w.vstate;
  g.vstride = vec_state_bytes(a.n);
  g.epoch = w.epoch;
  g.order = nullptr;
  cudaError_t e = cudaMemsetAsync(w.shared, 0, sizeof(SdShared), s);
  if (e != cudaSuccess) return e;
  if (a.noise_var && w.order && a.batch > 1) {
    int* order = w.order;
    unsigned int* cnt = reinterpret_cast<unsigned int*>(order + a.batch);
    e = cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * kOrderBuckets, s);
    if (e != cudaSuccess) return e;
    const int blocks = (a.batch + 255) / 256;
    sd_order_hist<<<blocks, 256, 0, s>>>(a.batch, a.noise_var, cnt);
    sd_order_scan<<<1, kOrderBuckets, 0, s>>>(cnt);
    sd_order_scatter<<<blocks, 256, 0, s>>>(a.batch, a.noise_var, cnt, order);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    g.order = order;
  }
  if (a.n <= 32) return launch_sd_group(g, num_sms, s);
  if (a.n <= 64) return launch_rows<2>(g, num_sms, s);
  if (a.n <= 128) return launch_rows<4>(g, num_sms, s);
  return launch_rows<7>(g, num_sms, s);
}

}  // namespace mdx
