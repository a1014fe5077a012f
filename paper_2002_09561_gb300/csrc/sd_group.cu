// Exact sphere decoder for n <= 32 real rows with several received vectors
// per warp: the same search as sd.cu (Algorithm 1 with the Best-FS /
// Schnorr-Euchner child order of Sec. IV-A, incremental partial distances of
// Eq. inc, subtree splitting between workers as the paper's dynamic load
// balancing, Sec. V-C), with a group of G lanes as the worker instead of a
// warp.
//
// Why.  One node step is a short dependent chain of control work (choose the
// next child in zig-zag order, its partial distance, the pruning test, push
// or pop a level) plus one FMA per row below the node.  With a warp per
// vector every lane repeats the control work, about 150 warp instructions per
// node for 32 useful FMAs.  With a group of G = 8 lanes per vector (rows
// r = g + 8 t of lane g) one warp advances four trees with every instruction.
//
// The node step.  Each pass evaluates one child of every busy group's current
// level and then pops, descends or reports a leaf, without branches: the
// shared-memory operands of both outcomes (the R column and residuals of a
// descent, the saved state of the level a pop returns to) are loaded first,
// independently of the child chosen, so their latency overlaps the choice.  A
// child inside the sphere is a visited node; the pass also evaluates that
// node's first child (the PAM index nearest u), and when it lies outside the
// sphere, so do all the others and the group does not descend.  It evaluates
// the child's next sibling as well: outside the sphere (the bound only
// shrinks, so it stays outside), no pass returns to the level, and a pop
// jumps over every such level to the nearest one with a sibling left inside
// (each level keeps that return level).  Almost every pass then visits a
// node: a failing evaluation no longer costs a pass of its own, nor does the
// climb back through levels with nothing left.  The new level's
// interference c_{i-1} = z_{i-1} - R_{i-1,i} a_i comes from row i - 1 of the
// R and residual columns, which every lane of the group loads (after a warp
// barrier: only the row's owner wrote the residual), not from a shuffle at
// the end of the residual update.  The zig-zag cursors and the current path
// are kept as floats, so choosing a child, forming its PAM level and
// recording it need no conversions.  Passes run kPassesPerVote at a time,
// from one copy of the node step in a loop (an unrolled copy per pass
// overflows the instruction cache); between them one warp vote decides the
// rare events (a leaf, the end of a task, work to fetch, the periodic check),
// and a group whose pass raised one sits out the rest of the passes until
// then.
//
// Shared memory.  Per group (one vector's task at a time): the vector's FP32
// R and the residual stack z, both with the columns in descending order
// (zoff: rows a lane writes past a column's end land in deeper columns), the
// per-level state {parent partial distance, c_i, zig-zag cursors},
// {R_ii, 1 / (2 alpha R_ii)}, the current path, and up to kCand leaf
// candidates of the running task.  The four groups of a warp are
// interleaved element by element (WarpLayout), so their lanes always touch
// disjoint banks, whichever levels their trees are at.  Every value a lane
// reads from its group's state it either wrote itself (all lanes of a group
// write the same level state and path entries) or reads after a warp
// barrier; residual rows are lane-owned.
//
// Each residual is the same FP32 FMA chain in the same order as in sd.cu
// (z_r = ybar_r - sum_{j > i} R_rj x_j, j from n-1 down), and each PAM level
// the same product (2k - (P-1)) alpha, so every partial distance, pruning
// decision and visited-node count of a sequential search equals the warp
// kernel's (a node not entered because its first child is outside the
// sphere is counted, as is that child's evaluation, and so is the failing
// evaluation of a sibling that ends its level).
//
// Work.  A task is a tree node of one vector (rows above it fixed), with the
// queue records and per-vector state of sd.cu.  Fresh vectors come first, in
// the launch's heaviest-first order.  A vector that never split is "solo":
// its group keeps the radius and the leaf candidates to itself and re-scores
// them in FP64 when the search ends, without touching the shared per-vector
// record.  Once the fresh vectors are gone, a group that needs work takes a
// ticket of the task queue (one atomicAdd on the head, no compare-and-swap
// retries: with thousands of waiting groups a CAS-claimed queue served well
// under a million tasks per second and left most groups idle for the last
// half of a heavy-tailed batch) and waits until that slot is published.
// While tickets outnumber the tasks reserved, a busy group that has searched
// kSplitMinNodes nodes of its task donates the in-sphere children of its
// top-most open level (at least kMinSplitLevel rows above the leaves); from
// then on the vector's radius is shared through atomicMin on its FP32 bits,
// its tasks merge their candidates into the vector's list under its lock,
// and the task that finishes last re-scores that list.  A search with a
// node budget does not split (the budget is an exact cap per vector).  An
// empty sphere doubles the radius (r^2 <- 2 r^2) and searches the root again.
//
// Waiting.  A group with a ticket looks at its slot every 16 passes while
// its warp has busy groups; a warp whose groups all wait polls the slots
// until one is published or no task is queued or running (a vector is
// counted as running before it is taken, so nothing can be handed to a group
// that has left).  Every spin-wait is bounded: the idle wait gives up only
// after about 2^22 polls in which no task ended or was donated anywhere, and
// like the other waits it reports through the launch's error word.
#include "sd_common.cuh"

namespace mdx {
namespace {

constexpr int kGroupN = 32;     // largest n of this kernel
// Lanes per vector.  Eight (four vectors per warp, rows g, g + 8, g + 16,
// g + 24 of lane g) measured faster than four on the 16x16 16-QAM batches
// (four lanes: fewer instructions per node, but half the warps per SM for
// the same trees, which exposes each pass's dependent chain).
#ifndef MDX_SDG_LANES
#define MDX_SDG_LANES 8
#endif
constexpr int kGroupLanes = MDX_SDG_LANES;
// warps per CTA: as many as let five CTAs share an SM's 228 KB
template <int G>
__host__ __device__ constexpr int group_warps() {
  return G >= 8 ? 2 : 1;
}
constexpr int kTri = 528;       // column-packed triangle of n = 32
// node-step passes per vote of the slow paths (divides 16 and kSplitEvery);
// a group that raised an event sits out the rest of them
#ifndef MDX_SDG_PASSES
#define MDX_SDG_PASSES 16
#endif
constexpr int kPassesPerVote = MDX_SDG_PASSES;
// copies of the node step in the pass loop: one.  The loop body must stay
// small enough for the instruction cache; on the 16x16 16-QAM sweep one copy
// searched in 40.5 ms, two in 43.4 ms, four in 52.7 ms (four passes per vote)
#ifndef MDX_SDG_UNROLL
#define MDX_SDG_UNROLL 1
#endif
constexpr int kPassUnroll = MDX_SDG_UNROLL;
static_assert(kPassesPerVote <= 16 && 16 % kPassesPerVote == 0, "the ticket check cadence");
static_assert(kSplitEvery % kPassesPerVote == 0, "the split check cadence");

// R and the residual stack in shared memory: column c (rows 0..c) starts at
// zoff(c) = kTri - (c + 1)(c + 2) / 2, the columns in descending order.  A
// lane may then write a whole column, rows past its end included: those land
// in deeper columns (or the padding after column 0), which are rewritten
// before they are read, so the node step stores every row without a test.
__host__ __device__ constexpr int zoff(int c) { return kTri - (((c + 1) * (c + 2)) >> 1); }

// Shared memory of one warp, in 4-byte words.  The NG = 32 / G groups of the
// warp are interleaved element by element (element e of group g at e NG + g),
// so that the G lanes of every group read consecutive elements at a stride of
// NG words: the groups of a warp always touch disjoint banks, whichever level
// each of their trees is at.
//   R       kTri x NG floats          FP32 R, columns at zoff(c)
//   Z       (kTri + 32) x NG floats   residual stack (level i: rows 0..i at zoff(i)), padded
//                                     for the rows written past column 0
//   ST      32 x NG float4     level state {parent partial distance, c_i, cursor lo, cursor hi}
//                              (u_i = c_i / (2 alpha R_ii) + (P - 1) / 2 and R_ii come from LR)
//   LR      32 x NG float2     {R_ii, 1 / (2 alpha R_ii)}
//   XS      32 x NG floats     current path (PAM indices as floats: no conversion on a descent)
//   RT      32 x NG bytes      return level of each level on the path (where a pop from it goes)
//   per group: kCand candidate partial distances and kCand x 32 path bytes
template <int G>
struct WarpLayout {
  static constexpr int NG = 32 / G;
  static constexpr int R = 0;
  static constexpr int Z = R + kTri * NG;
  static constexpr int ST = Z + (kTri + kGroupN) * NG;
  static constexpr int LR = ST + 4 * kGroupN * NG;
  static constexpr int XS = LR + 2 * kGroupN * NG;
  static constexpr int RT = XS + kGroupN * NG;
  static constexpr int CAND = RT + kGroupN * NG / 4;
  static constexpr int CAND_WORDS = kCand + kCand * kGroupN / 4;  // per group
  static constexpr int WORDS = CAND + NG * CAND_WORDS;
  static_assert(ST % 4 == 0 && LR % 2 == 0, "16- and 8-byte alignment of the level arrays");
};

template <int G>
__host__ __device__ constexpr size_t group_cta_bytes() {
  return (size_t)group_warps<G>() * WarpLayout<G>::WORDS * 4 + 8 * sizeof(double);
}

// FP64 ||ybar - R x||^2 of path x (n <= 32) by the G lanes of a group: lane
// g accumulates rows g, g + G, ...; the PAM levels come from a table.
template <int G>
__device__ __forceinline__ double rescore_fp64_group(int n, const double* lev64, const double* __restrict__ R64,
                                                     const double* __restrict__ y64, const uint8_t* x, bool x_global,
                                                     int gl, unsigned gmask) {
  constexpr int RPL = kGroupN / G;
  double rr[RPL];
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int r = gl + G * t;
    rr[t] = (r < n) ? y64[r] : 0.0;
  }
  for (int j = 0; j < n; ++j) {
    const int k = x_global ? (int)__ldcg(x + j) : (int)x[j];
    const double xj = lev64[k];
    const double* col = R64 + col_off(j);
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int r = gl + G * t;
      if (r <= j) rr[t] = fma(-col[r], xj, rr[t]);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < RPL; ++t) s = fma(rr[t], rr[t], s);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, G);
  return s;
}

#ifndef MDX_SDG_MIN_BLOCKS
#define MDX_SDG_MIN_BLOCKS 5
#endif

// kBudget: the launch has a node budget (tested on every descent; without one
// the node step carries no budget test)
template <int G, bool kBudget>
__global__ void __launch_bounds__(group_warps<G>() * 32, MDX_SDG_MIN_BLOCKS) sd_group_kernel(SdArgs g) {
  constexpr int NG = 32 / G;        // groups per warp
  constexpr int RPL = kGroupN / G;  // rows per lane
  extern __shared__ __align__(16) unsigned char smem[];
  const SearchArgs& a = g.a;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane / G, gl = lane % G, lead = gid * G;
  const unsigned gmask = ((1u << G) - 1u) << lead;
  const unsigned full = 0xffffffffu;
  const int n = a.n, P = a.P;
  const float Pf = (float)P;
  // A vector's tree is split between groups unless the search is sequential
  // or has a node budget: the budget is a cap per vector, which tasks running
  // at once could only check between passes (and it bounds the work of a
  // vector anyway)
  const bool may_split = !(a.flags & MDX_SEQUENTIAL_SEARCH) && !kBudget;
  const int ts = tri_stride32(n);
  const float alpha = a.alpha;
  const float uoff = 0.5f * (float)(P - 1);

  double* lev64 = reinterpret_cast<double*>(smem + group_cta_bytes<G>() - 8 * sizeof(double));
  if (threadIdx.x < 8) lev64[threadIdx.x] = (double)(2 * (int)threadIdx.x - (P - 1)) * a.alpha64;
  __syncthreads();

  using L = WarpLayout<G>;
  float* wbase = reinterpret_cast<float*>(smem) + (size_t)warp * L::WORDS;
  float* Rw = wbase + L::R;
  float* Zw = wbase + L::Z;
  float4* STw = reinterpret_cast<float4*>(wbase + L::ST);
  float2* LRw = reinterpret_cast<float2*>(wbase + L::LR);
  float* XSw = wbase + L::XS;
  uint8_t* RTw = reinterpret_cast<uint8_t*>(wbase + L::RT);
  float* cped = wbase + L::CAND + gid * L::CAND_WORDS;
  uint8_t* cx = reinterpret_cast<uint8_t*>(cped + kCand);
#define RW(e) Rw[(e) * NG + gid]
#define ZW(e) Zw[(e) * NG + gid]
#define ST(l) STw[(l) * NG + gid]
#define LR(l) LRw[(l) * NG + gid]
#define XS(j) XSw[(j) * NG + gid]
#define RT(l) RTw[(l) * NG + gid]

  // ---- per-group state (identical in the group's lanes)
  int mode = 0;     // 0: needs work, 1: busy, 2: idle (holding a queue ticket, or done)
  long long ticket = -1;  // the group leader's unanswered ticket of the task queue
  int staged = -1;  // vector whose R is in this group's shared memory
  int v = -1, top = n - 1, i = n - 1;
  int ci = zoff(n - 1);  // zoff(i), kept with i
  // the level a pop from level i goes to: the nearest level above i whose
  // next child was inside the sphere when the path left it (top + 1: none,
  // the task ends); levels in between have no child left to try
  int rt = n;
  // the level's state: parent partial distance, interference c_i, u_i (the
  // real-valued PAM index of c_i / R_ii), R_ii, and the zig-zag cursors (the
  // next lower / higher PAM index, as floats; lo < 0 or hi >= P: exhausted)
  float ped_par = 0.0f, c = 0.0f, u = 0.0f, rii = 1.0f, flo = 0.0f, fhi = 0.0f;
  float r2 = INFINITY, bnd = INFINITY, E = 0.0f;
  bool solo = false;
  int ncl = 0;  // leaf candidates of the running task
  long long nodes = 0, peds = 0, flops = 0, committed = 0;
  int n32 = 0, p32 = 0, lsum = 0, left32 = 0x7fffffff;
  int task_nodes = 0;  // nodes of the running task up to the last periodic check
  int restarts = 0;           // radius doublings so far (solo)
  float r2_start = INFINITY;  // radius of the current pass (solo)
  bool budget_hit = false;
  const int node_flops0 = 2 * (n - 1) + 4 * P;
  int since = 0;
  bool recheck = true;  // idle groups try the queue again
  bool ev_leaf = false, ev_done = false;
  float leaf_ped = 0.0f;
  float leaf_kf = 0.0f;

  // the level a group enters (task node, root restart): cursors from u
  auto enter_level = [&](int lvl, float pp) {
    i = lvl;
    ci = zoff(lvl);
    rt = lvl + 1;
    ped_par = pp;
    c = ZW(zoff(lvl) + lvl);
    const float2 rl = LR(lvl);
    rii = rl.x;
    u = fmaf(c, rl.y, uoff);
    flo = fminf(fmaxf(ceilf(u - 0.5f), 0.0f), Pf - 1.0f);
    fhi = flo + 1.0f;
  };

  for (;;) {
    // ==================================================== events and work
    const bool want = (mode == 0) || (mode == 2 && (recheck || (since & 15) == 16 - kPassesPerVote));
    // one vote per pass decides whether anything but the node step runs:
    // events of the last pass, groups that want work, the periodic check
    if (__any_sync(full, ev_leaf || ev_done || want || since >= kSplitEvery)) {
      // ---------------------------------------------------- periodic check
      if (since >= kSplitEvery) {
        since = 0;
        recheck = true;
        const bool busy = mode == 1 && !ev_done;
        SdVec* vs = busy ? vec_of(g, v) : nullptr;
        if (busy) {
          task_nodes += n32;
          nodes += n32;
          peds += p32;
          flops += (long long)n32 * node_flops0 - 2ll * lsum;
          n32 = p32 = lsum = 0;
          if (!solo) {
            unsigned int rb = 0;
            if (gl == 0) rb = *(volatile unsigned int*)&vs->r2bits;
            const float gr2 = __uint_as_float(__shfl_sync(gmask, rb, lead));
            if (gr2 < r2) {
              r2 = gr2;
              bnd = prune_bound(r2, E, n);
            }
          }
          if (kBudget) {
            unsigned long long tot = 0;
            int bh = 0;
            if (gl == 0) {
              tot = atomicAdd(&vs->nodes, (unsigned long long)nodes) + (unsigned long long)nodes;
              atomicAdd(&vs->peds, (unsigned long long)peds);
              atomicAdd(&vs->flops, (unsigned long long)flops);
              if (tot >= (unsigned long long)a.budget) atomicExch(&vs->budget_hit, 1);
              bh = *(volatile int*)&vs->budget_hit;
            }
            tot = __shfl_sync(gmask, tot, lead);
            bh = __shfl_sync(gmask, bh, lead);
            nodes = peds = flops = 0;  // committed to vs
            committed = (long long)tot;
            if (tot >= (unsigned long long)a.budget || bh) {
              budget_hit = true;
              left32 = 0;
            } else {
              const long long left = a.budget - committed;
              left32 = left > 0x7fffffffll ? 0x7fffffff : (int)left;
            }
          }
        }
        // donation while more groups wait than tasks are queued for them
        int wantd = 0;
        if (busy && may_split && task_nodes >= kSplitMinNodes && gl == 0) {
          // tickets taken beyond the tasks reserved so far: groups waiting for work
          const int waiting = (int)(*(volatile unsigned int*)&g.sh->q_head - *(volatile unsigned int*)&g.sh->q_tail);
          wantd = waiting > 0 ? 1 : 0;
        }
        wantd = __shfl_sync(full, wantd, lead);
        if (__any_sync(full, wantd)) {
          if (wantd) {
            if (gl == 0) atomicAdd(&g.sh->split_checks, 1u);
            if (solo) {
              // the vector's state becomes shared: publish the radius first
              if (gl == 0) {
                atomicMin(&vs->r2bits, __float_as_uint(r2));
                __threadfence();
              }
              solo = false;
            }
            int given = 0;
            // the top-most open level (the current node's own level only at the task's root)
            const int lmin = (i == top) ? i : i + 1;
            for (int l = top; l >= lmin && l >= kMinSplitLevel && given == 0; --l) {
              float llo, lhi, lc, lu, lped, lrii;
              if (l == i) {
                llo = flo;
                lhi = fhi;
                lc = c;
                lu = u;
                lped = ped_par;
                lrii = rii;
              } else {
                const float4 st = ST(l);
                const float2 lr = LR(l);
                llo = st.z;
                lhi = st.w;
                lped = st.x;
                lc = st.y;
                lu = fmaf(lc, lr.y, uoff);
                lrii = lr.x;
              }
              if (llo < 0.0f && lhi >= Pf) continue;
              // children inside the sphere, in Schnorr-Euchner order: counted first, then written
              int cnt = 0;
              {
                float a_lo = llo, a_hi = lhi;
                while (a_lo >= 0.0f || a_hi < Pf) {
                  float kk;
                  if (a_hi >= Pf || (a_lo >= 0.0f && fabsf(lu - a_lo) <= fabsf(a_hi - lu))) {
                    kk = a_lo;
                    a_lo -= 1.0f;
                  } else {
                    kk = a_hi;
                    a_hi += 1.0f;
                  }
                  const float d = fmaf(-lrii, fmaf(kk, 2.0f, -(Pf - 1.0f)) * alpha, lc);
                  if (!(fmaf(d, d, lped) < bnd)) break;
                  ++cnt;
                }
              }
              long long base_slot = -1;
              if (cnt > 0 && gl == 0) {
                atomicAdd(&vs->pending, cnt);
                atomicAdd(&g.sh->outstanding, cnt);
                // tickets may run ahead of the tail, so slots are reserved by
                // atomicAdd; a slot is rewritten only after its previous task was
                // copied out (slot_writable)
                base_slot = (long long)atomicAdd(&g.sh->q_tail, (unsigned)cnt);
                atomicAdd(&g.sh->donated, (unsigned)cnt);
                atomicAdd(&g.sh->progress, 1u);
              }
              base_slot = __shfl_sync(gmask, base_slot, lead);
              if (cnt > 0 && base_slot < 0) break;  // queue full: keep the rest
              for (int q = 0; q < cnt; ++q) {
                float kk;
                if (lhi >= Pf || (llo >= 0.0f && fabsf(lu - llo) <= fabsf(lhi - lu))) {
                  kk = llo;
                  llo -= 1.0f;
                } else {
                  kk = lhi;
                  lhi += 1.0f;
                }
                const float d = fmaf(-lrii, fmaf(kk, 2.0f, -(Pf - 1.0f)) * alpha, lc);
                const float pd = fmaf(d, d, lped);
                const unsigned long long sl = (unsigned long long)base_slot + q;
                SdTask* t = g.queue + ((unsigned)sl & (g.qcap - 1));
                int wok = 1;
                if (gl == 0) {
                  wok = slot_writable(g, t, sl);
                  if (!wok) {
                    atomicExch(&g.sh->error, 3);
                    atomicSub(&vs->pending, 1);
                    atomicSub(&g.sh->outstanding, 1);
                  }
                }
                wok = __shfl_sync(gmask, wok, lead);
                if (!wok) continue;
                for (int j = l + 1 + gl; j < n; j += G) t->x[j] = (uint8_t)(int)XS(j);
                if (gl == 0) {
                  t->x[l] = (uint8_t)(int)kk;
                  t->v = v;
                  t->level = l - 1;
                  t->ped = pd;
                }
                __threadfence();
                __syncwarp(gmask);
                if (gl == 0) atomicExch(&t->seq, (g.epoch << 32) | (sl + 1ull));
              }
              given += cnt;
              // the donated (or out-of-sphere) children are gone from this group's search
              if (l == i) {
                flo = -1.0f;
                fhi = Pf;
              } else {
                ST(l).z = -1.0f;
                ST(l).w = Pf;
              }
            }
            if (gl == 0) {
              if (given > 0) atomicAdd(&g.sh->splits, 1u);
              else atomicAdd(&g.sh->no_level, 1u);
            }
          }
          __syncwarp();
        }
      }

      // --------------------------------------------------------- a leaf
      if (__any_sync(full, ev_leaf)) {
        if (ev_leaf) {
          XS(0) = leaf_kf;
          int slot = -1;
          if (ncl < kCand) {
            slot = ncl++;
          } else {
            float worst = -1.0f;
            int w = -1;
            for (int q = 0; q < kCand; ++q)
              if (cped[q] > worst) {
                worst = cped[q];
                w = q;
              }
            if (leaf_ped < worst) slot = w;
          }
          if (slot >= 0) {
            uint8_t* dst = cx + slot * kGroupN;
            for (int j = gl; j < n; j += G) dst[j] = (uint8_t)(int)XS(j);
            cped[slot] = leaf_ped;
          }
          if (!solo && gl == 0) atomicMin(&vec_of(g, v)->r2bits, __float_as_uint(leaf_ped));
          if (leaf_ped < r2) {
            r2 = leaf_ped;
            bnd = prune_bound(r2, E, n);
          }
        }
        __syncwarp();
        ev_leaf = false;
      }

      // --------------------------------------------------- a task ended
      if (__any_sync(full, ev_done)) {
        bool rescore = false, restart = false, use_global = false;
        int nc = 0;
        if (ev_done) {
          nodes += n32;
          peds += p32;
          flops += (long long)n32 * node_flops0 - 2ll * lsum;
          n32 = p32 = lsum = 0;
          SdVec* vs = vec_of(g, v);
          if (solo) {
            if (ncl == 0 && !budget_hit && r2_start < INFINITY && restarts < 64) {
              // empty sphere: r^2 <- 2 r^2 and the root again
              restart = true;
              r2_start *= 2.0f;
              ++restarts;
              if (gl == 0) {
                vs->r2_start = r2_start;
                vs->r2bits = __float_as_uint(r2_start);
                vs->restarts = restarts;
              }
              r2 = r2_start;
            } else {
              rescore = true;
              nc = ncl;
            }
          } else {
            // merge this task's candidates into the vector's list, then account
            int last = 0, gnc = 0, rs = 0, bh = 0;
            float r2s = 0.0f;
            if (gl == 0) {
              if (ncl > 0) {
                if (lock_acquire(&vs->lock)) {
                  volatile SdVec* vv = vs;
                  for (int q = 0; q < ncl; ++q) {
                    int sl = -1;
                    const int cur = vv->ncand;
                    if (cur < kCand) {
                      sl = cur;
                      vv->ncand = cur + 1;
                    } else {
                      float worst = -1.0f;
                      for (int w = 0; w < kCand; ++w)
                        if (vv->cand_ped[w] > worst) {
                          worst = vv->cand_ped[w];
                          sl = w;
                        }
                      if (!(cped[q] < worst)) sl = -1;
                    }
                    if (sl >= 0) {
                      uint8_t* dst = cand_path(vs, sl, n);
                      for (int j = 0; j < n; ++j) dst[j] = cx[q * kGroupN + j];
                      vv->cand_ped[sl] = cped[q];
                    }
                  }
                  lock_release(&vs->lock);
                } else {
                  atomicExch(&g.sh->error, 1);
                }
              }
              atomicAdd(&vs->nodes, (unsigned long long)nodes);
              atomicAdd(&vs->peds, (unsigned long long)peds);
              atomicAdd(&vs->flops, (unsigned long long)flops);
              if (budget_hit) atomicExch(&vs->budget_hit, 1);
              __threadfence();
              last = (atomicSub(&vs->pending, 1) == 1);
              if (last) {
                __threadfence();
                volatile SdVec* vv = vs;
                gnc = vv->ncand;
                bh = vv->budget_hit;
                r2s = vv->r2_start;
                rs = vv->restarts;
              }
            }
            last = __shfl_sync(gmask, last, lead);
            gnc = __shfl_sync(gmask, gnc, lead);
            bh = __shfl_sync(gmask, bh, lead);
            r2s = __shfl_sync(gmask, r2s, lead);
            rs = __shfl_sync(gmask, rs, lead);
            nodes = peds = flops = 0;
            if (last) {
              if (gnc == 0 && !bh && r2s < INFINITY && rs < 64) {
                // empty sphere over all tasks: the root again with r^2 <- 2 r^2,
                // as a single task of this group (outstanding unchanged); the
                // counts so far are in vs
                restart = true;
                r2_start = 2.0f * r2s;
                restarts = rs + 1;
                if (gl == 0) {
                  vs->r2_start = r2_start;
                  vs->r2bits = __float_as_uint(r2_start);
                  vs->restarts = restarts;
                  vs->pending = 1;
                  __threadfence();
                }
                r2 = r2_start;
                committed = 0;
                solo = true;
                budget_hit = false;
              } else {
                rescore = true;
                use_global = true;
                nc = gnc;
                budget_hit = bh != 0;
              }
            }
          }
        }
        __syncwarp();
        if (restart) {
          // the root's residuals (no rows fixed) are ybar itself
          const float* yb = a.yb32 + (size_t)v * vec_stride32(n);
          for (int r = gl; r < n; r += G) ZW(zoff(n - 1) + r) = yb[r];
        }
        __syncwarp();
        if (restart) {
          top = n - 1;
          ncl = 0;
          bnd = prune_bound(r2, E, n);
          enter_level(top, 0.0f);
          n32 = 1;
          lsum = top;
          task_nodes = 0;
        }
        if (rescore) {
          // FP64 re-scoring of the candidates within FP32 error of the best
          SdVec* vs = vec_of(g, v);
          volatile SdVec* vv = vs;
          float best = INFINITY;
          for (int q = 0; q < nc; ++q) best = fminf(best, use_global ? vv->cand_ped[q] : cped[q]);
          const float keep = prune_bound(best, E, n);
          const double* R64 = a.R64 + (size_t)v * tri_stride64(n);
          const double* y64 = a.yb64 + (size_t)v * vec_stride64(n);
          int win = -1;
          double win_m = INFINITY;
          long long rescored = 0;
          for (int q = 0; q < nc; ++q) {
            const float cp = use_global ? vv->cand_ped[q] : cped[q];
            if (!(cp <= keep)) continue;
            const uint8_t* px = use_global ? cand_path(vs, q, n) : cx + q * kGroupN;
            double m;
            if (a.flags & MDX_NO_RESCORE) {
              m = (double)cp;
            } else {
              m = rescore_fp64_group<G>(n, lev64, R64, y64, px, use_global, gl, gmask);
              ++rescored;
            }
            bool better = m < win_m;
            if (!better && m == win_m && win >= 0) {
              // tie: lexicographically smaller index vector, top row first
              const uint8_t* wx = use_global ? cand_path(vs, win, n) : cx + win * kGroupN;
              for (int j = n - 1; j >= 0; --j) {
                const uint8_t w1 = use_global ? __ldcg(px + j) : px[j];
                const uint8_t w2 = use_global ? __ldcg(wx + j) : wx[j];
                if (w1 != w2) {
                  better = w1 < w2;
                  break;
                }
              }
            }
            if (better) {
              win = q;
              win_m = m;
            }
          }
          const uint8_t* wx = win >= 0 ? (use_global ? cand_path(vs, win, n) : cx + win * kGroupN) : nullptr;
          for (int j = gl; j < a.n_tx; j += G) {
            uint8_t q = 0;
            if (wx) {
              const int kre = use_global ? __ldcg(wx + 2 * j) : wx[2 * j];
              const int kim = use_global ? __ldcg(wx + 2 * j + 1) : wx[2 * j + 1];
              q = (uint8_t)(kre * P + kim);
            }
            a.sym_out[(size_t)v * a.n_tx + j] = q;
          }
          if (gl == 0) {
            a.metric_out[v] = (win >= 0) ? win_m : (double)INFINITY;
            const int rs = use_global ? vv->restarts : restarts;
            a.vstatus[v] = budget_hit ? MDX_V_BUDGET_EXCEEDED : (rs > 0 ? MDX_V_EMPTY_RETRIED : MDX_V_OK);
            if (a.stats) {
              // vs holds the counts committed under a node budget and those of
              // earlier passes or tasks; this group's own are added
              a.stats[(size_t)v * kStats + 0] = (long long)vv->nodes + nodes;
              a.stats[(size_t)v * kStats + 1] = (long long)vv->peds + peds;
              a.stats[(size_t)v * kStats + 2] = rs;
              a.stats[(size_t)v * kStats + 3] = rescored;
              a.stats[(size_t)v * kStats + 4] = (long long)vv->flops + flops;
            }
            atomicAdd(&g.sh->progress, 1u);
            atomicSub(&g.sh->outstanding, 1);
          }
          mode = 0;
        } else if (ev_done && !restart) {
          // a task of a split vector ended and others remain
          if (gl == 0) {
            atomicAdd(&g.sh->progress, 1u);
            atomicSub(&g.sh->outstanding, 1);
          }
          mode = 0;
        }
        __syncwarp();
        ev_done = false;
      }

      // ------------------------------------------------- acquire work
      const bool wants = (mode == 0) || (mode == 2 && (recheck || (since & 15) == 16 - kPassesPerVote));
      if (__any_sync(full, wants)) {
        // 0: nothing, 1: queued task, 2: fresh vector.  Fresh vectors come
        // first; once they are gone a group takes a ticket of the task queue
        // (one atomicAdd, no retries) and keeps it until that slot is published
        int got = 0, tv = -1, tlevel = 0;
        float tped = 0.0f;
        long long slot = -1;
        if (wants && gl == 0) {
          if (ticket < 0 && *(volatile unsigned int*)&g.sh->vec_next < (unsigned)a.batch) {
            // counted as running before it is taken: a waiting group that sees
            // every vector taken and nothing running may leave with its ticket
            atomicAdd(&g.sh->outstanding, 1);
            __threadfence();
            tv = (int)atomicAdd(&g.sh->vec_next, 1u);
            got = (tv < a.batch) ? 2 : 0;
            if (got == 2 && g.order) tv = g.order[tv];
            if (got == 0) atomicSub(&g.sh->outstanding, 1);
          }
          if (got == 0 && ticket < 0 && may_split)
            ticket = (long long)atomicAdd(&g.sh->q_head, 1u);
          if (got == 0 && ticket >= 0) {
            SdTask* t = g.queue + ((unsigned)ticket & (g.qcap - 1));
            if (*(volatile unsigned long long*)&t->seq == ((g.epoch << 32) | ((unsigned long long)ticket + 1ull))) {
              __threadfence();
              tv = *(volatile int*)&t->v;
              tlevel = *(volatile int*)&t->level;
              tped = *(volatile float*)&t->ped;
              got = (tv >= 0 && tv < a.batch && tlevel >= 0 && tlevel < n) ? 1 : -2;
              slot = ticket;
              ticket = -1;
            }
          }
        }
        got = __shfl_sync(full, got, lead);
        tv = __shfl_sync(full, tv, lead);
        tlevel = __shfl_sync(full, tlevel, lead);
        tped = __shfl_sync(full, tped, lead);
        slot = __shfl_sync(full, slot, lead);
        // copy the task's path, then free the slot
        if (got == 1)
          for (int j = tlevel + 1 + gl; j < n; j += G)
            XS(j) = (float)((volatile uint8_t*)g.queue[(unsigned)slot & (g.qcap - 1)].x)[j];
        __syncwarp();
        if ((got == 1 || got == -2) && gl == 0) {
          __threadfence();
          atomicExch(&g.queue[(unsigned)slot & (g.qcap - 1)].seq, g.epoch << 32);
          if (got == -2) {
            // a malformed record: counted as a finished task so the launch can end
            atomicExch(&g.sh->error, 2);
            atomicSub(&g.sh->outstanding, 1);
          }
        }
        if (got < 0) got = 0;
        if (wants && got == 0) mode = 2;
        // a fresh singular vector: zero outputs, no search
        if (got == 2 && a.singular && a.singular[tv]) {
          for (int j = gl; j < a.n_tx; j += G) a.sym_out[(size_t)tv * a.n_tx + j] = 0;
          if (gl == 0) {
            a.metric_out[tv] = 0.0;
            a.vstatus[tv] = MDX_V_SINGULAR;
            if (a.stats)
              for (int q = 0; q < kStats; ++q) a.stats[(size_t)tv * kStats + q] = 0;
            atomicSub(&g.sh->outstanding, 1);
          }
          got = 0;
          mode = 0;  // look again on the next pass
        }
        // stage R (and the per-row diagonal terms) of a new vector
        const bool stage = got != 0 && staged != tv;
        if (stage) {
          const float* src = a.R32 + (size_t)tv * ts;
          for (int cc = 0; cc < n; ++cc)
            for (int r = gl; r <= cc; r += G) RW(zoff(cc) + r) = src[col_off(cc) + r];
        }
        __syncwarp();
        if (stage) {
          for (int r = gl; r < n; r += G) {
            const float rr = RW(zoff(r) + r);
            LR(r) = make_float2(rr, 0.5f / (alpha * rr));
          }
          staged = tv;
        }
        __syncwarp();
        if (got != 0) {
          v = tv;
          SdVec* vs = vec_of(g, v);
          const float* yb = a.yb32 + (size_t)v * vec_stride32(n);
          if (got == 2) {
            // fresh vector: its FP32 error scale and initial radius
            const float amax = alpha * (float)(P - 1);
            float e2 = 0.0f;
            for (int r = gl; r < n; r += G) {
              float T = fabsf(yb[r]);
              for (int j = r; j < n; ++j) T += amax * fabsf(RW(zoff(j) + r));
              const float w = (float)(n - r + 1) * T;
              e2 += w * w;
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) e2 += __shfl_xor_sync(gmask, e2, o, G);
            E = sqrtf(e2) * kU32;
            float rr;
            if (a.radius_mode == RADIUS_NONE) rr = INFINITY;
            else if (a.radius_mode == RADIUS_PAPER) rr = (float)((double)a.n_rx * a.n_tx * a.noise_var[v]);
            else if (a.radius_mode == RADIUS_PER_VECTOR) rr = a.r2_vec[v];
            else rr = (float)a.radius_value;
            if (!(rr > 0.0f)) rr = INFINITY;
            r2 = rr;
            r2_start = rr;
            restarts = 0;
            budget_hit = false;
            solo = true;
            top = n - 1;
            tped = 0.0f;
            committed = 0;
            if (gl == 0) {
              vs->r2bits = __float_as_uint(rr);
              vs->pending = 1;
              vs->lock = 0;
              vs->ncand = 0;
              vs->nodes = vs->peds = vs->flops = 0ull;
              vs->restarts = 0;
              vs->budget_hit = 0;
              vs->E = E;
              vs->r2_start = rr;
              __threadfence();
            }
          } else {
            // queued task of a split vector: the vector's shared state
            float e = 0.0f, rr = 0.0f;
            unsigned long long cm = 0ull;
            int bh = 0;
            if (gl == 0) {
              e = *(volatile float*)&vs->E;
              rr = __uint_as_float(*(volatile unsigned int*)&vs->r2bits);
              cm = *(volatile unsigned long long*)&vs->nodes;
              bh = *(volatile int*)&vs->budget_hit;
            }
            E = __shfl_sync(gmask, e, lead);
            r2 = __shfl_sync(gmask, rr, lead);
            committed = (long long)__shfl_sync(gmask, cm, lead);
            budget_hit = __shfl_sync(gmask, bh, lead) != 0;
            solo = false;
            top = tlevel;
          }
          // residuals of the task node: z_r = ybar_r - sum_{j > top} R_rj x_j, r <= top
#pragma unroll
          for (int t = 0; t < RPL; ++t) {
            const int r = gl + G * t;
            if (r <= top) {
              float z = yb[r];
              for (int j = n - 1; j > top; --j)
                z = fmaf(-RW(zoff(j) + r), fmaf(XS(j), 2.0f, -(Pf - 1.0f)) * alpha, z);
              ZW(zoff(top) + r) = z;
            }
          }
        }
        __syncwarp();
        if (got != 0) {
          bnd = prune_bound(r2, E, n);
          enter_level(top, tped);
          nodes = peds = flops = 0;
          n32 = 1;
          p32 = 0;
          lsum = top;
          task_nodes = 0;
          ncl = 0;
          left32 = 0x7fffffff;
          if (a.budget > 0) {
            const long long left = a.budget - committed;
            left32 = left < 0 ? 0 : (left > 0x7fffffffll ? 0x7fffffff : (int)left);
          }
          if (budget_hit) left32 = 0;
          mode = 1;
        }
      }
      recheck = false;

      // ------------------------------------------ the whole warp waits
      if (!__any_sync(full, mode == 1)) {
        if (__any_sync(full, mode == 0)) continue;  // a group just ended a vector: look again
        // every group holds a ticket (or, in a search that does not split, has
        // nothing left to take): wait until a ticket's slot is published, fresh vectors
        // appear, or no task is queued or running any more.  The wait is bounded
        // by progress: it gives up (error word 4) only after about 2^22 polls in
        // which no task ended anywhere.
        int leave = 0;
        if (!may_split) {
          leave = 1;
        } else {
          unsigned int seen = 0;
          int quiet = 0;
          if (lane == 0) seen = *(volatile unsigned int*)&g.sh->progress;
          for (;;) {
            int ready = 0, stop = 0;
            if (gl == 0 && ticket >= 0) {
              const SdTask* t = g.queue + ((unsigned)ticket & (g.qcap - 1));
              ready = *(volatile unsigned long long*)&t->seq == ((g.epoch << 32) | ((unsigned long long)ticket + 1ull));
            }
            if (lane == 0) {
              if (*(volatile unsigned int*)&g.sh->vec_next < (unsigned)a.batch) {
                ready = 1;
              } else if (*(volatile int*)&g.sh->outstanding == 0) {
                stop = 1;
              } else {
                const unsigned int pr = *(volatile unsigned int*)&g.sh->progress;
                if (pr != seen) {
                  seen = pr;
                  quiet = 0;
                } else if (++quiet > (1 << 22)) {
                  atomicExch(&g.sh->error, 4);
                  stop = 1;
                }
              }
            }
            if (__any_sync(full, ready)) break;
            if (__shfl_sync(full, stop, 0)) {
              leave = 1;
              break;
            }
            __nanosleep(256);
          }
        }
        if (leave) break;
        recheck = true;
        continue;
      }
    }

    // ============================================================ node step
    // One child of the current level, in Schnorr-Euchner order: its partial
    // distance, then pop (none left inside the sphere), a leaf (slow path),
    // or descend.  Everything the step may need from shared memory is loaded
    // first, independently of the child chosen.  The step has no branch: the
    // groups of a warp that pop, descend, or have no task run the same
    // instructions under their own predicates (a branch would serialise the
    // outcomes and stall on its resolution every pass).  kPassesPerVote
    // passes run per vote of the slow paths; a group whose pass raised an
    // event (a leaf, the end of its task) sits the rest of them out.
#pragma unroll kPassUnroll
    for (int sub = 0; sub < kPassesPerVote; ++sub) {
      // rows i - 1 of the R and residual columns are read below by every lane
      // of the group, while only the row's owner wrote the residual (in an
      // earlier pass): the warp barrier orders those writes before the reads
      __syncwarp();
      const bool held = sub > 0 && (ev_leaf || ev_done);
      const bool busy = mode == 1 && !held;
      // rt = n (a task at the root) and im = -1 (a leaf) index past the level
      // arrays into their neighbours in shared memory; those values are never
      // used (no pop past the task's top level, no descent from level 0)
      const int im = i - 1;
      const int cm = ci + i + 1;  // zoff(i - 1)
      float rcv[RPL], zinv[RPL];
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        rcv[t] = RW(ci + gl + G * t);
        zinv[t] = ZW(ci + gl + G * t);
      }
      // row i - 1 of this level's R column and residuals, read by every lane
      // (the next level's interference without a shuffle from its owner)
      const float rim = RW(ci + im), zim = ZW(ci + im);
      const float4 stp = ST(rt);
      const float2 lrp = LR(rt);
      const int rtp = RT(rt);
      const float2 lrn = LR(im);
      const bool has_lo = flo >= 0.0f, has_hi = fhi < Pf;
      const bool has = busy && (has_lo || has_hi);
      const bool take_lo = has_lo && (!has_hi || fabsf(u - flo) <= fabsf(fhi - u));
      const float kf = take_lo ? flo : fhi;
      flo = (has && take_lo) ? flo - 1.0f : flo;
      fhi = (has && !take_lo) ? fhi + 1.0f : fhi;
      const float av = fmaf(kf, 2.0f, -(Pf - 1.0f)) * alpha;  // (2k - (P - 1)) alpha
      const float d = fmaf(-rii, av, c);
      const float ped = fmaf(d, d, ped_par);
      if (has) ++p32;
      const bool ok = has && ped < bnd;
      // The child's next sibling in Schnorr-Euchner order, evaluated now with
      // the same operations as the pass that would take it.  The pruning
      // bound only shrinks, so a sibling outside the sphere now is outside
      // then: the level ends with this child, and no pass comes back to it.
      const bool has_lo2 = flo >= 0.0f, has_hi2 = fhi < Pf;
      const bool take_lo2 = has_lo2 && (!has_hi2 || fabsf(u - flo) <= fabsf(fhi - u));
      const float kf2 = take_lo2 ? flo : fhi;
      const float d2 = fmaf(-rii, fmaf(kf2, 2.0f, -(Pf - 1.0f)) * alpha, c);
      const bool has2 = has_lo2 || has_hi2;
      const bool exh = !(has2 && fmaf(d2, d2, ped_par) < bnd);
      const bool deep = ok && i > 0;
      const bool leaf = ok && i == 0;
      bool visit = deep, bstop = false;  // the child is a visited (branched) node
      if (kBudget) {
        visit = deep && n32 < left32;
        bstop = deep && n32 >= left32;
        budget_hit = budget_hit || bstop;
      }
      // the new level's residuals (rows 0..i-1 matter; the rest spill into
      // deeper columns)
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const float zn = fmaf(-rcv[t], av, zinv[t]);
        if (visit) ZW(cm + gl + G * t) = zn;
      }
      if (visit) {
        ST(i) = make_float4(ped_par, c, flo, fhi);
        XS(i) = kf;
        RT(i) = (uint8_t)rt;
      }
      const float cnew = fmaf(-rim, av, zim);  // the same FMA as row i - 1's residual
      const float unew = fmaf(cnew, lrn.y, uoff);
      const float flonew = fminf(fmaxf(ceilf(unew - 0.5f), 0.0f), Pf - 1.0f);
      // The visited node's first child in Schnorr-Euchner order, evaluated
      // as the next pass would: flonew = ceil(u - 1/2) clamped to the
      // constellation is the PAM index nearest u (the lower one on a tie),
      // and the zig-zag takes it first.  Outside the sphere it rules out
      // every child of the node, so the group does not descend: the node and
      // that one evaluation are counted, and the group goes on with the next
      // child of level i, or leaves the level when none is inside.  (The
      // stores above, made for a descent, touch only state that a group at
      // level i never reads.)
      const float d1 = fmaf(-lrn.x, fmaf(flonew, 2.0f, -(Pf - 1.0f)) * alpha, cnew);
      const bool enter = fmaf(d1, d1, ped) < bnd;
      const bool desc = visit && enter;
      // the level is left: its child was outside the sphere (or none was
      // left), or the child (a leaf, or a node not entered) was the last one
      // inside
      const bool leave = busy && (!ok || (exh && (leaf || (visit && !enter))));
      const bool pop = leave && rt <= top;
      if (!held) {
        ev_done = (leave && rt > top) || bstop;
        ev_leaf = leaf;
        leaf_ped = ped;
        leaf_kf = kf;
      }
      const int zrt = kTri - (((rt + 1) * (rt + 2)) >> 1);  // zoff(rt)
      ci = desc ? cm : (pop ? zrt : ci);
      const int iold = i;
      i = desc ? im : (pop ? rt : i);
      ped_par = desc ? ped : (pop ? stp.x : ped_par);
      c = desc ? cnew : (pop ? stp.y : c);
      // the level's u is recomputed exactly as it was formed on the way down
      u = desc ? unew : (pop ? fmaf(stp.y, lrp.y, uoff) : u);
      rii = desc ? lrn.x : (pop ? lrp.x : rii);
      flo = desc ? flonew : (pop ? stp.z : flo);
      fhi = desc ? flonew + 1.0f : (pop ? stp.w : fhi);
      rt = desc ? (exh ? rt : iold) : (pop ? rtp : rt);
      if (visit) {
        ++n32;
        lsum += im;
        if (!enter) ++p32;
      }
      // the sibling's evaluation, when it ends the level, is one the
      // sequential search makes too
      if ((visit || leaf) && has2 && exh) ++p32;
    }

    since += kPassesPerVote;
  }
}

#undef RW
#undef ZW
#undef ST
#undef LR
#undef XS
#undef RT

template <int G, bool kBudget>
cudaError_t launch_group(const SdArgs& g, int num_sms, cudaStream_t s) {
  const size_t smem = group_cta_bytes<G>();
  cudaError_t e =
      cudaFuncSetAttribute(sd_group_kernel<G, kBudget>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sd_group_kernel<G, kBudget>, group_warps<G>() * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  sd_group_kernel<G, kBudget><<<per_sm * num_sms, group_warps<G>() * 32, smem, s>>>(g);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sd_group(const SdArgs& g, int num_sms, cudaStream_t s) {
  if (g.a.n > kGroupN) return cudaErrorInvalidConfiguration;
  return g.a.budget > 0 ? launch_group<kGroupLanes, true>(g, num_sms, s)
                        : launch_group<kGroupLanes, false>(g, num_sms, s);
}

}  // namespace mdx
