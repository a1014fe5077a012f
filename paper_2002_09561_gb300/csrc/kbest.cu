// K-best (Sec. VI) and the hybrid SD / K-best (Sec. VI), one CTA per
// received vector, vectors taken from a global counter.
//
// K-best level step, real tree (cta_kbest_levels below): every survivor's
// interference c_i = ybar_i - sum_{j>i} R_ij x_j (Eq. 4, shared by the node's
// P children, Eq. inc), then one 64-bit key per child (FP32 partial distance
// bits, then parent rank and child index), so that ordering the keys orders
// the level's candidates by (distance, parent rank, child) and the first K
// are the survivors; candidates outside the pruning bound get an all-ones key
// and sort last.  Keys are sorted in registers per warp and merged across
// warps (K <= 128; for larger K one bitonic sort in shared memory,
// kbest_levels); the new survivors copy their parent's path (4-byte words; the path
// stride is an odd number of words so that threads reading their own paths
// hit distinct banks) and append their child.  Complex tree (one level per
// antenna, Q = P^2 children, cta_kbest_levels_complex): the same selection
// over the S Q keys of a level (one bitonic sort in shared memory when K Q is
// too large for register runs, kbest_levels_complex).
//
// Hybrid.  The master part enumerates every depth-d prefix (rows n-1..n-d),
// keeps those inside the initial sphere and sorts them by partial distance;
// the CTA then finishes them best-first, each by a K-best run over the
// remaining rows under the current radius (a run stops as soon as all its
// survivors leave the sphere), and shrinks the radius with the run's best
// leaf: the best prefix on the whole CTA (cta_kbest_levels), the others one
// per warp (warp_kbest) on the warps that hold a K-best workspace.  Prefixes are taken while their own partial distance is inside the
// sphere; the first one outside ends the vector, since all later ones are
// farther.  The answer is the best K-best leaf over the prefixes inside the
// initial sphere, whatever the order, because a radius above the answer only
// removes nodes that could not lead to it.
//
// Both kernels keep the final leaves within FP32 error of the best and
// re-score them in FP64 against the FP64 R and ybar.
#include "mdx_internal.cuh"
#include "warp_kbest.cuh"

namespace mdx {
namespace {

struct KbLayout {
  int n, K, P, keys_cap, pp, ts;
  int T, E, G, lp;  // real tree: CTA level steps (cta_kbest_levels) geometry
  size_t off_R, off_yb, off_keys, off_xa, off_xb, off_pa, off_pb, off_cx, off_cp, off_cc, off_misc, off_m, bytes;
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
    off_cc = o;  // complex levels: the two rows' interference per survivor
    o += 2 * sizeof(float) * round_up(K, 4);
    off_misc = o;
    o += 64;
    off_m = o;  // FP64 metrics of the re-scored candidates
    o += sizeof(double) * kCandMax;
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
  float* cc;  // complex levels: [2][K] interference of rows 2j+1 and 2j per survivor
};

// ---------------------------------------------------------------------------
// K-best level steps by a whole CTA (T = 32 W threads), for one run from one
// node; the radius must not change during the run.  Per level: survivor t's
// interference (row_interference, G threads per survivor, the same bits as a
// warp's single-lane chains), then one key per child e = t P + k held in
// registers (E per thread, warp w holding the 32 E elements from 32 E w).
// With SE (the hybrid) a key orders the children as the tournament of
// warp_kbest emits them: its distance field is the running maximum of the
// partial distances along the survivor's Schnorr-Euchner order (a stream ends
// at its first child outside the bound, and a child leaves its stream only
// after the ones before it), then parent rank, Schnorr-Euchner rank, child;
// without SE (detect_kbest) it is (distance, parent rank, child).  Each warp
// sorts its keys in registers (bitonic: shuffles below stride 32, in-thread
// exchanges above); the warps' sorted runs are then merged pairwise through
// shared memory, keeping the 32 E smallest at each step (elementwise minimum
// against the partner's reversed run, then a bitonic merge), so that warp 0
// ends with the level's survivors.  Levels whose S P children fit in 32 lanes
// run on warp 0 alone (warp_level_small) while the other warps wait.
struct CtaRun {
  float* cc;      // [Kp] interference per survivor
  uint64_t* buf;  // [W][32 E] merge runs; [0, K) the level's survivor keys
  int* cnt;       // valid keys of the level
};

// Ascending sort of a bitonic run (size 64 E: every element ascends).
template <int E>
__device__ __forceinline__ void run_merge(uint64_t (&key)[E], int lane) {
#pragma unroll
  for (int stride = 16 * E; stride > 0; stride >>= 1) run_stage<E>(key, lane, 64 * E, stride);
}

template <int E, bool SE>
__device__ int cta_kbest_levels(const float* Rc, const float* yb, int n, int P, int lp, int K, int pp,
                                float alpha, int G, int top, const unsigned int* r2bits, float Es,
                                const CtaRun& w, uint8_t** xcur, uint8_t** xnxt, float** pcur, float** pnxt,
                                long long* nodes, long long* flops) {
  constexpr int R = 32 * E;
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, W = T >> 5;
  const float uoff = 0.5f * (float)(P - 1);
  const int wpp = pp >> 2;
  int S = 1, i = top;
  while (i >= 0 && S > 0) {
    if (S * P <= 32 && P <= 8) {
      // levels whose children fit in one warp: warp 0 alone, no CTA barrier
      if (warp == 0) {
        int steps = 0;
        // nothing else changes the radius during a CTA's run
        const float b = prune_bound(__uint_as_float(*(volatile const unsigned int*)r2bits), Es, n);
        while (i >= 0 && S > 0 && S * P <= 32) {
          const int kept = warp_level_small<SE>(Rc, yb, n, P, K, pp, alpha, i, b, S, *xcur, *xnxt, *pcur, *pnxt, lane);
          *nodes += S;
          *flops += (long long)S * (2 * (n - 1 - i) + 4 * P);
          uint8_t* tx = *xcur;
          *xcur = *xnxt;
          *xnxt = tx;
          float* tp = *pcur;
          *pcur = *pnxt;
          *pnxt = tp;
          S = kept;
          --i;
          ++steps;
        }
        if (lane == 0) {
          w.cnt[1] = S;
          w.cnt[2] = i;
          w.cnt[3] = steps;
        }
      }
      __syncthreads();
      S = w.cnt[1];
      i = w.cnt[2];
      if (warp != 0 && (w.cnt[3] & 1)) {
        uint8_t* tx = *xcur;
        *xcur = *xnxt;
        *xnxt = tx;
        float* tp = *pcur;
        *pcur = *pnxt;
        *pnxt = tp;
      }
      continue;
    }
    const float bnd = prune_bound(__uint_as_float(*(volatile const unsigned int*)r2bits), Es, n);
    if (G == 1) {
      // one thread per survivor, several survivors per thread when S > T
      for (int t = tid; t < S; t += T) w.cc[t] = row_interference<1>(Rc, yb, *xcur + (size_t)t * pp, n, P, alpha, i, 0);
    } else {
      const int t = tid / G, s = tid - t * G;
      const bool act = t < S;
      const uint8_t* xp = *xcur + (size_t)(act ? t : 0) * pp;
      float ci;
      if (G == 8) ci = row_interference<8>(Rc, yb, xp, n, P, alpha, i, s);
      else if (G == 4) ci = row_interference<4>(Rc, yb, xp, n, P, alpha, i, s);
      else ci = row_interference<2>(Rc, yb, xp, n, P, alpha, i, s);
      if (act && s == 0) w.cc[t] = ci;
    }
    __syncthreads();
    const float rii = Rc[col_off(i) + i];
    const float rinv = 0.5f / (alpha * rii);
    uint64_t key[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int e = warp * R + r * 32 + lane;
      const int t = e >> lp, k = e & (P - 1);
      const bool act = t < S;
      const float c = act ? w.cc[t] : 0.0f;
      const float p0 = act ? (*pcur)[t] : 0.0f;
      const float u = fmaf(c, rinv, uoff);
      const float d = fmaf(-rii, (float)(2 * k - (P - 1)) * alpha, c);
      const float ped = fmaf(d, d, p0);
      key[r] = child_key<SE>(ped, u, t, k, P, act, bnd, lane);
    }
    run_sort<E>(key, lane);
    for (int h = 1; h < W; h <<= 1) {
      if ((warp & (2 * h - 1)) == h) {
#pragma unroll
        for (int r = 0; r < E; ++r) w.buf[warp * R + r * 32 + lane] = key[r];
      }
      __syncthreads();
      if ((warp & (2 * h - 1)) == 0 && warp + h < W) {
#pragma unroll
        for (int r = 0; r < E; ++r) key[r] = kmin(key[r], w.buf[(warp + h) * R + (R - 1 - (r * 32 + lane))]);
        run_merge<E>(key, lane);
      }
    }
    if (warp == 0) {
      int valid = 0;
#pragma unroll
      for (int r = 0; r < E; ++r) {
        valid += __popc(__ballot_sync(0xffffffffu, key[r] != kInfKey));
        if (r * 32 + lane < K) w.buf[r * 32 + lane] = key[r];
      }
      if (lane == 0) *w.cnt = valid;
    }
    __syncthreads();
    const int kept = min(K, *w.cnt);
    for (int idx = tid; idx < kept * wpp; idx += T) {
      const int s = idx / wpp, wd = idx - s * wpp;
      const unsigned lo = (unsigned)w.buf[s];
      const int t = (int)(lo >> 8), k = (int)(lo & 15u);
      uint32_t word = reinterpret_cast<const uint32_t*>(*xcur + (size_t)t * pp)[wd];
      if (wd == (i >> 2)) {
        const int sh = 8 * (i & 3);
        word = (word & ~(0xffu << sh)) | ((uint32_t)k << sh);
      }
      reinterpret_cast<uint32_t*>(*xnxt + (size_t)s * pp)[wd] = word;
      if (wd == 0) {
        const float d = fmaf(-rii, (float)(2 * k - (P - 1)) * alpha, w.cc[t]);
        (*pnxt)[s] = fmaf(d, d, (*pcur)[t]);
      }
    }
    *nodes += S;
    *flops += (long long)S * (2 * (n - 1 - i) + 4 * P);
    __syncthreads();
    uint8_t* tx = *xcur;
    *xcur = *xnxt;
    *xnxt = tx;
    float* tp = *pcur;
    *pcur = *pnxt;
    *pnxt = tp;
    S = kept;
    --i;
  }
  return S;
}

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
        // child-major slots: consecutive threads write consecutive keys
        c.keys[k * S + tid] = (ped < bnd) ? (((uint64_t)__float_as_uint(ped) << 32) | id) : kInfKey;
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

// Complex-tree level steps (one level per complex antenna j: real rows 2j+1
// then 2j, Q = P^2 children): thread t computes the interference of both rows
// for survivor t and the partial distances of its Q children; keys
// (distance, parent rank * Q + q) are sorted as in kbest_levels.
__device__ int kbest_levels_complex(const KbCtx& c, int S, uint8_t** xcur, uint8_t** xnxt, float** pcur,
                                    float** pnxt, const float* r2s, float E, long long* nodes, long long* peds,
                                    long long* flops) {
  const int n = c.n, P = c.P, Q = P * P, K = c.K, pp = c.pp, tid = c.tid, T = c.T;
  for (int j = n / 2 - 1; j >= 0 && S > 0; --j) {
    const int r1 = 2 * j + 1, r0 = 2 * j;
    const float bnd = prune_bound(*r2s, E, n);
    const int SQ = S * Q;
    const int Cs = pow2ceil(SQ < 2 ? 2 : SQ);
    // interference of both rows, one thread per survivor
    for (int t = tid; t < S; t += T) {
      const uint8_t* xp = *xcur + (size_t)t * pp;
      float c1 = c.yb[r1], c0 = c.yb[r0];
      for (int jj = n - 1; jj > r1; --jj) {
        const float a = (float)(2 * (int)xp[jj] - (P - 1)) * c.alpha;
        c1 = fmaf(-c.Rc[col_off(jj) + r1], a, c1);
        c0 = fmaf(-c.Rc[col_off(jj) + r0], a, c0);
      }
      c.cc[t] = c1;
      c.cc[K + t] = c0;
    }
    __syncthreads();
    // the S Q children over all threads, child-major
    const float r11 = c.Rc[col_off(r1) + r1], r01 = c.Rc[col_off(r1) + r0], r00 = c.Rc[col_off(r0) + r0];
    for (int e = tid; e < SQ; e += T) {
      const int q = e / S, t = e - q * S;
      const int kre = q / P, kim = q - kre * P;
      const float aim = (float)(2 * kim - (P - 1)) * c.alpha, are = (float)(2 * kre - (P - 1)) * c.alpha;
      const float d1 = fmaf(-r11, aim, c.cc[t]);
      const float p1 = fmaf(d1, d1, (*pcur)[t]);
      const float d0 = fmaf(-r00, are, fmaf(-r01, aim, c.cc[K + t]));
      const float pd = fmaf(d0, d0, p1);
      const unsigned id = (unsigned)(t * Q + q);
      c.keys[e] = (pd < bnd) ? (((uint64_t)__float_as_uint(pd) << 32) | id) : kInfKey;
    }
    for (int q = SQ + tid; q < Cs; q += T) c.keys[q] = kInfKey;
    if (tid == 0) c.misc[0] = 0;
    __syncthreads();
    bitonic_sort(c.keys, Cs, tid, T);
    for (int q = tid; q < Cs; q += T)
      if (c.keys[q] != kInfKey && (q + 1 == Cs || c.keys[q + 1] == kInfKey)) c.misc[0] = q + 1;
    __syncthreads();
    const int valid = c.misc[0];
    const int kept = valid < K ? valid : K;
    for (int t = tid; t < kept; t += T) {
      const uint64_t key = c.keys[t];
      const unsigned id = (unsigned)(key & 0xffffffffu);
      const int par = (int)(id / (unsigned)Q), q = (int)(id % (unsigned)Q);
      const uint32_t* src = reinterpret_cast<const uint32_t*>(*xcur + (size_t)par * pp);
      uint32_t* dst = reinterpret_cast<uint32_t*>(*xnxt + (size_t)t * pp);
      for (int w = 0; w < pp / 4; ++w) dst[w] = src[w];
      (*xnxt)[(size_t)t * pp + r1] = (uint8_t)(q % P);
      (*xnxt)[(size_t)t * pp + r0] = (uint8_t)(q / P);
      (*pnxt)[t] = __uint_as_float((unsigned)(key >> 32));
    }
    *nodes += S;
    *peds += SQ;
    *flops += (long long)S * (4 * (n - 2 - r0) + 10 * Q);
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

// Complex-tree K-best level steps by a whole CTA (one level per antenna j:
// real rows 2j+1 and 2j, Q = P^2 children): each survivor's interference of
// both rows (one thread per survivor, as in kbest_levels_complex), then one
// key (distance, parent rank * Q + q) per child, E per thread, sorted in
// registers per warp and merged across warps as in cta_kbest_levels.
template <int E>
__device__ int cta_kbest_levels_complex(const KbCtx& c, int lq, const CtaRun& w, uint8_t** xcur, uint8_t** xnxt,
                                        float** pcur, float** pnxt, const float* r2s, float Es, long long* nodes,
                                        long long* peds, long long* flops) {
  constexpr int R = 32 * E;
  const int n = c.n, P = c.P, Q = P * P, K = c.K, pp = c.pp, tid = c.tid, T = c.T;
  const int lane = tid & 31, warp = tid >> 5, W = T >> 5, wpp = pp >> 2;
  int S = 1;
  for (int j = n / 2 - 1; j >= 0 && S > 0; --j) {
    const int r1 = 2 * j + 1, r0 = 2 * j;
    const float bnd = prune_bound(*r2s, Es, n);
    for (int t = tid; t < S; t += T) {
      const uint8_t* xp = *xcur + (size_t)t * pp;
      float c1 = c.yb[r1], c0 = c.yb[r0];
      for (int jj = n - 1; jj > r1; --jj) {
        const float a = (float)(2 * (int)xp[jj] - (P - 1)) * c.alpha;
        c1 = fmaf(-c.Rc[col_off(jj) + r1], a, c1);
        c0 = fmaf(-c.Rc[col_off(jj) + r0], a, c0);
      }
      w.cc[t] = c1;
      w.cc[K + t] = c0;
    }
    __syncthreads();
    const float r11 = c.Rc[col_off(r1) + r1], r01 = c.Rc[col_off(r1) + r0], r00 = c.Rc[col_off(r0) + r0];
    uint64_t key[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int e = warp * R + r * 32 + lane;
      const int t = e >> lq, q = e & (Q - 1);
      key[r] = kInfKey;
      if (t < S) {
        const int kre = q / P, kim = q - kre * P;
        const float aim = (float)(2 * kim - (P - 1)) * c.alpha, are = (float)(2 * kre - (P - 1)) * c.alpha;
        const float d1 = fmaf(-r11, aim, w.cc[t]);
        const float p1 = fmaf(d1, d1, (*pcur)[t]);
        const float d0 = fmaf(-r00, are, fmaf(-r01, aim, w.cc[K + t]));
        const float pd = fmaf(d0, d0, p1);
        if (pd < bnd) key[r] = ((uint64_t)__float_as_uint(pd) << 32) | (unsigned)e;
      }
    }
    run_sort<E>(key, lane);
    for (int h = 1; h < W; h <<= 1) {
      if ((warp & (2 * h - 1)) == h) {
#pragma unroll
        for (int r = 0; r < E; ++r) w.buf[warp * R + r * 32 + lane] = key[r];
      }
      __syncthreads();
      if ((warp & (2 * h - 1)) == 0 && warp + h < W) {
#pragma unroll
        for (int r = 0; r < E; ++r) key[r] = kmin(key[r], w.buf[(warp + h) * R + (R - 1 - (r * 32 + lane))]);
        run_merge<E>(key, lane);
      }
    }
    if (warp == 0) {
      int valid = 0;
#pragma unroll
      for (int r = 0; r < E; ++r) {
        valid += __popc(__ballot_sync(0xffffffffu, key[r] != kInfKey));
        if (r * 32 + lane < K) w.buf[r * 32 + lane] = key[r];
      }
      if (lane == 0) *w.cnt = valid;
    }
    __syncthreads();
    const int kept = min(K, *w.cnt);
    // new paths: rows 2j+1 (imaginary index) and 2j (real index) share a word
    const int wj = r0 >> 2, sh = 8 * (r0 & 3);
    for (int idx = tid; idx < kept * wpp; idx += T) {
      const int s = idx / wpp, wd = idx - s * wpp;
      const unsigned id = (unsigned)w.buf[s];
      const int t = (int)(id >> lq), q = (int)(id & (unsigned)(Q - 1));
      const int kre = q / P, kim = q - kre * P;
      uint32_t word = reinterpret_cast<const uint32_t*>(*xcur + (size_t)t * pp)[wd];
      if (wd == wj) word = (word & ~(0xffffu << sh)) | ((uint32_t)kre << sh) | ((uint32_t)kim << (sh + 8));
      reinterpret_cast<uint32_t*>(*xnxt + (size_t)s * pp)[wd] = word;
      if (wd == 0) {
        const float aim = (float)(2 * kim - (P - 1)) * c.alpha, are = (float)(2 * kre - (P - 1)) * c.alpha;
        const float d1 = fmaf(-r11, aim, w.cc[t]);
        const float p1 = fmaf(d1, d1, (*pcur)[t]);
        const float d0 = fmaf(-r00, are, fmaf(-r01, aim, w.cc[K + t]));
        (*pnxt)[s] = fmaf(d0, d0, p1);
      }
    }
    *nodes += S;
    *peds += (long long)S * Q;
    *flops += (long long)S * (4 * (n - 2 - r0) + 10 * Q);
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
  {
    // the FP64 R and ybar are read only by the final re-scoring: bring them
    // into L2 now, so that it does not wait on DRAM
    const char* r64 = reinterpret_cast<const char*>(a.R64 + (size_t)v * tri_stride64(a.n));
    const int rbytes = (int)sizeof(double) * tri_stride64(a.n);
    for (int off = tid * 128; off < rbytes; off += T * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(r64 + off));
  }
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

// FP64 ||ybar - R x||^2 of the path x with the columns split over the CTA's
// nw warps (warp w takes j = w, w + nw, ...; a chain of dependent FP64 FMAs is
// slow on this GPU, so shorter chains on all four schedulers finish sooner);
// warp 0 adds the warps' residual partials in warp order and returns the
// metric on its lanes (the other warps return 0).  part: nw * 224 doubles of
// shared memory.  Every thread of the CTA calls this.
__device__ double rescore_fp64_cta(int n, int P, double alpha64, const double* __restrict__ R64,
                                   const double* __restrict__ y64, const uint8_t* x, double* part) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double rr[7];
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    const int r = lane + 32 * t;
    rr[t] = (warp == 0 && r < n) ? y64[r] : 0.0;
  }
  const double lv = (double)(2 * (lane < P ? lane : 0) - (P - 1)) * alpha64;
  for (int j = warp; j < n; j += nw) {
    const double xj = __shfl_sync(0xffffffffu, lv, (int)x[j]);
    const double* col = R64 + col_off(j);
#pragma unroll
    for (int t = 0; t < 7; ++t) {
      const int r = lane + 32 * t;
      if (32 * t <= j && r <= j) rr[t] = fma(-col[r], xj, rr[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < 7; ++t) part[warp * 224 + lane + 32 * t] = rr[t];
  __syncthreads();
  double m = 0.0;
  if (warp == 0) {
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < 7; ++t) {
      const int r = lane + 32 * t;
      double z = 0.0;
      for (int w = 0; w < nw; ++w) z += part[w * 224 + r];
      if (r < n) s = fma(z, z, s);
    }
    m = __shfl_sync(0xffffffffu, warp_sum(s), 0);
  }
  __syncthreads();
  return m;
}

// Re-score candidate paths (cx, cped; count nc, sorted or not) in FP64 and
// write the outputs of vector v with warp 0 (every thread calls this).
// part == nullptr: one candidate per warp; else each candidate by the whole
// CTA (rescore_fp64_cta, part its scratch).  mbuf: kCandMax doubles of
// shared memory.
__device__ void finish_vector(const SearchArgs& a, int v, const uint8_t* cx, const float* cped,
                              int nc, int pp, float E, int status, long long nodes, long long peds,
                              long long restarts, long long flops, double* mbuf, double* part) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int n = a.n, P = a.P;
  float best = INFINITY;
  for (int q = 0; q < nc; ++q) best = fminf(best, cped[q]);
  const float keep = prune_bound(best, E, n);
  const double* R64 = a.R64 + (size_t)v * tri_stride64(n);
  const double* y64 = a.yb64 + (size_t)v * vec_stride64(n);
  if (part && !(a.flags & MDX_NO_RESCORE)) {
    for (int q = 0; q < nc; ++q) {
      const double m = (cped[q] <= keep) ? rescore_fp64_cta(n, P, a.alpha64, R64, y64, cx + (size_t)q * pp, part)
                                         : (double)INFINITY;
      if (tid == 0) mbuf[q] = m;
    }
  } else {
    for (int q = warp; q < nc; q += nw) {
      double m = INFINITY;
      if (cped[q] <= keep)
        m = (a.flags & MDX_NO_RESCORE) ? (double)cped[q]
                                       : rescore_fp64_warp(n, P, a.alpha64, R64, y64, cx + (size_t)q * pp, lane);
      if (lane == 0) mbuf[q] = m;
    }
  }
  __syncthreads();
  if (warp != 0) return;
  int win = -1;
  double win_m = INFINITY;
  long long rescored = 0;
  for (int q = 0; q < nc; ++q) {
    if (!(cped[q] <= keep)) continue;
    const double m = mbuf[q];
    if (!(a.flags & MDX_NO_RESCORE)) ++rescored;
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

__global__ void __launch_bounds__(1024) kbest_kernel(SearchArgs a, KbLayout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, T = blockDim.x;
  const int n = a.n, P = a.P;
  uint64_t* keys = reinterpret_cast<uint64_t*>(smem + L.off_keys);
  int* misc = reinterpret_cast<int*>(smem + L.off_misc);
  float* misc_f = reinterpret_cast<float*>(misc + 4);
  KbCtx c{n, P, a.K, L.pp, tid, T, a.alpha, reinterpret_cast<float*>(smem + L.off_R),
          reinterpret_cast<float*>(smem + L.off_yb), keys, misc, reinterpret_cast<float*>(smem + L.off_cc)};

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
      if ((a.flags & MDX_COMPLEX_TREE) && L.E == 0) {
        S = kbest_levels_complex(c, 1, &xcur, &xnxt, &pcur, &pnxt, &misc_f[1], E, &nodes, &peds, &flops);
      } else if (a.flags & MDX_COMPLEX_TREE) {
        const CtaRun run{c.cc, keys, misc + 8};
        if (L.E == 1)
          S = cta_kbest_levels_complex<1>(c, L.lp, run, &xcur, &xnxt, &pcur, &pnxt, &misc_f[1], E, &nodes, &peds,
                                          &flops);
        else if (L.E == 2)
          S = cta_kbest_levels_complex<2>(c, L.lp, run, &xcur, &xnxt, &pcur, &pnxt, &misc_f[1], E, &nodes, &peds,
                                          &flops);
        else
          S = cta_kbest_levels_complex<4>(c, L.lp, run, &xcur, &xnxt, &pcur, &pnxt, &misc_f[1], E, &nodes, &peds,
                                          &flops);
      } else if (L.E == 0) {
        S = kbest_levels(c, n - 1, 1, &xcur, &xnxt, &pcur, &pnxt, &misc_f[1], E, &nodes, &peds, &flops);
      } else {
        const CtaRun run{c.cc, keys, misc + 8};
        const unsigned int* r2b = reinterpret_cast<const unsigned int*>(&misc_f[1]);
        long long rn = 0, rf = 0;
        if (L.E == 1)
          S = cta_kbest_levels<1, false>(c.Rc, c.yb, n, P, L.lp, a.K, L.pp, a.alpha, L.G, n - 1, r2b, E, run, &xcur,
                                         &xnxt, &pcur, &pnxt, &rn, &rf);
        else if (L.E == 2)
          S = cta_kbest_levels<2, false>(c.Rc, c.yb, n, P, L.lp, a.K, L.pp, a.alpha, L.G, n - 1, r2b, E, run, &xcur,
                                         &xnxt, &pcur, &pnxt, &rn, &rf);
        else
          S = cta_kbest_levels<4, false>(c.Rc, c.yb, n, P, L.lp, a.K, L.pp, a.alpha, L.G, n - 1, r2b, E, run, &xcur,
                                         &xnxt, &pcur, &pnxt, &rn, &rf);
        nodes += rn;
        peds += rn * P;
        flops += rf;
      }
      if (S > 0 || !(misc_f[1] < INFINITY) || restarts >= 64) break;
      __syncthreads();
      if (tid == 0) misc_f[1] *= 2.0f;  // empty sphere: double the radius r^2
      ++restarts;
      __syncthreads();
    }
    const int nc = S < kCandMax ? S : kCandMax;
    finish_vector(a, v, xcur, pcur, nc, L.pp, E, restarts > 0 ? MDX_V_EMPTY_RETRIED : MDX_V_OK,
                  nodes, peds, restarts, flops, reinterpret_cast<double*>(smem + L.off_m), nullptr);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Hybrid with warp workers.  Shared memory: R and ybar (FP32), the sorted list
// of in-sphere prefixes (u16 indices), the vector's radius r2 (FP32 bits,
// shrunk with atomicMin by any warp) and leaf-candidate list (guarded by a
// shared-memory lock), and one K-best workspace per warp.  During the master
// phase the warp workspaces double as the prefix sort buffer.
struct HyLayout {
  int n, K, P, W, Wk, pp, ts, Cw;  // W warps per CTA, Wk of them with a K-best workspace; Cw: key capacity per warp
  size_t off_R, off_yb, off_idx, off_cx, off_cp, off_misc, off_m, off_warp, warp_bytes, bytes;
  // the best prefix's run by the whole CTA (cta = 0: by warp 0 alone): G threads
  // per survivor, E keys per thread, lp = log2 P; buffers at off_warp + run_*
  int cta, G, E, lp;
  size_t run_xa, run_xb, run_pa, run_pb, run_cc, run_buf, run_cnt, run_bytes;
};


__host__ __device__ inline size_t hy_warp_bytes(int n, int K, int P) {
  const size_t pp = path_stride(n);
  (void)P;
  const size_t b = 2 * sizeof(uint16_t) * round_up(K, 8) + 2 * pp * K + 2 * sizeof(float) * round_up(K, 4);
  return (b + 15) / 16 * 16;
}

__host__ __device__ inline void hy_layout(HyLayout& L, int n, int K, int P, int W, int Wk, size_t sort_bytes) {
  L.n = n;
  L.K = K;
  L.P = P;
  L.W = W;
  L.Wk = Wk;
  L.pp = path_stride(n);
  L.ts = tri_stride32(n);
  L.Cw = round_up(K, 8);
  size_t o = 0;
  L.off_R = o;
  o += sizeof(float) * L.ts;
  L.off_yb = o;
  o += sizeof(float) * round_up(n, 4);
  L.off_idx = o;
  o += sizeof(uint16_t) * 4096;
  L.off_cp = o;
  o += sizeof(float) * kCandMax;
  L.off_misc = o;
  o += 128;
  L.off_m = o;
  o += sizeof(double) * kCandMax;
  L.off_cx = o;
  o += (size_t)L.pp * kCandMax;
  o = (o + 15) / 16 * 16;
  L.off_warp = o;
  L.warp_bytes = hy_warp_bytes(n, K, P);
  // the warp workspaces double as the master's prefix sort buffer, as the
  // buffers of the CTA's run and as the re-scoring partials
  size_t need = ((sort_bytes + Wk - 1) / Wk + 15) / 16 * 16;
  const int T = 32 * W, Kp = pow2ceil(K);
  L.lp = 0;
  while ((1 << L.lp) < P) ++L.lp;
  L.E = 1;
  while (L.E <= 4 && (T * L.E < Kp * P || 32 * L.E < Kp)) L.E <<= 1;
  L.G = 1;
  while (L.G < 8 && 2 * L.G * Kp <= T) L.G <<= 1;
  L.cta = (Kp <= T && L.E <= 4 && (1 << L.lp) == P && P <= 16) ? 1 : 0;
  {
    size_t r = 0;
    auto take = [&](size_t bytes) {
      const size_t at = r;
      r += (bytes + 15) / 16 * 16;
      return at;
    };
    L.run_xa = take((size_t)L.pp * K);
    L.run_xb = take((size_t)L.pp * K);
    L.run_pa = take(sizeof(float) * K);
    L.run_pb = take(sizeof(float) * K);
    L.run_cc = take(sizeof(float) * Kp);
    L.run_buf = take(sizeof(uint64_t) * (size_t)T * L.E);
    L.run_cnt = take(16);
    L.run_bytes = r;
  }
  if (L.cta) {
    const size_t per = ((L.run_bytes + Wk - 1) / Wk + 15) / 16 * 16;
    if (need < per) need = per;
  }
  const size_t part = ((sizeof(double) * 224 * W + Wk - 1) / Wk + 15) / 16 * 16;  // one row block per CTA warp
  if (need < part) need = part;
  if (L.warp_bytes < need) L.warp_bytes = need;
  o += L.warp_bytes * Wk;
  L.bytes = o;
}

__global__ void hybrid_kernel(SearchArgs a, HyLayout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, T = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int n = a.n, P = a.P, d = a.depth, K = a.K;
  float* Rc = reinterpret_cast<float*>(smem + L.off_R);
  float* yb = reinterpret_cast<float*>(smem + L.off_yb);
  uint16_t* pidx = reinterpret_cast<uint16_t*>(smem + L.off_idx);
  float* cped = reinterpret_cast<float*>(smem + L.off_cp);
  uint8_t* cx = smem + L.off_cx;
  int* misc = reinterpret_cast<int*>(smem + L.off_misc);
  // misc: [0] vector, [1] valid prefixes, [2] next prefix, [3] ncand, [4] lock,
  //       [5] r2 bits, [6] E bits, [7] stop, [8] budget hit, [9] error
  unsigned int* r2bits = reinterpret_cast<unsigned int*>(&misc[5]);
  unsigned char* wbase = smem + L.off_warp + (size_t)warp * L.warp_bytes;
  uint16_t* wsel = reinterpret_cast<uint16_t*>(wbase);
  uint8_t* wxa = wbase + 2 * sizeof(uint16_t) * L.Cw;
  uint8_t* wxb = wxa + (size_t)L.pp * K;
  float* wpa = reinterpret_cast<float*>(wxb + (size_t)L.pp * K);
  float* wpb = wpa + round_up(K, 4);
  uint64_t* sortbuf = reinterpret_cast<uint64_t*>(smem + L.off_warp);  // master phase only
  int np = 1;
  for (int l = 0; l < d; ++l) np *= P;

  for (;;) {
    if (tid == 0) misc[0] = (int)atomicAdd(a.work_counter, 1u);
    __syncthreads();
    const int v = misc[0];
    __syncthreads();
    if (v >= a.batch) break;
    if (singular_vector(a, v)) continue;
    {
      KbLayout dummy;
      dummy.off_R = L.off_R;
      dummy.off_yb = L.off_yb;
      dummy.ts = L.ts;
      stage_vector(a, v, dummy, smem, reinterpret_cast<float*>(&misc[10]));
    }
    const float E = reinterpret_cast<float*>(&misc[10])[0];
    unsigned long long* acc_budget = reinterpret_cast<unsigned long long*>(&misc[12]);  // nodes (budgeted)
    unsigned long long* acc_nodes = reinterpret_cast<unsigned long long*>(&misc[14]);
    unsigned long long* acc_flops = reinterpret_cast<unsigned long long*>(&misc[16]);
    if (tid == 0) {
      misc[5] = (int)__float_as_uint(reinterpret_cast<float*>(&misc[10])[1]);
      misc[3] = 0;
      misc[4] = 0;
      misc[8] = 0;
      *acc_budget = 0ull;
      *acc_nodes = 0ull;
      *acc_flops = 0ull;
    }
    __syncthreads();
    long long nodes = 0, peds = 0, restarts = 0, flops = 0;
    for (;;) {
      // ---- master: every depth-d prefix inside the sphere, sorted by partial distance
      // (the in-sphere prefixes are compacted first, so that only they are sorted)
      const float bnd0 = prune_bound(__uint_as_float((unsigned)misc[5]), E, n);
      if (tid == 0) misc[18] = 0;
      __syncthreads();
      for (int q = tid; q < np; q += T) {
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
        if (ped < bnd0) sortbuf[atomicAdd(&misc[18], 1)] = ((uint64_t)__float_as_uint(ped) << 32) | (unsigned)q;
      }
      __syncthreads();
      const int nin = misc[18];
      const int Cs = pow2ceil(nin < 2 ? 2 : nin);
      for (int q = nin + tid; q < Cs; q += T) sortbuf[q] = kInfKey;
      __syncthreads();
      bitonic_sort(sortbuf, Cs, tid, T);
      for (int q = tid; q < nin; q += T) pidx[q] = (uint16_t)(sortbuf[q] & 0xffffu);
      if (tid == 0) misc[1] = nin;
      if (tid == 0) {
        misc[2] = 0;
        misc[7] = 0;
      }
      nodes += (tid == 0) ? 1 : 0;
      __syncthreads();
      const int nvalid = misc[1];
      // ---- workers: the best prefix is finished first (its leaf sets the
      // radius, as the paper's SD master explores best-first), by the whole CTA
      // or else by warp 0 alone; then every warp takes the remaining prefixes
      // in order
      long long wnodes = 0, wflops = 0;
      if (L.cta && nvalid > 0) {
        unsigned char* rb = smem + L.off_warp;
        uint8_t* xcur = rb + L.run_xa;
        uint8_t* xnxt = rb + L.run_xb;
        float* pcur = reinterpret_cast<float*>(rb + L.run_pa);
        float* pnxt = reinterpret_cast<float*>(rb + L.run_pb);
        const CtaRun run{reinterpret_cast<float*>(rb + L.run_cc), reinterpret_cast<uint64_t*>(rb + L.run_buf),
                         reinterpret_cast<int*>(rb + L.run_cnt)};
        const int q = pidx[0];
        float pped = 0.0f;
        {
          int rem = q;
          for (int l = 0; l < d; ++l) {
            const int i = n - 1 - l;
            const int k = rem % P;
            rem /= P;
            if (tid == 0) xcur[i] = (uint8_t)k;
            float ci = yb[i];
            int rr = q;
            for (int m = 0; m < l; ++m) {
              const int km = rr % P;
              rr /= P;
              ci = fmaf(-Rc[col_off(n - 1 - m) + i], (float)(2 * km - (P - 1)) * a.alpha, ci);
            }
            const float dd = fmaf(-Rc[col_off(i) + i], (float)(2 * k - (P - 1)) * a.alpha, ci);
            pped = fmaf(dd, dd, pped);
          }
        }
        const float r2 = __uint_as_float(*(volatile unsigned int*)r2bits);
        if (!(pped < prune_bound(r2, E, n))) {
          if (tid == 0) misc[7] = 1;  // sorted best-first: no prefix is inside the sphere
        } else {
          if (tid == 0) {
            pcur[0] = pped;
            misc[2] = 1;
            wnodes += 1;
            wflops += 2 * (d > 0 ? d - 1 : 0) + 4 * P;
          }
          __syncthreads();
          long long rn = 0, rf = 0;
          int S;
          if (L.E == 1)
            S = cta_kbest_levels<1, true>(Rc, yb, n, P, L.lp, K, L.pp, a.alpha, L.G, n - 1 - d, r2bits, E, run, &xcur,
                                    &xnxt, &pcur, &pnxt, &rn, &rf);
          else if (L.E == 2)
            S = cta_kbest_levels<2, true>(Rc, yb, n, P, L.lp, K, L.pp, a.alpha, L.G, n - 1 - d, r2bits, E, run, &xcur,
                                    &xnxt, &pcur, &pnxt, &rn, &rf);
          else
            S = cta_kbest_levels<4, true>(Rc, yb, n, P, L.lp, K, L.pp, a.alpha, L.G, n - 1 - d, r2bits, E, run, &xcur,
                                    &xnxt, &pcur, &pnxt, &rn, &rf);
          if (tid == 0) {
            wnodes += rn;
            wflops += rf;
          }
          if (S > 0) {
            // the run's leaves within FP32 error of its best start the candidate list
            const float lim = prune_bound(fminf(pcur[0], r2), E, n);
            int nc = 0;
            while (nc < S && nc < kCandMax && pcur[nc] <= lim) ++nc;
            const int wpp = L.pp / 4;
            for (int idx = tid; idx < nc * wpp; idx += T)
              reinterpret_cast<uint32_t*>(cx)[idx] = reinterpret_cast<const uint32_t*>(xcur)[idx];
            if (tid < nc) cped[tid] = pcur[tid];
            if (tid == 0) {
              misc[3] = nc;
              atomicMin(r2bits, __float_as_uint(pcur[0]));
            }
          }
          if (a.budget > 0 && tid == 0) {
            const unsigned long long tot = atomicAdd(acc_budget, (unsigned long long)wnodes) + wnodes;
            if ((long long)tot >= a.budget) misc[8] = 1;
            wnodes = 0;
          }
        }
        __syncthreads();
      }
      for (int phase = L.cta ? 1 : 0; phase < 2; ++phase) {
       if (phase == 1) __syncthreads();
       if ((phase == 1 && warp < L.Wk) || warp == 0) {
        for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&misc[2], 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= nvalid) break;
        int stopped = 0;
        if (lane == 0) stopped = *(volatile int*)&misc[7] | *(volatile int*)&misc[8];
        if (__shfl_sync(0xffffffffu, stopped, 0)) break;
        const int q = pidx[t];
        uint8_t* xcur = wxa;
        uint8_t* xnxt = wxb;
        float* pcur = wpa;
        float* pnxt = wpb;
        // the prefix's path and partial distance (recomputed, same FMA chain as the master)
        float pped = 0.0f;
        {
          int rem = q;
          for (int l = 0; l < d; ++l) {
            const int i = n - 1 - l;
            const int k = rem % P;
            rem /= P;
            if (lane == 0) xcur[i] = (uint8_t)k;
            float ci = yb[i];
            int rr = q;
            for (int m = 0; m < l; ++m) {
              const int km = rr % P;
              rr /= P;
              ci = fmaf(-Rc[col_off(n - 1 - m) + i], (float)(2 * km - (P - 1)) * a.alpha, ci);
            }
            const float dd = fmaf(-Rc[col_off(i) + i], (float)(2 * k - (P - 1)) * a.alpha, ci);
            pped = fmaf(dd, dd, pped);
          }
        }
        float r2 = 0.0f;
        if (lane == 0) r2 = __uint_as_float(*(volatile unsigned int*)r2bits);
        r2 = __shfl_sync(0xffffffffu, r2, 0);
        if (!(pped < prune_bound(r2, E, n))) {
          // sorted best-first: every later prefix is outside the sphere too
          if (lane == 0) atomicExch(&misc[7], 1);
          break;
        }
        if (lane == 0) pcur[0] = pped;
        __syncwarp();
        wnodes += 1;
        wflops += 2 * (d > 0 ? d - 1 : 0) + 4 * P;
        const int S = warp_kbest_any(Rc, yb, n, P, K, L.pp, a.alpha, n - 1 - d, r2bits, E, wsel, &xcur, &xnxt,
                                     &pcur, &pnxt, lane, &wnodes, &wflops);
        if (S > 0) {
          // this run's leaves within FP32 error of its best join the candidate list
          float cur = 0.0f;
          if (lane == 0) cur = __uint_as_float(*(volatile unsigned int*)r2bits);
          cur = __shfl_sync(0xffffffffu, cur, 0);
          const float lim = prune_bound(fminf(pcur[0], cur), E, n);
          for (int sidx = 0; sidx < S && sidx < kCandMax; ++sidx) {
            const float ps = pcur[sidx];
            if (!(ps <= lim)) break;
            int slot = -1;
            if (lane == 0) {
              bool got = false;
              for (int it = 0; it < (1 << 20); ++it) {
                if (atomicCAS(&misc[4], 0, 1) == 0) {
                  got = true;
                  break;
                }
                __nanosleep(32);
              }
              if (got) {
                const int nc = *(volatile int*)&misc[3];
                if (nc < kCandMax) {
                  slot = nc;
                  misc[3] = nc + 1;
                } else {
                  float worst = -1.0f;
                  int w = -1;
                  for (int c2 = 0; c2 < kCandMax; ++c2)
                    if (((volatile float*)cped)[c2] > worst) {
                      worst = ((volatile float*)cped)[c2];
                      w = c2;
                    }
                  if (ps < worst) slot = w;
                }
                if (slot < 0) {
                  __threadfence_block();
                  atomicExch(&misc[4], 0);
                }
              } else {
                atomicExch(&misc[9], 1);
              }
            }
            slot = __shfl_sync(0xffffffffu, slot, 0);
            if (slot >= 0) {
              const uint32_t* src = reinterpret_cast<const uint32_t*>(xcur + (size_t)sidx * L.pp);
              uint32_t* dst = reinterpret_cast<uint32_t*>(cx + (size_t)slot * L.pp);
              for (int w2 = lane; w2 < L.pp / 4; w2 += 32) dst[w2] = src[w2];
              __syncwarp();
              if (lane == 0) {
                cped[slot] = ps;
                __threadfence_block();
                atomicExch(&misc[4], 0);
              }
            }
          }
          if (lane == 0) atomicMin(r2bits, __float_as_uint(pcur[0]));
        }
        if (a.budget > 0) {
          // commit this warp's nodes; the vector stops once the budget is spent
          if (lane == 0) {
            const unsigned long long tot = atomicAdd(acc_budget, (unsigned long long)wnodes) + wnodes;
            if ((long long)tot >= a.budget) atomicExch(&misc[8], 1);
          }
          wnodes = 0;
        }
        __syncwarp();
        if (phase == 0) break;  // warp 0 hands over after the best prefix
        }
       }
      }
      if (lane == 0) {
        atomicAdd(acc_nodes, (unsigned long long)wnodes);
        atomicAdd(acc_flops, (unsigned long long)wflops);
      }
      __syncthreads();
      const int nc = misc[3];
      const float r2now = __uint_as_float((unsigned)misc[5]);
      if (nc > 0 || misc[8] || !(r2now < INFINITY) || restarts >= 64) break;
      // empty sphere: double the radius and run master and workers again
      if (tid == 0) misc[5] = (int)__float_as_uint(2.0f * r2now);
      ++restarts;
      __syncthreads();
    }
    nodes += (long long)*acc_nodes + (long long)*acc_budget;
    flops = (long long)*acc_flops;
    peds = nodes * P;
    const int status = misc[8] ? MDX_V_BUDGET_EXCEEDED : (restarts > 0 ? MDX_V_EMPTY_RETRIED : MDX_V_OK);
    finish_vector(a, v, cx, cped, misc[3], L.pp, E, status, nodes, peds, restarts, flops,
                  reinterpret_cast<double*>(smem + L.off_m), reinterpret_cast<double*>(smem + L.off_warp));
    __syncthreads();
  }
}

int kb_threads(int K, int P);

// Real tree: T threads, E keys per thread (T E >= Kp P slots, warp runs of
// 32 E >= Kp keys), G threads per survivor's interference (1 when Kp > T).
// Runs of 32 E keys sort in registers up to E = 4 (K <= 128); larger K keep
// the shared-memory bitonic step (E = 0), measured faster there (K = 256,
// 16x16 16-QAM: 132 against 150 ms per 100k vectors).
void kb_geometry(KbLayout& L, int n, int K, int P) {
  const int Kp = pow2ceil(K), C = Kp * P;
  int T = C / 4;
  if (T < 32) T = 32;
  if (T > 256) T = 256;
  int E = 1;
  while (T * E < C || 32 * E < Kp) E <<= 1;
  int G = 1;
  while (G < 8 && 2 * G * Kp <= T) G <<= 1;
  L.lp = 0;
  while ((1 << L.lp) < P) ++L.lp;
  if (E > 4) {
    L.T = kb_threads(K, P);
    L.E = 0;
    L.G = 1;
    L.init(n, K, P, C < 2 ? 2 : C);
    return;
  }
  L.T = T;
  L.E = E;
  L.G = G;
  L.init(n, K, P, T * E);
}

// Complex tree: the same with Q = P^2 children per survivor (lp holds log2 Q).
void kb_geometry_complex(KbLayout& L, int n, int K, int P) {
  const int Q = P * P, Kp = pow2ceil(K), C = Kp * Q;
  int T = C / 4;
  if (T < 32) T = 32;
  if (T > 512) T = 512;
  int E = 1;
  while (T * E < C || 32 * E < Kp) E <<= 1;
  L.lp = 0;
  while ((1 << L.lp) < Q) ++L.lp;
  L.G = 1;
  if (E > 4) {
    L.T = kb_threads(K, Q);
    L.E = 0;
    L.init(n, K, P, C < 2 ? 2 : C);
    return;
  }
  L.T = T;
  L.E = E;
  L.init(n, K, P, T * E);
}

int kb_threads(int K, int P) {
  int C = pow2ceil(K * P);
  int T = C / 2;
  if (T < 32) T = 32;
  if (T > 1024) T = 1024;
  return T;
}

cudaError_t launch_generic(const void* fn, const SearchArgs& a, const KbLayout& L, int T, int num_sms,
                           cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, T, L.bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = per_sm * num_sms;
  if (grid > a.batch) grid = a.batch;
  kbest_kernel<<<grid, T, L.bytes, s>>>(a, L);
  return cudaGetLastError();
}

}  // namespace

size_t kbest_smem_bytes(int n, int K, int P, bool complex_tree) {
  KbLayout L;
  if (complex_tree) {
    kb_geometry_complex(L, n, K, P);
  } else {
    kb_geometry(L, n, K, P);
  }
  return L.bytes;
}

cudaError_t launch_kbest(const SearchArgs& a, int num_sms, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  KbLayout L;
  if (a.flags & MDX_COMPLEX_TREE) {
    kb_geometry_complex(L, a.n, a.K, a.P);
    if (L.bytes > 227 * 1024) return cudaErrorInvalidConfiguration;
    return launch_generic((const void*)kbest_kernel, a, L, L.T, num_sms, s);
  }
  kb_geometry(L, a.n, a.K, a.P);
  if (L.bytes > 227 * 1024) return cudaErrorInvalidConfiguration;
  return launch_generic((const void*)kbest_kernel, a, L, L.T, num_sms, s);
}

// Eight warps per CTA with as many K-best workspaces as fit (the best prefix
// runs on the whole CTA, the other prefixes on the warps with a workspace);
// fewer warps only when not even one workspace fits beside eight warps' needs.
bool hy_fit(HyLayout& L, int n, int K, int P, size_t sort_bytes) {
  for (int W = 8; W >= 1; --W)
    for (int Wk = W; Wk >= 1; --Wk) {
      hy_layout(L, n, K, P, W, Wk, sort_bytes);
      if (L.bytes <= 227 * 1024) return true;
    }
  return false;
}

cudaError_t launch_hybrid(const SearchArgs& a, int num_sms, cudaStream_t s) {
  if (a.batch <= 0) return cudaSuccess;
  int np = 1;
  for (int l = 0; l < a.depth; ++l) np *= a.P;
  const size_t sort_bytes = sizeof(uint64_t) * pow2ceil(np < 2 ? 2 : np);
  HyLayout L;
  if (!hy_fit(L, a.n, a.K, a.P, sort_bytes)) return cudaErrorInvalidConfiguration;
  const int W = L.W;
  const void* fn = (const void*)hybrid_kernel;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, W * 32, L.bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = per_sm * num_sms;
  if (grid > a.batch) grid = a.batch;
  hybrid_kernel<<<grid, W * 32, L.bytes, s>>>(a, L);
  return cudaGetLastError();
}

size_t hybrid_smem_bytes(int n, int K, int P, int depth) {
  int np = 1;
  for (int l = 0; l < depth; ++l) np *= P;
  const size_t sort_bytes = sizeof(uint64_t) * pow2ceil(np < 2 ? 2 : np);
  HyLayout L;
  return hy_fit(L, n, K, P, sort_bytes) ? L.bytes : (size_t)-1;
}

}  // namespace mdx
