// Structures and protocols shared by the sphere decoder's two kernels: the
// warp-per-task kernel (sd.cu, any n) and the group kernel (sd_group.cu,
// n <= 32, several vectors per warp).  Both take work from the same task
// queue and keep the same per-vector state, described in sd.cu's header.
#pragma once

#include "mdx_internal.cuh"

namespace mdx {

// Global state of one SD launch (zeroed before the launch).
struct SdShared {
  unsigned int vec_next;
  unsigned int q_head;
  unsigned int q_tail;
  int outstanding;  // tasks queued or running (root tasks included)
  int idle;         // warps waiting for work
  int error;        // a bounded wait expired
  // event counters (read back by mdx_profile_read)
  unsigned int split_checks;   // periodic checks that saw idle warps
  unsigned int splits;         // checks that donated at least one task
  unsigned int donated;        // tasks donated
  unsigned int no_level;       // checks that found no level to split
  unsigned int progress;       // tasks ended (the group kernel's waits measure progress by it)
  int pad[5];
};

constexpr int kWarpsMax = 4;     // warps per CTA
constexpr int kCand = 8;         // leaf candidates kept per vector
constexpr int kSplitEvery = 128; // nodes between split / radius checks
constexpr int kTaskPath = 224;   // path bytes in a task record (n <= 224)
constexpr int kMinSplitLevel = 3; // donate only children with at least 3 rows below
constexpr int kSplitMinNodes = 512; // a task donates only after searching this many nodes

struct SdTask {
  unsigned long long seq;  // (epoch << 32) | (slot index + 1) once written
  int v;
  int level;  // row to expand; rows level+1..n-1 fixed in x[]
  float ped;
  int pad;
  uint8_t x[kTaskPath];
};
static_assert(sizeof(SdTask) == 248, "task record layout");

// Per-vector state in global memory.
struct SdVec {
  unsigned int r2bits;  // FP32 r^2 bits (non-negative floats order like uints)
  int pending;          // unfinished tasks of this vector
  int lock;             // candidate-list lock
  int ncand;
  unsigned long long nodes, peds, flops;
  int restarts;
  int budget_hit;
  float E;
  float r2_start;  // radius of the current pass (for doubling)
  float cand_ped[kCand];
  // followed by kCand paths of path_pad(n) bytes
};

__host__ __device__ inline int path_pad(int n) { return round_up(n, 16); }
__host__ __device__ inline size_t vec_state_bytes(int n) {
  return round_up((int)(sizeof(SdVec) + (size_t)kCand * path_pad(n)), 16);
}

__host__ __device__ inline size_t sd_warp_bytes(int n) {
  const size_t b = sizeof(float) * (2 * (size_t)tri_stride32(n) + 5 * (size_t)n) +
                   sizeof(int) * (size_t)n + (size_t)path_pad(n);
  return (b + 15) / 16 * 16;
}

struct SdArgs {
  SearchArgs a;
  SdShared* sh;
  SdTask* queue;
  unsigned int qcap;  // power of two
  unsigned char* vstate;
  size_t vstride;
  unsigned long long epoch;
  const int* order;  // fresh vectors in this order (heaviest first), or null
};

__device__ __forceinline__ SdVec* vec_of(const SdArgs& g, int v) {
  return reinterpret_cast<SdVec*>(g.vstate + (size_t)v * g.vstride);
}
__device__ __forceinline__ uint8_t* cand_path(SdVec* vs, int q, int n) {
  return reinterpret_cast<uint8_t*>(vs + 1) + (size_t)q * path_pad(n);
}

// Claim a queued task (lane 0); returns the slot index or -1 if the queue is empty.
__device__ inline long long queue_pop(const SdArgs& g) {
  volatile unsigned int* head = &g.sh->q_head;
  volatile unsigned int* tail = &g.sh->q_tail;
  for (int tries = 0; tries < 64; ++tries) {
    const unsigned int h = *head;
    if (h >= *tail) return -1;
    if (atomicCAS(&g.sh->q_head, h, h + 1) == h) return (long long)h;
  }
  return -1;
}

// Reserve cnt consecutive slots (lane 0); -1 if the ring has no room.  The
// head is read before the tail: the head never passes a tail read after it,
// so tail - head cannot underflow.
__device__ inline long long queue_reserve(const SdArgs& g, int cnt) {
  for (int tries = 0; tries < 4096; ++tries) {
    const unsigned int h = *(volatile unsigned int*)&g.sh->q_head;
    const unsigned int t = *(volatile unsigned int*)&g.sh->q_tail;
    if (t - h + (unsigned)cnt > g.qcap) return -1;
    if (atomicCAS(&g.sh->q_tail, t, t + (unsigned)cnt) == t) return (long long)t;
    __nanosleep(16);
  }
  return -1;
}

// A slot used before in this launch (index >= qcap) may be written only
// after the consumer of its previous occupant has copied it out and marked
// it free ((epoch << 32) | 0).  Lane 0; false if that never happened.
__device__ inline bool slot_writable(const SdArgs& g, SdTask* t, unsigned long long idx) {
  if (idx < g.qcap) return true;
  const unsigned long long freed = g.epoch << 32;
  for (int it = 0; it < (1 << 22); ++it) {
    if (*(volatile unsigned long long*)&t->seq == freed) {
      __threadfence();
      return true;
    }
    __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ bool lock_acquire(int* lk) {
  for (int it = 0; it < (1 << 22); ++it) {
    if (atomicCAS(lk, 0, 1) == 0) {
      __threadfence();
      return true;
    }
    __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void lock_release(int* lk) {
  __threadfence();
  atomicExch(lk, 0);
}

// The group kernel (sd_group.cu): four vectors per warp, n <= 32.
cudaError_t launch_sd_group(const SdArgs& g, int num_sms, cudaStream_t s);

}  // namespace mdx
