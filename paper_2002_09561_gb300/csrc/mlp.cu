// Learned initial radius and child ordering: a 2-hidden-layer MLP (width 256)
// evaluated and trained with BF16 operands and FP32 accumulation on the 5th
// generation tensor cores.  The paper has no learned component; the network
// only proposes a starting radius for the exact sphere decoder, which still
// returns the ML point (an empty sphere doubles the radius and searches again).
//
// Network, per received vector with real dimension n and P-PAM per row:
//   x  = [R upper triangle (column-packed order), ybar, SNR_dB / 30, 0 pad]   (D0 = pad64(n(n+1)/2 + n + 1))
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), o = W3 h2 + b3          (H = 256, DO = pad128(1 + n P))
//   o[0]            predicts t = log(d_ML / sigma^2) (pinball loss, tau = 0.9: over-predicts)
//   o[1 + r P + k]  logit that row r of the ML point takes PAM index k (cross-entropy)
//
// GEMM core (tc_gemm): D[M x N] = A[M x K] * B[N x K]^T with A and B K-major
// BF16 in global memory.  One CTA of 128 threads computes a 128 x TN tile:
// thread 0 streams 128x64 (A) and TNx64 (B) boxes into a 4-stage
// shared-memory ring with TMA (cp.async.bulk.tensor, 128-byte swizzle) and
// issues tcgen05.mma (M=128, N=TN, K=16) into a TMEM accumulator; each MMA
// group commits to the stage's "empty" barrier so the ring refills as soon as
// the tensor core is done with it.  After the last commit all four warps read
// their 32 TMEM lanes with tcgen05.ld and apply the fused epilogue (bias, ReLU,
// ReLU-mask for the backward pass, FP32 or BF16 output, optional transposed
// BF16 copy).  Every mbarrier wait is bounded: on expiry the kernel records
// an error, waits (bounded) for its copies in flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include "mdx_internal.cuh"

namespace mdx {
namespace {

constexpr int kTM = 128;    // tile rows
constexpr int kTK = 64;     // K per stage (one 128-byte swizzle row of BF16)
constexpr int kStages = 4;
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// true when the phase with parity `phase` has completed; bounded
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  const uint32_t a = smem_u32(bar);
  for (int it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile whose rows are 128 bytes with
// the 128-byte swizzle (8-row atoms of 1024 bytes; stride between atoms 1024).
__device__ __forceinline__ uint64_t sdesc_sw128(const void* p) {
  const uint32_t a = smem_u32(p);
  uint64_t d = 0;
  d |= (uint64_t)((a & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;               // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
  d |= (uint64_t)1 << 46;               // descriptor version
  d |= (uint64_t)2 << 61;               // 128-byte swizzle
  return d;
}

// Instruction descriptor for kind::f16 with BF16 A/B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

#define TMEM_LD32(taddr, r)                                                                                   \
  asm volatile(                                                                                               \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17," \
      "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                      \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),       \
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), \
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),            \
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),            \
        "=r"(r[30]), "=r"(r[31])                                                                              \
      : "r"(taddr))

}  // namespace

// Epilogue of one GEMM launch.
struct TcEpi {
  int mode;  // TC_F32, TC_BIAS_RELU, TC_MASK
  const float* bias;          // [N] (TC_F32 optional, TC_BIAS_RELU)
  const __nv_bfloat16* mask;  // [M][ldm] forward activation (TC_MASK)
  int ldm;
  float* outf;  // [M][ldf] FP32 output (TC_F32)
  int ldf;
  __nv_bfloat16* outb;  // [M][ldb] BF16 output (TC_BIAS_RELU, TC_MASK)
  int ldb;
  __nv_bfloat16* outt;  // [N][ldt] BF16 transposed copy, or null
  int ldt;
  int* err;
};
enum { TC_F32 = 0, TC_BIAS_RELU = 1, TC_MASK = 2 };

namespace {

template <int TN>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB, int K, TcEpi epi) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int A_BYTES = kTM * kTK * 2;
  constexpr int B_BYTES = TN * kTK * 2;
  constexpr int TMEM_COLS = TN <= 32 ? 32 : TN <= 64 ? 64 : TN <= 128 ? 128 : 256;
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * B_BYTES);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* fail = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * TN;
  const int nk = K / kTK;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // stages loaded (thread 0)
  if (tid == 0) {
    const uint32_t idesc = idesc_bf16(kTM, TN);
    const int pro = nk < kStages ? nk : kStages;
    for (int s = 0; s < pro; ++s) {
      mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
      tma_load_2d(sA + s * A_BYTES, &tmA, s * kTK, m0, &full[s]);
      tma_load_2d(sB + s * B_BYTES, &tmB, s * kTK, n0, &full[s]);
      ++issued;
    }
    bool ok = true;
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % kStages;
      const uint32_t ph = (uint32_t)(kb / kStages) & 1u;
      if (!mbar_wait(&full[s], ph)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kTK / 16; ++kk) {
        const uint64_t da = sdesc_sw128(sA + s * A_BYTES + kk * 32);
        const uint64_t db = sdesc_sw128(sB + s * B_BYTES + kk * 32);
        umma_bf16(tmem, da, db, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
      }
      umma_commit(&empty[s]);
      if (kb + kStages < nk) {
        if (!mbar_wait(&empty[s], ph)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
        tma_load_2d(sA + s * A_BYTES, &tmA, (kb + kStages) * kTK, m0, &full[s]);
        tma_load_2d(sB + s * B_BYTES, &tmB, (kb + kStages) * kTK, n0, &full[s]);
        ++issued;
      }
    }
    umma_commit(done);
    if (!ok) {
      *fail = 1;
      atomicExch(epi.err, 1);
    }
  }
  // wait for the last MMA group (one thread per warp polls, then the warp proceeds)
  int dok = 1;
  if (lane == 0) dok = mbar_wait(done, 0) ? 1 : 0;
  dok = __shfl_sync(0xffffffffu, dok, 0);
  __syncthreads();
  if (!dok || *fail) {
    if (tid == 0) {
      atomicExch(epi.err, 1);
      // wait (bounded) for every TMA load this CTA issued before releasing the
      // shared memory they target
      for (int j = 0; j < issued; ++j) mbar_wait(&full[j % kStages], (uint32_t)(j / kStages) & 1u);
    }
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    for (int c = 0; c < TN; c += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
      TMEM_LD32(taddr, r);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int col0 = n0 + c;
      // the thread's row, 32 columns: 16-byte loads and stores (the launcher
      // checks the alignment of every epilogue pointer and leading dimension)
      if (epi.mode == TC_F32) {
        float4* o = reinterpret_cast<float4*>(epi.outf + (size_t)row * epi.ldf + col0);
        const float4* b = epi.bias ? reinterpret_cast<const float4*>(epi.bias + col0) : nullptr;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float4 v = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                 __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
          if (b) {
            const float4 bb = b[q];
            v.x += bb.x;
            v.y += bb.y;
            v.z += bb.z;
            v.w += bb.w;
          }
          o[q] = v;
        }
      } else {
        __align__(16) __nv_bfloat16 vb[32];
        if (epi.mode == TC_BIAS_RELU) {
          const float4* b = reinterpret_cast<const float4*>(epi.bias + col0);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 bb = b[q];
            vb[4 * q] = __float2bfloat16(fmaxf(__uint_as_float(r[4 * q]) + bb.x, 0.0f));
            vb[4 * q + 1] = __float2bfloat16(fmaxf(__uint_as_float(r[4 * q + 1]) + bb.y, 0.0f));
            vb[4 * q + 2] = __float2bfloat16(fmaxf(__uint_as_float(r[4 * q + 2]) + bb.z, 0.0f));
            vb[4 * q + 3] = __float2bfloat16(fmaxf(__uint_as_float(r[4 * q + 3]) + bb.w, 0.0f));
          }
        } else {
          const uint4* m = reinterpret_cast<const uint4*>(epi.mask + (size_t)row * epi.ldm + col0);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            __align__(16) __nv_bfloat16 mk[8];
            *reinterpret_cast<uint4*>(mk) = m[q];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const float v = __uint_as_float(r[8 * q + j]);
              vb[8 * q + j] = __float2bfloat16(__bfloat162float(mk[j]) > 0.0f ? v : 0.0f);
            }
          }
        }
        uint4* o = reinterpret_cast<uint4*>(epi.outb + (size_t)row * epi.ldb + col0);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = reinterpret_cast<const uint4*>(vb)[q];
        if (epi.outt) {
#pragma unroll
          for (int j = 0; j < 32; ++j) epi.outt[(size_t)(col0 + j) * epi.ldt + row] = vb[j];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D BF16 tensor map over a row-major [rows][cols] matrix with leading
// dimension ld (elements); boxes of box_rows x 64 with the 128-byte swizzle.
bool make_tmap(CUtensorMap* tm, const void* base, int rows, int cols, int ld, int box_rows) {
  EncodeTiledFn f = encode_fn();
  if (!f) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return f(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int TN>
cudaError_t launch_tc(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const TcEpi& epi,
                      cudaStream_t s) {
  CUtensorMap ta, tb;
  if (!make_tmap(&ta, A, M, K, lda, kTM) || !make_tmap(&tb, B, N, K, ldb, TN)) return cudaErrorInvalidValue;
  const size_t smem = 1024 + (size_t)kStages * (kTM + TN) * kTK * 2 + 256;
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(M / kTM, N / TN);
  tc_gemm_kernel<TN><<<grid, 128, smem, s>>>(ta, tb, K, epi);
  return cudaGetLastError();
}

}  // namespace

// D[M x N] = A[M x K] B[N x K]^T, A and B row-major BF16 with leading
// dimensions lda, ldb (elements, multiples of 8); M % 128 == 0, K % 64 == 0,
// N % tile == 0 for tile in {256, 192, 128, 64}.
cudaError_t tc_gemm(const void* A, int lda, const void* B, int ldb, int M, int N, int K, const TcEpi& epi,
                    cudaStream_t s) {
  if (M % kTM || K % kTK || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  if ((lda % 8) || (ldb % 8)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) return cudaErrorInvalidValue;
  // the epilogue moves 16 bytes at a time along each output row
  auto misaligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; };
  if (epi.mode == TC_F32 && (!epi.outf || misaligned(epi.outf) || epi.ldf % 4)) return cudaErrorInvalidValue;
  if (epi.mode != TC_F32 && (!epi.outb || misaligned(epi.outb) || epi.ldb % 8)) return cudaErrorInvalidValue;
  if (epi.mode == TC_BIAS_RELU && (!epi.bias || misaligned(epi.bias))) return cudaErrorInvalidValue;
  if (epi.mode == TC_F32 && epi.bias && misaligned(epi.bias)) return cudaErrorInvalidValue;
  if (epi.mode == TC_MASK && (!epi.mask || misaligned(epi.mask) || epi.ldm % 8)) return cudaErrorInvalidValue;
  if (N % 256 == 0) return launch_tc<256>(A, lda, B, ldb, M, N, K, epi, s);
  if (N % 192 == 0) return launch_tc<192>(A, lda, B, ldb, M, N, K, epi, s);
  if (N % 128 == 0) return launch_tc<128>(A, lda, B, ldb, M, N, K, epi, s);
  if (N % 64 == 0) return launch_tc<64>(A, lda, B, ldb, M, N, K, epi, s);
  return cudaErrorInvalidValue;
}

}  // namespace mdx

// ======================================================================================
// MLP model, training and inference (orchestrates tc_gemm and the small kernels below)
// ======================================================================================
namespace mdx {
namespace {

constexpr int kH = 256;

__global__ void mlp_features_kernel(int batch, int rows, int n, int D0, const float* __restrict__ R32,
                                    const float* __restrict__ yb32, const double* __restrict__ nv,
                                    __nv_bfloat16* X, __nv_bfloat16* Xt, float* F) {
  // a warp per vector row, its lanes over the features (no index division)
  const int T = n * (n + 1) / 2;
  const int ts = tri_stride32(n), vs = vec_stride32(n);
  const int lane = threadIdx.x & 31;
  const int w0 = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)(((long long)gridDim.x * blockDim.x) >> 5);
  for (int v = w0; v < rows; v += nw) {
    for (int f = lane; f < D0; f += 32) {
      float x = 0.0f;
      if (v < batch) {
        if (f < T) x = R32[(size_t)v * ts + f];
        else if (f < T + n) x = yb32[(size_t)v * vs + (f - T)];
        else if (f == T + n) x = (float)(-10.0 * log10(nv[v]) / 30.0);
      }
      const __nv_bfloat16 b = __float2bfloat16(x);
      X[(size_t)v * D0 + f] = b;
      if (Xt) Xt[(size_t)f * rows + v] = b;
      if (F && v < batch) F[(size_t)v * D0 + f] = x;
    }
  }
}

// One warp per vector: pinball loss on o[0] (target log(d_ML / sigma^2)) and
// cross-entropy of every row's ML PAM index; writes dL/do (BF16, both layouts).
// Summary features of a large system (n_tx > 32), one warp per vector: log R_ii
// (n values), log(d_B / sigma^2) / 10 with d_B the FP32 distance of the Babai
// point (successive rounding, top row first, clipped to the PAM grid),
// log(||ybar||^2 / (n sigma^2)) / 10 and SNR_dB / 30; zero-padded to D0.
__global__ void reduced_features_kernel(int batch, int rows, int n, int P, float alpha, int D0,
                                        const float* __restrict__ R32, const float* __restrict__ yb32,
                                        const double* __restrict__ nv, __nv_bfloat16* X, __nv_bfloat16* Xt,
                                        float* F) {
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int ts = tri_stride32(n), vs = vec_stride32(n);
  for (int v = w0; v < rows; v += nw) {
    float db = 0.0f, ybn = 0.0f, s2 = 1.0f;
    const float* R = R32 + (size_t)v * ts;
    if (v < batch) {
      const float* yb = yb32 + (size_t)v * vs;
      s2 = (float)nv[v];
      float z[7];
#pragma unroll
      for (int t = 0; t < 7; ++t) {
        const int r = lane + 32 * t;
        z[t] = (r < n) ? yb[r] : 0.0f;
        ybn = fmaf(z[t], z[t], ybn);
      }
      ybn = warp_sum(ybn);
      for (int i = n - 1; i >= 0; --i) {
        float zi = 0.0f;
#pragma unroll
        for (int t = 0; t < 7; ++t)
          if (t == (i >> 5)) zi = z[t];
        const float c = __shfl_sync(0xffffffffu, zi, i & 31);
        const float rii = R[col_off(i) + i];
        const float u = c / (2.0f * alpha * rii) + 0.5f * (float)(P - 1);
        const float k = fminf(fmaxf(floorf(u + 0.5f), 0.0f), (float)(P - 1));
        const float a = (2.0f * k - (float)(P - 1)) * alpha;
        const float d = fmaf(-rii, a, c);
        db = fmaf(d, d, db);
#pragma unroll
        for (int t = 0; t < 7; ++t) {
          const int r = lane + 32 * t;
          if (r < i) z[t] = fmaf(-R[col_off(i) + r], a, z[t]);
        }
      }
    }
    for (int f = lane; f < D0; f += 32) {
      float x = 0.0f;
      if (v < batch) {
        if (f < n) x = logf(R[col_off(f) + f]);
        else if (f == n) x = logf(fmaxf(db, 1e-30f) / s2) / 10.0f;
        else if (f == n + 1) x = logf(fmaxf(ybn, 1e-30f) / ((float)n * s2)) / 10.0f;
        else if (f == n + 2) x = (float)(-10.0 * log10(nv[v]) / 30.0);
      }
      const __nv_bfloat16 b = __float2bfloat16(x);
      X[(size_t)v * D0 + f] = b;
      if (Xt) Xt[(size_t)f * rows + v] = b;
      if (F && v < batch) F[(size_t)v * D0 + f] = x;
    }
  }
}

__global__ void mlp_loss_kernel(int batch, int rows, int n, int P, int n_tx, int DO, const float* __restrict__ O,
                                const double* __restrict__ ml_metric, const double* __restrict__ nv,
                                const uint8_t* __restrict__ ml_sym, float tau, float lambda, int ce_rows,
                                __nv_bfloat16* dO, __nv_bfloat16* dOt, float* loss) {
  const int warps = blockDim.x / 32;
  const int v = blockIdx.x * warps + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (v >= rows) return;
  const float inv_b = 1.0f / (float)batch;
  float lr = 0.0f, lc = 0.0f;
  for (int j = lane; j < DO; j += 32) {
    float g = 0.0f;
    if (v < batch) {
      if (j == 0) {
        const float t = (float)log(ml_metric[v] / nv[v]);
        const float e = t - O[(size_t)v * DO];
        lr = (e >= 0.0f ? tau * e : (tau - 1.0f) * e);
        g = (e > 0.0f ? -tau : (1.0f - tau)) * inv_b;
      } else if (j < 1 + ce_rows * P) {
        const int r = (j - 1) / P, k = (j - 1) % P;
        const float* lg = O + (size_t)v * DO + 1 + r * P;
        float mx = lg[0];
        for (int q = 1; q < P; ++q) mx = fmaxf(mx, lg[q]);
        float s = 0.0f;
        for (int q = 0; q < P; ++q) s += __expf(lg[q] - mx);
        const int qs = ml_sym[(size_t)v * n_tx + r / 2];
        const int kt = (r & 1) ? (qs % P) : (qs / P);
        const float pk = __expf(lg[k] - mx) / s;
        g = lambda * (pk - (k == kt ? 1.0f : 0.0f)) * inv_b / (float)n;
        if (k == kt) lc += -logf(fmaxf(pk, 1e-30f)) / (float)n;
      }
    }
    const __nv_bfloat16 b = __float2bfloat16(g);
    dO[(size_t)v * DO + j] = b;
    dOt[(size_t)j * rows + v] = b;
  }
  lr = warp_sum(lr);
  lc = warp_sum(lc);
  if (lane == 0 && v < batch) {
    atomicAdd(&loss[0], lr * inv_b);
    atomicAdd(&loss[1], lc * inv_b);
  }
}

// grad[j] = sum over the batch of Mt[j][:] (rows of a transposed BF16 matrix).
__global__ void row_sum_kernel(int N, int cols, const __nv_bfloat16* __restrict__ Mt, float* __restrict__ out) {
  const int j = blockIdx.x;
  if (j >= N) return;
  float s = 0.0f;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) s += __bfloat162float(Mt[(size_t)j * cols + c]);
  __shared__ float red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0f;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[j] = t;
  }
}

__global__ void adam_kernel(long long count, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 copies of a [rows][cols] FP32 weight: W (row-major) and optionally W^T.
__global__ void pack_kernel(int rows, int cols, const float* __restrict__ w, __nv_bfloat16* wb,
                            __nv_bfloat16* wt) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e % cols);
    const __nv_bfloat16 b = __float2bfloat16(w[e]);
    wb[e] = b;
    if (wt) wt[(size_t)c * rows + r] = b;
  }
}

struct RadiusArgs {
  int batch, DO, n, P, n_rx, n_tx;
  bool learned, order;
  int base_mode;
  double base_value;
  float alpha;
  const float* O;
  const double* nv;
  const float* R32;
  const float* yb32;
  float* r2;
};

// Initial r^2 per vector: sigma^2 exp(o_0) (learned) or the given base
// radius, capped (order) by the FP32 distance of the leaf x^ whose row r
// takes the PAM index of largest logit o[1 + r P + k] (ties to the lower k),
// scaled by 1 + 2^-16 so that x^ stays inside the sphere under the search's
// own FP32 evaluation.
// Eight lanes per vector (four vectors per warp): the group's lanes take
// the rows' argmaxes and residuals r = g, g + 8, ... (consecutive lanes read
// consecutive entries of each R column), and the distance is summed over the
// rows in order on every lane of the group, so that each residual is the same
// FMA chain (columns r..n-1) and the distance the same sum (rows 0..n-1) as
// one thread computing the whole vector.
constexpr int kRadiusLanes = 8;
constexpr int kRadiusMaxN = 2 * kFullFeaturesMaxTx;  // the ordering head's rows at most
constexpr int kRadiusThreads = 128;

__global__ void __launch_bounds__(kRadiusThreads) radius_kernel(RadiusArgs a) {
  constexpr int G = kRadiusLanes, RPL = kRadiusMaxN / G;
  __shared__ uint8_t xh_all[kRadiusThreads / G][kRadiusMaxN];
  const int lane = threadIdx.x & 31, gl = lane & (G - 1), lead = lane & ~(G - 1);
  const int grp = threadIdx.x / G;
  const int v = (blockIdx.x * kRadiusThreads + threadIdx.x) / G;
  const bool act = v < a.batch;
  const int vv = act ? v : 0;  // lanes past the batch follow along for the shuffles
  double r2;
  if (a.learned) r2 = a.nv[vv] * exp((double)a.O[(size_t)vv * a.DO]);
  else if (a.base_mode == RADIUS_PAPER) r2 = (double)a.n_rx * a.n_tx * a.nv[vv];
  else if (a.base_mode == RADIUS_VALUE) r2 = a.base_value;
  else r2 = INFINITY;
  if (a.order) {
    const int n = a.n, P = a.P;
    const float* o = a.O + (size_t)vv * a.DO;
    uint8_t* xh = xh_all[grp];
    for (int r = gl; r < n; r += G) {
      int best = 0;
      float bl = o[1 + r * P];
      for (int k = 1; k < P; ++k)
        if (o[1 + r * P + k] > bl) {
          bl = o[1 + r * P + k];
          best = k;
        }
      xh[r] = (uint8_t)best;
    }
    __syncwarp();
    const float* R = a.R32 + (size_t)vv * tri_stride32(n);
    const float* yb = a.yb32 + (size_t)vv * vec_stride32(n);
    float e[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int r = gl + G * t;
      e[t] = 0.0f;
      if (r < n) {
        float et = yb[r];
        for (int c = r; c < n; ++c) et = fmaf(-R[col_off(c) + r], (float)(2 * (int)xh[c] - (P - 1)) * a.alpha, et);
        e[t] = et;
      }
    }
    float d = 0.0f;
#pragma unroll
    for (int r = 0; r < kRadiusMaxN; ++r) {
      const float er = __shfl_sync(0xffffffffu, e[r / G], lead + (r % G));
      if (r < n) d = fmaf(er, er, d);
    }
    const double cap = (double)d * (1.0 + 1.0 / 65536.0);
    if (cap > 0.0 && cap < r2) r2 = cap;
  }
  if (act && gl == 0) a.r2[v] = (float)r2;
}

int grid_for(long long total, int threads) {
  long long g = (total + threads - 1) / threads;
  if (g > 65535 * 4) g = 65535 * 4;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

struct MlpState {
  int n = 0, P = 0, n_tx = 0, qam = 0, D0 = 0, DO = 0, cap = 0;
  bool reduced = false;  // summary features (n_tx > 32), radius head only
  long long count = 0, step = 0;
  // FP32 master parameters, gradients, Adam moments (same layout)
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  // BF16 weights (row-major [out][in]) and transposes used by the backward pass
  __nv_bfloat16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *W2t = nullptr, *W3t = nullptr;
  // activations for up to cap rows
  __nv_bfloat16 *X = nullptr, *Xt = nullptr, *H1 = nullptr, *H1t = nullptr, *H2 = nullptr, *H2t = nullptr;
  __nv_bfloat16 *dO = nullptr, *dOt = nullptr, *dH2 = nullptr, *dH2t = nullptr, *dH1 = nullptr, *dH1t = nullptr;
  float *O = nullptr, *r2 = nullptr, *loss = nullptr;
  int* err = nullptr;
  size_t bytes = 0;

  // offsets of each tensor inside the parameter vector
  size_t oW1() const { return 0; }
  size_t ob1() const { return (size_t)kH * D0; }
  size_t oW2() const { return ob1() + kH; }
  size_t ob2() const { return oW2() + (size_t)kH * kH; }
  size_t oW3() const { return ob2() + kH; }
  size_t ob3() const { return oW3() + (size_t)DO * kH; }
};

void mlp_dims(int n_tx, int qam, int* D0, int* DO) {
  const int n = 2 * n_tx;
  const int P = qam == 4 ? 2 : qam == 16 ? 4 : 8;
  if (n_tx > kFullFeaturesMaxTx) {
    *D0 = round_up(n + 3, 64);
    *DO = 128;
    return;
  }
  *D0 = round_up(n * (n + 1) / 2 + n + 1, 64);
  *DO = round_up(1 + n * P, 128);
}

long long mlp_count(int n_tx, int qam) {
  int D0, DO;
  mlp_dims(n_tx, qam, &D0, &DO);
  return (long long)kH * D0 + kH + (long long)kH * kH + kH + (long long)DO * kH + DO;
}

void mlp_free(MlpState* s) {
  if (!s) return;
  void* p[] = {s->w,  s->g,   s->m,  s->v,   s->W1,  s->W2,  s->W3,   s->W2t,  s->W3t, s->X,  s->Xt,
               s->H1, s->H1t, s->H2, s->H2t, s->dO,  s->dOt, s->dH2,  s->dH2t, s->dH1, s->dH1t, s->O,
               s->r2, s->loss, s->err};
  for (void* q : p)
    if (q) cudaFree(q);
  delete s;
}

cudaError_t mlp_alloc(MlpState** out, int n_tx, int qam, int cap) {
  MlpState* s = new MlpState();
  s->n_tx = n_tx;
  s->qam = qam;
  s->n = 2 * n_tx;
  s->reduced = n_tx > kFullFeaturesMaxTx;
  s->P = qam == 4 ? 2 : qam == 16 ? 4 : 8;
  mlp_dims(n_tx, qam, &s->D0, &s->DO);
  s->cap = round_up(cap, 128);
  s->count = mlp_count(n_tx, qam);
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t elems) {
    if (e != cudaSuccess) return;
    const size_t b = sizeof(**p) * (elems ? elems : 1);
    e = cudaMalloc(reinterpret_cast<void**>(p), b);
    if (e == cudaSuccess) {
      s->bytes += b;
      e = cudaMemset(*p, 0, b);
    }
  };
  const size_t C = s->cap, D0 = s->D0, DO = s->DO, H = kH;
  A(&s->w, s->count);
  A(&s->g, s->count);
  A(&s->m, s->count);
  A(&s->v, s->count);
  A(&s->W1, H * D0);
  A(&s->W2, H * H);
  A(&s->W3, DO * H);
  A(&s->W2t, H * H);
  A(&s->W3t, H * DO);
  A(&s->X, C * D0);
  A(&s->Xt, C * D0);
  A(&s->H1, C * H);
  A(&s->H1t, C * H);
  A(&s->H2, C * H);
  A(&s->H2t, C * H);
  A(&s->dO, C * DO);
  A(&s->dOt, C * DO);
  A(&s->dH2, C * H);
  A(&s->dH2t, C * H);
  A(&s->dH1, C * H);
  A(&s->dH1t, C * H);
  A(&s->O, C * DO);
  A(&s->r2, C);
  A(&s->loss, 2);
  A(&s->err, 1);
  if (e != cudaSuccess) {
    mlp_free(s);
    return e;
  }
  *out = s;
  return cudaSuccess;
}

cudaError_t mlp_pack(MlpState* s, cudaStream_t st) {
  const int D0 = s->D0, DO = s->DO;
  pack_kernel<<<grid_for((long long)kH * D0, 256), 256, 0, st>>>(kH, D0, s->w + s->oW1(), s->W1, nullptr);
  pack_kernel<<<grid_for((long long)kH * kH, 256), 256, 0, st>>>(kH, kH, s->w + s->oW2(), s->W2, s->W2t);
  pack_kernel<<<grid_for((long long)DO * kH, 256), 256, 0, st>>>(DO, kH, s->w + s->oW3(), s->W3, s->W3t);
  return cudaGetLastError();
}

// Features of the first `batch` vectors (QR outputs R32 / yb32 already in the
// workspace) into s->X (and s->Xt when `train`), zero rows up to rows.
cudaError_t mlp_features(MlpState* s, int batch, int rows, const float* R32, const float* yb32, const double* nv,
                         bool train, float* F, cudaStream_t st) {
  if (s->reduced) {
    const float alpha = (float)sqrt(3.0 / (2.0 * (s->qam - 1)));
    reduced_features_kernel<<<grid_for((long long)rows * 32, 256), 256, 0, st>>>(
        batch, rows, s->n, s->P, alpha, s->D0, R32, yb32, nv, s->X, train ? s->Xt : nullptr, F);
    return cudaGetLastError();
  }
  mlp_features_kernel<<<grid_for((long long)rows * 32, 256), 256, 0, st>>>(
      batch, rows, s->n, s->D0, R32, yb32, nv, s->X, train ? s->Xt : nullptr, F);
  return cudaGetLastError();
}

// Forward pass over `rows` rows of s->X (rows % 128 == 0); keeps H1, H2
// (and their transposes when `train`) and the FP32 outputs in s->O.
cudaError_t mlp_forward(MlpState* s, int rows, bool train, cudaStream_t st) {
  TcEpi e{};
  e.err = s->err;
  e.mode = TC_BIAS_RELU;
  e.bias = s->w + s->ob1();
  e.outb = s->H1;
  e.ldb = kH;
  e.outt = train ? s->H1t : nullptr;
  e.ldt = rows;
  cudaError_t r = tc_gemm(s->X, s->D0, s->W1, s->D0, rows, kH, s->D0, e, st);
  if (r != cudaSuccess) return r;
  e.bias = s->w + s->ob2();
  e.outb = s->H2;
  e.outt = train ? s->H2t : nullptr;
  r = tc_gemm(s->H1, kH, s->W2, kH, rows, kH, kH, e, st);
  if (r != cudaSuccess) return r;
  TcEpi o{};
  o.err = s->err;
  o.mode = TC_F32;
  o.bias = s->w + s->ob3();
  o.outf = s->O;
  o.ldf = s->DO;
  return tc_gemm(s->H2, kH, s->W3, kH, rows, s->DO, kH, o, st);
}

// Backward pass: loss gradient, activations' gradients, weight and bias
// gradients into s->g (FP32, parameter layout).
cudaError_t mlp_backward(MlpState* s, int batch, int rows, const double* ml_metric, const double* nv,
                         const uint8_t* ml_sym, cudaStream_t st) {
  cudaError_t r = cudaMemsetAsync(s->loss, 0, 2 * sizeof(float), st);
  if (r != cudaSuccess) return r;
  mlp_loss_kernel<<<(rows + 7) / 8, 256, 0, st>>>(batch, rows, s->n, s->P, s->n_tx, s->DO, s->O, ml_metric, nv,
                                                  ml_sym, 0.9f, 0.2f, s->reduced ? 0 : s->n, s->dO, s->dOt,
                                                  s->loss);
  if ((r = cudaGetLastError()) != cudaSuccess) return r;
  TcEpi e{};
  e.err = s->err;
  // dH2 = (dO W3) * [H2 > 0]
  e.mode = TC_MASK;
  e.mask = s->H2;
  e.ldm = kH;
  e.outb = s->dH2;
  e.ldb = kH;
  e.outt = s->dH2t;
  e.ldt = rows;
  if ((r = tc_gemm(s->dO, s->DO, s->W3t, s->DO, rows, kH, s->DO, e, st)) != cudaSuccess) return r;
  // dH1 = (dH2 W2) * [H1 > 0]
  e.mask = s->H1;
  e.outb = s->dH1;
  e.outt = s->dH1t;
  if ((r = tc_gemm(s->dH2, kH, s->W2t, kH, rows, kH, kH, e, st)) != cudaSuccess) return r;
  // weight gradients: dW3 = dO^T H2, dW2 = dH2^T H1, dW1 = dH1^T X (reductions over the batch)
  TcEpi f{};
  f.err = s->err;
  f.mode = TC_F32;
  f.outf = s->g + s->oW3();
  f.ldf = kH;
  if ((r = tc_gemm(s->dOt, rows, s->H2t, rows, s->DO, kH, rows, f, st)) != cudaSuccess) return r;
  f.outf = s->g + s->oW2();
  if ((r = tc_gemm(s->dH2t, rows, s->H1t, rows, kH, kH, rows, f, st)) != cudaSuccess) return r;
  f.outf = s->g + s->oW1();
  f.ldf = s->D0;
  if ((r = tc_gemm(s->dH1t, rows, s->Xt, rows, kH, s->D0, rows, f, st)) != cudaSuccess) return r;
  row_sum_kernel<<<s->DO, 256, 0, st>>>(s->DO, rows, s->dOt, s->g + s->ob3());
  row_sum_kernel<<<kH, 256, 0, st>>>(kH, rows, s->dH2t, s->g + s->ob2());
  row_sum_kernel<<<kH, 256, 0, st>>>(kH, rows, s->dH1t, s->g + s->ob1());
  return cudaGetLastError();
}

cudaError_t mlp_adam(MlpState* s, float lr, cudaStream_t st) {
  s->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)s->step), c2 = 1.0f - powf(b2, (float)s->step);
  adam_kernel<<<grid_for(s->count, 256), 256, 0, st>>>(s->count, s->w, s->g, s->m, s->v, lr, b1, b2, 1e-8f, c1, c2);
  cudaError_t r = cudaGetLastError();
  if (r != cudaSuccess) return r;
  return mlp_pack(s, st);
}

cudaError_t mlp_radius(MlpState* s, int batch, const double* nv, bool learned, bool order, int base_mode,
                       double base_value, int n_rx, const float* R32, const float* yb32, cudaStream_t st) {
  RadiusArgs a{};
  a.batch = batch;
  a.DO = s->DO;
  a.n = s->n;
  a.P = s->P;
  a.n_rx = n_rx;
  a.n_tx = s->n_tx;
  a.learned = learned;
  a.order = order;
  a.base_mode = base_mode;
  a.base_value = base_value;
  a.alpha = (float)sqrt(3.0 / (2.0 * (s->qam - 1)));
  a.O = s->O;
  a.nv = nv;
  a.R32 = R32;
  a.yb32 = yb32;
  a.r2 = s->r2;
  radius_kernel<<<(int)(((long long)batch * kRadiusLanes + kRadiusThreads - 1) / kRadiusThreads), kRadiusThreads, 0,
                  st>>>(a);
  return cudaGetLastError();
}

}  // namespace mdx

namespace mdx {
float* mlp_params(MlpState* s) { return s->w; }
float* mlp_grads(MlpState* s) { return s->g; }
float* mlp_outputs(MlpState* s) { return s->O; }
float* mlp_r2(MlpState* s) { return s->r2; }
float* mlp_loss(MlpState* s) { return s->loss; }
int* mlp_err(MlpState* s) { return s->err; }
int mlp_cap(MlpState* s) { return s->cap; }
int mlp_ntx(MlpState* s) { return s->n_tx; }
int mlp_qam(MlpState* s) { return s->qam; }
bool mlp_reduced(MlpState* s) { return s->reduced; }
size_t mlp_bytes(MlpState* s) { return s->bytes; }
}  // namespace mdx
