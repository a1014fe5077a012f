// detect_kbest_noalloc: K-best detection without any device allocation.
//
// Some callers may not allocate device memory once they are running: a
// real-time receiver that reserves all of its memory at start-up and forbids
// allocation on the data path, or a process whose device memory is already
// held by another allocator.  They cannot create an mdx_ctx (mdx_create
// allocates its workspace), so this entry point runs the same QR and K-best
// kernels as detect_kbest with their scratch (the QR outputs R and ybar in
// FP64 and FP32, the per-vector singular flags and the work counter) placed
// in one statically sized device array that is part of the library itself.
//
// Costs and rules of that choice:
//   - the array (MDX_NOALLOC_SCRATCH_BYTES) is reserved on every GPU that
//     loads the library, until the process exits;
//   - sizes whose scratch does not fit are rejected with MDX_EUNSUPPORTED;
//   - all calls share the array: two calls whose work overlaps on the GPU
//     (different streams, or several host threads) race and corrupt each
//     other's results; serialise them on one stream;
//   - the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     before any stream capture begins.  The address is kept for the life of
//     the process, so a device reset (cudaDeviceReset) between calls is not
//     supported: it unloads the module and the kept address goes stale.
#include <math.h>

#include <mutex>

#include "mdx_internal.cuh"

namespace {

using namespace mdx;

// The scratch array.  In host code `g_noalloc_scratch` only names a host-side
// stand-in; kernels must be given the device address looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MDX_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (current), looked up once.
cudaError_t scratch_address(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[device];
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int pam_of(int qam) { return qam == 4 ? 2 : qam == 16 ? 4 : qam == 64 ? 8 : -1; }

bool on_device(const void* p, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == device);
}

}  // namespace

extern "C" mdx_status detect_kbest_noalloc(const mdx_params* p, int batch, const double* H,
                                           const double* y, const double* noise_var, uint8_t* sym_out,
                                           double* metric_out, int32_t* vstatus, int64_t* stats,
                                           void* stream) {
  if (!p || batch < 0) return MDX_EINVAL;
  if (batch == 0) return MDX_OK;
  const int M = p->n_tx, N = p->n_rx, P = pam_of(p->qam);
  if (M < 1 || N < M || P < 0) return MDX_EINVAL;
  if (M > MDX_MAX_TX || N > MDX_MAX_RX) return MDX_EUNSUPPORTED;
  if (p->K < 1 || p->K > MDX_MAX_K) return MDX_EINVAL;
  const double r0 = p->init_radius_sq;
  if (isnan(r0) || r0 == 0.0) return MDX_EINVAL;
  // the flags detect_kbest itself rejects, plus host buffers (which need the
  // context's staging buffers)
  if (p->flags & (MDX_HOST_BUFFERS | MDX_LEARNED_RADIUS | MDX_LEARNED_ORDER | MDX_ORDER_NATURAL))
    return MDX_EUNSUPPORTED;
  const int radius_mode = isinf(r0) ? (r0 > 0 ? RADIUS_NONE : RADIUS_PAPER) : (r0 < 0 ? RADIUS_PAPER : RADIUS_VALUE);
  if (radius_mode == RADIUS_PAPER && !noise_var) return MDX_EINVAL;
  if (!H || !y || !sym_out || !metric_out || !vstatus) return MDX_EINVAL;
  if ((reinterpret_cast<uintptr_t>(H) & 15u) || (reinterpret_cast<uintptr_t>(y) & 15u)) return MDX_EINVAL;
  const int n = 2 * M;
  // the same shared-memory check as detect_kbest, before anything is enqueued
  if (kbest_smem_bytes(n, p->K, P, (p->flags & MDX_COMPLEX_TREE) != 0) > 227 * 1024) return MDX_EUNSUPPORTED;

  // scratch layout: R64 | yb64 | R32 | yb32 | singular | work counter
  const size_t B = (size_t)batch;
  size_t off = 0;
  const size_t oR64 = off;
  off = align256(off + sizeof(double) * B * tri_stride64(n));
  const size_t oy64 = off;
  off = align256(off + sizeof(double) * B * vec_stride64(n));
  const size_t oR32 = off;
  off = align256(off + sizeof(float) * B * tri_stride32(n));
  const size_t oy32 = off;
  off = align256(off + sizeof(float) * B * vec_stride32(n));
  const size_t osing = off;
  off = align256(off + sizeof(int) * B);
  const size_t octr = off;
  off = align256(off + sizeof(unsigned int));
  if (off > (size_t)MDX_NOALLOC_SCRATCH_BYTES) return MDX_EUNSUPPORTED;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    cudaGetLastError();
    return MDX_ECUDA;
  }
  const void* ptrs[] = {H, y, sym_out, metric_out, vstatus};
  for (const void* q : ptrs)
    if (!on_device(q, device)) return MDX_EINVAL;
  if (noise_var && !on_device(noise_var, device)) return MDX_EINVAL;
  if (stats && !on_device(stats, device)) return MDX_EINVAL;

  unsigned char* base = nullptr;
  if (scratch_address(device, &base) != cudaSuccess) {
    cudaGetLastError();
    return MDX_ECUDA;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return MDX_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  QrOut q{reinterpret_cast<double*>(base + oR64), reinterpret_cast<double*>(base + oy64),
          reinterpret_cast<float*>(base + oR32), reinterpret_cast<float*>(base + oy32), nullptr, nullptr,
          reinterpret_cast<int*>(base + osing)};
  if (launch_qr(batch, N, M, H, y, q, s) != cudaSuccess) return MDX_ECUDA;

  SearchArgs a{};
  a.batch = batch;
  a.n = n;
  a.P = P;
  a.n_rx = N;
  a.n_tx = M;
  a.alpha64 = sqrt(3.0 / (2.0 * (p->qam - 1)));
  a.alpha = (float)a.alpha64;
  a.R32 = q.R32;
  a.yb32 = q.yb32;
  a.R64 = q.R64;
  a.yb64 = q.yb64;
  a.singular = q.singular;
  a.noise_var = noise_var;
  a.radius_mode = radius_mode;
  a.radius_value = r0;
  a.K = p->K;
  a.flags = p->flags;
  a.work_counter = reinterpret_cast<unsigned int*>(base + octr);
  a.sym_out = sym_out;
  a.metric_out = metric_out;
  a.vstatus = vstatus;
  a.stats = stats;
  // the work counter keeps the previous call's value: it must start at zero
  if (cudaMemsetAsync(a.work_counter, 0, sizeof(unsigned int), s) != cudaSuccess) return MDX_ECUDA;
  const cudaError_t e = launch_kbest(a, sms, s);
  if (e == cudaErrorInvalidConfiguration) return MDX_EUNSUPPORTED;
  return e == cudaSuccess ? MDX_OK : MDX_ECUDA;
}
