// bsort_sort_records_noalloc: the whole record sort (bucket by length, sort
// every bucket, gather) for callers that may not allocate device memory.
//
// Some callers cannot hand the library a workspace: their device memory is
// owned by a host framework's own pool or arena that forbids raw cudaMalloc
// (plugins of inference servers, game engines), or they run latency-bound
// loops where cudaMalloc / cudaFree, which may synchronise the device, are not
// acceptable.  For them this entry point keeps its scratch in the file-scope
// array below, which the CUDA runtime places in device memory when the module
// loads; every GPU that loads the library holds it until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call clears the part that must start at zero (the status
// header) itself.  Calls whose work overlaps on the GPU (two streams, or two
// host threads) race on the array and give undefined results: serialise them.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace bsort {

namespace {

// Most words one call may sort (any W up to 32); the array holds the
// workspace layout for this many 32-byte records.
constexpr uint32_t kNoAllocMaxWords = 32768;
constexpr size_t kNoAllocBytes = ws_layout(kNoAllocMaxWords, kMaxW).total;

__device__ __align__(256) uint8_t g_noalloc_ws[kNoAllocBytes];

std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (0 if there is none
// or the driver cannot say).  The driver functions are reached through the
// runtime's entry-point query, so the library needs no link to the driver.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {  // called with g_mu held
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    resolved = true;
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of g_noalloc_ws on the current device, set up once per
// device and context.  In host code the array's name is only a host-side
// stand-in, so the address must come from cudaGetSymbolAddress with that
// device current.  The address belongs to the context the module was loaded
// in: after cudaDeviceReset the device gets a new primary context (with a new
// id), and the address is looked up again instead of reusing a stale one.
cudaError_t noalloc_ptr(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_dev_ptr[dev] || ctx == 0 || ctx != g_ctx_id[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_ws);  // also makes the context current
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = p;
    g_ctx_id[dev] = current_context_id();
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

__global__ void noalloc_status_kernel(const WsHeader* hdr, int32_t* status) {
  const uint32_t f = hdr->status_flags;
  int32_t c = 0;
  for (int k = 1; k < 32; ++k)
    if (f & (1u << k)) {
      c = k;
      break;
    }
  *status = c;
}

}  // namespace

}  // namespace bsort

using namespace bsort;

extern "C" bsort_status bsort_sort_records_noalloc(const uint8_t* d_rec, const uint8_t* d_len,
                                                   uint32_t n, uint32_t W, bsort_alg alg,
                                                   const bsort_tune* tune, uint8_t* d_out_rec,
                                                   uint32_t* d_out_perm, uint32_t* d_off,
                                                   int32_t* d_status, cudaStream_t s) {
  if (W < 8 || W > kMaxW || W % 8 || !d_off) return BSORT_E_INVALID;
  if (alg != BSORT_ODD_EVEN && alg != BSORT_MERGE && alg != BSORT_AUTO) return BSORT_E_INVALID;
  if (n > kNoAllocMaxWords) return BSORT_E_CAPACITY;
  if (n && (!d_rec || !d_len || !d_out_rec || !d_out_perm)) return BSORT_E_INVALID;
  if (n && ((reinterpret_cast<uintptr_t>(d_rec) | reinterpret_cast<uintptr_t>(d_out_rec)) & 15u))
    return BSORT_E_INVALID;
  // Same knobs and defaults as bsort_sort_records.
  SortParams p;
  if (!resolve_params(alg, tune, W, &p)) return BSORT_E_INVALID;

  void* ws_ptr = nullptr;
  if (noalloc_ptr(&ws_ptr) != cudaSuccess) return BSORT_E_CUDA;
  const Ws ws = ws_view(ws_ptr, kNoAllocBytes, W);
  // the header (status word, per-bucket buffer flags) must start at zero
  if (cudaMemsetAsync(ws_ptr, 0, 4096, s) != cudaSuccess) return BSORT_E_CUDA;
  cudaError_t e = launch_bucket(d_rec, d_len, n, nullptr, W, d_off, ws, s);
  if (e == cudaSuccess) e = launch_sort(n, W, p, d_off, ws, s);
  if (e == cudaSuccess) e = launch_gather(n, nullptr, W, d_off, ws, d_out_rec, d_out_perm, s);
  if (e == cudaSuccess && d_status) {
    noalloc_status_kernel<<<1, 1, 0, s>>>(ws.hdr, d_status);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? BSORT_OK : BSORT_E_CUDA;
}
