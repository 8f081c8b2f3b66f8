// bl_moments_noalloc: the per-bunch moment reduction of bl_moments without
// any device allocation. The paper has no counterpart; this entry point
// exists for callers that must not allocate device memory themselves or let
// the library do it: code running under a framework whose caching allocator
// owns all device memory, hard real-time or embedded callers that reserve
// every byte up front, and callers that cannot afford cudaMalloc/cudaFree's
// implicit device synchronisation in the middle of their pipeline.
//
// The per-block partial sums live in a fixed, file-scope device array
// (g_noalloc_scratch below, BL_NOALLOC_SCRATCH_SLOTS slots of 28 doubles,
// about 7.3 MB). Every GPU that loads this library holds that array until the
// process exits. Host code never uses the array's name as an address: the
// device address is looked up with cudaGetSymbolAddress once per device and
// context (again after a cudaDeviceReset, which reloads the module).
#include <mutex>

#include <cuda.h>

#include "runtime.h"

namespace {

constexpr int64_t SLOTS = BL_NOALLOC_SCRATCH_SLOTS;

static __device__ __align__(256) double g_noalloc_scratch[SLOTS * 28];

// Device addresses of g_noalloc_scratch per device, with the context they
// were looked up in: a new context (after cudaDeviceReset) means a reloaded
// module and a new address.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};
void *g_ctx[MAX_DEVICES] = {};

// The current driver context, through the runtime's driver entry point (no
// link against libcuda); NULL if the entry point is unavailable.
void *current_context() {
  using GetCtx = CUresult (*)(CUcontext *);
  static GetCtx fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<GetCtx>(f);
  }();
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return reinterpret_cast<void *>(c);
}

// out must be memory the GPU can store to with this very pointer: device or
// managed memory, or page-locked host memory mapped at the same address.
bool device_writable(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error the failed query leaves behind
    return false;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

}  // namespace

extern "C" bl_status bl_moments_noalloc(const bl_bunch *b, double *out, bl_stream stream) {
  using namespace bl;
  std::string why;
  BL_CHECK(bunch_dims_ok(b, &why), why);
  BL_CHECK(out, "out is NULL");
  BL_CHECK(device_writable(out),
           "out is not device-accessible memory (device, managed or mapped page-locked host)");
  const int64_t slots = stream_slots(b->n, b->n_bunch);
  if (slots > SLOTS)
    return set_error(BL_ERR_INVALID_ARG,
                     "bl_moments_noalloc: blocks + bunches exceed the fixed scratch of " +
                         std::to_string((long long)SLOTS) +
                         " slots (at most about SLOTS*4096 particles); use bl_moments");
  int dev = -1;
  BL_CUDA(cudaGetDevice(&dev));
  BL_CHECK(dev >= 0 && dev < MAX_DEVICES, "device index out of range for bl_moments_noalloc");
  int major = 0, minor = 0;
  BL_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  BL_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
  if (!(major == 10 && minor == 3))
    return set_error(BL_ERR_UNSUPPORTED_ARCH, "this library is built for sm_103a (GB300)");
  void *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    void *ctx = current_context();
    if (!g_addr[dev] || g_ctx[dev] != ctx) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
      g_addr[dev] = p;
      g_ctx[dev] = ctx;
    }
    scratch = g_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t *off = b->n_bunch > 1 ? b->offsets_dev : nullptr;
  double *partials = static_cast<double *>(scratch);
  // Every slot that the finalize step reads is written earlier in the same
  // call by the block that owns it, so nothing has to be cleared first.
  int64_t unit = 0;
  if (b->dtype == BL_F32) {
    Soa<float> z = soa_of<float>(b);
    BL_CUDA(launch_stream<float>(z, z, b->n, off, b->n_bunch, nullptr, 0, nullptr, false, true,
                                 partials, st, &unit));
  } else {
    Soa<double> z = soa_of<double>(b);
    BL_CUDA(launch_stream<double>(z, z, b->n, off, b->n_bunch, nullptr, 0, nullptr, false, true,
                                  partials, st, &unit));
  }
  BL_CUDA(launch_moments_finalize(partials, off, b->n_bunch, b->n, unit, out, nullptr, st));
  return BL_OK;
}
