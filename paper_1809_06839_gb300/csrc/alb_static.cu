// alb_static.cu -- alb_apply_ragged_static: the per-transform ragged path for
// callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc or any allocating
// routine: code that runs inside a host allocator's callback, in a process
// whose device memory is fully pre-reserved by another framework, or in a
// real-time loop whose policy forbids allocation after start-up.  Those callers
// can still hand over their input and output images, but not a workspace.
// This entry point gives them the plain per-transform path with its scratch
// (work plan, per-image tables, per-image histograms) taken from one
// fixed-size array in device memory that belongs to the library.
//
// The array is a file-scope __device__ variable of kStaticScratchBytes bytes:
// every GPU that loads libalb.so holds it until the process exits.  Host code
// must not use the array's name as a device address (on the host it names a
// shadow object), so the first call on each device looks up the real device
// address with cudaGetSymbolAddress, with that device current, and caches it
// together with the id of the CUDA context it belongs to; a later call in a
// different context (after cudaDeviceReset) looks it up again.  A call that
// looks the address up does a runtime query, so the first call on a device
// (and the first after a reset) should happen before any stream capture.
// Every call shares the one array and leaves the last call's contents in it;
// calls whose kernels overlap on the GPU (different streams without
// ordering) race on it and must be serialised by the caller.
#include <mutex>

#include <cuda.h>

#include "alb_common.cuh"
#include "alb_kernels.cuh"

namespace alb {

constexpr int32_t kStaticMaxImages = 2048;
constexpr size_t kStaticScratchBytes = 8u << 20;   // 8 MiB
constexpr int32_t kStaticItemBytes = 16384;        // output bytes per work item

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
struct StaticAddr {
  void* addr;                  // device address of g_static_scratch
  unsigned long long ctx_id;   // the CUDA context it belongs to (0: unknown)
};
static StaticAddr g_static_addr[64] = {};

// Unique id of the calling thread's current CUDA context, 0 when there is
// none or the driver query is unavailable.  The driver functions are looked
// up through the runtime, so the library does not link the driver library.
static unsigned long long current_ctx_id() {
  typedef CUresult (*GetCurrentFn)(CUcontext*);
  typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetIdFn)f;
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of g_static_scratch in the current device's context, looked
// up once per context: a call after the context was destroyed and re-created
// (cudaDeviceReset) looks it up again instead of reusing a stale address.
static alb_status static_scratch(void** out) {
  int dev = -1;
  ALB_CUDA(cudaGetDevice(&dev));
  ALB_REQUIRE(dev >= 0 && dev < 64, ALB_EINVAL, "alb_apply_ragged_static: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  const unsigned long long id = current_ctx_id();
  StaticAddr& c = g_static_addr[dev];
  if (!c.addr || id == 0 || id != c.ctx_id) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return cuda_status(e, "cudaGetSymbolAddress(g_static_scratch)");
    c.addr = p;
    c.ctx_id = current_ctx_id();   // the lookup made the device's context current if it was not
  }
  *out = c.addr;
  return ALB_OK;
}

}  // namespace alb

using namespace alb;

extern "C" alb_status alb_apply_ragged_static(int32_t tid, int32_t n, const alb_params* params_dev,
                                              const alb_image* in_dev, const alb_image* out_dev,
                                              int32_t* dev_status, void* stream) {
  ALB_REQUIRE(tid >= ALB_HFLIP && tid <= ALB_ELASTIC && tid != ALB_CHAIN, ALB_EINVAL,
              "alb_apply_ragged_static: unknown transform id %d", tid);
  ALB_REQUIRE(n >= 0, ALB_EINVAL, "alb_apply_ragged_static: negative n");
  ALB_REQUIRE(n <= kStaticMaxImages, ALB_ECAPACITY,
              "alb_apply_ragged_static: %d images exceed the static scratch limit of %d images", n,
              kStaticMaxImages);
  if (n == 0) return ALB_OK;
  ALB_REQUIRE(params_dev && in_dev && out_dev, ALB_EINVAL, "alb_apply_ragged_static: null device array");
  void* base = nullptr;
  alb_status rc = static_scratch(&base);
  if (rc != ALB_OK) return rc;
  Carve cv{(char*)base, 0, kStaticScratchBytes};
  int32_t* prefix = cv.take<int32_t>(n + 1);
  int32_t* rpi = cv.take<int32_t>(n);
  uint8_t* luts = uses_lut(tid) ? cv.take<uint8_t>((size_t)n * 768) : nullptr;
  uint32_t* hist = tid == ALB_EQUALIZE ? cv.take<uint32_t>((size_t)n * 768) : nullptr;
  ALB_REQUIRE(prefix && rpi && (!uses_lut(tid) || luts) && (tid != ALB_EQUALIZE || hist), ALB_ECAPACITY,
              "alb_apply_ragged_static: %d images do not fit the %zu-byte static scratch", n, kStaticScratchBytes);
  cudaStream_t st = (cudaStream_t)stream;
  PrmList prm{params_dev, {}};
  ImgList li{in_dev, {}}, lo{out_dev, {}};
  // every scratch region is fully rewritten by the launches below (the plan by
  // k_plan, the tables by their build kernels, the histograms zeroed first),
  // so nothing left by an earlier call is read
  const PlanCheck chk{tid, 3, is_geometric(tid), li, prm, dev_status, 0};
  rc = launch_plan(lo, n, kStaticItemBytes, prefix, rpi, chk, st);
  if (rc != ALB_OK) return rc;
  Plan plan{prefix, rpi, n};
  return is_geometric(tid) ? launch_geometric(tid, plan, li, lo, prm, 3, false, dev_status, st)
                           : launch_photometric(tid, n, plan, li, lo, prm, luts, hist, dev_status, st);
}
