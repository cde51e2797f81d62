// alb_common.cuh -- internal helpers shared by the libalb kernels (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "alb.h"

static_assert(sizeof(alb_image) == 32, "alb_image layout");
static_assert(sizeof(alb_params) == 232, "alb_params layout");
static_assert(sizeof(alb_sample_cfg) == 88, "alb_sample_cfg layout");
static_assert(sizeof(alb_chain_cfg) == 72, "alb_chain_cfg layout");

#define ALB_HD __host__ __device__ __forceinline__
#define ALB_D __device__ __forceinline__

namespace alb {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
alb_status cuda_status(cudaError_t e, const char* what);
#define ALB_CUDA(call)                                              \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ::alb::cuda_status(e_, #call);    \
  } while (0)
#define ALB_REQUIRE(cond, code, ...)                                \
  do {                                                              \
    if (!(cond)) { ::alb::set_error(__VA_ARGS__); return (code); }  \
  } while (0)

int sm_count();     // SMs of the current device (cached per device)

// record the first device-side error in the caller's status word
ALB_D void dev_fail(int32_t* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ bounds-checked build
// Compiled with -DALB_CHECK_BOUNDS (build.build(check_bounds=True)), ALB_IN(cond)
// tests an index or address against the region it must stay in: when it
// fails, the source line of the first failing check and a count go to this
// translation unit's device counters and the guarded access is skipped (no
// trap, no fault); alb_bounds_violations reads the counters of every unit.
// In the normal build ALB_IN(cond) is `true` and costs nothing.
#ifdef ALB_CHECK_BOUNDS
static __device__ unsigned int g_alb_oob[2];   // count, first failing line
ALB_D bool alb_in_check(bool ok, int line) {
  if (!ok) {
    if (atomicAdd(&g_alb_oob[0], 1u) == 0u) g_alb_oob[1] = (unsigned)line;
  }
  return ok;
}
#define ALB_IN(cond) (::alb::alb_in_check((cond), __LINE__))
// per translation unit: read (and optionally clear) its counters
#define ALB_OOB_ACCESSOR(fname)                                                   \
  alb_status fname(unsigned int* count, unsigned int* line, bool reset) {         \
    unsigned int h[2] = {0u, 0u};                                                 \
    ALB_CUDA(cudaMemcpyFromSymbol(h, g_alb_oob, sizeof(h)));                     \
    if (reset) {                                                                  \
      const unsigned int z[2] = {0u, 0u};                                         \
      ALB_CUDA(cudaMemcpyToSymbol(g_alb_oob, z, sizeof(z)));                     \
    }                                                                             \
    *count += h[0];                                                               \
    if (!*line && h[1]) *line = h[1];                                             \
    return ALB_OK;                                                                \
  }
#else
#define ALB_IN(cond) (true)
#define ALB_OOB_ACCESSOR(fname) \
  alb_status fname(unsigned int*, unsigned int*, bool) { return ALB_OK; }
#endif

// a byte range [p, p + len) inside [base - slack, base + bytes + slack)
ALB_D bool bytes_within(const void* p, int64_t len, const void* base, int64_t bytes, int64_t slack = 0) {
  const intptr_t a = reinterpret_cast<intptr_t>(p), b = reinterpret_cast<intptr_t>(base);
  return a >= b - slack && a + len <= b + bytes + slack;
}
// the byte extent of an image: its first byte to its last pixel's last byte
ALB_D int64_t image_bytes(const alb_image& im) {
  return im.h > 0 && im.w > 0 ? (int64_t)(im.h - 1) * im.row_stride + (int64_t)im.w * im.c : 0;
}

// ------------------------------------------------------------------ integer helpers
ALB_HD int64_t floor_div(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b, r = a % b;
  return (r < 0) ? q - 1 : q;
}

// reflect-101 border (edge sample not repeated), any integer i, n >= 1
ALB_HD int32_t reflect101(int64_t i, int32_t n) {
  if (i >= 0 && i < n) return (int32_t)i;
  if (n == 1) return 0;
  if (i < 0 && i > -(int64_t)n) return (int32_t)(-i);                       // one fold at the left edge
  if (i >= n && i < 2 * (int64_t)n - 1) return (int32_t)(2 * (int64_t)(n - 1) - i);  // one fold at the right edge
  int64_t period = 2 * (int64_t)(n - 1);
  int64_t m = i % period;
  if (m < 0) m += period;
  if (m >= n) m = period - m;
  return (int32_t)m;
}

ALB_HD int32_t imin(int32_t a, int32_t b) { return a < b ? a : b; }
ALB_HD int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }

// ------------------------------------------------------------------ batch views
// A ragged batch: either device arrays (ptr != nullptr) or one inline entry
// passed by value (single-image alb_apply), so that no host->device copy is
// needed for the single-image call.
struct ImgList {
  const alb_image* dev;
  alb_image one;
  ALB_D alb_image get(int i) const { return dev ? dev[i] : one; }
};
struct PrmList {
  const alb_params* dev;
  alb_params one;
  ALB_D const alb_params& get(int i) const { return dev ? dev[i] : one; }
};

// Work plan of a ragged launch: image b owns items [prefix[b], prefix[b+1]);
// each item covers rows_per_item[b] output rows.
struct Plan {
  const int32_t* prefix;        // n + 1
  const int32_t* rows_per_item; // n
  int32_t n;
  // optional second tile plan ([n + 1], [n]), free for the image launch: the
  // resizes route their reductions through it (see launch_tile_geometric)
  int32_t* prefix2 = nullptr;
  int32_t* rows2 = nullptr;
};

// Blocked distribution of the plan's items over the grid: CTA j takes a
// contiguous range, so consecutive items mostly belong to the same image.
ALB_D void item_range(const Plan& p, int32_t& begin, int32_t& end) {
  int64_t total = p.prefix[p.n];
  begin = (int32_t)(total * blockIdx.x / gridDim.x);
  end = (int32_t)(total * (blockIdx.x + 1) / gridDim.x);
}

// image owning `item` (largest b with prefix[b] <= item)
ALB_D int32_t item_image(const Plan& p, int32_t item) {
  int32_t lo = 0, hi = p.n - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (p.prefix[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Walks the CTA's item range as runs of consecutive items of one image and
// calls f(b, r0, r1) once per run: output rows [r0, r1) of image b (r1 is not
// yet clamped to the image height).  A run is CTA-uniform, so f may hold
// block barriers.  Long runs let the streaming loops keep several vector
// loads in flight per thread instead of restarting every ~16 KB item.
template <class F>
ALB_D void for_each_run(const Plan& p, F&& f) {
  int32_t it0, it1;
  item_range(p, it0, it1);
  if (it0 >= it1) return;
  int32_t b = item_image(p, it0);
  for (int32_t item = it0; item < it1;) {
    while (item >= p.prefix[b + 1]) b++;
    const int32_t end = p.prefix[b + 1] < it1 ? p.prefix[b + 1] : it1;
    const int32_t rb = p.rows_per_item[b];
    f(b, (item - p.prefix[b]) * rb, (end - p.prefix[b]) * rb);
    item = end;
  }
}

// ------------------------------------------------------------------ workspace carving
struct Carve {
  char* base;
  size_t used, cap;
  template <class T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    return (used <= cap && base) ? reinterpret_cast<T*>(base + off) : nullptr;
  }
};

constexpr size_t plan_bytes(int32_t n) { return 256 + ((size_t)(n + 1) * 4 + 255) / 256 * 256 + ((size_t)n * 4 + 255) / 256 * 256 + 256; }

// Output size of a parameter record applied to an h x w input (C-ABI rules).
ALB_HD void record_out_shape(const alb_params& p, int32_t h, int32_t w, int32_t& oh, int32_t& ow) {
  oh = h; ow = w;
  switch (p.tid) {
    case ALB_RANDOM_CROP: case ALB_PAD_TO_SIZE: case ALB_RESIZE: case ALB_RANDOM_SIZED_CROP:
    case ALB_RANDOM_RESIZED_CROP: case ALB_CHAIN:
      oh = p.out_h; ow = p.out_w; break;
    case ALB_TRANSPOSE: oh = w; ow = h; break;
    case ALB_ROT90: if (p.apply && (p.k & 1)) { oh = w; ow = h; } break;
    default: break;
  }
}

// Per-image consistency of a ragged launch, checked on the device before any
// pixel is touched: 0, or the alb_status of the first violation.  want_c = 3
// for RGB image slots, 0 for masks (any c, equal in and out); geometric =
// whether the output follows the record's geometry (masks of photometric
// transforms keep the input size).
ALB_D int check_image_pair(int32_t tid, const alb_params& p, const alb_image& si, const alb_image& so,
                           int32_t want_c, bool geometric) {
  if (p.tid != tid) return ALB_EINVAL;
  if (si.c != so.c || si.c < 1 || (want_c && si.c != want_c)) return ALB_EINVAL;
  if (si.h < 0 || si.w < 0 || so.h < 0 || so.w < 0) return ALB_ESHAPE;
  if (si.row_stride < (int64_t)si.w * si.c || so.row_stride < (int64_t)so.w * so.c) return ALB_ESHAPE;
  int32_t oh = si.h, ow = si.w;
  if (geometric) record_out_shape(p, si.h, si.w, oh, ow);
  if (oh != so.h || ow != so.w) return ALB_ESHAPE;
  if (geometric && (tid == ALB_RANDOM_CROP || tid == ALB_RESIZE || tid == ALB_RANDOM_SIZED_CROP ||
                    tid == ALB_RANDOM_RESIZED_CROP)) {
    if (p.ch < 1 || p.cw < 1 || p.y0 < 0 || p.x0 < 0 || p.y0 + p.ch > si.h || p.x0 + p.cw > si.w) return ALB_ESHAPE;
    if (tid == ALB_RANDOM_CROP && (p.ch != so.h || p.cw != so.w)) return ALB_ESHAPE;
  }
  if (geometric && tid == ALB_PAD_TO_SIZE && (p.y0 < 0 || p.x0 < 0 || p.y0 + si.h > so.h || p.x0 + si.w > so.w))
    return ALB_ESHAPE;
  if (geometric && tid == ALB_GRID_DISTORTION && p.apply) {
    if (p.k < 1 || p.k > 12) return ALB_EINVAL;
    for (int j = 0; j < p.k; j++)
      if (((uint64_t)p.q[j >> 2] >> (16 * (j & 3)) & 0xFFFFu) == 0 ||
          ((uint64_t)p.q[(12 + j) >> 2] >> (16 * ((12 + j) & 3)) & 0xFFFFu) == 0)
        return ALB_EINVAL;
  }
  if (geometric && tid == ALB_ELASTIC && p.apply && (p.k < 0 || p.k > 131072 || p.cw < 2 || p.cw > 8))
    return ALB_EINVAL;
  return 0;
}

// Host launchers for the plan kernels (alb_geom.cu).  Images that fail
// check_image_pair get no work items and record their status.
struct PlanCheck {
  int32_t tid, want_c;
  bool geometric;
  ImgList in;
  PrmList prm;
  int32_t* status;
  int32_t filter_c;   // 0: all images; k > 0: only images with c == k; k < 0: only c != -k (others: no items, no error)
  int32_t reduce = 0; // resizes: 0 all images; else only one scale class: 2 windows no larger than the
                      // output, 1 reductions that fit the 66 x 34 box of 32 x 16 tiles, 3 the stronger ones
};

ALB_D bool plan_filtered_out(const PlanCheck& chk, const alb_image& im) {
  return (chk.filter_c > 0 && im.c != chk.filter_c) || (chk.filter_c < 0 && im.c == -chk.filter_c);
}
alb_status launch_plan(const ImgList& out, int32_t n, int32_t target_bytes, int32_t* prefix,
                       int32_t* rows_per_item, const PlanCheck& chk, cudaStream_t st);

}  // namespace alb
