// alb_capi.cu -- the extern "C" entry points of libalb.so: argument checks,
// workspace carving and dispatch to the kernels.  Nothing here computes pixels.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "alb_common.cuh"
#include "alb_kernels.cuh"
#include "alb_bulk.cuh"

namespace alb {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

alb_status cuda_status(cudaError_t e, const char* what) {
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  return ALB_ECUDA;
}

int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 152;
  }
  return cache[dev];
}

constexpr int32_t kItemBytes = 16384;   // output bytes per work item (row block)

static void out_shape(const alb_params& p, int32_t h, int32_t w, int32_t& oh, int32_t& ow) {
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

static size_t ragged_ws(int32_t tid, int32_t n) {
  size_t b = 2 * plan_bytes(n) + 256;
  if (uses_lut(tid)) b += (size_t)n * 768 + 256;
  if (tid == ALB_EQUALIZE) b += (size_t)n * 768 * 4 + 256;
  return b;
}

static alb_status check_image(const alb_image* im, const char* what) {
  ALB_REQUIRE(im->h >= 0 && im->w >= 0 && im->c >= 1, ALB_ESHAPE, "%s: bad size %dx%dx%d", what, im->h, im->w, im->c);
  ALB_REQUIRE(im->row_stride >= (int64_t)im->w * im->c, ALB_ESHAPE, "%s: row_stride %lld < w*c", what,
              (long long)im->row_stride);
  ALB_REQUIRE(im->data || im->h == 0 || im->w == 0, ALB_EINVAL, "%s: null data", what);
  return ALB_OK;
}

// Shared body of alb_apply (inline single entry) and alb_apply_ragged (device arrays).
static alb_status run_ragged(int32_t tid, int32_t n, const PrmList& prm, const ImgList& in, const ImgList& out,
                             const ImgList* min_, const ImgList* mout, const float* boxes, const int32_t* nbox,
                             int32_t cap, int32_t single_n, float* bout, int32_t* nbout, void* ws, size_t ws_bytes,
                             int32_t* status, cudaStream_t st) {
  if (n == 0) return ALB_OK;
  Carve cv{(char*)ws, 0, ws_bytes};
  const bool geo = is_geometric(tid);
  int32_t* prefix = cv.take<int32_t>(n + 1);
  int32_t* rpi = cv.take<int32_t>(n);
  int32_t* mprefix = cv.take<int32_t>(n + 1);
  int32_t* mrpi = cv.take<int32_t>(n);
  uint8_t* luts = uses_lut(tid) ? cv.take<uint8_t>((size_t)n * 768) : nullptr;
  uint32_t* hist = tid == ALB_EQUALIZE ? cv.take<uint32_t>((size_t)n * 768) : nullptr;
  ALB_REQUIRE(prefix && rpi && mprefix && mrpi && (!uses_lut(tid) || luts) && (tid != ALB_EQUALIZE || hist),
              ALB_EWORKSPACE, "workspace of %zu bytes is smaller than the %zu required", ws_bytes, ragged_ws(tid, n));
  if (out.dev || out.one.data) {
    // ragged image slots are RGB; a single image (validated on the host) may have any c for geometric transforms
    const int32_t img_c = in.dev ? 3 : in.one.c;
    const PlanCheck chk{tid, img_c, geo, in, prm, status, 0};
    alb_status rc = launch_plan(out, n, kItemBytes, prefix, rpi, chk, st);
    if (rc != ALB_OK) return rc;
    // the mask plan's arrays serve as the image launch's second tile plan;
    // the mask plan is written after the image kernels (stream order)
    Plan plan{prefix, rpi, n, mprefix, mrpi};
    rc = geo ? launch_geometric(tid, plan, in, out, prm, img_c, false, status, st)
             : launch_photometric(tid, n, plan, in, out, prm, luts, hist, status, st);
    if (rc != ALB_OK) return rc;
  }
  if (min_ && mout) {
    // The masks' channel count is known on the host only for a single image;
    // a ragged launch runs two mask passes: single-channel masks through the
    // specialised kernels, every other mask through the general ones (each
    // pass's plan gives the other pass's masks no items).
    const int npass = mout->dev ? 2 : 1;
    for (int pass = 0; pass < npass; pass++) {
      const int32_t chans = mout->dev ? (pass == 0 ? 1 : 0) : mout->one.c;
      const int32_t filter = mout->dev ? (pass == 0 ? 1 : -1) : 0;
      const PlanCheck mchk{tid, 0, geo, *min_, prm, status, filter};
      alb_status rc = launch_plan(*mout, n, kItemBytes, mprefix, mrpi, mchk, st);
      if (rc != ALB_OK) return rc;
      Plan mplan{mprefix, mrpi, n};
      if (geo) {
        rc = launch_geometric(tid, mplan, *min_, *mout, prm, chans, true, status, st);
      } else {
        // photometric transforms leave masks unchanged: copy with an identity flip record
        PrmList ident{nullptr, {}};
        ident.one.tid = ALB_HFLIP;
        ident.one.apply = 0;
        rc = launch_geometric(ALB_HFLIP, mplan, *min_, *mout, ident, chans, true, status, st);
      }
      if (rc != ALB_OK) return rc;
    }
  }
  if (boxes && bout && nbout) {
    alb_status rc = launch_boxes(n, prm, in, boxes, nbox, cap, single_n, bout, nbout, status, st);
    if (rc != ALB_OK) return rc;
  }
  return ALB_OK;
}

}  // namespace alb

using namespace alb;

extern "C" const char* alb_last_error(void) { return g_err; }
extern "C" const char* alb_version(void) { return "alb 1.0 sm_103a"; }

extern "C" alb_status alb_output_shape(const alb_params* p, int32_t h, int32_t w, int32_t* out_h, int32_t* out_w) {
  ALB_REQUIRE(p && out_h && out_w, ALB_EINVAL, "alb_output_shape: null argument");
  ALB_REQUIRE(p->tid >= ALB_HFLIP && p->tid <= ALB_ELASTIC, ALB_EINVAL, "alb_output_shape: unknown id %d", p->tid);
  out_shape(*p, h, w, *out_h, *out_w);
  return ALB_OK;
}

extern "C" size_t alb_workspace_size(int32_t tid, int32_t n) { return n <= 0 ? 256 : ragged_ws(tid, n); }

extern "C" alb_status alb_apply(const alb_params* params, const alb_image* in, const alb_image* out,
                                const alb_image* mask_in, const alb_image* mask_out, const float* boxes_in,
                                int32_t n_boxes, float* boxes_out, int32_t* n_boxes_out, void* workspace,
                                size_t workspace_bytes, void* stream) {
  ALB_REQUIRE(params && in, ALB_EINVAL, "alb_apply: params and in are required");
  const alb_params& p = *params;
  ALB_REQUIRE(p.tid >= ALB_HFLIP && p.tid <= ALB_ELASTIC && p.tid != ALB_CHAIN, ALB_EINVAL,
              "alb_apply: unknown transform id %d", p.tid);
  alb_status rc = check_image(in, "alb_apply(in)");
  if (rc != ALB_OK) return rc;
  int32_t oh, ow;
  out_shape(p, in->h, in->w, oh, ow);
  const bool geo = is_geometric(p.tid);
  if (out) {
    rc = check_image(out, "alb_apply(out)");
    if (rc != ALB_OK) return rc;
    ALB_REQUIRE(out->h == oh && out->w == ow && out->c == in->c, ALB_ESHAPE,
                "alb_apply: output is %dx%dx%d, transform %d gives %dx%dx%d", out->h, out->w, out->c, p.tid, oh, ow,
                in->c);
    ALB_REQUIRE(geo || in->c == 3, ALB_EINVAL, "alb_apply: transform %d needs an RGB image (c == 3)", p.tid);
    ALB_REQUIRE(!(geo && out->data == in->data && in->h > 0), ALB_EINVAL,
                "alb_apply: in-place is not allowed for geometric transform %d", p.tid);
  }
  if (p.tid == ALB_RANDOM_CROP || p.tid == ALB_RESIZE || p.tid == ALB_RANDOM_SIZED_CROP ||
      p.tid == ALB_RANDOM_RESIZED_CROP) {
    ALB_REQUIRE(p.ch >= 1 && p.cw >= 1 && p.y0 >= 0 && p.x0 >= 0 && p.y0 + p.ch <= in->h && p.x0 + p.cw <= in->w,
                ALB_ESHAPE, "alb_apply: window (%d,%d,%d,%d) outside the %dx%d image", p.y0, p.x0, p.ch, p.cw,
                in->h, in->w);
  }
  if (p.tid == ALB_PAD_TO_SIZE)
    ALB_REQUIRE(p.out_h >= in->h && p.out_w >= in->w && p.y0 >= 0 && p.x0 >= 0, ALB_ESHAPE, "alb_apply: bad pad");
  if (mask_in || mask_out) {
    ALB_REQUIRE(mask_in && mask_out, ALB_EINVAL, "alb_apply: mask_in and mask_out go together");
    rc = check_image(mask_in, "alb_apply(mask_in)");
    if (rc != ALB_OK) return rc;
    rc = check_image(mask_out, "alb_apply(mask_out)");
    if (rc != ALB_OK) return rc;
    ALB_REQUIRE(mask_in->h == in->h && mask_in->w == in->w && mask_out->c == mask_in->c, ALB_ESHAPE,
                "alb_apply: mask does not match the image");
    ALB_REQUIRE(mask_out->h == (geo ? oh : in->h) && mask_out->w == (geo ? ow : in->w), ALB_ESHAPE,
                "alb_apply: mask output has the wrong size");
  }
  if (boxes_in || boxes_out || n_boxes_out)
    ALB_REQUIRE(boxes_in && boxes_out && n_boxes_out && n_boxes >= 0, ALB_EINVAL,
                "alb_apply: boxes_in, boxes_out and n_boxes_out go together");
  ALB_REQUIRE(!(boxes_in && p.tid == ALB_ELASTIC), ALB_EINVAL,
              "alb_apply: boxes are not defined for the elastic transform");
  if (p.tid == ALB_GRID_DISTORTION && p.apply)
    ALB_REQUIRE(p.k >= 1 && p.k <= 12, ALB_EINVAL, "alb_apply: grid distortion needs 1..12 cells, got %d", p.k);
  if (p.tid == ALB_ELASTIC && p.apply)
    ALB_REQUIRE(p.k >= 0 && p.k <= 131072 && p.cw >= 2 && p.cw <= 8, ALB_EINVAL,
                "alb_apply: elastic amplitude %d or lattice exponent %d out of range", p.k, p.cw);
  ALB_REQUIRE(workspace && workspace_bytes >= ragged_ws(p.tid, 1), ALB_EWORKSPACE,
              "alb_apply: workspace of %zu bytes is smaller than %zu", workspace_bytes, ragged_ws(p.tid, 1));
  PrmList prm{nullptr, p};
  ImgList li{nullptr, *in};
  ImgList lo{nullptr, out ? *out : alb_image{}};
  ImgList mi{nullptr, mask_in ? *mask_in : alb_image{}};
  ImgList mo{nullptr, mask_out ? *mask_out : alb_image{}};
  return run_ragged(p.tid, 1, prm, li, lo, mask_in ? &mi : nullptr, mask_out ? &mo : nullptr, boxes_in, nullptr,
                    n_boxes, n_boxes, boxes_out, n_boxes_out, workspace, workspace_bytes, nullptr,
                    (cudaStream_t)stream);
}

extern "C" alb_status alb_apply_ragged(int32_t tid, int32_t n, const alb_params* params_dev, const alb_image* in_dev,
                                       const alb_image* out_dev, const alb_image* mask_in_dev,
                                       const alb_image* mask_out_dev, const float* boxes_dev,
                                       const int32_t* n_boxes_dev, int32_t box_cap, float* boxes_out_dev,
                                       int32_t* n_boxes_out_dev, void* workspace, size_t workspace_bytes,
                                       int32_t* dev_status, void* stream) {
  ALB_REQUIRE(tid >= ALB_HFLIP && tid <= ALB_ELASTIC && tid != ALB_CHAIN, ALB_EINVAL,
              "alb_apply_ragged: unknown transform id %d", tid);
  ALB_REQUIRE(n >= 0, ALB_EINVAL, "alb_apply_ragged: negative n");
  if (n == 0) return ALB_OK;
  ALB_REQUIRE(params_dev && in_dev, ALB_EINVAL, "alb_apply_ragged: params and in are required");
  ALB_REQUIRE(!mask_in_dev == !mask_out_dev, ALB_EINVAL, "alb_apply_ragged: mask_in and mask_out go together");
  if (boxes_dev || boxes_out_dev || n_boxes_out_dev)
    ALB_REQUIRE(boxes_dev && n_boxes_dev && boxes_out_dev && n_boxes_out_dev && box_cap > 0, ALB_EINVAL,
                "alb_apply_ragged: box arrays go together and need box_cap > 0");
  ALB_REQUIRE(!(boxes_dev && tid == ALB_ELASTIC), ALB_EINVAL,
              "alb_apply_ragged: boxes are not defined for the elastic transform");
  ALB_REQUIRE(workspace && workspace_bytes >= ragged_ws(tid, n), ALB_EWORKSPACE,
              "alb_apply_ragged: workspace of %zu bytes is smaller than %zu", workspace_bytes, ragged_ws(tid, n));
  PrmList prm{params_dev, {}};
  ImgList li{in_dev, {}}, lo{out_dev, {}}, mi{mask_in_dev, {}}, mo{mask_out_dev, {}};
  return run_ragged(tid, n, prm, li, lo, mask_in_dev ? &mi : nullptr, mask_out_dev ? &mo : nullptr, boxes_dev,
                    n_boxes_dev, box_cap, 0, boxes_out_dev, n_boxes_out_dev, workspace, workspace_bytes, dev_status,
                    (cudaStream_t)stream);
}

extern "C" alb_status alb_selftest_bounded_wait(int32_t spins, const void* src_dev, void* out_dev,
                                                int32_t* dev_status, void* stream) {
  ALB_REQUIRE(spins >= 1 && (uint32_t)spins <= kMbarSpinLimit, ALB_EINVAL,
              "alb_selftest_bounded_wait: spins %d outside [1, %u]", spins, kMbarSpinLimit);
  ALB_REQUIRE(src_dev && out_dev && dev_status, ALB_EINVAL, "alb_selftest_bounded_wait: null argument");
  ALB_REQUIRE(((uintptr_t)src_dev & 15) == 0, ALB_EALIGN, "alb_selftest_bounded_wait: src must be 16-byte aligned");
  return launch_wait_selftest((uint32_t)spins, (const uint8_t*)src_dev, (uint8_t*)out_dev, dev_status,
                              (cudaStream_t)stream);
}

extern "C" alb_status alb_bounds_violations(uint32_t* count, uint32_t* first_line, int32_t reset, int32_t* checked) {
  ALB_REQUIRE(count && first_line && checked, ALB_EINVAL, "alb_bounds_violations: null argument");
#ifdef ALB_CHECK_BOUNDS
  *checked = 1;
#else
  *checked = 0;
#endif
  unsigned int c = 0, line = 0;
  alb_status rc = oob_resample(&c, &line, reset != 0);
  if (rc == ALB_OK) rc = oob_fused(&c, &line, reset != 0);
  if (rc == ALB_OK) rc = oob_geom(&c, &line, reset != 0);
  if (rc == ALB_OK) rc = oob_diff(&c, &line, reset != 0);
  *count = c;
  *first_line = line;
  return rc;
}
