// alb_color.cu -- photometric transforms (Table I: Brightness, ShiftHSV,
// ShiftRGB, Gamma, Grayscale; Sec. II and Fig. 1: colour, contrast and
// brightness transforms) and per-channel histogram equalisation.
//
// LUT transforms run in two launches: k_build_luts computes each image's
// three 256-entry tables once in float64 (the tables are the exact rounding
// points of the definition), then k_apply_lut streams the pixels through a
// copy of the table held in shared memory.  Equalize adds k_histogram
// (per-CTA shared-memory histograms, one global merge per item) and builds its
// tables from the histograms with a 256-bin block scan.
#include "alb_common.cuh"
#include "alb_kernels.cuh"

namespace alb {

ALB_D uint8_t sat_rne(double v) {
  double r = rint(v);
  r = r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r);
  return (uint8_t)r;
}

ALB_D uint8_t sat_rne_f(float v) {
  float r = rintf(v);
  r = r < 0.0f ? 0.0f : (r > 255.0f ? 255.0f : r);
  return (uint8_t)r;
}

// round(num / den) half to even, num >= 0, den > 0
ALB_D uint64_t rne_div_u64(uint64_t num, uint64_t den) {
  uint64_t q = num / den, r = num - q * den;
  if (2 * r > den || (2 * r == den && (q & 1))) q++;
  return q;
}

// ------------------------------------------------------------------ LUT build
// One CTA of 256 threads per image; thread v fills entry v of the 3 tables.
__global__ void __launch_bounds__(256) k_build_luts(int32_t n, PrmList prm, uint8_t* __restrict__ luts) {
  const int b = blockIdx.x;
  if (b >= n) return;
  const alb_params& p = prm.get(b);
  const int v = threadIdx.x;
  const double x = (double)v;
  uint8_t* L = luts + (int64_t)b * 768;
  if (!p.apply) {
    L[v] = L[256 + v] = L[512 + v] = (uint8_t)v;
    return;
  }
  switch (p.tid) {
    case ALB_BRIGHTNESS: { const uint8_t o = sat_rne(x + p.beta); L[v] = L[256 + v] = L[512 + v] = o; break; }
    case ALB_CONTRAST: { const uint8_t o = sat_rne(p.alpha * x); L[v] = L[256 + v] = L[512 + v] = o; break; }
    case ALB_BRIGHTNESS_CONTRAST: {
      const double g = p.alpha * x;
      const uint8_t o = sat_rne(g + p.beta);
      L[v] = L[256 + v] = L[512 + v] = o;
      break;
    }
    case ALB_GAMMA: {
      const double r = x / 255.0;
      const uint8_t o = sat_rne(255.0 * pow(r, p.gamma));
      L[v] = L[256 + v] = L[512 + v] = o;
      break;
    }
    case ALB_SHIFT_RGB:
      for (int c = 0; c < 3; c++) L[256 * c + v] = sat_rne(x + p.shift[c]);
      break;
    default:
      L[v] = L[256 + v] = L[512 + v] = (uint8_t)v;
  }
}

// Equalize tables from per-image histograms hist[b][3][256]:
// LUT[v] = round_half_even(255 (cdf[v] - m) / (N - m)), m = count of the
// lowest occupied level; constant channel -> identity.
__global__ void __launch_bounds__(256) k_equalize_luts(int32_t n, PrmList prm, const uint32_t* __restrict__ hist,
                                                       uint8_t* __restrict__ luts) {
  __shared__ uint32_t wsum[8];
  __shared__ uint32_t first_count, total;
  __shared__ int32_t first_level;
  const int b = blockIdx.x;
  if (b >= n) return;
  const alb_params& p = prm.get(b);
  const int v = threadIdx.x, lane = v & 31, wid = v >> 5;
  for (int c = 0; c < 3; c++) {
    const uint32_t h = hist[((int64_t)b * 3 + c) * 256 + v];
    uint32_t s = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    if (v == 0) first_level = 256;
    if (lane == 31) wsum[wid] = s;
    __syncthreads();
    if (h > 0) atomicMin(&first_level, v);
    uint32_t before = 0;
    for (int w = 0; w < wid; w++) before += wsum[w];
    const uint32_t cdf = before + s;
    if (v == 255) total = cdf;
    __syncthreads();
    if (v == first_level) first_count = h;
    __syncthreads();
    uint8_t out = (uint8_t)v;
    if (p.apply && first_level < 256 && total != first_count) {
      out = v < first_level ? 0
                            : (uint8_t)rne_div_u64(255ull * (uint64_t)(cdf - first_count),
                                                   (uint64_t)(total - first_count));
    }
    luts[(int64_t)b * 768 + 256 * c + v] = out;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ histogram
__global__ void __launch_bounds__(256) k_histogram(Plan plan, ImgList in, uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[768];
  int32_t it0, it1;
  item_range(plan, it0, it1);
  if (it0 >= it1) return;
  int32_t b = item_image(plan, it0);
  int32_t cur = b;
  for (int i = threadIdx.x; i < 768; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (int32_t item = it0; item < it1; item++) {
    while (item >= plan.prefix[b + 1]) b++;
    if (b != cur) {  // flush the finished image
      __syncthreads();
      for (int i = threadIdx.x; i < 768; i += blockDim.x) {
        if (sh[i]) atomicAdd(&hist[(int64_t)cur * 768 + i], sh[i]);
        sh[i] = 0;
      }
      __syncthreads();
      cur = b;
    }
    const alb_image si = in.get(b);
    const int32_t rb = plan.rows_per_item[b];
    const int32_t r0 = (item - plan.prefix[b]) * rb, r1 = imin(r0 + rb, si.h);
    const int64_t L = (int64_t)si.w * 3;
    for (int32_t y = r0; y < r1; y++) {
      const uint8_t* row = (const uint8_t*)si.data + (int64_t)y * si.row_stride;
      for (int64_t ob = threadIdx.x; ob < L; ob += blockDim.x) {
        const int c = (int)(ob % 3);
        atomicAdd(&sh[256 * c + __ldg(row + ob)], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 768; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[(int64_t)cur * 768 + i], sh[i]);
}

// ------------------------------------------------------------------ LUT apply
__global__ void __launch_bounds__(256) k_apply_lut(Plan plan, ImgList in, ImgList out, const uint8_t* __restrict__ luts) {
  __shared__ uint8_t lut[768];
  int32_t it0, it1;
  item_range(plan, it0, it1);
  if (it0 >= it1) return;
  int32_t b = item_image(plan, it0);
  int32_t cached = -1;
  for (int32_t item = it0; item < it1; item++) {
    while (item >= plan.prefix[b + 1]) b++;
    if (b != cached) {
      __syncthreads();
      for (int i = threadIdx.x; i < 768; i += blockDim.x) lut[i] = luts[(int64_t)b * 768 + i];
      __syncthreads();
      cached = b;
    }
    const alb_image si = in.get(b), so = out.get(b);
    const int32_t rb = plan.rows_per_item[b];
    const int32_t r0 = (item - plan.prefix[b]) * rb, r1 = imin(r0 + rb, so.h);
    const int64_t L = (int64_t)so.w * 3;
    for (int32_t y = r0; y < r1; y++) {
      const uint8_t* irow = (const uint8_t*)si.data + (int64_t)y * si.row_stride;
      uint8_t* orow = (uint8_t*)so.data + (int64_t)y * so.row_stride;
      const int64_t head = ((uintptr_t)orow) & 3;
      const bool same_phase = (((uintptr_t)irow) & 3) == (uint64_t)head;
      const int64_t nslot = (head + L + 3) >> 2;
      for (int64_t s = threadIdx.x; s < nslot; s += blockDim.x) {
        const int64_t ob0 = s * 4 - head;
        const bool full = ob0 >= 0 && ob0 + 4 <= L;
        if (full && same_phase) {
          const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(irow + ob0));
          int c = (int)(ob0 % 3);
          uint32_t o = 0;
#pragma unroll
          for (int t = 0; t < 4; t++) {
            o |= (uint32_t)lut[256 * c + ((w >> (8 * t)) & 255)] << (8 * t);
            c = c == 2 ? 0 : c + 1;
          }
          *reinterpret_cast<uint32_t*>(orow + ob0) = o;
        } else {
          for (int t = 0; t < 4; t++) {
            const int64_t ob = ob0 + t;
            if (ob >= 0 && ob < L) orow[ob] = lut[256 * (int)(ob % 3) + irow[ob]];
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------ per-pixel ops
// Grayscale: round_half_even((299 R + 587 G + 114 B) / 1000), replicated x3.
ALB_D uint8_t gray_bt601(uint32_t r, uint32_t g, uint32_t b) {
  const uint32_t num = 299 * r + 587 * g + 114 * b;
  uint32_t q = num / 1000, rem = num - q * 1000;
  if (rem > 500 || (rem == 500 && (q & 1))) q++;
  return (uint8_t)q;
}

// ShiftHSV in float32 (Smith's hexcone; hue shift 2*dh degrees, sat/val by /255).
ALB_D void shift_hsv_px(float dh, float ds, float dv, uint8_t& R, uint8_t& G, uint8_t& B) {
  const float r = R, g = G, b = B;
  const float mx = fmaxf(r, fmaxf(g, b)), mn = fminf(r, fminf(g, b));
  const float chroma = mx - mn;
  float hue = 0.0f;
  if (chroma > 0.0f) {
    if (mx == r) hue = 60.0f * ((g - b) / chroma);
    else if (mx == g) hue = 60.0f * ((b - r) / chroma + 2.0f);
    else hue = 60.0f * ((r - g) / chroma + 4.0f);
    if (hue < 0.0f) hue += 360.0f;
  }
  const float sat = mx > 0.0f ? chroma / mx : 0.0f;
  const float val = mx / 255.0f;
  float h2 = fmodf(hue + 2.0f * dh, 360.0f);
  if (h2 < 0.0f) h2 += 360.0f;
  const float s2 = fminf(fmaxf(sat + ds / 255.0f, 0.0f), 1.0f);
  const float v2 = fminf(fmaxf(val + dv / 255.0f, 0.0f), 1.0f);
  const float c2 = v2 * s2;
  const float hp = h2 / 60.0f;
  const int sector = (int)floorf(hp);
  const float frac = hp - 2.0f * floorf(hp * 0.5f);
  const float x = c2 * (1.0f - fabsf(frac - 1.0f));
  const float m = v2 - c2;
  float r1, g1, b1;
  switch (sector) {
    case 0: r1 = c2; g1 = x; b1 = 0; break;
    case 1: r1 = x; g1 = c2; b1 = 0; break;
    case 2: r1 = 0; g1 = c2; b1 = x; break;
    case 3: r1 = 0; g1 = x; b1 = c2; break;
    case 4: r1 = x; g1 = 0; b1 = c2; break;
    default: r1 = c2; g1 = 0; b1 = x; break;
  }
  R = sat_rne_f(255.0f * (r1 + m));
  G = sat_rne_f(255.0f * (g1 + m));
  B = sat_rne_f(255.0f * (b1 + m));
}

template <int OP>  // 0 = Grayscale, 1 = ShiftHSV
__global__ void __launch_bounds__(256) k_pixel(Plan plan, ImgList in, ImgList out, PrmList prm) {
  int32_t it0, it1;
  item_range(plan, it0, it1);
  if (it0 >= it1) return;
  int32_t b = item_image(plan, it0);
  for (int32_t item = it0; item < it1; item++) {
    while (item >= plan.prefix[b + 1]) b++;
    const alb_image si = in.get(b), so = out.get(b);
    const alb_params& p = prm.get(b);
    const int32_t rb = plan.rows_per_item[b];
    const int32_t r0 = (item - plan.prefix[b]) * rb, r1 = imin(r0 + rb, so.h);
    const float dh = (float)p.shift[0], ds = (float)p.shift[1], dv = (float)p.shift[2];
    const int64_t npx = (int64_t)(r1 - r0) * so.w;
    for (int64_t i = threadIdx.x; i < npx; i += blockDim.x) {
      const int32_t y = r0 + (int32_t)(i / so.w), x = (int32_t)(i % so.w);
      const uint8_t* ip = (const uint8_t*)si.data + (int64_t)y * si.row_stride + 3 * (int64_t)x;
      uint8_t* op = (uint8_t*)so.data + (int64_t)y * so.row_stride + 3 * (int64_t)x;
      uint8_t R = ip[0], G = ip[1], B = ip[2];
      if (p.apply) {
        if (OP == 0) { R = G = B = gray_bt601(R, G, B); }
        else shift_hsv_px(dh, ds, dv, R, G, B);
      }
      op[0] = R; op[1] = G; op[2] = B;
    }
  }
}

// ------------------------------------------------------------------ launchers
static int grid_for(const void* fn, int threads) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
  return (per_sm < 1 ? 1 : per_sm) * sm_count();
}

alb_status launch_photometric(int32_t tid, int32_t n, const Plan& plan, const ImgList& in, const ImgList& out,
                              const PrmList& prm, uint8_t* luts, uint32_t* hist, int32_t* status,
                              cudaStream_t st) {
  switch (tid) {
    case ALB_BRIGHTNESS: case ALB_CONTRAST: case ALB_BRIGHTNESS_CONTRAST: case ALB_GAMMA: case ALB_SHIFT_RGB: {
      k_build_luts<<<n, 256, 0, st>>>(n, prm, luts);
      ALB_CUDA(cudaGetLastError());
      return launch_stream_lut(plan, in, out, luts, st);
    }
    case ALB_EQUALIZE: {
      ALB_CUDA(cudaMemsetAsync(hist, 0, (size_t)n * 768 * sizeof(uint32_t), st));
      alb_status rc = launch_stream_hist(plan, in, hist, st);
      if (rc != ALB_OK) return rc;
      k_equalize_luts<<<n, 256, 0, st>>>(n, prm, hist, luts);
      ALB_CUDA(cudaGetLastError());
      return launch_stream_lut(plan, in, out, luts, st);
    }
    case ALB_GRAYSCALE: case ALB_SHIFT_HSV:
      return launch_stream_pixel(tid, plan, in, out, prm, st);
    default:
      set_error("launch_photometric: transform %d is not photometric", tid);
      return ALB_EINVAL;
  }
}

}  // namespace alb
