// alb_color.cu -- photometric transforms (Table I: Brightness, ShiftHSV,
// ShiftRGB, Gamma, Grayscale; Sec. II and Fig. 1: colour, contrast and
// brightness transforms) and per-channel histogram equalisation.
//
// LUT transforms run in two launches: k_build_luts computes each image's
// three 256-entry tables once in float64 (the tables are the exact rounding
// points of the definition), then the streaming LUT kernel (alb_stream.cu)
// applies them from shared memory.  Equalize first builds per-image
// histograms (alb_stream.cu), then its tables here with a 256-bin block scan.
// Grayscale and ShiftHSV are per-pixel streaming kernels (alb_stream.cu).
#include "alb_common.cuh"
#include "alb_kernels.cuh"

namespace alb {

ALB_D uint8_t sat_rne(double v) {
  double r = rint(v);
  r = r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r);
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
      // float32 first: 255 (v/255)^g is then within 2e-4 of the exact value
      // (powf's documented bound of a few ulp at <= 255, the rounding of v/255
      // and of g to float), so unless it lies within 4e-3 of a rounding point
      // (a half-integer) it rounds like the float64 definition; the rare
      // others are evaluated in float64 (FP64 throughput is low on this GPU)
      const float y32 = 255.0f * powf((float)v / 255.0f, (float)p.gamma);
      const float frac = y32 - floorf(y32);
      uint8_t o;
      if (fabsf(frac - 0.5f) > 4e-3f) {
        o = sat_rne((double)rintf(y32));
      } else {
        o = sat_rne(255.0 * pow(x / 255.0, p.gamma));
      }
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

// ------------------------------------------------------------------ launchers
alb_status launch_photometric(int32_t tid, int32_t n, const Plan& plan, const ImgList& in, const ImgList& out,
                              const PrmList& prm, uint8_t* luts, uint32_t* hist, int32_t* status,
                              cudaStream_t st) {
  switch (tid) {
    case ALB_BRIGHTNESS: case ALB_CONTRAST: case ALB_BRIGHTNESS_CONTRAST: case ALB_GAMMA: case ALB_SHIFT_RGB: {
      k_build_luts<<<n, 256, 0, st>>>(n, prm, luts);
      ALB_CUDA(cudaGetLastError());
      return launch_stream_lut(plan, in, out, luts, status, st);
    }
    case ALB_EQUALIZE: {
      ALB_CUDA(cudaMemsetAsync(hist, 0, (size_t)n * 768 * sizeof(uint32_t), st));
      alb_status rc = launch_stream_hist(plan, in, hist, status, st);
      if (rc != ALB_OK) return rc;
      k_equalize_luts<<<n, 256, 0, st>>>(n, prm, hist, luts);
      ALB_CUDA(cudaGetLastError());
      return launch_stream_lut(plan, in, out, luts, status, st);
    }
    case ALB_GRAYSCALE: case ALB_SHIFT_HSV:
      return launch_stream_pixel(tid, plan, in, out, prm, status, st);
    default:
      set_error("launch_photometric: transform %d is not photometric", tid);
      return ALB_EINVAL;
  }
}

}  // namespace alb
