// alb_stream.cu -- streaming kernels for the transforms that touch each output
// byte once with a fixed source byte (Table I: HorizontalFlip, VerticalFlip,
// RandomCrop, PadToSize, Brightness, ShiftRGB, Gamma, Grayscale, ShiftHSV;
// Sec. II contrast; per-channel equalisation).
//
// Memory path: every warp moves whole 16-byte vectors.  Contiguous, 16-byte
// aligned images (the common case) are processed as one flat byte array:
// per-byte ops in 16-byte chunks, per-pixel ops in 48-byte units (16 RGB
// pixels, 3 vectors, always 16-byte aligned in the flat array).  Row-based
// copies (vertical flip, crop, pad interior) use per-row 16-byte output chunks
// whose source window, misaligned by a per-row constant, is read with aligned
// loads and realigned with funnel shifts.  Strided images and the bytes at row
// and item edges take a per-byte path.
#include "alb_common.cuh"
#include "alb_kernels.cuh"
#include "alb_vec.cuh"

namespace alb {

ALB_D uint8_t sat_rne_f(float v) {
  const float r = fminf(fmaxf(rintf(v), 0.0f), 255.0f);
  return (uint8_t)r;
}

// ================================================================== LUT ops
// Tables in shared memory, 32 copies interleaved so that lane l always reads
// bank l: byte v of channel c for lane l lives at c*8192 + (v & ~3)*32 + 4l + (v & 3).
constexpr int kLutBytes = 3 * 8192;

__device__ void build_lut_copies(const uint8_t* __restrict__ g, uint8_t* sh768, uint32_t* tab) {
  for (int i = threadIdx.x; i < 768; i += blockDim.x) sh768[i] = g[i];
  __syncthreads();
  for (int wi = threadIdx.x; wi < kLutBytes / 4; wi += blockDim.x) {
    const int c = wi >> 11, rem = wi & 2047, vq = rem >> 5;
    const uint8_t* s = sh768 + 256 * c + 4 * vq;
    tab[wi] = (uint32_t)s[0] | ((uint32_t)s[1] << 8) | ((uint32_t)s[2] << 16) | ((uint32_t)s[3] << 24);
  }
  __syncthreads();
}

ALB_D uint32_t lut_off(uint32_t v) { return ((v & 0xFCu) << 5) | (v & 3u); }

// one RGB pixel through the three tables (lb = this lane's table base)
ALB_D void lut_px(const uint8_t* tab, int lb, uint32_t& r, uint32_t& g, uint32_t& b) {
  r = tab[lb + lut_off(r)];
  g = tab[lb + 8192 + lut_off(g)];
  b = tab[lb + 16384 + lut_off(b)];
}

__global__ void __launch_bounds__(256) k_lut_stream(Plan plan, ImgList in, ImgList out,
                                                    const uint8_t* __restrict__ luts) {
  __shared__ __align__(16) uint32_t tab32[kLutBytes / 4];
  __shared__ uint8_t sh768[768];
  const uint8_t* tab = reinterpret_cast<const uint8_t*>(tab32);
  int32_t it0, it1;
  item_range(plan, it0, it1);
  if (it0 >= it1) return;
  const int lb = 4 * (threadIdx.x & 31);
  int32_t b = item_image(plan, it0);
  int32_t cached = -1;
  for (int32_t item = it0; item < it1; item++) {
    while (item >= plan.prefix[b + 1]) b++;
    if (b != cached) {
      __syncthreads();
      build_lut_copies(luts + (int64_t)b * 768, sh768, tab32);
      cached = b;
    }
    const alb_image si = in.get(b), so = out.get(b);
    const int32_t rb = plan.rows_per_item[b];
    const int32_t r0 = (item - plan.prefix[b]) * rb, r1 = imin(r0 + rb, so.h);
    const uint8_t* __restrict__ ip = (const uint8_t*)si.data;
    uint8_t* __restrict__ op = (uint8_t*)so.data;
    if (flat_aligned(si) && flat_aligned(so)) {
      const int64_t a = (int64_t)r0 * so.w, e = (int64_t)r1 * so.w;   // pixel range
      const int64_t u0 = (a + 15) >> 4, u1 = e >> 4;                    // whole 16-pixel units
      for (int64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        const uint8_t* src = ip + 48 * u;
        const uint4 v0 = ldg16(src), v1 = ldg16(src + 16), v2 = ldg16(src + 32);
        const uint32_t w[12] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w};
        uint32_t o[12];
#pragma unroll
        for (int m = 0; m < 12; m++) {
          uint32_t acc = 0;
#pragma unroll
          for (int t = 0; t < 4; t++) {
            const int k = 4 * m + t, c = k % 3;
            acc |= (uint32_t)tab[lb + 8192 * c + lut_off((w[m] >> (8 * t)) & 0xFFu)] << (8 * t);
          }
          o[m] = acc;
        }
        uint8_t* dst = op + 48 * u;
        stg16(dst, make_uint4(o[0], o[1], o[2], o[3]));
        stg16(dst + 16, make_uint4(o[4], o[5], o[6], o[7]));
        stg16(dst + 32, make_uint4(o[8], o[9], o[10], o[11]));
      }
      const int64_t h1 = u0 * 16 < e ? u0 * 16 : e;
      for (int64_t q = a + threadIdx.x; q < e; q += blockDim.x) {
        if (q >= h1 && q < u1 * 16) continue;
        uint32_t R = ip[3 * q], G = ip[3 * q + 1], B = ip[3 * q + 2];
        lut_px(tab, lb, R, G, B);
        op[3 * q] = (uint8_t)R; op[3 * q + 1] = (uint8_t)G; op[3 * q + 2] = (uint8_t)B;
      }
    } else {
      const int64_t npx = (int64_t)(r1 - r0) * so.w;
      for (int64_t i = threadIdx.x; i < npx; i += blockDim.x) {
        const int32_t y = r0 + (int32_t)(i / so.w), x = (int32_t)(i % so.w);
        const uint8_t* s0 = ip + (int64_t)y * si.row_stride + 3 * (int64_t)x;
        uint8_t* d = op + (int64_t)y * so.row_stride + 3 * (int64_t)x;
        uint32_t R = s0[0], G = s0[1], B = s0[2];
        lut_px(tab, lb, R, G, B);
        d[0] = (uint8_t)R; d[1] = (uint8_t)G; d[2] = (uint8_t)B;
      }
    }
  }
}

// ================================================================== per-pixel ops
ALB_D void gray_px(uint32_t& r, uint32_t& g, uint32_t& b) {
  const uint32_t num = 299 * r + 587 * g + 114 * b;
  uint32_t q = num / 1000, rem = num - q * 1000;
  if (rem > 500 || (rem == 500 && (q & 1))) q++;
  r = g = b = q;
}

// ShiftHSV, float32 (Smith's hexcone; hue shift 2*dh degrees; sat and val by
// /255).  Branch-free: the hue numerator/offset are selected, and the inverse
// hexcone uses the per-channel form f(n) = V - V S clamp(min(k, 4 - k), 0, 1),
// k = (n + H/60) mod 6 with n = 5, 3, 1 for R, G, B (identical to the sector
// table of the definition).
ALB_D uint32_t hsv_channel(float hp, float n, float V255, float C255) {
  float k = hp + n;
  k = k >= 6.0f ? k - 6.0f : k;
  const float t = __saturatef(fminf(k, 4.0f - k));
  return sat_rne_f(fmaf(-C255, t, V255));
}

ALB_D void hsv_px(float dh2, float ds, float dv, uint32_t& R, uint32_t& G, uint32_t& B) {
  const float r = (float)R, g = (float)G, b = (float)B;
  const float mx = fmaxf(r, fmaxf(g, b)), mn = fminf(r, fminf(g, b));
  const float chroma = mx - mn;
  const bool isr = mx == r, isg = !isr && mx == g;
  const float num = isr ? g - b : (isg ? b - r : r - g);
  const float off = isr ? 0.0f : (isg ? 120.0f : 240.0f);
  float hue = chroma > 0.0f ? fmaf(num, __fdividef(60.0f, chroma), off) : 0.0f;
  hue = hue < 0.0f ? hue + 360.0f : hue;
  const float sat = mx > 0.0f ? __fdividef(chroma, mx) : 0.0f;
  float h2 = hue + dh2;
  h2 = h2 >= 360.0f ? h2 - 360.0f : h2;
  h2 = h2 < 0.0f ? h2 + 360.0f : h2;
  const float s2 = __saturatef(sat + ds);
  const float v2 = __saturatef(fmaf(mx, 1.0f / 255.0f, dv));
  const float V255 = 255.0f * v2, C255 = V255 * s2;
  const float hp = h2 * (1.0f / 60.0f);
  R = hsv_channel(hp, 5.0f, V255, C255);
  G = hsv_channel(hp, 3.0f, V255, C255);
  B = hsv_channel(hp, 1.0f, V255, C255);
}

template <int OP>  // 0 = Grayscale, 1 = ShiftHSV
ALB_D void pixel_op(uint32_t& r, uint32_t& g, uint32_t& b, float dh2, float ds, float dv) {
  if (OP == 0) gray_px(r, g, b);
  else hsv_px(dh2, ds, dv, r, g, b);
}

template <int OP>
__global__ void __launch_bounds__(256) k_pixel_stream(Plan plan, ImgList in, ImgList out, PrmList prm) {
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
    const bool act = p.apply != 0;
    const float dh2 = (float)(2.0 * p.shift[0]), ds = (float)(p.shift[1] / 255.0), dv = (float)(p.shift[2] / 255.0);
    const uint8_t* __restrict__ ip = (const uint8_t*)si.data;
    uint8_t* __restrict__ op = (uint8_t*)so.data;
    if (flat_aligned(si) && flat_aligned(so)) {
      const int64_t a = (int64_t)r0 * so.w, e = (int64_t)r1 * so.w;   // pixel range
      const int64_t u0 = (a + 15) >> 4, u1 = e >> 4;                    // whole 16-pixel units
      for (int64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        const uint8_t* src = ip + 48 * u;
        uint4 v0 = ldg16(src), v1 = ldg16(src + 16), v2 = ldg16(src + 32);
        if (act) {
          uint32_t w[12] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w};
          uint32_t o[12] = {0};
#pragma unroll
          for (int px = 0; px < 16; px++) {
            uint32_t R = byte_of(w, 3 * px), G = byte_of(w, 3 * px + 1), B = byte_of(w, 3 * px + 2);
            pixel_op<OP>(R, G, B, dh2, ds, dv);
            o[(3 * px) >> 2] |= R << (8 * ((3 * px) & 3));
            o[(3 * px + 1) >> 2] |= G << (8 * ((3 * px + 1) & 3));
            o[(3 * px + 2) >> 2] |= B << (8 * ((3 * px + 2) & 3));
          }
          v0 = make_uint4(o[0], o[1], o[2], o[3]);
          v1 = make_uint4(o[4], o[5], o[6], o[7]);
          v2 = make_uint4(o[8], o[9], o[10], o[11]);
        }
        uint8_t* dst = op + 48 * u;
        stg16(dst, v0); stg16(dst + 16, v1); stg16(dst + 32, v2);
      }
      const int64_t h1 = u0 * 16 < e ? u0 * 16 : e;
      for (int64_t q = a + threadIdx.x; q < h1; q += blockDim.x) {
        uint32_t R = ip[3 * q], G = ip[3 * q + 1], B = ip[3 * q + 2];
        if (act) pixel_op<OP>(R, G, B, dh2, ds, dv);
        op[3 * q] = (uint8_t)R; op[3 * q + 1] = (uint8_t)G; op[3 * q + 2] = (uint8_t)B;
      }
      for (int64_t q = (u1 * 16 > h1 ? u1 * 16 : h1) + threadIdx.x; q < e; q += blockDim.x) {
        uint32_t R = ip[3 * q], G = ip[3 * q + 1], B = ip[3 * q + 2];
        if (act) pixel_op<OP>(R, G, B, dh2, ds, dv);
        op[3 * q] = (uint8_t)R; op[3 * q + 1] = (uint8_t)G; op[3 * q + 2] = (uint8_t)B;
      }
    } else {
      const int64_t npx = (int64_t)(r1 - r0) * so.w;
      for (int64_t i = threadIdx.x; i < npx; i += blockDim.x) {
        const int32_t y = r0 + (int32_t)(i / so.w), x = (int32_t)(i % so.w);
        const uint8_t* s = ip + (int64_t)y * si.row_stride + 3 * (int64_t)x;
        uint8_t* d = op + (int64_t)y * so.row_stride + 3 * (int64_t)x;
        uint32_t R = s[0], G = s[1], B = s[2];
        if (act) pixel_op<OP>(R, G, B, dh2, ds, dv);
        d[0] = (uint8_t)R; d[1] = (uint8_t)G; d[2] = (uint8_t)B;
      }
    }
  }
}

// ================================================================== horizontal flip
// Flat 16-pixel units: a unit inside one row reads the mirrored 16 pixels of
// the same row (a 48-byte window, misaligned by a per-row constant), reverses
// the pixel order in registers and stores 3 aligned vectors.
ALB_D constexpr int rev_src(int k) { return 3 * (15 - k / 3) + k % 3; }

__global__ void __launch_bounds__(256) k_hflip_stream(Plan plan, ImgList in, ImgList out, PrmList prm) {
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
    const int32_t W = so.w;
    const bool act = p.apply != 0;
    const uint8_t* __restrict__ ip = (const uint8_t*)si.data;
    uint8_t* __restrict__ op = (uint8_t*)so.data;
    if (flat_aligned(si) && flat_aligned(so)) {
      const int64_t a = (int64_t)r0 * W, e = (int64_t)r1 * W;
      const int64_t u0 = (a + 15) >> 4, u1 = e >> 4;
      for (int64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        const int64_t p0 = 16 * u;
        const int32_t y = (int32_t)((uint32_t)p0 / (uint32_t)W), x0 = (int32_t)(p0 - (int64_t)y * W);
        uint8_t* dst = op + 48 * u;
        if (!act) {
          stg16(dst, ldg16(ip + 48 * u)); stg16(dst + 16, ldg16(ip + 48 * u + 16));
          stg16(dst + 32, ldg16(ip + 48 * u + 32));
        } else if (x0 + 16 <= W) {
          const int64_t s0 = (int64_t)y * W + (W - 16 - x0);      // first source pixel
          uint32_t win[12];
          load_window<12>(ip + 3 * s0, win);
          uint32_t o[12];
#pragma unroll
          for (int m = 0; m < 12; m++) {
            o[m] = byte_of(win, rev_src(4 * m)) | (byte_of(win, rev_src(4 * m + 1)) << 8) |
                   (byte_of(win, rev_src(4 * m + 2)) << 16) | (byte_of(win, rev_src(4 * m + 3)) << 24);
          }
          stg16(dst, make_uint4(o[0], o[1], o[2], o[3]));
          stg16(dst + 16, make_uint4(o[4], o[5], o[6], o[7]));
          stg16(dst + 32, make_uint4(o[8], o[9], o[10], o[11]));
        } else {      // the unit straddles a row end (rows y, y + 1, ...)
          int32_t yy = y, xx = x0;
#pragma unroll 4
          for (int j = 0; j < 16; j++) {
            const uint8_t* s = ip + 3 * ((int64_t)yy * W + (W - 1 - xx));
            dst[3 * j] = s[0]; dst[3 * j + 1] = s[1]; dst[3 * j + 2] = s[2];
            if (++xx == W) { xx = 0; yy++; }
          }
        }
      }
      // pixels of the item outside whole units
      const int64_t h1 = u0 * 16 < e ? u0 * 16 : e;
      for (int64_t q = a + threadIdx.x; q < e; q += blockDim.x) {
        if (q >= h1 && q < u1 * 16) continue;
        const int32_t yy = (int32_t)((uint32_t)q / (uint32_t)W), xx = (int32_t)(q - (int64_t)yy * W);
        const uint8_t* s = ip + 3 * ((int64_t)yy * W + (act ? W - 1 - xx : xx));
        op[3 * q] = s[0]; op[3 * q + 1] = s[1]; op[3 * q + 2] = s[2];
      }
    } else {
      const int64_t npx = (int64_t)(r1 - r0) * W;
      for (int64_t i = threadIdx.x; i < npx; i += blockDim.x) {
        const int32_t y = r0 + (int32_t)(i / W), x = (int32_t)(i % W);
        const uint8_t* s = ip + (int64_t)y * si.row_stride + 3 * (int64_t)(act ? W - 1 - x : x);
        uint8_t* d = op + (int64_t)y * so.row_stride + 3 * (int64_t)x;
        d[0] = s[0]; d[1] = s[1]; d[2] = s[2];
      }
    }
  }
}

// ================================================================== row copies
// Vertical flip, crop and pad: output row y takes bytes of source row sy
// starting at a row-constant offset (crop: 3 x0; pad interior: -3 left); pad
// borders are reflected pixels.  Three lane-parallel loops per item: whole
// 16-byte chunks of the interior (realigned source window), the <= 15 interior
// bytes at each end outside whole chunks, and the pad borders.
template <int CT, int TID>
__global__ void __launch_bounds__(256) k_rowcopy(Plan plan, ImgList in, ImgList out, PrmList prm) {
  int32_t it0, it1;
  item_range(plan, it0, it1);
  if (it0 >= it1) return;
  int32_t b = item_image(plan, it0);
  for (int32_t item = it0; item < it1; item++) {
    while (item >= plan.prefix[b + 1]) b++;
    const alb_image si = in.get(b), so = out.get(b);
    const alb_params& p = prm.get(b);
    const int32_t C = CT ? CT : so.c;
    const int32_t rb = plan.rows_per_item[b];
    const int32_t r0 = (item - plan.prefix[b]) * rb, r1 = imin(r0 + rb, so.h);
    const int32_t nrow = r1 - r0;
    const bool act = p.apply != 0;
    const int32_t L = so.w * C;
    // interior output bytes [lo, hi) come from source byte x + shift
    int32_t lo = 0, hi = L, shift = 0;
    if (act && TID == ALB_RANDOM_CROP) shift = p.x0 * C;
    if (act && TID == ALB_PAD_TO_SIZE) { lo = p.x0 * C; hi = lo + si.w * C; shift = -lo; }
    const uint8_t* __restrict__ ip = (const uint8_t*)si.data;
    uint8_t* __restrict__ op = (uint8_t*)so.data;
    auto src_row = [&](int32_t y) -> int32_t {
      if (!act) return y;
      if (TID == ALB_VFLIP) return si.h - 1 - y;
      if (TID == ALB_RANDOM_CROP) return p.y0 + y;
      return reflect101((int64_t)y - p.y0, si.h);
    };
    // first and last whole chunk of the interior of row y
    auto chunk_bounds = [&](uint8_t* orow, int32_t& A, int32_t& B) {
      const int32_t ph = (int32_t)(reinterpret_cast<uintptr_t>(orow) & 15);
      A = ((ph + lo + 15) & ~15) - ph;
      B = ((ph + hi) & ~15) - ph;
      if (B < A) { A = hi; B = hi; }
    };
    const int32_t cpr = (hi - lo) / 16 + 1;
    for (int32_t i = threadIdx.x; i < nrow * cpr; i += blockDim.x) {
      const int32_t yy = i / cpr, j = i - yy * cpr, y = r0 + yy;
      uint8_t* orow = op + (int64_t)y * so.row_stride;
      int32_t A, B;
      chunk_bounds(orow, A, B);
      const int32_t x = A + 16 * j;
      if (x + 16 > B) continue;
      const uint8_t* srow = ip + (int64_t)src_row(y) * si.row_stride;
      uint32_t w[4];
      load_window<4>(srow + x + shift, w);
      stg16(orow + x, make_uint4(w[0], w[1], w[2], w[3]));
    }
    for (int32_t i = threadIdx.x; i < nrow * 32; i += blockDim.x) {
      const int32_t yy = i >> 5, k = i & 31, y = r0 + yy;
      uint8_t* orow = op + (int64_t)y * so.row_stride;
      int32_t A, B;
      chunk_bounds(orow, A, B);
      const int32_t x = k < 16 ? lo + k : B + (k - 16);
      if (k < 16 ? x >= A : x >= hi) continue;
      orow[x] = ip[(int64_t)src_row(y) * si.row_stride + x + shift];
    }
    if (TID == ALB_PAD_TO_SIZE && act) {
      const int32_t nb = lo + (L - hi);
      for (int32_t i = threadIdx.x; i < nrow * nb; i += blockDim.x) {
        const int32_t yy = i / nb, k = i - yy * nb, y = r0 + yy;
        const int32_t x = k < lo ? k : hi + (k - lo);
        const int32_t px = x / C, c = x - px * C;
        const int32_t sx = reflect101((int64_t)px - p.x0, si.w);
        op[(int64_t)y * so.row_stride + x] = ip[(int64_t)src_row(y) * si.row_stride + sx * C + c];
      }
    }
  }
}

// ================================================================== histogram
// Per-CTA shared-memory histograms (one copy per warp to spread contention on
// the smooth images' repeated values), merged into the image's global
// histogram with one atomic per bin when the CTA leaves the image.
__global__ void __launch_bounds__(256) k_hist_stream(Plan plan, ImgList in, uint32_t* __restrict__ hist) {
  constexpr int NWARP = 8;
  __shared__ uint32_t sh[NWARP][768];
  int32_t it0, it1;
  item_range(plan, it0, it1);
  if (it0 >= it1) return;
  const int wid = threadIdx.x >> 5;
  uint32_t* my = sh[wid];
  int32_t b = item_image(plan, it0);
  int32_t cur = b;
  for (int i = threadIdx.x; i < NWARP * 768; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  auto flush = [&](int32_t img) {
    __syncthreads();
    for (int i = threadIdx.x; i < 768; i += blockDim.x) {
      uint32_t s = 0;
#pragma unroll
      for (int w = 0; w < NWARP; w++) { s += sh[w][i]; sh[w][i] = 0; }
      if (s) atomicAdd(&hist[(int64_t)img * 768 + i], s);
    }
    __syncthreads();
  };
  for (int32_t item = it0; item < it1; item++) {
    while (item >= plan.prefix[b + 1]) b++;
    if (b != cur) { flush(cur); cur = b; }
    const alb_image si = in.get(b);
    const int32_t rb = plan.rows_per_item[b];
    const int32_t r0 = (item - plan.prefix[b]) * rb, r1 = imin(r0 + rb, si.h);
    const uint8_t* __restrict__ ip = (const uint8_t*)si.data;
    const int64_t L = (int64_t)si.w * 3;
    if (flat_aligned(si)) {
      const int64_t a = r0 * L, e = r1 * L;
      const int64_t c0 = (a + 15) >> 4, c1 = e >> 4;
      for (int64_t k = c0 + threadIdx.x; k < c1; k += blockDim.x) {
        const uint4 v = ldg16(ip + 16 * k);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        int c = (int)(k % 3);
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
          for (int t = 0; t < 4; t++) {
            atomicAdd(&my[256 * c + ((w[j] >> (8 * t)) & 0xFFu)], 1u);
            c = c == 2 ? 0 : c + 1;
          }
      }
      const int64_t h1 = 16 * c0 < e ? 16 * c0 : e;
      for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) {
        if (i >= h1 && i < 16 * c1) continue;
        atomicAdd(&my[256 * (int)(i % 3) + ip[i]], 1u);
      }
    } else {
      const int64_t n = (int64_t)(r1 - r0) * L;
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int32_t y = r0 + (int32_t)(i / L);
        const int64_t x = i - (int64_t)(y - r0) * L;
        atomicAdd(&my[256 * (int)(x % 3) + ip[(int64_t)y * si.row_stride + x]], 1u);
      }
    }
  }
  flush(cur);
}

// ================================================================== launchers
static int grid_for(const void* fn, int threads) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
  return (per_sm < 1 ? 1 : per_sm) * sm_count();
}

template <class... KArgs, class... Args>
static alb_status launch_k(void (*kern)(KArgs...), cudaStream_t st, Args... args) {
  kern<<<grid_for((const void*)kern, 256), 256, 0, st>>>(args...);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

// Streaming implementations; returns ALB_EINVAL (nothing launched) when the
// transform/channel combination has none, so the caller uses its general kernel.
alb_status launch_stream_geometric(int32_t tid, const Plan& plan, const ImgList& in, const ImgList& out,
                                   const PrmList& prm, int32_t channels, cudaStream_t st) {
  switch (tid) {
    case ALB_HFLIP:
      if (channels == 3) return launch_k(k_hflip_stream, st, plan, in, out, prm);
      break;
    case ALB_VFLIP:
      if (channels == 3) return launch_k(k_rowcopy<3, ALB_VFLIP>, st, plan, in, out, prm);
      if (channels == 1) return launch_k(k_rowcopy<1, ALB_VFLIP>, st, plan, in, out, prm);
      return launch_k(k_rowcopy<0, ALB_VFLIP>, st, plan, in, out, prm);
    case ALB_RANDOM_CROP:
      if (channels == 3) return launch_k(k_rowcopy<3, ALB_RANDOM_CROP>, st, plan, in, out, prm);
      if (channels == 1) return launch_k(k_rowcopy<1, ALB_RANDOM_CROP>, st, plan, in, out, prm);
      return launch_k(k_rowcopy<0, ALB_RANDOM_CROP>, st, plan, in, out, prm);
    case ALB_PAD_TO_SIZE:
      if (channels == 3) return launch_k(k_rowcopy<3, ALB_PAD_TO_SIZE>, st, plan, in, out, prm);
      if (channels == 1) return launch_k(k_rowcopy<1, ALB_PAD_TO_SIZE>, st, plan, in, out, prm);
      return launch_k(k_rowcopy<0, ALB_PAD_TO_SIZE>, st, plan, in, out, prm);
    default:
      break;
  }
  return ALB_EINVAL;
}

alb_status launch_stream_lut(const Plan& plan, const ImgList& in, const ImgList& out, const uint8_t* luts,
                             cudaStream_t st) {
  return launch_k(k_lut_stream, st, plan, in, out, luts);
}

alb_status launch_stream_pixel(int32_t tid, const Plan& plan, const ImgList& in, const ImgList& out,
                               const PrmList& prm, cudaStream_t st) {
  if (tid == ALB_GRAYSCALE) return launch_k(k_pixel_stream<0>, st, plan, in, out, prm);
  return launch_k(k_pixel_stream<1>, st, plan, in, out, prm);
}

alb_status launch_stream_hist(const Plan& plan, const ImgList& in, uint32_t* hist, cudaStream_t st) {
  return launch_k(k_hist_stream, st, plan, in, hist);
}

}  // namespace alb
