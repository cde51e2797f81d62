// alb_fused.cu -- the ragged-batch chain: RandomResizedCrop -> Q5 bilinear resize
// to out_h x out_w -> h-flip -> brightness/contrast table -> saturation (float32)
// -> Normalize -> bfloat16 NCHW.  (The paper's Sec. II-A example combines a flip
// with a random sized crop; Sec. II-C uses colour transforms; the chain is the
// ImageNet-style training pipeline built from them.)
//
// ALB_MODE_FUSED: one persistent kernel; CTAs pull (image, band of output rows)
// items from an atomic queue, every output value is computed from the source
// crop in registers and written once.
// ALB_MODE_PLAIN: five kernels with materialised intermediates (u8 resize, u8
// flip, u8 table, f32 saturation, bf16 normalise), the comparison path.
// Both modes call the same __device__ step functions, so outputs are identical.
#include <cuda_bf16.h>

#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "alb_common.cuh"
#include "alb_kernels.cuh"

namespace alb {

constexpr int kBandMax = 32;   // output rows per work item, at most
constexpr int kBandMaxP = 32;  // rows per pivot item

struct ChainK {
  float k[3], m[3];  // Normalize: y = fma(x, k_c, m_c)
  int32_t oh, ow;
};

ALB_D uint8_t sat_rne_d(double v) {
  double r = rint(v);
  r = r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r);
  return (uint8_t)r;
}

// ---------------------------------------------------------------- step functions
ALB_D int32_t chain_q5(int32_t d, int32_t n_in, int32_t n_out) {
  int64_t xq;
  if (n_in <= 2048 && n_out <= 2048) {    // |numerator| < 2^29: exact in 32-bit
    const int32_t num = 32 * ((2 * d + 1) * n_in - n_out) + n_out, den = 2 * n_out;
    const int32_t q = num / den;
    xq = (num % den != 0 && num < 0) ? q - 1 : q;
  } else {
    xq = floor_div(32 * ((int64_t)(2 * d + 1) * n_in - n_out) + n_out, 2 * (int64_t)n_out);
  }
  if (xq < 0) xq = 0;
  if ((xq >> 5) >= n_in - 1) xq = 32 * (int64_t)(n_in - 1);
  return (int32_t)xq;
}

// The 6 bytes at p (pixels ix, ix + 1 of a row) as lo = bytes 0..3, hi = 4..5,
// read as aligned words; the third word only when it holds a needed byte.
ALB_D void chain_pair(const uint8_t* p, uint32_t& lo, uint32_t& hi) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint32_t* w = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
  const int s = (int)(a & 3);
  const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = s == 3 ? __ldg(w + 2) : 0u;
  lo = __funnelshift_r(w0, w1, 8 * s);
  hi = __funnelshift_r(w1, w2, 8 * s);
}

// Q5 bilinear sample (3 channels) from the window's two tap rows ra (row iy)
// and rb (row min(iy + 1, ch - 1)) at the Q5 column xq, vertical fraction fy:
// (sum w_ij p_ij + 512) >> 10.  The tap pairs as {R0, R1, G0, G1} and {B0, B1}
// per row against the 16-bit weight pairs (wx0 wy, wx1 wy) of the top (wy =
// 32 - fy) and bottom (wy = fy) row: two dp2a per channel.
ALB_D void chain_bilerp(const uint8_t* __restrict__ ra, const uint8_t* __restrict__ rb, int32_t cw, int32_t xq,
                        int32_t fy, uint32_t rgb[3]) {
  int32_t ix = xq >> 5;
  const int32_t fx = xq & 31;
  if (!ALB_IN(ix >= 0 && ix < cw)) {
    rgb[0] = rgb[1] = rgb[2] = 0u;
    return;
  }
  uint32_t wxp = 32u + 65535u * (uint32_t)fx;       // {32 - fx, fx}: weights of pixels ix, ix + 1
  uint32_t tl, th, bl, bh;
  if (cw >= 2) {
    if (ix + 1 >= cw) {   // clamped last column (fx = 0): the pair (ix - 1, ix), all weight on the second
      ix -= 1;
      wxp = 32u << 16;
    }
    chain_pair(ra + 3 * ix, tl, th);
    chain_pair(rb + 3 * ix, bl, bh);
  } else {                // one-column window: both horizontal taps are that column
    const uint32_t t = (uint32_t)ra[0] | ((uint32_t)ra[1] << 8) | ((uint32_t)ra[2] << 16);
    const uint32_t u = (uint32_t)rb[0] | ((uint32_t)rb[1] << 8) | ((uint32_t)rb[2] << 16);
    tl = t | (t << 24); th = t >> 8; bl = u | (u << 24); bh = u >> 8;
    wxp = 32u;
  }
  const uint32_t wt = wxp * (uint32_t)(32 - fy), wb = wxp * (uint32_t)fy;
  const uint32_t pt = __byte_perm(tl, th, 0x4130), qt = __byte_perm(tl, th, 0x0052);
  const uint32_t pb = __byte_perm(bl, bh, 0x4130), qb = __byte_perm(bl, bh, 0x0052);
  rgb[0] = __dp2a_lo(wt, pt, __dp2a_lo(wb, pb, 512u)) >> 10;
  rgb[1] = __dp2a_hi(wt, pt, __dp2a_hi(wb, pb, 512u)) >> 10;
  rgb[2] = __dp2a_lo(wt, qt, __dp2a_lo(wb, qb, 512u)) >> 10;
}

// the same at Q5 coordinates (xq, yq) of the window
ALB_D void chain_bilinear(const uint8_t* __restrict__ win, int64_t stride, int32_t ch, int32_t cw, int32_t xq,
                          int32_t yq, uint32_t rgb[3]) {
  const int32_t iy = yq >> 5;
  if (!ALB_IN(iy >= 0 && iy < ch)) {
    rgb[0] = rgb[1] = rgb[2] = 0u;
    return;
  }
  chain_bilerp(win + (int64_t)iy * stride, win + (int64_t)imin(iy + 1, ch - 1) * stride, cw, xq, yq & 31, rgb);
}

// a byte as float through the 2^23 bias (exact; no integer conversion unit)
ALB_D float u8f(uint32_t v) { return __uint_as_float(0x4B000000u | v) - 8388608.0f; }

// saturation blend with the BT.601 grey value, float32, clamped, not rounded
ALB_D void chain_saturate(const uint32_t rgb[3], float s, float out[3]) {
  const float f[3] = {u8f(rgb[0]), u8f(rgb[1]), u8f(rgb[2])};
  const float grey = __fmaf_rn(0.114f, f[2], __fmaf_rn(0.587f, f[1], __fmul_rn(0.299f, f[0])));
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float v = __fmaf_rn(s, __fsub_rn(f[c], grey), grey);
    out[c] = fminf(fmaxf(v, 0.0f), 255.0f);
  }
}

ALB_D __nv_bfloat16 chain_normalize(float v, float k, float m) { return __float2bfloat16_rn(__fmaf_rn(v, k, m)); }

// ---------------------------------------------------------------- jitter mode 1
// Brightness (B = 0), contrast (C = 1) and saturation (S = 2) in a per-image
// order, permutation index k in 0..5 (lexicographic: BCS BSC CBS CSB SBC SCB),
// each op producing uint8: B and C through per-image tables (B: sat_rne(b v);
// C: sat_rne(m + c (v - m)) with m the image's contrast pivot, both float64),
// S per pixel in float32 fmas rounded half-even to uint8.
ALB_D int jitter_op(int k, int i) {
  // two bits per position, six bits per permutation
  constexpr uint64_t code = (uint64_t)(0 | 1 << 2 | 2 << 4) | (uint64_t)(0 | 2 << 2 | 1 << 4) << 6 |
                            (uint64_t)(1 | 0 << 2 | 2 << 4) << 12 | (uint64_t)(1 | 2 << 2 | 0 << 4) << 18 |
                            (uint64_t)(2 | 0 << 2 | 1 << 4) << 24 | (uint64_t)(2 | 1 << 2 | 0 << 4) << 30;
  return (int)((code >> (6 * k + 2 * i)) & 3u);
}

ALB_D uint32_t sat_rne_f(float v) {
  // clamping first and rounding after gives the same byte; adding 2^23 rounds
  // half to even into the low bits (no float-to-integer conversion)
  return __float_as_uint(fminf(fmaxf(v, 0.0f), 255.0f) + 8388608.0f) & 0xFFu;
}

// saturation of jitter mode 1: the float32 blend of chain_saturate, rounded to uint8
ALB_D void jitter_saturate(uint32_t rgb[3], float s) {
  const float f[3] = {u8f(rgb[0]), u8f(rgb[1]), u8f(rgb[2])};
  const float grey = __fmaf_rn(0.114f, f[2], __fmaf_rn(0.587f, f[1], __fmul_rn(0.299f, f[0])));
  uint32_t o[3];
#pragma unroll
  for (int c = 0; c < 3; c++) o[c] = sat_rne_f(__fmaf_rn(s, __fsub_rn(f[c], grey), grey));
  rgb[0] = o[0]; rgb[1] = o[1]; rgb[2] = o[2];
}

// integer BT.601 grey, round half to even: rne((299 R + 587 G + 114 B) / 1000)
ALB_D uint32_t grey_bt601(const uint32_t rgb[3]) {
  const uint32_t num = 299u * rgb[0] + 587u * rgb[1] + 114u * rgb[2];
  uint32_t q = num / 1000u;
  const uint32_t r = num - 1000u * q;
  if (r > 500u || (r == 500u && (q & 1u))) q++;
  return q;
}

// ops [from, to) of the image's order; tb / tc: its B and C tables
ALB_D void jitter_ops(uint32_t rgb[3], int k, int from, int to, const uint8_t* tb, const uint8_t* tc, float s) {
  for (int i = from; i < to; i++) {
    const int op = jitter_op(k, i);
    if (op == 2) {
      jitter_saturate(rgb, s);
    } else {
      const uint8_t* t = op == 0 ? tb : tc;
      rgb[0] = t[rgb[0]]; rgb[1] = t[rgb[1]]; rgb[2] = t[rgb[2]];
    }
  }
}

ALB_D int jitter_pos_c(int k) { return jitter_op(k, 0) == 1 ? 0 : (jitter_op(k, 1) == 1 ? 1 : 2); }

// Per image: B table (which == 0), or the C table from the image's grey sum (which == 1).
__global__ void k_jitter_luts(int32_t n, const alb_params* __restrict__ prm, const unsigned long long* __restrict__ sums,
                              int64_t npx, int32_t which, uint8_t* __restrict__ luts) {
  const int b = blockIdx.x, v = threadIdx.x;
  if (b >= n) return;
  const alb_params& p = prm[b];
  uint8_t* L = luts + (int64_t)b * 512;
  if (which == 0) {
    L[v] = sat_rne_d(p.beta * (double)v);
  } else {
    const uint64_t sum = sums[b];
    uint64_t q = sum / (uint64_t)npx;
    const uint64_t r = sum - q * (uint64_t)npx;
    if (2 * r > (uint64_t)npx || (2 * r == (uint64_t)npx && (q & 1))) q++;
    const double m = (double)q;
    L[256 + v] = sat_rne_d(m + p.alpha * ((double)v - m));
  }
}

// Contrast pivot sums of the fused path: per output pixel the resized value
// with the ops ordered before C applied, its integer grey, summed per image.
// Item = (image, band of rows), grid-stride; flip does not change the sum.
__global__ void __launch_bounds__(256) k_chain_pivot(int32_t n, const alb_params* __restrict__ prm,
                                                     const alb_image* __restrict__ imgs,
                                                     const uint8_t* __restrict__ luts, ChainK K, int32_t band,
                                                     unsigned long long* __restrict__ sums) {
  __shared__ uint8_t s_tb[256];
  __shared__ int32_t s_col[1024];
  __shared__ int32_t s_row[kBandMaxP];
  __shared__ unsigned long long s_part[8];
  const int32_t bands = (K.oh + band - 1) / band;
  const int64_t total = (int64_t)n * bands;
  int32_t cached = -1;
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int32_t b = (int32_t)(item / bands), r0 = (int32_t)(item - (int64_t)b * bands) * band;
    const int32_t r1 = imin(r0 + band, K.oh);
    const alb_params& p = prm[b];
    __syncthreads();
    if (b != cached) {
      for (int i = threadIdx.x; i < 256; i += blockDim.x) s_tb[i] = luts[(int64_t)b * 512 + i];
      for (int x = threadIdx.x; x < K.ow; x += blockDim.x) s_col[x] = chain_q5(x, p.cw, K.ow);
      cached = b;
    }
    if (threadIdx.x < r1 - r0) s_row[threadIdx.x] = chain_q5(r0 + threadIdx.x, p.ch, K.oh);
    __syncthreads();
    const alb_image im = imgs[b];
    const uint8_t* win = (const uint8_t*)im.data + (int64_t)p.y0 * im.row_stride + 3 * (int64_t)p.x0;
    const int pos_c = jitter_pos_c(p.k);
    const float s = (float)p.sat;
    uint32_t acc = 0;       // < 256 * 2 * 32 * 1024 per thread and item: fits 32 bits
    const int32_t hw = (K.ow + 1) >> 1;                 // pixel pairs per row (the last may be single)
    const int32_t npair = (r1 - r0) * hw;
    for (int32_t i = threadIdx.x; i < npair; i += blockDim.x) {
      const int32_t yy = i / hw, x = 2 * (i - yy * hw);
      const int32_t yq = s_row[yy];
      uint32_t a[3];
      chain_bilinear(win, im.row_stride, p.ch, p.cw, s_col[x], yq, a);
      jitter_ops(a, p.k, 0, pos_c, s_tb, s_tb, s);
      acc += grey_bt601(a);
      if (x + 1 < K.ow) {
        uint32_t c[3];
        chain_bilinear(win, im.row_stride, p.ch, p.cw, s_col[x + 1], yq, c);
        jitter_ops(c, p.k, 0, pos_c, s_tb, s_tb, s);
        acc += grey_bt601(c);
      }
    }
    unsigned long long acc64 = acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc64 += __shfl_down_sync(0xffffffffu, acc64, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc64;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_part[w];
      atomicAdd(&sums[b], t);
    }
  }
}

// per-image brightness-then-contrast table c (b v - 128) + 128 (float64, half even)
__global__ void k_chain_luts(int32_t n, const alb_params* __restrict__ prm, uint8_t* __restrict__ luts) {
  const int b = blockIdx.x, v = threadIdx.x;
  if (b >= n) return;
  const alb_params& p = prm[b];
  const double bv = p.beta * (double)v;
  const double d = bv - 128.0;
  const double cd = p.alpha * d;
  luts[(int64_t)b * 256 + v] = sat_rne_d(cd + 128.0);
}

// ---------------------------------------------------------------- fused kernel
// Item = (image, band of `band` output rows), pulled from one global counter.
// Per image the column coordinates (flip folded in) and the colour table live
// in shared memory; per band the row coordinates are computed once.  A thread
// produces two horizontally adjacent pixels, stored as one bf16x2 per channel.

// MODE 0: brightness/contrast table (fixed order, pivot 128), float saturation.
// MODE 1: jitter mode 1 (per-image order; B and C tables [n][512]; uint8 after each op).
// Instance-mask stacks of the chain: valid when the masks match the image and
// the output masks have the chain's output size and the same plane count.
ALB_D bool chain_mask_ok(const alb_image& im, const alb_image& mi, const alb_image& mo, const ChainK& K) {
  return mi.h == im.h && mi.w == im.w && mi.c >= 1 && mo.c == mi.c && mo.h == K.oh && mo.w == K.ow &&
         mi.row_stride >= (int64_t)mi.w * mi.c && mo.row_stride >= (int64_t)mo.w * mo.c && mi.data && mo.data;
}

ALB_D int32_t chain_nn(int32_t d, int32_t n_in, int32_t n_out) {   // nearest rule of the mask resize
  const int64_t i = ((int64_t)(2 * d + 1) * n_in) / (2 * (int64_t)n_out);
  return (int32_t)(i < n_in - 1 ? i : n_in - 1);
}

// rows [r0, r1) of image b's mask stack (nearest, flip folded into the column table)
ALB_D void chain_mask_rows(const alb_params& p, const alb_image& mi, const alb_image& mo, const int32_t* cnn,
                           const int32_t* rnn, int32_t r0, int32_t r1, int32_t ow) {
  const int32_t C = mi.c;
  const int32_t npx = (r1 - r0) * ow;        // at most 32 rows x 1024 columns
  const uint8_t* src = (const uint8_t*)mi.data + (int64_t)p.y0 * mi.row_stride + (int64_t)p.x0 * C;
  for (int32_t i = threadIdx.x; i < npx; i += blockDim.x) {
    const int32_t yy = i / ow, x = i - yy * ow;
    const uint8_t* s = src + (int64_t)rnn[yy] * mi.row_stride + (int64_t)cnn[x] * C;
    uint8_t* d = (uint8_t*)mo.data + (int64_t)(r0 + yy) * mo.row_stride + (int64_t)x * C;
    if (C == 1) {
      *d = __ldg(s);
    } else {
      for (int32_t c = 0; c < C; c++) d[c] = __ldg(s + c);
    }
  }
}

template <int MODE, bool MASKS>
__global__ void __launch_bounds__(256) k_chain_fused(int32_t n, const alb_params* __restrict__ prm,
                                                     const alb_image* __restrict__ imgs,
                                                     const uint8_t* __restrict__ luts, ChainK K, int32_t band,
                                                     int32_t* __restrict__ queue, __nv_bfloat16* __restrict__ out,
                                                     const alb_image* __restrict__ mask_in,
                                                     const alb_image* __restrict__ mask_out, int32_t* status) {
  constexpr int TAB = MODE == 0 ? 256 : 512;
  __shared__ int32_t s_item;
  __shared__ uint8_t s_lut[TAB];
  __shared__ int32_t s_col[1024];
  __shared__ int32_t s_row[kBandMax];
  __shared__ const uint8_t* s_ra[kBandMax];   // per band row: the window's two tap rows
  __shared__ const uint8_t* s_rb[kBandMax];
  __shared__ int32_t s_cnn[1024];      // masks: nearest source column of each output column (flip folded)
  __shared__ int32_t s_rnn[kBandMax];
  const int32_t bands = (K.oh + band - 1) / band;
  const int64_t total = (int64_t)n * bands;
  const int64_t plane = (int64_t)K.oh * K.ow;
  const bool pairs = (K.ow & 1) == 0;
  int32_t cached = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int32_t item = s_item;
    if (item >= total) break;
    const int32_t b = item / bands, r0 = (item - b * bands) * band, r1 = imin(r0 + band, K.oh);
    const alb_params& p = prm[b];
    if (b != cached) {
      for (int i = threadIdx.x; i < TAB; i += blockDim.x) s_lut[i] = luts[(int64_t)b * TAB + i];
      for (int x = threadIdx.x; x < K.ow; x += blockDim.x) {
        const int32_t xr = p.flip ? K.ow - 1 - x : x;  // output column x shows resized column xr
        s_col[x] = chain_q5(xr, p.cw, K.ow);
        if (MASKS) s_cnn[x] = chain_nn(xr, p.cw, K.ow);
      }
      cached = b;
    }
    const alb_image im = imgs[b];
    const uint8_t* win = (const uint8_t*)im.data + (int64_t)p.y0 * im.row_stride + 3 * (int64_t)p.x0;
    if (threadIdx.x < r1 - r0) {
      const int32_t yq = chain_q5(r0 + threadIdx.x, p.ch, K.oh), iy = yq >> 5;
      s_row[threadIdx.x] = yq;
      s_ra[threadIdx.x] = win + (int64_t)iy * im.row_stride;
      s_rb[threadIdx.x] = win + (int64_t)imin(iy + 1, p.ch - 1) * im.row_stride;
      if (MASKS) s_rnn[threadIdx.x] = chain_nn(r0 + threadIdx.x, p.ch, K.oh);
    }
    __syncthreads();
    const float s = (float)p.sat;
    __nv_bfloat16* ob = out + (int64_t)b * 3 * plane;
    if (pairs) {
      const int32_t hw = K.ow >> 1;
      const int32_t npair = (r1 - r0) * hw;
      // pair i = (band row yy, pair column xp), advanced by blockDim.x pairs a
      // step without dividing
      const int32_t dyy = (int32_t)blockDim.x / hw, dxp = (int32_t)blockDim.x - dyy * hw;
      int32_t yy = (int32_t)threadIdx.x / hw, xp = (int32_t)threadIdx.x - yy * hw;
      for (int32_t i = threadIdx.x; i < npair; i += blockDim.x) {
        const int32_t x = 2 * xp, y = r0 + yy;
        const int32_t fy = s_row[yy] & 31;
        const uint8_t* ra = s_ra[yy];
        const uint8_t* rb = s_rb[yy];
        xp += dxp; yy += dyy;
        if (xp >= hw) { xp -= hw; yy++; }
        uint32_t a[3], c[3];
        chain_bilerp(ra, rb, p.cw, s_col[x], fy, a);
        chain_bilerp(ra, rb, p.cw, s_col[x + 1], fy, c);
        float va[3], vc[3];
        if (MODE == 0) {
#pragma unroll
          for (int q = 0; q < 3; q++) { a[q] = s_lut[a[q]]; c[q] = s_lut[c[q]]; }
          chain_saturate(a, s, va);
          chain_saturate(c, s, vc);
        } else {
          jitter_ops(a, p.k, 0, 3, s_lut, s_lut + 256, s);
          jitter_ops(c, p.k, 0, 3, s_lut, s_lut + 256, s);
#pragma unroll
          for (int q = 0; q < 3; q++) { va[q] = u8f(a[q]); vc[q] = u8f(c[q]); }
        }
        const int64_t o = (int64_t)y * K.ow + x;
        if (!ALB_IN(y < K.oh && x + 1 < K.ow)) continue;
#pragma unroll
        for (int q = 0; q < 3; q++)   // both values rounded to bf16 by one packing conversion
          *reinterpret_cast<__nv_bfloat162*>(ob + q * plane + o) =
              __floats2bfloat162_rn(__fmaf_rn(va[q], K.k[q], K.m[q]), __fmaf_rn(vc[q], K.k[q], K.m[q]));
      }
    } else {
      const int32_t npx = (r1 - r0) * K.ow;
      for (int32_t i = threadIdx.x; i < npx; i += blockDim.x) {
        const int32_t yy = i / K.ow, x = i - yy * K.ow, y = r0 + yy;
        uint32_t rgb[3];
        chain_bilinear(win, im.row_stride, p.ch, p.cw, s_col[x], s_row[yy], rgb);
        float v[3];
        if (MODE == 0) {
#pragma unroll
          for (int q = 0; q < 3; q++) rgb[q] = s_lut[rgb[q]];
          chain_saturate(rgb, s, v);
        } else {
          jitter_ops(rgb, p.k, 0, 3, s_lut, s_lut + 256, s);
#pragma unroll
          for (int q = 0; q < 3; q++) v[q] = (float)rgb[q];
        }
        if (ALB_IN(y < K.oh && x < K.ow)) {
#pragma unroll
          for (int q = 0; q < 3; q++) ob[q * plane + (int64_t)y * K.ow + x] = chain_normalize(v[q], K.k[q], K.m[q]);
        }
      }
    }
    if (MASKS) {
      const alb_image mi = mask_in[b], mo = mask_out[b];
      if (chain_mask_ok(im, mi, mo, K)) chain_mask_rows(p, mi, mo, s_cnn, s_rnn, r0, r1, K.ow);
      else if (threadIdx.x == 0 && r0 == 0) dev_fail(status, ALB_ESHAPE);
    }
    __syncthreads();
  }
}

// Jitter mode 1 with the image held on chip: one CTA per image (pulled from a
// counter, one CTA per SM), the whole resized output image kept in shared
// memory between the two halves of the chain.  Pass 1: per output pixel the
// Q5 bilinear value with the ops ordered before contrast applied (uint8,
// stored unflipped), its integer BT.601 grey summed over the image; the
// image's C table from that pivot (the float64 rule of k_jitter_luts); pass 2:
// the remaining ops, the flip, Normalize and bf16 NCHW stores, from shared
// memory.  The source crop is read once and nothing is recomputed; the
// results are those of k_chain_pivot + k_jitter_luts + k_chain_fused<1>.
// Instance-mask stacks are copied in the same pass.
constexpr int kJitImgMax = 3 * 256 * 256;    // shared-memory image bytes, at most

template <bool MASKS>
__global__ void __launch_bounds__(1024, 1) k_chain_jitter_img(int32_t n, const alb_params* __restrict__ prm,
                                                              const alb_image* __restrict__ imgs,
                                                              const uint8_t* __restrict__ luts, ChainK K,
                                                              int32_t* __restrict__ queue,
                                                              __nv_bfloat16* __restrict__ out,
                                                              const alb_image* __restrict__ mask_in,
                                                              const alb_image* __restrict__ mask_out,
                                                              int32_t* status) {
  extern __shared__ __align__(16) uint8_t s_img[];
  __shared__ int32_t s_item;
  __shared__ uint8_t s_tb[256], s_tc[256];
  __shared__ int32_t s_col[1024], s_row[1024];
  __shared__ int32_t s_cnn[MASKS ? 1024 : 1], s_rnn[MASKS ? 1024 : 1];
  __shared__ unsigned long long s_part[32];
  const int tid = threadIdx.x, bs = blockDim.x;
  const int32_t OW = K.ow, OH = K.oh;
  const int64_t plane = (int64_t)OH * OW;
  const int32_t hw = (OW + 1) >> 1;                   // pixel pairs per row (the last may be single)
  const bool pairs = (OW & 1) == 0;                    // bf16x2 stores stay 4-byte aligned
  for (;;) {
    if (tid == 0) s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int32_t b = s_item;
    if (b >= n) break;
    const alb_params& p = prm[b];
    for (int i = tid; i < 256; i += bs) s_tb[i] = luts[(int64_t)b * 512 + i];
    for (int x = tid; x < OW; x += bs) {
      s_col[x] = chain_q5(x, p.cw, OW);
      if (MASKS) s_cnn[x] = chain_nn(p.flip ? OW - 1 - x : x, p.cw, OW);
    }
    for (int y = tid; y < OH; y += bs) {
      s_row[y] = chain_q5(y, p.ch, OH);
      if (MASKS) s_rnn[y] = chain_nn(y, p.ch, OH);
    }
    __syncthreads();
    const alb_image im = imgs[b];
    const uint8_t* win = (const uint8_t*)im.data + (int64_t)p.y0 * im.row_stride + 3 * (int64_t)p.x0;
    const int pos_c = jitter_pos_c(p.k);
    const float s = (float)p.sat;
    // ---- pass 1: ops before contrast, grey sum
    uint32_t acc = 0;        // at most 32 pairs of 2 * 255 per thread for images <= 256 x 256
    const int32_t npair = OH * hw;
    const int32_t dyy = bs / hw, dxp = bs - dyy * hw;   // pair indices advanced without division
    int32_t py = tid / hw, pxp = tid - py * hw;
    for (int32_t i = tid; i < npair; i += bs) {
      const int32_t y = py, x = 2 * pxp;
      pxp += dxp; py += dyy;
      if (pxp >= hw) { pxp -= hw; py++; }
      const int32_t yq = s_row[y], iy = yq >> 5;
      const uint8_t* ra = win + (int64_t)iy * im.row_stride;
      const uint8_t* rb = win + (int64_t)imin(iy + 1, p.ch - 1) * im.row_stride;
      uint8_t* d = s_img + 3 * (y * OW + x);
      uint32_t a[3];
      chain_bilerp(ra, rb, p.cw, s_col[x], yq & 31, a);
      jitter_ops(a, p.k, 0, pos_c, s_tb, s_tb, s);
      acc += grey_bt601(a);
      d[0] = (uint8_t)a[0]; d[1] = (uint8_t)a[1]; d[2] = (uint8_t)a[2];
      if (x + 1 < OW) {
        uint32_t c[3];
        chain_bilerp(ra, rb, p.cw, s_col[x + 1], yq & 31, c);
        jitter_ops(c, p.k, 0, pos_c, s_tb, s_tb, s);
        acc += grey_bt601(c);
        d[3] = (uint8_t)c[0]; d[4] = (uint8_t)c[1]; d[5] = (uint8_t)c[2];
      }
    }
    unsigned long long acc64 = acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc64 += __shfl_down_sync(0xffffffffu, acc64, o);
    if ((tid & 31) == 0) s_part[tid >> 5] = acc64;
    __syncthreads();
    // ---- the image's C table from its pivot
    if (tid < 256) {
      unsigned long long sum = 0;
      for (int w = 0; w < (bs >> 5); w++) sum += s_part[w];
      const uint64_t np = (uint64_t)plane;
      uint64_t q = sum / np;
      const uint64_t r = sum - q * np;
      if (2 * r > np || (2 * r == np && (q & 1))) q++;
      const double m = (double)q;
      s_tc[tid] = sat_rne_d(m + p.alpha * ((double)tid - m));
    }
    __syncthreads();
    // ---- pass 2: the remaining ops, flip, Normalize, bf16 NCHW
    __nv_bfloat16* ob = out + (int64_t)b * 3 * plane;
    py = tid / hw; pxp = tid - py * hw;
    for (int32_t i = tid; i < npair; i += bs) {
      const int32_t y = py, x = 2 * pxp;
      pxp += dxp; py += dyy;
      if (pxp >= hw) { pxp -= hw; py++; }
      const bool two = x + 1 < OW;
      const int32_t xa = p.flip ? OW - 1 - x : x, xb = p.flip ? OW - 2 - x : x + 1;   // resized columns shown
      const uint8_t* sa = s_img + 3 * ((int64_t)y * OW + xa);
      uint32_t a[3] = {sa[0], sa[1], sa[2]};
      jitter_ops(a, p.k, pos_c, 3, s_tb, s_tc, s);
      const int64_t o = (int64_t)y * OW + x;
      if (!ALB_IN(y < OH && x < OW)) continue;
      if (two) {
        const uint8_t* sb = s_img + 3 * ((int64_t)y * OW + xb);
        uint32_t c[3] = {sb[0], sb[1], sb[2]};
        jitter_ops(c, p.k, pos_c, 3, s_tb, s_tc, s);
        if (pairs) {
#pragma unroll
          for (int q = 0; q < 3; q++)
            *reinterpret_cast<__nv_bfloat162*>(ob + q * plane + o) =
                __floats2bfloat162_rn(__fmaf_rn(u8f(a[q]), K.k[q], K.m[q]), __fmaf_rn(u8f(c[q]), K.k[q], K.m[q]));
        } else {
#pragma unroll
          for (int q = 0; q < 3; q++) {
            ob[q * plane + o] = chain_normalize((float)a[q], K.k[q], K.m[q]);
            ob[q * plane + o + 1] = chain_normalize((float)c[q], K.k[q], K.m[q]);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < 3; q++) ob[q * plane + o] = chain_normalize((float)a[q], K.k[q], K.m[q]);
      }
    }
    if (MASKS) {
      const alb_image mi = mask_in[b], mo = mask_out[b];
      if (chain_mask_ok(im, mi, mo, K)) chain_mask_rows(p, mi, mo, s_cnn, s_rnn, 0, OH, OW);
      else if (tid == 0) dev_fail(status, ALB_ESHAPE);
    }
    __syncthreads();
  }
}

// Masks of the chain on their own (the plain path): item = (image, band of 32 rows), grid-stride.
__global__ void __launch_bounds__(256) k_chain_masks(int32_t n, const alb_params* __restrict__ prm,
                                                     const alb_image* __restrict__ imgs, ChainK K,
                                                     const alb_image* __restrict__ mask_in,
                                                     const alb_image* __restrict__ mask_out, int32_t* status) {
  __shared__ int32_t s_cnn[1024];
  __shared__ int32_t s_rnn[32];
  const int32_t bands = (K.oh + 31) / 32;
  int32_t cached = -1;
  for (int64_t item = blockIdx.x; item < (int64_t)n * bands; item += gridDim.x) {
    const int32_t b = (int32_t)(item / bands), r0 = (int32_t)(item - (int64_t)b * bands) * 32;
    const int32_t r1 = imin(r0 + 32, K.oh);
    const alb_params& p = prm[b];
    const alb_image im = imgs[b], mi = mask_in[b], mo = mask_out[b];
    const bool ok = chain_mask_ok(im, mi, mo, K);
    __syncthreads();
    if (ok && b != cached) {
      for (int x = threadIdx.x; x < K.ow; x += blockDim.x) s_cnn[x] = chain_nn(p.flip ? K.ow - 1 - x : x, p.cw, K.ow);
      cached = b;
    }
    if (threadIdx.x < r1 - r0) s_rnn[threadIdx.x] = chain_nn(r0 + threadIdx.x, p.ch, K.oh);
    __syncthreads();
    if (ok) chain_mask_rows(p, mi, mo, s_cnn, s_rnn, r0, r1, K.ow);
    else if (threadIdx.x == 0 && r0 == 0) dev_fail(status, ALB_ESHAPE);
  }
}

// Boxes of the chain: one warp per image; crop to the window (clip there),
// scale, flip, clip to the output, drop empty boxes, compact in order.
__global__ void k_chain_boxes(int32_t n, const alb_params* __restrict__ prm, ChainK K, const float* __restrict__ boxes,
                              const int32_t* __restrict__ nbox, int32_t cap, float* __restrict__ out,
                              int32_t* __restrict__ nout, int32_t* status) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= n) return;
  const alb_params& p = prm[b];
  const int32_t oh = K.oh, ow = K.ow;
  int32_t cnt = nbox[b];
  if (cnt > cap || cnt < 0) { if (lane == 0) dev_fail(status, ALB_ECAPACITY); cnt = cnt < 0 ? 0 : cap; }
  const float* bin = boxes + (int64_t)b * cap * 4;
  float* bout = out + (int64_t)b * cap * 4;
  int32_t kept_total = 0;
  for (int base = 0; base < cnt; base += 32) {
    const int i = base + lane;
    double a1 = 0, b1 = 0, a2 = 0, b2 = 0;
    bool keep = false;
    if (i < cnt) {
      double cx1 = bin[4 * i] - p.x0, cy1 = bin[4 * i + 1] - p.y0, cx2 = bin[4 * i + 2] - p.x0, cy2 = bin[4 * i + 3] - p.y0;
      if (cx1 < 0) cx1 = 0;
      if (cy1 < 0) cy1 = 0;
      if (cx2 > p.cw) cx2 = p.cw;
      if (cy2 > p.ch) cy2 = p.ch;
      a1 = cx1 * ow / p.cw; a2 = cx2 * ow / p.cw; b1 = cy1 * oh / p.ch; b2 = cy2 * oh / p.ch;
      if (p.flip) { const double t = a1; a1 = (double)ow - a2; a2 = (double)ow - t; }
      if (a1 < 0) a1 = 0;
      if (b1 < 0) b1 = 0;
      if (a2 > ow) a2 = ow;
      if (b2 > oh) b2 = oh;
      keep = !(a2 - a1 <= 0.0 || b2 - b1 <= 0.0);
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int slot = kept_total + __popc(m & ((1u << lane) - 1u));
      bout[4 * slot] = (float)a1; bout[4 * slot + 1] = (float)b1;
      bout[4 * slot + 2] = (float)a2; bout[4 * slot + 3] = (float)b2;
    }
    kept_total += __popc(m);
  }
  if (lane == 0) nout[b] = kept_total;
}

// ---------------------------------------------------------------- plain path
// The comparison path runs one step per launch through the library's own
// per-transform machinery, every intermediate materialised:
//   crop + resize  -> the ragged RandomResizedCrop launch (tile plan +
//                     k_resize_rows) into uint8 224 x 224 images,
//   h-flip         -> the ragged HorizontalFlip launch (k_pixmap3),
//   colour table   -> the bulk-copy LUT kernel (k_lut_bulk) with the chain's
//                     per-image tables,
//   saturation     -> uint8 -> float32 (mode 0) or the jitter steps uint8 ->
//                     uint8 (mode 1), 16-byte vectors,
//   Normalize      -> float32 / uint8 HWC -> bf16 NCHW, 16-byte vectors.
// The per-step kernels below take one image per grid row (blockIdx.y), so
// per-image constants are loaded once and no pixel index is divided; images
// whose plane is a multiple of 16 pixels take the vector path, others one
// pixel per thread.  Same rounding points as the fused kernel, so the output
// is identical.

// per image: the step records of the per-transform launches and the
// descriptors of the two uint8 intermediates
__global__ void k_plain_records(int32_t n, const alb_params* __restrict__ prm, ChainK K, uint8_t* a, uint8_t* b,
                                alb_params* __restrict__ rrc, alb_params* __restrict__ flip,
                                alb_params* __restrict__ lut, alb_image* __restrict__ da,
                                alb_image* __restrict__ db) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const alb_params p = prm[i];
  alb_params r = p;
  r.tid = ALB_RANDOM_RESIZED_CROP; r.apply = 1; r.out_h = K.oh; r.out_w = K.ow;
  rrc[i] = r;
  alb_params f = p;
  f.tid = ALB_HFLIP; f.apply = p.flip != 0; f.in_h = f.out_h = K.oh; f.in_w = f.out_w = K.ow;
  flip[i] = f;
  alb_params l = p;
  l.tid = ALB_BRIGHTNESS_CONTRAST; l.apply = 1; l.in_h = l.out_h = K.oh; l.in_w = l.out_w = K.ow;
  lut[i] = l;
  const int64_t plane = (int64_t)K.oh * K.ow * 3;
  alb_image im;
  im.h = K.oh; im.w = K.ow; im.c = 3; im.reserved = 0; im.row_stride = 3 * (int64_t)K.ow;
  im.data = a + (int64_t)i * plane;
  da[i] = im;
  im.data = b + (int64_t)i * plane;
  db[i] = im;
}

// the chain's colour table of each image, replicated for the three channels
// (the layout of the LUT kernel's per-image tables)
__global__ void k_plain_luts768(int32_t n, const uint8_t* __restrict__ luts256, uint8_t* __restrict__ luts768) {
  const int b = blockIdx.x, v = threadIdx.x;
  if (b >= n) return;
  const uint8_t t = luts256[(int64_t)b * 256 + v];
  uint8_t* o = luts768 + (int64_t)b * 768;
  o[v] = t; o[256 + v] = t; o[512 + v] = t;
}

ALB_D void ld48(const uint8_t* p, uint8_t (&v)[48]) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const uint4 t = q[k];
    const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int j = 0; j < 16; j++) v[16 * k + j] = (uint8_t)(w[j >> 2] >> (8 * (j & 3)));
  }
}

ALB_D void st48(uint8_t* p, const uint8_t (&v)[48]) {
  uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < 16; j++) w[j >> 2] |= (uint32_t)v[16 * k + j] << (8 * (j & 3));
    q[k] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// mode 0 saturation: uint8 RGB -> float32 blend (clamped, not rounded); four
// pixels a thread (three input words, three float4 outputs), consecutive
// threads on consecutive pixels so that a warp's stores cover 1.5 KB
__global__ void __launch_bounds__(256) k_plain_saturate(int32_t n, const alb_params* __restrict__ prm, int64_t P,
                                                        const uint8_t* __restrict__ in, float* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int b = blockIdx.y; b < n; b += gridDim.y) {
    const float s = (float)prm[b].sat;
    const uint8_t* ib = in + (int64_t)b * P * 3;
    float* ob = out + (int64_t)b * P * 3;
    if ((P & 15) == 0) {
      const uint32_t* iw = reinterpret_cast<const uint32_t*>(ib);
      float4* o4 = reinterpret_cast<float4*>(ob);
      for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < P / 4; g += stride) {
        const uint32_t w0 = __ldg(iw + 3 * g), w1 = __ldg(iw + 3 * g + 1), w2 = __ldg(iw + 3 * g + 2);
        const uint32_t w[3] = {w0, w1, w2};
        float f[12];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const uint32_t rgb[3] = {(w[(3 * j) >> 2] >> (8 * ((3 * j) & 3))) & 0xFFu,
                                   (w[(3 * j + 1) >> 2] >> (8 * ((3 * j + 1) & 3))) & 0xFFu,
                                   (w[(3 * j + 2) >> 2] >> (8 * ((3 * j + 2) & 3))) & 0xFFu};
          chain_saturate(rgb, s, f + 3 * j);
        }
        o4[3 * g] = make_float4(f[0], f[1], f[2], f[3]);
        o4[3 * g + 1] = make_float4(f[4], f[5], f[6], f[7]);
        o4[3 * g + 2] = make_float4(f[8], f[9], f[10], f[11]);
      }
    } else {
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
        const uint32_t rgb[3] = {ib[3 * i], ib[3 * i + 1], ib[3 * i + 2]};
        chain_saturate(rgb, s, ob + 3 * i);
      }
    }
  }
}

// Normalize: float32 HWC -> bf16 NCHW
__global__ void __launch_bounds__(256) k_plain_normalize(int32_t n, ChainK K, int64_t P, const float* __restrict__ in,
                                                         __nv_bfloat16* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int b = blockIdx.y; b < n; b += gridDim.y) {
    const float* ib = in + (int64_t)b * P * 3;
    __nv_bfloat16* ob = out + (int64_t)b * 3 * P;
    if ((P & 7) == 0) {
      for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < P / 8; g += stride) {
        const float4* i4 = reinterpret_cast<const float4*>(ib + 24 * g);
        float f[24];
#pragma unroll
        for (int q = 0; q < 6; q++) {
          const float4 t = i4[q];
          f[4 * q] = t.x; f[4 * q + 1] = t.y; f[4 * q + 2] = t.z; f[4 * q + 3] = t.w;
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 4; j++) {
            const __nv_bfloat16 lo = chain_normalize(f[3 * (2 * j) + c], K.k[c], K.m[c]);
            const __nv_bfloat16 hi = chain_normalize(f[3 * (2 * j + 1) + c], K.k[c], K.m[c]);
            w[j] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
          }
          *reinterpret_cast<uint4*>(ob + (int64_t)c * P + 8 * g) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
    } else {
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride)
        for (int c = 0; c < 3; c++) ob[(int64_t)c * P + i] = chain_normalize(ib[3 * i + c], K.k[c], K.m[c]);
    }
  }
}

// jitter mode 1: contrast-pivot sums (integer BT.601 grey) of the images
// whose op at position `step` is C, one block reduction and one atomic per
// block
__global__ void __launch_bounds__(256) k_plain_pivot(int32_t n, const alb_params* __restrict__ prm, int64_t P,
                                                     int32_t step, const uint8_t* __restrict__ in,
                                                     unsigned long long* __restrict__ sums) {
  __shared__ uint32_t red[8];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int b = blockIdx.y; b < n; b += gridDim.y) {
    if (jitter_op(prm[b].k, step) != 1) continue;         // block-uniform
    const uint8_t* ib = in + (int64_t)b * P * 3;
    uint32_t acc = 0;
    if ((P & 15) == 0) {
      for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < P / 16; g += stride) {
        uint8_t v[48];
        ld48(ib + 48 * g, v);
#pragma unroll
        for (int j = 0; j < 16; j++) {
          const uint32_t rgb[3] = {v[3 * j], v[3 * j + 1], v[3 * j + 2]};
          acc += grey_bt601(rgb);
        }
      }
    } else {
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
        const uint32_t rgb[3] = {ib[3 * i], ib[3 * i + 1], ib[3 * i + 2]};
        acc += grey_bt601(rgb);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
      if (t) atomicAdd(&sums[b], t);
    }
    __syncthreads();
  }
}

// jitter mode 1: each image's op at position `step` (B or C through its
// table, S as the rounded float32 blend), uint8 -> uint8
__global__ void __launch_bounds__(256) k_plain_jitter_step(int32_t n, const alb_params* __restrict__ prm, int64_t P,
                                                           int32_t step, const uint8_t* __restrict__ luts,
                                                           const uint8_t* __restrict__ in, uint8_t* __restrict__ out) {
  __shared__ uint8_t tab[256];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int b = blockIdx.y; b < n; b += gridDim.y) {
    const alb_params& p = prm[b];
    const int op = jitter_op(p.k, step);
    const float s = (float)p.sat;
    __syncthreads();
    if (op != 2) tab[threadIdx.x] = luts[(int64_t)b * 512 + (op == 1 ? 256 : 0) + threadIdx.x];
    __syncthreads();
    const uint8_t* ib = in + (int64_t)b * P * 3;
    uint8_t* ob = out + (int64_t)b * P * 3;
    if ((P & 15) == 0) {
      for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < P / 16; g += stride) {
        uint8_t v[48];
        ld48(ib + 48 * g, v);
        if (op == 2) {
#pragma unroll
          for (int j = 0; j < 16; j++) {
            uint32_t rgb[3] = {v[3 * j], v[3 * j + 1], v[3 * j + 2]};
            jitter_saturate(rgb, s);
            v[3 * j] = (uint8_t)rgb[0]; v[3 * j + 1] = (uint8_t)rgb[1]; v[3 * j + 2] = (uint8_t)rgb[2];
          }
        } else {
#pragma unroll
          for (int j = 0; j < 48; j++) v[j] = tab[v[j]];
        }
        st48(ob + 48 * g, v);
      }
    } else {
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
        uint32_t rgb[3] = {ib[3 * i], ib[3 * i + 1], ib[3 * i + 2]};
        if (op == 2) jitter_saturate(rgb, s);
        else { rgb[0] = tab[rgb[0]]; rgb[1] = tab[rgb[1]]; rgb[2] = tab[rgb[2]]; }
        for (int c = 0; c < 3; c++) ob[3 * i + c] = (uint8_t)rgb[c];
      }
    }
  }
}

// jitter mode 1 Normalize: uint8 HWC -> bf16 NCHW
__global__ void __launch_bounds__(256) k_plain_normalize_u8(int32_t n, ChainK K, int64_t P,
                                                            const uint8_t* __restrict__ in,
                                                            __nv_bfloat16* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int b = blockIdx.y; b < n; b += gridDim.y) {
    const uint8_t* ib = in + (int64_t)b * P * 3;
    __nv_bfloat16* ob = out + (int64_t)b * 3 * P;
    if ((P & 15) == 0) {
      for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < P / 16; g += stride) {
        uint8_t v[48];
        ld48(ib + 48 * g, v);
#pragma unroll
        for (int c = 0; c < 3; c++) {
          uint32_t w[8];
#pragma unroll
          for (int j = 0; j < 8; j++) {
            const __nv_bfloat16 lo = chain_normalize((float)v[3 * (2 * j) + c], K.k[c], K.m[c]);
            const __nv_bfloat16 hi = chain_normalize((float)v[3 * (2 * j + 1) + c], K.k[c], K.m[c]);
            w[j] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
          }
          uint4* o4 = reinterpret_cast<uint4*>(ob + (int64_t)c * P + 16 * g);
          o4[0] = make_uint4(w[0], w[1], w[2], w[3]);
          o4[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
      }
    } else {
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride)
        for (int c = 0; c < 3; c++) ob[(int64_t)c * P + i] = chain_normalize((float)ib[3 * i + c], K.k[c], K.m[c]);
    }
  }
}

// grid of the per-image step kernels: enough blocks per image to give every
// thread about one 16-pixel group, images on the grid's y axis
static dim3 plain_grid(int32_t n, int64_t P, int32_t px_per_thread = 16) {
  const int64_t groups = (P + px_per_thread - 1) / px_per_thread;
  const int64_t bx = (groups + 255) / 256;
  return dim3((unsigned)(bx < 1 ? 1 : (bx > 1024 ? 1024 : bx)), (unsigned)(n < 65535 ? n : 65535));
}
// ---------------------------------------------------------------- launcher
constexpr int32_t kPlainItemBytes = 16384;   // output bytes per work item of the plain path's ragged launches

size_t chain_workspace(const alb_chain_cfg& cfg, int32_t n, int32_t mode) {
  size_t px = (size_t)n * cfg.out_h * cfg.out_w;
  size_t b = 4096 + (size_t)n * 512 + (size_t)n * 8 + 512;   // queue, tables, pivot sums
  if (mode == ALB_MODE_PLAIN)   // intermediates, step records, descriptors, plan, 3-channel tables
    b += 2 * px * 3 + px * 3 * 4 + (size_t)n * 3 * sizeof(alb_params) + (size_t)n * 2 * sizeof(alb_image) +
         (size_t)(4 * n + 2) * 4 + (size_t)n * 768 + 10 * 256;
  return b;
}

static ChainK make_consts(const alb_chain_cfg& cfg) {
  ChainK K;
  for (int c = 0; c < 3; c++) {
    K.k[c] = (float)(1.0 / (255.0 * cfg.std[c]));
    K.m[c] = (float)(-cfg.mean[c] / cfg.std[c]);
  }
  K.oh = cfg.out_h;
  K.ow = cfg.out_w;
  return K;
}

// ---------------------------------------------------------------- schedule cache
// A schedule of the fused kernel is (rows per work item, resident CTAs per
// SM).  alb_autotune_batch times candidates on the caller's batch and keeps
// the fastest here, per (device, out_h, out_w, jitter mode, batch-size bucket
// = ceil(log2 n));
// a cfg with tile_h == 0 and ctas_per_sm == 0 runs with the cached schedule
// of its key, or the default (8 rows, occupancy limit) when there is none.
struct TuneEntry {
  int32_t dev, oh, ow, jitter, bucket;
  int32_t band, per_sm;
};
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;

static int32_t size_bucket(int32_t n) {
  int32_t b = 0;
  while (b < 31 && (int64_t(1) << b) < n) b++;
  return b;
}

static bool tune_lookup(int32_t dev, const alb_chain_cfg& cfg, int32_t n, int32_t& band, int32_t& per_sm) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const int32_t bk = size_bucket(n);
  for (const TuneEntry& e : g_tune)
    if (e.dev == dev && e.oh == cfg.out_h && e.ow == cfg.out_w && e.jitter == cfg.jitter && e.bucket == bk) {
      band = e.band;
      per_sm = e.per_sm;
      return true;
    }
  return false;
}

static void tune_store(int32_t dev, const alb_chain_cfg& cfg, int32_t n, int32_t band, int32_t per_sm) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const int32_t bk = size_bucket(n);
  for (TuneEntry& e : g_tune)
    if (e.dev == dev && e.oh == cfg.out_h && e.ow == cfg.out_w && e.jitter == cfg.jitter && e.bucket == bk) {
      e.band = band;
      e.per_sm = per_sm;
      return;
    }
  g_tune.push_back(TuneEntry{dev, cfg.out_h, cfg.out_w, cfg.jitter, bk, band, per_sm});
}

// ---- persistence of the schedule cache (JSON), keyed by device name and SM
// count instead of the process-local ordinal:
//   {"format": "alb-autotune-1", "entries": [{"device": "...", "sms": 152,
//    "out_h": 224, "out_w": 224, "jitter": 0, "bucket": 12,
//    "rows_per_item": 32, "ctas_per_sm": 6}, ...]}
struct TuneRecord {
  std::string device;
  int32_t sms = -1, oh = -1, ow = -1, jitter = -1, bucket = -1, band = -1, per_sm = -1;
};

static bool device_key(int dev, std::string& name, int32_t& sms) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return false;
  name.clear();
  for (const char* c = prop.name; *c && name.size() < 255; c++) name += (*c == '"' || *c == '\\') ? '_' : *c;
  sms = prop.multiProcessorCount;
  return true;
}

// A small reader for the format above: an object whose "entries" member is an
// array of flat objects with string or integer members.  Returns false on
// anything else.
struct JsonReader {
  const std::string& t;
  size_t i = 0;
  explicit JsonReader(const std::string& text) : t(text) {}
  void ws() { while (i < t.size() && (t[i] == ' ' || t[i] == '\n' || t[i] == '\r' || t[i] == '\t')) i++; }
  bool lit(char c) { ws(); if (i < t.size() && t[i] == c) { i++; return true; } return false; }
  bool str(std::string& out) {
    ws();
    if (i >= t.size() || t[i] != '"') return false;
    out.clear();
    for (i++; i < t.size() && t[i] != '"'; i++) {
      if (t[i] == '\\' || out.size() > 255) return false;
      out += t[i];
    }
    if (i >= t.size()) return false;
    i++;
    return true;
  }
  bool integer(int64_t& v) {
    ws();
    size_t j = i;
    bool neg = false;
    if (j < t.size() && t[j] == '-') { neg = true; j++; }
    if (j >= t.size() || t[j] < '0' || t[j] > '9') return false;
    int64_t x = 0;
    for (; j < t.size() && t[j] >= '0' && t[j] <= '9'; j++) {
      x = 10 * x + (t[j] - '0');
      if (x > (int64_t(1) << 40)) return false;
    }
    i = j;
    v = neg ? -x : x;
    return true;
  }
  bool record(TuneRecord& r) {
    if (!lit('{')) return false;
    if (lit('}')) return true;
    do {
      std::string key;
      if (!str(key) || !lit(':')) return false;
      if (key == "device") {
        if (!str(r.device)) return false;
        continue;
      }
      int64_t v = 0;
      if (!integer(v)) return false;
      const int32_t x = (int32_t)v;
      if (key == "sms") r.sms = x;
      else if (key == "out_h") r.oh = x;
      else if (key == "out_w") r.ow = x;
      else if (key == "jitter") r.jitter = x;
      else if (key == "bucket") r.bucket = x;
      else if (key == "rows_per_item") r.band = x;
      else if (key == "ctas_per_sm") r.per_sm = x;
      else return false;
    } while (lit(','));
    return lit('}');
  }
  bool document(std::vector<TuneRecord>& out, std::string& format) {
    if (!lit('{')) return false;
    bool have_entries = false;
    if (!lit('}')) {
      do {
        std::string key;
        if (!str(key) || !lit(':')) return false;
        if (key == "format") {
          if (!str(format)) return false;
        } else if (key == "entries") {
          if (!lit('[')) return false;
          have_entries = true;
          if (!lit(']')) {
            do {
              TuneRecord r;
              if (!record(r)) return false;
              out.push_back(r);
            } while (lit(','));
            if (!lit(']')) return false;
          }
        } else {
          return false;
        }
      } while (lit(','));
      if (!lit('}')) return false;
    }
    ws();
    return have_entries && i == t.size();
  }
};

static bool record_valid(const TuneRecord& r) {
  return !r.device.empty() && r.sms > 0 && r.oh > 0 && r.ow > 0 && r.ow <= 1024 && (r.jitter == 0 || r.jitter == 1) &&
         r.bucket >= 0 && r.bucket <= 31 && r.band >= 1 && r.band <= kBandMax && r.per_sm >= 1 && r.per_sm <= 64;
}

static int fused_max_per_sm(int jitter, bool masks = false) {
  int per_sm = 0;
  auto kern = jitter ? (masks ? k_chain_fused<1, true> : k_chain_fused<1, false>)
                     : (masks ? k_chain_fused<0, true> : k_chain_fused<0, false>);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
  return per_sm < 1 ? 1 : per_sm;
}

alb_status launch_chain(const alb_chain_cfg& cfg, int32_t n, const alb_params* params, const alb_image* in,
                        void* out, int32_t mode, Carve& ws, int32_t* status, cudaStream_t st,
                        const alb_image* mask_in, const alb_image* mask_out) {
  const ChainK K = make_consts(cfg);
  const int jit = cfg.jitter;
  const int64_t npx = (int64_t)cfg.out_h * cfg.out_w;
  int32_t* queue = ws.take<int32_t>(64);
  uint8_t* luts = ws.take<uint8_t>((size_t)n * (jit ? 512 : 256));
  unsigned long long* sums = jit ? ws.take<unsigned long long>((size_t)n) : nullptr;
  ALB_REQUIRE(queue && luts && (!jit || sums), ALB_EWORKSPACE, "alb_apply_batch: workspace too small");
  if (jit) {
    k_jitter_luts<<<n, 256, 0, st>>>(n, params, nullptr, npx, 0, luts);   // B tables
    ALB_CUDA(cudaMemsetAsync(sums, 0, (size_t)n * sizeof(unsigned long long), st));
  } else {
    k_chain_luts<<<n, 256, 0, st>>>(n, params, luts);
  }
  ALB_CUDA(cudaGetLastError());
  __nv_bfloat16* o = (__nv_bfloat16*)out;
  if (mode == ALB_MODE_FUSED) {
    ALB_REQUIRE(cfg.out_w <= 1024, ALB_ESHAPE, "alb_apply_batch: fused mode supports out_w <= 1024");
    int32_t band = 8, per_sm = 0;
    if (cfg.tile_h <= 0 && cfg.ctas_per_sm <= 0) {
      int dev = 0;
      ALB_CUDA(cudaGetDevice(&dev));
      tune_lookup(dev, cfg, n, band, per_sm);
    } else {
      if (cfg.tile_h > 0) band = imin(cfg.tile_h, kBandMax);
      per_sm = cfg.ctas_per_sm;
    }
    const int max_per_sm = fused_max_per_sm(jit, mask_in != nullptr);
    if (per_sm <= 0 || per_sm > max_per_sm) per_sm = max_per_sm;
    if (jit && 3 * npx <= kJitImgMax && cfg.out_h <= 1024) {
      // the whole chain per image on chip (one CTA per SM, the image in shared memory)
      const int smem = (int)(3 * npx);
      auto kj = mask_in ? k_chain_jitter_img<true> : k_chain_jitter_img<false>;
      ALB_CUDA(cudaFuncSetAttribute(kj, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      int pj = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pj, kj, 1024, smem);
      ALB_CUDA(cudaMemsetAsync(queue, 0, sizeof(int32_t), st));
      kj<<<(pj < 1 ? 1 : pj) * sm_count(), 1024, smem, st>>>(n, params, in, luts, K, queue, o, mask_in, mask_out,
                                                              status);
      ALB_CUDA(cudaGetLastError());
      return ALB_OK;
    }
    if (jit) {
      // the contrast pivots first (a reduction over each image), then the C tables
      int pv = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pv, k_chain_pivot, 256, 0);
      k_chain_pivot<<<(pv < 1 ? 1 : pv) * sm_count(), 256, 0, st>>>(n, params, in, luts, K, 32, sums);
      ALB_CUDA(cudaGetLastError());
      k_jitter_luts<<<n, 256, 0, st>>>(n, params, sums, npx, 1, luts);
      ALB_CUDA(cudaGetLastError());
    }
    ALB_CUDA(cudaMemsetAsync(queue, 0, sizeof(int32_t), st));
    auto kern = jit ? (mask_in ? k_chain_fused<1, true> : k_chain_fused<1, false>)
                    : (mask_in ? k_chain_fused<0, true> : k_chain_fused<0, false>);
    kern<<<per_sm * sm_count(), 256, 0, st>>>(n, params, in, luts, K, band, queue, o, mask_in, mask_out, status);
    ALB_CUDA(cudaGetLastError());
    return ALB_OK;
  }
  // plain path: one step per launch, intermediates materialised
  const int64_t P = (int64_t)cfg.out_h * cfg.out_w;
  const size_t px = (size_t)n * P;
  uint8_t* a = ws.take<uint8_t>(px * 3);
  uint8_t* b = ws.take<uint8_t>(px * 3);
  float* f = jit ? nullptr : ws.take<float>(px * 3);
  alb_params* rec = ws.take<alb_params>((size_t)n * 3);
  alb_image* desc = ws.take<alb_image>((size_t)n * 2);
  int32_t* prefix = ws.take<int32_t>((size_t)n + 1);
  int32_t* rpi = ws.take<int32_t>((size_t)n);
  int32_t* prefix2 = ws.take<int32_t>((size_t)n + 1);   // the resize step's second tile plan (reductions)
  int32_t* rpi2 = ws.take<int32_t>((size_t)n);
  uint8_t* luts768 = jit ? nullptr : ws.take<uint8_t>((size_t)n * 768);
  ALB_REQUIRE(a && b && (jit || (f && luts768)) && rec && desc && prefix && rpi && prefix2 && rpi2, ALB_EWORKSPACE,
              "alb_apply_batch: workspace too small for plain mode");
  alb_params *rrc = rec, *fl = rec + n, *lr = rec + 2 * n;
  alb_image *da = desc, *db = desc + n;
  k_plain_records<<<(n + 127) / 128, 128, 0, st>>>(n, params, K, a, b, rrc, fl, lr, da, db);
  ALB_CUDA(cudaGetLastError());
  const ImgList lin{in, {}}, la{da, {}}, lb{db, {}};
  const Plan plan{prefix, rpi, n, prefix2, rpi2};
  // crop + resize: the ragged RandomResizedCrop launch
  {
    const PrmList pr{rrc, {}};
    const PlanCheck chk{ALB_RANDOM_RESIZED_CROP, 3, true, lin, pr, status, 0};
    alb_status rc = launch_plan(la, n, kPlainItemBytes, prefix, rpi, chk, st);
    if (rc == ALB_OK) rc = launch_geometric(ALB_RANDOM_RESIZED_CROP, plan, lin, la, pr, 3, false, status, st);
    if (rc != ALB_OK) return rc;
  }
  // h-flip: the ragged HorizontalFlip launch
  {
    const PrmList pr{fl, {}};
    const PlanCheck chk{ALB_HFLIP, 3, true, la, pr, status, 0};
    alb_status rc = launch_plan(lb, n, kPlainItemBytes, prefix, rpi, chk, st);
    if (rc == ALB_OK) rc = launch_geometric(ALB_HFLIP, plan, la, lb, pr, 3, false, status, st);
    if (rc != ALB_OK) return rc;
  }
  const dim3 grid = plain_grid(n, P);
  if (jit) {
    // one launch per position of the order; before each, the pivots of the
    // images whose contrast runs at that position, and their C tables
    uint8_t* cur = b;
    uint8_t* nxt = a;
    for (int step = 0; step < 3; step++) {
      k_plain_pivot<<<grid, 256, 0, st>>>(n, params, P, step, cur, sums);
      ALB_CUDA(cudaGetLastError());
      k_jitter_luts<<<n, 256, 0, st>>>(n, params, sums, npx, 1, luts);
      ALB_CUDA(cudaGetLastError());
      k_plain_jitter_step<<<grid, 256, 0, st>>>(n, params, P, step, luts, cur, nxt);
      ALB_CUDA(cudaGetLastError());
      uint8_t* t = cur; cur = nxt; nxt = t;
    }
    k_plain_normalize_u8<<<grid, 256, 0, st>>>(n, K, P, cur, o);
    ALB_CUDA(cudaGetLastError());
  } else {
    // brightness / contrast table: the bulk-copy LUT kernel with the chain's tables
    k_plain_luts768<<<n, 256, 0, st>>>(n, luts, luts768);
    ALB_CUDA(cudaGetLastError());
    const PrmList pr{lr, {}};
    const PlanCheck chk{ALB_BRIGHTNESS_CONTRAST, 3, false, lb, pr, status, 0};
    alb_status rc = launch_plan(la, n, kPlainItemBytes, prefix, rpi, chk, st);
    if (rc == ALB_OK) rc = launch_stream_lut(plan, lb, la, luts768, status, st);
    if (rc != ALB_OK) return rc;
    k_plain_saturate<<<plain_grid(n, P, 4), 256, 0, st>>>(n, params, P, a, f);
    ALB_CUDA(cudaGetLastError());
    k_plain_normalize<<<grid, 256, 0, st>>>(n, K, P, f, o);
    ALB_CUDA(cudaGetLastError());
  }
  if (mask_in) {
    k_chain_masks<<<8 * sm_count(), 256, 0, st>>>(n, params, in, K, mask_in, mask_out, status);
    ALB_CUDA(cudaGetLastError());
  }
  return ALB_OK;
}

}  // namespace alb

using namespace alb;

extern "C" size_t alb_batch_workspace_size(const alb_chain_cfg* cfg, int32_t n, int32_t mode) {
  if (!cfg || n <= 0) return 4096;
  return chain_workspace(*cfg, n, mode);
}

extern "C" alb_status alb_apply_batch(const alb_chain_cfg* cfg, int32_t n, const alb_params* params_dev,
                                      const alb_image* in_dev, void* out_bf16, int32_t mode, void* workspace,
                                      size_t workspace_bytes, int32_t* dev_status, void* stream) {
  ALB_REQUIRE(cfg, ALB_EINVAL, "alb_apply_batch: null cfg");
  ALB_REQUIRE(n >= 0, ALB_EINVAL, "alb_apply_batch: negative n");
  if (n == 0) return ALB_OK;
  ALB_REQUIRE(params_dev && in_dev && out_bf16, ALB_EINVAL, "alb_apply_batch: null device array");
  ALB_REQUIRE(mode == ALB_MODE_FUSED || mode == ALB_MODE_PLAIN, ALB_EINVAL, "alb_apply_batch: bad mode %d", mode);
  ALB_REQUIRE(cfg->out_h > 0 && cfg->out_w > 0, ALB_ESHAPE, "alb_apply_batch: bad output size");
  ALB_REQUIRE(cfg->tile_w == 0 && cfg->tile_h >= 0 && cfg->tile_h <= kBandMax && cfg->ctas_per_sm >= 0, ALB_EINVAL,
              "alb_apply_batch: tile_h must be in [0, %d], tile_w 0, ctas_per_sm >= 0", kBandMax);
  ALB_REQUIRE(cfg->jitter == 0 || cfg->jitter == 1, ALB_EINVAL, "alb_apply_batch: jitter must be 0 or 1");
  for (int c = 0; c < 3; c++) ALB_REQUIRE(cfg->std[c] > 0, ALB_EINVAL, "alb_apply_batch: std must be > 0");
  ALB_REQUIRE(workspace && workspace_bytes >= chain_workspace(*cfg, n, mode), ALB_EWORKSPACE,
              "alb_apply_batch: workspace of %zu bytes is smaller than %zu", workspace_bytes,
              chain_workspace(*cfg, n, mode));
  Carve cv{(char*)workspace, 0, workspace_bytes};
  return launch_chain(*cfg, n, params_dev, in_dev, out_bf16, mode, cv, dev_status, (cudaStream_t)stream);
}

// Times every candidate schedule of the fused kernel on this batch (each run
// is a complete alb_apply_batch in fused mode: tables + fused kernel, output
// written) and caches the fastest.  Synchronises the stream; not for use while
// the stream is being captured into a graph.
extern "C" alb_status alb_autotune_batch(const alb_chain_cfg* cfg, int32_t n, const alb_params* params_dev,
                                         const alb_image* in_dev, void* out_bf16, void* workspace,
                                         size_t workspace_bytes, int32_t reps, alb_chain_cfg* best, void* stream) {
  ALB_REQUIRE(cfg && best, ALB_EINVAL, "alb_autotune_batch: null cfg");
  ALB_REQUIRE(n > 0, ALB_EINVAL, "alb_autotune_batch: n must be > 0");
  ALB_REQUIRE(params_dev && in_dev && out_bf16, ALB_EINVAL, "alb_autotune_batch: null device array");
  ALB_REQUIRE(cfg->out_h > 0 && cfg->out_w > 0 && cfg->out_w <= 1024, ALB_ESHAPE,
              "alb_autotune_batch: bad output size");
  ALB_REQUIRE(cfg->tile_w == 0, ALB_EINVAL, "alb_autotune_batch: tile_w must be 0");
  ALB_REQUIRE(cfg->jitter == 0 || cfg->jitter == 1, ALB_EINVAL, "alb_autotune_batch: jitter must be 0 or 1");
  for (int c = 0; c < 3; c++) ALB_REQUIRE(cfg->std[c] > 0, ALB_EINVAL, "alb_autotune_batch: std must be > 0");
  const size_t need = chain_workspace(*cfg, n, ALB_MODE_FUSED);
  ALB_REQUIRE(workspace && workspace_bytes >= need, ALB_EWORKSPACE,
              "alb_autotune_batch: workspace of %zu bytes is smaller than %zu", workspace_bytes, need);
  if (reps < 1) reps = 1;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  ALB_CUDA(cudaGetDevice(&dev));
  const int max_per_sm = fused_max_per_sm(cfg->jitter);
  const int32_t bands[] = {2, 4, 8, 16, 32};
  const int32_t residency[] = {max_per_sm, max_per_sm / 2};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ALB_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_status(cudaGetLastError(), "cudaEventCreate");
  }
  float best_ms = 0.0f;
  int32_t best_band = 8, best_per_sm = max_per_sm;
  alb_status rc = ALB_OK;
  for (int32_t band : bands) {
    for (int ri = 0; ri < 2 && rc == ALB_OK; ri++) {
      const int32_t per_sm = residency[ri];
      if (per_sm < 1 || (ri == 1 && per_sm == residency[0])) continue;
      alb_chain_cfg c = *cfg;
      c.tile_h = band;
      c.ctas_per_sm = per_sm;
      Carve cv{(char*)workspace, 0, workspace_bytes};
      rc = launch_chain(c, n, params_dev, in_dev, out_bf16, ALB_MODE_FUSED, cv, nullptr, st);   // warm-up
      if (rc != ALB_OK) break;
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && rc == ALB_OK; r++) {
        Carve cr{(char*)workspace, 0, workspace_bytes};
        rc = launch_chain(c, n, params_dev, in_dev, out_bf16, ALB_MODE_FUSED, cr, nullptr, st);
      }
      cudaEventRecord(e1, st);
      if (rc != ALB_OK) break;
      float ms = 0.0f;
      cudaError_t e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) { rc = cuda_status(e, "autotune timing"); break; }
      if (best_ms == 0.0f || ms < best_ms) { best_ms = ms; best_band = band; best_per_sm = per_sm; }
    }
    if (rc != ALB_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != ALB_OK) return rc;
  tune_store(dev, *cfg, n, best_band, best_per_sm);
  *best = *cfg;
  best->tile_h = best_band;
  best->ctas_per_sm = best_per_sm;
  return ALB_OK;
}

// The chain with its targets: instance-mask stacks (nearest, the same crop
// and flip) and boxes.  Fused mode writes the masks from the fused kernel's
// work items; plain mode in a launch of their own.
extern "C" alb_status alb_apply_batch_targets(const alb_chain_cfg* cfg, int32_t n, const alb_params* params_dev,
                                              const alb_image* in_dev, void* out_bf16, const alb_image* mask_in_dev,
                                              const alb_image* mask_out_dev, const float* boxes_dev,
                                              const int32_t* n_boxes_dev, int32_t box_cap, float* boxes_out_dev,
                                              int32_t* n_boxes_out_dev, int32_t mode, void* workspace,
                                              size_t workspace_bytes, int32_t* dev_status, void* stream) {
  ALB_REQUIRE(cfg, ALB_EINVAL, "alb_apply_batch_targets: null cfg");
  ALB_REQUIRE(n >= 0, ALB_EINVAL, "alb_apply_batch_targets: negative n");
  if (n == 0) return ALB_OK;
  ALB_REQUIRE(params_dev && in_dev && out_bf16, ALB_EINVAL, "alb_apply_batch_targets: null device array");
  ALB_REQUIRE(mode == ALB_MODE_FUSED || mode == ALB_MODE_PLAIN, ALB_EINVAL, "alb_apply_batch_targets: bad mode %d",
              mode);
  ALB_REQUIRE(cfg->out_h > 0 && cfg->out_w > 0 && cfg->out_w <= 1024, ALB_ESHAPE,
              "alb_apply_batch_targets: bad output size");
  ALB_REQUIRE(cfg->tile_w == 0 && cfg->tile_h >= 0 && cfg->tile_h <= kBandMax && cfg->ctas_per_sm >= 0, ALB_EINVAL,
              "alb_apply_batch_targets: tile_h must be in [0, %d], tile_w 0, ctas_per_sm >= 0", kBandMax);
  ALB_REQUIRE(cfg->jitter == 0 || cfg->jitter == 1, ALB_EINVAL, "alb_apply_batch_targets: jitter must be 0 or 1");
  for (int c = 0; c < 3; c++) ALB_REQUIRE(cfg->std[c] > 0, ALB_EINVAL, "alb_apply_batch_targets: std must be > 0");
  ALB_REQUIRE(!mask_in_dev == !mask_out_dev, ALB_EINVAL, "alb_apply_batch_targets: mask_in and mask_out go together");
  const bool boxes = boxes_dev || n_boxes_dev || boxes_out_dev || n_boxes_out_dev;
  ALB_REQUIRE(!boxes || (boxes_dev && n_boxes_dev && boxes_out_dev && n_boxes_out_dev && box_cap > 0), ALB_EINVAL,
              "alb_apply_batch_targets: box arrays go together and need box_cap > 0");
  ALB_REQUIRE(workspace && workspace_bytes >= chain_workspace(*cfg, n, mode), ALB_EWORKSPACE,
              "alb_apply_batch_targets: workspace of %zu bytes is smaller than %zu", workspace_bytes,
              chain_workspace(*cfg, n, mode));
  cudaStream_t st = (cudaStream_t)stream;
  Carve cv{(char*)workspace, 0, workspace_bytes};
  alb_status rc = launch_chain(*cfg, n, params_dev, in_dev, out_bf16, mode, cv, dev_status, st, mask_in_dev,
                               mask_out_dev);
  if (rc != ALB_OK) return rc;
  if (boxes) {
    const ChainK K = make_consts(*cfg);
    k_chain_boxes<<<(n + 3) / 4, 128, 0, st>>>(n, params_dev, K, boxes_dev, n_boxes_dev, box_cap, boxes_out_dev,
                                               n_boxes_out_dev, dev_status);
    ALB_CUDA(cudaGetLastError());
  }
  return ALB_OK;
}


// ---- schedule cache: lookup and persistence
extern "C" alb_status alb_autotune_lookup(const alb_chain_cfg* cfg, int32_t n, alb_chain_cfg* best,
                                          int32_t* found) {
  ALB_REQUIRE(cfg && best && found, ALB_EINVAL, "alb_autotune_lookup: null argument");
  ALB_REQUIRE(n > 0, ALB_EINVAL, "alb_autotune_lookup: n must be > 0");
  int dev = 0;
  ALB_CUDA(cudaGetDevice(&dev));
  int32_t band = 0, per_sm = 0;
  *found = tune_lookup(dev, *cfg, n, band, per_sm) ? 1 : 0;
  *best = *cfg;
  if (*found) {
    best->tile_h = band;
    best->ctas_per_sm = per_sm;
  }
  return ALB_OK;
}

extern "C" alb_status alb_autotune_save(const char* path) {
  ALB_REQUIRE(path && *path, ALB_EINVAL, "alb_autotune_save: empty path");
  std::vector<TuneEntry> entries;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    entries = g_tune;
  }
  std::string out = "{\"format\": \"alb-autotune-1\", \"entries\": [";
  for (size_t k = 0; k < entries.size(); k++) {
    const TuneEntry& e = entries[k];
    std::string name;
    int32_t sms = 0;
    if (!device_key(e.dev, name, sms)) return cuda_status(cudaGetLastError(), "alb_autotune_save: device query");
    char buf[512];
    snprintf(buf, sizeof(buf),
             "%s\n  {\"device\": \"%s\", \"sms\": %d, \"out_h\": %d, \"out_w\": %d, \"jitter\": %d, \"bucket\": %d, "
             "\"rows_per_item\": %d, \"ctas_per_sm\": %d}",
             k ? "," : "", name.c_str(), sms, e.oh, e.ow, e.jitter, e.bucket, e.band, e.per_sm);
    out += buf;
  }
  out += "\n]}\n";
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "wb");
  ALB_REQUIRE(f, ALB_EINVAL, "alb_autotune_save: cannot write %s", tmp.c_str());
  const bool ok = fwrite(out.data(), 1, out.size(), f) == out.size();
  const bool closed = fclose(f) == 0;
  ALB_REQUIRE(ok && closed, ALB_EINVAL, "alb_autotune_save: write to %s failed", tmp.c_str());
  ALB_REQUIRE(rename(tmp.c_str(), path) == 0, ALB_EINVAL, "alb_autotune_save: cannot rename to %s", path);
  return ALB_OK;
}

extern "C" alb_status alb_autotune_load(const char* path, int32_t* n_loaded) {
  ALB_REQUIRE(path && *path && n_loaded, ALB_EINVAL, "alb_autotune_load: null argument");
  *n_loaded = 0;
  FILE* f = fopen(path, "rb");
  ALB_REQUIRE(f, ALB_EINVAL, "alb_autotune_load: cannot open %s", path);
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0 && text.size() < (1u << 22)) text.append(buf, got);
  fclose(f);
  ALB_REQUIRE(text.size() < (1u << 22), ALB_EINVAL, "alb_autotune_load: %s is larger than 4 MiB", path);
  std::vector<TuneRecord> recs;
  std::string format;
  JsonReader rd(text);
  ALB_REQUIRE(rd.document(recs, format), ALB_EINVAL, "alb_autotune_load: %s is not an autotune cache (offset %zu)",
              path, rd.i);
  ALB_REQUIRE(format == "alb-autotune-1", ALB_EINVAL, "alb_autotune_load: unknown format \"%s\"", format.c_str());
  for (size_t k = 0; k < recs.size(); k++)
    ALB_REQUIRE(record_valid(recs[k]), ALB_EINVAL, "alb_autotune_load: entry %zu of %s is out of range", k, path);
  // nothing is loaded until the whole file has been read and checked
  int count = 0;
  ALB_CUDA(cudaGetDeviceCount(&count));
  int32_t loaded = 0;
  for (int dev = 0; dev < count; dev++) {
    std::string name;
    int32_t sms = 0;
    if (!device_key(dev, name, sms)) return cuda_status(cudaGetLastError(), "alb_autotune_load: device query");
    for (const TuneRecord& r : recs) {
      if (r.device != name || r.sms != sms) continue;
      alb_chain_cfg c{};
      c.out_h = r.oh;
      c.out_w = r.ow;
      c.jitter = r.jitter;
      tune_store(dev, c, int32_t(1) << (r.bucket > 30 ? 30 : r.bucket), r.band, r.per_sm);
      loaded++;
    }
  }
  *n_loaded = loaded;
  return ALB_OK;
}

namespace alb {
ALB_OOB_ACCESSOR(oob_fused)
}  // namespace alb
