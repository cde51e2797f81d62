/*
 * alb_oracle.c -- plain, slow CPU oracle for the augmentation hot path of
 * "Albumentations: fast and flexible image augmentations" (Buslaev et al.,
 * arXiv 1809.06839).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * product path (the CUDA library) never calls it, links it or shares any
 * code, header, table or constant with it.
 *
 * Everything here is a nested loop over output pixels, one image at a time,
 * in exact integer arithmetic or IEEE float64 (float32 only where the method
 * itself is defined in float32: the colour-jitter saturation and Normalize
 * steps of the fused chain).  No blocking, fusion or reordering.  Build with
 * -ffp-contract=off so that a*b+c is never contracted into an fma.
 *
 * The paper names its transforms (Table I: RandomCrop64, PadToSize512,
 * HorizontalFlip, VerticalFlip, Rotate, ShiftScaleRotate, Brightness,
 * ShiftHSV, ShiftRGB, Gamma, Grayscale; Sec. II: colour, contrast and
 * brightness transforms, horizontal flip + random sized crop on images,
 * boxes and masks, crops / rotations / reflections / scaling with masks
 * transformed the same way) but defines none of them mathematically.  The
 * definitions below are this project's readings of the paper (pixel-centre
 * coordinates, round-half-even saturation, reflect-101 borders, 5-bit
 * fixed-point bilinear weights, Q16 affine coefficients); each function
 * states the reading it follows.
 *
 * Parity status: every function is pinned by tests/test_oracle_*.py against
 * closed forms, library routines (numpy, Python fractions, colorsys, torch
 * bf16 casts), invariants or brute force.  See the per-function comments.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define EXPORT __attribute__((visibility("default")))

/* ---- transform ids (public numbering, shared by value with the C-ABI) ---- */
enum {
  T_HFLIP = 1, T_VFLIP = 2, T_RANDOM_CROP = 3, T_PAD_TO_SIZE = 4,
  T_BRIGHTNESS = 5, T_CONTRAST = 6, T_BRIGHTNESS_CONTRAST = 7, T_GAMMA = 8,
  T_SHIFT_RGB = 9, T_SHIFT_HSV = 10, T_GRAYSCALE = 11, T_EQUALIZE = 12,
  T_ROTATE = 13, T_SHIFT_SCALE_ROTATE = 14, T_RESIZE = 15,
  T_RANDOM_SIZED_CROP = 16, T_RANDOM_RESIZED_CROP = 17, T_TRANSPOSE = 18,
  T_ROT90 = 19, T_CHAIN = 20, T_GRID_DISTORTION = 21, T_ELASTIC = 22
};

/* Sampled parameter record of one transform for one image (oracle layout). */
typedef struct orc_params {
  int32_t tid, apply;            /* transform id; 0 = identity (p-draw failed) */
  int32_t in_h, in_w, out_h, out_w;
  int32_t y0, x0, ch, cw;        /* crop window, or pad top/left in y0/x0 */
  int32_t flip, k;               /* chain h-flip bit; rot90 count */
  double alpha, beta, gamma, sat;
  double shift[3];               /* ShiftRGB per channel; ShiftHSV (dh, ds, dv) */
  double angle, scale, dx, dy;   /* degrees; scale; shift as fractions of W, H */
  double m[6];                   /* forward map src->dst, pixel-centre coords */
  int64_t q[6];                  /* inverse map dst->src in Q16 integers */
} orc_params;

typedef struct orc_cfg {
  int32_t tid, out_h, out_w, _pad;
  double p;
  double lo[4], hi[4];
} orc_cfg;

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ESHAPE = 2 };

/* ======================================================================
 * Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror,
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).  One round
 * multiplies counter words 0 and 2 by the two published multipliers and
 * mixes the high/low halves with words 1, 3 and the key; the key is bumped
 * by the two Weyl constants between rounds.
 * ====================================================================== */
EXPORT void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                              uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The word stream of one (seed, stream id, image index): block j of
 * Philox with counter (j, index, stream lo, stream hi) and key (seed lo,
 * seed hi); words are taken in order 0,1,2,3 of block 0, then block 1 ... */
typedef struct orc_stream {
  uint32_t key[2], index, s_lo, s_hi, block;
  uint32_t buf[4];
  int pos;
} orc_stream;

static void stream_init(orc_stream* s, uint64_t seed, uint64_t stream_id, uint32_t index) {
  s->key[0] = (uint32_t)seed; s->key[1] = (uint32_t)(seed >> 32);
  s->index = index; s->s_lo = (uint32_t)stream_id; s->s_hi = (uint32_t)(stream_id >> 32);
  s->block = 0; s->pos = 4;
}

static uint32_t stream_word(orc_stream* s) {
  if (s->pos == 4) {
    uint32_t ctr[4] = {s->block, s->index, s->s_lo, s->s_hi};
    orc_philox4x32_10(ctr, s->key, s->buf);
    s->block++;
    s->pos = 0;
  }
  return s->buf[s->pos++];
}

/* Uniform double in [0,1): 27 high bits of one word and 26 of the next
 * form a 53-bit integer, scaled by 2^-53. */
static double stream_uniform01(orc_stream* s) {
  uint32_t a = stream_word(s) >> 5;
  uint32_t b = stream_word(s) >> 6;
  uint64_t v = (uint64_t)a * 67108864u + (uint64_t)b;
  return (double)v * (1.0 / 9007199254740992.0);
}

static double stream_uniform(orc_stream* s, double lo, double hi) {
  double u = stream_uniform01(s);
  double span = hi - lo;
  double t = span * u;
  return lo + t;
}

/* Unbiased integer in [0, n] (n >= 0): Lemire's multiply-shift with
 * rejection ("Fast random integer generation in an interval", 2019). */
static int32_t stream_randint(orc_stream* s, int32_t n) {
  uint32_t range = (uint32_t)n + 1u;
  uint32_t x = stream_word(s);
  uint64_t m = (uint64_t)x * (uint64_t)range;
  uint32_t low = (uint32_t)m;
  if (low < range) {
    uint32_t threshold = (uint32_t)(0u - range) % range;
    while (low < threshold) {
      x = stream_word(s);
      m = (uint64_t)x * (uint64_t)range;
      low = (uint32_t)m;
    }
  }
  return (int32_t)(m >> 32);
}

/* exported for the pins on the sampler primitives */
EXPORT void orc_stream_words(uint64_t seed, uint64_t stream_id, uint32_t index, int n, uint32_t* out) {
  orc_stream s; stream_init(&s, seed, stream_id, index);
  for (int i = 0; i < n; i++) out[i] = stream_word(&s);
}
EXPORT void orc_stream_uniform01(uint64_t seed, uint64_t stream_id, uint32_t index, int n, double* out) {
  orc_stream s; stream_init(&s, seed, stream_id, index);
  for (int i = 0; i < n; i++) out[i] = stream_uniform01(&s);
}
EXPORT void orc_stream_randint(uint64_t seed, uint64_t stream_id, uint32_t index, int32_t hi, int n, int32_t* out) {
  orc_stream s; stream_init(&s, seed, stream_id, index);
  for (int i = 0; i < n; i++) out[i] = stream_randint(&s, hi);
}

/* ======================================================================
 * Small exact helpers
 * ====================================================================== */
static int64_t floor_div(int64_t a, int64_t b) {     /* b > 0 */
  int64_t q = a / b, r = a % b;
  if (r != 0 && r < 0) q -= 1;
  return q;
}

/* reflect-101 border: ...dcb|abcd|cba...; the edge sample is not repeated.
 * Period 2(n-1); a length-1 axis maps everything to 0. */
static int64_t reflect101(int64_t i, int64_t n) {
  if (n == 1) return 0;
  int64_t period = 2 * (n - 1);
  int64_t m = i % period;
  if (m < 0) m += period;
  if (m >= n) m = period - m;
  return m;
}

/* float64 -> uint8 with round-half-even then saturation to [0,255]. */
static uint8_t sat_rne(double v) {
  double r = rint(v);            /* default rounding mode: nearest, ties to even */
  if (r < 0.0) r = 0.0;
  if (r > 255.0) r = 255.0;
  return (uint8_t)r;
}

/* round(num/den) with ties to even, num >= 0, den > 0, exact integers. */
static int64_t rne_div(int64_t num, int64_t den) {
  int64_t q = num / den, r = num % den;
  int64_t twice = 2 * r;
  if (twice > den || (twice == den && (q & 1))) q += 1;
  return q;
}

/* ======================================================================
 * Parameter geometry: affine maps about the pixel-centre image centre, and
 * the half-pixel resize map
 * ====================================================================== */

/* Rotation about the image centre c = ((W-1)/2, (H-1)/2) by angle degrees
 * (positive = counter-clockwise on screen, y pointing down), scale s, then a
 * shift t = (dx*W, dy*H):  dst = s*R(angle)*(src - c) + c + t with
 * R = [[cos, sin], [-sin, cos]].  The inverse src = A*(dst - c - t) + c with
 * A = R^-1 / s is quantised once to Q16 integers (round half even). */
static void warp_geometry(orc_params* p, int h, int w) {
  double rad = p->angle * (M_PI / 180.0);
  double cs = cos(rad), sn = sin(rad);
  double s = p->scale;
  double cx = (double)(w - 1) * 0.5, cy = (double)(h - 1) * 0.5;
  double tx = p->dx * (double)w, ty = p->dy * (double)h;
  /* forward */
  double m00 = s * cs, m01 = s * sn, m10 = -(s * sn), m11 = s * cs;
  p->m[0] = m00; p->m[1] = m01; p->m[3] = m10; p->m[4] = m11;
  p->m[2] = (cx + tx) - (m00 * cx + m01 * cy);
  p->m[5] = (cy + ty) - (m10 * cx + m11 * cy);
  /* inverse */
  double a00 = cs / s, a01 = -sn / s, a10 = sn / s, a11 = cs / s;
  double ox = cx + tx, oy = cy + ty;
  double b0 = cx - (a00 * ox + a01 * oy);
  double b1 = cy - (a10 * ox + a11 * oy);
  p->q[0] = llrint(a00 * 65536.0); p->q[1] = llrint(a01 * 65536.0); p->q[2] = llrint(b0 * 65536.0);
  p->q[3] = llrint(a10 * 65536.0); p->q[4] = llrint(a11 * 65536.0); p->q[5] = llrint(b1 * 65536.0);
}

EXPORT void orc_warp_geometry(orc_params* p, int h, int w) { warp_geometry(p, h, w); }

/* Output size of a transform applied to an h x w input. */
EXPORT int orc_output_shape(const orc_params* p, int h, int w, int* oh, int* ow) {
  switch (p->tid) {
    case T_RANDOM_CROP: case T_PAD_TO_SIZE: case T_RESIZE:
    case T_RANDOM_SIZED_CROP: case T_RANDOM_RESIZED_CROP: case T_CHAIN:
      *oh = p->out_h; *ow = p->out_w; return ORC_OK;
    case T_TRANSPOSE:
      *oh = w; *ow = h; return ORC_OK;
    case T_ROT90:
      if (p->apply && (p->k & 1)) { *oh = w; *ow = h; } else { *oh = h; *ow = w; }
      return ORC_OK;
    default:
      *oh = h; *ow = w; return ORC_OK;
  }
}

/* ======================================================================
 * Parameter sampling: one Philox word stream per
 * (seed, stream id, image index); the probability draw comes first and all
 * parameter draws follow whether or not the transform is applied.
 * Size-changing transforms are always applied.
 * ====================================================================== */
static int sample_rrc(orc_stream* s, int h, int w, double slo, double shi,
                      double rlo, double rhi, int* y0, int* x0, int* ch, int* cw) {
  double area = (double)h * (double)w;
  double lrlo = log(rlo), lrhi = log(rhi);
  for (int attempt = 0; attempt < 10; attempt++) {
    double target = area * stream_uniform(s, slo, shi);
    double ar = exp(stream_uniform(s, lrlo, lrhi));
    double fw = rint(sqrt(target * ar));
    double fh = rint(sqrt(target / ar));
    if (fw > 0.0 && fh > 0.0 && fw <= (double)w && fh <= (double)h) {
      *cw = (int)fw; *ch = (int)fh;
      *y0 = stream_randint(s, h - *ch);
      *x0 = stream_randint(s, w - *cw);
      return 0;
    }
  }
  /* fallback: the largest centred crop whose aspect lies in [rlo, rhi] */
  double in_ratio = (double)w / (double)h;
  if (in_ratio < rlo) { *cw = w; *ch = (int)rint((double)w / rlo); }
  else if (in_ratio > rhi) { *ch = h; *cw = (int)rint((double)h * rhi); }
  else { *cw = w; *ch = h; }
  if (*ch > h) *ch = h;
  if (*cw > w) *cw = w;
  *y0 = (h - *ch) / 2; *x0 = (w - *cw) / 2;
  return 1;
}

/* ======================================================================
 * Grid distortion and elastic transform (Sec. II-C: non-rigid distortions
 * for medical images).  The paper names them only; the readings here:
 *
 * Grid distortion.  Each axis of length n is cut into G cells of equal
 * width in the output; cell i keeps a positive factor d_i (Q14 integers).
 * The source cells have widths proportional to d_i and together span the
 * same [0, n-1] (pixel centres), so the source coordinate of output sample
 * x in cell i = min(G-1, floor(G x / (n-1))) is the exact rational
 *   src(x) = ((n-1) P_i + (G x - i (n-1)) d_i) / D,  P_i = sum_{j<i} d_j,
 *   D = sum_j d_j,
 * quantised to Q5 with round half up.  Images: Q5 bilinear (taps inside the
 * image; the +1 tap clamped); masks: nearest floor((Xq + 16) / 32).
 *
 * Elastic transform.  A lattice of control points every S = 2^s px (from
 * (0, 0), ceil(W/S) + 1 by ceil(H/S) + 1 points) carries integer Q5
 * displacements in [-A, A]; point t = i * nx + j takes the Philox4x32-10
 * block with counter (t, image index, stream id lo, stream id hi ^ 2^31) and
 * key = seed: dx = floor(w0 (2A + 1) / 2^32) - A, dy the same from w1.  A
 * pixel's displacement is the bilinear blend of its cell's four points with
 * integer weights (S - fx)(S - fy), ..., rounded half up: floor((sum +
 * S^2/2) / S^2).  The source coordinate is (32 x + dx, 32 y + dy) in Q5;
 * images: Q5 bilinear with reflect-101 taps; masks: nearest, reflected.
 * ====================================================================== */
EXPORT void orc_grid_set_factor(orc_params* p, int slot, int32_t d) {
  uint64_t w = (uint64_t)p->q[slot >> 2];
  int sh = 16 * (slot & 3);
  w = (w & ~((uint64_t)0xFFFF << sh)) | ((uint64_t)(uint16_t)d << sh);
  p->q[slot >> 2] = (int64_t)w;
}

EXPORT int32_t orc_grid_factor(const orc_params* p, int slot) {
  return (int32_t)(((uint64_t)p->q[slot >> 2] >> (16 * (slot & 3))) & 0xFFFFu);
}

/* Q5 source coordinate of output sample x on an axis of n samples
 * (axis 0 = x: factor slots 0..G-1, axis 1 = y: slots 12..12+G-1). */
EXPORT int64_t orc_grid_q5(const orc_params* p, int axis, int64_t x, int64_t n) {
  int g = p->k;
  if (n <= 1) return 0;
  int64_t d[12], D = 0;
  for (int j = 0; j < g; j++) { d[j] = orc_grid_factor(p, 12 * axis + j); D += d[j]; }
  int64_t i = (g * x) / (n - 1);
  if (i > g - 1) i = g - 1;
  int64_t P = 0;
  for (int j = 0; j < i; j++) P += d[j];
  int64_t N = (n - 1) * P + (g * x - i * (n - 1)) * d[i];
  int64_t xq = floor_div(64 * N + D, 2 * D);
  if (xq < 0) xq = 0;
  if (xq > 32 * (n - 1)) xq = 32 * (n - 1);
  return xq;
}

/* Output edge coordinate of source edge coordinate e on a grid-distorted
 * axis of n samples: the inverse of the (unquantised) piecewise-linear
 * src(x) in centre coordinates between the first and last pixel centres
 * (both fixed points of the map); the outer half pixels map to themselves,
 * so the image edges stay the image edges. */
EXPORT double orc_grid_edge_inverse(const orc_params* p, int axis, double e, int64_t n) {
  int g = p->k;
  if (n <= 1) return e;
  double d[12], D = 0.0, c[13];
  for (int j = 0; j < g; j++) { d[j] = (double)orc_grid_factor(p, 12 * axis + j); D += d[j]; }
  double P = 0.0;
  for (int j = 0; j <= g; j++) { c[j] = (double)(n - 1) * P / D; if (j < g) P += d[j]; }
  double t = e - 0.5;
  if (t <= 0.0 || t >= (double)(n - 1)) return e;
  int i = 0;
  while (i < g - 1 && t >= c[i + 1]) i++;
  double Pi = 0.0;
  for (int j = 0; j < i; j++) Pi += d[j];
  double x = (D * t - (double)(n - 1) * Pi) / ((double)g * d[i]) + (double)i * (double)(n - 1) / (double)g;
  return x + 0.5;
}

/* Lattice displacements of an elastic record (Q5): dx, dy of point t. */
EXPORT void orc_elastic_point(const orc_params* p, int64_t t, int32_t* dx, int32_t* dy) {
  uint64_t seed = (uint64_t)p->q[0], sid = (uint64_t)p->q[1];
  uint32_t ctr[4] = {(uint32_t)t, (uint32_t)p->q[2], (uint32_t)sid, (uint32_t)(sid >> 32) ^ 0x80000000u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  uint64_t span = 2 * (uint64_t)p->k + 1;
  *dx = (int32_t)((o[0] * span) >> 32) - p->k;
  *dy = (int32_t)((o[1] * span) >> 32) - p->k;
}

/* Q5 displacement of pixel (x, y) of an image w pixels wide. */
EXPORT void orc_elastic_disp(const orc_params* p, int64_t x, int64_t y, int w, int32_t* dx, int32_t* dy) {
  int sh = p->cw;
  int64_t S = (int64_t)1 << sh;
  int64_t nx = ((w + S - 1) >> sh) + 1;
  int64_t ci = y >> sh, cj = x >> sh, fy = y & (S - 1), fx = x & (S - 1);
  int32_t ax[4], ay[4];
  orc_elastic_point(p, ci * nx + cj, &ax[0], &ay[0]);
  orc_elastic_point(p, ci * nx + cj + 1, &ax[1], &ay[1]);
  orc_elastic_point(p, (ci + 1) * nx + cj, &ax[2], &ay[2]);
  orc_elastic_point(p, (ci + 1) * nx + cj + 1, &ax[3], &ay[3]);
  int64_t w00 = (S - fx) * (S - fy), w01 = fx * (S - fy), w10 = (S - fx) * fy, w11 = fx * fy;
  *dx = (int32_t)floor_div(w00 * ax[0] + w01 * ax[1] + w10 * ax[2] + w11 * ax[3] + S * S / 2, S * S);
  *dy = (int32_t)floor_div(w00 * ay[0] + w01 * ay[1] + w10 * ay[2] + w11 * ay[3] + S * S / 2, S * S);
}

EXPORT int orc_sample_params(const orc_cfg* cfg, uint64_t seed, uint64_t stream_id,
                             uint32_t index, int h, int w, orc_params* p) {
  memset(p, 0, sizeof(*p));
  if (h <= 0 || w <= 0) return ORC_ESHAPE;
  orc_stream s; stream_init(&s, seed, stream_id, index);
  p->tid = cfg->tid; p->in_h = h; p->in_w = w; p->out_h = h; p->out_w = w;
  p->alpha = 1.0; p->beta = 0.0; p->gamma = 1.0; p->sat = 1.0; p->scale = 1.0;
  double u = stream_uniform01(&s);
  p->apply = u < cfg->p;
  switch (cfg->tid) {
    case T_HFLIP: case T_VFLIP: case T_GRAYSCALE: case T_EQUALIZE: case T_TRANSPOSE:
      break;
    case T_ROT90:
      p->k = stream_randint(&s, 3);
      break;
    case T_RANDOM_CROP:
      p->apply = 1;
      if (cfg->out_h > h || cfg->out_w > w || cfg->out_h <= 0 || cfg->out_w <= 0) return ORC_ESHAPE;
      p->out_h = cfg->out_h; p->out_w = cfg->out_w; p->ch = cfg->out_h; p->cw = cfg->out_w;
      p->y0 = stream_randint(&s, h - cfg->out_h);
      p->x0 = stream_randint(&s, w - cfg->out_w);
      break;
    case T_PAD_TO_SIZE:
      p->apply = 1;
      p->out_h = h > cfg->out_h ? h : cfg->out_h;
      p->out_w = w > cfg->out_w ? w : cfg->out_w;
      p->y0 = (p->out_h - h) / 2; p->x0 = (p->out_w - w) / 2;
      break;
    case T_BRIGHTNESS:
      p->beta = stream_uniform(&s, cfg->lo[0], cfg->hi[0]);
      break;
    case T_CONTRAST:
      p->alpha = stream_uniform(&s, cfg->lo[0], cfg->hi[0]);
      break;
    case T_BRIGHTNESS_CONTRAST:
      p->alpha = stream_uniform(&s, cfg->lo[0], cfg->hi[0]);
      p->beta = stream_uniform(&s, cfg->lo[1], cfg->hi[1]);
      break;
    case T_GAMMA:
      p->gamma = stream_uniform(&s, cfg->lo[0], cfg->hi[0]);
      break;
    case T_SHIFT_RGB: case T_SHIFT_HSV:
      for (int c = 0; c < 3; c++) p->shift[c] = stream_uniform(&s, cfg->lo[c], cfg->hi[c]);
      break;
    case T_ROTATE:
      p->angle = stream_uniform(&s, cfg->lo[0], cfg->hi[0]);
      warp_geometry(p, h, w);
      break;
    case T_SHIFT_SCALE_ROTATE:
      p->dx = stream_uniform(&s, cfg->lo[0], cfg->hi[0]);
      p->dy = stream_uniform(&s, cfg->lo[0], cfg->hi[0]);
      p->scale = stream_uniform(&s, cfg->lo[1], cfg->hi[1]);
      p->angle = stream_uniform(&s, cfg->lo[2], cfg->hi[2]);
      warp_geometry(p, h, w);
      break;
    case T_RESIZE:
      p->apply = 1;
      if (cfg->out_h <= 0 || cfg->out_w <= 0) return ORC_ESHAPE;
      p->out_h = cfg->out_h; p->out_w = cfg->out_w;
      p->y0 = 0; p->x0 = 0; p->ch = h; p->cw = w;
      break;
    case T_RANDOM_SIZED_CROP: {
      p->apply = 1;
      if (cfg->out_h <= 0 || cfg->out_w <= 0) return ORC_ESHAPE;
      p->out_h = cfg->out_h; p->out_w = cfg->out_w;
      int mside = h < w ? h : w;
      int lo = (int)ceil(cfg->lo[0] * (double)mside);
      int hi = (int)floor(cfg->hi[0] * (double)mside);
      if (lo < 1) lo = 1;
      if (hi > mside) hi = mside;
      if (hi < lo) return ORC_ESHAPE;
      int side = lo + stream_randint(&s, hi - lo);
      p->ch = side; p->cw = side;
      p->y0 = stream_randint(&s, h - side);
      p->x0 = stream_randint(&s, w - side);
      break;
    }
    case T_RANDOM_RESIZED_CROP:
      p->apply = 1;
      if (cfg->out_h <= 0 || cfg->out_w <= 0) return ORC_ESHAPE;
      p->out_h = cfg->out_h; p->out_w = cfg->out_w;
      sample_rrc(&s, h, w, cfg->lo[0], cfg->hi[0], cfg->lo[1], cfg->hi[1], &p->y0, &p->x0, &p->ch, &p->cw);
      break;
    case T_GRID_DISTORTION: {
      /* G cells per axis (lo[1], default 5, at most 12); a factor per cell,
       * 1 + U[lo[0], hi[0]], kept as Q14 integers (x cells, then y cells) */
      int g = cfg->lo[1] > 0 ? (int)cfg->lo[1] : 5;
      if (g < 1 || g > 12) return ORC_EINVAL;
      p->k = g;
      for (int j = 0; j < 2 * g; j++) {
        double d = 1.0 + stream_uniform(&s, cfg->lo[0], cfg->hi[0]);
        int64_t dq = (int64_t)rint(d * 16384.0);
        if (dq < 1) dq = 1;
        if (dq > 32767) dq = 32767;
        orc_grid_set_factor(p, j < g ? j : 12 + (j - g), (int32_t)dq);
      }
      break;
    }
    case T_ELASTIC: {
      /* amplitude alpha = lo[0] px (Q5: k = rne(32 alpha)), lattice spacing
       * 2^cw px with cw = lo[1] (default 5); the lattice itself is drawn from
       * the image's own Philox block stream (orc_elastic_lattice) */
      double a = cfg->lo[0];
      int sh = cfg->lo[1] > 0 ? (int)cfg->lo[1] : 5;
      if (a < 0.0 || a > 4096.0 || sh < 2 || sh > 8) return ORC_EINVAL;
      p->k = (int32_t)rint(a * 32.0);
      p->cw = sh;
      p->q[0] = (int64_t)seed; p->q[1] = (int64_t)stream_id; p->q[2] = (int64_t)index;
      break;
    }
    case T_CHAIN:
      /* RandomResizedCrop, then h-flip with probability 1/2, then brightness,
       * contrast and saturation factors, each uniform in [lo[2], hi[2]]. */
      p->apply = 1;
      if (cfg->out_h <= 0 || cfg->out_w <= 0) return ORC_ESHAPE;
      p->out_h = cfg->out_h; p->out_w = cfg->out_w;
      sample_rrc(&s, h, w, cfg->lo[0], cfg->hi[0], cfg->lo[1], cfg->hi[1], &p->y0, &p->x0, &p->ch, &p->cw);
      p->flip = stream_uniform01(&s) < 0.5;
      p->beta = stream_uniform(&s, cfg->lo[2], cfg->hi[2]);   /* brightness factor b */
      p->alpha = stream_uniform(&s, cfg->lo[2], cfg->hi[2]);  /* contrast factor c */
      p->sat = stream_uniform(&s, cfg->lo[2], cfg->hi[2]);    /* saturation factor s */
      p->k = stream_randint(&s, 5);   /* order of the three jitter ops, 0..5 (used by jitter mode 1) */
      break;
    default:
      return ORC_EINVAL;
  }
  return ORC_OK;
}

/* ======================================================================
 * Per-channel 256-entry look-up tables, each entry computed in float64 and
 * saturated with round-half-even
 * ====================================================================== */
EXPORT int orc_build_lut(const orc_params* p, uint8_t lut[3][256]) {
  for (int c = 0; c < 3; c++)
    for (int v = 0; v < 256; v++) {
      double x = (double)v, y;
      switch (p->tid) {
        case T_BRIGHTNESS: y = x + p->beta; break;
        case T_CONTRAST: y = p->alpha * x; break;
        case T_BRIGHTNESS_CONTRAST: { double g = p->alpha * x; y = g + p->beta; break; }
        case T_GAMMA: { double r = x / 255.0; y = 255.0 * pow(r, p->gamma); break; }
        case T_SHIFT_RGB: y = x + p->shift[c]; break;
        case T_CHAIN: {   /* brightness b then contrast c about the fixed pivot 128 */
          double bv = p->beta * x;
          double d = bv - 128.0;
          double cd = p->alpha * d;
          y = cd + 128.0;
          break;
        }
        default: return ORC_EINVAL;
      }
      lut[c][v] = p->apply ? sat_rne(y) : (uint8_t)v;
    }
  return ORC_OK;
}

/* Histogram equalisation of one channel: cdf of the 256-bin histogram,
 * m = count of the lowest occupied level, N pixels;
 * LUT[v] = round_half_even(255 (cdf[v] - m) / (N - m)); a constant channel
 * (N == m) keeps the identity map. */
EXPORT void orc_equalize_lut(const uint64_t hist[256], uint8_t lut[256]) {
  uint64_t n = 0;
  for (int v = 0; v < 256; v++) n += hist[v];
  int first = -1;
  for (int v = 0; v < 256; v++) if (hist[v] > 0) { first = v; break; }
  if (first < 0) { for (int v = 0; v < 256; v++) lut[v] = (uint8_t)v; return; }
  uint64_t m = hist[first];
  if (n == m) { for (int v = 0; v < 256; v++) lut[v] = (uint8_t)v; return; }
  uint64_t cdf = 0;
  for (int v = 0; v < 256; v++) {
    cdf += hist[v];
    if (v < first) { lut[v] = 0; continue; }
    lut[v] = (uint8_t)rne_div((int64_t)(255 * (cdf - m)), (int64_t)(n - m));
  }
}

/* ======================================================================
 * Colour space: Smith's hexcone HSV, float64.
 * ====================================================================== */
static void shift_hsv_pixel(const double shift[3], const uint8_t in[3], uint8_t out[3]) {
  double r = in[0], g = in[1], b = in[2];
  double mx = r, mn = r;
  if (g > mx) mx = g;
  if (b > mx) mx = b;
  if (g < mn) mn = g;
  if (b < mn) mn = b;
  double chroma = mx - mn;
  double hue = 0.0;
  if (chroma > 0.0) {
    if (mx == r) hue = 60.0 * ((g - b) / chroma);
    else if (mx == g) hue = 60.0 * ((b - r) / chroma + 2.0);
    else hue = 60.0 * ((r - g) / chroma + 4.0);
    if (hue < 0.0) hue += 360.0;
  }
  double sat = mx > 0.0 ? chroma / mx : 0.0;
  double val = mx / 255.0;
  /* shift: hue in OpenCV half-degree units (x2), sat/val in 1/255 units */
  double h2 = fmod(hue + 2.0 * shift[0], 360.0);
  if (h2 < 0.0) h2 += 360.0;
  double s2 = sat + shift[1] / 255.0;
  if (s2 < 0.0) s2 = 0.0;
  if (s2 > 1.0) s2 = 1.0;
  double v2 = val + shift[2] / 255.0;
  if (v2 < 0.0) v2 = 0.0;
  if (v2 > 1.0) v2 = 1.0;
  /* back to RGB */
  double c2 = v2 * s2;
  double hp = h2 / 60.0;
  int sector = (int)floor(hp);
  double frac = hp - 2.0 * floor(hp / 2.0);           /* hp mod 2 */
  double x = c2 * (1.0 - fabs(frac - 1.0));
  double m = v2 - c2;
  double r1, g1, b1;
  switch (sector) {
    case 0: r1 = c2; g1 = x; b1 = 0; break;
    case 1: r1 = x; g1 = c2; b1 = 0; break;
    case 2: r1 = 0; g1 = c2; b1 = x; break;
    case 3: r1 = 0; g1 = x; b1 = c2; break;
    case 4: r1 = x; g1 = 0; b1 = c2; break;
    default: r1 = c2; g1 = 0; b1 = x; break;
  }
  out[0] = sat_rne(255.0 * (r1 + m));
  out[1] = sat_rne(255.0 * (g1 + m));
  out[2] = sat_rne(255.0 * (b1 + m));
}

EXPORT void orc_shift_hsv_pixel(const double shift[3], const uint8_t in[3], uint8_t out[3]) {
  shift_hsv_pixel(shift, in, out);
}

/* ======================================================================
 * Images.  in: h x w x c bytes, row stride is; out: out_h x out_w x c,
 * row stride os.
 * ====================================================================== */
#define PX(base, stride, c, y, x) ((base) + (int64_t)(y) * (stride) + (int64_t)(x) * (c))

/* Q5 bilinear sample of channel k at the Q5 source coordinates (Xq, Yq):
 * taps floor(Xq/32) and +1 (same for y) go through the border map; weights
 * (32-fx)(32-fy), fx(32-fy), (32-fx)fy, fx fy sum to 1024;
 * out = (sum + 512) / 1024 rounded down (round half up). */
static uint8_t q5_bilinear(const uint8_t* in, int h, int w, int c, int64_t is,
                           int k, int64_t xq, int64_t yq, int border_reflect) {
  int64_t ix = floor_div(xq, 32), fx = xq - 32 * ix;
  int64_t iy = floor_div(yq, 32), fy = yq - 32 * iy;
  int64_t xa, xb, ya, yb;
  if (border_reflect) {
    xa = reflect101(ix, w); xb = reflect101(ix + 1, w);
    ya = reflect101(iy, h); yb = reflect101(iy + 1, h);
  } else {   /* caller guarantees ix, iy in range; the +1 tap is clamped */
    xa = ix; xb = ix + 1 < w ? ix + 1 : w - 1;
    ya = iy; yb = iy + 1 < h ? iy + 1 : h - 1;
  }
  int64_t p00 = PX(in, is, c, ya, xa)[k], p01 = PX(in, is, c, ya, xb)[k];
  int64_t p10 = PX(in, is, c, yb, xa)[k], p11 = PX(in, is, c, yb, xb)[k];
  int64_t acc = (32 - fx) * (32 - fy) * p00 + fx * (32 - fy) * p01
              + (32 - fx) * fy * p10 + fx * fy * p11;
  return (uint8_t)((acc + 512) / 1024);
}

/* Half-pixel resize coordinate in Q5 (reading C-R): the source coordinate
 * of output sample d is (d + 0.5) * n_in / n_out - 0.5, rounded half up to
 * 1/32 px in exact integers, clamped below at 0; at or beyond the last
 * input sample it is pinned there with zero fraction. */
static int64_t resize_q5(int64_t d, int64_t n_in, int64_t n_out) {
  int64_t xq = floor_div(32 * ((2 * d + 1) * n_in - n_out) + n_out, 2 * n_out);
  if (xq < 0) xq = 0;
  if (floor_div(xq, 32) >= n_in - 1) xq = 32 * (n_in - 1);
  return xq;
}

/* nearest-neighbour resize index: the input sample that contains the
 * centre of output sample d. */
static int64_t resize_nearest(int64_t d, int64_t n_in, int64_t n_out) {
  int64_t i = floor_div((2 * d + 1) * n_in, 2 * n_out);
  return i < n_in - 1 ? i : n_in - 1;
}

static void apply_lut_image(const uint8_t lut[3][256], const uint8_t* in, int h, int w,
                            int64_t is, uint8_t* out, int64_t os) {
  for (int y = 0; y < h; y++)
    for (int x = 0; x < w; x++)
      for (int k = 0; k < 3; k++)
        PX(out, os, 3, y, x)[k] = lut[k][PX(in, is, 3, y, x)[k]];
}

/* The geometric index maps shared by images (bilinear or exact copy) and
 * masks (nearest): nearest != 0 selects the mask rule. */
static int apply_geometric(const orc_params* p, const uint8_t* in, int h, int w, int c,
                           int64_t is, uint8_t* out, int64_t os, int nearest) {
  int oh, ow;
  orc_output_shape(p, h, w, &oh, &ow);
  for (int y = 0; y < oh; y++)
    for (int x = 0; x < ow; x++)
      for (int k = 0; k < c; k++) {
        uint8_t* o = PX(out, os, c, y, x) + k;
        if (!p->apply) { *o = PX(in, is, c, y, x)[k]; continue; }
        switch (p->tid) {
          case T_HFLIP: *o = PX(in, is, c, y, w - 1 - x)[k]; break;
          case T_VFLIP: *o = PX(in, is, c, h - 1 - y, x)[k]; break;
          case T_TRANSPOSE: *o = PX(in, is, c, x, y)[k]; break;
          case T_ROT90: {
            /* k quarter turns counter-clockwise on screen */
            int64_t sy, sx;
            switch (p->k & 3) {
              case 0: sy = y; sx = x; break;
              case 1: sy = x; sx = w - 1 - y; break;
              case 2: sy = h - 1 - y; sx = w - 1 - x; break;
              default: sy = h - 1 - x; sx = y; break;
            }
            *o = PX(in, is, c, sy, sx)[k];
            break;
          }
          case T_RANDOM_CROP: *o = PX(in, is, c, p->y0 + y, p->x0 + x)[k]; break;
          case T_PAD_TO_SIZE:
            *o = PX(in, is, c, reflect101(y - p->y0, h), reflect101(x - p->x0, w))[k];
            break;
          case T_ROTATE: case T_SHIFT_SCALE_ROTATE: {
            int64_t X = p->q[0] * x + p->q[1] * y + p->q[2];
            int64_t Y = p->q[3] * x + p->q[4] * y + p->q[5];
            if (nearest) {
              int64_t sx = reflect101(floor_div(X + 32768, 65536), w);
              int64_t sy = reflect101(floor_div(Y + 32768, 65536), h);
              *o = PX(in, is, c, sy, sx)[k];
            } else {
              int64_t xq = floor_div(X + 1024, 2048), yq = floor_div(Y + 1024, 2048);
              *o = q5_bilinear(in, h, w, c, is, k, xq, yq, 1);
            }
            break;
          }
          case T_RESIZE: case T_RANDOM_SIZED_CROP: case T_RANDOM_RESIZED_CROP: {
            const uint8_t* win = PX(in, is, c, p->y0, p->x0);
            if (nearest) {
              int64_t sx = resize_nearest(x, p->cw, ow), sy = resize_nearest(y, p->ch, oh);
              *o = PX(win, is, c, sy, sx)[k];
            } else {
              int64_t xq = resize_q5(x, p->cw, ow), yq = resize_q5(y, p->ch, oh);
              *o = q5_bilinear(win, p->ch, p->cw, c, is, k, xq, yq, 0);
            }
            break;
          }
          case T_GRID_DISTORTION: {
            int64_t xq = orc_grid_q5(p, 0, x, w), yq = orc_grid_q5(p, 1, y, h);
            if (nearest) *o = PX(in, is, c, floor_div(yq + 16, 32), floor_div(xq + 16, 32))[k];
            else *o = q5_bilinear(in, h, w, c, is, k, xq, yq, 0);
            break;
          }
          case T_ELASTIC: {
            int32_t dx, dy;
            orc_elastic_disp(p, x, y, w, &dx, &dy);
            int64_t xq = 32 * (int64_t)x + dx, yq = 32 * (int64_t)y + dy;
            if (nearest) *o = PX(in, is, c, reflect101(floor_div(yq + 16, 32), h), reflect101(floor_div(xq + 16, 32), w))[k];
            else *o = q5_bilinear(in, h, w, c, is, k, xq, yq, 1);
            break;
          }
          default: return ORC_EINVAL;
        }
      }
  return ORC_OK;
}

EXPORT int orc_apply_image(const orc_params* p, const uint8_t* in, int h, int w, int c, int64_t is,
                           uint8_t* out, int64_t os) {
  switch (p->tid) {
    case T_BRIGHTNESS: case T_CONTRAST: case T_BRIGHTNESS_CONTRAST: case T_GAMMA: case T_SHIFT_RGB: {
      if (c != 3) return ORC_EINVAL;
      uint8_t lut[3][256];
      orc_build_lut(p, lut);
      apply_lut_image((const uint8_t(*)[256])lut, in, h, w, is, out, os);
      return ORC_OK;
    }
    case T_SHIFT_HSV:
      if (c != 3) return ORC_EINVAL;
      for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
          if (p->apply) shift_hsv_pixel(p->shift, PX(in, is, 3, y, x), PX(out, os, 3, y, x));
          else memcpy(PX(out, os, 3, y, x), PX(in, is, 3, y, x), 3);
        }
      return ORC_OK;
    case T_GRAYSCALE:
      if (c != 3) return ORC_EINVAL;
      for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
          const uint8_t* s = PX(in, is, 3, y, x);
          uint8_t* o = PX(out, os, 3, y, x);
          if (!p->apply) { memcpy(o, s, 3); continue; }
          int64_t g = rne_div(299 * (int64_t)s[0] + 587 * (int64_t)s[1] + 114 * (int64_t)s[2], 1000);
          o[0] = o[1] = o[2] = (uint8_t)g;
        }
      return ORC_OK;
    case T_EQUALIZE: {
      if (c != 3) return ORC_EINVAL;
      uint8_t lut[3][256];
      for (int k = 0; k < 3; k++) {
        uint64_t hist[256] = {0};
        for (int y = 0; y < h; y++)
          for (int x = 0; x < w; x++) hist[PX(in, is, 3, y, x)[k]]++;
        if (p->apply) orc_equalize_lut(hist, lut[k]);
        else for (int v = 0; v < 256; v++) lut[k][v] = (uint8_t)v;
      }
      apply_lut_image((const uint8_t(*)[256])lut, in, h, w, is, out, os);
      return ORC_OK;
    }
    default:
      return apply_geometric(p, in, h, w, c, is, out, os, 0);
  }
}

/* Masks follow the image's geometry with nearest sampling; transforms that
 * do not move pixels leave the mask unchanged. */
EXPORT int orc_apply_mask(const orc_params* p, const uint8_t* in, int h, int w, int c, int64_t is,
                          uint8_t* out, int64_t os) {
  switch (p->tid) {
    case T_BRIGHTNESS: case T_CONTRAST: case T_BRIGHTNESS_CONTRAST: case T_GAMMA: case T_SHIFT_RGB:
    case T_SHIFT_HSV: case T_GRAYSCALE: case T_EQUALIZE:
      for (int y = 0; y < h; y++) memcpy(out + (int64_t)y * os, in + (int64_t)y * is, (size_t)w * c);
      return ORC_OK;
    default:
      return apply_geometric(p, in, h, w, c, is, out, os, 1);
  }
}

/* ======================================================================
 * Boxes: float32 [n][4] xyxy in pixel-edge coordinates (the image spans
 * [0,W] x [0,H]).  Transformed in float64, clipped to the output image,
 * boxes with no area left are dropped, order kept.  Returns the count.
 * ====================================================================== */
EXPORT int orc_apply_boxes(const orc_params* p, int h, int w, const float* in, int n, float* out) {
  int oh, ow;
  orc_output_shape(p, h, w, &oh, &ow);
  int kept = 0;
  for (int i = 0; i < n; i++) {
    double x1 = in[4 * i], y1 = in[4 * i + 1], x2 = in[4 * i + 2], y2 = in[4 * i + 3];
    double a1 = x1, b1 = y1, a2 = x2, b2 = y2;
    if (p->apply) switch (p->tid) {
      case T_HFLIP: a1 = (double)w - x2; a2 = (double)w - x1; break;
      case T_VFLIP: b1 = (double)h - y2; b2 = (double)h - y1; break;
      case T_TRANSPOSE: a1 = y1; b1 = x1; a2 = y2; b2 = x2; break;
      case T_ROT90:
        switch (p->k & 3) {
          case 0: break;
          case 1: a1 = y1; a2 = y2; b1 = (double)w - x2; b2 = (double)w - x1; break;
          case 2: a1 = (double)w - x2; a2 = (double)w - x1; b1 = (double)h - y2; b2 = (double)h - y1; break;
          default: a1 = (double)h - y2; a2 = (double)h - y1; b1 = x1; b2 = x2; break;
        }
        break;
      case T_RANDOM_CROP:
        a1 = x1 - p->x0; a2 = x2 - p->x0; b1 = y1 - p->y0; b2 = y2 - p->y0; break;
      case T_PAD_TO_SIZE:
        a1 = x1 + p->x0; a2 = x2 + p->x0; b1 = y1 + p->y0; b2 = y2 + p->y0; break;
      case T_RESIZE: case T_RANDOM_SIZED_CROP: case T_RANDOM_RESIZED_CROP: {
        /* crop to the window (clip there first), then scale to the output */
        double cx1 = x1 - p->x0, cx2 = x2 - p->x0, cy1 = y1 - p->y0, cy2 = y2 - p->y0;
        if (cx1 < 0) cx1 = 0;
        if (cy1 < 0) cy1 = 0;
        if (cx2 > p->cw) cx2 = p->cw;
        if (cy2 > p->ch) cy2 = p->ch;
        a1 = cx1 * ow / p->cw; a2 = cx2 * ow / p->cw;
        b1 = cy1 * oh / p->ch; b2 = cy2 * oh / p->ch;
        break;
      }
      case T_ROTATE: case T_SHIFT_SCALE_ROTATE: {
        double xs[4] = {x1, x2, x1, x2}, ys[4] = {y1, y1, y2, y2};
        for (int j = 0; j < 4; j++) {
          double u = xs[j] - 0.5, v = ys[j] - 0.5;
          double tx = (p->m[0] * u + p->m[1] * v + p->m[2]) + 0.5;
          double ty = (p->m[3] * u + p->m[4] * v + p->m[5]) + 0.5;
          if (j == 0 || tx < a1) a1 = tx;
          if (j == 0 || tx > a2) a2 = tx;
          if (j == 0 || ty < b1) b1 = ty;
          if (j == 0 || ty > b2) b2 = ty;
        }
        break;
      }
      case T_GRID_DISTORTION:
        a1 = orc_grid_edge_inverse(p, 0, x1, w); a2 = orc_grid_edge_inverse(p, 0, x2, w);
        b1 = orc_grid_edge_inverse(p, 1, y1, h); b2 = orc_grid_edge_inverse(p, 1, y2, h);
        break;
      case T_ELASTIC:
        return -1;      /* boxes are not defined for a non-parametric distortion */
      default: break;   /* photometric: boxes unchanged */
    }
    if (a1 < 0) a1 = 0;
    if (b1 < 0) b1 = 0;
    if (a2 > ow) a2 = ow;
    if (b2 > oh) b2 = oh;
    if (a2 - a1 <= 0.0 || b2 - b1 <= 0.0) continue;
    out[4 * kept] = (float)a1; out[4 * kept + 1] = (float)b1;
    out[4 * kept + 2] = (float)a2; out[4 * kept + 3] = (float)b2;
    kept++;
  }
  return kept;
}

/* ======================================================================
 * Fused chain: RandomResizedCrop window resized
 * to out_h x out_w (Q5 bilinear), optional h-flip, brightness/contrast LUT,
 * saturation in float32, Normalize to bfloat16 NCHW.  Written as the plain
 * sequence of its steps with every intermediate materialised.
 * ====================================================================== */
static uint16_t f32_to_bf16_rne(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return (uint16_t)((u >> 16) | 0x40);
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}
EXPORT uint16_t orc_f32_to_bf16(float f) { return f32_to_bf16_rne(f); }

/* per-channel Normalize constants: k_c = 1/(255 std_c), m_c = -mean_c/std_c,
 * computed in float64 and rounded to float32. */
EXPORT void orc_normalize_consts(const double mean[3], const double stdv[3], float k[3], float m[3]) {
  for (int c = 0; c < 3; c++) {
    k[c] = (float)(1.0 / (255.0 * stdv[c]));
    m[c] = (float)(-mean[c] / stdv[c]);
  }
}

static uint8_t sat_rne_f32(float v) {
  float r = rintf(v);
  if (r < 0.0f) r = 0.0f;
  if (r > 255.0f) r = 255.0f;
  return (uint8_t)r;
}

/* The three jitter ops of mode 1 in the order of permutation index k
 * (0 BCS, 1 BSC, 2 CBS, 3 CSB, 4 SBC, 5 SCB; B = 0, C = 1, S = 2). */
EXPORT int orc_jitter_op(int k, int i) {
  static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  if (k < 0 || k > 5 || i < 0 || i > 2) return -1;
  return perm[k][i];
}

/* Contrast pivot of a uint8 RGB image: the round-half-even mean of the
 * integer BT.601 grey values rne((299 R + 587 G + 114 B) / 1000). */
EXPORT int orc_contrast_pivot(const uint8_t* img, size_t npx) {
  int64_t sum = 0;
  for (size_t i = 0; i < npx; i++) {
    sum += rne_div(299 * (int64_t)img[3 * i] + 587 * (int64_t)img[3 * i + 1] + 114 * (int64_t)img[3 * i + 2], 1000);
  }
  return (int)rne_div(sum, (int64_t)npx);
}

/* Colour jitter, mode 1 (the torchvision / PIL reading: a random order of
 * the three ops, each producing a uint8 image):
 *   B: v -> sat_rne(b v)                                  (float64)
 *   C: v -> sat_rne(m + c (v - m)), m = contrast pivot of the image as it
 *      is when C runs                                     (float64)
 *   S: per pixel, grey = 0.299 R + 0.587 G + 0.114 B in float32 fmas,
 *      v -> sat_rne(fmaf(s, v - grey, grey))              (float32)
 * applied in place to npx RGB pixels. */
EXPORT void orc_jitter_mode1(const orc_params* p, uint8_t* img, size_t npx) {
  for (int i = 0; i < 3; i++) {
    int op = orc_jitter_op(p->k, i);
    if (op == 0) {
      for (size_t j = 0; j < 3 * npx; j++) img[j] = sat_rne(p->beta * (double)img[j]);
    } else if (op == 1) {
      double m = (double)orc_contrast_pivot(img, npx);
      for (size_t j = 0; j < 3 * npx; j++) img[j] = sat_rne(m + p->alpha * ((double)img[j] - m));
    } else {
      float sf = (float)p->sat;
      for (size_t j = 0; j < npx; j++) {
        float r = img[3 * j], g = img[3 * j + 1], b = img[3 * j + 2];
        float grey = fmaf(0.114f, b, fmaf(0.587f, g, 0.299f * r));
        for (int c = 0; c < 3; c++) img[3 * j + c] = sat_rne_f32(fmaf(sf, (float)img[3 * j + c] - grey, grey));
      }
    }
  }
}

/* The chain with jitter mode 1: crop + resize, h-flip, the three jitter
 * ops in the record's order (uint8 after each), Normalize -> bf16 NCHW. */
EXPORT int orc_chain_image_jitter(const orc_params* p, const double mean[3], const double stdv[3],
                                  const uint8_t* in, int h, int w, int64_t is, uint16_t* out) {
  int oh = p->out_h, ow = p->out_w;
  size_t npx = (size_t)oh * ow;
  uint8_t* resized = (uint8_t*)malloc(npx * 3);
  uint8_t* cur = (uint8_t*)malloc(npx * 3);
  if (!resized || !cur) { free(resized); free(cur); return ORC_EINVAL; }
  orc_params rp = *p;
  rp.tid = T_RANDOM_RESIZED_CROP; rp.apply = 1;
  apply_geometric(&rp, in, h, w, 3, is, resized, (int64_t)ow * 3, 0);
  orc_params fp = *p;
  fp.tid = T_HFLIP; fp.apply = p->flip;
  apply_geometric(&fp, resized, oh, ow, 3, (int64_t)ow * 3, cur, (int64_t)ow * 3, 0);
  orc_jitter_mode1(p, cur, npx);
  float kc[3], mc[3];
  orc_normalize_consts(mean, stdv, kc, mc);
  for (int c = 0; c < 3; c++)
    for (size_t i = 0; i < npx; i++) out[(size_t)c * npx + i] = f32_to_bf16_rne(fmaf((float)cur[3 * i + c], kc[c], mc[c]));
  free(resized); free(cur);
  return ORC_OK;
}

EXPORT int orc_chain_image(const orc_params* p, const double mean[3], const double stdv[3],
                           const uint8_t* in, int h, int w, int64_t is, uint16_t* out) {
  int oh = p->out_h, ow = p->out_w;
  size_t npx = (size_t)oh * ow;
  uint8_t* resized = (uint8_t*)malloc(npx * 3);
  uint8_t* flipped = (uint8_t*)malloc(npx * 3);
  uint8_t* lutted = (uint8_t*)malloc(npx * 3);
  float* satd = (float*)malloc(npx * 3 * sizeof(float));
  if (!resized || !flipped || !lutted || !satd) { free(resized); free(flipped); free(lutted); free(satd); return ORC_EINVAL; }
  /* 1. crop + resize */
  orc_params rp = *p;
  rp.tid = T_RANDOM_RESIZED_CROP; rp.apply = 1;
  apply_geometric(&rp, in, h, w, 3, is, resized, (int64_t)ow * 3, 0);
  /* 2. h-flip */
  orc_params fp = *p;
  fp.tid = T_HFLIP; fp.apply = p->flip;
  apply_geometric(&fp, resized, oh, ow, 3, (int64_t)ow * 3, flipped, (int64_t)ow * 3, 0);
  /* 3. brightness/contrast LUT */
  uint8_t lut[3][256];
  orc_params lp = *p;
  lp.tid = T_CHAIN; lp.apply = 1;
  orc_build_lut(&lp, lut);
  apply_lut_image((const uint8_t(*)[256])lut, flipped, oh, ow, (int64_t)ow * 3, lutted, (int64_t)ow * 3);
  /* 4. saturation: blend each channel with the BT.601 grey value, float32 */
  float sf = (float)p->sat;
  for (size_t i = 0; i < npx; i++) {
    float r = lutted[3 * i], g = lutted[3 * i + 1], b = lutted[3 * i + 2];
    float grey = fmaf(0.114f, b, fmaf(0.587f, g, 0.299f * r));
    for (int c = 0; c < 3; c++) {
      float v = fmaf(sf, (float)lutted[3 * i + c] - grey, grey);
      if (v < 0.0f) v = 0.0f;
      if (v > 255.0f) v = 255.0f;
      satd[3 * i + c] = v;
    }
  }
  /* 5. Normalize -> bf16 NCHW */
  float kc[3], mc[3];
  orc_normalize_consts(mean, stdv, kc, mc);
  for (int c = 0; c < 3; c++)
    for (size_t i = 0; i < npx; i++)
      out[(size_t)c * npx + i] = f32_to_bf16_rne(fmaf(satd[3 * i + c], kc[c], mc[c]));
  free(resized); free(flipped); free(lutted); free(satd);
  return ORC_OK;
}

/* ======================================================================
 * Differentiable float path.
 * x: [B][C][H][W]; per image angle (deg), scale, tx, ty (fractions of W, H),
 * alpha, beta, gamma.  w = bilinear warp of x with zero border;
 * z = alpha w + beta; y = clamp(z, 0, 1)^gamma.
 *
 * Source coordinates come in two classes (`coords`):
 *   64: the inverse map evaluated in float64 -- the definition of the warp;
 *   32: the float32 coordinate class: the six inverse-map entries (computed
 *       in float64) rounded to float32 once, then
 *       sx = fma(a00, ox, fma(a01, oy, b0)) and sy = fma(a10, ox, fma(a11, oy, b1))
 *       as correctly rounded float32 fused multiply-adds.  This is the
 *       coordinate a float32 implementation of the warp samples at, so its
 *       floor cells -- and with them the piecewise-bilinear pieces whose
 *       boundaries gradients cannot cross smoothly -- are the same as the
 *       implementation's.  Everything after the coordinate (weights, taps,
 *       photometric step, gradients) stays float64 in both classes.
 * ====================================================================== */
typedef struct {
  double a00, a01, a10, a11, b0, b1, cs, sn, s, cx, cy, W, H, txp, typ;
  float f00, f01, f10, f11, fb0, fb1;   /* the float32 coordinate class */
} fwarp;

static void fwarp_setup(fwarp* g, double angle, double scale, double tx, double ty, int h, int w) {
  double rad = angle * (M_PI / 180.0);
  g->cs = cos(rad); g->sn = sin(rad); g->s = scale;
  g->cx = (double)(w - 1) * 0.5; g->cy = (double)(h - 1) * 0.5;
  g->W = w; g->H = h;
  g->txp = tx * (double)w; g->typ = ty * (double)h;
  g->a00 = g->cs / scale; g->a01 = -g->sn / scale; g->a10 = g->sn / scale; g->a11 = g->cs / scale;
  double ox = g->cx + g->txp, oy = g->cy + g->typ;
  g->b0 = g->cx - (g->a00 * ox + g->a01 * oy);
  g->b1 = g->cy - (g->a10 * ox + g->a11 * oy);
  g->f00 = (float)g->a00; g->f01 = (float)g->a01; g->f10 = (float)g->a10; g->f11 = (float)g->a11;
  g->fb0 = (float)g->b0; g->fb1 = (float)g->b1;
}

/* source coordinate (sx, sy) of output pixel (ox, oy) in coordinate class `coords` */
static void fwarp_coord(const fwarp* g, int coords, int ox, int oy, double* sx, double* sy) {
  if (coords == 32) {
    *sx = (double)fmaf(g->f00, (float)ox, fmaf(g->f01, (float)oy, g->fb0));
    *sy = (double)fmaf(g->f10, (float)ox, fmaf(g->f11, (float)oy, g->fb1));
  } else {
    *sx = g->a00 * ox + g->a01 * oy + g->b0;
    *sy = g->a10 * ox + g->a11 * oy + g->b1;
  }
}

static double tap(const double* img, int h, int w, int64_t x, int64_t y) {
  if (x < 0 || y < 0 || x >= w || y >= h) return 0.0;
  return img[y * w + x];
}

EXPORT void orc_warp_photo_fwd(int B, int C, int H, int W, int coords, const double* x,
                               const double* angle, const double* scale, const double* tx, const double* ty,
                               const double* alpha, const double* beta, const double* gamma,
                               double* warped, double* y) {
  for (int b = 0; b < B; b++) {
    fwarp g; fwarp_setup(&g, angle[b], scale[b], tx[b], ty[b], H, W);
    for (int c = 0; c < C; c++) {
      const double* img = x + ((size_t)b * C + c) * H * W;
      for (int oy = 0; oy < H; oy++)
        for (int ox = 0; ox < W; ox++) {
          double sx, sy;
          fwarp_coord(&g, coords, ox, oy, &sx, &sy);
          double fx0 = floor(sx), fy0 = floor(sy);
          double fx = sx - fx0, fy = sy - fy0;
          int64_t ix = (int64_t)fx0, iy = (int64_t)fy0;
          double v = (1 - fx) * (1 - fy) * tap(img, H, W, ix, iy) + fx * (1 - fy) * tap(img, H, W, ix + 1, iy)
                   + (1 - fx) * fy * tap(img, H, W, ix, iy + 1) + fx * fy * tap(img, H, W, ix + 1, iy + 1);
          size_t o = (((size_t)b * C + c) * H + oy) * W + ox;
          if (warped) warped[o] = v;
          double z = alpha[b] * v + beta[b];
          double zc = z < 0 ? 0 : (z > 1 ? 1 : z);
          y[o] = zc > 0 ? pow(zc, gamma[b]) : 0.0;
        }
    }
  }
}

/* Analytic adjoint of orc_warp_photo_fwd (same coordinate class).
 * dparams: [B][7] = (d angle [per degree], d scale, d tx, d ty, d alpha,
 * d beta, d gamma).  Optional (NULL = not wanted): adx [B][C][H][W] and
 * adparams [B][7] receive the sums of the absolute values of the terms each
 * gradient entry is a sum of -- for a parameter of the map, the terms are
 * the products of the coordinate partials dL/dsx, dL/dsy with each part of
 * the coordinate's derivative, taken apart as the map's rotation and
 * translation parts -- the scale against which the rounding error of any
 * finite-precision evaluation of the same sums is measured. */
EXPORT void orc_warp_photo_bwd(int B, int C, int H, int W, int coords, const double* x,
                               const double* angle, const double* scale, const double* tx, const double* ty,
                               const double* alpha, const double* beta, const double* gamma,
                               const double* gy, double* dx, double* dparams, double* adx, double* adparams) {
  memset(dx, 0, sizeof(double) * (size_t)B * C * H * W);
  if (adx) memset(adx, 0, sizeof(double) * (size_t)B * C * H * W);
  for (int b = 0; b < B; b++) {
    fwarp g; fwarp_setup(&g, angle[b], scale[b], tx[b], ty[b], H, W);
    double dang = 0, dsc = 0, dtx = 0, dty = 0, dal = 0, dbe = 0, dga = 0;
    double aang = 0, asc = 0, atx = 0, aty = 0, aal = 0, abe = 0, aga = 0;
    for (int c = 0; c < C; c++) {
      const double* img = x + ((size_t)b * C + c) * H * W;
      double* dimg = dx + ((size_t)b * C + c) * H * W;
      double* aimg = adx ? adx + ((size_t)b * C + c) * H * W : NULL;
      for (int oy = 0; oy < H; oy++)
        for (int ox = 0; ox < W; ox++) {
          double sx, sy;
          fwarp_coord(&g, coords, ox, oy, &sx, &sy);
          double fx0 = floor(sx), fy0 = floor(sy);
          double fx = sx - fx0, fy = sy - fy0;
          int64_t ix = (int64_t)fx0, iy = (int64_t)fy0;
          double v00 = tap(img, H, W, ix, iy), v10 = tap(img, H, W, ix + 1, iy);
          double v01 = tap(img, H, W, ix, iy + 1), v11 = tap(img, H, W, ix + 1, iy + 1);
          double v = (1 - fx) * (1 - fy) * v00 + fx * (1 - fy) * v10 + (1 - fx) * fy * v01 + fx * fy * v11;
          double z = alpha[b] * v + beta[b];
          size_t o = (((size_t)b * C + c) * H + oy) * W + ox;
          double g_out = gy[o];
          if (!(z > 0.0 && z < 1.0)) continue;       /* clamp: zero gradient */
          double zg = pow(z, gamma[b]);
          double gz = g_out * gamma[b] * pow(z, gamma[b] - 1.0);
          dga += g_out * zg * log(z);
          dal += gz * v;
          dbe += gz;
          aga += fabs(g_out * zg * log(z));
          aal += fabs(gz * v);
          abe += fabs(gz);
          double gw = gz * alpha[b];
          /* image adjoint: scatter to the in-range taps */
          double wk[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
          int64_t tx_[4] = {ix, ix + 1, ix, ix + 1}, ty_[4] = {iy, iy, iy + 1, iy + 1};
          for (int k = 0; k < 4; k++)
            if (tx_[k] >= 0 && tx_[k] < W && ty_[k] >= 0 && ty_[k] < H) {
              dimg[ty_[k] * W + tx_[k]] += gw * wk[k];
              if (aimg) aimg[ty_[k] * W + tx_[k]] += fabs(gw * wk[k]);
            }
          /* coordinate partials */
          double dsx = gw * ((1 - fy) * (v10 - v00) + fy * (v11 - v01));
          double dsy = gw * ((1 - fx) * (v01 - v00) + fx * (v11 - v10));
          double xp = ox - g.cx - g.txp, yp = oy - g.cy - g.typ;
          double dsx_dth = (-g.sn * xp - g.cs * yp) / g.s;
          double dsy_dth = (g.cs * xp - g.sn * yp) / g.s;
          dang += dsx * dsx_dth + dsy * dsy_dth;
          dsc += dsx * (-(sx - g.cx) / g.s) + dsy * (-(sy - g.cy) / g.s);
          dtx += dsx * (-g.cs * g.W / g.s) + dsy * (-g.sn * g.W / g.s);
          dty += dsx * (g.sn * g.H / g.s) + dsy * (-g.cs * g.H / g.s);
          aang += (fabs(dsx) * (fabs(g.sn * xp) + fabs(g.cs * yp)) + fabs(dsy) * (fabs(g.cs * xp) + fabs(g.sn * yp))) / g.s;
          asc += (fabs(dsx) * fabs(sx - g.cx) + fabs(dsy) * fabs(sy - g.cy)) / g.s;
          atx += (fabs(dsx) * fabs(g.cs) + fabs(dsy) * fabs(g.sn)) * g.W / g.s;
          aty += (fabs(dsx) * fabs(g.sn) + fabs(dsy) * fabs(g.cs)) * g.H / g.s;
        }
    }
    double* dp = dparams + 7 * (size_t)b;
    dp[0] = dang * (M_PI / 180.0); dp[1] = dsc; dp[2] = dtx; dp[3] = dty;
    dp[4] = dal; dp[5] = dbe; dp[6] = dga;
    if (adparams) {
      double* ap = adparams + 7 * (size_t)b;
      ap[0] = aang * (M_PI / 180.0); ap[1] = asc; ap[2] = atx; ap[3] = aty;
      ap[4] = aal; ap[5] = abe; ap[6] = aga;
    }
  }
}

/* ======================================================================
 * Targets of the fused chain (Sec. II-A: a crop + flip applied to an image
 * together with its masks and boxes; Fig. 2 detection).
 *
 * Masks: an N-plane uint8 mask (HWC, c = N instance planes) goes through the
 * chain's crop window with nearest resampling to out_h x out_w (the resize
 * rule of the masks) and the same h-flip.
 * Boxes: crop to the window (clip there), scale to the output, flip, clip
 * to the output and drop boxes with no area left, order kept.
 * Box-safe windows: the chain's crop window is drawn so that it contains the
 * union of the image's boxes: with the union clipped to the image and
 * widened to whole pixels [ux0, ux1) x [uy0, uy1), x0 = randint[0, ux0],
 * x1 = ux1 + randint[0, W - ux1] (window [x0, x1)), then the same for y;
 * without boxes (or an empty union) the chain's RandomResizedCrop draw is
 * used.  The flip and jitter draws follow as in the chain.
 * ====================================================================== */
EXPORT int orc_chain_mask(const orc_params* p, const uint8_t* in, int h, int w, int c, int64_t is,
                          uint8_t* out, int64_t os) {
  int oh = p->out_h, ow = p->out_w;
  if (p->y0 < 0 || p->x0 < 0 || p->y0 + p->ch > h || p->x0 + p->cw > w) return ORC_ESHAPE;
  for (int y = 0; y < oh; y++)
    for (int x = 0; x < ow; x++) {
      int xr = p->flip ? ow - 1 - x : x;
      int64_t sy = p->y0 + resize_nearest(y, p->ch, oh), sx = p->x0 + resize_nearest(xr, p->cw, ow);
      for (int k = 0; k < c; k++) PX(out, os, c, y, x)[k] = PX(in, is, c, sy, sx)[k];
    }
  return ORC_OK;
}

EXPORT int orc_chain_boxes(const orc_params* p, const float* in, int n, float* out) {
  int oh = p->out_h, ow = p->out_w, kept = 0;
  for (int i = 0; i < n; i++) {
    double cx1 = in[4 * i] - p->x0, cy1 = in[4 * i + 1] - p->y0, cx2 = in[4 * i + 2] - p->x0, cy2 = in[4 * i + 3] - p->y0;
    if (cx1 < 0) cx1 = 0;
    if (cy1 < 0) cy1 = 0;
    if (cx2 > p->cw) cx2 = p->cw;
    if (cy2 > p->ch) cy2 = p->ch;
    double a1 = cx1 * ow / p->cw, a2 = cx2 * ow / p->cw, b1 = cy1 * oh / p->ch, b2 = cy2 * oh / p->ch;
    if (p->flip) { double t = a1; a1 = (double)ow - a2; a2 = (double)ow - t; }
    if (a1 < 0) a1 = 0;
    if (b1 < 0) b1 = 0;
    if (a2 > ow) a2 = ow;
    if (b2 > oh) b2 = oh;
    if (a2 - a1 <= 0.0 || b2 - b1 <= 0.0) continue;
    out[4 * kept] = (float)a1; out[4 * kept + 1] = (float)b1;
    out[4 * kept + 2] = (float)a2; out[4 * kept + 3] = (float)b2;
    kept++;
  }
  return kept;
}

EXPORT int orc_sample_chain_box_safe(const orc_cfg* cfg, uint64_t seed, uint64_t stream_id, uint32_t index,
                                     int h, int w, const float* boxes, int nb, orc_params* p) {
  if (cfg->tid != T_CHAIN) return ORC_EINVAL;
  memset(p, 0, sizeof(*p));
  if (h <= 0 || w <= 0) return ORC_ESHAPE;
  if (cfg->out_h <= 0 || cfg->out_w <= 0) return ORC_ESHAPE;
  orc_stream s; stream_init(&s, seed, stream_id, index);
  p->tid = T_CHAIN; p->in_h = h; p->in_w = w;
  p->alpha = 1.0; p->beta = 0.0; p->gamma = 1.0; p->sat = 1.0; p->scale = 1.0;
  (void)stream_uniform01(&s);                 /* the probability draw; the chain always applies */
  p->apply = 1;
  p->out_h = cfg->out_h; p->out_w = cfg->out_w;
  double ux1 = 0, uy1 = 0, ux2 = 0, uy2 = 0;
  int have = 0;
  for (int i = 0; i < nb; i++) {
    double a = boxes[4 * i], b = boxes[4 * i + 1], c = boxes[4 * i + 2], d = boxes[4 * i + 3];
    if (a < 0) a = 0;
    if (b < 0) b = 0;
    if (c > w) c = w;
    if (d > h) d = h;
    if (c <= a || d <= b) continue;
    if (!have || a < ux1) ux1 = a;
    if (!have || b < uy1) uy1 = b;
    if (!have || c > ux2) ux2 = c;
    if (!have || d > uy2) uy2 = d;
    have = 1;
  }
  if (have) {
    int x0i = (int)floor(ux1), y0i = (int)floor(uy1), x1i = (int)ceil(ux2), y1i = (int)ceil(uy2);
    int x0 = stream_randint(&s, x0i);
    int x1 = x1i + stream_randint(&s, w - x1i);
    int y0 = stream_randint(&s, y0i);
    int y1 = y1i + stream_randint(&s, h - y1i);
    p->x0 = x0; p->cw = x1 - x0; p->y0 = y0; p->ch = y1 - y0;
  } else {
    sample_rrc(&s, h, w, cfg->lo[0], cfg->hi[0], cfg->lo[1], cfg->hi[1], &p->y0, &p->x0, &p->ch, &p->cw);
  }
  p->flip = stream_uniform01(&s) < 0.5;
  p->beta = stream_uniform(&s, cfg->lo[2], cfg->hi[2]);
  p->alpha = stream_uniform(&s, cfg->lo[2], cfg->hi[2]);
  p->sat = stream_uniform(&s, cfg->lo[2], cfg->hi[2]);
  p->k = stream_randint(&s, 5);
  return ORC_OK;
}

