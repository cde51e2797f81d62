// alb_sample.cu -- parameter sampling (Sec. II: transforms are applied with
// sampled parameters).  One __host__ __device__ implementation serves the host
// entry point alb_sample_params and the device kernel of alb_sample_params_batch.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  The word
// stream of image `index` is the sequence of Philox blocks with counter
// (j, index, stream lo, stream hi), key (seed lo, seed hi), words 0..3 of block
// 0, then block 1, ...  Uniform doubles take 27 + 26 bits of two words;
// integers in [0, n] use Lemire's multiply-shift with rejection (2019).
#include <cmath>
#include <cstring>

#include "alb_common.cuh"
#include "alb_distort.cuh"

namespace alb {

struct Philox {
  uint32_t key0, key1, index, s_lo, s_hi, block;
  uint32_t buf[4];
  int pos;
};

ALB_HD void ph_init(Philox& s, uint64_t seed, uint64_t sid, uint32_t index) {
  s.key0 = (uint32_t)seed; s.key1 = (uint32_t)(seed >> 32);
  s.index = index; s.s_lo = (uint32_t)sid; s.s_hi = (uint32_t)(sid >> 32);
  s.block = 0; s.pos = 4;
}

ALB_HD uint32_t ph_word(Philox& s) {
  if (s.pos == 4) {
    philox_block(s.block, s.index, s.s_lo, s.s_hi, s.key0, s.key1, s.buf);
    s.block++;
    s.pos = 0;
  }
  return s.buf[s.pos++];
}

ALB_HD double ph_u01(Philox& s) {
  uint32_t a = ph_word(s) >> 5;
  uint32_t b = ph_word(s) >> 6;
  uint64_t v = (uint64_t)a * 67108864ull + b;
  return (double)v * (1.0 / 9007199254740992.0);
}

ALB_HD double ph_uniform(Philox& s, double lo, double hi) {
  double u = ph_u01(s);
  double span = hi - lo;
  double t = span * u;
  return lo + t;
}

ALB_HD int32_t ph_randint(Philox& s, int32_t n) {  // [0, n]
  uint32_t range = (uint32_t)n + 1u;
  uint64_t m = (uint64_t)ph_word(s) * range;
  uint32_t low = (uint32_t)m;
  if (low < range) {
    uint32_t thr = (0u - range) % range;
    while (low < thr) {
      m = (uint64_t)ph_word(s) * range;
      low = (uint32_t)m;
    }
  }
  return (int32_t)(m >> 32);
}

// Warp geometry (rotation about the centre, scale, shift): forward matrix in
// float64 and the inverse quantised to Q16 (round half even).
ALB_HD void warp_geometry(alb_params& p, int32_t h, int32_t w) {
  const double kDeg = 3.14159265358979323846 / 180.0;
  double rad = p.angle * kDeg;
  double cs = cos(rad), sn = sin(rad);
  double s = p.scale;
  double cx = (double)(w - 1) * 0.5, cy = (double)(h - 1) * 0.5;
  double tx = p.dx * (double)w, ty = p.dy * (double)h;
  double m00 = s * cs, m01 = s * sn, m10 = -(s * sn), m11 = s * cs;
  p.m[0] = m00; p.m[1] = m01; p.m[3] = m10; p.m[4] = m11;
  p.m[2] = (cx + tx) - (m00 * cx + m01 * cy);
  p.m[5] = (cy + ty) - (m10 * cx + m11 * cy);
  double a00 = cs / s, a01 = -sn / s, a10 = sn / s, a11 = cs / s;
  double ox = cx + tx, oy = cy + ty;
  double b0 = cx - (a00 * ox + a01 * oy);
  double b1 = cy - (a10 * ox + a11 * oy);
  p.q[0] = llrint(a00 * 65536.0); p.q[1] = llrint(a01 * 65536.0); p.q[2] = llrint(b0 * 65536.0);
  p.q[3] = llrint(a10 * 65536.0); p.q[4] = llrint(a11 * 65536.0); p.q[5] = llrint(b1 * 65536.0);
}

// RandomResizedCrop window: ten attempts of (area fraction, log-aspect),
// sides rounded half even; else the widest centred crop in the aspect range.
ALB_HD void sample_rrc(Philox& s, int32_t h, int32_t w, double slo, double shi, double rlo, double rhi,
                       alb_params& p) {
  double area = (double)h * (double)w;
  double lrlo = log(rlo), lrhi = log(rhi);
  for (int attempt = 0; attempt < 10; attempt++) {
    double target = area * ph_uniform(s, slo, shi);
    double ar = exp(ph_uniform(s, lrlo, lrhi));
    double fw = rint(sqrt(target * ar));
    double fh = rint(sqrt(target / ar));
    if (fw > 0.0 && fh > 0.0 && fw <= (double)w && fh <= (double)h) {
      p.cw = (int32_t)fw; p.ch = (int32_t)fh;
      p.y0 = ph_randint(s, h - p.ch);
      p.x0 = ph_randint(s, w - p.cw);
      return;
    }
  }
  double in_ratio = (double)w / (double)h;
  if (in_ratio < rlo) { p.cw = w; p.ch = (int32_t)rint((double)w / rlo); }
  else if (in_ratio > rhi) { p.ch = h; p.cw = (int32_t)rint((double)h * rhi); }
  else { p.cw = w; p.ch = h; }
  if (p.ch > h) p.ch = h;
  if (p.cw > w) p.cw = w;
  p.y0 = (h - p.ch) / 2;
  p.x0 = (w - p.cw) / 2;
}

ALB_HD void params_identity(alb_params& p, int32_t tid, int32_t h, int32_t w) {
  memset(&p, 0, sizeof(p));
  p.tid = tid; p.in_h = h; p.in_w = w; p.out_h = h; p.out_w = w;
  p.alpha = 1.0; p.gamma = 1.0; p.sat = 1.0; p.scale = 1.0;
}

ALB_HD int sample_one(const alb_sample_cfg& cfg, uint64_t seed, uint64_t sid, uint32_t index, int32_t h,
                      int32_t w, alb_params& p) {
  params_identity(p, cfg.tid, h, w);
  if (h <= 0 || w <= 0) return ALB_ESHAPE;
  Philox s;
  ph_init(s, seed, sid, index);
  p.apply = ph_u01(s) < cfg.p;
  switch (cfg.tid) {
    case ALB_HFLIP: case ALB_VFLIP: case ALB_GRAYSCALE: case ALB_EQUALIZE: case ALB_TRANSPOSE:
      break;
    case ALB_ROT90:
      p.k = ph_randint(s, 3);
      break;
    case ALB_RANDOM_CROP:
      p.apply = 1;
      if (cfg.out_h <= 0 || cfg.out_w <= 0 || cfg.out_h > h || cfg.out_w > w) return ALB_ESHAPE;
      p.out_h = cfg.out_h; p.out_w = cfg.out_w; p.ch = cfg.out_h; p.cw = cfg.out_w;
      p.y0 = ph_randint(s, h - cfg.out_h);
      p.x0 = ph_randint(s, w - cfg.out_w);
      break;
    case ALB_PAD_TO_SIZE:
      p.apply = 1;
      p.out_h = h > cfg.out_h ? h : cfg.out_h;
      p.out_w = w > cfg.out_w ? w : cfg.out_w;
      p.y0 = (p.out_h - h) / 2;
      p.x0 = (p.out_w - w) / 2;
      break;
    case ALB_BRIGHTNESS:
      p.beta = ph_uniform(s, cfg.lo[0], cfg.hi[0]);
      break;
    case ALB_CONTRAST:
      p.alpha = ph_uniform(s, cfg.lo[0], cfg.hi[0]);
      break;
    case ALB_BRIGHTNESS_CONTRAST:
      p.alpha = ph_uniform(s, cfg.lo[0], cfg.hi[0]);
      p.beta = ph_uniform(s, cfg.lo[1], cfg.hi[1]);
      break;
    case ALB_GAMMA:
      p.gamma = ph_uniform(s, cfg.lo[0], cfg.hi[0]);
      break;
    case ALB_SHIFT_RGB: case ALB_SHIFT_HSV:
      for (int c = 0; c < 3; c++) p.shift[c] = ph_uniform(s, cfg.lo[c], cfg.hi[c]);
      break;
    case ALB_ROTATE:
      p.angle = ph_uniform(s, cfg.lo[0], cfg.hi[0]);
      warp_geometry(p, h, w);
      break;
    case ALB_SHIFT_SCALE_ROTATE:
      p.dx = ph_uniform(s, cfg.lo[0], cfg.hi[0]);
      p.dy = ph_uniform(s, cfg.lo[0], cfg.hi[0]);
      p.scale = ph_uniform(s, cfg.lo[1], cfg.hi[1]);
      p.angle = ph_uniform(s, cfg.lo[2], cfg.hi[2]);
      warp_geometry(p, h, w);
      break;
    case ALB_RESIZE:
      p.apply = 1;
      if (cfg.out_h <= 0 || cfg.out_w <= 0) return ALB_ESHAPE;
      p.out_h = cfg.out_h; p.out_w = cfg.out_w;
      p.ch = h; p.cw = w;   // the window is the whole image
      break;
    case ALB_RANDOM_SIZED_CROP: {
      p.apply = 1;
      if (cfg.out_h <= 0 || cfg.out_w <= 0) return ALB_ESHAPE;
      p.out_h = cfg.out_h; p.out_w = cfg.out_w;
      int32_t mside = h < w ? h : w;
      int32_t lo = (int32_t)ceil(cfg.lo[0] * (double)mside);
      int32_t hi = (int32_t)floor(cfg.hi[0] * (double)mside);
      if (lo < 1) lo = 1;
      if (hi > mside) hi = mside;
      if (hi < lo) return ALB_ESHAPE;
      int32_t side = lo + ph_randint(s, hi - lo);
      p.ch = side; p.cw = side;
      p.y0 = ph_randint(s, h - side);
      p.x0 = ph_randint(s, w - side);
      break;
    }
    case ALB_RANDOM_RESIZED_CROP:
      p.apply = 1;
      if (cfg.out_h <= 0 || cfg.out_w <= 0) return ALB_ESHAPE;
      p.out_h = cfg.out_h; p.out_w = cfg.out_w;
      sample_rrc(s, h, w, cfg.lo[0], cfg.hi[0], cfg.lo[1], cfg.hi[1], p);
      break;
    case ALB_GRID_DISTORTION: {
      // G cells per axis (lo[1], default 5, at most 12); per cell 1 + U[lo[0], hi[0]]
      // kept as Q14 integers, x cells then y cells
      const int g = cfg.lo[1] > 0 ? (int)cfg.lo[1] : 5;
      if (g < 1 || g > kGridMaxCells) return ALB_EINVAL;
      p.k = g;
      for (int j = 0; j < 2 * g; j++) {
        const double d = 1.0 + ph_uniform(s, cfg.lo[0], cfg.hi[0]);
        int64_t dq = (int64_t)rint(d * 16384.0);
        if (dq < 1) dq = 1;
        if (dq > 32767) dq = 32767;
        const int slot = j < g ? j : 12 + (j - g);
        uint64_t w = (uint64_t)p.q[slot >> 2];
        const int sh = 16 * (slot & 3);
        w = (w & ~((uint64_t)0xFFFF << sh)) | ((uint64_t)(uint16_t)dq << sh);
        p.q[slot >> 2] = (int64_t)w;
      }
      break;
    }
    case ALB_ELASTIC: {
      // amplitude lo[0] px (Q5: k = rne(32 a)), lattice spacing 2^cw px (lo[1], default 5);
      // the lattice comes from the image's own Philox blocks (alb_distort.cuh)
      const double a = cfg.lo[0];
      const int sh = cfg.lo[1] > 0 ? (int)cfg.lo[1] : 5;
      if (!(a >= 0.0 && a <= 4096.0) || sh < 2 || sh > 8) return ALB_EINVAL;
      p.k = (int32_t)rint(a * 32.0);
      p.cw = sh;
      p.q[0] = (int64_t)seed; p.q[1] = (int64_t)sid; p.q[2] = (int64_t)index;
      break;
    }
    case ALB_CHAIN:
      p.apply = 1;
      if (cfg.out_h <= 0 || cfg.out_w <= 0) return ALB_ESHAPE;
      p.out_h = cfg.out_h; p.out_w = cfg.out_w;
      sample_rrc(s, h, w, cfg.lo[0], cfg.hi[0], cfg.lo[1], cfg.hi[1], p);
      p.flip = ph_u01(s) < 0.5;
      p.beta = ph_uniform(s, cfg.lo[2], cfg.hi[2]);   // brightness factor
      p.alpha = ph_uniform(s, cfg.lo[2], cfg.hi[2]);  // contrast factor
      p.sat = ph_uniform(s, cfg.lo[2], cfg.hi[2]);    // saturation factor
      p.k = ph_randint(s, 5);                          // order of the jitter ops, 0..5 (jitter mode 1)
      break;
    default:
      return ALB_EINVAL;
  }
  return ALB_OK;
}

// The chain's record with a box-safe crop window: the window contains the
// union of the image's boxes (clipped to the image, widened to whole pixels
// [ux0, ux1) x [uy0, uy1)): x0 = randint[0, ux0], x1 = ux1 + randint[0, W - ux1],
// then y; without boxes (or an empty union) the chain's RandomResizedCrop
// draw.  The probability, flip and jitter draws are those of the chain.
ALB_HD int sample_chain_box_safe(const alb_sample_cfg& cfg, uint64_t seed, uint64_t sid, uint32_t index, int32_t h,
                                 int32_t w, const float* boxes, int32_t nb, alb_params& p) {
  params_identity(p, ALB_CHAIN, h, w);
  if (cfg.tid != ALB_CHAIN) return ALB_EINVAL;
  if (h <= 0 || w <= 0 || cfg.out_h <= 0 || cfg.out_w <= 0) return ALB_ESHAPE;
  Philox s;
  ph_init(s, seed, sid, index);
  (void)ph_u01(s);                 // the probability draw; the chain always applies
  p.apply = 1;
  p.out_h = cfg.out_h; p.out_w = cfg.out_w;
  double ux1 = 0, uy1 = 0, ux2 = 0, uy2 = 0;
  bool have = false;
  for (int32_t i = 0; i < nb; i++) {
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
    have = true;
  }
  if (have) {
    const int32_t x0i = (int32_t)floor(ux1), y0i = (int32_t)floor(uy1), x1i = (int32_t)ceil(ux2), y1i = (int32_t)ceil(uy2);
    const int32_t x0 = ph_randint(s, x0i);
    const int32_t x1 = x1i + ph_randint(s, w - x1i);
    const int32_t y0 = ph_randint(s, y0i);
    const int32_t y1 = y1i + ph_randint(s, h - y1i);
    p.x0 = x0; p.cw = x1 - x0; p.y0 = y0; p.ch = y1 - y0;
  } else {
    sample_rrc(s, h, w, cfg.lo[0], cfg.hi[0], cfg.lo[1], cfg.hi[1], p);
  }
  p.flip = ph_u01(s) < 0.5;
  p.beta = ph_uniform(s, cfg.lo[2], cfg.hi[2]);
  p.alpha = ph_uniform(s, cfg.lo[2], cfg.hi[2]);
  p.sat = ph_uniform(s, cfg.lo[2], cfg.hi[2]);
  p.k = ph_randint(s, 5);
  return ALB_OK;
}

__global__ void k_sample_box_safe(alb_sample_cfg cfg, uint64_t seed, uint64_t sid, uint32_t first, int32_t n,
                                  const alb_image* __restrict__ imgs, const float* __restrict__ boxes,
                                  const int32_t* __restrict__ nbox, int32_t cap, alb_params* __restrict__ out,
                                  int32_t* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const alb_image im = imgs[i];
  int32_t nb = nbox[i];
  if (nb < 0 || nb > cap) { dev_fail(status, ALB_ECAPACITY); nb = nb < 0 ? 0 : cap; }
  alb_params p;
  int rc = sample_chain_box_safe(cfg, seed, sid, first + (uint32_t)i, im.h, im.w, boxes + (int64_t)i * cap * 4, nb, p);
  if (rc != ALB_OK) {
    params_identity(p, ALB_CHAIN, im.h, im.w);
    dev_fail(status, rc);
  }
  out[i] = p;
}

__global__ void k_sample(alb_sample_cfg cfg, uint64_t seed, uint64_t sid, uint32_t first, int32_t n,
                         const alb_image* __restrict__ imgs, alb_params* __restrict__ out, int32_t* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  alb_image im = imgs[i];
  alb_params p;
  int rc = sample_one(cfg, seed, sid, first + (uint32_t)i, im.h, im.w, p);
  if (rc != ALB_OK) {
    params_identity(p, cfg.tid, im.h, im.w);
    dev_fail(status, rc);
  }
  out[i] = p;
}

}  // namespace alb

using namespace alb;

extern "C" alb_status alb_sample_params(const alb_sample_cfg* cfg, uint64_t seed, uint64_t stream_id,
                                        uint32_t index, int32_t h, int32_t w, alb_params* out) {
  ALB_REQUIRE(cfg && out, ALB_EINVAL, "alb_sample_params: null argument");
  int rc = sample_one(*cfg, seed, stream_id, index, h, w, *out);
  if (rc == ALB_EINVAL) set_error("alb_sample_params: unknown transform id %d", cfg->tid);
  if (rc == ALB_ESHAPE) set_error("alb_sample_params: transform %d does not fit a %dx%d image", cfg->tid, h, w);
  return (alb_status)rc;
}

extern "C" alb_status alb_sample_params_batch(const alb_sample_cfg* cfg, uint64_t seed, uint64_t stream_id,
                                              uint32_t first_index, int32_t n, const alb_image* images_dev,
                                              alb_params* params_dev, int32_t* dev_status, void* stream) {
  ALB_REQUIRE(cfg, ALB_EINVAL, "alb_sample_params_batch: null cfg");
  ALB_REQUIRE(n >= 0, ALB_EINVAL, "alb_sample_params_batch: negative n");
  if (n == 0) return ALB_OK;
  ALB_REQUIRE(images_dev && params_dev, ALB_EINVAL, "alb_sample_params_batch: null device array");
  ALB_REQUIRE(cfg->tid >= ALB_HFLIP && cfg->tid <= ALB_ELASTIC, ALB_EINVAL,
              "alb_sample_params_batch: unknown transform id %d", cfg->tid);
  cudaStream_t st = (cudaStream_t)stream;
  k_sample<<<(n + 127) / 128, 128, 0, st>>>(*cfg, seed, stream_id, first_index, n, images_dev, params_dev,
                                            dev_status);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

extern "C" alb_status alb_sample_chain_box_safe(const alb_sample_cfg* cfg, uint64_t seed, uint64_t stream_id,
                                                 uint32_t index, int32_t h, int32_t w, const float* boxes,
                                                 int32_t n_boxes, alb_params* out) {
  ALB_REQUIRE(cfg && out && n_boxes >= 0 && (boxes || n_boxes == 0), ALB_EINVAL,
              "alb_sample_chain_box_safe: bad argument");
  ALB_REQUIRE(cfg->tid == ALB_CHAIN, ALB_EINVAL, "alb_sample_chain_box_safe: cfg tid must be ALB_CHAIN");
  int rc = sample_chain_box_safe(*cfg, seed, stream_id, index, h, w, boxes, n_boxes, *out);
  if (rc != ALB_OK) {
    set_error("alb_sample_chain_box_safe: status %d for a %dx%d image", rc, h, w);
    return (alb_status)rc;
  }
  return ALB_OK;
}

extern "C" alb_status alb_sample_chain_box_safe_batch(const alb_sample_cfg* cfg, uint64_t seed, uint64_t stream_id,
                                                       uint32_t first_index, int32_t n, const alb_image* images_dev,
                                                       const float* boxes_dev, const int32_t* n_boxes_dev,
                                                       int32_t box_cap, alb_params* params_dev, int32_t* dev_status,
                                                       void* stream) {
  ALB_REQUIRE(cfg, ALB_EINVAL, "alb_sample_chain_box_safe_batch: null cfg");
  ALB_REQUIRE(cfg->tid == ALB_CHAIN, ALB_EINVAL, "alb_sample_chain_box_safe_batch: cfg tid must be ALB_CHAIN");
  ALB_REQUIRE(n >= 0, ALB_EINVAL, "alb_sample_chain_box_safe_batch: negative n");
  if (n == 0) return ALB_OK;
  ALB_REQUIRE(images_dev && params_dev && boxes_dev && n_boxes_dev && box_cap > 0, ALB_EINVAL,
              "alb_sample_chain_box_safe_batch: null device array or box_cap <= 0");
  k_sample_box_safe<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*cfg, seed, stream_id, first_index, n,
                                                                      images_dev, boxes_dev, n_boxes_dev, box_cap,
                                                                      params_dev, dev_status);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

