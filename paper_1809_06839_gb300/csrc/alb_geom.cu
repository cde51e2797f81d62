// alb_geom.cu -- geometric transforms of images and masks (Table I: RandomCrop,
// PadToSize, HorizontalFlip, VerticalFlip, Rotate, ShiftScaleRotate; Sec. II-A/B:
// random sized crop, rotations, reflections, scaling, masks transformed "in the
// same way"), and the box transforms (Sec. II-A: bounding boxes).
//
// Work decomposition (all kernels here): a ragged batch is split into items of
// (image, block of output rows) by k_plan; a persistent grid (SMs x CTAs/SM)
// takes contiguous ranges of items.  Threads of a CTA walk the item's output
// bytes in aligned 4-byte slots (consecutive lanes -> consecutive slots), so
// every warp store is a coalesced 128-byte line and every warp gather of one
// byte position touches at most a few consecutive source lines.
#include "alb_common.cuh"
#include "alb_kernels.cuh"
#include "alb_distort.cuh"

namespace alb {

// ------------------------------------------------------------------ plan
__global__ void k_plan(ImgList out, int32_t n, int32_t target, int32_t* __restrict__ prefix,
                       int32_t* __restrict__ rows_per_item, PlanCheck chk) {
  __shared__ int32_t wsum[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    int i = base + threadIdx.x;
    int32_t cnt = 0;
    if (i < n) {
      alb_image im = out.get(i);
      int64_t row = (int64_t)im.w * im.c;
      int32_t rb = row > 0 ? (int32_t)((target + row - 1) / row) : 1;
      rb = imax(1, imin(rb, imax(im.h, 1)));
      cnt = im.h > 0 && im.w > 0 ? (im.h + rb - 1) / rb : 0;
      rows_per_item[i] = rb;
      const int bad = check_image_pair(chk.tid, chk.prm.get(i), chk.in.get(i), im, chk.want_c, chk.geometric);
      if (bad) { cnt = 0; dev_fail(chk.status, bad); }
      if (plan_filtered_out(chk, im)) cnt = 0;
    }
    int32_t v = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (lane == 31) wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
      int32_t s = lane < nw ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
      }
      if (lane < nw) wsum[lane] = s;
    }
    __syncthreads();
    int32_t excl = carry + (wid ? wsum[wid - 1] : 0) + v - cnt;
    if (i < n) prefix[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + cnt;
    __syncthreads();
  }
  if (threadIdx.x == 0) prefix[n] = carry;
}

alb_status launch_plan(const ImgList& out, int32_t n, int32_t target_bytes, int32_t* prefix,
                       int32_t* rows_per_item, const PlanCheck& chk, cudaStream_t st) {
  k_plan<<<1, 1024, 0, st>>>(out, n, target_bytes, prefix, rows_per_item, chk);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

// ------------------------------------------------------------------ index maps
// Source pixel of output pixel (y, x) for the pure index-map transforms.
struct MapRow {
  int32_t tid, apply, k, y0, x0, H, W;
  ALB_D int32_t src_y(int32_t y, int32_t x) const {
    if (!apply) return y;
    switch (tid) {
      case ALB_VFLIP: return H - 1 - y;
      case ALB_RANDOM_CROP: return y0 + y;
      case ALB_PAD_TO_SIZE: return reflect101((int64_t)y - y0, H);
      case ALB_TRANSPOSE: return x;
      case ALB_ROT90:
        switch (k & 3) { case 0: return y; case 1: return x; case 2: return H - 1 - y; default: return H - 1 - x; }
      default: return y;  // HFLIP
    }
  }
  ALB_D int32_t src_x(int32_t y, int32_t x) const {
    if (!apply) return x;
    switch (tid) {
      case ALB_HFLIP: return W - 1 - x;
      case ALB_RANDOM_CROP: return x0 + x;
      case ALB_PAD_TO_SIZE: return reflect101((int64_t)x - x0, W);
      case ALB_TRANSPOSE: return y;
      case ALB_ROT90:
        switch (k & 3) { case 0: return x; case 1: return W - 1 - y; case 2: return W - 1 - x; default: return y; }
      default: return x;  // VFLIP
    }
  }
  // true when the source row depends on the output row only
  ALB_D bool row_separable() const {
    return !(apply && (tid == ALB_TRANSPOSE || (tid == ALB_ROT90 && (k & 1))));
  }
};

// Pure index-map copy (flips, crop, pad, transpose, rot90; masks and images).
template <int CT>  // CT = compile-time channels (1 or 3), 0 = runtime
__global__ void __launch_bounds__(256) k_index_map(Plan plan, ImgList in, ImgList out, PrmList prm,
                                                   int32_t* status) {
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
    MapRow m{p.tid, p.apply, p.k, p.y0, p.x0, si.h, si.w};
    const int64_t L = (int64_t)so.w * C;
    const uint8_t* __restrict__ src = (const uint8_t*)si.data;
    uint8_t* __restrict__ dst = (uint8_t*)so.data;
    const bool sep = m.row_separable();
    for (int32_t y = r0; y < r1; y++) {
      uint8_t* orow = dst + (int64_t)y * so.row_stride;
      const int64_t head = ((uintptr_t)orow) & 3;        // bytes before the first aligned slot
      const int64_t nslot = (head + L + 3) >> 2;
      const uint8_t* srow = sep ? src + (int64_t)m.src_y(y, 0) * si.row_stride : nullptr;
      for (int64_t s = threadIdx.x; s < nslot; s += blockDim.x) {
        uint32_t word = 0;
        int nvalid = 0;
        const int64_t ob0 = s * 4 - head;
#pragma unroll
        for (int t = 0; t < 4; t++) {
          const int64_t ob = ob0 + t;
          if (ob < 0 || ob >= L) continue;
          const int32_t x = (int32_t)(ob / C), c = (int32_t)(ob - (int64_t)x * C);
          const int32_t sx = m.src_x(y, x);
          if (!ALB_IN(sx >= 0 && sx < si.w && m.src_y(y, x) >= 0 && m.src_y(y, x) < si.h)) continue;
          const uint8_t* sp = sep ? srow : src + (int64_t)m.src_y(y, x) * si.row_stride;
          word |= (uint32_t)__ldg(sp + (int64_t)sx * C + c) << (8 * t);
          nvalid++;
        }
        uint8_t* op = orow + ob0;
        if (nvalid == 4) {
          *reinterpret_cast<uint32_t*>(op) = word;
        } else {
#pragma unroll
          for (int t = 0; t < 4; t++) {
            const int64_t ob = ob0 + t;
            if (ob >= 0 && ob < L) op[t] = (uint8_t)(word >> (8 * t));
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------ Q5 warps
// Rotate / ShiftScaleRotate (C6): X = q0 x + q1 y + q2 (Q16, int64 exact);
// bilinear: Xq = floor((X + 1024) / 2048) (Q5), taps reflect-101, weights per
// C5; nearest (masks): floor((X + 32768) / 65536).
template <int CT, bool NEAREST>
__global__ void __launch_bounds__(256) k_warp_affine_u8(Plan plan, ImgList in, ImgList out, PrmList prm,
                                                        int32_t* status) {
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
    const int64_t q0 = p.apply ? p.q[0] : 65536, q1 = p.apply ? p.q[1] : 0, q2 = p.apply ? p.q[2] : 0;
    const int64_t q3 = p.apply ? p.q[3] : 0, q4 = p.apply ? p.q[4] : 65536, q5 = p.apply ? p.q[5] : 0;
    const int32_t H = si.h, W = si.w;
    const uint8_t* __restrict__ src = (const uint8_t*)si.data;
    uint8_t* __restrict__ dst = (uint8_t*)so.data;
    const int64_t npx = (int64_t)(r1 - r0) * so.w;
    for (int64_t i = threadIdx.x; i < npx; i += blockDim.x) {
      const int32_t y = r0 + (int32_t)(i / so.w), x = (int32_t)(i % so.w);
      const int64_t X = q0 * x + q1 * y + q2;
      const int64_t Y = q3 * x + q4 * y + q5;
      uint8_t* op = dst + (int64_t)y * so.row_stride + (int64_t)x * C;
      if (NEAREST) {
        // arithmetic right shifts of int64 are floor divisions by powers of two
        const int32_t sx = reflect101((X + 32768) >> 16, W);
        const int32_t sy = reflect101((Y + 32768) >> 16, H);
        const uint8_t* sp = src + (int64_t)sy * si.row_stride + (int64_t)sx * C;
        for (int c = 0; c < C; c++) op[c] = __ldg(sp + c);
      } else {
        const int64_t xq = (X + 1024) >> 11, yq = (Y + 1024) >> 11;  // arithmetic shift = floor
        const int64_t ix = xq >> 5, iy = yq >> 5;
        const int32_t fx = (int32_t)(xq & 31), fy = (int32_t)(yq & 31);
        const int32_t xa = reflect101(ix, W), xb = reflect101(ix + 1, W);
        const int32_t ya = reflect101(iy, H), yb = reflect101(iy + 1, H);
        const uint8_t* ra = src + (int64_t)ya * si.row_stride;
        const uint8_t* rbp = src + (int64_t)yb * si.row_stride;
        const int32_t w00 = (32 - fx) * (32 - fy), w01 = fx * (32 - fy), w10 = (32 - fx) * fy, w11 = fx * fy;
        for (int c = 0; c < C; c++) {
          const int32_t acc = w00 * __ldg(ra + (int64_t)xa * C + c) + w01 * __ldg(ra + (int64_t)xb * C + c) +
                              w10 * __ldg(rbp + (int64_t)xa * C + c) + w11 * __ldg(rbp + (int64_t)xb * C + c);
          op[c] = (uint8_t)((acc + 512) >> 10);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ resize
// Half-pixel Q5 coordinate (C-R): floor((32((2d+1) n_in - n_out) + n_out) / (2 n_out)),
// clamped to [0, 32 (n_in - 1)]; nearest: min(floor((2d+1) n_in / (2 n_out)), n_in - 1).
ALB_D int32_t resize_q5(int32_t d, int32_t n_in, int32_t n_out) {
  int64_t num = 32 * ((int64_t)(2 * d + 1) * n_in - n_out) + n_out;
  int64_t xq = floor_div(num, 2 * (int64_t)n_out);
  if (xq < 0) xq = 0;
  if ((xq >> 5) >= n_in - 1) xq = 32 * (int64_t)(n_in - 1);
  return (int32_t)xq;
}
ALB_D int32_t resize_nn(int32_t d, int32_t n_in, int32_t n_out) {
  int64_t i = ((int64_t)(2 * d + 1) * n_in) / (2 * (int64_t)n_out);
  return (int32_t)(i < n_in - 1 ? i : n_in - 1);
}

constexpr int kResizeColCap = 4096;

template <int CT, bool NEAREST>
__global__ void __launch_bounds__(256) k_resize_u8(Plan plan, ImgList in, ImgList out, PrmList prm,
                                                   int32_t* status) {
  __shared__ int32_t colq[kResizeColCap];
  int32_t it0, it1;
  item_range(plan, it0, it1);
  if (it0 >= it1) return;
  int32_t b = item_image(plan, it0);
  int32_t cached_b = -1;
  for (int32_t item = it0; item < it1; item++) {
    while (item >= plan.prefix[b + 1]) b++;
    const alb_image si = in.get(b), so = out.get(b);
    const alb_params& p = prm.get(b);
    const int32_t C = CT ? CT : so.c;
    const int32_t rb = plan.rows_per_item[b];
    const int32_t r0 = (item - plan.prefix[b]) * rb, r1 = imin(r0 + rb, so.h);
    const int32_t cw = p.cw, ch = p.ch, ow = so.w, oh = so.h;
    const bool table = ow <= kResizeColCap;
    if (table && cached_b != b) {
      __syncthreads();
      for (int x = threadIdx.x; x < ow; x += blockDim.x) colq[x] = NEAREST ? resize_nn(x, cw, ow) : resize_q5(x, cw, ow);
      __syncthreads();
      cached_b = b;
    }
    const uint8_t* __restrict__ win = (const uint8_t*)si.data + (int64_t)p.y0 * si.row_stride + (int64_t)p.x0 * C;
    uint8_t* __restrict__ dst = (uint8_t*)so.data;
    const int64_t npx = (int64_t)(r1 - r0) * ow;
    for (int64_t i = threadIdx.x; i < npx; i += blockDim.x) {
      const int32_t y = r0 + (int32_t)(i / ow), x = (int32_t)(i % ow);
      uint8_t* op = dst + (int64_t)y * so.row_stride + (int64_t)x * C;
      if (NEAREST) {
        const int32_t sx = table ? colq[x] : resize_nn(x, cw, ow);
        const int32_t sy = resize_nn(y, ch, oh);
        const uint8_t* sp = win + (int64_t)sy * si.row_stride + (int64_t)sx * C;
        for (int c = 0; c < C; c++) op[c] = __ldg(sp + c);
      } else {
        const int32_t xq = table ? colq[x] : resize_q5(x, cw, ow);
        const int32_t yq = resize_q5(y, ch, oh);
        const int32_t ix = xq >> 5, fx = xq & 31, iy = yq >> 5, fy = yq & 31;
        const int32_t ixb = imin(ix + 1, cw - 1), iyb = imin(iy + 1, ch - 1);
        const uint8_t* ra = win + (int64_t)iy * si.row_stride;
        const uint8_t* rbp = win + (int64_t)iyb * si.row_stride;
        const int32_t w00 = (32 - fx) * (32 - fy), w01 = fx * (32 - fy), w10 = (32 - fx) * fy, w11 = fx * fy;
        for (int c = 0; c < C; c++) {
          const int32_t acc = w00 * __ldg(ra + (int64_t)ix * C + c) + w01 * __ldg(ra + (int64_t)ixb * C + c) +
                              w10 * __ldg(rbp + (int64_t)ix * C + c) + w11 * __ldg(rbp + (int64_t)ixb * C + c);
          op[c] = (uint8_t)((acc + 512) >> 10);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ boxes
// One warp per image: each lane transforms boxes in float64 (same formulas as
// the definitions of Sec. II-A's box targets: exact affine maps for
// flip/crop/pad/resize, four corners through the forward matrix for warps),
// clips to the output, drops empty boxes and compacts with a ballot prefix.
__global__ void k_boxes(int32_t n, PrmList prm, ImgList in, const float* __restrict__ boxes,
                        const int32_t* __restrict__ nbox, int32_t cap, int32_t single_n, float* __restrict__ out,
                        int32_t* __restrict__ nout, int32_t* status) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= n) return;
  const alb_params& p = prm.get(b);
  const alb_image im = in.get(b);
  const int32_t h = im.h, w = im.w;
  int32_t oh = h, ow = w;
  switch (p.tid) {
    case ALB_RANDOM_CROP: case ALB_PAD_TO_SIZE: case ALB_RESIZE: case ALB_RANDOM_SIZED_CROP:
    case ALB_RANDOM_RESIZED_CROP: oh = p.out_h; ow = p.out_w; break;
    case ALB_TRANSPOSE: oh = w; ow = h; break;
    case ALB_ROT90: if (p.apply && (p.k & 1)) { oh = w; ow = h; } break;
    default: break;
  }
  int32_t cnt = nbox ? nbox[b] : single_n;
  if (cnt > cap) { dev_fail(status, ALB_ECAPACITY); cnt = cap; }
  const float* bin = boxes + (int64_t)b * cap * 4;
  float* bout = out + (int64_t)b * cap * 4;
  int32_t kept_total = 0;
  for (int base = 0; base < cnt; base += 32) {
    const int i = base + lane;
    double a1 = 0, b1 = 0, a2 = 0, b2 = 0;
    bool keep = false;
    if (i < cnt) {
      const double x1 = bin[4 * i], y1 = bin[4 * i + 1], x2 = bin[4 * i + 2], y2 = bin[4 * i + 3];
      a1 = x1; b1 = y1; a2 = x2; b2 = y2;
      if (p.apply) switch (p.tid) {
        case ALB_HFLIP: a1 = (double)w - x2; a2 = (double)w - x1; break;
        case ALB_VFLIP: b1 = (double)h - y2; b2 = (double)h - y1; break;
        case ALB_TRANSPOSE: a1 = y1; b1 = x1; a2 = y2; b2 = x2; break;
        case ALB_ROT90:
          switch (p.k & 3) {
            case 0: break;
            case 1: a1 = y1; a2 = y2; b1 = (double)w - x2; b2 = (double)w - x1; break;
            case 2: a1 = (double)w - x2; a2 = (double)w - x1; b1 = (double)h - y2; b2 = (double)h - y1; break;
            default: a1 = (double)h - y2; a2 = (double)h - y1; b1 = x1; b2 = x2; break;
          }
          break;
        case ALB_RANDOM_CROP:
          a1 = x1 - p.x0; a2 = x2 - p.x0; b1 = y1 - p.y0; b2 = y2 - p.y0; break;
        case ALB_PAD_TO_SIZE:
          a1 = x1 + p.x0; a2 = x2 + p.x0; b1 = y1 + p.y0; b2 = y2 + p.y0; break;
        case ALB_RESIZE: case ALB_RANDOM_SIZED_CROP: case ALB_RANDOM_RESIZED_CROP: {
          double cx1 = x1 - p.x0, cx2 = x2 - p.x0, cy1 = y1 - p.y0, cy2 = y2 - p.y0;
          if (cx1 < 0) cx1 = 0;
          if (cy1 < 0) cy1 = 0;
          if (cx2 > p.cw) cx2 = p.cw;
          if (cy2 > p.ch) cy2 = p.ch;
          a1 = cx1 * ow / p.cw; a2 = cx2 * ow / p.cw;
          b1 = cy1 * oh / p.ch; b2 = cy2 * oh / p.ch;
          break;
        }
        case ALB_ROTATE: case ALB_SHIFT_SCALE_ROTATE: {
          const double xs[4] = {x1, x2, x1, x2}, ys[4] = {y1, y1, y2, y2};
#pragma unroll
          for (int j = 0; j < 4; j++) {
            const double u = xs[j] - 0.5, v = ys[j] - 0.5;
            const double tx = (p.m[0] * u + p.m[1] * v + p.m[2]) + 0.5;
            const double ty = (p.m[3] * u + p.m[4] * v + p.m[5]) + 0.5;
            if (j == 0 || tx < a1) a1 = tx;
            if (j == 0 || tx > a2) a2 = tx;
            if (j == 0 || ty < b1) b1 = ty;
            if (j == 0 || ty > b2) b2 = ty;
          }
          break;
        }
        case ALB_GRID_DISTORTION:
          a1 = grid_edge_inverse(p.q, p.k, 0, x1, w); a2 = grid_edge_inverse(p.q, p.k, 0, x2, w);
          b1 = grid_edge_inverse(p.q, p.k, 1, y1, h); b2 = grid_edge_inverse(p.q, p.k, 1, y2, h);
          break;
        default: break;
      }
      if (a1 < 0) a1 = 0;
      if (b1 < 0) b1 = 0;
      if (a2 > ow) a2 = ow;
      if (b2 > oh) b2 = oh;
      keep = (a2 - a1 > 0.0) && (b2 - b1 > 0.0);
    }
    const uint32_t mask = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int slot = kept_total + __popc(mask & ((1u << lane) - 1u));
      bout[4 * slot] = (float)a1; bout[4 * slot + 1] = (float)b1;
      bout[4 * slot + 2] = (float)a2; bout[4 * slot + 3] = (float)b2;
    }
    kept_total += __popc(mask);
  }
  if (lane == 0) nout[b] = kept_total;
}

// ------------------------------------------------------------------ launchers
static int grid_for(const void* fn, int threads, size_t smem) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (per_sm < 1) per_sm = 1;
  return per_sm * sm_count();
}

// ------------------------------------------------------------------ distortions
// Grid distortion and elastic transform (any channel count): one thread per
// output pixel over the plan's row items.  Images: Q5 bilinear (grid: taps
// inside the image, the +1 tap clamped; elastic: reflect-101 taps); masks:
// nearest floor((Xq + 16) / 32) (elastic: reflected).
template <int CT>
ALB_D void q5_taps_store(const uint8_t* __restrict__ src, int64_t ss, int32_t C, int32_t xa, int32_t xb, int32_t ya,
                         int32_t yb, int32_t fx, int32_t fy, uint8_t* op) {
  const uint8_t* ra = src + (int64_t)ya * ss;
  const uint8_t* rbp = src + (int64_t)yb * ss;
  const int32_t w00 = (32 - fx) * (32 - fy), w01 = fx * (32 - fy), w10 = (32 - fx) * fy, w11 = fx * fy;
  for (int c = 0; c < C; c++) {
    const int32_t acc = w00 * __ldg(ra + (int64_t)xa * C + c) + w01 * __ldg(ra + (int64_t)xb * C + c) +
                        w10 * __ldg(rbp + (int64_t)xa * C + c) + w11 * __ldg(rbp + (int64_t)xb * C + c);
    op[c] = (uint8_t)((acc + 512) >> 10);
  }
}

template <int CT, bool NEAREST>
__global__ void __launch_bounds__(256) k_grid_u8(Plan plan, ImgList in, ImgList out, PrmList prm, int32_t* status) {
  __shared__ int32_t colq[kResizeColCap];
  int32_t it0, it1;
  item_range(plan, it0, it1);
  if (it0 >= it1) return;
  int32_t b = item_image(plan, it0);
  int32_t cached_b = -1;
  for (int32_t item = it0; item < it1; item++) {
    while (item >= plan.prefix[b + 1]) b++;
    const alb_image si = in.get(b), so = out.get(b);
    const alb_params& p = prm.get(b);
    const int32_t C = CT ? CT : so.c;
    const int32_t rb = plan.rows_per_item[b];
    const int32_t r0 = (item - plan.prefix[b]) * rb, r1 = imin(r0 + rb, so.h);
    const int32_t W = si.w, H = si.h;
    const bool act = p.apply != 0;
    const bool table = W <= kResizeColCap;
    if (table && cached_b != b) {
      __syncthreads();
      for (int x = threadIdx.x; x < W; x += blockDim.x) colq[x] = act ? grid_q5(p.q, p.k, 0, x, W) : 32 * x;
      __syncthreads();
      cached_b = b;
    }
    const uint8_t* __restrict__ src = (const uint8_t*)si.data;
    uint8_t* __restrict__ dst = (uint8_t*)so.data;
    const int64_t npx = (int64_t)(r1 - r0) * W;
    for (int64_t i = threadIdx.x; i < npx; i += blockDim.x) {
      const int32_t y = r0 + (int32_t)(i / W), x = (int32_t)(i % W);
      uint8_t* op = dst + (int64_t)y * so.row_stride + (int64_t)x * C;
      const int32_t xq = table ? colq[x] : (act ? grid_q5(p.q, p.k, 0, x, W) : 32 * x);
      const int32_t yq = act ? grid_q5(p.q, p.k, 1, y, H) : 32 * y;
      if (NEAREST) {
        if (!ALB_IN(((yq + 16) >> 5) >= 0 && ((yq + 16) >> 5) < H && ((xq + 16) >> 5) >= 0 && ((xq + 16) >> 5) < W))
          continue;
        const uint8_t* sp = src + (int64_t)((yq + 16) >> 5) * si.row_stride + (int64_t)((xq + 16) >> 5) * C;
        for (int c = 0; c < C; c++) op[c] = __ldg(sp + c);
      } else {
        const int32_t ix = xq >> 5, iy = yq >> 5;
        if (!ALB_IN(ix >= 0 && ix < W && iy >= 0 && iy < H)) continue;
        q5_taps_store<CT>(src, si.row_stride, C, ix, imin(ix + 1, W - 1), iy, imin(iy + 1, H - 1), xq & 31, yq & 31,
                          op);
      }
    }
  }
}

constexpr int kLatticeCap = 4096;   // lattice points cached per CTA and item

template <int CT, bool NEAREST>
__global__ void __launch_bounds__(256) k_elastic_u8(Plan plan, ImgList in, ImgList out, PrmList prm, int32_t* status) {
  __shared__ int2 lat[kLatticeCap];
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
    if (r1 <= r0) continue;
    const int32_t W = si.w, H = si.h;
    const bool act = p.apply != 0;
    const int sh = act ? p.cw : 2;
    const int32_t S = 1 << sh;
    const int32_t nx = ((W + S - 1) >> sh) + 1;
    const int32_t ci0 = r0 >> sh, ci1 = ((r1 - 1) >> sh) + 1;     // lattice rows the item blends
    const int64_t npts = (int64_t)(ci1 - ci0 + 1) * nx;
    const bool cached = act && npts <= kLatticeCap;
    __syncthreads();
    if (cached)
      for (int32_t t = threadIdx.x; t < npts; t += blockDim.x) {
        int32_t dx, dy;
        elastic_point(p.q, p.k, (int64_t)ci0 * nx + t, dx, dy);
        lat[t] = make_int2(dx, dy);
      }
    __syncthreads();
    auto point = [&](int32_t ci, int32_t cj) -> int2 {
      if (cached) return lat[(ci - ci0) * nx + cj];
      int32_t dx, dy;
      elastic_point(p.q, p.k, (int64_t)ci * nx + cj, dx, dy);
      return make_int2(dx, dy);
    };
    const uint8_t* __restrict__ src = (const uint8_t*)si.data;
    uint8_t* __restrict__ dst = (uint8_t*)so.data;
    const int64_t npx = (int64_t)(r1 - r0) * W;
    for (int64_t i = threadIdx.x; i < npx; i += blockDim.x) {
      const int32_t y = r0 + (int32_t)(i / W), x = (int32_t)(i % W);
      uint8_t* op = dst + (int64_t)y * so.row_stride + (int64_t)x * C;
      int64_t xq = 32 * (int64_t)x, yq = 32 * (int64_t)y;
      if (act) {
        const int32_t ci = y >> sh, cj = x >> sh, fy = y & (S - 1), fx = x & (S - 1);
        const int2 a = point(ci, cj), bq = point(ci, cj + 1), c = point(ci + 1, cj), d = point(ci + 1, cj + 1);
        const int64_t w00 = (int64_t)(S - fx) * (S - fy), w01 = (int64_t)fx * (S - fy), w10 = (int64_t)(S - fx) * fy,
                      w11 = (int64_t)fx * fy;
        const int64_t SS = (int64_t)S * S;
        // floor((sum + S^2 / 2) / S^2): S^2 is a power of two, an arithmetic shift floors
        xq += (w00 * a.x + w01 * bq.x + w10 * c.x + w11 * d.x + SS / 2) >> (2 * sh);
        yq += (w00 * a.y + w01 * bq.y + w10 * c.y + w11 * d.y + SS / 2) >> (2 * sh);
      }
      if (NEAREST) {
        const int32_t sx = reflect101((xq + 16) >> 5, W), sy = reflect101((yq + 16) >> 5, H);   // floor
        const uint8_t* sp = src + (int64_t)sy * si.row_stride + (int64_t)sx * C;
        for (int c = 0; c < C; c++) op[c] = __ldg(sp + c);
      } else {
        const int64_t ix = xq >> 5, iy = yq >> 5;   // arithmetic shifts floor
        q5_taps_store<CT>(src, si.row_stride, C, reflect101(ix, W), reflect101(ix + 1, W), reflect101(iy, H),
                          reflect101(iy + 1, H), (int32_t)(xq - 32 * ix), (int32_t)(yq - 32 * iy), op);
      }
    }
  }
}

template <class K>
static alb_status launch_items(K kernel, const Plan& plan, const ImgList& in, const ImgList& out,
                               const PrmList& prm, int32_t* status, cudaStream_t st) {
  const int grid = grid_for((const void*)kernel, 256, 0);
  kernel<<<grid, 256, 0, st>>>(plan, in, out, prm, status);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

alb_status launch_geometric(int32_t tid, const Plan& plan, const ImgList& in, const ImgList& out,
                            const PrmList& prm, int32_t channels, bool mask, int32_t* status, cudaStream_t st) {
  const PlanCheck chk{tid, mask ? 0 : channels, true, in, prm, status, mask ? (channels == 1 ? 1 : -1) : 0};
  const bool c3 = channels == 3, c1 = channels == 1;
  if (launch_stream_geometric(tid, plan, in, out, prm, channels, st) == ALB_OK) return ALB_OK;
  if (launch_tile_geometric(tid, plan, in, out, prm, channels, mask, chk, st) == ALB_OK) return ALB_OK;
  switch (tid) {
    case ALB_HFLIP: case ALB_VFLIP: case ALB_RANDOM_CROP: case ALB_PAD_TO_SIZE: case ALB_TRANSPOSE:
    case ALB_ROT90:
      if (c3) return launch_items(k_index_map<3>, plan, in, out, prm, status, st);
      if (c1) return launch_items(k_index_map<1>, plan, in, out, prm, status, st);
      return launch_items(k_index_map<0>, plan, in, out, prm, status, st);
    case ALB_ROTATE: case ALB_SHIFT_SCALE_ROTATE:
      if (mask) {
        if (c1) return launch_items(k_warp_affine_u8<1, true>, plan, in, out, prm, status, st);
        return launch_items(k_warp_affine_u8<0, true>, plan, in, out, prm, status, st);
      }
      if (c3) return launch_items(k_warp_affine_u8<3, false>, plan, in, out, prm, status, st);
      return launch_items(k_warp_affine_u8<0, false>, plan, in, out, prm, status, st);
    case ALB_GRID_DISTORTION:
      if (mask) {
        if (c1) return launch_items(k_grid_u8<1, true>, plan, in, out, prm, status, st);
        return launch_items(k_grid_u8<0, true>, plan, in, out, prm, status, st);
      }
      if (c3) return launch_items(k_grid_u8<3, false>, plan, in, out, prm, status, st);
      return launch_items(k_grid_u8<0, false>, plan, in, out, prm, status, st);
    case ALB_ELASTIC:
      if (mask) {
        if (c1) return launch_items(k_elastic_u8<1, true>, plan, in, out, prm, status, st);
        return launch_items(k_elastic_u8<0, true>, plan, in, out, prm, status, st);
      }
      if (c3) return launch_items(k_elastic_u8<3, false>, plan, in, out, prm, status, st);
      return launch_items(k_elastic_u8<0, false>, plan, in, out, prm, status, st);
    case ALB_RESIZE: case ALB_RANDOM_SIZED_CROP: case ALB_RANDOM_RESIZED_CROP:
      if (mask) {
        if (c1) return launch_items(k_resize_u8<1, true>, plan, in, out, prm, status, st);
        return launch_items(k_resize_u8<0, true>, plan, in, out, prm, status, st);
      }
      if (c3) return launch_items(k_resize_u8<3, false>, plan, in, out, prm, status, st);
      return launch_items(k_resize_u8<0, false>, plan, in, out, prm, status, st);
    default:
      set_error("launch_geometric: transform %d is not geometric", tid);
      return ALB_EINVAL;
  }
}

alb_status launch_boxes(int32_t n, const PrmList& prm, const ImgList& in, const float* boxes, const int32_t* nbox,
                        int32_t cap, int32_t single_n, float* out, int32_t* nout, int32_t* status, cudaStream_t st) {
  const int warps = 4;
  k_boxes<<<(n + warps - 1) / warps, 32 * warps, 0, st>>>(n, prm, in, boxes, nbox, cap, single_n, out, nout, status);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

}  // namespace alb

namespace alb {
ALB_OOB_ACCESSOR(oob_geom)
}  // namespace alb
