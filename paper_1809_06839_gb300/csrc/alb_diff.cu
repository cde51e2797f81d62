// alb_diff.cu -- differentiable float32 augmentation: the affine warp of the u8
// path (rotation about the centre, scale, shift; Table I "ShiftScaleRotate")
// with bilinear sampling and a zero border, and the photometric map
// y = clamp(alpha x + beta, 0, 1)^gamma (Sec. II / Fig. 1 brightness, contrast,
// gamma).  Backward kernels recompute every sampling coordinate from the
// per-image parameters (nothing is stored by the forward).
//
// x, y, g: float32 NCHW [B][C][H][W].  Warp parameters [B][4] = (angle deg,
// scale, tx, ty) with the shift in fractions of W and H; photometric [B][3] =
// (alpha, beta, gamma).
//
// Input adjoint of the warp: a gather over the output samples whose taps touch
// each source pixel (no atomics); parameter gradients: per-CTA block
// reductions written to a partials buffer and reduced by one CTA per image in
// a fixed order.  Both are deterministic.
#include "alb_common.cuh"

namespace alb {

struct WarpF {
  float a00, a01, a10, a11, b0, b1;  // inverse map, float32 (rounded from float64)
  float cs, sn, s, cx, cy, txp, typ, W, H;
};

ALB_D WarpF warp_setup(const float* prm, int b, int H, int W) {
  const double kDeg = 3.14159265358979323846 / 180.0;
  const double angle = prm[4 * b], scale = prm[4 * b + 1], tx = prm[4 * b + 2], ty = prm[4 * b + 3];
  const double rad = angle * kDeg;
  const double cs = cos(rad), sn = sin(rad);
  const double cx = (double)(W - 1) * 0.5, cy = (double)(H - 1) * 0.5;
  const double txp = tx * W, typ = ty * H;
  const double a00 = cs / scale, a01 = -sn / scale, a10 = sn / scale, a11 = cs / scale;
  const double ox = cx + txp, oy = cy + typ;
  WarpF g;
  g.a00 = (float)a00; g.a01 = (float)a01; g.a10 = (float)a10; g.a11 = (float)a11;
  g.b0 = (float)(cx - (a00 * ox + a01 * oy));
  g.b1 = (float)(cy - (a10 * ox + a11 * oy));
  g.cs = (float)cs; g.sn = (float)sn; g.s = (float)scale; g.cx = (float)cx; g.cy = (float)cy;
  g.txp = (float)txp; g.typ = (float)typ; g.W = (float)W; g.H = (float)H;
  return g;
}

ALB_D float tapf(const float* __restrict__ img, int H, int W, int x, int y) {
  return (x >= 0 && y >= 0 && x < W && y < H) ? __ldg(img + (int64_t)y * W + x) : 0.0f;
}

// ------------------------------------------------------------------ warp
// Both warp kernels work on 32x16 pixel tiles with 256 threads (two pixels a
// thread, rows r and r+8) and stage the tile's counterpart in shared memory:
// the forward stages the source box its outputs sample, the backward the
// output box whose samples touch its source tile.  Work units are (tile,
// group of up to three channels); a CTA owns every gridDim.x-th tile of one
// image and copies unit u+1's box in with cp.async (zero-filled outside the
// image) while it computes unit u from the other buffer.  With W a multiple
// of four (AL) boxes are widened to 16-byte columns and copied 16 bytes at a
// time; otherwise 4 bytes at a time.  A box that does not fit a buffer
// (extreme zoom) is read from global memory instead; results are identical
// either way.
constexpr int kWT_W = 32, kWT_H = 16, kWT_THREADS = 256;
constexpr int kWT_CG = 3;                 // channels staged per unit
constexpr int kWT_BUF = 6144;             // floats per staging buffer (two buffers: 48 KB)

struct WarpBox {
  int x0, y0, x1, y1;  // inclusive box corners (x1 < x0: empty)
  int pitch;           // row pitch in floats of the staged copy
  int staged;          // the box of `cn` channels fits one buffer
};

// pitch and fit of a box; AL widens it to 16-byte columns (x0 down, x1 up to
// multiples of four) with a pitch of an odd number of 16-byte columns
template <bool AL>
ALB_D void warp_box_finish(WarpBox& bx, int cn) {
  if (AL && bx.x1 >= bx.x0) {
    bx.x0 &= ~3;
    bx.x1 = bx.x0 + (((bx.x1 - bx.x0 + 1) + 3) & ~3) - 1;
  }
  const int w = bx.x1 - bx.x0 + 1, h = bx.y1 - bx.y0 + 1;
  bx.pitch = AL ? (((w >> 2) | 1) << 2) : (w | 1);  // rotated access patterns spread over banks
  bx.staged = (w > 0 && h > 0 && (int64_t)cn * h * bx.pitch <= kWT_BUF) ? 1 : 0;
}

ALB_D void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
ALB_D void cp_async16z(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
ALB_D void cp_async_commit_f() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
ALB_D void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// issue the copies of channels [0, cn) of the box of a [C][H][W] plane stack
// (src points at the group's first plane); zero outside the image, which is
// the warp's zero border.  Copy items (row, column) are spread over all
// threads; the row is recovered with a float reciprocal, exact for the item
// counts of a buffer.
template <bool AL>
ALB_D void warp_stage_async(float* __restrict__ sm, const float* __restrict__ src, int cn, int H, int W,
                            const WarpBox& bx) {
  const int h = bx.y1 - bx.y0 + 1;
  const int ncol = AL ? (bx.x1 - bx.x0 + 1) >> 2 : bx.x1 - bx.x0 + 1;  // copy items per row
  const int items = h * ncol;
  const float rinv = 1.0f / (float)ncol;
  for (int k = 0; k < cn; k++) {
    const float* img = src + (int64_t)k * H * W;
    float* dst = sm + k * h * bx.pitch;
    for (int t = threadIdx.x; t < items; t += kWT_THREADS) {
      const int r = (int)__fmul_rn(__fadd_rn((float)t, 0.5f), rinv);
      const int c = t - r * ncol;
      const int y = bx.y0 + r;
      const int xx = bx.x0 + (AL ? 4 * c : c);
      const bool in = y >= 0 && y < H && xx >= 0 && xx < W;  // AL: a 16-byte column is wholly in or out
      const float* gp = in ? img + (int64_t)y * W + xx : img;
      if (AL)
        cp_async16z(dst + r * bx.pitch + 4 * c, gp, in);
      else
        cp_async4(dst + r * bx.pitch + c, gp, in);
    }
  }
}

// source box of an output tile: the tile's corners mapped by the inverse map,
// one pixel of margin for the taps and for rounding (computed identically by
// every thread)
template <bool AL>
ALB_D WarpBox warp_fwd_box(const WarpF& g, int ox0, int oy0, int H, int W, int cn) {
  const float xa = (float)ox0, xb = (float)min(ox0 + kWT_W, W) - 1.0f;
  const float ya = (float)oy0, yb = (float)min(oy0 + kWT_H, H) - 1.0f;
  float sxl = 3e38f, sxh = -3e38f, syl = 3e38f, syh = -3e38f;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const float ox = (k & 1) ? xb : xa, oy = (k & 2) ? yb : ya;
    const float sx = __fmaf_rn(g.a00, ox, __fmaf_rn(g.a01, oy, g.b0));
    const float sy = __fmaf_rn(g.a10, ox, __fmaf_rn(g.a11, oy, g.b1));
    sxl = fminf(sxl, sx); sxh = fmaxf(sxh, sx); syl = fminf(syl, sy); syh = fmaxf(syh, sy);
  }
  WarpBox bx{0, 0, -1, -1, 1, 0};
  if (fabsf(sxl) < 1e7f && fabsf(sxh) < 1e7f && fabsf(syl) < 1e7f && fabsf(syh) < 1e7f) {
    bx.x0 = (int)floorf(sxl) - 1; bx.x1 = (int)floorf(sxh) + 2;
    bx.y0 = (int)floorf(syl) - 1; bx.y1 = (int)floorf(syh) + 2;
  }
  warp_box_finish<AL>(bx, cn);
  return bx;
}

// (tile origin, first channel) of unit u of this CTA.  No integer division on
// the common path: one channel group needs none, and the tile row comes from a
// float reciprocal of tiles_x, exact for tile indices below 2^21 and tiles_x up
// to 2048 (checked on every such pair); larger grids divide.
ALB_D void warp_unit(int u, int groups, int tiles_x, float rtx, int& X0, int& Y0, int& c0) {
  int tu = u;
  c0 = 0;
  if (groups != 1) {
    tu = u / groups;
    c0 = (u - tu * groups) * kWT_CG;
  }
  const int t = blockIdx.x + tu * gridDim.x;
  const int ty = (t < (1 << 21) && tiles_x <= 2048) ? (int)__fmul_rn(__fadd_rn((float)t, 0.5f), rtx) : t / tiles_x;
  X0 = (t - ty * tiles_x) * kWT_W;
  Y0 = ty * kWT_H;
}

ALB_D int warp_units(int tiles, int groups) {
  const int mine = tiles > (int)blockIdx.x ? (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  return mine * groups;
}

// forward: grid (CTAs per image, B); each CTA sets up its image's map once
// and runs the unit pipeline.  F3: every channel group is full (C a multiple
// of three), so no channel test is left in the loops.
template <bool AL, bool F3>
__global__ void __launch_bounds__(kWT_THREADS) k_warp_f32_fwd(int B, int C, int H, int W, int tiles_x, int tiles,
                                                              const float* __restrict__ x,
                                                              const float* __restrict__ prm, float* __restrict__ y) {
  extern __shared__ __align__(16) float sm[];
  __shared__ WarpF sg;
  const int b = blockIdx.y;
  if (threadIdx.x == 0) sg = warp_setup(prm, b, H, W);
  __syncthreads();
  const float a00 = sg.a00, a01 = sg.a01, a10 = sg.a10, a11 = sg.a11, b0 = sg.b0, b1 = sg.b1;
  const WarpF g = sg;
  const int plane = H * W;
  const float* xb = x + (int64_t)b * C * plane;
  float* yb = y + (int64_t)b * C * plane;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int groups = (C + kWT_CG - 1) / kWT_CG;
  const int units = warp_units(tiles, groups);
  const float rtx = 1.0f / (float)tiles_x;
  WarpBox nb{0, 0, -1, -1, 1, 0};
  if (units > 0) {
    int X0, Y0, c0;
    warp_unit(0, groups, tiles_x, rtx, X0, Y0, c0);
    const int cn0 = F3 ? kWT_CG : min(C - c0, kWT_CG);
    nb = warp_fwd_box<AL>(g, X0, Y0, H, W, cn0);
    if (nb.staged) warp_stage_async<AL>(sm, xb + (int64_t)c0 * plane, cn0, H, W, nb);
  }
  cp_async_commit_f();
  for (int u = 0; u < units; u++) {
    const WarpBox bx = nb;
    int ox0, oy0, c0;
    warp_unit(u, groups, tiles_x, rtx, ox0, oy0, c0);
    const int cn = F3 ? kWT_CG : min(C - c0, kWT_CG);
    if (u + 1 < units) {
      int X1, Y1, c1;
      warp_unit(u + 1, groups, tiles_x, rtx, X1, Y1, c1);
      const int cn1 = F3 ? kWT_CG : min(C - c1, kWT_CG);
      nb = warp_fwd_box<AL>(g, X1, Y1, H, W, cn1);
      if (nb.staged) warp_stage_async<AL>(sm + ((u + 1) & 1) * kWT_BUF, xb + (int64_t)c1 * plane, cn1, H, W, nb);
    }
    cp_async_commit_f();
    cp_async_wait_prev();
    __syncthreads();
    const float* buf = sm + (u & 1) * kWT_BUF;
    const float* src = xb + (int64_t)c0 * plane;
    float* dstp = yb + (int64_t)c0 * plane;
    const int bw = bx.x1 - bx.x0 + 1, bh = bx.y1 - bx.y0 + 1, bp = bx.pitch, bpl = bh * bx.pitch;
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const int ox = ox0 + tx, oy = oy0 + ty + 8 * j;
      if (ox >= W || oy >= H) continue;
      const float sx = __fmaf_rn(a00, (float)ox, __fmaf_rn(a01, (float)oy, b0));
      const float sy = __fmaf_rn(a10, (float)ox, __fmaf_rn(a11, (float)oy, b1));
      const float fx0 = floorf(sx), fy0 = floorf(sy);
      const float fx = sx - fx0, fy = sy - fy0;
      const int ix = (int)fx0, iy = (int)fy0;
      const float w00 = (1.0f - fx) * (1.0f - fy), w10 = fx * (1.0f - fy), w01 = (1.0f - fx) * fy, w11 = fx * fy;
      const int lx = ix - bx.x0, ly = iy - bx.y0;
      const int o = oy * W + ox;
      if (bx.staged && (unsigned)lx < (unsigned)(bw - 1) && (unsigned)ly < (unsigned)(bh - 1)) {
        const int s0 = ly * bp + lx;
#pragma unroll
        for (int k = 0; k < kWT_CG; k++) {
          if ((F3 || k < cn) && ALB_IN(k * bpl + s0 + bp + 1 < kWT_BUF && s0 >= 0)) {
            const float* s = buf + k * bpl + s0;
            dstp[k * plane + o] = w00 * s[0] + w10 * s[1] + w01 * s[bp] + w11 * s[bp + 1];
          }
        }
      } else {
        for (int k = 0; k < cn; k++) {
          const float* img = src + (int64_t)k * plane;
          dstp[k * plane + o] = w00 * tapf(img, H, W, ix, iy) + w10 * tapf(img, H, W, ix + 1, iy) +
                                w01 * tapf(img, H, W, ix, iy + 1) + w11 * tapf(img, H, W, ix + 1, iy + 1);
        }
      }
    }
    __syncthreads();  // buffer (u & 1) is refilled by unit u + 2
  }
}

ALB_D float block_sum(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  float t = 0.0f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
  return t;  // valid in thread 0
}

struct WarpInv {
  float m00, m01, m10, m11;  // forward map (inverse of the sampling map's linear part)
};

// output box of the source region [X0-1, X0+32] x [Y0-1, Y0+16] of a source
// tile: its corners mapped by the forward map, two pixels of margin, clipped
// to the image (computed identically by every thread)
template <bool AL>
ALB_D WarpBox warp_bwd_box(const WarpF& g, const WarpInv& M, bool finite, int X0, int Y0, int H, int W, int cn) {
  WarpBox bx{0, 0, -1, -1, 1, 0};
  if (finite) {
    float ol = 3e38f, oh = -3e38f, pl = 3e38f, ph = -3e38f;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const float sx = ((k & 1) ? (float)(X0 + kWT_W) : (float)(X0 - 1)) - g.b0;
      const float sy = ((k & 2) ? (float)(Y0 + kWT_H) : (float)(Y0 - 1)) - g.b1;
      const float ox = M.m00 * sx + M.m01 * sy, oy = M.m10 * sx + M.m11 * sy;
      ol = fminf(ol, ox); oh = fmaxf(oh, ox); pl = fminf(pl, oy); ph = fmaxf(ph, oy);
    }
    ol = fmaxf(ol - 2.0f, 0.0f); oh = fminf(oh + 2.0f, (float)(W - 1));
    pl = fmaxf(pl - 2.0f, 0.0f); ph = fminf(ph + 2.0f, (float)(H - 1));
    if (ol <= oh && pl <= ph) {
      bx.x0 = (int)floorf(ol); bx.x1 = (int)ceilf(oh);
      bx.y0 = (int)floorf(pl); bx.y1 = (int)ceilf(ph);
    }
  }
  warp_box_finish<AL>(bx, cn);
  return bx;
}

// one slab constraint of the gather search: a*ox within [u - r, u + r]
ALB_D void warp_slab(float a, float ra, float u, float r, float& lo, float& hi) {
  if (fabsf(a) > 1e-30f) {
    const float t0 = (u - r) * ra, t1 = (u + r) * ra;
    lo = fmaxf(lo, fminf(t0, t1));
    hi = fminf(hi, fmaxf(t0, t1));
  } else if (fabsf(u) > r) {
    hi = -1.0f;  // never satisfied
    lo = 1.0f;
  }
}

// per-image constants of the gather search
struct GatherK {
  float a00, a01, a10, a11, b0, b1, ra00, ra10;
  float m10, m11, ry, rs, rs2, dout, oxc, oyc, cx, cy;
};

// Gather of two horizontally adjacent source pixels p = (px, py) and
// p' = (px + 1, py) (p' absent when has1 is false): their candidate outputs are
// those sampled in [px - 1, px + 2) x [py - 1, py + 1), searched row by row
// once for both.  A candidate with floor(sx) - px in {-1, 0, 1} is a tap of p
// (px - floor(sx) in {0, 1}), of p' (px + 1 - floor(sx) in {0, 1}) or of both;
// its gradient values are read once, each pixel's input gradient accumulates
// g w in acc0 / acc1, and the two pixels' terms of the same output are folded
// into dL/dsx, dL/dsy before the eight parameter sums S.  G: the gradient rows
// (staged box: `gp` row pitch, `gpl` channel pitch, rows and columns relative
// to (oxb, oyb); or the image itself).
template <bool F3, typename GPtr>
ALB_D void warp_gather_pair(const GatherK& K, const WarpBox& bx, GPtr G, int gp, int gpl, int oxb, int oyb,
                            int px, int py, int cn, bool has1, const float (&xa)[kWT_CG], const float (&xc)[kWT_CG],
                            float (&acc0)[kWT_CG], float (&acc1)[kWT_CG], float (&S)[8]) {
  const float u0 = (float)px - K.b0, v0 = (float)py - K.b1;
  const float oc = K.m10 * u0 + K.m11 * v0;
  const float ocl = fminf(oc, oc + K.m10), och = fmaxf(oc, oc + K.m10);
  const int ylo = max(bx.y0, (int)ceilf(fmaxf(ocl - K.ry, -1.0f)));
  const int yhi = min(bx.y1, (int)floorf(fminf(och + K.ry, 3e7f)));
  for (int oy = ylo; oy <= yhi; oy++) {
    const float oyf = (float)oy;
    const float txr = __fmaf_rn(K.a01, oyf, K.b0), tyr = __fmaf_rn(K.a11, oyf, K.b1);
    float lo = -1.0f, hi = 3e7f;
    warp_slab(K.a00, K.ra00, (float)px + 0.5f - txr, K.rs2, lo, hi);
    warp_slab(K.a10, K.ra10, (float)py - tyr, K.rs, lo, hi);
    const int xlo = max(bx.x0, (int)ceilf(fmaxf(lo - K.dout, -1.0f)));
    const int xhi = min(bx.x1, (int)floorf(fminf(hi + K.dout, 3e7f)));
    const int rowoff = (oy - oyb) * gp - oxb;
    const float yp = oyf - K.oyc;
    float oxf = (float)xlo;
    for (int ox = xlo; ox <= xhi; ox++, oxf += 1.0f) {
      const float sx = __fmaf_rn(K.a00, oxf, txr);
      const float sy = __fmaf_rn(K.a10, oxf, tyr);
      const float fx0 = floorf(sx), fy0 = floorf(sy);
      const int dxa = px - (int)fx0, dy = py - (int)fy0;
      if ((unsigned)(dxa + 1) > 2u || (unsigned)dy > 1u) continue;
      const bool h0 = dxa >= 0, h1 = has1 && dxa <= 0;
      const float fx = sx - fx0, fy = sy - fy0;
      const float wy = dy ? fy : 1.0f - fy;
      const float wx0 = dxa == 1 ? fx : 1.0f - fx;   // p: right tap when dxa = 1
      const float wx1 = dxa == 0 ? fx : 1.0f - fx;   // p': right tap when dxa = 0
      const float w0 = wx0 * wy, w1 = wx1 * wy;
      float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
      for (int k = 0; k < kWT_CG; k++) {
        if (F3 || k < cn) {
          const float gv = G[k * gpl + rowoff + ox];
          if (h0) {
            acc0[k] = __fmaf_rn(gv, w0, acc0[k]);
            a0 = __fmaf_rn(gv, xa[k], a0);
          }
          if (h1) {
            acc1[k] = __fmaf_rn(gv, w1, acc1[k]);
            a1 = __fmaf_rn(gv, xc[k], a1);
          }
        }
      }
      // d w / d sx is +wy for a right tap, -wy for a left one; d w / d sy is
      // +wx for a lower tap, -wx for an upper one
      const float ex = (dxa == 1 ? a0 : -a0) + (dxa == 0 ? a1 : -a1);   // a0 = 0 unless h0, a1 = 0 unless h1
      const float ey = __fmaf_rn(a0, wx0, a1 * wx1);
      const float dsx = ex * wy;
      const float dsy = dy ? ey : -ey;
      const float xp = oxf - K.oxc;
      S[0] = __fmaf_rn(dsx, xp, S[0]);
      S[1] = __fmaf_rn(dsx, yp, S[1]);
      S[2] = __fmaf_rn(dsy, xp, S[2]);
      S[3] = __fmaf_rn(dsy, yp, S[3]);
      S[4] = __fmaf_rn(dsx, sx - K.cx, S[4]);
      S[5] = __fmaf_rn(dsy, sy - K.cy, S[5]);
      S[6] += dsx;
      S[7] += dsy;
    }
  }
}

// Backward as a gather.  Source pixel p is a tap of output q exactly when
// floor(sx_q) is px-1 or px and floor(sy_q) is py-1 or py, with (sx_q, sy_q)
// the float32 coordinate the forward computes.  Each source pixel walks the
// output rows of the parallelogram q = M (p + [-1,1]^2 - b) (M the forward map,
// widened by a rounding margin), solves each row for its ox interval, and
// re-tests every candidate with the forward's own arithmetic, so it sums
// exactly the forward's (q, weight) pairs, in a fixed order (rows, then
// columns): the input gradient is deterministic and needs no atomics.  The
// same pairs carry the parameter gradient: pair (p, q) adds g_q x_p times the
// weight's derivative to dL/dsx_q, dL/dsy_q, and those are folded against the
// coordinate's derivatives through eight running sums per thread.
// F3: every channel group is full (C a multiple of three).
template <bool AL, bool F3>
__global__ void __launch_bounds__(kWT_THREADS, 4) k_warp_f32_bwd(int B, int C, int H, int W, int tiles_x, int tiles,
                                                              const float* __restrict__ x,
                                                              const float* __restrict__ prm,
                                                              const float* __restrict__ gy, float* __restrict__ gx,
                                                              float* __restrict__ partials) {
  extern __shared__ __align__(16) float sm[];
  __shared__ WarpF sg;
  __shared__ float sM[6];  // forward map rows (m00, m01, m10, m11), search margins (source, output)
  __shared__ float red[32];
  const int b = blockIdx.y;
  const int plane = H * W;
  if (threadIdx.x == 0) {
    const WarpF g = warp_setup(prm, b, H, W);
    sg = g;
    const double det = (double)g.a00 * g.a11 - (double)g.a01 * g.a10;
    sM[0] = (float)(g.a11 / det); sM[1] = (float)(-g.a01 / det);
    sM[2] = (float)(-g.a10 / det); sM[3] = (float)(g.a00 / det);
    // source-space margin: a few float32 ulps of the largest coordinate
    const float big = 2.0f * (float)(H > W ? H : W) + fabsf(g.b0) + fabsf(g.b1);
    sM[4] = 1e-3f + 8.0f * big * 1.1920929e-7f;
    sM[5] = 1e-3f + 1e-6f * (float)(H + W);
  }
  __syncthreads();
  const WarpF g = sg;
  const WarpInv M{sM[0], sM[1], sM[2], sM[3]};
  const float dsrc = sM[4];
  const bool finite = isfinite(M.m00) && isfinite(M.m01) && isfinite(M.m10) && isfinite(M.m11) && isfinite(g.b0) &&
                      isfinite(g.b1);
  GatherK K;
  K.a00 = g.a00; K.a01 = g.a01; K.a10 = g.a10; K.a11 = g.a11; K.b0 = g.b0; K.b1 = g.b1;
  K.ra00 = 1.0f / g.a00; K.ra10 = 1.0f / g.a10;
  K.m10 = M.m10; K.m11 = M.m11;
  K.ry = (1.0f + dsrc) * (fabsf(M.m10) + fabsf(M.m11)) + sM[5];
  K.rs = 1.0f + dsrc; K.rs2 = 1.5f + dsrc; K.dout = sM[5];
  K.oxc = g.cx + g.txp; K.oyc = g.cy + g.typ; K.cx = g.cx; K.cy = g.cy;
  const int tp = threadIdx.x & 15, tr = threadIdx.x >> 4;   // pixel pair 2 tp, 2 tp + 1 of tile row tr
  const float* xb = x + (int64_t)b * C * plane;
  const float* gyb = gy + (int64_t)b * C * plane;
  float* gxb = gx + (int64_t)b * C * plane;
  const int groups = (C + kWT_CG - 1) / kWT_CG;
  const int units = warp_units(tiles, groups);
  const float rtx = 1.0f / (float)tiles_x;
  float S[8];
#pragma unroll
  for (int k = 0; k < 8; k++) S[k] = 0.0f;

  WarpBox nb{0, 0, -1, -1, 1, 0};
  if (units > 0) {
    int X0, Y0, c0;
    warp_unit(0, groups, tiles_x, rtx, X0, Y0, c0);
    const int cn0 = F3 ? kWT_CG : min(C - c0, kWT_CG);
    nb = warp_bwd_box<AL>(g, M, finite, X0, Y0, H, W, cn0);
    if (nb.staged) warp_stage_async<AL>(sm, gyb + (int64_t)c0 * plane, cn0, H, W, nb);
  }
  cp_async_commit_f();
  for (int u = 0; u < units; u++) {
    const WarpBox bx = nb;
    int X0, Y0, c0;
    warp_unit(u, groups, tiles_x, rtx, X0, Y0, c0);
    const int cn = F3 ? kWT_CG : min(C - c0, kWT_CG);
    if (u + 1 < units) {
      int X1, Y1, c1;
      warp_unit(u + 1, groups, tiles_x, rtx, X1, Y1, c1);
      const int cn1 = F3 ? kWT_CG : min(C - c1, kWT_CG);
      nb = warp_bwd_box<AL>(g, M, finite, X1, Y1, H, W, cn1);
      if (nb.staged) warp_stage_async<AL>(sm + ((u + 1) & 1) * kWT_BUF, gyb + (int64_t)c1 * plane, cn1, H, W, nb);
    }
    cp_async_commit_f();
    // this unit's source values, loaded while its copies land: each thread
    // owns the horizontal pixel pair (px, px + 1) of tile row tr
    const int px = X0 + 2 * tp, py = Y0 + tr;
    const bool in0 = px < W && py < H, has1 = in0 && px + 1 < W;
    float xa[kWT_CG], xc[kWT_CG];
    {
      const int o = in0 ? py * W + px : 0;
#pragma unroll
      for (int k = 0; k < kWT_CG; k++) {
        xa[k] = (in0 && (F3 || k < cn)) ? __ldg(xb + (int64_t)(c0 + k) * plane + o) : 0.0f;
        xc[k] = (has1 && (F3 || k < cn)) ? __ldg(xb + (int64_t)(c0 + k) * plane + o + 1) : 0.0f;
      }
    }
    cp_async_wait_prev();
    __syncthreads();
    const int bh = bx.y1 - bx.y0 + 1;
    const float* buf = sm + (u & 1) * kWT_BUF;
    if (in0) {
      float acc0[kWT_CG], acc1[kWT_CG];
#pragma unroll
      for (int k = 0; k < kWT_CG; k++) acc0[k] = acc1[k] = finite ? 0.0f : __int_as_float(0x7fc00000);
      if (finite && bx.x1 >= bx.x0) {
        if (bx.staged)
          warp_gather_pair<F3>(K, bx, buf, bx.pitch, bh * bx.pitch, bx.x0, bx.y0, px, py, cn, has1, xa, xc, acc0, acc1,
                           S);
        else
          warp_gather_pair<F3>(K, bx, gyb + (int64_t)c0 * plane, W, plane, 0, 0, px, py, cn, has1, xa, xc, acc0, acc1, S);
      }
      const int o = py * W + px;
#pragma unroll
      for (int k = 0; k < kWT_CG; k++) {
        if (F3 || k < cn) {
          gxb[(int64_t)(c0 + k) * plane + o] = acc0[k];
          if (has1) gxb[(int64_t)(c0 + k) * plane + o + 1] = acc1[k];
        }
      }
    }
    __syncthreads();  // buffer (u & 1) is refilled by unit u + 2
  }
  float R[8];
#pragma unroll
  for (int k = 0; k < 8; k++) R[k] = block_sum(S[k], red);
  if (threadIdx.x == 0) {
    float* pp = partials + ((int64_t)b * gridDim.x + blockIdx.x) * 4;
    const float is = 1.0f / g.s;
    const float dth = (-g.sn * R[0] - g.cs * R[1] + g.cs * R[2] - g.sn * R[3]) * is;
    const float nan = __int_as_float(0x7fc00000);
    pp[0] = finite ? dth * (float)(3.14159265358979323846 / 180.0) : nan;
    pp[1] = finite ? -(R[4] + R[5]) * is : nan;
    pp[2] = finite ? -(g.cs * R[6] + g.sn * R[7]) * g.W * is : nan;
    pp[3] = finite ? (g.sn * R[6] - g.cs * R[7]) * g.H * is : nan;
  }
}

// fixed-order reduction of per-CTA partials: one CTA per image
__global__ void k_reduce_partials(int nblk, int k, const float* __restrict__ partials, float* __restrict__ out) {
  const int b = blockIdx.x;
  __shared__ float red[32];
  for (int j = 0; j < k; j++) {
    float v = 0.f;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) v += partials[((int64_t)b * nblk + i) * k + j];
    v = block_sum(v, red);
    if (threadIdx.x == 0) out[(int64_t)b * k + j] = v;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ photometric
// Elementwise over [C][H][W] per image, four values a thread a step (one
// 16-byte access when the image's element count is a multiple of four, which
// keeps every image's base 16-byte aligned), two steps in flight.
ALB_D float photo_fwd1(float al, float be, float ga, float v) {
  const float z = __fmaf_rn(al, v, be);
  const float zc = fminf(fmaxf(z, 0.0f), 1.0f);
  return zc > 0.0f ? __powf(zc, ga) : 0.0f;  // fast power: a few ulp, far inside the float path's 2e-6
}

template <bool VEC>
ALB_D void ld4(const float* p, int64_t i, int64_t n, float (&v)[4]) {
  if (VEC) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p + i));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = i + k < n ? __ldg(p + i + k) : 0.0f;
  }
}

template <bool VEC>
ALB_D void st4(float* p, int64_t i, int64_t n, const float (&v)[4]) {
  if (VEC) {
    *reinterpret_cast<float4*>(p + i) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int k = 0; k < 4; k++)
      if (i + k < n) p[i + k] = v[k];
  }
}

template <bool VEC>
__global__ void __launch_bounds__(256) k_photo_f32_fwd(int B, int C, int H, int W, const float* __restrict__ x,
                                                       const float* __restrict__ prm, float* __restrict__ y) {
  const int b = blockIdx.y;
  const float al = prm[3 * b], be = prm[3 * b + 1], ga = prm[3 * b + 2];
  const int64_t n = (int64_t)C * H * W;
  const float* xb = x + (int64_t)b * n;
  float* yb = y + (int64_t)b * n;
  const int64_t step = (int64_t)gridDim.x * blockDim.x * 4;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i < n; i += 2 * step) {
    const int64_t i2 = i + step;
    float v[4], w[4];
    ld4<VEC>(xb, i, n, v);
    if (i2 < n) ld4<VEC>(xb, i2, n, w);
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = photo_fwd1(al, be, ga, v[k]);
    st4<VEC>(yb, i, n, v);
    if (i2 < n) {
#pragma unroll
      for (int k = 0; k < 4; k++) w[k] = photo_fwd1(al, be, ga, w[k]);
      st4<VEC>(yb, i2, n, w);
    }
  }
}

// input gradient of one value; accumulates the parameter gradients
ALB_D float photo_bwd1(float al, float be, float ga, float xv, float g, float& da, float& db, float& dg) {
  const float z = __fmaf_rn(al, xv, be);
  if (!(z > 0.0f && z < 1.0f)) return 0.0f;
  const float lz = logf(z);
  const float zg = expf(ga * lz);                    // z^gamma
  const float gz = g * ga * expf((ga - 1.0f) * lz);  // g * gamma * z^(gamma-1)
  dg += g * zg * lz;
  da += gz * xv;
  db += gz;
  return gz * al;
}

template <bool VEC>
__global__ void __launch_bounds__(256) k_photo_f32_bwd(int B, int C, int H, int W, const float* __restrict__ x,
                                                       const float* __restrict__ prm, const float* __restrict__ gy,
                                                       float* __restrict__ gx, float* __restrict__ partials) {
  const int b = blockIdx.y;
  __shared__ float red[32];
  const float al = prm[3 * b], be = prm[3 * b + 1], ga = prm[3 * b + 2];
  const int64_t n = (int64_t)C * H * W;
  const float* xb = x + (int64_t)b * n;
  const float* gb = gy + (int64_t)b * n;
  float* dxb = gx + (int64_t)b * n;
  float da = 0.f, db = 0.f, dg = 0.f;
  const int64_t step = (int64_t)gridDim.x * blockDim.x * 4;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i < n; i += 2 * step) {
    const int64_t i2 = i + step;
    float xv[4], gv[4], xw[4], gw[4];
    ld4<VEC>(xb, i, n, xv);
    ld4<VEC>(gb, i, n, gv);
    if (i2 < n) {
      ld4<VEC>(xb, i2, n, xw);
      ld4<VEC>(gb, i2, n, gw);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) xv[k] = i + k < n ? photo_bwd1(al, be, ga, xv[k], gv[k], da, db, dg) : 0.0f;
    st4<VEC>(dxb, i, n, xv);
    if (i2 < n) {
#pragma unroll
      for (int k = 0; k < 4; k++) xw[k] = i2 + k < n ? photo_bwd1(al, be, ga, xw[k], gw[k], da, db, dg) : 0.0f;
      st4<VEC>(dxb, i2, n, xw);
    }
  }
  const float r0 = block_sum(da, red), r1 = block_sum(db, red), r2 = block_sum(dg, red);
  if (threadIdx.x == 0) {
    float* pp = partials + ((int64_t)b * gridDim.x + blockIdx.x) * 3;
    pp[0] = r0; pp[1] = r1; pp[2] = r2;
  }
}

// the warp kernels' two staging buffers plus their static shared variables
// exceed the default 48 KB: opt in once per device
static alb_status warp_smem_optin() {
  static bool done[64] = {false};
  int dev = 0;
  ALB_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && done[dev]) return ALB_OK;
  const int bytes = 2 * kWT_BUF * (int)sizeof(float);
  const void* kernels[8] = {(const void*)k_warp_f32_fwd<true, true>,  (const void*)k_warp_f32_fwd<true, false>,
                            (const void*)k_warp_f32_fwd<false, true>, (const void*)k_warp_f32_fwd<false, false>,
                            (const void*)k_warp_f32_bwd<true, true>,  (const void*)k_warp_f32_bwd<true, false>,
                            (const void*)k_warp_f32_bwd<false, true>, (const void*)k_warp_f32_bwd<false, false>};
  for (const void* k : kernels) ALB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return ALB_OK;
}

// CTAs per image of the tiled warp kernels: about eight waves of resident
// CTAs over the whole batch (the per-image map is set up once per CTA, which
// then loops over tiles), at most one per tile and at most 1024
static int warp_ctas_per_image(const void* kernel, int tiles, int B) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kWT_THREADS, 2 * kWT_BUF * sizeof(float)) !=
          cudaSuccess || occ < 1)
    occ = 1;
  const int64_t want = ((int64_t)sm_count() * occ * 8 + B - 1) / B;
  int64_t n = want < tiles ? want : tiles;
  if (n > 1024) n = 1024;
  return n < 1 ? 1 : (int)n;
}

// CTAs per image of the elementwise kernels: four full waves of resident
// 256-thread CTAs over the batch, rounded down so that no nearly-empty last
// wave doubles the time; at most one CTA per 256 units and at most 1024
static int blocks_per_image(const void* kernel, int64_t units, int B) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, 0) != cudaSuccess || occ < 1) occ = 1;
  int64_t per = (int64_t)sm_count() * occ * 4 / B;
  const int64_t cap = (units + 255) / 256;
  if (per > cap) per = cap;
  if (per < 1) per = 1;
  if (per > 1024) per = 1024;
  return (int)per;
}

}  // namespace alb

using namespace alb;

static alb_status check_f32(int32_t B, int32_t C, int32_t H, int32_t W, const void* a, const void* b, const void* c) {
  ALB_REQUIRE(B >= 0 && C >= 1 && H >= 1 && W >= 1, ALB_ESHAPE, "f32 path: bad shape %dx%dx%dx%d", B, C, H, W);
  ALB_REQUIRE(B == 0 || (a && b && c), ALB_EINVAL, "f32 path: null pointer");
  return ALB_OK;
}

extern "C" size_t alb_f32_workspace_size(int32_t B, int32_t C, int32_t H, int32_t W) {
  return (size_t)(B > 0 ? B : 1) * 1024 * 4 * sizeof(float) + 256;
}

// warp shapes: batch within the grid's y limit, per-image offsets of a channel
// group within int32
static alb_status check_warp_shape(int32_t B, int32_t H, int32_t W, const char* what) {
  ALB_REQUIRE(B <= 65535, ALB_ESHAPE, "%s: batch %d above 65535", what, B);
  ALB_REQUIRE((int64_t)(kWT_CG + 1) * H * W < (1LL << 31), ALB_ESHAPE, "%s: image %dx%d too large", what, H, W);
  return ALB_OK;
}

// 16-byte staging of the staged tensor: W a multiple of four and 16-byte
// aligned planes
static bool warp_aligned(int32_t W, const void* staged) {
  return W % 4 == 0 && ((uintptr_t)staged % 16) == 0;
}

extern "C" alb_status alb_warp_affine_f32_fwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                              const float* prm, float* y, void* stream) {
  alb_status rc = check_f32(B, C, H, W, x, prm, y);
  if (rc != ALB_OK || B == 0) return rc;
  rc = check_warp_shape(B, H, W, "alb_warp_affine_f32_fwd");
  if (rc != ALB_OK) return rc;
  rc = warp_smem_optin();
  if (rc != ALB_OK) return rc;
  const int tiles_x = (W + kWT_W - 1) / kWT_W, tiles_y = (H + kWT_H - 1) / kWT_H;
  const int tiles = tiles_x * tiles_y;
  const bool al = warp_aligned(W, x), f3 = C % kWT_CG == 0;
  void (*kern)(int, int, int, int, int, int, const float*, const float*, float*) =
      al ? (f3 ? k_warp_f32_fwd<true, true> : k_warp_f32_fwd<true, false>)
         : (f3 ? k_warp_f32_fwd<false, true> : k_warp_f32_fwd<false, false>);
  const int nblk = warp_ctas_per_image((const void*)kern, tiles, B);
  kern<<<dim3(nblk, B), kWT_THREADS, 2 * kWT_BUF * sizeof(float), (cudaStream_t)stream>>>(B, C, H, W, tiles_x, tiles,
                                                                                        x, prm, y);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

extern "C" alb_status alb_warp_affine_f32_bwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                              const float* prm, const float* gy, float* gx, float* gprm,
                                              void* workspace, size_t workspace_bytes, void* stream) {
  alb_status rc = check_f32(B, C, H, W, x, prm, gy);
  if (rc != ALB_OK || B == 0) return rc;
  ALB_REQUIRE(gx && gprm, ALB_EINVAL, "alb_warp_affine_f32_bwd: null output");
  rc = check_warp_shape(B, H, W, "alb_warp_affine_f32_bwd");
  if (rc != ALB_OK) return rc;
  rc = warp_smem_optin();
  if (rc != ALB_OK) return rc;
  const int tiles_x = (W + kWT_W - 1) / kWT_W, tiles_y = (H + kWT_H - 1) / kWT_H;
  const int tiles = tiles_x * tiles_y;
  const bool al = warp_aligned(W, gy), f3 = C % kWT_CG == 0;
  void (*kern)(int, int, int, int, int, int, const float*, const float*, const float*, float*, float*) =
      al ? (f3 ? k_warp_f32_bwd<true, true> : k_warp_f32_bwd<true, false>)
         : (f3 ? k_warp_f32_bwd<false, true> : k_warp_f32_bwd<false, false>);
  const int nblk = warp_ctas_per_image((const void*)kern, tiles, B);
  ALB_REQUIRE(workspace && workspace_bytes >= (size_t)B * nblk * 4 * sizeof(float), ALB_EWORKSPACE,
              "alb_warp_affine_f32_bwd: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  kern<<<dim3(nblk, B), kWT_THREADS, 2 * kWT_BUF * sizeof(float), st>>>(B, C, H, W, tiles_x, tiles, x, prm, gy, gx,
                                                                      (float*)workspace);
  ALB_CUDA(cudaGetLastError());
  k_reduce_partials<<<B, 256, 0, st>>>(nblk, 4, (const float*)workspace, gprm);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

extern "C" alb_status alb_photometric_f32_fwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                              const float* prm, float* y, void* stream) {
  alb_status rc = check_f32(B, C, H, W, x, prm, y);
  if (rc != ALB_OK || B == 0) return rc;
  ALB_REQUIRE(B <= 65535, ALB_ESHAPE, "alb_photometric_f32_fwd: batch %d above 65535", B);
  const int64_t n = (int64_t)C * H * W;
  const bool vec = n % 4 == 0 && ((uintptr_t)x % 16) == 0 && ((uintptr_t)y % 16) == 0;
  const void* kern = vec ? (const void*)k_photo_f32_fwd<true> : (const void*)k_photo_f32_fwd<false>;
  dim3 grid(blocks_per_image(kern, (n + 3) / 4, B), B);
  if (vec)
    k_photo_f32_fwd<true><<<grid, 256, 0, (cudaStream_t)stream>>>(B, C, H, W, x, prm, y);
  else
    k_photo_f32_fwd<false><<<grid, 256, 0, (cudaStream_t)stream>>>(B, C, H, W, x, prm, y);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

extern "C" alb_status alb_photometric_f32_bwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                              const float* prm, const float* gy, float* gx, float* gprm,
                                              void* workspace, size_t workspace_bytes, void* stream) {
  alb_status rc = check_f32(B, C, H, W, x, prm, gy);
  if (rc != ALB_OK || B == 0) return rc;
  ALB_REQUIRE(gx && gprm, ALB_EINVAL, "alb_photometric_f32_bwd: null output");
  ALB_REQUIRE(B <= 65535, ALB_ESHAPE, "alb_photometric_f32_bwd: batch %d above 65535", B);
  const int64_t n = (int64_t)C * H * W;
  const bool vec = n % 4 == 0 && ((uintptr_t)x % 16) == 0 && ((uintptr_t)gy % 16) == 0 && ((uintptr_t)gx % 16) == 0;
  const void* kern = vec ? (const void*)k_photo_f32_bwd<true> : (const void*)k_photo_f32_bwd<false>;
  const int nblk = blocks_per_image(kern, (n + 3) / 4, B);
  ALB_REQUIRE(workspace && workspace_bytes >= (size_t)B * nblk * 3 * sizeof(float), ALB_EWORKSPACE,
              "alb_photometric_f32_bwd: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  if (vec)
    k_photo_f32_bwd<true><<<dim3(nblk, B), 256, 0, st>>>(B, C, H, W, x, prm, gy, gx, (float*)workspace);
  else
    k_photo_f32_bwd<false><<<dim3(nblk, B), 256, 0, st>>>(B, C, H, W, x, prm, gy, gx, (float*)workspace);
  ALB_CUDA(cudaGetLastError());
  k_reduce_partials<<<B, 256, 0, st>>>(nblk, 3, (const float*)workspace, gprm);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

namespace alb {
ALB_OOB_ACCESSOR(oob_diff)
}  // namespace alb
