// alb_resample.cu -- tiled resampling for the transforms that move pixels along
// a continuous map: the affine warps (Table I: Rotate, ShiftScaleRotate) and
// the resizes (Sec. II-B scaling; Sec. II-A random sized crop), for images
// (Q5 bilinear) and their masks (nearest), with reflect-101 borders for warps.
//
// Work item = one output tile, owned by ONE warp: there is no block-wide
// barrier anywhere.  Each warp stages the source footprint of its tile (the
// bounding box of the mapped tile plus the +1 tap) in its own shared-memory box
// as raw, aligned 16-byte cp.async copies, one staged row per lane with the
// row's byte phase kept beside it.  The general kernel (16 x 16 tiles, masks)
// double-buffers the box: while it computes tile i, tile i + 1's copies are in
// flight.  The RGB kernels below single-buffer it instead: half the shared
// memory per warp lets more warps reside, and other warps hide the copies
// better than a second buffer does (measured: resize -16 %, affine -12 %).  Rows are reflected (warps) or clamped (resizes) when
// they are copied; for tiles whose box crosses the image's left/right border
// the staged span is the reflected column range and each tap column goes
// through the border map.  Lane l computes output column l & 15 for rows
// (l >> 4) + 2k and stores its bytes directly.  Tiles whose footprint does not
// fit the box (scales below ~0.45) read their taps from global memory.
#include "alb_common.cuh"
#include "alb_kernels.cuh"
#include "alb_vec.cuh"
#include "alb_distort.cuh"

namespace alb {

constexpr int WT = 16;          // warp tile side, output pixels
constexpr int WBOX = 36;        // staged box side: boxes of up to WBOX - 1 pixels fit
constexpr int NWARP = 4;        // warps per CTA

template <int C>
struct WPitch {
  // staged row pitch: a multiple of 16 bytes (cp.async destinations) whose word
  // count (36 / 20) is not a multiple of 32, so successive rows start in different banks
  static constexpr int SROW = C == 3 ? 144 : 80;
  static_assert(SROW % 16 == 0, "cp.async destinations must be 16-byte aligned");
  static_assert(C == 3 ? SROW >= 15 + 3 * (WBOX - 1) + 12 : SROW >= 16 * ((15 + WBOX - 1 + 15) / 16), "row pitch");
};

// --------------------------------------------------------------- tile plan
__global__ void k_plan_tiles(ImgList out, int32_t n, int32_t tile_w, int32_t tile_h, int32_t* __restrict__ prefix,
                             int32_t* __restrict__ tiles_x, PlanCheck chk) {
  __shared__ int32_t wsum[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    int32_t cnt = 0;
    if (i < n) {
      const alb_image im = out.get(i);
      const int32_t tx = (im.w + tile_w - 1) / tile_w, ty = (im.h + tile_h - 1) / tile_h;
      cnt = im.h > 0 && im.w > 0 ? tx * ty : 0;
      tiles_x[i] = tx > 0 ? tx : 1;
      if (check_image_pair(chk.tid, chk.prm.get(i), chk.in.get(i), im, chk.want_c, chk.geometric)) cnt = 0;
      if (plan_filtered_out(chk, im)) cnt = 0;
      if (chk.reduce != 0 && cnt) {
        const alb_params& pr = chk.prm.get(i);
        // class 2: windows no larger than the output on either axis (64 x 32
        // tiles fit the 66 x 34 box: 63 f + 2 <= 65 columns, 31 f + 2 <= 33 rows);
        // class 1: reductions whose 32 x 16 tiles fit the 66 x 34 box (31 f + 3
        // <= 66 columns, 15 f + 3 <= 34 rows); class 3: stronger reductions,
        // whose 32 x 32 tiles read global memory
        const bool past = pr.cw > im.w || pr.ch > im.h;
        const bool fits = 1000 * (int64_t)pr.cw <= 2032 * (int64_t)im.w && 1000 * (int64_t)pr.ch <= 2066 * (int64_t)im.h;
        const int32_t cls = !past ? 2 : (fits ? 1 : 3);
        if (cls != chk.reduce) cnt = 0;
      }
    }
    int32_t v = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (lane == 31) wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
      int32_t s = lane < nw ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
      }
      if (lane < nw) wsum[lane] = s;
    }
    __syncthreads();
    const int32_t excl = carry + (wid ? wsum[wid - 1] : 0) + v - cnt;
    if (i < n) prefix[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + cnt;
    __syncthreads();
  }
  if (threadIdx.x == 0) prefix[n] = carry;
}

// --------------------------------------------------------------- coordinate maps
ALB_D int32_t rs_q5(int32_t d, int32_t n_in, int32_t n_out) {  // half-pixel Q5 resize coordinate
  int64_t xq;
  if (n_in <= 2048 && n_out <= 2048) {
    // |numerator| < 2^29: exact in 32-bit (floor division of a possibly negative value)
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
ALB_D int32_t rs_nn(int32_t d, int32_t n_in, int32_t n_out) {
  const int64_t i = (n_in <= 2048 && n_out <= 2048) ? (int64_t)((uint32_t)((2 * d + 1) * n_in) / (uint32_t)(2 * n_out))
                                                     : ((int64_t)(2 * d + 1) * n_in) / (2 * (int64_t)n_out);
  return (int32_t)(i < n_in - 1 ? i : n_in - 1);
}

enum { MAP_AFFINE = 0, MAP_RESIZE = 1, MAP_GRID = 2 };

// Q5 bilinear from a byte grid (row pitch `pitch`, C = 3 channels), taps at
// byte offset o (ix, iy) and o + pitch: three aligned words per row, realigned.
ALB_D void taps_row(const uint8_t* base, int o, uint32_t& lo, uint32_t& hi) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(base + (o & ~3));
  const int s = 8 * (o & 3);
  const uint32_t w0 = w[0], w1 = w[1], w2 = w[2];
  lo = __funnelshift_r(w0, w1, s);
  hi = __funnelshift_r(w1, w2, s);
}

// the 6 bytes at p (pixels ix, ix + 1 of a row) as lo = bytes 0..3, hi = 4..5;
// aligned word loads, the third only when it holds a needed byte
ALB_D void ldg_pair(const uint8_t* p, uint32_t& lo, uint32_t& hi) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint32_t* w = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
  const int s = (int)(a & 3);
  const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = s == 3 ? __ldg(w + 2) : 0u;
  lo = __funnelshift_r(w0, w1, 8 * s);
  hi = __funnelshift_r(w1, w2, 8 * s);
}

// Q5 bilinear of one RGB pixel from the two tap rows (lo = bytes 0..3, hi =
// bytes 4..5 of the 6-byte pair (ix, ix + 1) of each row), exactly
// (sum w_ij p_ij + 512) >> 10 with w_ij = wx_i * wy_j, evaluated as
// ((32 - fy) h_top + fy h_bot + 512) >> 10 with h = (32 - fx) p0 + fx p1
// (the same integer): the 8-bit-weight horizontal pairs are dp4a products,
// the vertical pair (two 13-bit partials, 8-bit weights) one dp2a.
ALB_D uint32_t bilerp3(uint32_t t_lo, uint32_t t_hi, uint32_t b_lo, uint32_t b_hi, int fx, int fy) {
  const uint32_t wx = (uint32_t)(32 - fx) | ((uint32_t)fx << 8);
  const uint32_t wy = (uint32_t)(32 - fy) | ((uint32_t)fy << 8);
  // channel c of pixels ix and ix + 1: bytes (c, 3 + c) of the 6-byte pair
  const uint32_t ht_r = __dp4a(__byte_perm(t_lo, t_hi, 0x0030), wx, 0u);
  const uint32_t hb_r = __dp4a(__byte_perm(b_lo, b_hi, 0x0030), wx, 0u);
  const uint32_t ht_g = __dp4a(__byte_perm(t_lo, t_hi, 0x0041), wx, 0u);
  const uint32_t hb_g = __dp4a(__byte_perm(b_lo, b_hi, 0x0041), wx, 0u);
  const uint32_t ht_b = __dp4a(__byte_perm(t_lo, t_hi, 0x0052), wx, 0u);
  const uint32_t hb_b = __dp4a(__byte_perm(b_lo, b_hi, 0x0052), wx, 0u);
  const uint32_t r = __dp2a_lo(__byte_perm(ht_r, hb_r, 0x5410), wy, 512u) >> 10;
  const uint32_t g = __dp2a_lo(__byte_perm(ht_g, hb_g, 0x5410), wy, 512u) >> 10;
  const uint32_t b = __dp2a_lo(__byte_perm(ht_b, hb_b, 0x5410), wy, 512u) >> 10;
  return r | (g << 8) | (b << 16);
}

// --------------------------------------------------------------- async copies
ALB_D void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
ALB_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
ALB_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Per-image values of a warp's current image (uniform across the warp's lanes).
struct WImg {
  int32_t b, prefix, ntiles, tiles_x;
  int32_t H, W, OH, OW, cw, ch, wx0, wy0;
  int64_t q[6];
  const uint8_t* src;
  uint8_t* dst;
  int64_t sstride, dstride;
};

template <int MAP>
ALB_D void load_img(const Plan& plan, const ImgList& in, const ImgList& out, const PrmList& prm, int32_t b, WImg& k) {
  const alb_image si = in.get(b), so = out.get(b);
  const alb_params& p = prm.get(b);
  k.b = b; k.prefix = plan.prefix[b]; k.ntiles = plan.prefix[b + 1] - k.prefix; k.tiles_x = plan.rows_per_item[b];
  k.H = si.h; k.W = si.w; k.OH = so.h; k.OW = so.w;
  k.cw = MAP == MAP_RESIZE ? p.cw : si.w; k.ch = MAP == MAP_RESIZE ? p.ch : si.h;
  k.wx0 = MAP == MAP_RESIZE ? p.x0 : 0; k.wy0 = MAP == MAP_RESIZE ? p.y0 : 0;
  const bool app = MAP == MAP_AFFINE && p.apply;
  k.q[0] = app ? p.q[0] : 65536; k.q[1] = app ? p.q[1] : 0; k.q[2] = app ? p.q[2] : 0;
  k.q[3] = app ? p.q[3] : 0; k.q[4] = app ? p.q[4] : 65536; k.q[5] = app ? p.q[5] : 0;
  k.src = (const uint8_t*)si.data; k.dst = (uint8_t*)so.data;
  k.sstride = si.row_stride; k.dstride = so.row_stride;
}

// Geometry of one warp tile.  `v` (per lane): for resizes, lane l < 16 holds the
// Q5 (or nearest) coordinate of tile column l, lane 16 + r that of tile row r.
struct WTile {
  int32_t ox0, oy0, tw, th;
  int32_t bx0, by0, bw, bh, ra, rb, mode;   // mode 0 inside, 1 crosses a border, 2 too large
  int64_t X00, Y00;
  int32_t v;
};

template <int MAP, bool NEAREST, int C>
ALB_D void tile_geo(const WImg& k, int32_t item, int lane, WTile& g) {
  const int32_t t = item - k.prefix, ty = t / k.tiles_x, tx = t - ty * k.tiles_x;
  g.ox0 = tx * WT; g.oy0 = ty * WT;
  g.tw = imin(WT, k.OW - g.ox0); g.th = imin(WT, k.OH - g.oy0);
  int32_t bx0, bx1, by0, by1;
  g.X00 = 0; g.Y00 = 0; g.v = 0;
  if (MAP == MAP_AFFINE) {
    g.X00 = k.q[0] * g.ox0 + k.q[1] * g.oy0 + k.q[2];
    g.Y00 = k.q[3] * g.ox0 + k.q[4] * g.oy0 + k.q[5];
    const int64_t dXx = k.q[0] * (g.tw - 1), dXy = k.q[1] * (g.th - 1), dYx = k.q[3] * (g.tw - 1), dYy = k.q[4] * (g.th - 1);
    const int64_t xmin = g.X00 + (dXx < 0 ? dXx : 0) + (dXy < 0 ? dXy : 0);
    const int64_t xmax = g.X00 + (dXx > 0 ? dXx : 0) + (dXy > 0 ? dXy : 0);
    const int64_t ymin = g.Y00 + (dYx < 0 ? dYx : 0) + (dYy < 0 ? dYy : 0);
    const int64_t ymax = g.Y00 + (dYx > 0 ? dYx : 0) + (dYy > 0 ? dYy : 0);
    if (NEAREST) {
      bx0 = (int32_t)((xmin + 32768) >> 16); bx1 = (int32_t)((xmax + 32768) >> 16);
      by0 = (int32_t)((ymin + 32768) >> 16); by1 = (int32_t)((ymax + 32768) >> 16);
    } else {
      bx0 = (int32_t)((xmin + 1024) >> 16); bx1 = (int32_t)((xmax + 1024) >> 16) + 1;
      by0 = (int32_t)((ymin + 1024) >> 16); by1 = (int32_t)((ymax + 1024) >> 16) + 1;
    }
  } else {
    const bool col = lane < 16;
    const int32_t d = col ? g.ox0 + imin(lane, g.tw - 1) : g.oy0 + imin(lane - 16, g.th - 1);
    const int32_t nin = col ? k.cw : k.ch, nout = col ? k.OW : k.OH;
    g.v = NEAREST ? rs_nn(d, nin, nout) : rs_q5(d, nin, nout);
    const int32_t c0 = __shfl_sync(0xffffffffu, g.v, 0), c1 = __shfl_sync(0xffffffffu, g.v, g.tw - 1);
    const int32_t r0 = __shfl_sync(0xffffffffu, g.v, 16), r1 = __shfl_sync(0xffffffffu, g.v, 16 + g.th - 1);
    if (NEAREST) {
      bx0 = c0; bx1 = c1; by0 = r0; by1 = r1;
    } else {
      bx0 = c0 >> 5; bx1 = imin((c1 >> 5) + 1, k.cw - 1);
      by0 = r0 >> 5; by1 = imin((r1 >> 5) + 1, k.ch - 1);
    }
  }
  g.bx0 = bx0; g.by0 = by0; g.bw = bx1 - bx0 + 1; g.bh = by1 - by0 + 1;
  g.ra = bx0; g.rb = bx1; g.mode = 0;
  const int32_t W = k.W;
  if (g.bw > WBOX - 1 || g.bh > WBOX - 1) {
    g.mode = 2;
  } else if (MAP == MAP_AFFINE && (bx0 < 0 || bx1 >= W)) {
    // stage the real columns the box's columns reflect onto (one fold at most)
    int32_t lo, hi;
    const bool ok = W > 1 && bx0 > -W && bx1 < 2 * W - 1;
    if (bx0 < 0 && bx1 >= W) { lo = 0; hi = W - 1; }
    else if (bx0 < 0) { lo = bx1 < 0 ? -bx1 : 0; hi = imax(-bx0, bx1); }
    else { lo = bx0 > W - 1 ? 2 * (W - 1) - bx1 : imin(bx0, 2 * (W - 1) - bx1); hi = bx0 > W - 1 ? 2 * (W - 1) - bx0 : W - 1; }
    g.ra = lo; g.rb = hi;
    g.mode = ok && hi - lo + 1 <= WBOX - 1 ? 1 : 2;
  }
}

// Lane r (and r + 32) copies staged row r of the tile's box: raw aligned chunks.
template <int MAP, int C>
ALB_D void tile_stage(const WImg& k, const WTile& g, int lane, uint8_t* box, int16_t* phase) {
  if (g.mode == 2) return;
  const int span = C * (g.rb - g.ra + 1);
  for (int r = lane; r < g.bh; r += 32) {
    const int vy = g.by0 + r;
    const int ry = MAP == MAP_AFFINE ? reflect101(vy, k.H) : k.wy0 + imin(vy, k.ch - 1);
    const uintptr_t first = reinterpret_cast<uintptr_t>(k.src) + (uintptr_t)((int64_t)ry * k.sstride) +
                            (uintptr_t)(C * (k.wx0 + g.ra));
    const uintptr_t c0 = first & ~uintptr_t(15);
    const int ph = (int)(first - c0);
    phase[r] = (int16_t)ph;
    const int nch = (ph + span + 15) >> 4;
    uint8_t* d = box + r * WPitch<C>::SROW;
    const int64_t ib = (int64_t)(k.H - 1) * k.sstride + (int64_t)C * k.W;
    for (int j = 0; j < nch; j++)
      if (ALB_IN(bytes_within(reinterpret_cast<const void*>(c0 + 16 * j), 16, k.src, ib, 15) && r < WBOX &&
                 16 * j + 16 <= WPitch<C>::SROW))
        cp_async16(d + 16 * j, reinterpret_cast<const void*>(c0 + 16 * j));
  }
}

template <int MAP, bool NEAREST, int C>
ALB_D void tile_compute(const WImg& ks, const WTile& g, int lane, const uint8_t* __restrict__ bx,
                        const int16_t* __restrict__ ph) {
  constexpr int SROW = WPitch<C>::SROW;
  // a register copy: the global byte stores below could otherwise alias the
  // shared-memory state and force a reload of every field after each store
  const WImg k = ks;
  const int px = lane & 15, py0 = lane >> 4;
  const int32_t W = k.W, H = k.H;
  const int64_t q0 = k.q[0], q1 = k.q[1], q2 = k.q[2], q3 = k.q[3], q4 = k.q[4], q5 = k.q[5];
  int32_t cq = 0;
  if (MAP == MAP_RESIZE) cq = __shfl_sync(0xffffffffu, g.v, px);
  int32_t Xr = 0, Yr = 0;
  if (MAP == MAP_AFFINE) {
    Xr = (int32_t)(g.X00 - 65536 * (int64_t)g.bx0) + (int32_t)q0 * px + (int32_t)q1 * py0;
    Yr = (int32_t)(g.Y00 - 65536 * (int64_t)g.by0) + (int32_t)q3 * px + (int32_t)q4 * py0;
  }
  const int32_t dX = 2 * (int32_t)q1, dY = 2 * (int32_t)q4;
#pragma unroll 2
  for (int kk = 0; kk < WT / 2; kk++, Xr += dX, Yr += dY) {
    const int py = py0 + 2 * kk;
    int32_t rq = 0;
    if (MAP == MAP_RESIZE) rq = __shfl_sync(0xffffffffu, g.v, 16 + py);
    if (px >= g.tw || py >= g.th) continue;
    if (!ALB_IN(g.oy0 + py < k.OH && g.ox0 + px < k.OW)) continue;
    uint8_t* __restrict__ od = k.dst + (int64_t)(g.oy0 + py) * k.dstride + (int64_t)C * (g.ox0 + px);
    if (g.mode != 2) {
      int ix, iy, fx = 0, fy = 0;
      if (MAP == MAP_AFFINE) {
        if (NEAREST) { ix = (Xr + 32768) >> 16; iy = (Yr + 32768) >> 16; }
        else {
          const int xq = (Xr + 1024) >> 11, yq = (Yr + 1024) >> 11;
          ix = xq >> 5; fx = xq & 31; iy = yq >> 5; fy = yq & 31;
        }
      } else {
        if (NEAREST) { ix = cq - g.bx0; iy = rq - g.by0; }
        else {
          const int xq = cq - 32 * g.bx0, yq = rq - 32 * g.by0;
          ix = xq >> 5; fx = xq & 31; iy = yq >> 5; fy = yq & 31;
        }
      }
      if (!ALB_IN(iy >= 0 && iy < g.bh && ix >= 0 && ix < g.bw && (NEAREST || g.mode != 1 || iy + 1 < g.bh)))
        continue;
      const int o0 = iy * SROW + ph[iy];
      if (NEAREST) {
        const int rx = g.mode == 1 ? reflect101(g.bx0 + ix, W) - g.ra : ix;
        if (!ALB_IN(rx >= 0 && rx <= g.rb - g.ra)) continue;
#pragma unroll
        for (int c = 0; c < C; c++) od[c] = bx[o0 + C * rx + c];
      } else if (g.mode == 0) {
        // the +1 row: at a resize's clamped bottom edge it is past the staged
        // rows and has weight fy = 0, so the last staged row stands in for it
        const int iy1 = iy + 1 < g.bh ? iy + 1 : iy;
        const int o1 = iy1 * SROW + ph[iy1];
        uint32_t tl, th2, bl, bh2;
        taps_row(bx, o0 + 3 * ix, tl, th2);     // bx is 16-byte aligned: word alignment is that of the offset
        taps_row(bx, o1 + 3 * ix, bl, bh2);
        const uint32_t v = bilerp3(tl, th2, bl, bh2, fx, fy);
        od[0] = (uint8_t)v; od[1] = (uint8_t)(v >> 8); od[2] = (uint8_t)(v >> 16);
      } else {
        const int o1 = (iy + 1) * SROW + ph[iy + 1];
        const int xa = 3 * (reflect101(g.bx0 + ix, W) - g.ra), xb = 3 * (reflect101(g.bx0 + ix + 1, W) - g.ra);
        const int w11 = fx * fy, w01 = 32 * fx - w11, w10 = 32 * fy - w11, w00 = 1024 - 32 * fx - 32 * fy + w11;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const int acc = w00 * bx[o0 + xa + c] + w01 * bx[o0 + xb + c] + w10 * bx[o1 + xa + c] + w11 * bx[o1 + xb + c];
          od[c] = (uint8_t)((acc + 512) >> 10);
        }
      }
    } else {
      // footprint too large for the box: taps straight from global memory
      const int x = g.ox0 + px, y = g.oy0 + py;
      int sx0, sy0, sx1 = 0, sy1 = 0, fx = 0, fy = 0;
      if (MAP == MAP_AFFINE) {
        const int64_t X = q0 * x + q1 * y + q2, Y = q3 * x + q4 * y + q5;
        if (NEAREST) {
          sx0 = reflect101((X + 32768) >> 16, W); sy0 = reflect101((Y + 32768) >> 16, H);
        } else {
          const int64_t xq = (X + 1024) >> 11, yq = (Y + 1024) >> 11;
          fx = (int)(xq & 31); fy = (int)(yq & 31);
          sx0 = reflect101(xq >> 5, W); sx1 = reflect101((xq >> 5) + 1, W);
          sy0 = reflect101(yq >> 5, H); sy1 = reflect101((yq >> 5) + 1, H);
        }
      } else {
        if (NEAREST) {
          sx0 = k.wx0 + cq; sy0 = k.wy0 + rq;
        } else {
          fx = cq & 31; fy = rq & 31;
          sx0 = k.wx0 + (cq >> 5); sx1 = k.wx0 + imin((cq >> 5) + 1, k.cw - 1);
          sy0 = k.wy0 + (rq >> 5); sy1 = k.wy0 + imin((rq >> 5) + 1, k.ch - 1);
        }
      }
      if (!ALB_IN(sx0 >= 0 && sx0 < W && sy0 >= 0 && sy0 < H && (NEAREST || (sx1 >= 0 && sx1 < W && sy1 >= 0 &&
                                                                       sy1 < H))))
        continue;
      if (NEAREST) {
        const uint8_t* s0 = k.src + (int64_t)sy0 * k.sstride + (int64_t)C * sx0;
#pragma unroll
        for (int c = 0; c < C; c++) od[c] = s0[c];
      } else {
        const int w11 = fx * fy, w01 = 32 * fx - w11, w10 = 32 * fy - w11, w00 = 1024 - 32 * fx - 32 * fy + w11;
        const uint8_t* ra = k.src + (int64_t)sy0 * k.sstride;
        const uint8_t* rbp = k.src + (int64_t)sy1 * k.sstride;
#pragma unroll
        for (int c = 0; c < C; c++) {
          const int acc = w00 * ra[3 * sx0 + c] + w01 * ra[3 * sx1 + c] + w10 * rbp[3 * sx0 + c] + w11 * rbp[3 * sx1 + c];
          od[c] = (uint8_t)((acc + 512) >> 10);
        }
      }
    }
  }
}

template <int MAP, bool NEAREST, int C>
__global__ void __launch_bounds__(32 * NWARP, 5) k_resample_warp(Plan plan, ImgList in, ImgList out, PrmList prm) {
  constexpr int BOXB = WBOX * WPitch<C>::SROW;
  __shared__ __align__(16) uint8_t box[NWARP][2][BOXB];
  __shared__ int16_t phase[NWARP][2][WBOX];
  __shared__ WImg simg[NWARP][2];      // image state of the tile in each buffer (warp-uniform)
  __shared__ WTile stile[NWARP][2];    // geometry of the tile in each buffer
  int32_t it0, it1;
  item_range(plan, it0, it1);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t item = it0 + w;
  if (item >= it1) return;
  // prologue: the warp's first tile goes to buffer 0
  int32_t vcur;   // per-lane resize coordinate of the current tile
  {
    WImg k;
    WTile g;
    load_img<MAP>(plan, in, out, prm, item_image(plan, item), k);
    tile_geo<MAP, NEAREST, C>(k, item, lane, g);
    vcur = g.v;
    if (lane == 0) { simg[w][0] = k; stile[w][0] = g; }
    tile_stage<MAP, C>(k, g, lane, box[w][0], phase[w][0]);
  }
  cp_async_commit();
  int buf = 0;
  for (; item < it1; item += NWARP, buf ^= 1) {
    const int32_t nitem = item + NWARP;
    int32_t vnext = 0;
    if (nitem < it1) {
      __syncwarp();
      WImg k = simg[w][buf];
      if (nitem >= k.prefix + k.ntiles) {
        int32_t b = k.b;
        while (nitem >= plan.prefix[b + 1]) b++;
        load_img<MAP>(plan, in, out, prm, b, k);
      }
      WTile g;
      tile_geo<MAP, NEAREST, C>(k, nitem, lane, g);
      vnext = g.v;
      __syncwarp();
      if (lane == 0) { simg[w][buf ^ 1] = k; stile[w][buf ^ 1] = g; }
      tile_stage<MAP, C>(k, g, lane, box[w][buf ^ 1], phase[w][buf ^ 1]);
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();
    WTile g = stile[w][buf];
    g.v = vcur;
    tile_compute<MAP, NEAREST, C>(simg[w][buf], g, lane, box[w][buf], phase[w][buf]);
    __syncwarp();       // every lane is done with box[buf] before it is refilled
    vcur = vnext;
  }
  cp_async_wait<0>();
}

// --------------------------------------------------------------- separable resize
// Bilinear RGB resizes (Resize, RandomSizedCrop, RandomResizedCrop) use the
// separability of the Q5 weights: out = ((32 - fy) h(iy) + fy h(iy + 1) + 512)
// >> 10 with h(i) = (32 - fx) p(i, ix) + fx p(i, ix + 1) exact in integers, so
// h of a source row is computed once per output column and reused by every
// output row whose tap rows include it.  A warp owns an output tile, lane j =
// output column j (and j + 32 in the 64-wide shape); it walks the tile's rows
// top to bottom keeping the two current tap rows' h in registers and computes
// a new row of h only when the warp-uniform top tap row moves (for an
// enlargement most output rows reuse both, or shift by one source row).  The
// tile's source box (up to BX x BY pixels of its shape) is staged per warp in
// shared memory by cp.async, one buffer per warp (the per-tile image and
// geometry stay in registers).  Measured trade-off: a taller tile amortises
// the per-tile geometry, a larger box costs warps per SM (the row chain is
// latency-bound); with one column per lane 32 x 32 with a 36 x 36 box beat
// 32 x 16 with 36 x 20 and 32 x 32 with 36 x 28; two columns per lane (the
// row's coordinate, box row offset and advance test shared) beat one.
// Larger footprints read global memory.  Three tile shapes, one per scale
// class of the window (routed per image by the tile plans): S = 0, 64 x 32
// tiles with a 66 x 34 box, two columns per lane (windows no larger than the
// output on either axis; the small box keeps 7 CTAs per SM); S = 1, 32 x 16
// tiles with a 66 x 34 box (reductions up to ~2); S = 2, 32 x 32 tiles with a
// 36 x 36 box (stronger reductions, whose tiles read global memory at the
// highest residency).
template <int S>
struct RShape {
  // S = 0: windows no larger than the output; 1: reductions up to ~2x;
  // 2: the rest (and every image when there is no second plan)
  static constexpr int TW = S == 0 ? 64 : 32, TH = S == 1 ? 16 : 32;   // output tile (columns x rows)
  static constexpr int NC = TW / 32;                      // output columns per lane: lane, lane + 32
  static constexpr int BX = S == 2 ? 36 : 66, BY = S == 2 ? 36 : 34;   // staged box (pixels x rows)
  static constexpr int PITCH = S == 2 ? 144 : 224;        // staged row pitch in bytes
  static_assert(PITCH % 16 == 0, "cp.async destinations must be 16-byte aligned");
  static_assert(PITCH >= 15 + 3 * (BX - 1) + 12, "a tap read (3 words from the pair's word) stays in its row");
  static_assert(BY >= TH + 1 && BX >= TW + 2, "the box holds an unscaled tile");
  static_assert(TH <= 32 && (TH & (TH - 1)) == 0, "lane r holds the coordinate of tile row r");
};
constexpr int RWARP = 4;              // warps per CTA

struct RImg {          // per-image values of a warp's current image (warp-uniform)
  int32_t b, prefix, ntiles, tiles_x;
  int32_t OH, OW, cw, ch, wx0, wy0;
  const uint8_t* src;
  uint8_t* dst;
  int64_t sstride, dstride;
};
struct RTile {         // geometry of one tile
  int32_t ox0, oy0, tw, th, bx0, by0, bw, bh, big;
};

template <int MAP>
ALB_D void r_load_img(const Plan& plan, const ImgList& in, const ImgList& out, const PrmList& prm, int32_t b,
                      RImg& k) {
  const alb_image si = in.get(b), so = out.get(b);
  const alb_params& p = prm.get(b);
  k.b = b; k.prefix = plan.prefix[b]; k.ntiles = plan.prefix[b + 1] - k.prefix; k.tiles_x = plan.rows_per_item[b];
  k.OH = so.h; k.OW = so.w;
  if (MAP == MAP_GRID) {
    k.cw = si.w; k.ch = si.h; k.wx0 = 0; k.wy0 = 0;
  } else {
    k.cw = p.cw; k.ch = p.ch; k.wx0 = p.x0; k.wy0 = p.y0;
  }
  k.src = (const uint8_t*)si.data; k.dst = (uint8_t*)so.data;
  k.sstride = si.row_stride; k.dstride = so.row_stride;
}

// Tile geometry; per lane: vcol[c] = Q5 coordinate of tile column
// lane + 32 c, vrow = that of tile row `lane` (lanes < TH), both clamped to
// the tile.
template <int MAP, int S>
ALB_D void r_tile_geo(const RImg& k, const PrmList& prm, int32_t item, int lane, RTile& g,
                      int32_t (&vcol)[RShape<S>::NC], int32_t& vrow) {
  using SH = RShape<S>;
  const int32_t t = item - k.prefix, ty = t / k.tiles_x, tx = t - ty * k.tiles_x;
  g.ox0 = tx * SH::TW; g.oy0 = ty * SH::TH;
  g.tw = imin(SH::TW, k.OW - g.ox0); g.th = imin(SH::TH, k.OH - g.oy0);
  const int32_t ry = g.oy0 + imin(lane & (SH::TH - 1), g.th - 1);
  if (MAP == MAP_GRID) {
    const alb_params& p = prm.get(k.b);            // the cell factors stay in the record
#pragma unroll
    for (int c = 0; c < SH::NC; c++) {
      const int32_t cx = g.ox0 + imin(lane + 32 * c, g.tw - 1);
      vcol[c] = p.apply ? grid_q5(p.q, p.k, 0, cx, k.cw) : 32 * cx;
    }
    vrow = p.apply ? grid_q5(p.q, p.k, 1, ry, k.ch) : 32 * ry;
  } else {
#pragma unroll
    for (int c = 0; c < SH::NC; c++) vcol[c] = rs_q5(g.ox0 + imin(lane + 32 * c, g.tw - 1), k.cw, k.OW);
    vrow = rs_q5(ry, k.ch, k.OH);
  }
  const int32_t last = g.tw - 1;
  const int32_t vl = (SH::NC > 1 && last >= 32) ? vcol[SH::NC - 1] : vcol[0];
  const int32_t c0 = __shfl_sync(0xffffffffu, vcol[0], 0), c1 = __shfl_sync(0xffffffffu, vl, last & 31);
  const int32_t r0 = __shfl_sync(0xffffffffu, vrow, 0), r1 = __shfl_sync(0xffffffffu, vrow, g.th - 1);
  g.bx0 = c0 >> 5; g.by0 = r0 >> 5;
  g.bw = imin((c1 >> 5) + 1, k.cw - 1) - g.bx0 + 1;
  g.bh = imin((r1 >> 5) + 1, k.ch - 1) - g.by0 + 1;
  g.big = g.bw > SH::BX || g.bh > SH::BY;
}

// Lane r (and r + 32) stages box row r: raw aligned 16-byte chunks;
// rowoff[r] = r * pitch + the row's byte phase.
template <int S>
ALB_D void r_tile_stage(const RImg& k, const RTile& g, int lane, uint8_t* box, int32_t* rowoff) {
  using SH = RShape<S>;
  if (g.big) return;
  const int span = 3 * g.bw;
  for (int r = lane; r < g.bh; r += 32) {
    const int sy = k.wy0 + g.by0 + r;            // by0 + bh - 1 <= ch - 1: inside the window
    const uintptr_t first = reinterpret_cast<uintptr_t>(k.src) + (uintptr_t)((int64_t)sy * k.sstride) +
                            (uintptr_t)(3 * (k.wx0 + g.bx0));
    const uintptr_t c0 = first & ~uintptr_t(15);
    const int ph = (int)(first - c0);
    rowoff[r] = r * SH::PITCH + ph;
    const int nch = (ph + span + 15) >> 4;
    uint8_t* d = box + r * SH::PITCH;
    const int64_t ib = (int64_t)(k.ch - 1 + k.wy0) * k.sstride + 3 * (int64_t)(k.cw + k.wx0);
    for (int j = 0; j < nch; j++)
      if (ALB_IN(bytes_within(reinterpret_cast<const void*>(c0 + 16 * j), 16, k.src, ib, 15) && r < SH::BY &&
                 16 * j + 16 <= SH::PITCH))
        cp_async16(d + 16 * j, reinterpret_cast<const void*>(c0 + 16 * j));
  }
}

// h of one tap row for the three channels: (32 - fx) p(ix) + fx p(ix + 1).
ALB_D void r_hrow(uint32_t lo, uint32_t hi, uint32_t wx, uint32_t (&h)[3]) {
  h[0] = __dp4a(__byte_perm(lo, hi, 0x0030), wx, 0u);
  h[1] = __dp4a(__byte_perm(lo, hi, 0x0041), wx, 0u);
  h[2] = __dp4a(__byte_perm(lo, hi, 0x0052), wx, 0u);
}

// the output pixel from the two tap rows' h, stored channel by channel
ALB_D void r_vert_store(const uint32_t (&ha)[3], const uint32_t (&hb)[3], uint32_t wy, bool store, uint8_t* od) {
  const uint32_t r = __dp2a_lo(__byte_perm(ha[0], hb[0], 0x5410), wy, 512u) >> 10;
  const uint32_t g = __dp2a_lo(__byte_perm(ha[1], hb[1], 0x5410), wy, 512u) >> 10;
  const uint32_t b = __dp2a_lo(__byte_perm(ha[2], hb[2], 0x5410), wy, 512u) >> 10;
  if (store) { od[0] = (uint8_t)r; od[1] = (uint8_t)g; od[2] = (uint8_t)b; }
}

// NC output columns per lane (lane, lane + 32): the per-row work that does not
// depend on the column (the row's Q5 coordinate, its box row offset, the
// advance test) is shared by the lane's columns.
template <int NC>
ALB_D void r_tile_compute(const RImg& k, const RTile& g, int lane, const int32_t (&vcol)[NC], int32_t vrow,
                          const uint8_t* __restrict__ box, const int32_t* __restrict__ rowoff) {
  uint32_t wx[NC];
  bool store[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) {
    wx[c] = (uint32_t)(32 + 255 * (vcol[c] & 31));    // (32 - fx) | fx << 8
    store[c] = lane + 32 * c < g.tw;
  }
  uint8_t* od = k.dst + (int64_t)g.oy0 * k.dstride + 3 * (int64_t)(g.ox0 + lane);
  uint32_t ha[NC][3], hb[NC][3];
#pragma unroll
  for (int c = 0; c < NC; c++)
#pragma unroll
    for (int j = 0; j < 3; j++) ha[c][j] = hb[c][j] = 0u;
  int32_t ia = -2;                                   // box row whose h is in ha (hb: the row below)
  auto vert = [&](int r, int32_t fy) {
    const uint32_t wy = (uint32_t)(32 + 255 * fy);
#pragma unroll
    for (int c = 0; c < NC; c++)
      r_vert_store(ha[c], hb[c], wy, store[c] && ALB_IN(g.oy0 + r < k.OH && g.ox0 + lane + 32 * c < k.OW),
                   od + 96 * c);
  };
  if (!g.big) {
    int32_t ocol[NC];
#pragma unroll
    for (int c = 0; c < NC; c++) ocol[c] = 3 * ((vcol[c] >> 5) - g.bx0);
    // h of box row i for every column of the lane (one row offset load)
    auto hrow = [&](int32_t i, uint32_t (&h)[NC][3]) {
      const bool iok = ALB_IN(i >= 0 && i < g.bh);
      const int32_t ro = iok ? rowoff[i] : 0;
#pragma unroll
      for (int c = 0; c < NC; c++) {
        uint32_t lo = 0u, hi = 0u;
        if (iok && ALB_IN(ocol[c] >= 0 && ocol[c] < 3 * g.bw)) taps_row(box, ro + ocol[c], lo, hi);
        r_hrow(lo, hi, wx[c], h[c]);
      }
    };
    // at a clamped bottom edge the row below the last tap row is not staged
    // and has weight fy = 0: the last staged row stands in for it
    const int32_t last = g.bh - 1;
    // the tap rows advance warp-uniformly: a row of h is computed only when
    // the top tap row moves (enlargements reuse it for the next output rows)
    for (int r = 0; r < g.th; r++, od += k.dstride) {
      const int32_t rq = __shfl_sync(0xffffffffu, vrow, r);
      const int32_t iy = (rq >> 5) - g.by0, fy = rq & 31;
      if (iy != ia) {                              // warp-uniform
        if (iy == ia + 1) {
#pragma unroll
          for (int c = 0; c < NC; c++)
#pragma unroll
            for (int j = 0; j < 3; j++) ha[c][j] = hb[c][j];
        } else {
          hrow(iy, ha);
        }
        hrow(imin(iy + 1, last), hb);
        ia = iy;
      }
      vert(r, fy);
    }
  } else {
    // footprint larger than the box: taps straight from the source window,
    // the pair (sx0, sx0 + 1) as aligned words (every word read holds a byte
    // of the pair); at the clamped last column (sx1 == sx0, weight fx = 0)
    // byte by byte
    int32_t sx0[NC], sx1[NC];
#pragma unroll
    for (int c = 0; c < NC; c++) {
      sx0[c] = k.wx0 + (vcol[c] >> 5);
      sx1[c] = k.wx0 + imin((vcol[c] >> 5) + 1, k.cw - 1);
    }
    auto hrow = [&](int32_t sy, uint32_t (&h)[NC][3]) {
      const uint8_t* row = k.src + (int64_t)sy * k.sstride;
#pragma unroll
      for (int c = 0; c < NC; c++) {
        uint32_t lo = 0u, hi = 0u;
        if (!ALB_IN(sy >= k.wy0 && sy < k.wy0 + k.ch && sx0[c] >= k.wx0 && sx1[c] < k.wx0 + k.cw &&
                    sx1[c] >= sx0[c])) {
        } else if (sx1[c] == sx0[c] + 1) {
          ldg_pair(row + 3 * sx0[c], lo, hi);
        } else {
          lo = (uint32_t)row[3 * sx0[c]] | ((uint32_t)row[3 * sx0[c] + 1] << 8) |
               ((uint32_t)row[3 * sx0[c] + 2] << 16) | ((uint32_t)row[3 * sx1[c]] << 24);
          hi = (uint32_t)row[3 * sx1[c] + 1] | ((uint32_t)row[3 * sx1[c] + 2] << 8);
        }
        r_hrow(lo, hi, wx[c], h[c]);
      }
    };
    for (int r = 0; r < g.th; r++, od += k.dstride) {
      const int32_t rq = __shfl_sync(0xffffffffu, vrow, r);
      const int32_t iy = rq >> 5, fy = rq & 31;
      if (iy != ia) {
        hrow(k.wy0 + iy, ha);
        hrow(k.wy0 + imin(iy + 1, k.ch - 1), hb);
        ia = iy;
      }
      vert(r, fy);
    }
  }
}

template <int S>
struct RShared {       // dynamic shared memory of k_resize_rows: one staging box per warp
  uint8_t box[RWARP][RShape<S>::BY * RShape<S>::PITCH + 16];   // +16: the last row's tap read past the staged bytes
  int32_t rowoff[RWARP][RShape<S>::BY];
};

template <int MAP, int S>
__global__ void __launch_bounds__(32 * RWARP) k_resize_rows(Plan plan, ImgList in, ImgList out, PrmList prm) {
  extern __shared__ __align__(16) uint8_t rs_dyn[];
  RShared<S>& sm = *reinterpret_cast<RShared<S>*>(rs_dyn);
  int32_t it0, it1;
  item_range(plan, it0, it1);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t item = it0 + w;
  if (item >= it1) return;
  RImg k;
  r_load_img<MAP>(plan, in, out, prm, item_image(plan, item), k);
  for (; item < it1; item += RWARP) {
    if (item >= k.prefix + k.ntiles) {
      int32_t b = k.b;
      while (item >= plan.prefix[b + 1]) b++;
      r_load_img<MAP>(plan, in, out, prm, b, k);
    }
    RTile g;
    int32_t ccol[RShape<S>::NC], crow;
    r_tile_geo<MAP, S>(k, prm, item, lane, g, ccol, crow);
    __syncwarp();
    r_tile_stage<S>(k, g, lane, sm.box[w], sm.rowoff[w]);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    r_tile_compute(k, g, lane, ccol, crow, sm.box[w], sm.rowoff[w]);
  }
}

// --------------------------------------------------------------- affine warp (RGB, bilinear)
// Rotate / ShiftScaleRotate on RGB images.  A warp owns a 32 x 20 output tile,
// lane j = output column j, and walks the tile's rows: the Q16 source
// coordinates of a lane advance by (q1, q4) per row, already offset to the
// tile's staged box and biased by the Q16 -> Q5 rounding constant.  The box
// (up to AB - 1 = 47 pixels each way: the whole tile at any angle for scales
// >= 0.9, whose footprint is at most 52 * 0.71 / 0.9 + 2 = 43 pixels)
// is staged per warp by cp.async, rows reflected at copy time, one buffer per
// warp with the image and tile state in registers (at most 85 registers: six
// CTAs, 24 warps per SM -- the kernel is latency-bound, so resident warps
// matter more than a second buffer; with one buffer a taller tile pays:
// 32 x 20 beat 32 x 12 by 4 %, 32 x 24 and 32 x 28 lost on Rotate); a per-row
// table holds row * pitch + byte
// phase, so a tap row's
// offset is one shared load.  Tiles whose box crosses the left/right image
// border stage the reflected column range in source order and map the two tap
// columns through the fold, reading a mirrored pair as the staged pair with
// its horizontal weights swapped; tiles whose footprint does not fit read
// their taps from global memory.
constexpr int AT_W = 32, AT_H = 20;   // output tile (columns x rows)
constexpr int AB = 48;                // staged box side (pixels)
constexpr int APITCH = 176;           // staged row pitch in bytes
constexpr int AWARP = 4;              // warps per CTA
static_assert(APITCH % 16 == 0, "cp.async destinations must be 16-byte aligned");
static_assert(APITCH >= 15 + 3 * (AB - 1) + 12, "a tap read (3 words from the pair's word) stays in its row");

struct AImg {          // per-image values of a warp's current image (warp-uniform)
  int32_t b, prefix, ntiles, tiles_x;
  int32_t H, W, OH, OW;
  int64_t q[6];
  const uint8_t* src;
  uint8_t* dst;
  int64_t sstride, dstride;
};
struct ATile {         // geometry of one tile
  int32_t ox0, oy0, tw, th;
  int32_t bx0, by0, bw, bh, ra, rb, mode;   // mode 0 inside, 1 crosses a left/right border, 2 too large
  int64_t X00, Y00;                          // Q16 source coordinates of the tile's pixel (0, 0)
};

ALB_D void a_load_img(const Plan& plan, const ImgList& in, const ImgList& out, const PrmList& prm, int32_t b,
                      AImg& k) {
  const alb_image si = in.get(b), so = out.get(b);
  const alb_params& p = prm.get(b);
  k.b = b; k.prefix = plan.prefix[b]; k.ntiles = plan.prefix[b + 1] - k.prefix; k.tiles_x = plan.rows_per_item[b];
  k.H = si.h; k.W = si.w; k.OH = so.h; k.OW = so.w;
  const bool app = p.apply != 0;
  k.q[0] = app ? p.q[0] : 65536; k.q[1] = app ? p.q[1] : 0; k.q[2] = app ? p.q[2] : 0;
  k.q[3] = app ? p.q[3] : 0; k.q[4] = app ? p.q[4] : 65536; k.q[5] = app ? p.q[5] : 0;
  k.src = (const uint8_t*)si.data; k.dst = (uint8_t*)so.data;
  k.sstride = si.row_stride; k.dstride = so.row_stride;
}

ALB_D void a_tile_geo(const AImg& k, int32_t item, ATile& g) {
  const int32_t t = item - k.prefix, ty = t / k.tiles_x, tx = t - ty * k.tiles_x;
  g.ox0 = tx * AT_W; g.oy0 = ty * AT_H;
  g.tw = imin(AT_W, k.OW - g.ox0); g.th = imin(AT_H, k.OH - g.oy0);
  g.X00 = k.q[0] * g.ox0 + k.q[1] * g.oy0 + k.q[2];
  g.Y00 = k.q[3] * g.ox0 + k.q[4] * g.oy0 + k.q[5];
  const int64_t dXx = k.q[0] * (g.tw - 1), dXy = k.q[1] * (g.th - 1), dYx = k.q[3] * (g.tw - 1), dYy = k.q[4] * (g.th - 1);
  const int64_t xmin = g.X00 + (dXx < 0 ? dXx : 0) + (dXy < 0 ? dXy : 0);
  const int64_t xmax = g.X00 + (dXx > 0 ? dXx : 0) + (dXy > 0 ? dXy : 0);
  const int64_t ymin = g.Y00 + (dYx < 0 ? dYx : 0) + (dYy < 0 ? dYy : 0);
  const int64_t ymax = g.Y00 + (dYx > 0 ? dYx : 0) + (dYy > 0 ? dYy : 0);
  // Q5 cells of the extreme coordinates, +1 for the second tap
  const int32_t bx0 = (int32_t)((xmin + 1024) >> 16), bx1 = (int32_t)((xmax + 1024) >> 16) + 1;
  const int32_t by0 = (int32_t)((ymin + 1024) >> 16), by1 = (int32_t)((ymax + 1024) >> 16) + 1;
  g.bx0 = bx0; g.by0 = by0; g.bw = bx1 - bx0 + 1; g.bh = by1 - by0 + 1;
  g.ra = bx0; g.rb = bx1; g.mode = 0;
  const int32_t W = k.W;
  if (g.bw > AB - 1 || g.bh > AB - 1) {
    g.mode = 2;
  } else if (bx0 < 0 || bx1 >= W) {
    // stage the real columns the box's columns reflect onto (one fold at most)
    int32_t lo, hi;
    const bool ok = W > 1 && bx0 > -W && bx1 < 2 * W - 1;
    if (bx0 < 0 && bx1 >= W) { lo = 0; hi = W - 1; }
    else if (bx0 < 0) { lo = bx1 < 0 ? -bx1 : 0; hi = imax(-bx0, bx1); }
    else { lo = bx0 > W - 1 ? 2 * (W - 1) - bx1 : imin(bx0, 2 * (W - 1) - bx1); hi = bx0 > W - 1 ? 2 * (W - 1) - bx0 : W - 1; }
    g.ra = lo; g.rb = hi;
    g.mode = ok && hi - lo + 1 <= AB - 1 ? 1 : 2;
  }
}
// reflect-101 of a column within one fold (|i| < n for i < 0, i <= 2 (n - 1) above)
ALB_D int32_t refl1(int32_t i, int32_t n) { return i < 0 ? -i : (i >= n ? 2 * (n - 1) - i : i); }

// The mapped tile as a convex parallelogram (box-relative pixel units, with
// the Q16 -> Q5 rounding bias): its y-range and its left and right chains.
// The least x over a horizontal band is the left chain at the band point
// nearest to the leftmost vertex (the chain is convex), and likewise on the
// right; the chains' slopes are computed once per tile.
struct AChains {
  float ymin, ymax;
  float xl, yl, kl_up, kl_dn;   // leftmost vertex; dx/dy of the chain above and below it
  float xr, yr, kr_up, kr_dn;   // rightmost vertex
};

ALB_D void a_chains(const AImg& k, const ATile& g, AChains& c) {
  // inside tiles span at most AB pixels, so every Q16 value here fits 32 bits
  // (64-bit integer to float conversions run on the slow double-precision pipe)
  const float s = 1.0f / 65536.0f;
  const float x0 = (float)(int32_t)(g.X00 + 1024 - 65536 * (int64_t)g.bx0) * s;
  const float y0 = (float)(int32_t)(g.Y00 + 1024 - 65536 * (int64_t)g.by0) * s;
  const float ux = (float)((int32_t)k.q[0] * (g.tw - 1)) * s, uy = (float)((int32_t)k.q[3] * (g.tw - 1)) * s;
  const float wx = (float)((int32_t)k.q[1] * (g.th - 1)) * s, wy = (float)((int32_t)k.q[4] * (g.th - 1)) * s;
  const float vx[4] = {x0, x0 + ux, x0 + ux + wx, x0 + wx}, vy[4] = {y0, y0 + uy, y0 + uy + wy, y0 + wy};
  // running extreme vertices as values (indexed arrays would live in local memory)
  float lx = vx[0], ly = vy[0], rx = vx[0], ry = vy[0];
  float tlx = vx[0], tly = vy[0], blx = vx[0], bly = vy[0], trx = vx[0], try_ = vy[0], brx = vx[0], bry = vy[0];
#pragma unroll
  for (int i = 1; i < 4; i++) {
    const float x = vx[i], y = vy[i];
    if (x < lx) { lx = x; ly = y; }
    if (x > rx) { rx = x; ry = y; }
    // top / bottom vertex, ties broken to the left (left chain) or right (right chain)
    if (y < tly || (y == tly && x < tlx)) { tlx = x; tly = y; }
    if (y > bly || (y == bly && x < blx)) { blx = x; bly = y; }
    if (y < try_ || (y == try_ && x > trx)) { trx = x; try_ = y; }
    if (y > bry || (y == bry && x > brx)) { brx = x; bry = y; }
  }
  c.ymin = tly; c.ymax = bly;
  c.xl = lx; c.yl = ly; c.xr = rx; c.yr = ry;
  c.kl_up = ly > tly ? (lx - tlx) / (ly - tly) : 0.0f;
  c.kl_dn = bly > ly ? (blx - lx) / (bly - ly) : 0.0f;
  c.kr_up = ry > try_ ? (rx - trx) / (ry - try_) : 0.0f;
  c.kr_dn = bry > ry ? (brx - rx) / (bry - ry) : 0.0f;
}

// x-extent [lo, hi] of the parallelogram inside the band [ya, yb]; lo > hi when they do not meet
ALB_D void a_band(const AChains& c, float ya, float yb, float& lo, float& hi) {
  const float y0 = fmaxf(ya, c.ymin), y1 = fminf(yb, c.ymax);
  if (y0 > y1) { lo = 1.0f; hi = 0.0f; return; }
  const float yl = fminf(fmaxf(c.yl, y0), y1), yr = fminf(fmaxf(c.yr, y0), y1);
  lo = fmaf(yl - c.yl, yl < c.yl ? c.kl_up : c.kl_dn, c.xl);
  hi = fmaf(yr - c.yr, yr < c.yr ? c.kr_up : c.kr_dn, c.xr);
}

ALB_D void a_tile_stage(const AImg& k, const ATile& g, int lane, uint8_t* box, int32_t* rowoff) {
  if (g.mode == 2) return;
  const int span = 3 * (g.rb - g.ra + 1);
  // inside tiles stage, per box row, only the columns that the tile's taps
  // can read: the mapped tile meets row r's band [r - 1, r + 1) of tap rows;
  // columns floor(x) and floor(x) + 1 of that extent, with a margin
  AChains ch;
  if (g.mode == 0) a_chains(k, g, ch);
  for (int r = lane; r < g.bh; r += 32) {
    const int32_t yr = g.by0 + r;
    int32_t ry = yr;
    if ((uint32_t)yr >= (uint32_t)k.H) {
      const int32_t t1 = refl1(yr, k.H);
      ry = (k.H > 1 && (uint32_t)t1 < (uint32_t)k.H) ? t1 : reflect101(yr, k.H);
    }
    const uintptr_t first = reinterpret_cast<uintptr_t>(k.src) + (uintptr_t)((int64_t)ry * k.sstride) +
                            (uintptr_t)(3 * g.ra);
    const uintptr_t c0 = first & ~uintptr_t(15);
    const int ph = (int)(first - c0);
    rowoff[r] = r * APITCH + ph;
    int j0 = 0, j1 = ((ph + span + 15) >> 4) - 1;
    if (g.mode == 0) {
      float lo, hi;
      a_band(ch, (float)r - 1.05f, (float)r + 1.05f, lo, hi);
      if (lo > hi) continue;                                   // no tap reads this row
      const int cl = imax((int)floorf(lo - 0.05f), 0), chh = imin((int)floorf(hi + 0.05f) + 1, g.bw - 1);
      if (cl > chh) continue;
      j0 = (ph + 3 * cl) >> 4;
      j1 = imin(j1, (ph + 3 * chh + 2) >> 4);
    }
    uint8_t* d = box + r * APITCH;
    const int64_t ib = (int64_t)(k.H - 1) * k.sstride + 3 * (int64_t)k.W;
    for (int j = j0; j <= j1; j++)
      if (ALB_IN(bytes_within(reinterpret_cast<const void*>(c0 + 16 * j), 16, k.src, ib, 15) && r < AB && j >= 0 &&
                 16 * j + 16 <= APITCH))
        cp_async16(d + 16 * j, reinterpret_cast<const void*>(c0 + 16 * j));
  }
}

// Q5 bilinear of one RGB pixel from the raw tap pairs of its two rows (lo =
// bytes 0..3, hi = bytes 4..5 of pixels (x, x + 1)): the pairs as {R0, R1, G0,
// G1} and {B0, B1} against the 16-bit weight pairs (wxp.lo wy, wxp.hi wy) of
// the top (wy = 32 - fy) and bottom (wy = fy) row, where wxp holds the
// horizontal weights of the first and second pixel; two dp2a per channel
// give sum w_ij p_ij + 512 exactly
ALB_D void a_bilerp(uint32_t tl, uint32_t th2, uint32_t bl, uint32_t bh2, uint32_t wxp, int32_t fy, uint32_t& vr,
                    uint32_t& vg, uint32_t& vb) {
  const uint32_t wt = wxp * (uint32_t)(32 - fy), wb = wxp * (uint32_t)fy;
  const uint32_t pt = __byte_perm(tl, th2, 0x4130), qt = __byte_perm(tl, th2, 0x0052);
  const uint32_t pb = __byte_perm(bl, bh2, 0x4130), qb = __byte_perm(bl, bh2, 0x0052);
  vr = __dp2a_lo(wt, pt, __dp2a_lo(wb, pb, 512u)) >> 10;
  vg = __dp2a_hi(wt, pt, __dp2a_hi(wb, pb, 512u)) >> 10;
  vb = __dp2a_lo(wt, qt, __dp2a_lo(wb, qb, 512u)) >> 10;
}

ALB_D void a_store3(uint8_t* od, uint32_t r, uint32_t g, uint32_t b) {
  od[0] = (uint8_t)r; od[1] = (uint8_t)g; od[2] = (uint8_t)b;
}

ALB_D void a_tile_compute(const AImg& k, const ATile& g, int lane, const uint8_t* __restrict__ box,
                          const int32_t* __restrict__ rowoff) {
  const int32_t col = imin(lane, g.tw - 1);             // lanes past the tile edge follow its last column
  const bool store = lane < g.tw;
  uint8_t* od = k.dst + (int64_t)g.oy0 * k.dstride + 3 * (int64_t)(g.ox0 + lane);
  const int32_t q1 = (int32_t)k.q[1], q4 = (int32_t)k.q[4];
  if (g.mode != 2) {
    // box-relative Q16 coordinates plus the Q16 -> Q5 rounding bias
    int32_t X = (int32_t)(g.X00 - 65536 * (int64_t)g.bx0) + (int32_t)k.q[0] * col + 1024;
    int32_t Y = (int32_t)(g.Y00 - 65536 * (int64_t)g.by0) + (int32_t)k.q[3] * col + 1024;
    if (g.mode == 0) {
#pragma unroll 2
      for (int r = 0; r < g.th; r++, X += q1, Y += q4, od += k.dstride) {
        const int32_t ix = X >> 16, fx = (X >> 11) & 31, iy = Y >> 16, fy = (Y >> 11) & 31;
        const int o = 3 * ix;
        uint32_t tl = 0u, th2 = 0u, bl = 0u, bh2 = 0u;
        if (ALB_IN(ix >= 0 && ix + 1 < g.bw && iy >= 0 && iy + 1 < g.bh)) {
          taps_row(box, rowoff[iy] + o, tl, th2);
          taps_row(box, rowoff[iy + 1] + o, bl, bh2);
        }
        uint32_t vr, vg, vb;
        a_bilerp(tl, th2, bl, bh2, 32u + 65535u * (uint32_t)fx, fy, vr, vg, vb);   // {32 - fx, fx}
        if (store && ALB_IN(g.oy0 + r < k.OH && g.ox0 + lane < k.OW)) a_store3(od, vr, vg, vb);
      }
    } else {
      // the box spans one fold at most: the two tap columns map through it with
      // one comparison each; a mirrored pair (x, x - 1) is the staged pair
      // (x - 1, x) with the horizontal weights swapped
      const int32_t W = k.W, span3 = 3 * (g.rb - g.ra);
      for (int r = 0; r < g.th; r++, X += q1, Y += q4, od += k.dstride) {
        const int32_t ix = X >> 16, fx = (X >> 11) & 31, iy = Y >> 16, fy = (Y >> 11) & 31;
        const int32_t xa = refl1(g.bx0 + ix, W), xb = refl1(g.bx0 + ix + 1, W);
        const bool swp = xb < xa;
        const int32_t o = 3 * ((swp ? xb : xa) - g.ra);
        uint32_t tl = 0u, th2 = 0u, bl = 0u, bh2 = 0u;
        if (ALB_IN(iy >= 0 && iy + 1 < g.bh && o >= 0 && o + 3 <= span3)) {
          taps_row(box, rowoff[iy] + o, tl, th2);
          taps_row(box, rowoff[iy + 1] + o, bl, bh2);
        }
        const uint32_t wxp = swp ? (32u << 16) - 65535u * (uint32_t)fx : 32u + 65535u * (uint32_t)fx;
        uint32_t vr, vg, vb;
        a_bilerp(tl, th2, bl, bh2, wxp, fy, vr, vg, vb);
        if (store && ALB_IN(g.oy0 + r < k.OH && g.ox0 + lane < k.OW)) a_store3(od, vr, vg, vb);
      }
    }
  } else {
    // footprint too large for the box: taps straight from global memory
    const int32_t W = k.W, H = k.H;
    int64_t X = g.X00 + k.q[0] * col + 1024, Y = g.Y00 + k.q[3] * col + 1024;
    for (int r = 0; r < g.th; r++, X += k.q[1], Y += k.q[4], od += k.dstride) {
      const int64_t xq = X >> 11, yq = Y >> 11;
      const int fx = (int)(xq & 31), fy = (int)(yq & 31);
      const int sx0 = reflect101(xq >> 5, W), sx1 = reflect101((xq >> 5) + 1, W);
      const int sy0 = reflect101(yq >> 5, H), sy1 = reflect101((yq >> 5) + 1, H);
      if (!ALB_IN(sx0 >= 0 && sx0 < W && sx1 >= 0 && sx1 < W && sy0 >= 0 && sy0 < H && sy1 >= 0 && sy1 < H)) continue;
      const int w11 = fx * fy, w01 = 32 * fx - w11, w10 = 32 * fy - w11, w00 = 1024 - 32 * fx - 32 * fy + w11;
      const uint8_t* ra = k.src + (int64_t)sy0 * k.sstride;
      const uint8_t* rbp = k.src + (int64_t)sy1 * k.sstride;
      uint32_t v[3];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const int acc = w00 * ra[3 * sx0 + c] + w01 * ra[3 * sx1 + c] + w10 * rbp[3 * sx0 + c] + w11 * rbp[3 * sx1 + c];
        v[c] = (uint32_t)((acc + 512) >> 10);
      }
      if (store && ALB_IN(g.oy0 + r < k.OH && g.ox0 + lane < k.OW)) a_store3(od, v[0], v[1], v[2]);
    }
  }
}

struct AShared {       // dynamic shared memory of k_warp_affine3: one staging box per warp
  uint8_t box[AWARP][AB * APITCH + 16];   // +16: the last row's tap read past the staged bytes
  int32_t rowoff[AWARP][AB];
};

__global__ void __launch_bounds__(32 * AWARP, 6) k_warp_affine3(Plan plan, ImgList in, ImgList out, PrmList prm) {
  extern __shared__ __align__(16) uint8_t aw_dyn[];
  AShared& sm = *reinterpret_cast<AShared*>(aw_dyn);
  int32_t it0, it1;
  item_range(plan, it0, it1);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t item = it0 + w;
  if (item >= it1) return;
  AImg k;
  a_load_img(plan, in, out, prm, item_image(plan, item), k);
  for (; item < it1; item += AWARP) {
    if (item >= k.prefix + k.ntiles) {
      int32_t b = k.b;
      while (item >= plan.prefix[b + 1]) b++;
      a_load_img(plan, in, out, prm, b, k);
    }
    ATile g;
    a_tile_geo(k, item, g);
    __syncwarp();
    a_tile_stage(k, g, lane, sm.box[w], sm.rowoff[w]);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    a_tile_compute(k, g, lane, sm.box[w], sm.rowoff[w]);
  }
}

// --------------------------------------------------------------- elastic (RGB, bilinear)
// A warp owns a 32 x 16 output tile, lane j = output column j.  The tile's
// lattice points (at most 10 x 6 for the densest lattice, S = 4) are drawn by
// the lanes into shared memory; per output pixel the displacement is the
// exact integer blend of its cell's four points, and the two tap pixels of
// each tap row are read as aligned words from global memory (L1-cached: the
// field is smooth, neighbouring lanes read neighbouring bytes), reflected
// per tap at the image border.
constexpr int ET_W = 32, ET_H = 16, EWARP = 4, ELAT = 64;

// the same pair format from two arbitrary (reflected) pixels
ALB_D void gather_pair(const uint8_t* row, int32_t xa, int32_t xb, uint32_t& lo, uint32_t& hi) {
  const uint8_t* a = row + 3 * (int64_t)xa;
  const uint8_t* b = row + 3 * (int64_t)xb;
  lo = (uint32_t)__ldg(a) | ((uint32_t)__ldg(a + 1) << 8) | ((uint32_t)__ldg(a + 2) << 16) | ((uint32_t)__ldg(b) << 24);
  hi = (uint32_t)__ldg(b + 1) | ((uint32_t)__ldg(b + 2) << 8);
}

__global__ void __launch_bounds__(32 * EWARP) k_elastic3(Plan plan, ImgList in, ImgList out, PrmList prm) {
  __shared__ int2 lat[EWARP][ELAT];
  int32_t it0, it1;
  item_range(plan, it0, it1);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t item = it0 + w;
  if (item >= it1) return;
  int32_t b = item_image(plan, item);
  for (; item < it1; item += EWARP) {
    while (item >= plan.prefix[b + 1]) b++;
    const alb_image si = in.get(b), so = out.get(b);
    const alb_params& p = prm.get(b);
    const int32_t t = item - plan.prefix[b], tiles_x = plan.rows_per_item[b];
    const int32_t ty = t / tiles_x, tx = t - ty * tiles_x;
    const int32_t ox0 = tx * ET_W, oy0 = ty * ET_H;
    const int32_t tw = imin(ET_W, so.w - ox0), th = imin(ET_H, so.h - oy0);
    const int32_t W = si.w, H = si.h;
    const bool act = p.apply != 0;
    const int sh = act ? p.cw : 2;
    const int32_t S = 1 << sh;
    const int32_t ci0 = oy0 >> sh, cj0 = ox0 >> sh;
    const int32_t ncols = ((ox0 + tw - 1) >> sh) + 2 - cj0;
    __syncwarp();                                     // the previous tile's reads of lat[w] are done
    if (act) {
      const int32_t nrows = ((oy0 + th - 1) >> sh) + 2 - ci0;
      const int32_t nx = ((W + S - 1) >> sh) + 1;
      for (int32_t k = lane; k < nrows * ncols; k += 32) {
        const int32_t r = k / ncols, c = k - r * ncols;
        int32_t dx, dy;
        elastic_point(p.q, p.k, (int64_t)(ci0 + r) * nx + cj0 + c, dx, dy);
        lat[w][k] = make_int2(dx, dy);
      }
    }
    __syncwarp();
    const int32_t x = ox0 + imin(lane, tw - 1);
    const int32_t cj = (x >> sh) - cj0, fx = x & (S - 1);
    const bool store = lane < tw;
    const uint8_t* __restrict__ src = (const uint8_t*)si.data;
    const int64_t ss = si.row_stride;
    uint8_t* od = (uint8_t*)so.data + (int64_t)oy0 * so.row_stride + 3 * (int64_t)(ox0 + lane);
    const int64_t SS = (int64_t)S * S;
    // per lane, the horizontal blends (S - fx) p_left + fx p_right of the two
    // lattice rows around the current output row, refreshed when the row of
    // lattice cells changes (warp-uniform); 32-bit when A S^2 fits
    const bool narrow = (int64_t)p.k * SS < (int64_t(1) << 30);
    int32_t crow = -1;
    int64_t hax = 0, hay = 0, hbx = 0, hby = 0;
    for (int r = 0; r < th; r++, od += so.row_stride) {
      const int32_t y = oy0 + r;
      int32_t X = 32 * x, Y = 32 * y;
      if (act) {
        const int32_t ci = (y >> sh) - ci0, fy = y & (S - 1);
        if (ci != crow && ALB_IN(ci >= 0 && cj >= 0 && cj + 1 < ncols && (ci + 1) * ncols + cj + 1 < ELAT)) {
          const int2 a = lat[w][ci * ncols + cj], bq = lat[w][ci * ncols + cj + 1];
          const int2 c = lat[w][(ci + 1) * ncols + cj], d = lat[w][(ci + 1) * ncols + cj + 1];
          hax = (int64_t)(S - fx) * a.x + (int64_t)fx * bq.x;
          hay = (int64_t)(S - fx) * a.y + (int64_t)fx * bq.y;
          hbx = (int64_t)(S - fx) * c.x + (int64_t)fx * d.x;
          hby = (int64_t)(S - fx) * c.y + (int64_t)fx * d.y;
          crow = ci;
        }
        // floor((sum + S^2 / 2) / S^2): S^2 is a power of two, an arithmetic shift floors
        if (narrow) {
          X += ((S - fy) * (int32_t)hax + fy * (int32_t)hbx + (int32_t)(SS / 2)) >> (2 * sh);
          Y += ((S - fy) * (int32_t)hay + fy * (int32_t)hby + (int32_t)(SS / 2)) >> (2 * sh);
        } else {
          X += (int32_t)(((int64_t)(S - fy) * hax + (int64_t)fy * hbx + SS / 2) >> (2 * sh));
          Y += (int32_t)(((int64_t)(S - fy) * hay + (int64_t)fy * hby + SS / 2) >> (2 * sh));
        }
      }
      const int32_t ix = X >> 5, fxq = X & 31, iy = Y >> 5, fyq = Y & 31;
      uint32_t tl, th2, bl, bh2;
      if (ix >= 0 && ix + 1 < W && iy >= 0 && iy + 1 < H) {
        const uint8_t* ra = src + (int64_t)iy * ss + 3 * (int64_t)ix;
        ldg_pair(ra, tl, th2);
        ldg_pair(ra + ss, bl, bh2);
      } else {
        const int32_t xa = reflect101(ix, W), xb = reflect101(ix + 1, W);
        gather_pair(src + (int64_t)reflect101(iy, H) * ss, xa, xb, tl, th2);
        gather_pair(src + (int64_t)reflect101(iy + 1, H) * ss, xa, xb, bl, bh2);
      }
      const uint32_t v = bilerp3(tl, th2, bl, bh2, fxq, fyq);
      if (store && ALB_IN(oy0 + r < so.h && ox0 + lane < so.w)) {
        od[0] = (uint8_t)v; od[1] = (uint8_t)(v >> 8); od[2] = (uint8_t)(v >> 16);
      }
    }
  }
}

// --------------------------------------------------------------- launcher
template <class... KArgs, class... Args>
static alb_status launch_k(void (*kern)(KArgs...), cudaStream_t st, Args... args) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * NWARP, 0);
  kern<<<(per_sm < 1 ? 1 : per_sm) * sm_count(), 32 * NWARP, 0, st>>>(args...);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

// Returns ALB_EINVAL (nothing launched) when no tiled kernel covers the case.
alb_status launch_tile_geometric(int32_t tid, const Plan& plan, const ImgList& in, const ImgList& out,
                                 const PrmList& prm, int32_t channels, bool mask, const PlanCheck& chk,
                                 cudaStream_t st) {
  const bool affine = tid == ALB_ROTATE || tid == ALB_SHIFT_SCALE_ROTATE;
  const bool resize = tid == ALB_RESIZE || tid == ALB_RANDOM_SIZED_CROP || tid == ALB_RANDOM_RESIZED_CROP;
  const bool grid = tid == ALB_GRID_DISTORTION;
  if (!affine && !resize && !grid && tid != ALB_ELASTIC) return ALB_EINVAL;
  if (!(channels == 3 && !mask) && !(channels == 1 && mask)) return ALB_EINVAL;
  // the row plan's arrays are rewritten as a tile plan (stream-ordered)
  int32_t* prefix = const_cast<int32_t*>(plan.prefix);
  int32_t* tiles_x = const_cast<int32_t*>(plan.rows_per_item);
  if ((resize || grid) && !mask) {
    // resizes with a second plan: three classes by the window's scale, each
    // through its own tile shape (see k_plan_tiles); the first plan's arrays
    // are rebuilt for the third class once the first class's kernel has read
    // them (stream order)
    const bool split = resize && plan.prefix2 && plan.rows2;
    auto run = [&](auto kern, int smem, const Plan& pl) -> alb_status {
      ALB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * RWARP, smem);
      kern<<<(per_sm < 1 ? 1 : per_sm) * sm_count(), 32 * RWARP, smem, st>>>(pl, in, out, prm);
      ALB_CUDA(cudaGetLastError());
      return ALB_OK;
    };
    auto tiles = [&](int tw, int th, int32_t* pf, int32_t* tx, int32_t cls) -> alb_status {
      PlanCheck c = chk;
      c.reduce = cls;
      k_plan_tiles<<<1, 1024, 0, st>>>(out, plan.n, tw, th, pf, tx, c);
      ALB_CUDA(cudaGetLastError());
      return ALB_OK;
    };
    alb_status rc;
    if (grid) {
      // grid distortion: cell factors up to ~1.9 stretch many tiles' footprints
      // past the small box, so every image takes the 66 x 34 box of the 32 x 16 tiles
      rc = tiles(RShape<1>::TW, RShape<1>::TH, prefix, tiles_x, 0);
      if (rc != ALB_OK) return rc;
      return run(k_resize_rows<MAP_GRID, 1>, (int)sizeof(RShared<1>), plan);
    }
    if (!split) {
      rc = tiles(RShape<2>::TW, RShape<2>::TH, prefix, tiles_x, 0);
      if (rc != ALB_OK) return rc;
      return run(k_resize_rows<MAP_RESIZE, 2>, (int)sizeof(RShared<2>), plan);
    }
    rc = tiles(RShape<0>::TW, RShape<0>::TH, prefix, tiles_x, 2);
    if (rc == ALB_OK) rc = run(k_resize_rows<MAP_RESIZE, 0>, (int)sizeof(RShared<0>), plan);
    if (rc == ALB_OK) rc = tiles(RShape<2>::TW, RShape<2>::TH, prefix, tiles_x, 3);
    if (rc == ALB_OK) rc = run(k_resize_rows<MAP_RESIZE, 2>, (int)sizeof(RShared<2>), plan);
    if (rc == ALB_OK) rc = tiles(RShape<1>::TW, RShape<1>::TH, plan.prefix2, plan.rows2, 1);
    if (rc != ALB_OK) return rc;
    const Plan p2{plan.prefix2, plan.rows2, plan.n};
    return run(k_resize_rows<MAP_RESIZE, 1>, (int)sizeof(RShared<1>), p2);
  }
  if (grid) return ALB_EINVAL;   // masks of a grid distortion: the general kernel
  if (tid == ALB_ELASTIC) {
    if (mask) return ALB_EINVAL;   // masks: the general kernel
    k_plan_tiles<<<1, 1024, 0, st>>>(out, plan.n, ET_W, ET_H, prefix, tiles_x, chk);
    ALB_CUDA(cudaGetLastError());
    return launch_k(k_elastic3, st, plan, in, out, prm);
  }
  if (affine && !mask) {
    k_plan_tiles<<<1, 1024, 0, st>>>(out, plan.n, AT_W, AT_H, prefix, tiles_x, chk);
    ALB_CUDA(cudaGetLastError());
    const int smem = (int)sizeof(AShared);
    ALB_CUDA(cudaFuncSetAttribute(k_warp_affine3, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_warp_affine3, 32 * AWARP, smem);
    k_warp_affine3<<<(per_sm < 1 ? 1 : per_sm) * sm_count(), 32 * AWARP, smem, st>>>(plan, in, out, prm);
    ALB_CUDA(cudaGetLastError());
    return ALB_OK;
  }
  // single-plane masks of the warps and resizes (RGB images returned above)
  k_plan_tiles<<<1, 1024, 0, st>>>(out, plan.n, WT, WT, prefix, tiles_x, chk);
  ALB_CUDA(cudaGetLastError());
  if (affine) return launch_k(k_resample_warp<MAP_AFFINE, true, 1>, st, plan, in, out, prm);
  return launch_k(k_resample_warp<MAP_RESIZE, true, 1>, st, plan, in, out, prm);
}

}  // namespace alb

namespace alb {
ALB_OOB_ACCESSOR(oob_resample)
}  // namespace alb
