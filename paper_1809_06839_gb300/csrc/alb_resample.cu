// alb_resample.cu -- tiled resampling for the transforms that move pixels along
// a continuous map: the affine warps (Table I: Rotate, ShiftScaleRotate) and
// the resizes (Sec. II-B "scaling"; Sec. II-A random sized crop), for images
// (Q5 bilinear) and their masks (nearest), with reflect-101 borders for warps.
//
// One work item = one 32 x 32 output tile.  The tile's source footprint (the
// bounding box of the mapped tile, plus the +1 tap) is staged into shared
// memory: 16-byte chunks of a box row that lie inside the image are copied
// with aligned 16-byte loads and a funnel-shift realignment; chunks that cross
// the image border are gathered byte by byte through the border map.  Each
// warp then computes an 8 x 4 output patch, whose taps cover a compact source
// region (few shared-memory bank conflicts), into an output tile in shared
// memory, which is written back with 16-byte stores.  Tiles whose footprint
// exceeds the staging box (scales below ~0.4) read their taps from global memory.
#include "alb_common.cuh"
#include "alb_kernels.cuh"
#include "alb_vec.cuh"

namespace alb {

constexpr int TW = 32, TH = 32;

// --------------------------------------------------------------- tile plan
__global__ void k_plan_tiles(ImgList out, int32_t n, int32_t* __restrict__ prefix, int32_t* __restrict__ tiles_x) {
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
      const int32_t tx = (im.w + TW - 1) / TW, ty = (im.h + TH - 1) / TH;
      cnt = im.h > 0 && im.w > 0 ? tx * ty : 0;
      tiles_x[i] = tx > 0 ? tx : 1;
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

enum { MAP_AFFINE = 0, MAP_RESIZE = 1 };

// Q5 bilinear from a byte grid (row pitch `pitch`, C = 3 channels), taps at
// byte offset o (ix, iy) and o + pitch: three aligned words per row, realigned.
ALB_D void taps_row(const uint8_t* base, int o, uint32_t& lo, uint32_t& hi) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(base + (o & ~3));
  const int s = 8 * (o & 3);
  const uint32_t w0 = w[0], w1 = w[1], w2 = w[2];
  lo = __funnelshift_r(w0, w1, s);
  hi = __funnelshift_r(w1, w2, s);
}

ALB_D uint32_t bilerp3(uint32_t t_lo, uint32_t t_hi, uint32_t b_lo, uint32_t b_hi, int fx, int fy) {
  const int w11 = fx * fy, w01 = 32 * fx - w11, w10 = 32 * fy - w11, w00 = 1024 - 32 * fx - 32 * fy + w11;
  // pixel 0 = bytes 0..2 of lo; pixel 1 = byte 3 of lo, bytes 0..1 of hi
  const int r = w00 * (int)(t_lo & 255) + w01 * (int)(t_lo >> 24) + w10 * (int)(b_lo & 255) + w11 * (int)(b_lo >> 24);
  const int g = w00 * (int)((t_lo >> 8) & 255) + w01 * (int)(t_hi & 255) + w10 * (int)((b_lo >> 8) & 255) +
                w11 * (int)(b_hi & 255);
  const int b = w00 * (int)((t_lo >> 16) & 255) + w01 * (int)((t_hi >> 8) & 255) + w10 * (int)((b_lo >> 16) & 255) +
                w11 * (int)((b_hi >> 8) & 255);
  return (uint32_t)((r + 512) >> 10) | ((uint32_t)((g + 512) >> 10) << 8) | ((uint32_t)((b + 512) >> 10) << 16);
}

// --------------------------------------------------------------- async copies
ALB_D void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
ALB_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
ALB_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Geometry of one tile (computed once per tile by thread 0 into shared memory).
struct TileGeo {
  int32_t b, ox0, oy0, tw, th;
  int32_t bx0, by0, bw, bh;     // footprint box (virtual source coordinates)
  int32_t ra, rb;               // staged real columns [ra, rb]
  int32_t mode;                 // 0 box inside the image, 1 box crosses a border, 2 box too large
  int32_t wx0, wy0, cw, ch;     // resize window
  int64_t X00, Y00;             // Q16 source coordinates of the tile's first pixel (affine)
};

constexpr int BOXR = 72;                   // staged rows (box height <= BOXR - 1)

template <int C>
struct Pitch {
  static constexpr int SROW = C == 3 ? 272 : 112;   // 68 / 28 words: successive rows start in different banks
  static constexpr int OROW = TW * C;
  static constexpr int BWMAX = C == 3 ? 79 : 79;    // box width limit (the +1 tap and the phase fit SROW)
};

// Per-image values the geometry thread needs, reloaded only when the image changes.
struct ImgCache {
  int32_t b;
  int32_t prefix, tiles_x, H, W, OH, OW, cw, ch, wx0, wy0;
  int64_t q[6];
};

template <int MAP>
ALB_D void cache_image(const Plan& plan, const ImgList& in, const ImgList& out, const PrmList& prm, int32_t b,
                       ImgCache& k) {
  const alb_image si = in.get(b), so = out.get(b);
  const alb_params& p = prm.get(b);
  k.b = b; k.prefix = plan.prefix[b]; k.tiles_x = plan.rows_per_item[b];
  k.H = si.h; k.W = si.w; k.OH = so.h; k.OW = so.w;
  k.cw = MAP == MAP_RESIZE ? p.cw : si.w; k.ch = MAP == MAP_RESIZE ? p.ch : si.h;
  k.wx0 = MAP == MAP_RESIZE ? p.x0 : 0; k.wy0 = MAP == MAP_RESIZE ? p.y0 : 0;
  const bool app = MAP == MAP_AFFINE && p.apply;
  k.q[0] = app ? p.q[0] : 65536; k.q[1] = app ? p.q[1] : 0; k.q[2] = app ? p.q[2] : 0;
  k.q[3] = app ? p.q[3] : 0; k.q[4] = app ? p.q[4] : 65536; k.q[5] = app ? p.q[5] : 0;
}

template <int MAP, bool NEAREST, int C>
ALB_D void tile_geometry(const ImgCache& k, int32_t item, TileGeo& g) {
  const int32_t t = item - k.prefix, ty = t / k.tiles_x, tx = t - ty * k.tiles_x;
  g.b = k.b; g.ox0 = tx * TW; g.oy0 = ty * TH;
  g.tw = imin(TW, k.OW - g.ox0); g.th = imin(TH, k.OH - g.oy0);
  const int32_t W = k.W;
  g.cw = k.cw; g.ch = k.ch; g.wx0 = k.wx0; g.wy0 = k.wy0;
  struct { int32_t w, h; } so{k.OW, k.OH};
  int32_t bx0, bx1, by0, by1;
  g.X00 = 0; g.Y00 = 0;
  if (MAP == MAP_AFFINE) {
    const int64_t q0 = k.q[0], q1 = k.q[1], q2 = k.q[2], q3 = k.q[3], q4 = k.q[4], q5 = k.q[5];
    g.X00 = q0 * g.ox0 + q1 * g.oy0 + q2;
    g.Y00 = q3 * g.ox0 + q4 * g.oy0 + q5;
    const int64_t dXx = q0 * (g.tw - 1), dXy = q1 * (g.th - 1), dYx = q3 * (g.tw - 1), dYy = q4 * (g.th - 1);
    const int64_t Xs[4] = {g.X00, g.X00 + dXx, g.X00 + dXy, g.X00 + dXx + dXy};
    const int64_t Ys[4] = {g.Y00, g.Y00 + dYx, g.Y00 + dYy, g.Y00 + dYx + dYy};
    int64_t xmin = Xs[0], xmax = Xs[0], ymin = Ys[0], ymax = Ys[0];
#pragma unroll
    for (int k = 1; k < 4; k++) {
      xmin = Xs[k] < xmin ? Xs[k] : xmin; xmax = Xs[k] > xmax ? Xs[k] : xmax;
      ymin = Ys[k] < ymin ? Ys[k] : ymin; ymax = Ys[k] > ymax ? Ys[k] : ymax;
    }
    if (NEAREST) {
      bx0 = (int32_t)((xmin + 32768) >> 16); bx1 = (int32_t)((xmax + 32768) >> 16);
      by0 = (int32_t)((ymin + 32768) >> 16); by1 = (int32_t)((ymax + 32768) >> 16);
    } else {
      bx0 = (int32_t)(((xmin + 1024) >> 11) >> 5); bx1 = (int32_t)(((xmax + 1024) >> 11) >> 5) + 1;
      by0 = (int32_t)(((ymin + 1024) >> 11) >> 5); by1 = (int32_t)(((ymax + 1024) >> 11) >> 5) + 1;
    }
  } else {
    if (NEAREST) {
      bx0 = rs_nn(g.ox0, g.cw, so.w); bx1 = rs_nn(g.ox0 + g.tw - 1, g.cw, so.w);
      by0 = rs_nn(g.oy0, g.ch, so.h); by1 = rs_nn(g.oy0 + g.th - 1, g.ch, so.h);
    } else {
      bx0 = rs_q5(g.ox0, g.cw, so.w) >> 5; bx1 = imin((rs_q5(g.ox0 + g.tw - 1, g.cw, so.w) >> 5) + 1, g.cw - 1);
      by0 = rs_q5(g.oy0, g.ch, so.h) >> 5; by1 = imin((rs_q5(g.oy0 + g.th - 1, g.ch, so.h) >> 5) + 1, g.ch - 1);
    }
  }
  g.bx0 = bx0; g.by0 = by0; g.bw = bx1 - bx0 + 1; g.bh = by1 - by0 + 1;
  g.ra = bx0; g.rb = bx1;
  g.mode = 0;
  if (g.bw > Pitch<C>::BWMAX || g.bh > BOXR - 1) {
    g.mode = 2;
  } else if (MAP == MAP_AFFINE && (bx0 < 0 || bx1 >= W)) {
    // border tile: stage the real columns the box's columns reflect onto (one
    // fold at most; boxes reaching further than one image width read globally)
    int32_t lo, hi;
    bool ok = W > 1 && bx0 > -W && bx1 < 2 * W - 1;
    if (bx0 < 0 && bx1 >= W) { lo = 0; hi = W - 1; }
    else if (bx0 < 0) { lo = bx1 < 0 ? -bx1 : 0; hi = imax(-bx0, bx1); }
    else { lo = bx0 > W - 1 ? 2 * (W - 1) - bx1 : imin(bx0, 2 * (W - 1) - bx1); hi = bx0 > W - 1 ? 2 * (W - 1) - bx0 : W - 1; }
    g.ra = lo; g.rb = hi;
    g.mode = ok && hi - lo + 1 <= Pitch<C>::BWMAX ? 1 : 2;
  }
}

// Issue the asynchronous copies of a tile's staged rows (raw aligned 16-byte
// chunks): warp w copies rows w, w + 8, ...; lane j copies chunk j of the row.
template <int MAP, int C>
ALB_D void tile_prefetch(const TileGeo& g, const alb_image& si, uint8_t* box, int16_t* phase) {
  if (g.mode == 2) return;
  const int lane = threadIdx.x & 31;
  const int span = C * (g.rb - g.ra + 1);
  for (int r = threadIdx.x >> 5; r < g.bh; r += blockDim.x >> 5) {
    const int vy = g.by0 + r;
    const int ry = MAP == MAP_AFFINE ? reflect101(vy, si.h) : g.wy0 + imin(vy, g.ch - 1);
    const uintptr_t first = reinterpret_cast<uintptr_t>(si.data) + (uintptr_t)((int64_t)ry * si.row_stride) +
                            (uintptr_t)(C * (g.wx0 + g.ra));
    const uintptr_t c0 = first & ~uintptr_t(15);
    const int ph = (int)(first - c0);
    if (lane == 0) phase[r] = (int16_t)ph;
    if (16 * lane < ph + span) cp_async16(box + r * Pitch<C>::SROW + 16 * lane, reinterpret_cast<const void*>(c0 + 16 * lane));
  }
}

template <int MAP, bool NEAREST, int C>
__global__ void __launch_bounds__(256) k_resample_tile(Plan plan, ImgList in, ImgList out, PrmList prm) {
  using PT = Pitch<C>;
  __shared__ __align__(16) uint8_t box[2][BOXR * PT::SROW];
  __shared__ __align__(16) uint8_t otile[TH * PT::OROW + 16];
  __shared__ int16_t phase[2][BOXR];
  __shared__ TileGeo geo[2];
  __shared__ int32_t colq[TW], rowq[TH];
  int32_t it0, it1;
  item_range(plan, it0, it1);
  if (it0 >= it1) return;
  int32_t bnext = item_image(plan, it0);
  // prologue: geometry + copies of the first tile
  __shared__ ImgCache kc;   // used by thread 0 only
  if (threadIdx.x == 0) {
    cache_image<MAP>(plan, in, out, prm, bnext, kc);
    tile_geometry<MAP, NEAREST, C>(kc, it0, geo[0]);
  }
  __syncthreads();
  tile_prefetch<MAP, C>(geo[0], in.get(bnext), box[0], phase[0]);
  cp_async_commit();
  int buf = 0;
  for (int32_t item = it0; item < it1; item++, buf ^= 1) {
    // geometry + copies of the next tile into the other buffer
    if (item + 1 < it1) {
      if (threadIdx.x == 0) {
        if (item + 1 >= kc.prefix + kc.tiles_x * ((kc.OH + TH - 1) / TH)) {   // next tile starts a new image
          while (item + 1 >= plan.prefix[bnext + 1]) bnext++;
          cache_image<MAP>(plan, in, out, prm, bnext, kc);
        }
        tile_geometry<MAP, NEAREST, C>(kc, item + 1, geo[buf ^ 1]);
      }
      __syncthreads();
      tile_prefetch<MAP, C>(geo[buf ^ 1], in.get(geo[buf ^ 1].b), box[buf ^ 1], phase[buf ^ 1]);
    }
    cp_async_commit();
    cp_async_wait<1>();          // this tile's copies have landed (the next tile's may be in flight)
    const TileGeo g = geo[buf];
    const alb_image si = in.get(g.b), so = out.get(g.b);
    const alb_params& p = prm.get(g.b);
    if (MAP == MAP_RESIZE) {
      if (threadIdx.x < TW) {
        const int x = g.ox0 + imin(threadIdx.x, g.tw - 1);
        colq[threadIdx.x] = NEAREST ? rs_nn(x, g.cw, so.w) : rs_q5(x, g.cw, so.w);
      } else if (threadIdx.x < TW + TH) {
        const int y = g.oy0 + imin(threadIdx.x - TW, g.th - 1);
        rowq[threadIdx.x - TW] = NEAREST ? rs_nn(y, g.ch, so.h) : rs_q5(y, g.ch, so.h);
      }
    }
    __syncthreads();
    const uint8_t* bx = box[buf];
    const int16_t* ph = phase[buf];
    const int32_t H = si.h, W = si.w;
    int64_t q0 = 65536, q1 = 0, q2 = 0, q3 = 0, q4 = 65536, q5 = 0;
    if (MAP == MAP_AFFINE && p.apply) { q0 = p.q[0]; q1 = p.q[1]; q2 = p.q[2]; q3 = p.q[3]; q4 = p.q[4]; q5 = p.q[5]; }
    const int32_t Xc = (int32_t)(g.X00 - 65536 * (int64_t)g.bx0), Yc = (int32_t)(g.Y00 - 65536 * (int64_t)g.by0);
    const uint8_t* __restrict__ src = (const uint8_t*)si.data;
    // thread = output column px, rows py = warp, warp + 8, ... (per-column terms once)
    const int px = threadIdx.x & 31, wy = threadIdx.x >> 5, ystep = blockDim.x >> 5;
    if (px < g.tw && g.mode != 2) {
      int32_t Xr = 0, Yr = 0, dX = 0, dY = 0, cq = 0;
      if (MAP == MAP_AFFINE) {
        Xr = Xc + (int32_t)q0 * px + (int32_t)q1 * wy;
        Yr = Yc + (int32_t)q3 * px + (int32_t)q4 * wy;
        dX = (int32_t)q1 * ystep; dY = (int32_t)q4 * ystep;
      } else {
        cq = NEAREST ? colq[px] - g.bx0 : colq[px] - 32 * g.bx0;
      }
      for (int py = wy; py < g.th; py += ystep, Xr += dX, Yr += dY) {
        uint8_t* od = otile + py * PT::OROW + C * px;
        int ix, iy, fx = 0, fy = 0;
        if (MAP == MAP_AFFINE) {
          if (NEAREST) { ix = (Xr + 32768) >> 16; iy = (Yr + 32768) >> 16; }
          else {
            const int xq = (Xr + 1024) >> 11, yq = (Yr + 1024) >> 11;
            ix = xq >> 5; fx = xq & 31; iy = yq >> 5; fy = yq & 31;
          }
        } else {
          if (NEAREST) { ix = cq; iy = rowq[py] - g.by0; }
          else {
            const int yq = rowq[py] - 32 * g.by0;
            ix = cq >> 5; fx = cq & 31; iy = yq >> 5; fy = yq & 31;
          }
        }
        const int o0 = iy * PT::SROW + ph[iy];
        if (NEAREST) {
          const int rx = g.mode == 1 ? reflect101(g.bx0 + ix, W) - g.ra : ix;
#pragma unroll
          for (int c = 0; c < C; c++) od[c] = bx[o0 + C * rx + c];
        } else if (g.mode == 0) {
          // the +1 row: at a resize's clamped bottom edge it is past the staged
          // rows and has weight fy = 0, so the last staged row stands in for it
          const int iy1 = iy + 1 < g.bh ? iy + 1 : iy;
          const int o1 = iy1 * PT::SROW + ph[iy1];
          uint32_t tl, th2, bl, bh2;
          taps_row(bx, o0 + 3 * ix, tl, th2);     // bx is 16-byte aligned: word alignment is that of the offset
          taps_row(bx, o1 + 3 * ix, bl, bh2);
          const uint32_t v = bilerp3(tl, th2, bl, bh2, fx, fy);
          od[0] = (uint8_t)v; od[1] = (uint8_t)(v >> 8); od[2] = (uint8_t)(v >> 16);
        } else {
          // border tile: taps through the reflect-101 column map
          const int o1 = (iy + 1) * PT::SROW + ph[iy + 1];
          const int xa = 3 * (reflect101(g.bx0 + ix, W) - g.ra), xb = 3 * (reflect101(g.bx0 + ix + 1, W) - g.ra);
          const int w11 = fx * fy, w01 = 32 * fx - w11, w10 = 32 * fy - w11, w00 = 1024 - 32 * fx - 32 * fy + w11;
#pragma unroll
          for (int c = 0; c < 3; c++) {
            const int acc = w00 * bx[o0 + xa + c] + w01 * bx[o0 + xb + c] + w10 * bx[o1 + xa + c] + w11 * bx[o1 + xb + c];
            od[c] = (uint8_t)((acc + 512) >> 10);
          }
        }
      }
    } else if (px < g.tw) {
      // footprint too large for the box: taps straight from global memory
      for (int py = wy; py < g.th; py += ystep) {
        uint8_t* od = otile + py * PT::OROW + C * px;
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
            sx0 = g.wx0 + rs_nn(x, g.cw, so.w); sy0 = g.wy0 + rs_nn(y, g.ch, so.h);
          } else {
            const int xq = rs_q5(x, g.cw, so.w), yq = rs_q5(y, g.ch, so.h);
            fx = xq & 31; fy = yq & 31;
            sx0 = g.wx0 + (xq >> 5); sx1 = g.wx0 + imin((xq >> 5) + 1, g.cw - 1);
            sy0 = g.wy0 + (yq >> 5); sy1 = g.wy0 + imin((yq >> 5) + 1, g.ch - 1);
          }
        }
        if (NEAREST) {
          const uint8_t* s0 = src + (int64_t)sy0 * si.row_stride + (int64_t)C * sx0;
#pragma unroll
          for (int c = 0; c < C; c++) od[c] = s0[c];
        } else {
          const int w11 = fx * fy, w01 = 32 * fx - w11, w10 = 32 * fy - w11, w00 = 1024 - 32 * fx - 32 * fy + w11;
          const uint8_t* ra = src + (int64_t)sy0 * si.row_stride;
          const uint8_t* rbp = src + (int64_t)sy1 * si.row_stride;
#pragma unroll
          for (int c = 0; c < C; c++) {
            const int acc = w00 * ra[3 * sx0 + c] + w01 * ra[3 * sx1 + c] + w10 * rbp[3 * sx0 + c] + w11 * rbp[3 * sx1 + c];
            od[c] = (uint8_t)((acc + 512) >> 10);
          }
        }
      }
    }
    __syncthreads();
    // ---- write the output tile: per row, aligned 16-byte chunks + edge bytes
    const int seg = C * g.tw;
    const int nch = (seg + 15) / 16 + 1;
    for (int i = threadIdx.x; i < g.th * nch; i += blockDim.x) {
      const int r = i / nch, j = i - r * nch;
      uint8_t* grow = (uint8_t*)so.data + (int64_t)(g.oy0 + r) * so.row_stride + (int64_t)C * g.ox0;
      const int pg = (int)(reinterpret_cast<uintptr_t>(grow) & 15);
      const int x = 16 * j - pg;
      const uint8_t* srow = otile + r * PT::OROW;
      if (x >= 0 && x + 16 <= seg) {
        const uint32_t* w = reinterpret_cast<const uint32_t*>(srow + (x & ~3));
        const int sh = 8 * (x & 3);
        const uint32_t a0 = w[0], a1 = w[1], a2 = w[2], a3 = w[3], a4 = (x & 3) ? w[4] : 0u;
        *reinterpret_cast<uint4*>(grow + x) =
            make_uint4(__funnelshift_r(a0, a1, sh), __funnelshift_r(a1, a2, sh), __funnelshift_r(a2, a3, sh),
                       __funnelshift_r(a3, a4, sh));
      } else {
        for (int kk = 0; kk < 16; kk++) {
          const int xx = x + kk;
          if (xx >= 0 && xx < seg) grow[xx] = srow[xx];
        }
      }
    }
    // the next iteration's first barrier orders this tile's reads of otile/box
    // before they are overwritten
  }
  cp_async_wait<0>();
}

// --------------------------------------------------------------- launcher
template <class... KArgs, class... Args>
static alb_status launch_k(void (*kern)(KArgs...), cudaStream_t st, Args... args) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
  kern<<<(per_sm < 1 ? 1 : per_sm) * sm_count(), 256, 0, st>>>(args...);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

// Returns ALB_EINVAL (nothing launched) when no tiled kernel covers the case.
alb_status launch_tile_geometric(int32_t tid, const Plan& plan, const ImgList& in, const ImgList& out,
                                 const PrmList& prm, int32_t channels, bool mask, cudaStream_t st) {
  const bool affine = tid == ALB_ROTATE || tid == ALB_SHIFT_SCALE_ROTATE;
  const bool resize = tid == ALB_RESIZE || tid == ALB_RANDOM_SIZED_CROP || tid == ALB_RANDOM_RESIZED_CROP;
  if (!affine && !resize) return ALB_EINVAL;
  if (!(channels == 3 && !mask) && !(channels == 1 && mask)) return ALB_EINVAL;
  // the row plan's arrays are rewritten as a tile plan (stream-ordered)
  int32_t* prefix = const_cast<int32_t*>(plan.prefix);
  int32_t* tiles_x = const_cast<int32_t*>(plan.rows_per_item);
  k_plan_tiles<<<1, 1024, 0, st>>>(out, plan.n, prefix, tiles_x);
  ALB_CUDA(cudaGetLastError());
  if (affine) {
    if (mask) return launch_k(k_resample_tile<MAP_AFFINE, true, 1>, st, plan, in, out, prm);
    return launch_k(k_resample_tile<MAP_AFFINE, false, 3>, st, plan, in, out, prm);
  }
  if (mask) return launch_k(k_resample_tile<MAP_RESIZE, true, 1>, st, plan, in, out, prm);
  return launch_k(k_resample_tile<MAP_RESIZE, false, 3>, st, plan, in, out, prm);
}

}  // namespace alb
