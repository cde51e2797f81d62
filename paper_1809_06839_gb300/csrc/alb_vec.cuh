// alb_vec.cuh -- 16-byte vector helpers for packed uint8 RGB streams.
#pragma once

#include "alb_common.cuh"

namespace alb {

// A packed image whose rows are contiguous (row_stride == w*c) and whose base
// is 16-byte aligned: its bytes form one flat, aligned array.
ALB_D bool flat_aligned(const alb_image& a) {
  return a.row_stride == (int64_t)a.w * a.c && ((reinterpret_cast<uintptr_t>(a.data) & 15) == 0);
}

ALB_D uint4 ldg16(const uint8_t* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }
ALB_D void stg16(uint8_t* p, uint4 v) { *reinterpret_cast<uint4*>(p) = v; }

// Bytes [p, p + 4*NW) for an arbitrary p, read with aligned 16-byte loads of
// the chunks that hold them (never a chunk without a needed byte) and
// realigned with funnel shifts.  NW = 4 (16 bytes) or 12 (48 bytes).  Split
// in two halves so that a loop can issue the loads of its next unit (raw_load)
// before it realigns and uses the current one (raw_align).
template <int NW>
struct RawWin {
  uint32_t w[NW + 4];
  int r;          // byte phase of p within its 16-byte chunk
};

template <int NW>
ALB_D void raw_load(const uint8_t* p, RawWin<NW>& rw) {
  constexpr int NC = NW / 4;                 // aligned chunks when p is aligned
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint4* q = reinterpret_cast<const uint4*>(a & ~uintptr_t(15));
  rw.r = (int)(a & 15);
#pragma unroll
  for (int i = 0; i < NC; i++) {
    const uint4 v = __ldg(q + i);
    rw.w[4 * i] = v.x; rw.w[4 * i + 1] = v.y; rw.w[4 * i + 2] = v.z; rw.w[4 * i + 3] = v.w;
  }
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (rw.r) v = __ldg(q + NC);
  rw.w[4 * NC] = v.x; rw.w[4 * NC + 1] = v.y; rw.w[4 * NC + 2] = v.z; rw.w[4 * NC + 3] = v.w;
}

template <int NW>
ALB_D void raw_align(const RawWin<NW>& rw, uint32_t (&out)[NW]) {
  constexpr int NC = NW / 4;
  const int qq = rw.r >> 2, s = (rw.r & 3) * 8;
  uint32_t t1[4 * NC + 3];
#pragma unroll
  for (int i = 0; i < 4 * NC + 3; i++) t1[i] = (qq & 1) ? rw.w[i + 1] : rw.w[i];
  uint32_t t2[NW + 1];
#pragma unroll
  for (int i = 0; i < NW + 1; i++) t2[i] = (qq & 2) ? t1[i + 2] : t1[i];
#pragma unroll
  for (int i = 0; i < NW; i++) out[i] = __funnelshift_r(t2[i], t2[i + 1], s);
}

template <int NW>
ALB_D void load_window(const uint8_t* p, uint32_t (&out)[NW]) {
  RawWin<NW> rw;
  raw_load<NW>(p, rw);
  raw_align<NW>(rw, out);
}

// Three aligned 16-byte vectors (one 48-byte unit of 16 RGB pixels).
struct U48 {
  uint4 v0, v1, v2;
};
ALB_D void ld48(const uint8_t* p, U48& u) { u.v0 = ldg16(p); u.v1 = ldg16(p + 16); u.v2 = ldg16(p + 32); }
ALB_D void st48(uint8_t* p, const uint32_t (&o)[12]) {
  stg16(p, make_uint4(o[0], o[1], o[2], o[3]));
  stg16(p + 16, make_uint4(o[4], o[5], o[6], o[7]));
  stg16(p + 32, make_uint4(o[8], o[9], o[10], o[11]));
}
ALB_D void words48(const U48& u, uint32_t (&w)[12]) {
  w[0] = u.v0.x; w[1] = u.v0.y; w[2] = u.v0.z; w[3] = u.v0.w;
  w[4] = u.v1.x; w[5] = u.v1.y; w[6] = u.v1.z; w[7] = u.v1.w;
  w[8] = u.v2.x; w[9] = u.v2.y; w[10] = u.v2.z; w[11] = u.v2.w;
}

// Row and column of flat pixel index p in an image `w` pixels wide.
ALB_D void flat_rc(int64_t p, int32_t w, int32_t& y, int32_t& x) {
  if (p < (int64_t(1) << 32)) {
    y = (int32_t)((uint32_t)p / (uint32_t)w);
  } else {
    y = (int32_t)(p / w);
  }
  x = (int32_t)(p - (int64_t)y * w);
}

template <int NW>
ALB_D uint32_t byte_of(const uint32_t (&w)[NW], int i) {  // i: compile-time after unrolling
  return (w[i >> 2] >> (8 * (i & 3))) & 0xFFu;
}

}  // namespace alb
