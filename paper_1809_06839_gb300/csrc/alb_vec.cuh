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
// realigned with funnel shifts.  NW = 4 (16 bytes) or 12 (48 bytes).
template <int NW>
ALB_D void load_window(const uint8_t* p, uint32_t (&out)[NW]) {
  constexpr int NC = NW / 4;                 // aligned chunks when p is aligned
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint4* q = reinterpret_cast<const uint4*>(a & ~uintptr_t(15));
  const int r = (int)(a & 15);
  uint32_t w[4 * NC + 4];
#pragma unroll
  for (int i = 0; i < NC; i++) {
    const uint4 v = __ldg(q + i);
    w[4 * i] = v.x; w[4 * i + 1] = v.y; w[4 * i + 2] = v.z; w[4 * i + 3] = v.w;
  }
  if (r == 0) {
#pragma unroll
    for (int i = 0; i < NW; i++) out[i] = w[i];
    return;
  }
  {
    const uint4 v = __ldg(q + NC);
    w[4 * NC] = v.x; w[4 * NC + 1] = v.y; w[4 * NC + 2] = v.z; w[4 * NC + 3] = v.w;
  }
  const int qq = r >> 2, s = (r & 3) * 8;
  uint32_t t1[4 * NC + 3];
#pragma unroll
  for (int i = 0; i < 4 * NC + 3; i++) t1[i] = (qq & 1) ? w[i + 1] : w[i];
  uint32_t t2[NW + 1];
#pragma unroll
  for (int i = 0; i < NW + 1; i++) t2[i] = (qq & 2) ? t1[i + 2] : t1[i];
#pragma unroll
  for (int i = 0; i < NW; i++) out[i] = __funnelshift_r(t2[i], t2[i + 1], s);
}

template <int NW>
ALB_D uint32_t byte_of(const uint32_t (&w)[NW], int i) {  // i: compile-time after unrolling
  return (w[i >> 2] >> (8 * (i & 3))) & 0xFFu;
}

}  // namespace alb
