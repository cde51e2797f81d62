// alb_distort.cuh -- Philox4x32-10 block function and the coordinate maps of
// the non-rigid distortions (Sec. II-C: grid distortion and elastic transform
// for medical images), shared by the sampler, the plan checks and the kernels.
//
// Grid distortion: each axis of n samples is cut into G equal output cells;
// cell i keeps a factor d_i (Q14 integers in the record: slot j of q[j / 4]
// bits 16 (j % 4), x cells in slots 0..11, y cells in 12..23).  The source
// cells have widths proportional to d_i and span the same [0, n - 1], so
// the source coordinate of output sample x in cell i = min(G - 1,
// floor(G x / (n - 1))) is the exact rational ((n - 1) P_i + (G x - i (n - 1))
// d_i) / D (P_i = sum of the factors before cell i, D = their total), taken
// to Q5 with round half up.
//
// Elastic transform: lattice points every S = 2^s pixels (ceil(W / S) + 1 per
// row) carry integer Q5 displacements in [-A, A]; point t uses the Philox
// block with counter (t, image index, stream lo, stream hi ^ 2^31) and key =
// seed (both from the record's q[0..2]): dx = floor(w0 (2A + 1) / 2^32) - A,
// dy likewise from w1.  A pixel's displacement blends its cell's four points
// with integer bilinear weights, rounded half up.
#pragma once

#include "alb_common.cuh"

namespace alb {

ALB_HD void philox_block(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                         uint32_t out[4]) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t a = (uint64_t)0xD2511F53u * c0;
    uint64_t b = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(b >> 32) ^ c1 ^ k0;
    uint32_t n2 = (uint32_t)(a >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)b;
    c3 = (uint32_t)a;
    c0 = n0;
    c2 = n2;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}


constexpr int kGridMaxCells = 12;

ALB_HD int32_t grid_factor(const int64_t q[6], int slot) {
  return (int32_t)(((uint64_t)q[slot >> 2] >> (16 * (slot & 3))) & 0xFFFFu);
}

// Q5 source coordinate of output sample x on axis 0 (x) or 1 (y) of n samples
ALB_HD int32_t grid_q5(const int64_t q[6], int32_t g, int axis, int32_t x, int32_t n) {
  if (n <= 1) return 0;
  int64_t D = 0, P = 0, di = 0;
  int32_t i = (int32_t)(((int64_t)g * x) / (n - 1));
  if (i > g - 1) i = g - 1;
  for (int j = 0; j < g; j++) {
    const int64_t d = grid_factor(q, 12 * axis + j);
    D += d;
    if (j < i) P += d;
    if (j == i) di = d;
  }
  const int64_t N = (int64_t)(n - 1) * P + ((int64_t)g * x - (int64_t)i * (n - 1)) * di;
  int64_t xq = floor_div(64 * N + D, 2 * D);
  if (xq < 0) xq = 0;
  if (xq > 32 * (int64_t)(n - 1)) xq = 32 * (int64_t)(n - 1);
  return (int32_t)xq;
}

// Output edge coordinate of source edge coordinate e (boxes): the inverse of
// the unquantised cell map between the first and last pixel centres (both
// fixed points); the outer half pixels map to themselves.  float64, in the
// operation order of the definition.
ALB_HD double grid_edge_inverse(const int64_t q[6], int32_t g, int axis, double e, int32_t n) {
  if (n <= 1) return e;
  double d[kGridMaxCells], c[kGridMaxCells + 1], D = 0.0;
  for (int j = 0; j < g; j++) { d[j] = (double)grid_factor(q, 12 * axis + j); D += d[j]; }
  double P = 0.0;
  for (int j = 0; j <= g; j++) { c[j] = (double)(n - 1) * P / D; if (j < g) P += d[j]; }
  const double t = e - 0.5;
  if (t <= 0.0 || t >= (double)(n - 1)) return e;
  int i = 0;
  while (i < g - 1 && t >= c[i + 1]) i++;
  double Pi = 0.0;
  for (int j = 0; j < i; j++) Pi += d[j];
  const double x = (D * t - (double)(n - 1) * Pi) / ((double)g * d[i]) + (double)i * (double)(n - 1) / (double)g;
  return x + 0.5;
}

// Q5 displacement (dx, dy) of lattice point t of an elastic record
ALB_HD void elastic_point(const int64_t q[6], int32_t amp, int64_t t, int32_t& dx, int32_t& dy) {
  const uint64_t seed = (uint64_t)q[0], sid = (uint64_t)q[1];
  uint32_t o[4];
  philox_block((uint32_t)t, (uint32_t)q[2], (uint32_t)sid, (uint32_t)(sid >> 32) ^ 0x80000000u, (uint32_t)seed,
               (uint32_t)(seed >> 32), o);
  const uint64_t span = 2 * (uint64_t)amp + 1;
  dx = (int32_t)((o[0] * span) >> 32) - amp;
  dy = (int32_t)((o[1] * span) >> 32) - amp;
}

}  // namespace alb
