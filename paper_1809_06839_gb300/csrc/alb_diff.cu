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
// Input adjoint of the warp: each output sample scatters g * weight to its four
// taps with fire-and-forget atomic adds (red.global.add.f32); parameter
// gradients: per-CTA block reductions written to a partials buffer and reduced
// by one CTA per image in a fixed order (deterministic).
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
// one thread per output pixel (all channels); blocks of 256 over H*W, grid.y = B
__global__ void __launch_bounds__(256) k_warp_f32_fwd(int B, int C, int H, int W, const float* __restrict__ x,
                                                      const float* __restrict__ prm, float* __restrict__ y) {
  const int b = blockIdx.y;
  __shared__ WarpF sg;
  if (threadIdx.x == 0) sg = warp_setup(prm, b, H, W);
  __syncthreads();
  const WarpF g = sg;
  const int64_t plane = (int64_t)H * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x) {
    const int oy = (int)(i / W), ox = (int)(i - (int64_t)oy * W);
    const float sx = __fmaf_rn(g.a00, (float)ox, __fmaf_rn(g.a01, (float)oy, g.b0));
    const float sy = __fmaf_rn(g.a10, (float)ox, __fmaf_rn(g.a11, (float)oy, g.b1));
    const float fx0 = floorf(sx), fy0 = floorf(sy);
    const float fx = sx - fx0, fy = sy - fy0;
    const int ix = (int)fx0, iy = (int)fy0;
    const float w00 = (1.0f - fx) * (1.0f - fy), w10 = fx * (1.0f - fy), w01 = (1.0f - fx) * fy, w11 = fx * fy;
    for (int c = 0; c < C; c++) {
      const float* img = x + ((int64_t)b * C + c) * plane;
      const float v = w00 * tapf(img, H, W, ix, iy) + w10 * tapf(img, H, W, ix + 1, iy) +
                      w01 * tapf(img, H, W, ix, iy + 1) + w11 * tapf(img, H, W, ix + 1, iy + 1);
      y[((int64_t)b * C + c) * plane + i] = v;
    }
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

__global__ void __launch_bounds__(256) k_warp_f32_bwd(int B, int C, int H, int W, const float* __restrict__ x,
                                                      const float* __restrict__ prm, const float* __restrict__ gy,
                                                      float* __restrict__ gx, float* __restrict__ partials) {
  const int b = blockIdx.y;
  __shared__ WarpF sg;
  __shared__ float red[32];
  if (threadIdx.x == 0) sg = warp_setup(prm, b, H, W);
  __syncthreads();
  const WarpF g = sg;
  const int64_t plane = (int64_t)H * W;
  float dth = 0.f, dsc = 0.f, dtx = 0.f, dty = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x) {
    const int oy = (int)(i / W), ox = (int)(i - (int64_t)oy * W);
    const float sx = __fmaf_rn(g.a00, (float)ox, __fmaf_rn(g.a01, (float)oy, g.b0));
    const float sy = __fmaf_rn(g.a10, (float)ox, __fmaf_rn(g.a11, (float)oy, g.b1));
    const float fx0 = floorf(sx), fy0 = floorf(sy);
    const float fx = sx - fx0, fy = sy - fy0;
    const int ix = (int)fx0, iy = (int)fy0;
    const bool in00 = ix >= 0 && ix < W && iy >= 0 && iy < H;
    const bool in10 = ix + 1 >= 0 && ix + 1 < W && iy >= 0 && iy < H;
    const bool in01 = ix >= 0 && ix < W && iy + 1 >= 0 && iy + 1 < H;
    const bool in11 = ix + 1 >= 0 && ix + 1 < W && iy + 1 >= 0 && iy + 1 < H;
    float dsx = 0.f, dsy = 0.f;
    for (int c = 0; c < C; c++) {
      const int64_t base = ((int64_t)b * C + c) * plane;
      const float gw = __ldg(gy + base + i);
      if (gw == 0.0f) continue;
      const float* img = x + base;
      float* dimg = gx + base;
      const float v00 = tapf(img, H, W, ix, iy), v10 = tapf(img, H, W, ix + 1, iy);
      const float v01 = tapf(img, H, W, ix, iy + 1), v11 = tapf(img, H, W, ix + 1, iy + 1);
      if (in00) atomicAdd(dimg + (int64_t)iy * W + ix, gw * (1.0f - fx) * (1.0f - fy));
      if (in10) atomicAdd(dimg + (int64_t)iy * W + ix + 1, gw * fx * (1.0f - fy));
      if (in01) atomicAdd(dimg + (int64_t)(iy + 1) * W + ix, gw * (1.0f - fx) * fy);
      if (in11) atomicAdd(dimg + (int64_t)(iy + 1) * W + ix + 1, gw * fx * fy);
      dsx += gw * ((1.0f - fy) * (v10 - v00) + fy * (v11 - v01));
      dsy += gw * ((1.0f - fx) * (v01 - v00) + fx * (v11 - v10));
    }
    const float xp = (float)ox - g.cx - g.txp, yp = (float)oy - g.cy - g.typ;
    dth += dsx * ((-g.sn * xp - g.cs * yp) / g.s) + dsy * ((g.cs * xp - g.sn * yp) / g.s);
    dsc += dsx * (-(sx - g.cx) / g.s) + dsy * (-(sy - g.cy) / g.s);
    dtx += dsx * (-g.cs * g.W / g.s) + dsy * (-g.sn * g.W / g.s);
    dty += dsx * (g.sn * g.H / g.s) + dsy * (-g.cs * g.H / g.s);
  }
  const float r0 = block_sum(dth, red), r1 = block_sum(dsc, red), r2 = block_sum(dtx, red), r3 = block_sum(dty, red);
  if (threadIdx.x == 0) {
    float* pp = partials + ((int64_t)b * gridDim.x + blockIdx.x) * 4;
    pp[0] = r0 * (float)(3.14159265358979323846 / 180.0);
    pp[1] = r1; pp[2] = r2; pp[3] = r3;
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
__global__ void __launch_bounds__(256) k_photo_f32_fwd(int B, int C, int H, int W, const float* __restrict__ x,
                                                       const float* __restrict__ prm, float* __restrict__ y) {
  const int b = blockIdx.y;
  const float al = prm[3 * b], be = prm[3 * b + 1], ga = prm[3 * b + 2];
  const int64_t n = (int64_t)C * H * W;
  const float* xb = x + (int64_t)b * n;
  float* yb = y + (int64_t)b * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float z = __fmaf_rn(al, __ldg(xb + i), be);
    const float zc = fminf(fmaxf(z, 0.0f), 1.0f);
    yb[i] = zc > 0.0f ? powf(zc, ga) : 0.0f;
  }
}

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
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float xv = __ldg(xb + i), g = __ldg(gb + i);
    const float z = __fmaf_rn(al, xv, be);
    float gxv = 0.0f;
    if (z > 0.0f && z < 1.0f) {
      const float lz = logf(z);
      const float zg = expf(ga * lz);                 // z^gamma
      const float gz = g * ga * expf((ga - 1.0f) * lz);  // g * gamma * z^(gamma-1)
      dg += g * zg * lz;
      da += gz * xv;
      db += gz;
      gxv = gz * al;
    }
    dxb[i] = gxv;
  }
  const float r0 = block_sum(da, red), r1 = block_sum(db, red), r2 = block_sum(dg, red);
  if (threadIdx.x == 0) {
    float* pp = partials + ((int64_t)b * gridDim.x + blockIdx.x) * 3;
    pp[0] = r0; pp[1] = r1; pp[2] = r2;
  }
}

static int blocks_per_image(int64_t elems, int B) {
  const int64_t want = (int64_t)sm_count() * 8;
  int64_t per = (want + B - 1) / B;
  const int64_t cap = (elems + 255) / 256;
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

extern "C" alb_status alb_warp_affine_f32_fwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                              const float* prm, float* y, void* stream) {
  alb_status rc = check_f32(B, C, H, W, x, prm, y);
  if (rc != ALB_OK || B == 0) return rc;
  dim3 grid(blocks_per_image((int64_t)H * W, B), B);
  k_warp_f32_fwd<<<grid, 256, 0, (cudaStream_t)stream>>>(B, C, H, W, x, prm, y);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

extern "C" alb_status alb_warp_affine_f32_bwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                              const float* prm, const float* gy, float* gx, float* gprm,
                                              void* workspace, size_t workspace_bytes, void* stream) {
  alb_status rc = check_f32(B, C, H, W, x, prm, gy);
  if (rc != ALB_OK || B == 0) return rc;
  ALB_REQUIRE(gx && gprm, ALB_EINVAL, "alb_warp_affine_f32_bwd: null output");
  const int nblk = blocks_per_image((int64_t)H * W, B);
  ALB_REQUIRE(workspace && workspace_bytes >= (size_t)B * nblk * 4 * sizeof(float), ALB_EWORKSPACE,
              "alb_warp_affine_f32_bwd: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  ALB_CUDA(cudaMemsetAsync(gx, 0, (size_t)B * C * H * W * sizeof(float), st));
  k_warp_f32_bwd<<<dim3(nblk, B), 256, 0, st>>>(B, C, H, W, x, prm, gy, gx, (float*)workspace);
  ALB_CUDA(cudaGetLastError());
  k_reduce_partials<<<B, 256, 0, st>>>(nblk, 4, (const float*)workspace, gprm);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

extern "C" alb_status alb_photometric_f32_fwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                              const float* prm, float* y, void* stream) {
  alb_status rc = check_f32(B, C, H, W, x, prm, y);
  if (rc != ALB_OK || B == 0) return rc;
  dim3 grid(blocks_per_image((int64_t)C * H * W, B), B);
  k_photo_f32_fwd<<<grid, 256, 0, (cudaStream_t)stream>>>(B, C, H, W, x, prm, y);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

extern "C" alb_status alb_photometric_f32_bwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                              const float* prm, const float* gy, float* gx, float* gprm,
                                              void* workspace, size_t workspace_bytes, void* stream) {
  alb_status rc = check_f32(B, C, H, W, x, prm, gy);
  if (rc != ALB_OK || B == 0) return rc;
  ALB_REQUIRE(gx && gprm, ALB_EINVAL, "alb_photometric_f32_bwd: null output");
  const int nblk = blocks_per_image((int64_t)C * H * W, B);
  ALB_REQUIRE(workspace && workspace_bytes >= (size_t)B * nblk * 3 * sizeof(float), ALB_EWORKSPACE,
              "alb_photometric_f32_bwd: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  k_photo_f32_bwd<<<dim3(nblk, B), 256, 0, st>>>(B, C, H, W, x, prm, gy, gx, (float*)workspace);
  ALB_CUDA(cudaGetLastError());
  k_reduce_partials<<<B, 256, 0, st>>>(nblk, 3, (const float*)workspace, gprm);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}
