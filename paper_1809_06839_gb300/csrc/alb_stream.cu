// alb_stream.cu -- streaming kernels for the transforms that touch each output
// byte once with a fixed source byte (Table I: HorizontalFlip, VerticalFlip,
// RandomCrop, PadToSize, Brightness, ShiftRGB, Gamma, Grayscale, ShiftHSV;
// Sec. II contrast; per-channel equalisation).
//
// Memory path: every warp moves whole 16-byte vectors.  Contiguous, 16-byte
// aligned images (the common case) are processed as one flat byte array:
// per-byte ops in 16-byte chunks, per-pixel ops in 48-byte units (16 RGB
// pixels, 3 vectors, always 16-byte aligned in the flat array).  Row-based
// copies (vertical flip, crop, pad interior) use per-row 16-byte output chunks
// whose source window, misaligned by a per-row constant, is read with aligned
// loads and realigned with funnel shifts.  Strided images and the bytes at row
// and item edges take a per-byte path.
#include "alb_common.cuh"
#include "alb_kernels.cuh"
#include "alb_vec.cuh"
#include "alb_bulk.cuh"

namespace alb {

// ================================================================== LUT ops
// Tables in shared memory, 32 copies interleaved so that lane l always reads
// bank l: byte v of channel c for lane l lives at c*8192 + (v & ~3)*32 + 4l + (v & 3).
constexpr int kLutBytes = 3 * 8192;

__device__ void build_lut_copies(const uint8_t* __restrict__ g, uint8_t* sh768, uint32_t* tab) {
  for (int i = threadIdx.x; i < 768; i += blockDim.x) sh768[i] = g[i];
  __syncthreads();
  for (int wi = threadIdx.x; wi < kLutBytes / 4; wi += blockDim.x) {
    const int c = wi >> 11, rem = wi & 2047, vq = rem >> 5;
    const uint8_t* s = sh768 + 256 * c + 4 * vq;
    tab[wi] = (uint32_t)s[0] | ((uint32_t)s[1] << 8) | ((uint32_t)s[2] << 16) | ((uint32_t)s[3] << 24);
  }
  __syncthreads();
}

ALB_D uint32_t lut_off(uint32_t v) { return ((v & 0xFCu) << 5) | (v & 3u); }

// one RGB pixel through the three tables (lb = this lane's table base)
ALB_D void lut_px(const uint8_t* tab, int lb, uint32_t& r, uint32_t& g, uint32_t& b) {
  r = tab[lb + lut_off(r)];
  g = tab[lb + 8192 + lut_off(g)];
  b = tab[lb + 16384 + lut_off(b)];
}

// LUT ops through the bulk-copy engine.  Per CTA, thread 0 runs a pipeline
// of kBulkStages shared-memory stages of kBulkChunk bytes: bulk loads of the
// run's 16-byte-aligned core (completion counted on one mbarrier per stage),
// all threads look the bytes up in place (16-byte vectors; the channel of a
// byte follows its offset mod 3), then one bulk store writes the stage back
// and the stage is refilled once that store has read it.  The <= 15 bytes at
// each end of a run and images that are not contiguous and 16-byte aligned take
// a per-byte / per-pixel path.
constexpr int kBulkChunk = 12288;   // bytes per stage: 768 vectors, a multiple of 3 and 16
constexpr int kBulkStages = 3;
static_assert(kBulkChunk % 48 == 0, "a stage starts on the same channel phase as the previous one");

// After a bounded wait gave up: wait (bounded again) for the copies of chunks
// [first, last) of the sequence -- exactly the chunks whose bulk loads were
// issued and not yet consumed, so that no load into the CTA's shared memory
// is still in flight when it stops -- and record ALB_ETIMEOUT.  A chunk whose
// copy was never issued must not be in the range: its phase cannot complete.
// Called by the thread that issued the loads.
ALB_D void bulk_drain(uint64_t* full, uint32_t seq, int32_t first, int32_t last, int32_t* status) {
  for (int32_t k = first; k < last; k++) {
    const uint32_t q = seq + (uint32_t)k;
    mbar_wait(&full[q % kBulkStages], (q / kBulkStages) & 1u);
  }
  dev_fail(status, ALB_ETIMEOUT);
}

// Streams bytes [0, total) of src (and, with dst, back to dst) through the
// CTA's stages.  body(stage, bytes, offset) runs on every thread for each
// chunk; with dst it may rewrite the stage in place, which is then stored.
// seq counts the CTA's chunk loads (stage = seq % stages, phase parity =
// (seq / stages) & 1) and continues across calls.  Returns false when a
// bounded wait gave up (status set, loads in flight drained): the caller stops.
// Called by all threads of the CTA; src/dst/total 16-byte aligned.
template <class F>
ALB_D bool bulk_pipeline(uint8_t (*stage)[kBulkChunk], uint64_t* full, uint32_t& seq, const uint8_t* src,
                         uint8_t* dst, int64_t total, int32_t* status, F&& body) {
  const int tid = threadIdx.x;
  const int32_t nch = (int32_t)((total + kBulkChunk - 1) / kBulkChunk);
  if (nch == 0) return true;
  auto bytes_of = [&](int32_t j) -> uint32_t {
    const int64_t rest = total - (int64_t)j * kBulkChunk;
    return (uint32_t)(rest < kBulkChunk ? rest : kBulkChunk);
  };
  auto issue = [&](int32_t j) {
    const uint32_t q = seq + (uint32_t)j, st = q % kBulkStages;
    mbar_arrive_expect_tx(&full[st], bytes_of(j));
    bulk_load(stage[st], src + (int64_t)j * kBulkChunk, bytes_of(j), &full[st]);
  };
  if (tid == 0) {
    if (dst) bulk_wait_read<0>();                // every earlier store has read its stage
    for (int32_t j = 0; j < nch && j < kBulkStages - 1; j++) issue(j);
  }
  int32_t j = 0;
  bool dead = false;
  for (; j < nch; j++) {
    const uint32_t q = seq + (uint32_t)j, st = q % kBulkStages;
    const bool ok = mbar_wait(&full[st], (q / kBulkStages) & 1u);
    if (__syncthreads_or(!ok)) { dead = true; break; }
    body(stage[st], (int)bytes_of(j), (int64_t)j * kBulkChunk);
    if (dst) fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      if (dst) {
        bulk_store(dst + (int64_t)j * kBulkChunk, stage[st], bytes_of(j));
        bulk_commit();
      }
      const int32_t jn = j + kBulkStages - 1;    // refills the stage of chunk j - 1
      if (jn < nch) {
        if (dst) bulk_wait_read<1>();
        issue(jn);
      }
    }
  }
  if (dead) {
    // chunks j .. j + stages - 2 had their copies issued (chunk j's wait is
    // the one that gave up); none beyond
    if (tid == 0) bulk_drain(full, seq, j, imin(nch, j + kBulkStages - 1), status);
    return false;
  }
  seq += (uint32_t)nch;
  return true;
}

// the run's bytes [S0, E0) split into head [S0, A), 16-byte-aligned core [A, E), tail [E, E0)
ALB_D void aligned_core(int64_t S0, int64_t E0, int64_t& A, int64_t& E) {
  A = (S0 + 15) & ~int64_t(15);
  E = E0 & ~int64_t(15);
  if (A > E0) A = E0;
  if (E < A) E = A;
}

struct LutBulkSmem {
  uint8_t stage[kBulkStages][kBulkChunk];
  uint32_t tab32[kLutBytes / 4];
  uint64_t full[kBulkStages];
  uint8_t sh768[768];
};

__global__ void __launch_bounds__(256) k_lut_bulk(Plan plan, ImgList in, ImgList out, const uint8_t* __restrict__ luts,
                                                  int32_t* status) {
  extern __shared__ __align__(128) uint8_t lut_dyn[];
  LutBulkSmem& sm = *reinterpret_cast<LutBulkSmem*>(lut_dyn);
  const int lb = 4 * (threadIdx.x & 31);
  const uint8_t* tab0 = reinterpret_cast<const uint8_t*>(sm.tab32);
  const uint8_t* tab = tab0 + lb;
  const int tid = threadIdx.x, bs = blockDim.x;
  if (tid == 0) {
    for (int i = 0; i < kBulkStages; i++) mbar_init(&sm.full[i], 1);
    mbar_init_fence();
  }
  __syncthreads();
  uint32_t seq = 0;
  bool dead = false;
  for_each_run(plan, [&](int32_t b, int32_t r0, int32_t r1) {
    if (dead) return;
    __syncthreads();
    build_lut_copies(luts + (int64_t)b * 768, sm.sh768, sm.tab32);
    const alb_image si = in.get(b), so = out.get(b);
    r1 = imin(r1, so.h);
    const uint8_t* __restrict__ ip = (const uint8_t*)si.data;
    uint8_t* __restrict__ op = (uint8_t*)so.data;
    if (!(flat_aligned(si) && flat_aligned(so))) {
      const int64_t npx = (int64_t)(r1 - r0) * so.w;
      for (int64_t i = tid; i < npx; i += bs) {
        const int32_t y = r0 + (int32_t)(i / so.w), x = (int32_t)(i % so.w);
        const uint8_t* s0 = ip + (int64_t)y * si.row_stride + 3 * (int64_t)x;
        uint8_t* d = op + (int64_t)y * so.row_stride + 3 * (int64_t)x;
        uint32_t R = s0[0], G = s0[1], B = s0[2];
        lut_px(tab0, lb, R, G, B);
        d[0] = (uint8_t)R; d[1] = (uint8_t)G; d[2] = (uint8_t)B;
      }
      return;
    }
    int64_t A, E;
    const int64_t S0 = 3 * (int64_t)r0 * so.w, E0 = 3 * (int64_t)r1 * so.w;
    aligned_core(S0, E0, A, E);
    for (int64_t q = S0 + tid; q < A; q += bs) op[q] = tab[8192 * (int)(q % 3) + lut_off(ip[q])];
    for (int64_t q = E + tid; q < E0; q += bs) op[q] = tab[8192 * (int)(q % 3) + lut_off(ip[q])];
    const int phi = (int)(A % 3);   // channel of the core's first byte; chunks keep it (kBulkChunk % 3 == 0)
    dead = !bulk_pipeline(sm.stage, sm.full, seq, ip + A, op + A, E - A, status,
                          [&](uint8_t* sb, int nbytes, int64_t) {
      const int nv = nbytes >> 4;
      for (int v = tid; v < nv; v += bs) {
        const uint4 x = *reinterpret_cast<const uint4*>(sb + 16 * v);
        const int rho = (phi + v) % 3;             // 16 = 1 mod 3: channel of the vector's first byte
        const uint8_t* t0 = tab + 8192 * rho;
        const uint8_t* t1 = tab + 8192 * (rho == 2 ? 0 : rho + 1);
        const uint8_t* t2 = tab + 8192 * (rho == 0 ? 2 : rho - 1);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
        uint32_t o[4];
#pragma unroll
        for (int m = 0; m < 4; m++) {
          uint32_t acc = 0;
#pragma unroll
          for (int t = 0; t < 4; t++) {
            const int k = 4 * m + t;
            const uint8_t* tb = k % 3 == 0 ? t0 : (k % 3 == 1 ? t1 : t2);
            acc |= (uint32_t)tb[lut_off((w[m] >> (8 * t)) & 0xFFu)] << (8 * t);
          }
          o[m] = acc;
        }
        *reinterpret_cast<uint4*>(sb + 16 * v) = make_uint4(o[0], o[1], o[2], o[3]);
      }
    });
  });
  if (tid == 0) bulk_wait_all();
}

// Per-channel histograms through the bulk-copy stages (read only): one shared
// histogram per CTA held as 8 interleaved copies, word (256 c + v) * 8 +
// (lane & 7), merged into the image's global histogram at the end of each run
// (one image per run).  A lane's word lies in bank 8 (v mod 4) + (lane & 7),
// so at most the 4 lanes of one residue class of lane & 7 can meet in a bank,
// where per-warp copies let all 32 lanes collide at random.
struct HistBulkSmem {
  uint8_t stage[kBulkStages][kBulkChunk];
  uint32_t sh[768 * 8];
  uint64_t full[kBulkStages];
};

__global__ void __launch_bounds__(256) k_hist_bulk(Plan plan, ImgList in, uint32_t* __restrict__ hist,
                                                   int32_t* status) {
  extern __shared__ __align__(128) uint8_t hist_dyn[];
  HistBulkSmem& sm = *reinterpret_cast<HistBulkSmem*>(hist_dyn);
  const int tid = threadIdx.x, bs = blockDim.x;
  // bin (256 c + v) of this lane's copy: my[8 * bin]
  uint32_t* my = sm.sh + (tid & 7);
  for (int i = tid; i < 8 * 768; i += bs) sm.sh[i] = 0;
  if (tid == 0) {
    for (int i = 0; i < kBulkStages; i++) mbar_init(&sm.full[i], 1);
    mbar_init_fence();
  }
  __syncthreads();
  uint32_t seq = 0;
  bool dead = false;
  for_each_run(plan, [&](int32_t b, int32_t r0, int32_t r1) {
    if (dead) return;
    const alb_image si = in.get(b);
    r1 = imin(r1, si.h);
    const uint8_t* __restrict__ ip = (const uint8_t*)si.data;
    if (flat_aligned(si)) {
      int64_t A, E;
      const int64_t S0 = 3 * (int64_t)r0 * si.w, E0 = 3 * (int64_t)r1 * si.w;
      aligned_core(S0, E0, A, E);
      for (int64_t q = S0 + tid; q < A; q += bs) atomicAdd(&my[8 * (256 * (int)(q % 3) + ip[q])], 1u);
      for (int64_t q = E + tid; q < E0; q += bs) atomicAdd(&my[8 * (256 * (int)(q % 3) + ip[q])], 1u);
      const int phi = (int)(A % 3);
      dead = !bulk_pipeline(sm.stage, sm.full, seq, ip + A, nullptr, E - A, status,
                            [&](uint8_t* sb, int nbytes, int64_t) {
        const int nv = nbytes >> 4;
        for (int v = tid; v < nv; v += bs) {
          const uint4 x = *reinterpret_cast<const uint4*>(sb + 16 * v);
          const int rho = (phi + v) % 3;
          uint32_t* h0 = my + 2048 * rho;
          uint32_t* h1 = my + 2048 * (rho == 2 ? 0 : rho + 1);
          uint32_t* h2 = my + 2048 * (rho == 0 ? 2 : rho - 1);
          const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int k = 0; k < 16; k++) {
            uint32_t* hb = k % 3 == 0 ? h0 : (k % 3 == 1 ? h1 : h2);
            atomicAdd(&hb[8 * ((w[k >> 2] >> (8 * (k & 3))) & 0xFFu)], 1u);
          }
        }
      });
      if (dead) return;
    } else {
      const int64_t npx = (int64_t)(r1 - r0) * si.w;
      for (int64_t i = tid; i < npx; i += bs) {
        const int32_t y = r0 + (int32_t)(i / si.w), x = (int32_t)(i % si.w);
        const uint8_t* s = ip + (int64_t)y * si.row_stride + 3 * (int64_t)x;
#pragma unroll
        for (int c = 0; c < 3; c++) atomicAdd(&my[8 * (256 * c + s[c])], 1u);
      }
    }
    __syncthreads();
    for (int i = tid; i < 768; i += bs) {
      uint32_t sum = 0;
#pragma unroll
      for (int w = 0; w < 8; w++) { sum += sm.sh[8 * i + w]; sm.sh[8 * i + w] = 0; }
      if (sum) atomicAdd(&hist[(int64_t)b * 768 + i], sum);
    }
    __syncthreads();
  });
}

// ================================================================== per-pixel ops
ALB_D void gray_px(uint32_t& r, uint32_t& g, uint32_t& b) {
  const uint32_t num = 299 * r + 587 * g + 114 * b;
  uint32_t q = num / 1000, rem = num - q * 1000;
  if (rem > 500 || (rem == 500 && (q & 1))) q++;
  r = g = b = q;
}

// ShiftHSV, float32 (Smith's hexcone; hue shift 2*dh degrees; sat and val by
// /255), with the hue kept in sextants (H/60, in [0, 6)).  Every value is a
// BIASED float 2^23 + v: the bit pattern of a byte v is 0x4B000000 | v, so a
// channel is unpacked with one byte permute, differences of two channels are
// exact, the integer chroma and max are differences of bit patterns, and
// adding 2^23 to a result in [0, 255] rounds it to the nearest integer (ties
// to even) into the low byte of its bit pattern, ready to be packed.  The two
// reciprocals (1 / chroma, 1 / max) come from a 256-entry table of correctly
// rounded 1 / c (entry 0 = 0: a grey pixel has hue 0 and saturation 0).
// Branch-free: the hue numerator/offset are selected, and the inverse hexcone
// uses the per-channel form f(n) = V - V S t(k), t(k) = clamp(min(k, 4 - k),
// 0, 1) for k = (n + H/60) mod 6, n = 5, 3, 1 for R, G, B (identical to the
// sector table of the definition).  k = H/60 + n lies in [1, 11), where t is
// 2 - (the distance to the nearer of 2 and 8), clamped, so no wrap is needed.
// The result lies in [V - VS, V] within [0, 255], so only the rounding remains.
constexpr float kBias = 8388608.0f;   // 2^23

ALB_D float hsv_channel_b(float hp, float n, float V255, float C255) {
  const float d = fminf(fabsf(hp + (n - 2.0f)), fabsf(hp + (n - 8.0f)));
  return fmaf(-C255, __saturatef(2.0f - d), V255) + kBias;
}

ALB_D void hsv_px_b(const float* __restrict__ rcp, float dh6, float ds, float dv, float& R, float& G, float& B) {
  const float r = R, g = G, b = B;
  const float mx = fmaxf(r, fmaxf(g, b)), mn = fminf(r, fminf(g, b));
  const uint32_t ic = __float_as_uint(mx) - __float_as_uint(mn), im = __float_as_uint(mx) & 0xFFu;
  const float chroma = mx - mn, mxv = mx - kBias;
  const bool isr = mx == r, isg = !isr && mx == g;
  const float num = isr ? g - b : (isg ? b - r : r - g);
  const float off = isr ? 0.0f : (isg ? 2.0f : 4.0f);
  float hue = fmaf(num, rcp[ic], off);
  hue = hue < 0.0f ? hue + 6.0f : hue;
  const float sat = chroma * rcp[im];
  float hp = hue + dh6;
  hp = hp >= 6.0f ? hp - 6.0f : hp;
  hp = hp < 0.0f ? hp + 6.0f : hp;
  const float s2 = __saturatef(sat + ds);
  const float v2 = __saturatef(fmaf(mxv, 1.0f / 255.0f, dv));
  const float V255 = 255.0f * v2, C255 = V255 * s2;
  R = hsv_channel_b(hp, 5.0f, V255, C255);
  G = hsv_channel_b(hp, 3.0f, V255, C255);
  B = hsv_channel_b(hp, 1.0f, V255, C255);
}

// byte i (compile-time after unrolling) of the words as a biased float
template <int NW>
ALB_D float biased_byte(const uint32_t (&w)[NW], int i) {
  return __uint_as_float(__byte_perm(w[i >> 2], 0x4B000000u, 0x7440u | (uint32_t)(i & 3)));
}
ALB_D float biased(uint32_t v) { return __uint_as_float(0x4B000000u | v); }
ALB_D uint8_t unbias(float f) { return (uint8_t)__float_as_uint(f); }

struct PixArgs {
  const float* rcp;
  float dh6, ds, dv;
};

template <int OP>  // 0 = Grayscale, 1 = ShiftHSV
ALB_D void pixel_op(uint32_t& r, uint32_t& g, uint32_t& b, const PixArgs& a) {
  if (OP == 0) {
    gray_px(r, g, b);
  } else {
    float R = biased(r), G = biased(g), B = biased(b);
    hsv_px_b(a.rcp, a.dh6, a.ds, a.dv, R, G, B);
    r = unbias(R); g = unbias(G); b = unbias(B);
  }
}

template <int OP>
ALB_D void pixel_unit(const U48& u, uint32_t (&o)[12], const PixArgs& a) {
  uint32_t w[12];
  words48(u, w);
  if (OP == 0) {
#pragma unroll
    for (int m = 0; m < 12; m++) o[m] = 0;
#pragma unroll
    for (int px = 0; px < 16; px++) {
      uint32_t R = byte_of(w, 3 * px), G = byte_of(w, 3 * px + 1), B = byte_of(w, 3 * px + 2);
      gray_px(R, G, B);
      o[(3 * px) >> 2] |= R << (8 * ((3 * px) & 3));
      o[(3 * px + 1) >> 2] |= G << (8 * ((3 * px + 1) & 3));
      o[(3 * px + 2) >> 2] |= B << (8 * ((3 * px + 2) & 3));
    }
  } else {
    // 48 results as biased floats; each output word packs the low bytes of four
    float f[48];
#pragma unroll
    for (int px = 0; px < 16; px++) {
      float R = biased_byte(w, 3 * px), G = biased_byte(w, 3 * px + 1), B = biased_byte(w, 3 * px + 2);
      hsv_px_b(a.rcp, a.dh6, a.ds, a.dv, R, G, B);
      f[3 * px] = R; f[3 * px + 1] = G; f[3 * px + 2] = B;
    }
#pragma unroll
    for (int m = 0; m < 12; m++) {
      const uint32_t lo = __byte_perm(__float_as_uint(f[4 * m]), __float_as_uint(f[4 * m + 1]), 0x0040u);
      const uint32_t hi = __byte_perm(__float_as_uint(f[4 * m + 2]), __float_as_uint(f[4 * m + 3]), 0x0040u);
      o[m] = __byte_perm(lo, hi, 0x5410u);
    }
  }
}

template <int OP>
__global__ void __launch_bounds__(256) k_pixel_stream(Plan plan, ImgList in, ImgList out, PrmList prm) {
  __shared__ float s_rcp[256];
  if (OP == 1) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) s_rcp[i] = i ? 1.0f / (float)i : 0.0f;
    __syncthreads();
  }
  for_each_run(plan, [&](int32_t b, int32_t r0, int32_t r1) {
    const alb_image si = in.get(b), so = out.get(b);
    const alb_params& p = prm.get(b);
    r1 = imin(r1, so.h);
    const bool act = p.apply != 0;
    // the per-image shifts in float (from the record's doubles), formed by one
    // lane per warp: double-precision work is slow on this part
    float dh6 = 0.0f, ds = 0.0f, dv = 0.0f;
    if (OP == 1) {
      if ((threadIdx.x & 31) == 0) {
        dh6 = (float)(2.0 * p.shift[0]) * (1.0f / 60.0f);
        ds = (float)(p.shift[1] / 255.0);
        dv = (float)(p.shift[2] / 255.0);
      }
      dh6 = __shfl_sync(0xffffffffu, dh6, 0);
      ds = __shfl_sync(0xffffffffu, ds, 0);
      dv = __shfl_sync(0xffffffffu, dv, 0);
    }
    const PixArgs pa{s_rcp, dh6, ds, dv};
    const uint8_t* __restrict__ ip = (const uint8_t*)si.data;
    uint8_t* __restrict__ op = (uint8_t*)so.data;
    if (flat_aligned(si) && flat_aligned(so)) {
      const int64_t a = (int64_t)r0 * so.w, e = (int64_t)r1 * so.w;   // pixel range
      const int64_t u0 = (a + 15) >> 4, u1 = e >> 4;                    // whole 16-pixel units
      int64_t u = u0 + threadIdx.x;
      U48 nx;
      if (u < u1) ld48(ip + 48 * u, nx);
      for (; u < u1; u += blockDim.x) {
        const U48 cur = nx;
        if (u + blockDim.x < u1) ld48(ip + 48 * (u + blockDim.x), nx);
        uint32_t o[12];
        if (act) {
          pixel_unit<OP>(cur, o, pa);
        } else {
          words48(cur, o);
        }
        st48(op + 48 * u, o);
      }
      const int64_t h1 = u0 * 16 < e ? u0 * 16 : e;
      for (int64_t q = a + threadIdx.x; q < e; q += blockDim.x) {
        if (q >= h1 && q < u1 * 16) continue;
        uint32_t R = ip[3 * q], G = ip[3 * q + 1], B = ip[3 * q + 2];
        if (act) pixel_op<OP>(R, G, B, pa);
        op[3 * q] = (uint8_t)R; op[3 * q + 1] = (uint8_t)G; op[3 * q + 2] = (uint8_t)B;
      }
    } else {
      const int64_t npx = (int64_t)(r1 - r0) * so.w;
      for (int64_t i = threadIdx.x; i < npx; i += blockDim.x) {
        const int32_t y = r0 + (int32_t)(i / so.w), x = (int32_t)(i % so.w);
        const uint8_t* s = ip + (int64_t)y * si.row_stride + 3 * (int64_t)x;
        uint8_t* d = op + (int64_t)y * so.row_stride + 3 * (int64_t)x;
        uint32_t R = s[0], G = s[1], B = s[2];
        if (act) pixel_op<OP>(R, G, B, pa);
        d[0] = (uint8_t)R; d[1] = (uint8_t)G; d[2] = (uint8_t)B;
      }
    }
  });
}

// ================================================================== pixel maps
// HorizontalFlip, VerticalFlip, RandomCrop and PadToSize on RGB images: output
// pixel (y, x) is source pixel (src_y(y), src_x(x)), with src_x of slope +1
// or -1 between reflection points.  Flat 16-pixel output units (48 aligned
// bytes): when src_x over the unit's 16 pixels is one run of slope +1 the
// unit is a 48-byte source window (realigned with funnel shifts); slope -1 is
// the same window with the pixel order reversed in registers; a unit that
// holds a reflection point or a row end takes the per-pixel path.  The next
// unit's window loads are issued before the current unit is assembled.
template <int TID>
struct PixMap {
  int32_t H, W, x0, y0;
  bool act;
  ALB_D int32_t sy(int32_t y) const {
    if (!act) return y;
    if (TID == ALB_VFLIP) return H - 1 - y;
    if (TID == ALB_RANDOM_CROP) return y0 + y;
    if (TID == ALB_PAD_TO_SIZE) return reflect101(y - y0, H);
    return y;
  }
  ALB_D int32_t sx(int32_t x) const {
    if (!act) return x;
    if (TID == ALB_HFLIP) return W - 1 - x;
    if (TID == ALB_RANDOM_CROP) return x0 + x;
    if (TID == ALB_PAD_TO_SIZE) return reflect101(x - x0, W);
    return x;
  }
  // How output pixels x .. x + 15 map: 0 = source pixels start .. start + 15,
  // 1 = the same 16 pixels in reverse order, 2 = neither (a reflection point)
  ALB_D int run16(int32_t x, int32_t& start) const {
    start = x;
    if (!act) return 0;
    if (TID == ALB_HFLIP) { start = W - 16 - x; return 1; }
    if (TID == ALB_RANDOM_CROP) { start = x0 + x; return 0; }
    if (TID == ALB_PAD_TO_SIZE) {
      const int32_t d = x - x0;
      if (d >= 0 && d + 15 < W) { start = d; return 0; }
      if (d + 15 < 0 && d > -W) { start = -(d + 15); return 1; }                   // left border, one fold
      if (d >= W && d + 15 <= 2 * W - 2) { start = 2 * (W - 1) - (d + 15); return 1; }  // right border, one fold
      return 2;
    }
    return 0;
  }
};

ALB_HD constexpr int rev_src(int k) { return 3 * (15 - k / 3) + k % 3; }
ALB_HD constexpr int rev_word(int k, int j) { return rev_src(4 * k + j) >> 2; }
ALB_HD constexpr int rev_lo(int k) {
  int lo = rev_word(k, 0);
  for (int j = 1; j < 4; j++) lo = rev_word(k, j) < lo ? rev_word(k, j) : lo;
  return lo;
}

// The 16 RGB pixels of a 48-byte window in reverse order, channel order kept.
// Output word k takes its bytes from at most three consecutive source words:
// one byte permute of the first two, a second one for the third.
ALB_D void reverse16(const uint32_t (&win)[12], uint32_t (&o)[12]) {
#pragma unroll
  for (int k = 0; k < 12; k++) {
    const int lo = rev_lo(k);
    uint32_t sel1 = 0, sel2 = 0;
    bool three = false;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int d = rev_word(k, j) - lo, byte = rev_src(4 * k + j) & 3;
      if (d <= 1) {
        sel1 |= (uint32_t)(4 * d + byte) << (4 * j);
        sel2 |= (uint32_t)j << (4 * j);
      } else {
        three = true;
        sel2 |= (uint32_t)(4 + byte) << (4 * j);
      }
    }
    const uint32_t a = __byte_perm(win[lo], win[lo + 1 < 12 ? lo + 1 : 11], sel1);
    o[k] = three ? __byte_perm(a, win[lo + 2 < 12 ? lo + 2 : 11], sel2) : a;
  }
}

template <int TID>
__global__ void __launch_bounds__(256, 3) k_pixmap3(Plan plan, ImgList in, ImgList out, PrmList prm) {
  for_each_run(plan, [&](int32_t b, int32_t r0, int32_t r1) {
    const alb_image si = in.get(b), so = out.get(b);
    const alb_params& p = prm.get(b);
    r1 = imin(r1, so.h);
    PixMap<TID> m{si.h, si.w, p.x0, p.y0, p.apply != 0};
    const int32_t OW = so.w;
    const uint8_t* __restrict__ ip = (const uint8_t*)si.data;
    uint8_t* __restrict__ op = (uint8_t*)so.data;
    const int64_t ss = si.row_stride;
    auto src_px = [&](int32_t y, int32_t x) { return ip + (int64_t)m.sy(y) * ss + 3 * (int64_t)m.sx(x); };
    if (!flat_aligned(so)) {
      const int64_t npx = (int64_t)(r1 - r0) * OW;
      for (int64_t i = threadIdx.x; i < npx; i += blockDim.x) {
        const int32_t y = r0 + (int32_t)(i / OW), x = (int32_t)(i % OW);
        const uint8_t* s = src_px(y, x);
        uint8_t* d = op + (int64_t)y * so.row_stride + 3 * (int64_t)x;
        d[0] = s[0]; d[1] = s[1]; d[2] = s[2];
      }
      return;
    }
    const int64_t a = (int64_t)r0 * OW, e = (int64_t)r1 * OW;
    const int64_t u0 = (a + 15) >> 4, u1 = e >> 4;
    // kind 0: forward window, 1: reversed window, 2: per pixel
    auto fetch = [&](int64_t u, RawWin<12>& rw, int& kind) {
      int32_t y, x;
      flat_rc(16 * u, OW, y, x);
      kind = 2;
      if (x + 16 > OW) return;
      int32_t start;
      kind = m.run16(x, start);
      if (kind == 2) return;
      raw_load<12>(ip + (int64_t)m.sy(y) * ss + 3 * (int64_t)start, rw);
    };
    // every lane of a warp runs the same iterations (the bound is tested per
    // lane), so the warp can take its per-pixel units together
    const int lane = threadIdx.x & 31;
    int64_t ub = u0;
    RawWin<12> nx;
    int nkind = 2;
    if (ub + threadIdx.x < u1) fetch(ub + threadIdx.x, nx, nkind);
    for (; ub < u1; ub += blockDim.x) {
      const int64_t u = ub + threadIdx.x;
      const bool valid = u < u1;
      const RawWin<12> cur = nx;
      const int kind = nkind;
      if (u + blockDim.x < u1) fetch(u + blockDim.x, nx, nkind);
      if (valid && kind != 2) {
        uint32_t win[12], o[12];
        raw_align<12>(cur, win);
        if (kind == 0) {
#pragma unroll
          for (int k = 0; k < 12; k++) o[k] = win[k];
        } else {
          reverse16(win, o);
        }
        st48(op + 48 * u, o);
      }
      // units with a reflection point or a row end inside: their pixels,
      // listed unit by unit, are spread over the lanes (one pixel per lane
      // and round), so the warp waits one load latency for up to two units
      const uint32_t todo = __ballot_sync(0xffffffffu, valid && kind == 2);
      const int npx = 16 * __popc(todo);
      for (int base = 0; base < npx; base += 32) {
        const int idx = base + lane;
        int src = 0;                       // lane holding the (idx / 16)-th such unit
        if (idx < npx) {
          uint32_t mm = todo;
          for (int k = idx >> 4; k > 0; k--) mm &= mm - 1;   // clear the lower set bits
          src = __ffs(mm) - 1;
        }
        const int64_t su = __shfl_sync(0xffffffffu, u, src);
        if (idx < npx) {
          const int j = idx & 15;
          int32_t y, x;
          flat_rc(16 * su + j, OW, y, x);
          const uint8_t* s = src_px(y, x);
          uint8_t* d = op + 48 * su + 3 * j;
          d[0] = s[0]; d[1] = s[1]; d[2] = s[2];
        }
      }
    }
    // pixels of the run outside whole units
    const int64_t h1 = u0 * 16 < e ? u0 * 16 : e;
    for (int64_t q = a + threadIdx.x; q < e; q += blockDim.x) {
      if (q >= h1 && q < u1 * 16) continue;
      int32_t y, x;
      flat_rc(q, OW, y, x);
      const uint8_t* s = src_px(y, x);
      op[3 * q] = s[0]; op[3 * q + 1] = s[1]; op[3 * q + 2] = s[2];
    }
  });
}

// ================================================================== row copies
// Vertical flip, crop and pad: output row y takes bytes of source row sy
// starting at a row-constant offset (crop: 3 x0; pad interior: -3 left); pad
// borders are reflected pixels.  Three lane-parallel loops per item: whole
// 16-byte chunks of the interior (realigned source window), the <= 15 interior
// bytes at each end outside whole chunks, and the pad borders.
template <int CT, int TID>
__global__ void __launch_bounds__(256) k_rowcopy(Plan plan, ImgList in, ImgList out, PrmList prm) {
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
    const int32_t nrow = r1 - r0;
    const bool act = p.apply != 0;
    const int32_t L = so.w * C;
    // interior output bytes [lo, hi) come from source byte x + shift
    int32_t lo = 0, hi = L, shift = 0;
    if (act && TID == ALB_RANDOM_CROP) shift = p.x0 * C;
    if (act && TID == ALB_PAD_TO_SIZE) { lo = p.x0 * C; hi = lo + si.w * C; shift = -lo; }
    const uint8_t* __restrict__ ip = (const uint8_t*)si.data;
    uint8_t* __restrict__ op = (uint8_t*)so.data;
    auto src_row = [&](int32_t y) -> int32_t {
      if (!act) return y;
      if (TID == ALB_VFLIP) return si.h - 1 - y;
      if (TID == ALB_RANDOM_CROP) return p.y0 + y;
      return reflect101((int64_t)y - p.y0, si.h);
    };
    // first and last whole chunk of the interior of row y
    auto chunk_bounds = [&](uint8_t* orow, int32_t& A, int32_t& B) {
      const int32_t ph = (int32_t)(reinterpret_cast<uintptr_t>(orow) & 15);
      A = ((ph + lo + 15) & ~15) - ph;
      B = ((ph + hi) & ~15) - ph;
      if (B < A) { A = hi; B = hi; }
    };
    const int32_t cpr = (hi - lo) / 16 + 1;
    for (int32_t i = threadIdx.x; i < nrow * cpr; i += blockDim.x) {
      const int32_t yy = i / cpr, j = i - yy * cpr, y = r0 + yy;
      uint8_t* orow = op + (int64_t)y * so.row_stride;
      int32_t A, B;
      chunk_bounds(orow, A, B);
      const int32_t x = A + 16 * j;
      if (x + 16 > B) continue;
      const uint8_t* srow = ip + (int64_t)src_row(y) * si.row_stride;
      uint32_t w[4];
      load_window<4>(srow + x + shift, w);
      stg16(orow + x, make_uint4(w[0], w[1], w[2], w[3]));
    }
    for (int32_t i = threadIdx.x; i < nrow * 32; i += blockDim.x) {
      const int32_t yy = i >> 5, k = i & 31, y = r0 + yy;
      uint8_t* orow = op + (int64_t)y * so.row_stride;
      int32_t A, B;
      chunk_bounds(orow, A, B);
      const int32_t x = k < 16 ? lo + k : B + (k - 16);
      if (k < 16 ? x >= A : x >= hi) continue;
      orow[x] = ip[(int64_t)src_row(y) * si.row_stride + x + shift];
    }
    if (TID == ALB_PAD_TO_SIZE && act) {
      const int32_t nb = lo + (L - hi);
      for (int32_t i = threadIdx.x; i < nrow * nb; i += blockDim.x) {
        const int32_t yy = i / nb, k = i - yy * nb, y = r0 + yy;
        const int32_t x = k < lo ? k : hi + (k - lo);
        const int32_t px = x / C, c = x - px * C;
        const int32_t sx = reflect101((int64_t)px - p.x0, si.w);
        op[(int64_t)y * so.row_stride + x] = ip[(int64_t)src_row(y) * si.row_stride + sx * C + c];
      }
    }
  }
}

// ================================================================== launchers
static int grid_for(const void* fn, int threads) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
  return (per_sm < 1 ? 1 : per_sm) * sm_count();
}

template <class... KArgs, class... Args>
static alb_status launch_k(void (*kern)(KArgs...), cudaStream_t st, Args... args) {
  kern<<<grid_for((const void*)kern, 256), 256, 0, st>>>(args...);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

// Streaming implementations; returns ALB_EINVAL (nothing launched) when the
// transform/channel combination has none, so the caller uses its general kernel.
alb_status launch_stream_geometric(int32_t tid, const Plan& plan, const ImgList& in, const ImgList& out,
                                   const PrmList& prm, int32_t channels, cudaStream_t st) {
  if (channels == 3) {
    switch (tid) {
      case ALB_HFLIP: return launch_k(k_pixmap3<ALB_HFLIP>, st, plan, in, out, prm);
      case ALB_VFLIP: return launch_k(k_pixmap3<ALB_VFLIP>, st, plan, in, out, prm);
      case ALB_RANDOM_CROP: return launch_k(k_pixmap3<ALB_RANDOM_CROP>, st, plan, in, out, prm);
      case ALB_PAD_TO_SIZE: return launch_k(k_pixmap3<ALB_PAD_TO_SIZE>, st, plan, in, out, prm);
      default: break;
    }
  }
  switch (tid) {
    case ALB_VFLIP:
      if (channels == 1) return launch_k(k_rowcopy<1, ALB_VFLIP>, st, plan, in, out, prm);
      return launch_k(k_rowcopy<0, ALB_VFLIP>, st, plan, in, out, prm);
    case ALB_RANDOM_CROP:
      if (channels == 1) return launch_k(k_rowcopy<1, ALB_RANDOM_CROP>, st, plan, in, out, prm);
      return launch_k(k_rowcopy<0, ALB_RANDOM_CROP>, st, plan, in, out, prm);
    case ALB_PAD_TO_SIZE:
      if (channels == 1) return launch_k(k_rowcopy<1, ALB_PAD_TO_SIZE>, st, plan, in, out, prm);
      return launch_k(k_rowcopy<0, ALB_PAD_TO_SIZE>, st, plan, in, out, prm);
    default:
      break;
  }
  return ALB_EINVAL;
}

alb_status launch_stream_lut(const Plan& plan, const ImgList& in, const ImgList& out, const uint8_t* luts,
                             int32_t* status, cudaStream_t st) {
  const int smem = (int)sizeof(LutBulkSmem);
  ALB_CUDA(cudaFuncSetAttribute(k_lut_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lut_bulk, 256, smem);
  k_lut_bulk<<<(per_sm < 1 ? 1 : per_sm) * sm_count(), 256, smem, st>>>(plan, in, out, luts, status);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

alb_status launch_stream_pixel(int32_t tid, const Plan& plan, const ImgList& in, const ImgList& out,
                               const PrmList& prm, int32_t* status, cudaStream_t st) {
  (void)status;   // the register-pipelined kernels have no bounded waits
  if (tid == ALB_GRAYSCALE) return launch_k(k_pixel_stream<0>, st, plan, in, out, prm);
  return launch_k(k_pixel_stream<1>, st, plan, in, out, prm);
}

alb_status launch_stream_hist(const Plan& plan, const ImgList& in, uint32_t* hist, int32_t* status,
                              cudaStream_t st) {
  const int smem = (int)sizeof(HistBulkSmem);
  ALB_CUDA(cudaFuncSetAttribute(k_hist_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hist_bulk, 256, smem);
  k_hist_bulk<<<(per_sm < 1 ? 1 : per_sm) * sm_count(), 256, smem, st>>>(plan, in, hist, status);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

// Self-test of the bounded wait and of the drain that follows it.  One CTA,
// one thread: stages 1 and 2 get real 16-byte bulk loads from src; stage 0
// gets the arrival announcing 16 bytes but no copy, so its phase can never
// complete.  The wait on stage 0 (at most `spins` tries, the same routine as
// the pipelines') gives up; bulk_drain then waits for the two copies that
// were issued -- and only those -- and records ALB_ETIMEOUT.  The drained
// stages are copied to out[0, 32) so the caller can see that they landed
// before the CTA ended.
__global__ void k_wait_selftest(uint32_t spins, const uint8_t* __restrict__ src, uint8_t* __restrict__ out,
                                int32_t* status) {
  __shared__ __align__(128) uint8_t stage[kBulkStages][kBulkChunk > 64 ? 64 : kBulkChunk];
  __shared__ __align__(8) uint64_t full[kBulkStages];
  if (threadIdx.x != 0) return;
  for (int i = 0; i < kBulkStages; i++) mbar_init(&full[i], 1);
  mbar_init_fence();
  mbar_arrive_expect_tx(&full[0], 16);                 // announced, never issued
  for (int k = 1; k < kBulkStages; k++) {
    mbar_arrive_expect_tx(&full[k], 16);
    bulk_load(stage[k], src + 16 * (k - 1), 16, &full[k]);
  }
  if (mbar_wait(&full[0], 0u, spins)) return;          // cannot happen: nothing completes stage 0
  bulk_drain(full, 0u, 1, kBulkStages, status);
  for (int k = 1; k < kBulkStages; k++)
    for (int b = 0; b < 16; b++) out[16 * (k - 1) + b] = stage[k][b];
}

alb_status launch_wait_selftest(uint32_t spins, const uint8_t* src, uint8_t* out, int32_t* status,
                                cudaStream_t st) {
  static_assert(kBulkStages == 3, "the self-test issues copies into stages 1 and 2");
  k_wait_selftest<<<1, 32, 0, st>>>(spins, src, out, status);
  ALB_CUDA(cudaGetLastError());
  return ALB_OK;
}

}  // namespace alb
