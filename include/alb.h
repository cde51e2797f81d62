/*
 * alb.h -- C ABI of libalb.so, the GB300 (sm_103a) augmentation hot path of
 * Buslaev et al., "Albumentations: fast and flexible image augmentations"
 * (arXiv 1809.06839).
 *
 * The paper's method: a transform with sampled parameters is applied to an
 * image and, with the same geometry, to its targets -- segmentation masks and
 * bounding boxes (Sec. II, Sec. II-A, Sec. II-B); Table I (Sec. III) lists
 * the benchmarked transforms.  The paper defines none of the operations
 * mathematically; the definitions this library implements (coordinate
 * conventions, border mode, rounding, sampling) are written out with each
 * entry point below and in the project's design notes.
 *
 * Conventions for every call
 *  - Images are uint8, HWC, channels interleaved, rows `row_stride` bytes
 *    apart (row_stride >= w*c).  Image data pointers are DEVICE pointers,
 *    owned by the caller.  RGB images have c == 3; masks have c >= 1.
 *  - Boxes are float32 [n][4] (x1, y1, x2, y2) in pixel-edge coordinates:
 *    the image covers [0, w] x [0, h].
 *  - Unless stated otherwise the library allocates nothing.  Scratch memory
 *    comes from a caller-provided device `workspace` of at least the size
 *    the matching *_workspace_size call returns.
 *  - Launches are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream).  Every call returns an alb_status; on failure nothing
 *    was launched and alb_last_error() (thread-local) holds a message.
 *    Errors found by kernels (a parameter record that does not fit its
 *    image, a box buffer that is too small) are written to the optional
 *    device word `dev_status` (first error wins; the caller zeroes it).
 *  - No call falls back to the CPU.
 */
#ifndef ALB_H
#define ALB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ALB_API __attribute__((visibility("default")))
#else
#define ALB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
typedef enum alb_status {
  ALB_OK = 0,
  ALB_EINVAL = 1,     /* bad argument (null pointer, unknown id, c != 3 for RGB ops) */
  ALB_ESHAPE = 2,     /* sizes inconsistent with the parameters (e.g. crop > image) */
  ALB_EALIGN = 3,     /* misaligned pointer or stride */
  ALB_ECAPACITY = 4,  /* box buffer or batch capacity exceeded */
  ALB_ECUDA = 5,      /* a CUDA runtime call failed */
  ALB_ETIMEOUT = 6,   /* a bounded device wait gave up */
  ALB_EWORKSPACE = 7  /* workspace missing or smaller than required */
} alb_status;

/* ---- transform ids (Table I of the paper plus the transforms of Sec. II) ---- */
typedef enum alb_tid {
  ALB_HFLIP = 1,                 /* Table I "HorizontalFlip" */
  ALB_VFLIP = 2,                 /* Table I "VerticalFlip" */
  ALB_RANDOM_CROP = 3,           /* Table I "RandomCrop64" */
  ALB_PAD_TO_SIZE = 4,           /* Table I "PadToSize512" */
  ALB_BRIGHTNESS = 5,            /* Table I "Brightness" */
  ALB_CONTRAST = 6,              /* Sec. II, Fig. 1 contrast transform */
  ALB_BRIGHTNESS_CONTRAST = 7,   /* brightness and contrast as one table */
  ALB_GAMMA = 8,                 /* Table I "Gamma" */
  ALB_SHIFT_RGB = 9,             /* Table I "ShiftRGB" */
  ALB_SHIFT_HSV = 10,            /* Table I "ShiftHSV" */
  ALB_GRAYSCALE = 11,            /* Table I "Grayscale" */
  ALB_EQUALIZE = 12,             /* per-channel histogram equalisation */
  ALB_ROTATE = 13,               /* Table I "Rotate" */
  ALB_SHIFT_SCALE_ROTATE = 14,   /* Table I "ShiftScaleRotate" */
  ALB_RESIZE = 15,               /* Sec. II-B scaling */
  ALB_RANDOM_SIZED_CROP = 16,    /* Sec. II-A, Fig. 2 random sized crop */
  ALB_RANDOM_RESIZED_CROP = 17,  /* crop of sampled area and aspect, resized */
  ALB_TRANSPOSE = 18,            /* Sec. II-B, Dih4 element */
  ALB_ROT90 = 19,                /* Sec. II-B, Dih4 rotations */
  ALB_CHAIN = 20,                /* the fused ragged-batch chain (alb_apply_batch) */
  ALB_GRID_DISTORTION = 21,      /* Sec. II-C: grid distortion (separable piecewise-linear map) */
  ALB_ELASTIC = 22               /* Sec. II-C: elastic transform (smooth random displacement field) */
} alb_tid;

/* One image (or mask) in device memory.  32 bytes. */
typedef struct alb_image {
  void* data;           /* device pointer to byte (0,0,0); caller-owned */
  int32_t h, w, c;      /* rows, columns, interleaved channels */
  int32_t reserved;     /* must be 0 */
  int64_t row_stride;   /* bytes from one row to the next, >= w*c */
} alb_image;

/* The sampled parameters of one transform for one image (Sec. II: the
 * transform's parameters).  Produced by alb_sample_params[_batch];
 * callers may also fill it themselves.  Fields unused by a transform are 0
 * (scale, alpha, gamma and sat default to 1).  232 bytes. */
typedef struct alb_params {
  int32_t tid;           /* alb_tid */
  int32_t apply;         /* 1 = applied, 0 = identity (the probability draw failed) */
  int32_t in_h, in_w;    /* input size the record was sampled for */
  int32_t out_h, out_w;  /* output size */
  int32_t y0, x0;        /* crop window origin; PadToSize: top/left padding */
  int32_t ch, cw;        /* crop window size (RandomCrop, Resize, RSC, RRC, chain);
                            ELASTIC: cw = log2 of the lattice spacing (2..8) */
  int32_t flip;          /* chain: 1 = horizontal flip */
  int32_t k;             /* ROT90: quarter turns counter-clockwise; CHAIN: order of the
                            jitter ops 0..5; GRID_DISTORTION: cells per axis G (1..12);
                            ELASTIC: displacement amplitude A in 1/32 px */
  double alpha;          /* contrast gain; chain: contrast factor */
  double beta;           /* brightness shift (pixel units); chain: brightness factor */
  double gamma;          /* gamma exponent */
  double sat;            /* chain: saturation factor */
  double shift[3];       /* ShiftRGB per channel; ShiftHSV (hue half-degrees, sat, val /255) */
  double angle;          /* warp angle, degrees, counter-clockwise on screen */
  double scale;          /* warp scale */
  double dx, dy;         /* warp shift, fractions of w and h */
  double m[6];           /* forward map src -> dst, pixel-centre coordinates, row-major 2x3 */
  int64_t q[6];          /* Rotate/SSR: inverse map dst -> src, Q16 fixed point (round half
                            even).  GRID_DISTORTION: per-cell factors, Q14, 16 bits each
                            (slot j in bits 16 (j % 4) of q[j / 4]; x cells in slots 0..11,
                            y cells in 12..23).  ELASTIC: the lattice's Philox seed, stream
                            id and image index in q[0..2] */
} alb_params;

/* Sampling configuration of one transform.  Meaning of the ranges:
 *  BRIGHTNESS lo/hi[0] = beta;  CONTRAST [0] = alpha;  BRIGHTNESS_CONTRAST
 *  [0] = alpha, [1] = beta;  GAMMA [0] = gamma;  SHIFT_RGB [0..2] per channel;
 *  SHIFT_HSV [0] hue, [1] sat, [2] val;  ROTATE [0] angle;
 *  SHIFT_SCALE_ROTATE [0] shift (each axis), [1] scale, [2] angle;
 *  RANDOM_SIZED_CROP [0] side as a fraction of min(h, w);
 *  RANDOM_RESIZED_CROP / CHAIN [0] area fraction, [1] aspect w/h,
 *  CHAIN [2] brightness, contrast and saturation factors.
 *  GRID_DISTORTION [0] cell factor offset (factor 1 + U[lo, hi]); lo[1] cells
 *  per axis (1..12, 0 = 5).  ELASTIC lo[0] amplitude in px (0..4096), lo[1]
 *  log2 of the lattice spacing (2..8, 0 = 5); no random range.
 *  out_h/out_w: crop / pad / resize target size. */
typedef struct alb_sample_cfg {
  int32_t tid, out_h, out_w, reserved;
  double p;              /* probability the transform is applied */
  double lo[4], hi[4];
} alb_sample_cfg;

/* Configuration of the fused chain (alb_apply_batch). */
typedef struct alb_chain_cfg {
  int32_t out_h, out_w;  /* output size (224 x 224 for the ImageNet-style chain) */
  double mean[3];        /* Normalize mean per channel (fraction of 255) */
  double std[3];         /* Normalize std per channel (fraction of 255) */
  int32_t tile_h;        /* fused kernel: output rows per work item (1..32) */
  int32_t tile_w;        /* must be 0: a work item spans the full output width */
  int32_t ctas_per_sm;   /* fused kernel: resident CTAs per SM.  tile_h == 0 and
                            ctas_per_sm == 0: the schedule alb_autotune_batch cached
                            for this (device, out_h, out_w, batch-size bucket), else
                            8 rows at the occupancy limit */
  int32_t jitter;        /* colour jitter: 0 = brightness b then contrast c about 128 as one
                            table, then saturation s in float32 (not rounded); 1 = the three
                            ops in the record's random order k (0..5: BCS BSC CBS CSB SBC SCB),
                            each producing uint8: B v -> rne(b v); C v -> rne(m + c (v - m)),
                            m = rounded mean of the integer BT.601 grey of the image at that
                            point (a per-image reduction); S the float32 blend, rounded */
} alb_chain_cfg;        /* 72 bytes */

enum { ALB_MODE_FUSED = 0, ALB_MODE_PLAIN = 1 };

/* ------------------------------------------------------------------ */
/* Parameter sampling (Sec. II: each transform is applied with parameters drawn at
 * random).  Philox4x32-10 (Salmon et al., SC'11): the word stream of
 * image `index` is Philox blocks with counter (j, index, stream_id lo,
 * stream_id hi) and key seed; uniform doubles take 27+26 bits of two words;
 * integers use Lemire's multiply-shift with rejection.  The probability draw
 * comes first; size-changing transforms are always applied.  Host only;
 * `out` is a host pointer.  Returns ALB_ESHAPE when the transform cannot fit
 * (crop larger than the image). */
ALB_API alb_status alb_sample_params(const alb_sample_cfg* cfg, uint64_t seed, uint64_t stream_id,
                             uint32_t index, int32_t h, int32_t w, alb_params* out);

/* The same sampler as a device kernel for n images: image i uses index
 * first_index + i and the size in images_dev[i].  images_dev and params_dev
 * are device arrays of n entries.  A record that cannot fit writes
 * ALB_ESHAPE to dev_status (if non-NULL) and an identity record. */
ALB_API alb_status alb_sample_params_batch(const alb_sample_cfg* cfg, uint64_t seed, uint64_t stream_id,
                                   uint32_t first_index, int32_t n, const alb_image* images_dev,
                                   alb_params* params_dev, int32_t* dev_status, void* stream);

/* Output size of a transform with parameters p applied to an h x w input. */
ALB_API alb_status alb_output_shape(const alb_params* p, int32_t h, int32_t w, int32_t* out_h, int32_t* out_w);

/* Scratch bytes alb_apply / alb_apply_ragged need for n images of transform tid. */
ALB_API size_t alb_workspace_size(int32_t tid, int32_t n);

/* ------------------------------------------------------------------ */
/* Apply one transform to one image and, optionally, its mask and boxes
 * (Sec. II-A: masks and boxes are transformed together with the image;
 * Sec. II-B: binary masks follow the image geometry).
 *  params:  HOST pointer to one record.
 *  in/out:  HOST structs describing DEVICE images; out must have the size
 *           alb_output_shape gives and the same c.  NULL out skips the image.
 *           In-place (out->data == in->data) is allowed only for transforms
 *           that keep the size and move no pixels (LUT ops, ShiftHSV,
 *           Grayscale, Equalize).
 *  mask_in/mask_out: optional (NULL) mask of any c, same h x w as the image;
 *           geometric transforms resample it with nearest-neighbour, the
 *           others copy it unchanged.
 *  boxes_in: DEVICE float [n_boxes][4]; boxes_out: DEVICE float [n_boxes][4];
 *           n_boxes_out: DEVICE int32, the number of boxes kept (boxes left
 *           with no area after clipping are dropped, order kept).
 *  workspace: DEVICE scratch of alb_workspace_size(params->tid, 1) bytes. */
ALB_API alb_status alb_apply(const alb_params* params, const alb_image* in, const alb_image* out,
                     const alb_image* mask_in, const alb_image* mask_out,
                     const float* boxes_in, int32_t n_boxes, float* boxes_out, int32_t* n_boxes_out,
                     void* workspace, size_t workspace_bytes, void* stream);

/* Apply transform tid to a ragged batch of n images in one pass (the plain,
 * one-transform-per-launch GPU path).  All arrays are DEVICE arrays of n
 * entries: params_dev[i].tid must equal tid; out_dev[i] must have the
 * output size of params_dev[i].  Masks (optional, NULL) as in alb_apply.
 * Boxes (optional, NULL): boxes_dev is float [n][box_cap][4] with
 * n_boxes_dev[i] valid entries; results go to boxes_out_dev (same layout)
 * and n_boxes_out_dev. */
ALB_API alb_status alb_apply_ragged(int32_t tid, int32_t n, const alb_params* params_dev,
                            const alb_image* in_dev, const alb_image* out_dev,
                            const alb_image* mask_in_dev, const alb_image* mask_out_dev,
                            const float* boxes_dev, const int32_t* n_boxes_dev, int32_t box_cap,
                            float* boxes_out_dev, int32_t* n_boxes_out_dev,
                            void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream);

/* Allocation-free variant of alb_apply_ragged (images only: no masks, no
 * boxes).  The paper has no counterpart: this exists for callers that cannot
 * allocate device memory (an allocator callback, a process whose device
 * memory another framework has fully reserved, a real-time loop that forbids
 * allocation), so they cannot provide a workspace.  Scratch comes from one
 * static 8 MiB device array inside the library (held by every GPU that loads
 * the library until exit); at most 2048 images per call, more returns
 * ALB_ECAPACITY.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and should come before any stream capture;
 * the address is cached per CUDA context, so after cudaDeviceReset the next
 * call looks it up again (and should also come before any capture).
 * All calls share the array: calls that overlap on the GPU race and must be
 * ordered by the caller.  Arguments as in alb_apply_ragged; allocates nothing. */
ALB_API alb_status alb_apply_ragged_static(int32_t tid, int32_t n, const alb_params* params_dev,
                                           const alb_image* in_dev, const alb_image* out_dev,
                                           int32_t* dev_status, void* stream);

/* ------------------------------------------------------------------ */
/* The fused ragged-batch chain: per image, RandomResizedCrop window
 * resized (Q5 bilinear, half-pixel) to out_h x out_w, h-flip if
 * params.flip, brightness factor beta then contrast factor alpha about a
 * fixed pivot 128 as one per-image table, saturation blend in float32 with
 * factor sat, Normalize with float32 constants 1/(255 std), -mean/std,
 * bfloat16 round-to-nearest-even, written NCHW to out_bf16
 * [n][3][out_h][out_w].
 *  mode ALB_MODE_FUSED: one persistent kernel, each output pixel written
 *  once.  ALB_MODE_PLAIN: one kernel per step with materialised
 *  intermediates; bit-identical output.
 *  params_dev / in_dev: DEVICE arrays of n entries (params tid = ALB_CHAIN). */
ALB_API size_t alb_batch_workspace_size(const alb_chain_cfg* cfg, int32_t n, int32_t mode);
ALB_API alb_status alb_apply_batch(const alb_chain_cfg* cfg, int32_t n, const alb_params* params_dev,
                           const alb_image* in_dev, void* out_bf16, int32_t mode,
                           void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream);

/* The chain with its targets (Sec. II-A: a crop and flip applied to an image
 * and to its masks and boxes in the same way; Fig. 2 detection): as
 * alb_apply_batch, plus optional per-image instance-mask stacks and boxes.
 *  mask_in_dev / mask_out_dev: DEVICE arrays of n descriptors (both or
 *  neither): uint8 HWC with c = N instance planes (N >= 1, per image); the
 *  input mask has the image's h x w, the output out_h x out_w and the same N.
 *  A mask is resampled with the nearest rule of the mask resize through the
 *  same crop window and flip.  An image whose masks do not match records
 *  ALB_ESHAPE in dev_status and its masks are not written.
 *  boxes_dev: DEVICE float [n][box_cap][4] xyxy pixel-edge coordinates,
 *  n_boxes_dev [n]; boxes_out_dev / n_boxes_out_dev likewise: each box is
 *  cropped to the window (clipped there), scaled, flipped, clipped to the
 *  output and dropped when it has no area left; order kept.
 * Fused mode writes the masks from the fused kernel's work items; plain mode
 * in a launch of their own.  Workspace as for alb_apply_batch. */
ALB_API alb_status alb_apply_batch_targets(const alb_chain_cfg* cfg, int32_t n, const alb_params* params_dev,
                                   const alb_image* in_dev, void* out_bf16, const alb_image* mask_in_dev,
                                   const alb_image* mask_out_dev, const float* boxes_dev,
                                   const int32_t* n_boxes_dev, int32_t box_cap, float* boxes_out_dev,
                                   int32_t* n_boxes_out_dev, int32_t mode, void* workspace,
                                   size_t workspace_bytes, int32_t* dev_status, void* stream);

/* Box-safe crop windows for the chain (for detection): the chain's record
 * (cfg tid = ALB_CHAIN) with a crop window that contains the union of the
 * image's boxes, clipped to the image and widened to whole pixels
 * [ux0, ux1) x [uy0, uy1): x0 = randint[0, ux0], x1 = ux1 + randint[0, W - ux1],
 * then the same for y (integers by the sampler's rule); without boxes the
 * chain's RandomResizedCrop draw.  The flip and jitter draws follow as in
 * alb_sample_params.  Host form: boxes is a HOST float [n_boxes][4]; `out`
 * a host record.  Batch form: images_dev [n], boxes_dev [n][box_cap][4],
 * n_boxes_dev [n], params_dev [n] are DEVICE arrays; a count outside
 * [0, box_cap] records ALB_ECAPACITY and is clamped. */
ALB_API alb_status alb_sample_chain_box_safe(const alb_sample_cfg* cfg, uint64_t seed, uint64_t stream_id,
                                     uint32_t index, int32_t h, int32_t w, const float* boxes, int32_t n_boxes,
                                     alb_params* out);
ALB_API alb_status alb_sample_chain_box_safe_batch(const alb_sample_cfg* cfg, uint64_t seed, uint64_t stream_id,
                                           uint32_t first_index, int32_t n, const alb_image* images_dev,
                                           const float* boxes_dev, const int32_t* n_boxes_dev, int32_t box_cap,
                                           alb_params* params_dev, int32_t* dev_status, void* stream);

/* Autotuner of the fused kernel's schedule (the paper has no counterpart: it is
 * part of running the chain on a GPU).  Runs alb_apply_batch in fused mode once
 * as warm-up and `reps` times under CUDA events for every candidate (rows per
 * item in {2, 4, 8, 16, 32} x CTAs per SM in {occupancy limit, half of it}) on
 * the caller's own batch, keeps the fastest in a process-wide cache keyed by
 * (current device, out_h, out_w, ceil(log2 n)), and returns it in *best (a copy
 * of *cfg with tile_h and ctas_per_sm set).  Arguments as for alb_apply_batch
 * (workspace for ALB_MODE_FUSED); out_bf16 is overwritten with the chain's
 * output, identical for every schedule.  Synchronises `stream`: do not call it
 * while the stream is captured.  Errors: ALB_EINVAL / ALB_ESHAPE /
 * ALB_EWORKSPACE on bad arguments, ALB_ECUDA when a launch or timing fails. */
ALB_API alb_status alb_autotune_batch(const alb_chain_cfg* cfg, int32_t n, const alb_params* params_dev,
                              const alb_image* in_dev, void* out_bf16, void* workspace,
                              size_t workspace_bytes, int32_t reps, alb_chain_cfg* best, void* stream);

/* The schedule cache of alb_autotune_batch, read and persisted (no
 * counterpart in the paper).  alb_autotune_lookup: the cached schedule of
 * (current device, cfg->out_h, cfg->out_w, cfg->jitter, ceil(log2 n)) in
 * *best (a copy of *cfg with tile_h, ctas_per_sm set) and *found = 1, or
 * *found = 0 and *best = *cfg; host pointers.  alb_autotune_save: writes
 * every cached entry to the JSON file `path` (written to path.tmp, then
 * renamed), keyed by device name and SM count:
 *   {"format": "alb-autotune-1", "entries": [{"device": "...", "sms": N,
 *    "out_h": H, "out_w": W, "jitter": J, "bucket": K, "rows_per_item": R,
 *    "ctas_per_sm": C}, ...]}
 * alb_autotune_load: reads such a file, checks every entry (ALB_EINVAL, and
 * nothing loaded, if the file is missing, malformed or out of range), then
 * stores the entries whose device name and SM count match a device of this
 * process, replacing entries of the same key; *n_loaded receives their
 * number.  ALB_ECUDA when a device query fails.  None of them launches
 * work or allocates device memory. */
ALB_API alb_status alb_autotune_lookup(const alb_chain_cfg* cfg, int32_t n, alb_chain_cfg* best, int32_t* found);
ALB_API alb_status alb_autotune_save(const char* path);
ALB_API alb_status alb_autotune_load(const char* path, int32_t* n_loaded);

/* ------------------------------------------------------------------ */
/* Differentiable float32 path.  x: DEVICE float [B][C][H][W] (NCHW, values
 * nominally in [0,1]); prm: DEVICE float [B][4] = (angle in degrees, scale,
 * tx, ty) for the warp, [B][3] = (alpha, beta, gamma) for the photometric op.
 * Warp: the C6 map of the u8 warps in float32 with bilinear sampling and a
 * zero border.  Photometric: y = clamp(alpha x + beta, 0, 1)^gamma.
 * Backward kernels recompute sampling coordinates from prm (nothing is
 * stored by the forward), write the input gradient gx (same layout as x)
 * and ACCUMULATE nothing: gprm [B][4] / [B][3] is overwritten.  The warp's
 * input gradient is a gather over the forward's exact (output, weight)
 * pairs and every reduction runs in a fixed order, so both backward calls
 * are bitwise repeatable.  Limits: B <= 65535 and 4*H*W < 2^31 for the warp
 * (ALB_ESHAPE otherwise); workspace of alb_f32_workspace_size bytes for the
 * backward calls (ALB_EWORKSPACE when smaller). */
ALB_API size_t alb_f32_workspace_size(int32_t B, int32_t C, int32_t H, int32_t W);
ALB_API alb_status alb_warp_affine_f32_fwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                   const float* prm, float* y, void* stream);
ALB_API alb_status alb_warp_affine_f32_bwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                   const float* prm, const float* gy, float* gx, float* gprm,
                                   void* workspace, size_t workspace_bytes, void* stream);
ALB_API alb_status alb_photometric_f32_fwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                   const float* prm, float* y, void* stream);
ALB_API alb_status alb_photometric_f32_bwd(int32_t B, int32_t C, int32_t H, int32_t W, const float* x,
                                   const float* prm, const float* gy, float* gx, float* gprm,
                                   void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* Diagnostic (no counterpart in the paper: part of the library's failure
 * handling).  The bulk-copy kernels wait on their shared-memory barriers
 * with an iteration limit; when a wait gives up they wait (bounded again)
 * for the copies they had issued and not yet consumed, record ALB_ETIMEOUT
 * in their status word and stop.  This call runs that path on purpose: one
 * thread issues two 16-byte bulk loads from src_dev[0, 32) into two stages,
 * announces a third copy that it never issues, waits for the third with at
 * most `spins` tries (1 <= spins <= 2^22), drains the two real copies,
 * records ALB_ETIMEOUT in *dev_status (device int32, set only if it is 0)
 * and copies the two drained stages to out_dev[0, 32).  A caller sees a
 * working timeout path as *dev_status == ALB_ETIMEOUT and out == src.
 * src_dev must be 16-byte aligned (ALB_EALIGN otherwise); all pointers are
 * device pointers owned by the caller.  Asynchronous on `stream`. */
ALB_API alb_status alb_selftest_bounded_wait(int32_t spins, const void* src_dev, void* out_dev,
                                             int32_t* dev_status, void* stream);

/* Diagnostic (no counterpart in the paper).  In the bounds-checked build of
 * the library (compiled with ALB_CHECK_BOUNDS) every instrumented gather,
 * staging copy and store of the resampling, chain, index-map and float warp
 * kernels tests its index or address against the region it must stay in; a
 * failing check skips the access and is counted on the device.  This call
 * adds up the counts of every kernel file into *count (host), puts the source
 * line of the first failing check into *first_line (0 if none), clears the
 * counters when reset != 0, and sets *checked to 1 in the checked build, 0 in
 * the normal build (whose counts are always 0).  Synchronous (it reads device
 * memory); ALB_ECUDA when that fails. */
ALB_API alb_status alb_bounds_violations(uint32_t* count, uint32_t* first_line, int32_t reset, int32_t* checked);

/* ------------------------------------------------------------------ */
/* Thread-local message for the last failing call on this thread. */
ALB_API const char* alb_last_error(void);
/* Library version, e.g. "alb 1.0 sm_103a". */
ALB_API const char* alb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ALB_H */
