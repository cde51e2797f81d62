// alb_kernels.cuh -- host launchers shared between the libalb translation units.
#pragma once

#include "alb_common.cuh"

namespace alb {

// alb_geom.cu
alb_status launch_geometric(int32_t tid, const Plan& plan, const ImgList& in, const ImgList& out,
                            const PrmList& prm, int32_t channels, bool mask, int32_t* status, cudaStream_t st);
alb_status launch_boxes(int32_t n, const PrmList& prm, const ImgList& in, const float* boxes, const int32_t* nbox,
                        int32_t cap, int32_t single_n, float* out, int32_t* nout, int32_t* status, cudaStream_t st);

// alb_stream.cu (vectorised streaming kernels)
alb_status launch_stream_geometric(int32_t tid, const Plan& plan, const ImgList& in, const ImgList& out,
                                   const PrmList& prm, int32_t channels, cudaStream_t st);
alb_status launch_stream_lut(const Plan& plan, const ImgList& in, const ImgList& out, const uint8_t* luts,
                             int32_t* status, cudaStream_t st);
alb_status launch_stream_pixel(int32_t tid, const Plan& plan, const ImgList& in, const ImgList& out,
                               const PrmList& prm, int32_t* status, cudaStream_t st);
alb_status launch_stream_hist(const Plan& plan, const ImgList& in, uint32_t* hist, int32_t* status,
                              cudaStream_t st);
alb_status launch_wait_selftest(uint32_t spins, const uint8_t* src, uint8_t* out, int32_t* status,
                                cudaStream_t st);

// alb_resample.cu (tiled warps and resizes)
alb_status launch_tile_geometric(int32_t tid, const Plan& plan, const ImgList& in, const ImgList& out,
                                 const PrmList& prm, int32_t channels, bool mask, const PlanCheck& chk,
                                 cudaStream_t st);

// alb_color.cu
alb_status launch_photometric(int32_t tid, int32_t n, const Plan& plan, const ImgList& in, const ImgList& out,
                              const PrmList& prm, uint8_t* luts, uint32_t* hist, int32_t* status,
                              cudaStream_t st);

// alb_fused.cu
alb_status launch_chain(const alb_chain_cfg& cfg, int32_t n, const alb_params* params, const alb_image* in,
                        void* out, int32_t mode, Carve& ws, int32_t* status, cudaStream_t st,
                        const alb_image* mask_in = nullptr, const alb_image* mask_out = nullptr);
size_t chain_workspace(const alb_chain_cfg& cfg, int32_t n, int32_t mode);

// per translation unit: the bounds-checked build's violation counters (count
// added to *count, first failing source line into *line when it is 0)
alb_status oob_resample(unsigned int* count, unsigned int* line, bool reset);
alb_status oob_fused(unsigned int* count, unsigned int* line, bool reset);
alb_status oob_geom(unsigned int* count, unsigned int* line, bool reset);
alb_status oob_diff(unsigned int* count, unsigned int* line, bool reset);

inline bool is_geometric(int32_t tid) {
  switch (tid) {
    case ALB_HFLIP: case ALB_VFLIP: case ALB_RANDOM_CROP: case ALB_PAD_TO_SIZE: case ALB_ROTATE:
    case ALB_SHIFT_SCALE_ROTATE: case ALB_RESIZE: case ALB_RANDOM_SIZED_CROP: case ALB_RANDOM_RESIZED_CROP:
    case ALB_TRANSPOSE: case ALB_ROT90: case ALB_GRID_DISTORTION: case ALB_ELASTIC:
      return true;
    default:
      return false;
  }
}
inline bool uses_lut(int32_t tid) {
  switch (tid) {
    case ALB_BRIGHTNESS: case ALB_CONTRAST: case ALB_BRIGHTNESS_CONTRAST: case ALB_GAMMA: case ALB_SHIFT_RGB:
    case ALB_EQUALIZE:
      return true;
    default:
      return false;
  }
}

}  // namespace alb
