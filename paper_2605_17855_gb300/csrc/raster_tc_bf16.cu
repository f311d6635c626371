// Tensor-core rasterizer, BF16 operands: the coefficients split three ways (hi + mid + lo) over two
// K blocks of 16 (K = 32), since BF16 keeps 8 significand bits against FP16's 11. The kernel itself
// is in raster_tc_impl.cuh; this translation unit holds its BF16 instantiations.
#include "raster_tc_impl.cuh"

namespace tgs {

tgs_status launch_raster_tc_bf16(const tgs_projected& p, const tgs_bins& b, int width, int height,
                                 int gw, int gh, const tgs_raster_opts& o, float* out_rgb,
                                 float* out_T, int32_t* n_contrib, cudaStream_t st) {
  return launch_raster_tc_typed<true>(p, b, width, height, gw, gh, o, out_rgb, out_T, n_contrib, st);
}

tgs_status launch_raster_tc_batch_bf16(const RasterFrame* frames, int count, int gw, int gh,
                                       const tgs_raster_opts& o, int* next_item, uint64_t wait_ns,
                                       cudaStream_t st, int share_div) {
  return launch_raster_tc_batch_typed<true>(frames, count, gw, gh, o, next_item, wait_ns, st,
                                            share_div);
}

}  // namespace tgs
