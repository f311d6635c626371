// Tensor-core rasterizer, FP16 operands (hi + lo coefficient split in one K block of 16), and the
// dispatch to the BF16 variant. The kernel itself is in raster_tc_impl.cuh.
#include "raster_tc_impl.cuh"

namespace tgs {

tgs_status launch_raster_tc(const tgs_projected& p, const tgs_bins& b, int width, int height, int gw,
                            int gh, const tgs_raster_opts& o, float* out_rgb, float* out_T,
                            int32_t* n_contrib, cudaStream_t st) {
  if (o.precision == TGS_PRECISION_BF16_TC)
    return launch_raster_tc_bf16(p, b, width, height, gw, gh, o, out_rgb, out_T, n_contrib, st);
  return launch_raster_tc_typed<false>(p, b, width, height, gw, gh, o, out_rgb, out_T, n_contrib, st);
}

tgs_status launch_raster_tc_batch(const RasterFrame* frames, int count, int gw, int gh,
                                  const tgs_raster_opts& o, int* next_item, uint64_t wait_ns,
                                  cudaStream_t st, int share_div) {
  if (o.precision == TGS_PRECISION_BF16_TC)
    return launch_raster_tc_batch_bf16(frames, count, gw, gh, o, next_item, wait_ns, st, share_div);
  return launch_raster_tc_batch_typed<false>(frames, count, gw, gh, o, next_item, wait_ns, st,
                                             share_div);
}

}  // namespace tgs
