// Instantiation of the tile kernels for degree 3 (one translation unit per
// degree keeps the parallel build short).
#include "tile_kernels.cuh"

namespace mfcg {
cudaError_t launch_tile_deg3(int mode, const TileArgs& a, const OperatorCoeffs& c, cudaStream_t s) {
  return launch_tile_p<3>(mode, a, c, s);
}
cudaError_t launch_tail_deg3(int mode, const TileArgs& a, cudaStream_t s) { return launch_tail_p<3>(mode, a, s); }
cudaError_t prepare_tile_deg3(int geom, int prec, size_t smem) { return prepare_tile_p<3>(geom, prec, smem); }
int tile_occupancy_deg3(int mode, int geom, int prec, int ncomp, size_t smem) {
  return tile_occupancy_p<3>(mode, geom, prec, ncomp, smem);
}
}  // namespace mfcg
