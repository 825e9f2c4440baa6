// Instantiation of the tile kernels for degree 2 (one translation unit per
// degree keeps the parallel build short).
#include "tile_kernels.cuh"

namespace mfcg {
cudaError_t launch_tile_deg2(int mode, const TileArgs& a, const OperatorCoeffs& c, cudaStream_t s) {
  return launch_tile_p<2>(mode, a, c, s);
}
cudaError_t launch_tail_deg2(int mode, const TileArgs& a, cudaStream_t s) { return launch_tail_p<2>(mode, a, s); }
cudaError_t prepare_tile_deg2(int geom, int prec, size_t smem) { return prepare_tile_p<2>(geom, prec, smem); }
int tile_occupancy_deg2(int mode, int geom, int prec, int ncomp, size_t smem) {
  return tile_occupancy_p<2>(mode, geom, prec, ncomp, smem);
}
}  // namespace mfcg
