// Degree dispatch of the tile kernels (the kernels themselves are instantiated
// one degree per translation unit in tile_p<degree>.cu).
#include "tile_kernels.cuh"

namespace mfcg {

#define MFCG_DECLARE_DEG(P)                                                                         \
  cudaError_t launch_tile_deg##P(int mode, const TileArgs& a, const OperatorCoeffs& c, cudaStream_t s); \
  cudaError_t launch_tail_deg##P(int mode, const TileArgs& a, cudaStream_t s);                      \
  cudaError_t prepare_tile_deg##P(int geom, int prec, size_t smem);                                 \
  int tile_occupancy_deg##P(int mode, int geom, int prec, int ncomp, size_t smem);
MFCG_DECLARE_DEG(1)
MFCG_DECLARE_DEG(2)
MFCG_DECLARE_DEG(3)
MFCG_DECLARE_DEG(4)
MFCG_DECLARE_DEG(5)
MFCG_DECLARE_DEG(6)
MFCG_DECLARE_DEG(7)
MFCG_DECLARE_DEG(8)
#undef MFCG_DECLARE_DEG

cudaError_t launch_tile(int degree, int mode, const TileArgs& a, const OperatorCoeffs& c, cudaStream_t s) {
  switch (degree) {
    case 1: return launch_tile_deg1(mode, a, c, s);
    case 2: return launch_tile_deg2(mode, a, c, s);
    case 3: return launch_tile_deg3(mode, a, c, s);
    case 4: return launch_tile_deg4(mode, a, c, s);
    case 5: return launch_tile_deg5(mode, a, c, s);
    case 6: return launch_tile_deg6(mode, a, c, s);
    case 7: return launch_tile_deg7(mode, a, c, s);
    case 8: return launch_tile_deg8(mode, a, c, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tail(int degree, int mode, const TileArgs& a, cudaStream_t s) {
  switch (degree) {
    case 1: return launch_tail_deg1(mode, a, s);
    case 2: return launch_tail_deg2(mode, a, s);
    case 3: return launch_tail_deg3(mode, a, s);
    case 4: return launch_tail_deg4(mode, a, s);
    case 5: return launch_tail_deg5(mode, a, s);
    case 6: return launch_tail_deg6(mode, a, s);
    case 7: return launch_tail_deg7(mode, a, s);
    case 8: return launch_tail_deg8(mode, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prepare_tile(int degree, int geom, int prec, size_t smem) {
  switch (degree) {
    case 1: return prepare_tile_deg1(geom, prec, smem);
    case 2: return prepare_tile_deg2(geom, prec, smem);
    case 3: return prepare_tile_deg3(geom, prec, smem);
    case 4: return prepare_tile_deg4(geom, prec, smem);
    case 5: return prepare_tile_deg5(geom, prec, smem);
    case 6: return prepare_tile_deg6(geom, prec, smem);
    case 7: return prepare_tile_deg7(geom, prec, smem);
    case 8: return prepare_tile_deg8(geom, prec, smem);
    default: return cudaErrorInvalidValue;
  }
}

int tile_occupancy(int degree, int mode, int geom, int prec, int ncomp, size_t smem) {
  switch (degree) {
    case 1: return tile_occupancy_deg1(mode, geom, prec, ncomp, smem);
    case 2: return tile_occupancy_deg2(mode, geom, prec, ncomp, smem);
    case 3: return tile_occupancy_deg3(mode, geom, prec, ncomp, smem);
    case 4: return tile_occupancy_deg4(mode, geom, prec, ncomp, smem);
    case 5: return tile_occupancy_deg5(mode, geom, prec, ncomp, smem);
    case 6: return tile_occupancy_deg6(mode, geom, prec, ncomp, smem);
    case 7: return tile_occupancy_deg7(mode, geom, prec, ncomp, smem);
    case 8: return tile_occupancy_deg8(mode, geom, prec, ncomp, smem);
    default: return 0;
  }
}

size_t tile_smem_bytes(int degree, int geom, int prec, const TileGeom& g, int mode) {
  return tile_smem_elems(degree, geom, prec_bytes(prec), g, mode, prec) * prec_bytes(prec);
}

}  // namespace mfcg
