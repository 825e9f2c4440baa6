// Operator application that performs no device allocation.
//
// mfcg_setup allocates every work buffer of a problem with cudaMalloc.  Some
// callers cannot do that: programs that hand all device memory to their own
// pool allocator at start-up and may not allocate behind its back, and
// latency-sensitive loops that must not call cudaMalloc/cudaFree because those
// calls can synchronise the whole device.  mfcg_apply_operator_static serves
// them: it computes dst = A src for an affine (Cartesian) mesh in FP64 with
// the same kernels and the same vector ordering as mfcg_apply_operator on a
// problem set up with default options, and keeps the only scratch it needs --
// the partial sums of the nodes shared between tiles -- in a fixed array in
// device memory that every GPU loading the library holds until the process
// exits.
//
// The kernels are instantiated in this translation unit, so their launch
// attributes are independent of the ones mfcg_setup sets for its own copies.
#include <mutex>

#include "tile_kernels.cuh"

namespace mfcg {
void build_coeffs(int p, const double h[3], double amplitude, int coef, OperatorCoeffs& c);
}  // namespace mfcg

using namespace mfcg;

namespace {

// 16 MiB of face partials: for example Q4 on up to about 40^3 cells, Q2 on 84^3.
constexpr size_t kStaticScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
size_t g_smem_set[kMaxDevices][kMaxDegree + 1] = {};
int g_ahead[kMaxDevices][kMaxDegree + 1];  // prefetch distance per device and degree, -1 = not yet queried
int g_max_smem[kMaxDevices] = {};
int g_n_sm[kMaxDevices] = {};
std::mutex g_mutex;

// default tile edge per degree of affine problems (the table mfcg_setup uses)
int default_affine_tile(int p) {
  static const int t[9] = {0, 16, 8, 5, 4, 3, 3, 2, 2};
  return t[p];
}

// shared memory of the kernel's launch, and whether it fits the device's opt-in limit
template <int P>
size_t static_operator_smem(const TileGeom& g) {
  return tile_smem_elems(P, GEOM_AFFINE, (int)sizeof(double), g, MODE_OPERATOR) * sizeof(double);
}

template <int P>
cudaError_t launch_static_operator(TileArgs& a, const OperatorCoeffs& c, cudaStream_t s, size_t& smem_set,
                                   int n_sm, int& ahead) {
  auto tile = tile_kernel<P, MODE_OPERATOR, GEOM_AFFINE, PREC_F64, 1>;
  const size_t smem = static_operator_smem<P>(a.g);
  if (smem > smem_set) {
    const cudaError_t e = cudaFuncSetAttribute(tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  if (ahead < 0) {
    // L2 look-ahead prefetch distance of the regular operator pass: the CTAs
    // resident in one wave (an occupancy query allocates nothing)
    int occ = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tile, kThreads, smem);
    if (e != cudaSuccess) return e;
    ahead = n_sm * occ;
  }
  a.prefetch_ahead = ahead;
  tile<<<(unsigned)a.g.n_tiles, kThreads, smem, s>>>(a, c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tail_kernel<P, MODE_OPERATOR, PREC_F64><<<(unsigned)a.tail_ctas, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

extern "C" int mfcg_apply_operator_static(const mfcg_mesh* mesh, int degree, const double* src, double* dst,
                                          void* cuda_stream) {
  if (!mesh || !src || !dst || src == dst) return MFCG_INVALID_ARG;
  if (degree < 1 || degree > kMaxDegree) return MFCG_UNSUPPORTED_DEGREE;
  if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || mesh->amplitude != 0.0) return MFCG_INVALID_ARG;
  const int N[3] = {mesh->nx, mesh->ny, mesh->nz};
  for (int d = 0; d < 3; ++d)
    if ((int64_t)degree * N[d] + 1 > (1 << 20)) return MFCG_INVALID_ARG;
  int T[3];
  for (int d = 0; d < 3; ++d) T[d] = default_affine_tile(degree);
  // mfcg_setup's default FP64 tiles at degree 4 are 4 x 4 x 3 cells (the
  // shape of its tensor-core operator): the same vector order here
  if (degree == 4) T[2] = 3;
  TileArgs a{};
  init_tile_geom(degree, N, T, a.g, a.fam, &a.tdiv);
  if ((size_t)a.g.n_tiles * (size_t)a.g.face_stride * sizeof(double) > kStaticScratchBytes)
    return MFCG_SCRATCH_TOO_SMALL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MFCG_CUDA_ERROR;

  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    // first call on this device: the device address of the static array and
    // the device limits (none of these queries allocates)
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return MFCG_CUDA_ERROR;
    if (cudaDeviceGetAttribute(&g_max_smem[dev], cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g_n_sm[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return MFCG_CUDA_ERROR;
    for (int q = 0; q <= kMaxDegree; ++q) g_ahead[dev][q] = -1;
    g_scratch_addr[dev] = ptr;
  }
  // a tile that does not fit the shared memory of one CTA is an argument
  // error, as in mfcg_setup (the static shared arrays of the kernel included)
  {
    const size_t static_smem = 8 * (kThreads / 32) * sizeof(double) + 2 * kMaxColorCells * sizeof(int);
    size_t smem = 0;
    switch (degree) {
      case 1: smem = static_operator_smem<1>(a.g); break;
      case 2: smem = static_operator_smem<2>(a.g); break;
      case 3: smem = static_operator_smem<3>(a.g); break;
      case 4: smem = static_operator_smem<4>(a.g); break;
      case 5: smem = static_operator_smem<5>(a.g); break;
      case 6: smem = static_operator_smem<6>(a.g); break;
      case 7: smem = static_operator_smem<7>(a.g); break;
      case 8: smem = static_operator_smem<8>(a.g); break;
    }
    if (smem + static_smem > (size_t)g_max_smem[dev]) return MFCG_INVALID_ARG;
  }
  a.tail_nodes = a.fam[0] + a.fam[1] + a.fam[2];
  const int64_t ctas = (a.tail_nodes + 4 * kThreads - 1) / (4 * kThreads);
  a.tail_ctas = (int)(ctas < 1 ? 1 : (ctas > 152 * 16 ? 152 * 16 : ctas));
  a.shell = g_scratch_addr[dev];
  a.in0 = src;
  a.out0 = dst;
  a.geom = GEOM_AFFINE;
  a.prec = PREC_F64;
  a.ncomp = 1;
  a.op_kind = OP_LAPLACE;
  a.comp_stride = a.g.n_dofs;
  a.shell_comp_stride = a.g.n_tiles * a.g.face_stride;
  OperatorCoeffs c{};
  const double h[3] = {1.0 / N[0], 1.0 / N[1], 1.0 / N[2]};
  build_coeffs(degree, h, 0.0, MFCG_COEF_CONSTANT, c);
  const cudaStream_t s = (cudaStream_t)cuda_stream;
  size_t& smem_set = g_smem_set[dev][degree];
  int& ahead = g_ahead[dev][degree];
  const int n_sm = g_n_sm[dev];
  cudaError_t e = cudaErrorInvalidValue;
  switch (degree) {
    case 1: e = launch_static_operator<1>(a, c, s, smem_set, n_sm, ahead); break;
    case 2: e = launch_static_operator<2>(a, c, s, smem_set, n_sm, ahead); break;
    case 3: e = launch_static_operator<3>(a, c, s, smem_set, n_sm, ahead); break;
    case 4: e = launch_static_operator<4>(a, c, s, smem_set, n_sm, ahead); break;
    case 5: e = launch_static_operator<5>(a, c, s, smem_set, n_sm, ahead); break;
    case 6: e = launch_static_operator<6>(a, c, s, smem_set, n_sm, ahead); break;
    case 7: e = launch_static_operator<7>(a, c, s, smem_set, n_sm, ahead); break;
    case 8: e = launch_static_operator<8>(a, c, s, smem_set, n_sm, ahead); break;
  }
  return e == cudaSuccess ? MFCG_OK : MFCG_CUDA_ERROR;
}
