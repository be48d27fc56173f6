// Instantiation of the step / field kernels for one storage type.  Included
// by lbe_step_<storage>.cu with LBE_ST (policy), LBE_SUFFIX and LBE_ALL_TILES
// defined.
#include "lbe_launch.h"
#include "lbe_tile.cuh"
#if LBE_STRIP
#include "lbe_strip.cuh"
#endif
#if LBE_STASH
#include "lbe_stash.cuh"
#endif

#define LBE_CAT2(a, b) a##b
#define LBE_CAT(a, b) LBE_CAT2(a, b)

namespace lbe {

namespace {
template <int TX, int TY>
cudaError_t launch_one(const InstDev* d, int n, int64_t total, int parity, int grid,
                       cudaStream_t s) {
  if (grid <= 0) grid = 1;
  if ((int64_t)grid > total) grid = (int)total;
  tile_kernel<LBE_ST, TX, TY, 0><<<grid, TX * TY, 0, s>>>(d, n, total, parity, nullptr);
  return cudaGetLastError();
}
template <int TX, int TY>
int occ_one() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, tile_kernel<LBE_ST, TX, TY, 0>, TX * TY,
                                                    0) != cudaSuccess)
    return 0;
  return b;
}
}  // namespace

cudaError_t LBE_CAT(launch_step_, LBE_SUFFIX)(int tile, const InstDev* d, int n, int64_t total,
                                               int parity, int grid, cudaStream_t s) {
  switch (tile) {
    case 0: return launch_one<32, 8>(d, n, total, parity, grid, s);
#if LBE_ALL_TILES
    case 1: return launch_one<64, 4>(d, n, total, parity, grid, s);
    case 2: return launch_one<32, 16>(d, n, total, parity, grid, s);
    case 3: return launch_one<64, 8>(d, n, total, parity, grid, s);
    case 4: return launch_one<128, 4>(d, n, total, parity, grid, s);
#endif
    default: return cudaErrorInvalidValue;
  }
}

int LBE_CAT(occupancy_, LBE_SUFFIX)(int tile) {
  switch (tile) {
    case 0: return occ_one<32, 8>();
#if LBE_ALL_TILES
    case 1: return occ_one<64, 4>();
    case 2: return occ_one<32, 16>();
    case 3: return occ_one<64, 8>();
    case 4: return occ_one<128, 4>();
#endif
    default: return 0;
  }
}

cudaError_t LBE_CAT(fields_, LBE_SUFFIX)(const InstDev* d, int64_t tiles, int parity, double* out,
                                          cudaStream_t s) {
  if (tiles <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)(tiles < 2147483647 ? tiles : 2147483647);
  tile_kernel<LBE_ST, 32, 8, 1><<<grid, 256, 0, s>>>(d, 1, tiles, parity, out);
  return cudaGetLastError();
}

#if LBE_STRIP
namespace {
template <int NC, int R>
bool strip_attr() {
  // the dynamic shared-memory opt-in, once per device
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  if (!done[dev]) {
    if (cudaFuncSetAttribute(strip_kernel<LBE_ST, NC, R>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Strip<LBE_ST, NC, R>::SMEM) != cudaSuccess)
      return false;
    done[dev] = true;
  }
  return true;
}
template <int NC, int R>
cudaError_t strip_one(const InstDev* d, const TmapSet* maps, int n, int64_t items, int seg,
                      int parity, int grid, int* err, cudaStream_t s) {
  if (!strip_attr<NC, R>()) return cudaErrorInvalidValue;
  if (grid <= 0) grid = 1;
  if ((int64_t)grid > items) grid = (int)items;
  strip_kernel<LBE_ST, NC, R>
      <<<grid, NC, Strip<LBE_ST, NC, R>::SMEM, s>>>(d, maps, n, items, seg, parity, err);
  return cudaGetLastError();
}
template <int NC, int R>
int strip_occ() {
  if (!strip_attr<NC, R>()) return 0;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, strip_kernel<LBE_ST, NC, R>, NC,
                                                    Strip<LBE_ST, NC, R>::SMEM) != cudaSuccess)
    return 0;
  return b;
}
}  // namespace

#if LBE_STASH
namespace {
template <int NC>
bool stash_attr() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  if (!done[dev]) {
    if (cudaFuncSetAttribute(stash_kernel<LBE_ST, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             StashCfg<LBE_ST, NC>::SMEM) != cudaSuccess)
      return false;
    done[dev] = true;
  }
  return true;
}
template <int NC>
cudaError_t stash_one(const InstDev* d, const TmapSet* maps, int n, int64_t items, int seg,
                      int parity, int grid, int* err, cudaStream_t s) {
  if (!stash_attr<NC>()) return cudaErrorInvalidValue;
  if (grid <= 0) grid = 1;
  if ((int64_t)grid > items) grid = (int)items;
  stash_kernel<LBE_ST, NC>
      <<<grid, NC, StashCfg<LBE_ST, NC>::SMEM, s>>>(d, maps, n, items, seg, parity, err);
  return cudaGetLastError();
}
template <int NC>
int stash_occ() {
  if (!stash_attr<NC>()) return 0;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, stash_kernel<LBE_ST, NC>, NC,
                                                    StashCfg<LBE_ST, NC>::SMEM) != cudaSuccess)
    return 0;
  return b;
}
}  // namespace
#endif

cudaError_t LBE_CAT(launch_strip_, LBE_SUFFIX)(int variant, const InstDev* d, const TmapSet* maps,
                                                int n, int64_t items, int seg, int parity, int grid,
                                                int* err, cudaStream_t s) {
  switch (variant) {
    case 0: return strip_one<128, LBE_R128>(d, maps, n, items, seg, parity, grid, err, s);
    case 1: return strip_one<64, LBE_R64>(d, maps, n, items, seg, parity, grid, err, s);
#if LBE_STASH
    case 2: return stash_one<128>(d, maps, n, items, seg, parity, grid, err, s);
#endif
    default: return cudaErrorInvalidValue;
  }
}
int LBE_CAT(strip_occupancy_, LBE_SUFFIX)(int variant) {
  switch (variant) {
    case 0: return strip_occ<128, LBE_R128>();
    case 1: return strip_occ<64, LBE_R64>();
#if LBE_STASH
    case 2: return stash_occ<128>();
#endif
    default: return 0;
  }
}
#endif

}  // namespace lbe
