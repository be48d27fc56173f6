// Instantiation of the step / field kernels for one storage type.  Included
// by lbe_step_<storage>.cu with LBE_ST (policy), LBE_SUFFIX and LBE_ALL_TILES
// defined.
#include "lbe_launch.h"
#include "lbe_tile.cuh"
#if LBE_STASH
#include "lbe_stash.cuh"
#endif

#define LBE_CAT2(a, b) a##b
#define LBE_CAT(a, b) LBE_CAT2(a, b)

namespace lbe {

namespace {
template <int TX, int TY>
cudaError_t launch_one(const InstDev* d, int n, int64_t total, int parity, int grid,
                       const uint32_t* seed, cudaStream_t s) {
  if (grid <= 0) grid = 1;
  if ((int64_t)grid > total) grid = (int)total;
  tile_kernel<LBE_ST, TX, TY, 0><<<grid, TX * TY, 0, s>>>(d, n, total, parity, nullptr, seed);
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
                                               int parity, int grid, const uint32_t* seed,
                                               cudaStream_t s) {
  switch (tile) {
    case 0: return launch_one<32, 8>(d, n, total, parity, grid, seed, s);
#if LBE_ALL_TILES
    case 1: return launch_one<64, 4>(d, n, total, parity, grid, seed, s);
    case 2: return launch_one<32, 16>(d, n, total, parity, grid, seed, s);
    case 3: return launch_one<64, 8>(d, n, total, parity, grid, seed, s);
    case 4: return launch_one<128, 4>(d, n, total, parity, grid, seed, s);
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

#if LBE_PCORR
// Varying density: the corrected p of every cell of every instance into its
// pcorr (tiles of shape 0 over a work list of that shape), before the step.
cudaError_t LBE_CAT(pcorr_, LBE_SUFFIX)(const InstDev* d, int n, int64_t total, int parity,
                                         int grid, cudaStream_t s) {
  if (grid <= 0) grid = 1;
  if ((int64_t)grid > total) grid = (int)total;
  tile_kernel<LBE_ST, 32, 8, 2><<<grid, 256, 0, s>>>(d, n, total, parity, nullptr, nullptr);
  return cudaGetLastError();
}
#endif

cudaError_t LBE_CAT(fields_, LBE_SUFFIX)(const InstDev* d, int64_t tiles, int parity, double* out,
                                          cudaStream_t s) {
  if (tiles <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)(tiles < 2147483647 ? tiles : 2147483647);
  tile_kernel<LBE_ST, 32, 8, 1><<<grid, 256, 0, s>>>(d, 1, tiles, parity, out, nullptr);
  return cudaGetLastError();
}

#if LBE_STASH
namespace {
template <int NC, bool VAR, bool OWN>
bool stash_attr() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  if (!done[dev]) {
    if (cudaFuncSetAttribute(stash_kernel<LBE_ST, NC, VAR, OWN>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             StashCfg<LBE_ST, NC>::SMEM) != cudaSuccess)
      return false;
    done[dev] = true;
  }
  return true;
}
template <int NC, bool VAR, bool OWN>
cudaError_t stash_one(const InstDev* d, int n, int64_t items, int seg, int parity, int grid,
                      int* err, int poll_lim, int withhold, const uint32_t* seed,
                      cudaStream_t s) {
  if (!stash_attr<NC, VAR, OWN>()) return cudaErrorInvalidValue;
  if (grid <= 0) grid = 1;
  if ((int64_t)grid > items) grid = (int)items;
  stash_kernel<LBE_ST, NC, VAR, OWN>
      <<<grid, NC, StashCfg<LBE_ST, NC>::SMEM, s>>>(d, n, items, seg, parity, err, poll_lim,
                                                    withhold, seed);
  return cudaGetLastError();
}
template <int NC, bool VAR, bool OWN>
int stash_occ() {
  if (!stash_attr<NC, VAR, OWN>()) return 0;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, stash_kernel<LBE_ST, NC, VAR, OWN>, NC,
                                                    StashCfg<LBE_ST, NC>::SMEM) != cudaSuccess)
    return 0;
  return b;
}
}  // namespace

cudaError_t LBE_CAT(launch_stash_, LBE_SUFFIX)(const InstDev* d, int n, int64_t items, int seg,
                                                int parity, int grid, int* err, int poll_lim,
                                                int withhold, const uint32_t* seed, bool var,
                                                bool own_ghosts, cudaStream_t s) {
#define LBE_STASH_ONE(V, O) \
  stash_one<128, V, O>(d, n, items, seg, parity, grid, err, poll_lim, withhold, seed, s)
  if (var) return own_ghosts ? LBE_STASH_ONE(true, true) : LBE_STASH_ONE(true, false);
  return own_ghosts ? LBE_STASH_ONE(false, true) : LBE_STASH_ONE(false, false);
#undef LBE_STASH_ONE
}
// resident CTAs per SM (the smaller of the two builds)
int LBE_CAT(stash_occupancy_, LBE_SUFFIX)() {
  const int o[4] = {stash_occ<128, false, false>(), stash_occ<128, true, false>(),
                    stash_occ<128, false, true>(), stash_occ<128, true, true>()};
  int m = o[0];
  for (int j = 1; j < 4; j++) m = o[j] < m ? o[j] : m;
  return m;
}
#endif

}  // namespace lbe
