// Internal interface between the host API and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbe_common.cuh"

namespace lbe {

struct TileShape {
  int tx, ty;
};
// Kernel ids: 0..4 tile kernel with these tile shapes; 5, 6 retired (strip
// kernels with a TMA ring of whole source rows, superseded by the stash
// kernel; not built); 7 strip kernel with a per-warp stash of pulled
// populations, 128 output columns (16/32-bit storages; ty = 0: a strip
// marches over its rows), the periodic ghost columns refreshed by
// ghost_kernel after the step; 8 the same kernel writing the ghost columns
// itself (the owner of an edge cell stores it twice).
constexpr int NUM_TILE_SHAPES = 5;
constexpr int NUM_TILES = 9;
constexpr int STRIP_FIRST = 5;
constexpr int STASH_ID = 7;
constexpr int STASH_OWN_ID = 8;
// bytes allocated after an instance's two population buffers, covering the
// widest read past the end of a row of the stash kernel: a stash row of 136
// elements of up to 8 bytes from a strip start x0 <= nx - 1, against a
// pitch of at least nx + 8 elements (at most 127 x 8 bytes)
constexpr size_t ARENA_TAIL = 2048;
constexpr TileShape TILE_SHAPES[NUM_TILES] = {{32, 8},  {64, 4},  {32, 16}, {64, 8},
                                              {128, 4}, {124, 0}, {60, 0},  {128, 0},
                                              {128, 0}};
inline bool is_strip(int tile) { return tile >= STRIP_FIRST && tile < NUM_TILES; }
inline bool is_stash(int tile) { return tile == STASH_ID || tile == STASH_OWN_ID; }

// Does the step kernel of this storage exist for this kernel id?
bool tile_available(int storage, int tile);

// Stash strip kernel (16/32-bit storages): one step of every instance over
// `items` work items (strips x segments of seg rows); reads buf[parity],
// writes buf[parity ^ 1]; *err is set if a copy wait runs out of its
// poll_lim polls.  withhold >= 0 (test hook): the copies of that source row
// are not issued, so that the waits for it run out.
constexpr int STASH_POLLS = 1 << 22;       // polls of one bounded copy wait
constexpr int STASH_POLLS_TEST = 1 << 12;  // with the withhold test hook
// seed: the handle's step counter (device), read for the random bits of the
// stochastic rounding of the 16-bit forms.  var: some instance uses a
// boundary or property variant (the kernel built with them).
cudaError_t launch_stash(int storage, const InstDev* d, int n, int64_t items, int seg, int parity,
                         int grid, int* err, int poll_lim, int withhold, const uint32_t* seed,
                         bool var, bool own_ghosts, cudaStream_t s);
int stash_occupancy(int storage);
cudaError_t launch_stash_f32(const InstDev* d, int n, int64_t items, int seg, int parity, int grid,
                             int* err, int poll_lim, int withhold,
                             const uint32_t* seed, bool var,
                             bool own_ghosts, cudaStream_t s);
cudaError_t launch_stash_f16(const InstDev* d, int n, int64_t items, int seg, int parity, int grid,
                             int* err, int poll_lim, int withhold,
                             const uint32_t* seed, bool var,
                             bool own_ghosts, cudaStream_t s);
cudaError_t launch_stash_bf16(const InstDev* d, int n, int64_t items, int seg, int parity,
                              int grid, int* err, int poll_lim, int withhold,
                             const uint32_t* seed, bool var,
                             bool own_ghosts, cudaStream_t s);
cudaError_t launch_stash_mix(const InstDev* d, int n, int64_t items, int seg, int parity,
                             int grid, int* err, int poll_lim, int withhold,
                             const uint32_t* seed, bool var,
                             bool own_ghosts, cudaStream_t s);
int stash_occupancy_f32();
int stash_occupancy_f16();
int stash_occupancy_bf16();
int stash_occupancy_mix();

// One step of every instance in d_inst[0..n_inst): persistent grid of `grid`
// CTAs over total_tiles tiles; reads buf[parity], writes buf[parity ^ 1].
cudaError_t launch_step(int storage, int tile, const InstDev* d_inst, int n_inst,
                        int64_t total_tiles, int parity, int grid, const uint32_t* seed,
                        cudaStream_t s);

// Resident CTAs per SM of the step kernel (0 if unavailable).
int step_occupancy(int storage, int tile);

// Fields c, p, ux, uy, T of one instance (d_one, tiles of shape 0, whose
// tile_begin must be 0) into out[5][ny][nx] (double).
cudaError_t launch_fields(int storage, const InstDev* d_one, int64_t tiles, int parity,
                          double* out, cudaStream_t s);

// Per-storage entry points (defined in lbe_step_<storage>.cu).
cudaError_t launch_step_f64(int tile, const InstDev* d, int n, int64_t total, int parity,
                            int grid, const uint32_t* seed, cudaStream_t s);
cudaError_t launch_step_f32(int tile, const InstDev* d, int n, int64_t total, int parity,
                            int grid, const uint32_t* seed, cudaStream_t s);
cudaError_t launch_step_f16(int tile, const InstDev* d, int n, int64_t total, int parity,
                            int grid, const uint32_t* seed, cudaStream_t s);
cudaError_t launch_step_bf16(int tile, const InstDev* d, int n, int64_t total, int parity,
                             int grid, const uint32_t* seed, cudaStream_t s);
cudaError_t launch_step_mix(int tile, const InstDev* d, int n, int64_t total, int parity,
                            int grid, const uint32_t* seed, cudaStream_t s);
int occupancy_f64(int tile);
int occupancy_f32(int tile);
int occupancy_f16(int tile);
int occupancy_bf16(int tile);
int occupancy_mix(int tile);
cudaError_t fields_f64(const InstDev* d, int64_t tiles, int parity, double* out, cudaStream_t s);
// Varying density (FP64 storage only): the corrected p of Eq. 13 of every
// cell into each instance's pcorr; d is a work list of tile shape 0.
cudaError_t pcorr_f64(const InstDev* d, int n, int64_t total, int parity, int grid,
                      cudaStream_t s);
// FP32 storage: the pre-pass of the dissipation term (u of every cell)
cudaError_t pcorr_f32(const InstDev* d, int n, int64_t total, int parity, int grid,
                      cudaStream_t s);
cudaError_t fields_f32(const InstDev* d, int64_t tiles, int parity, double* out, cudaStream_t s);
cudaError_t fields_f16(const InstDev* d, int64_t tiles, int parity, double* out, cudaStream_t s);
cudaError_t fields_bf16(const InstDev* d, int64_t tiles, int parity, double* out, cudaStream_t s);
cudaError_t fields_mix(const InstDev* d, int64_t tiles, int parity, double* out, cudaStream_t s);

// Auxiliary kernels (lbe_aux.cu).
// The rest state of every cell from c0, T0 (device, [ny][nx]) into
// rest[3][ny][nx]: H_0, H_i (g_i = w_i H_i) and rho c_v T0 (hbar_i = w_i rho
// c_v T0); f = 0.
cudaError_t launch_rest_state(const InstDev* d_one, int nx, int ny, const double* c0,
                              const double* T0, double* rest, cudaStream_t s);
// pre[27][ny][nx] (double, pre-collision) -> buf[parity] (inverse of the
// pull); rest != 0: pre is rest[3][ny][nx] of launch_rest_state.
cudaError_t launch_push(int storage, const InstDev* d_one, int nx, int ny, const double* pre,
                        int parity, int rest, cudaStream_t s);
// buf[parity] -> pre[27][ny][nx] (the pull).
cudaError_t launch_pull(int storage, const InstDev* d_one, int nx, int ny, double* pre,
                        int parity, cudaStream_t s);
// FP64 sums over cur[5][n] and prev[5][n] (or prev = nullptr): out[6] =
// sum c, sum p, sum T, sum |u - u_prev|^2, sum |u|^2, non-finite count.
// partial must hold 6 * sums_blocks() doubles.
int sums_blocks();
cudaError_t launch_sums(const double* cur, const double* prev, int64_t n, double* partial,
                        double* out, cudaStream_t s);
cudaError_t launch_f64_to_f32(const double* in, float* out, int64_t n, cudaStream_t s);
// Periodic ghost columns of buffer `parity` of n_inst instances (16/32-bit
// storages), after a step of the stash kernel.
// (also advances the handle's step counter *seed by one)
cudaError_t launch_ghosts(const InstDev* d, int n_inst, int max_ny, int parity, uint32_t* seed,
                          cudaStream_t s);
// The handle's step counter: +1 after every step (the ghost-column kernel
// does it for the strip kernel; this one after a tile-kernel step), or set.
cudaError_t launch_seed_tick(uint32_t* seed, cudaStream_t s);
cudaError_t launch_seed_set(uint32_t* seed, uint32_t value, cudaStream_t s);

// Adjoint kernels (lbe_adjoint.cu), FP64, one instance d_one of nx x ny.
// Scratch: adjoint_scratch_doubles(nx, ny) doubles.
int64_t adjoint_scratch_doubles(int nx, int ny);
// out4[0] = sum c u_y, out4[1] = sum c of the state Q[27][ny][nx] (device).
cudaError_t launch_observable(const InstDev* d_one, int nx, int ny, const double* Q,
                              double* scratch, double* out4, cudaStream_t s);
// a_out = Post'(Q)^T Pull^T a_next + wl dl/dQ with obs = {sum c u_y, sum c} of
// Q (device, read only if wl != 0); theta_acc[0..2] (device) += the parameter
// partials.  a_next may be nullptr (zero).  fp32: the per-cell products in
// FP32 arithmetic (the planes and the parameter sums stay FP64).
cudaError_t launch_adjoint_step(const InstDev* d_one, int nx, int ny, const double* Q,
                                const double* a_next, double wl, const double* obs,
                                double* a_out, double* theta_acc, double* scratch, bool fp32,
                                cudaStream_t s);
// dT0[k] = rho c_v sum_i w_i a[18 + i][k]
cudaError_t launch_adjoint_dT0(const InstDev* d_one, int nx, int ny, const double* a,
                               double* dT0, cudaStream_t s);

// Sets the message lbe_last_error(NULL) returns on this thread (lbe_api.cu).
void set_thread_error(const char* msg);

}  // namespace lbe
