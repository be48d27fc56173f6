#include <algorithm>
// Auxiliary kernels: initial state, state conversion (push / pull between the
// pre-collision form and a storage buffer), FP64 reductions, dtype casts,
// and the storage dispatch of the step / field launchers.
#include "lbe_launch.h"
#include "lbe_tile.cuh"

namespace lbe {

// ------------------------------------------------------------------ dispatch
bool tile_available(int storage, int tile) {
  if (tile < 0 || tile >= NUM_TILES) return false;
  if (storage == ST_F64) return tile == 0;
  // ids 5 and 6 are retired (TMA-ring strips); the stash kernel is 16/32-bit
  if (is_strip(tile) && !is_stash(tile)) return false;
  return true;
}

cudaError_t launch_stash(int storage, const InstDev* d, int n, int64_t items, int seg, int parity,
                         int grid, int* err, int poll_lim, int withhold, const uint32_t* seed,
                         bool var, bool own_ghosts, cudaStream_t s) {
  switch (storage) {
    case ST_F32:
      return launch_stash_f32(d, n, items, seg, parity, grid, err, poll_lim, withhold, seed, var,
                              own_ghosts, s);
    case ST_F16DEV:
      return launch_stash_f16(d, n, items, seg, parity, grid, err, poll_lim, withhold, seed, var,
                              own_ghosts, s);
    case ST_BF16DEV:
      return launch_stash_bf16(d, n, items, seg, parity, grid, err, poll_lim, withhold, seed, var,
                              own_ghosts, s);
    case ST_F16MIX:
      return launch_stash_mix(d, n, items, seg, parity, grid, err, poll_lim, withhold, seed, var,
                              own_ghosts, s);
  }
  return cudaErrorInvalidValue;
}

int stash_occupancy(int storage) {
  switch (storage) {
    case ST_F32: return stash_occupancy_f32();
    case ST_F16DEV: return stash_occupancy_f16();
    case ST_BF16DEV: return stash_occupancy_bf16();
    case ST_F16MIX: return stash_occupancy_mix();
  }
  return 0;
}

cudaError_t launch_step(int storage, int tile, const InstDev* d, int n, int64_t total, int parity,
                        int grid, const uint32_t* seed, cudaStream_t s) {
  switch (storage) {
    case ST_F64: return launch_step_f64(tile, d, n, total, parity, grid, seed, s);
    case ST_F32: return launch_step_f32(tile, d, n, total, parity, grid, seed, s);
    case ST_F16DEV: return launch_step_f16(tile, d, n, total, parity, grid, seed, s);
    case ST_BF16DEV: return launch_step_bf16(tile, d, n, total, parity, grid, seed, s);
    case ST_F16MIX: return launch_step_mix(tile, d, n, total, parity, grid, seed, s);
  }
  return cudaErrorInvalidValue;
}

int step_occupancy(int storage, int tile) {
  switch (storage) {
    case ST_F64: return occupancy_f64(tile);
    case ST_F32: return occupancy_f32(tile);
    case ST_F16DEV: return occupancy_f16(tile);
    case ST_BF16DEV: return occupancy_bf16(tile);
    case ST_F16MIX: return occupancy_mix(tile);
  }
  return 0;
}

cudaError_t launch_fields(int storage, const InstDev* d, int64_t tiles, int parity, double* out,
                          cudaStream_t s) {
  switch (storage) {
    case ST_F64: return fields_f64(d, tiles, parity, out, s);
    case ST_F32: return fields_f32(d, tiles, parity, out, s);
    case ST_F16DEV: return fields_f16(d, tiles, parity, out, s);
    case ST_BF16DEV: return fields_bf16(d, tiles, parity, out, s);
    case ST_F16MIX: return fields_mix(d, tiles, parity, out, s);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------- initial state
// At rest (u = 0, p = 0): f_i = f_eq(0, 0) = 0; g_i = g_eq(c0, mu0, 0) with
// mu0 = 2 beta c0 (c0-1)(2c0-1) - eps^2 lap c0 (Eq. 21-22), lap c0 by the
// isotropic stencil with mirrored ghost rows; hbar_i = w_i rho(c0) c_v T0
// (Eq. aEq9 at u = 0).  The rest state of a cell is three numbers, g_i =
// w_i H_i (H_0 and the common H_i) and hbar_i = w_i rho c_v T0: rest[0..2]
// [ny][nx] hold them, and the push below builds the 27 populations of every
// cell from its neighbours' three.  (Grids: x over blocks, rows over
// blockIdx.y, strided.)
__global__ void rest_state_kernel(const InstDev* __restrict__ d, int nx, int ny,
                                  const double* __restrict__ c0, const double* __restrict__ T0,
                                  double* __restrict__ rest) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int64_t N = (int64_t)nx * ny;
  const InstDev& I = *d;
  const Phys<double>& P = I.pd;
  // c0 with its ghost rows (the mirror, plus the wetting flux at a wetting
  // wall), periodic in x
  auto cat = [&](int xx, int yy) -> double {
    xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
    if (yy < 0) return wet_ghost(I.pd, c0[(int64_t)(-1 - yy) * nx + xx], -1 - yy);
    if (yy >= ny) return wet_ghost(I.pd, c0[(int64_t)(2 * ny - 1 - yy) * nx + xx], yy - ny);
    return c0[(int64_t)yy * nx + xx];
  };
  for (int y = blockIdx.y; y < ny; y += gridDim.y) {
    const int64_t k = (int64_t)y * nx + x;
    const double v0 = c0[k];
    // Laplacian (2/c_s^2) sum_i w_i (c(x + xi_i) - c(x)), terms in index order
    const double wa = WGT<double>(1), wd = WGT<double>(5);
    double t = wa * (cat(x + 1, y) - v0);
    t = t + wa * (cat(x, y + 1) - v0);
    t = t + wa * (cat(x - 1, y) - v0);
    t = t + wa * (cat(x, y - 1) - v0);
    t = t + wd * (cat(x + 1, y + 1) - v0);
    t = t + wd * (cat(x - 1, y + 1) - v0);
    t = t + wd * (cat(x - 1, y - 1) - v0);
    t = t + wd * (cat(x + 1, y - 1) - v0);
    const double cs2 = 1.0 / 3.0;
    const double lap = 2.0 * t / cs2;
    const double mu = P.beta2 * v0 * (v0 - 1.0) * (2.0 * v0 - 1.0) - P.eps2 * lap;
    const double W0 = WGT<double>(0);
    rest[k] = (v0 - (1.0 - W0) * P.Gm * mu / cs2) / W0;  // H_0
    rest[N + k] = P.Gm * mu / cs2;                        // H_i, i > 0
    rest[2 * N + k] = rho_at(P, v0) * P.cv * T0[k];      // rho c_v T0
  }
}

cudaError_t launch_rest_state(const InstDev* d, int nx, int ny, const double* c0,
                              const double* T0, double* rest, cudaStream_t s) {
  const dim3 grid((nx + 127) / 128, ny < 65535 ? ny : 65535);
  rest_state_kernel<<<grid, 128, 0, s>>>(d, nx, ny, c0, T0, rest);
  return cudaGetLastError();
}

// -------------------------------------------------------------- push / pull
// The pull P_i(x) = P*_i(x - xi_i) is a permutation of the buffer entries
// (each post-collision value either streams to x + xi_i or, at a wall,
// returns reversed to x), so it has an exact inverse, the push:
//   P*_j(x) = P_j(x + xi_j)                 if x + xi_j is a cell,
//   P*_j(x) = P_jbar(x)                      at a wall for f and g,
//   P*_j(x) = 2 w_j rho c_v T_w - P_jbar(x)  at a wall for hbar,
// rho that of the cell's c = sum_i g_i (with a varying density).  pre(kk, j,
// k): pre-collision population (kk, j) of cell k.
template <class S, class Pre>
__device__ __forceinline__ void push_cell(const InstDev& I, int nx, int ny, int x, int y,
                                          int parity, Pre&& pre) {
  using C = typename S::C;
  char* buf = I.buf[parity];
  const int64_t k = (int64_t)y * nx + x;
  const size_t rowbase = (size_t)y * I.pitch;
  // hbar deviation reference of this row (storage forms other than FP64)
  const double rref = dev_h<S>() ? I.pd.rho * I.pd.cv * (I.hr0 + I.hr1 * y) : 0.0;
  double cn = 0.0;
  for (int j = 0; j < 9; j++) cn += pre(1, j, k);
  const double rc = rho_at(I.pd, cn);
#pragma unroll
  for (int j = 0; j < 9; j++) {
    int xt = x + EX(j);
    xt = xt < 0 ? xt + nx : (xt >= nx ? xt - nx : xt);
    const int yt = y + EY(j);
    const bool wall = (yt < 0) || (yt >= ny);
    for (int kk = 0; kk < 3; kk++) {
      double v;
      if (!wall) {
        v = pre(kk, j, (int64_t)yt * nx + xt);
      } else {
        const double pb = pre(kk, OPP(j), k);
        if (kk < 2) {
          v = pb;
        } else {
          // the inverse of the pull's anti-bounce-back of population
          // OPP(j), whose link crosses the wall at x + xi_jx/2
          const double* Twall = (yt < 0) ? I.Tbot : I.Ttop;
          double Tw = Twall[x];
          if (I.pd.wmid != 0.0 && EX(j) != 0) Tw = 0.5 * (Tw + Twall[xt]);
          v = 2.0 * WGT<double>(j) * rc * I.pd.cv * Tw - pb;
        }
      }
      if (kk == 2) v -= WGT<double>(j) * rref;
      st_cell<S>(I, buf, kk, j, rowbase, x, (C)v);
      if constexpr (S::kind != ST_F64) {
        // g_0 = hi + lo: the low part of the rest population
        if (kk == 1 && j == 0) st_cell_g0lo<S>(I, buf, rowbase, x, (float)(v - (double)(C)v));
      }
    }
  }
}

// push of a [27][ny][nx] pre-collision state (rest == 0), or of the rest
// state of rest_state_kernel (rest != 0: the same values as the state f_i =
// 0, g_i = w_i H_i, hbar_i = rho c_v T0 w_i)
template <class S>
__global__ void push_kernel(const InstDev* __restrict__ d, int nx, int ny,
                            const double* __restrict__ pre, int parity, int rest) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int64_t N = (int64_t)nx * ny;
  for (int y = blockIdx.y; y < ny; y += gridDim.y) {
    if (rest) {
      push_cell<S>(*d, nx, ny, x, y, parity, [&](int kk, int j, int64_t k) -> double {
        const double w = WGT<double>(j);
        if (kk == 0) return 0.0;
        if (kk == 1) return w * (j == 0 ? pre[k] : pre[N + k]);
        return pre[2 * N + k] * w;
      });
    } else {
      push_cell<S>(*d, nx, ny, x, y, parity,
                   [&](int kk, int j, int64_t k) { return pre[(int64_t)(kk * 9 + j) * N + k]; });
    }
  }
}

template <class S>
__global__ void pull_kernel(const InstDev* __restrict__ d, int nx, int ny, double* __restrict__ pre,
                            int parity) {
  using C = typename S::C;
  const InstDev& I = *d;
  const int64_t N = (int64_t)nx * ny;
  const char* buf = I.buf[parity];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(k % nx), y = (int)(k / nx);
    const Cell<S> q = make_cell<S>(x, y, nx);
    const Phys<C>& P = phys<C>(I);
    C v[9];
    pull9<S, 0>(I, P, buf, q, v);
    for (int i = 0; i < 9; i++) pre[(int64_t)i * N + k] = (double)v[i];
    pull9<S, 1>(I, P, buf, q, v);
    for (int i = 0; i < 9; i++) pre[(int64_t)(9 + i) * N + k] = (double)v[i];
    if constexpr (S::kind != ST_F64)
      pre[(int64_t)9 * N + k] += (double)ld_g0lo<S>(I, buf, (size_t)y * I.pitch + XG + x);
    C cn = C(0);
    for (int i = 0; i < 9; i++) cn += v[i];
    pull9<S, 2>(I, P, buf, q, v, rho_at(P, cn));
    const double rref = dev_h<S>() ? I.pd.rho * I.pd.cv * (I.hr0 + I.hr1 * y) : 0.0;
    for (int i = 0; i < 9; i++)
      pre[(int64_t)(18 + i) * N + k] = (double)v[i] + WGT<double>(i) * rref;
  }
}

template <class S>
static cudaError_t push_t(const InstDev* d, int nx, int ny, const double* pre, int parity,
                          int rest, cudaStream_t s) {
  const dim3 grid((nx + 127) / 128, ny < 65535 ? ny : 65535);
  push_kernel<S><<<grid, 128, 0, s>>>(d, nx, ny, pre, parity, rest);
  return cudaGetLastError();
}
template <class S>
static cudaError_t pull_t(const InstDev* d, int nx, int ny, double* pre, int parity,
                          cudaStream_t s) {
  const int64_t N = (int64_t)nx * ny;
  const int grid = (int)((N + 255) / 256 < 65535 ? (N + 255) / 256 : 65535);
  pull_kernel<S><<<grid, 256, 0, s>>>(d, nx, ny, pre, parity);
  return cudaGetLastError();
}

cudaError_t launch_push(int storage, const InstDev* d, int nx, int ny, const double* pre,
                        int parity, int rest, cudaStream_t s) {
  switch (storage) {
    case ST_F64: return push_t<StF64>(d, nx, ny, pre, parity, rest, s);
    case ST_F32: return push_t<StF32>(d, nx, ny, pre, parity, rest, s);
    case ST_F16DEV: return push_t<StF16>(d, nx, ny, pre, parity, rest, s);
    case ST_BF16DEV: return push_t<StBF16>(d, nx, ny, pre, parity, rest, s);
    case ST_F16MIX: return push_t<StMix>(d, nx, ny, pre, parity, rest, s);
  }
  return cudaErrorInvalidValue;
}
cudaError_t launch_pull(int storage, const InstDev* d, int nx, int ny, double* pre, int parity,
                        cudaStream_t s) {
  switch (storage) {
    case ST_F64: return pull_t<StF64>(d, nx, ny, pre, parity, s);
    case ST_F32: return pull_t<StF32>(d, nx, ny, pre, parity, s);
    case ST_F16DEV: return pull_t<StF16>(d, nx, ny, pre, parity, s);
    case ST_BF16DEV: return pull_t<StBF16>(d, nx, ny, pre, parity, s);
    case ST_F16MIX: return pull_t<StMix>(d, nx, ny, pre, parity, s);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------- FP64 sums
// Two passes, fixed block count and fixed reduction order: deterministic.
constexpr int SUM_BLOCKS = 304;
constexpr int SUM_THREADS = 256;
int sums_blocks() { return SUM_BLOCKS; }

// ------------------------------------------------------------ ghost columns
// Periodic ghost columns of the buffer `parity` of every instance (16/32-bit
// storages): in a row, elements 0..XG-1 repeat cells nx-XG..nx-1 and elements
// nx+XG..nx+2XG-1 repeat cells 0..XG-1 (element XG + x holds cell x).  Planes:
// FP32: 9 (f, g) pairs + 9 hbar + the FP16 g_0 low part; 16-bit: 8 (f, g)
// pairs + f_0 + 9 hbar + the FP32 g_0 + the low part; F16MIX: 9 planes of
// 8-byte words + the FP32 g_0.  One thread per ghost element: 8 neighbouring
// threads copy one row's 2 XG elements (the sources and the ghosts are
// disjoint for nx >= XG, which the strip kernel requires).
template <class T>
__device__ __forceinline__ void wrap_one(char* plane, size_t row, int dstE, int srcE) {
  T* q = reinterpret_cast<T*>(plane) + row;
  q[dstE] = q[srcE];
}

constexpr int GHOST_THREADS = 256;
constexpr int GHOST_PLANES = 20;

// blockIdx.y: plane; blockIdx.x walks (instance, chunk of GHOST_THREADS / 2 XG
// rows) pairs, chunks = row chunks of the tallest instance.
__global__ void __launch_bounds__(GHOST_THREADS)
ghost_kernel(const InstDev* __restrict__ insts, int n_inst, int chunks, int parity, uint32_t* seed) {
  // the step is complete: advance the handle's step counter
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *seed += 1u;
  const int p = blockIdx.y;
  const int j = threadIdx.x % (2 * XG);
  const int64_t pairs = (int64_t)n_inst * chunks;
  for (int64_t g = blockIdx.x; g < pairs; g += gridDim.x) {
    const InstDev& I = insts[g / chunks];
    const int y = (int)(g % chunks) * (GHOST_THREADS / (2 * XG)) + (int)threadIdx.x / (2 * XG);
    if (y >= I.ny) continue;
    char* b = I.buf[parity];
    const int nx = I.nx;
    const int dstE = j < XG ? j : nx + j;  // left ghosts, then right
    const int srcE = j < XG ? nx + j : j;  // cells nx-XG+j, then j-XG
    const size_t row = (size_t)y * (size_t)I.pitch;
    const int st = I.storage;
    if (st == ST_F16MIX) {
      if (p < 9) wrap_one<uint64_t>(b + (size_t)p * I.pair_bytes, row, dstE, srcE);
      else if (p == 9) wrap_one<uint32_t>(b + I.g0_off, row, dstE, srcE);
    } else if (st == ST_F16DEV || st == ST_BF16DEV) {
      if (p < 8) wrap_one<uint32_t>(b + (size_t)p * I.pair_bytes, row, dstE, srcE);
      else if (p == 8) wrap_one<uint16_t>(b + I.f0_off, row, dstE, srcE);
      else if (p < 18)
        wrap_one<uint16_t>(b + I.h_off + (size_t)(p - 9) * I.plane_bytes, row, dstE, srcE);
      else if (p == 18) wrap_one<uint32_t>(b + I.g0_off, row, dstE, srcE);
      else wrap_one<uint16_t>(b + I.g0lo_off, row, dstE, srcE);
    } else {  // FP32
      if (p < 9) wrap_one<uint64_t>(b + (size_t)p * I.pair_bytes, row, dstE, srcE);
      else if (p < 18)
        wrap_one<uint32_t>(b + I.h_off + (size_t)(p - 9) * I.plane_bytes, row, dstE, srcE);
      else if (p == 18) wrap_one<uint16_t>(b + I.g0lo_off, row, dstE, srcE);
    }
  }
}

cudaError_t launch_ghosts(const InstDev* d, int n_inst, int max_ny, int parity, uint32_t* seed,
                          cudaStream_t s) {
  constexpr int rows = GHOST_THREADS / (2 * XG);
  const int chunks = (max_ny + rows - 1) / rows;
  const int64_t pairs = (int64_t)n_inst * chunks;
  const int bx = (int)std::min<int64_t>(pairs, 1 << 16);
  ghost_kernel<<<dim3(bx, GHOST_PLANES), GHOST_THREADS, 0, s>>>(d, n_inst, chunks, parity, seed);
  return cudaGetLastError();
}

__global__ void seed_kernel(uint32_t* seed, uint32_t value, int set) {
  *seed = set ? value : *seed + 1u;
}
cudaError_t launch_seed_tick(uint32_t* seed, cudaStream_t s) {
  seed_kernel<<<1, 1, 0, s>>>(seed, 0u, 0);
  return cudaGetLastError();
}
cudaError_t launch_seed_set(uint32_t* seed, uint32_t value, cudaStream_t s) {
  seed_kernel<<<1, 1, 0, s>>>(seed, value, 1);
  return cudaGetLastError();
}

__device__ __forceinline__ void block_sum6(double v[6], double* sh) {
  // sh: 6 * SUM_THREADS doubles
  for (int j = 0; j < 6; j++) sh[j * SUM_THREADS + threadIdx.x] = v[j];
  __syncthreads();
  for (int st = SUM_THREADS / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int j = 0; j < 6; j++)
        sh[j * SUM_THREADS + threadIdx.x] += sh[j * SUM_THREADS + threadIdx.x + st];
    __syncthreads();
  }
  for (int j = 0; j < 6; j++) v[j] = sh[j * SUM_THREADS];
}

__global__ void __launch_bounds__(SUM_THREADS)
sums_pass1(const double* __restrict__ cur, const double* __restrict__ prev, int64_t n,
           double* __restrict__ partial) {
  __shared__ double sh[6 * SUM_THREADS];
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t k = blockIdx.x * (int64_t)SUM_THREADS + threadIdx.x; k < n;
       k += (int64_t)SUM_BLOCKS * SUM_THREADS) {
    const double c = cur[k], p = cur[n + k], ux = cur[2 * n + k], uy = cur[3 * n + k],
                 T = cur[4 * n + k];
    v[0] += c;
    v[1] += p;
    v[2] += T;
    if (prev) {
      const double dx = ux - prev[2 * n + k], dy = uy - prev[3 * n + k];
      v[3] += dx * dx + dy * dy;
    }
    v[4] += ux * ux + uy * uy;
    v[5] += (double)(!isfinite(c)) + (double)(!isfinite(p)) + (double)(!isfinite(ux)) +
            (double)(!isfinite(uy)) + (double)(!isfinite(T));
  }
  block_sum6(v, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < 6; j++) partial[blockIdx.x * 6 + j] = v[j];
}

__global__ void __launch_bounds__(SUM_THREADS)
sums_pass2(const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[6 * SUM_THREADS];
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < SUM_BLOCKS; b += SUM_THREADS)
    for (int j = 0; j < 6; j++) v[j] += partial[b * 6 + j];
  block_sum6(v, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < 6; j++) out[j] = v[j];
}

cudaError_t launch_sums(const double* cur, const double* prev, int64_t n, double* partial,
                        double* out, cudaStream_t s) {
  sums_pass1<<<SUM_BLOCKS, SUM_THREADS, 0, s>>>(cur, prev, n, partial);
  sums_pass2<<<1, SUM_THREADS, 0, s>>>(partial, out);
  return cudaGetLastError();
}

__global__ void f64_to_f32_kernel(const double* __restrict__ in, float* __restrict__ out,
                                  int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (float)in[k];
}
cudaError_t launch_f64_to_f32(const double* in, float* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
  f64_to_f32_kernel<<<grid, 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace lbe
