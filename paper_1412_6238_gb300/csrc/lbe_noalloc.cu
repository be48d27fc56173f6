// Allocation-free variant of the FP64 diagnostic sums (lbe_sums_fields_noalloc).
//
// Some callers cannot let the library call cudaMalloc: a framework whose
// caching allocator owns all device memory and must not see foreign
// allocations, a latency-critical monitoring loop where cudaMalloc/cudaFree
// would synchronize the device, or a process whose device-memory budget is
// fixed at start-up.  This entry point therefore keeps its only scratch (the
// per-block partial sums) in a file-scope __device__ array that is part of the
// loaded module: every GPU that loads the library holds it until the process
// exits, and no call allocates or frees anything.
//
// The caller passes the inputs (field arrays in device memory) and the output
// (5 doubles in device memory); the work is enqueued on the caller's stream.
#include <cstdio>
#include <mutex>

#include "../../include/lbe.h"
#include "lbe_launch.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 16;                        // elements per thread
constexpr int64_t NA_PER_BLOCK = (int64_t)NA_THREADS * NA_PER_THREAD;
constexpr int NA_MAX_BLOCKS = 8192;                      // 8192 x 6 x 8 B = 384 KiB
constexpr int64_t NA_MAX_CELLS = NA_PER_BLOCK * NA_MAX_BLOCKS;  // 33,554,432

// The scratch: per-block partial sums, 6 per block.  Shared by every call on
// a device; each call writes the partials of exactly the blocks it launches
// before reading them, so nothing has to be cleared between calls.
static __device__ __align__(256) double na_partials[NA_MAX_BLOCKS * 6];

constexpr int MAX_DEVICES = 64;
std::mutex na_mutex;
// device address of na_partials per device, and the context it was looked up
// in (a caller that makes another context current on the device, through the
// driver API, gets the array's address in that context)
double* na_ptr[MAX_DEVICES] = {};
void* na_ctx[MAX_DEVICES] = {};

// The current driver context, through the runtime's driver entry point (no
// link dependency on the driver library); nullptr if unavailable.
void* na_current_context() {
  using GetCurrent = int (*)(void**);
  static GetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<GetCurrent>(f);
  }();
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

// errors are reported like those of the other calls: lbe_last_error(NULL)
lbe_status na_fail(lbe_status st, const char* msg) {
  lbe::set_thread_error(msg);
  return st;
}

__device__ __forceinline__ void na_block_sum6(double v[6], double* sh) {
  for (int j = 0; j < 6; j++) sh[j * NA_THREADS + threadIdx.x] = v[j];
  __syncthreads();
  for (int st = NA_THREADS / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st)
      for (int j = 0; j < 6; j++)
        sh[j * NA_THREADS + threadIdx.x] += sh[j * NA_THREADS + threadIdx.x + st];
    __syncthreads();
  }
  for (int j = 0; j < 6; j++) v[j] = sh[j * NA_THREADS];
}

struct Fields5 {
  const double* f[5];  // c, p, ux, uy, T
};

// Pass 1: block b reduces elements [b*NA_PER_BLOCK, (b+1)*NA_PER_BLOCK).
__global__ void __launch_bounds__(NA_THREADS)
na_pass1(Fields5 cur, const double* __restrict__ pux, const double* __restrict__ puy, int64_t n,
         double* __restrict__ partial) {
  __shared__ double sh[6 * NA_THREADS];
  double v[6] = {0, 0, 0, 0, 0, 0};
  const int64_t base = (int64_t)blockIdx.x * NA_PER_BLOCK;
  for (int r = 0; r < NA_PER_THREAD; r++) {
    const int64_t k = base + (int64_t)r * NA_THREADS + threadIdx.x;
    if (k >= n) break;
    const double c = cur.f[0][k], p = cur.f[1][k], ux = cur.f[2][k], uy = cur.f[3][k],
                 T = cur.f[4][k];
    v[0] += c;
    v[1] += p;
    v[2] += T;
    if (pux) {
      const double dx = ux - pux[k], dy = uy - puy[k];
      v[3] += dx * dx + dy * dy;
    }
    v[4] += ux * ux + uy * uy;
    v[5] += (double)(!isfinite(c)) + (double)(!isfinite(p)) + (double)(!isfinite(ux)) +
            (double)(!isfinite(uy)) + (double)(!isfinite(T));
  }
  na_block_sum6(v, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < 6; j++) partial[blockIdx.x * 6 + j] = v[j];
}

// Pass 2: one block reduces the nb partials in a fixed order and writes the
// five outputs with the definitions of lbe_sums.
__global__ void __launch_bounds__(NA_THREADS)
na_pass2(const double* __restrict__ partial, int nb, double rho_cv, int has_prev,
         double* __restrict__ out) {
  __shared__ double sh[6 * NA_THREADS];
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nb; b += NA_THREADS)
    for (int j = 0; j < 6; j++) v[j] += partial[b * 6 + j];
  na_block_sum6(v, sh);
  if (threadIdx.x == 0) {
    out[0] = v[0];
    out[1] = v[1];
    out[2] = v[2] * rho_cv;
    out[3] = (has_prev && v[4] > 0) ? sqrt(v[3]) / sqrt(v[4]) : 0.0;
    out[4] = v[5];
  }
}

}  // namespace

extern "C" lbe_status lbe_sums_fields_noalloc(const double* const cur[5],
                                              const double* const prev[5], int64_t n,
                                              double rho_cv, double* out, void* stream) {
  if (!cur || !out) return na_fail(LBE_EINVAL, "cur and out must not be NULL");
  for (int k = 0; k < 5; k++)
    if (!cur[k]) return na_fail(LBE_EINVAL, "cur[k] must not be NULL");
  if (prev && (!prev[2] || !prev[3]))
    return na_fail(LBE_EINVAL, "prev[2] and prev[3] (ux, uy) must not be NULL");
  if (n < 1) return na_fail(LBE_EINVAL, "n must be >= 1");
  if (n > NA_MAX_CELLS)
    return na_fail(LBE_EINVAL,
                   "n exceeds the 33554432-cell maximum of the allocation-free sums "
                   "(its static scratch holds 8192 blocks of 4096 cells)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
    return na_fail(LBE_ECUDA, "no usable current CUDA device");
  // an error left on this thread by earlier, unrelated work is not ours
  (void)cudaGetLastError();
  double* partial;
  {
    // set-up, once per device (and context), with that device current: the
    // host-side name na_partials is only a stand-in, the kernels need the
    // device address
    std::lock_guard<std::mutex> lock(na_mutex);
    void* ctx = na_current_context();
    if (!na_ptr[dev] || na_ctx[dev] != ctx) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, na_partials);
      if (e != cudaSuccess || !p) {
        char m[256];
        snprintf(m, sizeof m, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return na_fail(LBE_ECUDA, m);
      }
      na_ptr[dev] = static_cast<double*>(p);
      na_ctx[dev] = ctx;
    }
    partial = na_ptr[dev];
  }
  const int nb = (int)((n + NA_PER_BLOCK - 1) / NA_PER_BLOCK);
  Fields5 f;
  for (int k = 0; k < 5; k++) f.f[k] = cur[k];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto launched = [](const char* which) -> lbe_status {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return LBE_OK;
    char m[256];
    snprintf(m, sizeof m, "lbe_sums_fields_noalloc %s launch: %s", which, cudaGetErrorString(e));
    return na_fail(LBE_ECUDA, m);
  };
  na_pass1<<<nb, NA_THREADS, 0, s>>>(f, prev ? prev[2] : nullptr, prev ? prev[3] : nullptr, n,
                                     partial);
  if (lbe_status st = launched("pass 1")) return st;
  na_pass2<<<1, NA_THREADS, 0, s>>>(partial, nb, rho_cv, prev ? 1 : 0, out);
  return launched("pass 2");
}
