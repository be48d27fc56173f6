// Host side of the C ABI declared in include/lbe.h: parameter validation,
// device memory, stream and graph management, bounded waits, checkpoints.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lbe.h"
#include "lbe_launch.h"

using namespace lbe;

namespace {

thread_local std::string g_thread_err;

struct InstHost {
  lbe_params p{};
  int nx = 0, ny = 0, pitch = 0;
  uint64_t plane_bytes = 0, g0_off = 0, g0lo_off = 0, buf_bytes = 0;
  uint64_t pair_bytes = 0, h_off = 0, f0_off = 0;  // pair layouts
  char* arena = nullptr;  // two buffers of buf_bytes
  double* walls = nullptr;  // device: Tbot[nx], Ttop[nx], then 4 float tables
  double* pcorr = nullptr;  // device [ny][nx]: corrected p (varying density only)
  double* uvel = nullptr;   // device [2][ny][nx]: u of every cell (dissipation term only)
  std::vector<double> Tbot, Ttop;
  std::vector<float> wdev;  // host copy of the T_w - T_r tables
};

}  // namespace

struct lbe_handle {
  int n = 0;
  int storage = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int num_sms = 0;
  std::vector<InstHost> inst;
  std::vector<InstDev> idev;     // step descriptors (tile_begin for the step shape)
  InstDev* d_inst = nullptr;     // [n] for the step kernel
  InstDev* d_finst = nullptr;    // [n] for the field kernel (shape 0, tile_begin 0)
  bool vrho = false;             // varying density (rho2 != rho; FP64 storage)
  bool variants = false;         // some instance uses interp / wall_mid / cos_wet
  bool dissip = false;           // some instance keeps the dissipation term (FP64)
  InstDev* d_pinst = nullptr;    // [n] shape-0 work list of the pcorr pass (vrho)
  int64_t p_tiles = 0;           // its tiles
  int p_grid = 0;                // its CTAs
  int tile = 0;
  int grid_req = 0;              // 0 = auto, -1 = one CTA per tile, >0 = CTAs
  int grid = 0;
  int seg_req = 0;               // strip kernel: rows per work item (0 = auto)
  int seg = 0;
  int* d_err = nullptr;          // device error word (strip kernel wait time-outs)
  uint32_t* d_seed = nullptr;    // step counter (random bits of the stochastic rounding)
  int poll_lim = STASH_POLLS;    // polls of one bounded copy wait
  int withhold = -1;             // test hook: source row whose copies are not issued
  int64_t total_tiles = 0;
  int max_ny = 0;                // largest ny of the instances
  int parity = 0;
  int64_t steps = 0;
  bool prev_valid = false;       // buf[parity^1] holds the previous step
  bool bad = false;              // after LBE_ENAN / LBE_ECUDA
  cudaGraphExec_t gexec = nullptr;
  bool graph_failed = false;
  cudaEvent_t ev = nullptr;
  double* scratch = nullptr;     // fields of two states: 10 * max_cells doubles
  int64_t max_cells = 0;
  double* d_partial = nullptr;   // sums partials
  double* d_sums = nullptr;      // 6 doubles
  std::string err;
};

namespace {

lbe_status fail(lbe_handle* h, lbe_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) {
    h->err = buf;
    if (st == LBE_ECUDA || st == LBE_ENAN) h->bad = true;
  } else {
    g_thread_err = buf;
  }
  return st;
}

#define CU(h, call)                                                                         \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail((h), e_ == cudaErrorMemoryAllocation ? LBE_ENOMEM : LBE_ECUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                           \
  } while (0)

long timeout_ms() {
  const char* s = getenv("LBE_TIMEOUT_MS");
  long v = s ? atol(s) : 600000;
  return v > 0 ? v : 600000;
}

bool fault_alloc() {
  const char* s = getenv("LBE_FAULT");
  return s && strcmp(s, "alloc") == 0;
}

// Bounded wait for all work enqueued on the handle's stream so far.
lbe_status wait_stream(lbe_handle* h) {
  CU(h, cudaEventRecord(h->ev, h->stream));
  const auto t0 = std::chrono::steady_clock::now();
  const long lim = timeout_ms();
  int spins = 0;
  for (;;) {
    cudaError_t e = cudaEventQuery(h->ev);
    if (e == cudaSuccess) return LBE_OK;
    if (e != cudaErrorNotReady)
      return fail(h, LBE_ECUDA, "while waiting for the stream: %s", cudaGetErrorString(e));
    const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                        std::chrono::steady_clock::now() - t0).count();
    if (ms > lim) return fail(h, LBE_ETIMEOUT, "stream not done after %ld ms", lim);
    if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Device -> host copy at the end of the handle's stream.  A copy into pageable
// host memory blocks the calling thread until the stream reaches it, so the
// stream is first waited for with the bounded wait; the copy then waits only
// for its own transfer.
lbe_status to_host(lbe_handle* h, void* dst, const void* src, size_t bytes) {
  lbe_status st = wait_stream(h);
  if (st) return st;
  CU(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream));
  return LBE_OK;
}

// Bounded wait, then the device error word of the strip kernel: a copy wait
// that ran out in any step since the word was last cleared (lbe_init,
// lbe_set_state, lbe_load) makes every later wait report LBE_ECUDA.
lbe_status wait(lbe_handle* h) {
  lbe_status st = wait_stream(h);
  if (st || !h->d_err) return st;
  int e = 0;
  CU(h, cudaMemcpyAsync(&e, h->d_err, sizeof e, cudaMemcpyDeviceToHost, h->stream));
  if ((st = wait_stream(h))) return st;
  if (e)
    return fail(h, LBE_ECUDA, "%s (device error word %d); the state is lost: set a state or "
                "load a checkpoint",
                (e & 1) ? "a strip-kernel wait (for copies or a stash slot) ran out of its poll "
                          "limit"
                        : "a strip-kernel work range did not advance",
                e);
  return LBE_OK;
}

// LBE_FAULT=withhold:<row> (test hook): the strip kernel issues no copies of
// source row <row>, and a copy wait gives up after STASH_POLLS_TEST polls.
int fault_withhold() {
  const char* s = getenv("LBE_FAULT");
  if (!s || strncmp(s, "withhold:", 9) != 0) return -1;
  const int r = atoi(s + 9);
  return r >= 0 ? r : -1;
}

// Density of phase c = 1 differs from that of phase c = 0 (rho2 = 0 means
// rho2 = rho).
bool varying_rho(const lbe_params& p) { return p.rho2 > 0 && p.rho2 != p.rho; }

lbe_status check_params(const lbe_params& p, int index) {
  auto bad = [&](const char* what) {
    return fail(nullptr, LBE_EINVAL, "instance %d: %s", index, what);
  };
  if (p.nx < 1) return bad("nx must be >= 1");
  if (p.ny < 2) return bad("ny must be >= 2");
  if ((int64_t)p.nx * p.ny > (int64_t)1 << 31) return bad("nx*ny must be < 2^31");
  if (p.storage < LBE_F64 || p.storage > LBE_F16MIX) return bad("unknown storage");
  if (p.check_every < 0) return bad("check_every must be >= 0");
  if (!(p.rho > 0) || !(p.cv > 0)) return bad("rho and cv must be > 0");
  if (!(p.eta1 > 0) || !(p.eta2 > 0)) return bad("eta1, eta2 must be > 0 (0 < omega_f < 2)");
  if (!(p.lam1 >= 0) || !(p.lam2 >= 0)) return bad("lam1, lam2 must be >= 0");
  if (!(p.eps > 0)) return bad("eps must be > 0");
  if (!(p.tau_g > 0.5)) return bad("tau_g must be > 1/2 (0 < omega_g < 2)");
  if (!(p.mobility >= 0)) return bad("mobility must be >= 0");
  if (!(p.eta_n > 0)) return bad("eta_n must be > 0");
  const double vals[] = {p.beta, p.sigma0, p.sigmaT, p.Tref, p.ax, p.ay};
  for (double v : vals)
    if (!std::isfinite(v)) return bad("non-finite parameter");
  if (!(p.rho2 >= 0) || !std::isfinite(p.rho2)) return bad("rho2 must be >= 0 (0: rho2 = rho)");
  if (p.interp != 0 && p.interp != 1) return bad("interp must be 0 (linear) or 1 (harmonic)");
  if (p.interp == 1 && !(p.lam1 > 0 && p.lam2 > 0))
    return bad("the harmonic law (interp = 1) needs lam1, lam2 > 0");
  if (p.wall_mid != 0 && p.wall_mid != 1) return bad("wall_mid must be 0 or 1");
  if (!(p.cos_wet >= -1.0 && p.cos_wet <= 1.0)) return bad("cos_wet must be in [-1, 1]");
  if (p.dissip != 0 && p.dissip != 1) return bad("dissip must be 0 or 1");
  if (p.dissip == 1 && p.storage != LBE_F64 && p.storage != LBE_F32)
    return bad("the dissipation term (dissip = 1) needs FP64 or FP32 storage");
  if (p.reserved != 0) return bad("reserved must be 0");
  if (varying_rho(p) && p.storage != LBE_F64)
    return bad("a density ratio (rho2 != rho) needs FP64 storage");
  return LBE_OK;
}

void fill_desc(lbe_handle* h, int j, InstDev& D) {
  const InstHost& H = h->inst[j];
  const lbe_params& p = H.p;
  memset(&D, 0, sizeof D);
  D.nx = H.nx;
  D.ny = H.ny;
  D.pitch = H.pitch;
  D.storage = h->storage;
  D.plane_bytes = H.plane_bytes;
  D.g0_off = H.g0_off;
  D.g0lo_off = H.g0lo_off;
  D.pair_bytes = H.pair_bytes;
  D.h_off = H.h_off;
  D.f0_off = H.f0_off;
  D.buf[0] = H.arena;
  D.buf[1] = H.arena + H.buf_bytes;
  D.salt = (uint32_t)j;
  D.Tbot = H.walls;
  D.Ttop = H.walls + H.nx;
  Phys<double>& P = D.pd;
  P.rho = p.rho;
  P.inv_rho = 1.0 / p.rho;
  P.cv = p.cv;
  P.rho_cv = p.rho * p.cv;
  P.inv_rho_cv = 1.0 / (p.rho * p.cv);
  P.rcs2 = p.rho * (1.0 / 3.0);
  P.rcvcs2 = (p.rho * p.cv) * (1.0 / 3.0);
  P.eta1 = p.eta1;
  P.deta = p.eta2 - p.eta1;
  P.lam1 = p.lam1;
  P.dlam = p.lam2 - p.lam1;
  P.sigma0 = p.sigma0;
  P.sigmaT = p.sigmaT;
  P.Tref = p.Tref;
  P.eps2 = p.eps * p.eps;
  P.ea = p.eps * (6.0 * std::sqrt(2.0));  // alpha = 6 sqrt 2 (Sec. II)
  P.beta2 = 2.0 * p.beta;
  P.omega_g = 1.0 / p.tau_g;
  P.Gm = p.mobility / (p.tau_g - 0.5);
  P.Fbx = p.rho * p.ax;
  P.Fby = p.rho * p.ay;
  P.ax = p.ax;
  P.ay = p.ay;
  P.drho = varying_rho(p) ? p.rho2 - p.rho : 0.0;
  P.harm = p.interp == 1 ? 1.0 : 0.0;
  P.eta2 = p.eta2;
  P.lam2 = p.lam2;
  P.ie1 = 1.0 / p.eta1;
  P.ie2 = 1.0 / p.eta2;
  P.il1 = p.lam1 > 0 ? 1.0 / p.lam1 : 0.0;
  P.il2 = p.lam2 > 0 ? 1.0 / p.lam2 : 0.0;
  P.wmid = p.wall_mid == 1 ? 1.0 : 0.0;
  P.kw = p.cos_wet * std::sqrt(2.0 * p.beta) / p.eps;
  D.pcorr = H.pcorr;
  D.uvel = H.uvel;
  P.eta_n2 = p.eta_n * p.eta_n;
  // hbar reference: linear profile between the mean wall temperatures
  double tb = 0, tt = 0;
  for (int x = 0; x < H.nx; x++) {
    tb += H.Tbot[x];
    tt += H.Ttop[x];
  }
  tb /= H.nx;
  tt /= H.nx;
  D.hr1 = (tt - tb) / H.ny;
  D.hr0 = tb + 0.5 * D.hr1;
  P.hr0 = D.hr0;
  P.hr1 = D.hr1;
  P.dh = P.rho_cv * D.hr1;
  // power-of-two scales keep the 16-bit deviations in the normal range with
  // a wide margin below the FP16 maximum (65504)
  double dev = 1e-6 * (std::fabs(tb) + std::fabs(tt) + 1.0);
  for (int x = 0; x < H.nx; x++) {
    dev = std::fmax(dev, std::fabs(H.Tbot[x] - tb));
    dev = std::fmax(dev, std::fabs(H.Ttop[x] - tt));
  }
  dev = std::fmax(dev, 0.05 * std::fabs(tt - tb));
  const double hmax = (4.0 / 9.0) * p.rho * p.cv * dev;
  int eh = (int)std::floor(std::log2(65504.0 / 64.0 / hmax));
  eh = eh < -30 ? -30 : (eh > 30 ? 30 : eh);
  const int e[3] = {12, 12, eh};
  for (int k = 0; k < 3; k++) {
    // 16-bit values: g and hbar of F16MIX, all three lattices of F16DEV / BF16DEV
    const bool sixteen = h->storage == LBE_F16DEV || h->storage == LBE_BF16DEV ||
                         (h->storage == LBE_F16MIX && k > 0);
    D.s[k] = sixteen ? std::ldexp(1.0f, e[k]) : 1.0f;
    P.inv_s[k] = sixteen ? std::ldexp(1.0, -e[k]) : 1.0;
  }
  // the same constants in FP32 for the FP32 arithmetic
  Phys<float>& F = D.pf;
  const double* src = &P.rho;
  float* dstf = &F.rho;
  const int nfield = (int)(sizeof(Phys<double>) / sizeof(double));
  for (int k = 0; k < nfield; k++) dstf[k] = (float)src[k];
  // T_w - T_r at the first / last row and at the wall positions
  D.wdev[0] = reinterpret_cast<const float*>(H.walls + 2 * H.nx);
  D.wdev[1] = D.wdev[0] + H.nx;
  D.wdev[2] = D.wdev[1] + H.nx;
  D.wdev[3] = D.wdev[2] + H.nx;
}

void free_handle(lbe_handle* h) {
  if (!h) return;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  for (auto& H : h->inst) {
    if (H.arena) cudaFree(H.arena);
    if (H.walls) cudaFree(H.walls);
    if (H.pcorr) cudaFree(H.pcorr);
    if (H.uvel) cudaFree(H.uvel);
  }
  if (h->d_inst) cudaFree(h->d_inst);
  if (h->d_pinst) cudaFree(h->d_pinst);
  if (h->d_err) cudaFree(h->d_err);
  if (h->d_seed) cudaFree(h->d_seed);
  if (h->d_finst) cudaFree(h->d_finst);
  if (h->scratch) cudaFree(h->scratch);
  if (h->d_partial) cudaFree(h->d_partial);
  if (h->d_sums) cudaFree(h->d_sums);
  if (h->ev) cudaEventDestroy(h->ev);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// (Re)build the step descriptors for the current tile shape and upload them.
lbe_status setup_tiles(lbe_handle* h) {
  if (is_strip(h->tile)) {
    const int nc = TILE_SHAPES[h->tile].tx;  // output columns per strip
    const int occ = stash_occupancy(h->storage);
    if (occ <= 0) return fail(h, LBE_ECUDA, "strip kernel %d cannot be resident", h->tile);
    h->grid = h->grid_req > 0 ? h->grid_req : occ * h->num_sms;
    int max_ny = 1;
    for (auto& H : h->inst) max_ny = std::max(max_ny, H.ny);
    h->max_ny = max_ny;
    // default: balanced row ranges for instances of different sizes, items
    // of a fixed row count for one grid size.  Measured on the 64-drop
    // sweep (four grid sizes, 36 M cells; FP32, 3 CTAs per SM): balanced
    // 22.8 GLUPS, fixed items of 72 / 96 / 128 rows 21.6 / 22.2 / 22.2 (the
    // last wave partly idle); on one 4096^2 grid fixed items of 72 rows (4
    // whole waves) 24.0, balanced ranges 23.4 (also when cut into pieces of
    // 48 to 160 rows).
    bool one_size = true;
    for (auto& H : h->inst)
      one_size = one_size && H.nx == h->inst[0].nx && H.ny == h->inst[0].ny;
    if (h->seg_req > 0 || (h->seg_req < 0 && h->grid_req != -1)) {
      h->seg = h->seg_req;
    } else if (h->grid_req != -1 && !one_size) {
      h->seg = 0;  // balanced contiguous row ranges, one per CTA
    } else {
      // rows per item that minimise (waves of the persistent grid, or of the
      // resident CTAs with one CTA per item) x (rows per item + the warm-up
      // rows every item recomputes, about 6 for the stash kernel)
      const int64_t slots = h->grid_req == -1 ? (int64_t)occ * h->num_sms : h->grid;
      const bool stash = is_stash(h->tile);
      const int seg_lo = std::min(8, max_ny);
      const int seg_hi = stash ? std::min(96, max_ny) : max_ny;
      const int warm = stash ? 6 : 4;
      double best = 1e300;
      int best_seg = seg_hi;
      for (int seg = seg_lo; seg <= seg_hi; seg++) {
        int64_t items = 0;
        for (auto& H : h->inst)
          items += (int64_t)((H.nx + nc - 1) / nc) * ((H.ny + seg - 1) / seg);
        const double waves = (double)((items + slots - 1) / slots);
        const double cost = waves * (seg + warm);
        if (cost < best * (1 - 1e-9)) {
          best = cost;
          best_seg = seg;
        }
      }
      h->seg = best_seg;
    }
    // tile_begin: the instance's first item (seg > 0) or first strip row
    // (seg == 0: the rows of all strips end to end, tiles_y the band height
    // of the band-by-band order, about one CTA's share of the rows)
    int64_t begin = 0, rows = 0;
    for (auto& H : h->inst) rows += (int64_t)((H.nx + nc - 1) / nc) * H.ny;
    const int64_t ctas = h->grid_req == -1 ? 1 : std::max(1, h->grid);
    const int64_t band = std::max<int64_t>(1, (rows + ctas - 1) / ctas);
    for (int j = 0; j < h->n; j++) {
      InstDev& D = h->idev[j];
      D.tiles_x = (D.nx + nc - 1) / nc;
      D.tiles_y = h->seg > 0 ? (D.ny + h->seg - 1) / h->seg
                             : (int)std::min<int64_t>(band, D.ny);
      D.tile_begin = begin;
      begin += (int64_t)D.tiles_x * (h->seg > 0 ? D.tiles_y : D.ny);
    }
    h->total_tiles = begin;
    if (h->grid_req == -1) h->grid = (int)std::min<int64_t>(begin, 2147483647);
    CU(h, cudaMemcpyAsync(h->d_inst, h->idev.data(), sizeof(InstDev) * h->n,
                          cudaMemcpyHostToDevice, h->stream));
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    h->graph_failed = false;
    return wait(h);
  }
  const TileShape ts = TILE_SHAPES[h->tile];
  int64_t begin = 0;
  for (int j = 0; j < h->n; j++) {
    InstDev& D = h->idev[j];
    D.tiles_x = (D.nx + ts.tx - 1) / ts.tx;
    D.tiles_y = (D.ny + ts.ty - 1) / ts.ty;
    D.tile_begin = begin;
    begin += (int64_t)D.tiles_x * D.tiles_y;
  }
  h->total_tiles = begin;
  CU(h, cudaMemcpyAsync(h->d_inst, h->idev.data(), sizeof(InstDev) * h->n,
                        cudaMemcpyHostToDevice, h->stream));
  const int occ = step_occupancy(h->storage, h->tile);
  if (occ <= 0) return fail(h, LBE_ECUDA, "step kernel for tile %d cannot be resident", h->tile);
  if (h->grid_req == -1)
    h->grid = (int)(h->total_tiles < 2147483647 ? h->total_tiles : 2147483647);
  else if (h->grid_req > 0)
    h->grid = h->grid_req;
  else
    h->grid = occ * h->num_sms;
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  h->graph_failed = false;
  return wait(h);
}

cudaError_t launch_one_step(lbe_handle* h, int parity) {
  if (is_strip(h->tile)) {
    // the withhold test hook applies to one launch (never inside a graph:
    // run_steps launches that step directly)
    const int wh = h->withhold, pl = h->poll_lim;
    if (wh >= 0) {
      h->withhold = -1;
      h->poll_lim = STASH_POLLS;
    }
    const bool own = h->tile == STASH_OWN_ID;
    cudaError_t e = launch_stash(h->storage, h->d_inst, h->n, h->total_tiles, h->seg, parity,
                                 h->grid, h->d_err, pl, wh, h->d_seed, h->variants, own,
                                 h->stream);
    // kernel 7 leaves the periodic ghost columns to ghost_kernel, which also
    // advances the step counter; kernel 8 writes them itself
    if (e == cudaSuccess)
      e = own ? launch_seed_tick(h->d_seed, h->stream)
              : launch_ghosts(h->d_inst, h->n, h->max_ny, parity ^ 1, h->d_seed, h->stream);
    return e;
  }
  cudaError_t e = cudaSuccess;
  // varying density: the corrected p of Eq. 13 (and so its gradient) needs
  // u of every cell first, and the dissipation term the gradients of u: a
  // pass of its own
  if (h->vrho || h->dissip)
    e = h->storage == LBE_F64
            ? pcorr_f64(h->d_pinst, h->n, h->p_tiles, parity, h->p_grid, h->stream)
            : pcorr_f32(h->d_pinst, h->n, h->p_tiles, parity, h->p_grid, h->stream);
  if (e == cudaSuccess)
    e = launch_step(h->storage, h->tile, h->d_inst, h->n, h->total_tiles, parity, h->grid,
                    h->d_seed, h->stream);
  if (e == cudaSuccess) e = launch_seed_tick(h->d_seed, h->stream);
  return e;
}

lbe_status launch_steps_direct(lbe_handle* h, int64_t k) {
  for (int64_t s = 0; s < k; s++) {
    cudaError_t e = launch_one_step(h, h->parity);
    if (e != cudaSuccess) return fail(h, LBE_ECUDA, "step launch: %s", cudaGetErrorString(e));
    h->parity ^= 1;
    h->steps++;
    h->prev_valid = true;
  }
  return LBE_OK;
}

// Graph of two steps (parity 0 -> 1 -> 0), captured once per tile setup.
void ensure_graph(lbe_handle* h) {
  if (h->gexec || h->graph_failed) return;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    h->graph_failed = true;
    return;
  }
  cudaError_t e1 = launch_one_step(h, 0);
  cudaError_t e2 = launch_one_step(h, 1);
  cudaError_t e3 = cudaStreamEndCapture(h->stream, &g);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || !g ||
      cudaGraphInstantiate(&h->gexec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    h->gexec = nullptr;
    h->graph_failed = true;
  }
  if (g) cudaGraphDestroy(g);
}

lbe_status run_steps(lbe_handle* h, int64_t k) {
  if (k <= 0) return LBE_OK;
  if (h->withhold >= 0 && is_strip(h->tile)) {  // test hook: this step outside the graph
    lbe_status st = launch_steps_direct(h, 1);
    if (st) return st;
    k--;
  }
  if (k > 0 && h->parity == 1) {
    lbe_status st = launch_steps_direct(h, 1);
    if (st) return st;
    k--;
  }
  ensure_graph(h);
  if (h->gexec) {
    for (; k >= 2; k -= 2) {
      cudaError_t e = cudaGraphLaunch(h->gexec, h->stream);
      if (e != cudaSuccess) return fail(h, LBE_ECUDA, "graph launch: %s", cudaGetErrorString(e));
      h->steps += 2;
      h->prev_valid = true;
    }
  }
  return launch_steps_direct(h, k);
}

lbe_status ensure_scratch(lbe_handle* h) {
  if (h->scratch) return LBE_OK;
  CU(h, cudaMalloc(&h->scratch, sizeof(double) * 10 * (size_t)h->max_cells));
  CU(h, cudaMalloc(&h->d_partial, sizeof(double) * 6 * sums_blocks()));
  CU(h, cudaMalloc(&h->d_sums, sizeof(double) * 6));
  return LBE_OK;
}

lbe_status compute_fields(lbe_handle* h, int j, int which_parity, double* out) {
  const InstHost& H = h->inst[j];
  const TileShape ts = TILE_SHAPES[0];
  const int64_t tiles = (int64_t)((H.nx + ts.tx - 1) / ts.tx) * ((H.ny + ts.ty - 1) / ts.ty);
  cudaError_t e = launch_fields(h->storage, h->d_finst + j, tiles, which_parity, out, h->stream);
  if (e != cudaSuccess) return fail(h, LBE_ECUDA, "field kernel: %s", cudaGetErrorString(e));
  return LBE_OK;
}

// sums of instance j into host out6 (c, p, T, |du|^2, |u|^2, nonfinite)
lbe_status sums6(lbe_handle* h, int j, double out6[6]) {
  lbe_status st = ensure_scratch(h);
  if (st) return st;
  const InstHost& H = h->inst[j];
  const int64_t N = (int64_t)H.nx * H.ny;
  double* cur = h->scratch;
  double* prev = h->scratch + 5 * (size_t)h->max_cells;
  if ((st = compute_fields(h, j, h->parity, cur))) return st;
  const bool hp = h->prev_valid;
  if (hp && (st = compute_fields(h, j, h->parity ^ 1, prev))) return st;
  cudaError_t e = launch_sums(cur, hp ? prev : nullptr, N, h->d_partial, h->d_sums, h->stream);
  if (e != cudaSuccess) return fail(h, LBE_ECUDA, "sums kernel: %s", cudaGetErrorString(e));
  if ((st = to_host(h, out6, h->d_sums, 6 * sizeof(double)))) return st;
  return wait(h);
}

lbe_status create(int32_t n, const lbe_params* params, const lbe_init_fields* init, void* stream,
                  lbe_handle** out) {
  if (!out) return fail(nullptr, LBE_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !params || !init) return fail(nullptr, LBE_EINVAL, "need n >= 1, params, init");
  for (int j = 0; j < n; j++) {
    lbe_status st = check_params(params[j], j);
    if (st) return st;
    if (params[j].storage != params[0].storage)
      return fail(nullptr, LBE_EINVAL, "all instances must use the same storage");
    if (!init[j].c0 || !init[j].T0 || !init[j].Tbot || !init[j].Ttop)
      return fail(nullptr, LBE_EINVAL, "instance %d: NULL initial field", j);
  }
  if (fault_alloc()) return fail(nullptr, LBE_ENOMEM, "allocation failed (LBE_FAULT=alloc)");
  lbe_handle* h = new lbe_handle();
  h->n = n;
  h->storage = params[0].storage;
  h->inst.resize(n);
  h->idev.resize(n);
  auto bail = [&](lbe_status st) {
    std::string m = h->err;
    free_handle(h);
    g_thread_err = m;
    return st;
  };
#define CUB(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return bail(fail(h, e_ == cudaErrorMemoryAllocation ? LBE_ENOMEM : LBE_ECUDA, "%s: %s", \
                       #call, cudaGetErrorString(e_)));                                     \
  } while (0)
  CUB(cudaGetDevice(&h->device));
  CUB(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    CUB(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  CUB(cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming));
  const int st = h->storage;
  const size_t esz = st == LBE_F64 ? 8 : ((st == LBE_F32 || st == LBE_F16MIX) ? 4 : 2);
  for (int j = 0; j < n; j++) {
    InstHost& H = h->inst[j];
    H.p = params[j];
    H.nx = params[j].nx;
    H.ny = params[j].ny;
    H.pitch = round_up(H.nx + 2 * XG, 64);  // periodic ghost columns on both sides
    H.plane_bytes = ((uint64_t)H.ny * H.pitch * esz + 255) / 256 * 256;
    // the FP16 plane of the g_0 low part (16/32-bit forms) follows the
    // population planes
    const uint64_t lo_bytes = ((uint64_t)H.ny * H.pitch * 2 + 255) / 256 * 256;
    if (st == LBE_F16MIX) {
      // 9 planes of 8-byte words (f_i FP32 and two FP16 values), FP32 g_0
      H.pair_bytes = ((uint64_t)H.ny * H.pitch * 8 + 255) / 256 * 256;
      H.g0_off = 9 * H.pair_bytes;
      H.h_off = 0;
      H.f0_off = 0;
      H.g0lo_off = 0;  // in the words of plane 0
      H.buf_bytes = H.g0_off + H.plane_bytes;
    } else if (st == LBE_F16DEV || st == LBE_BF16DEV) {
      // 8 (f_i, g_i) pair planes (i >= 1), f_0, 9 hbar, FP32 g_0, low part
      H.pair_bytes = ((uint64_t)H.ny * H.pitch * 4 + 255) / 256 * 256;
      H.f0_off = 8 * H.pair_bytes;
      H.h_off = H.f0_off + H.plane_bytes;
      H.g0_off = H.h_off + 9 * H.plane_bytes;
      H.g0lo_off = H.g0_off + (((uint64_t)H.ny * H.pitch * 4 + 255) / 256 * 256);
      H.buf_bytes = H.g0lo_off + lo_bytes;
    } else if (st == LBE_F32) {
      // 9 (f_i, g_i) pair planes, 9 hbar planes, the g_0 low part
      H.g0_off = 0;
      H.pair_bytes = ((uint64_t)H.ny * H.pitch * 8 + 255) / 256 * 256;
      H.h_off = 9 * H.pair_bytes;
      H.g0lo_off = H.h_off + 9 * H.plane_bytes;
      H.buf_bytes = H.g0lo_off + lo_bytes;
    } else {
      H.g0_off = 0;
      H.g0lo_off = 0;
      H.buf_bytes = 27 * H.plane_bytes;
    }
    // ARENA_TAIL: reads of a strip's last warp may run past the last row of
    // the last plane (into pitch padding, never used); keep them allocated
    CUB(cudaMalloc(&H.arena, 2 * H.buf_bytes + ARENA_TAIL));
    CUB(cudaMemsetAsync(H.arena, 0, 2 * H.buf_bytes + ARENA_TAIL, h->stream));
    // walls: Tbot[nx], Ttop[nx] (double), then 4 x nx floats of T_w - T_r
    CUB(cudaMalloc(&H.walls, sizeof(double) * 2 * H.nx + sizeof(float) * 4 * H.nx));
    H.Tbot.assign(init[j].Tbot, init[j].Tbot + H.nx);
    H.Ttop.assign(init[j].Ttop, init[j].Ttop + H.nx);
    CUB(cudaMemcpyAsync(H.walls, H.Tbot.data(), sizeof(double) * H.nx, cudaMemcpyHostToDevice,
                        h->stream));
    CUB(cudaMemcpyAsync(H.walls + H.nx, H.Ttop.data(), sizeof(double) * H.nx,
                        cudaMemcpyHostToDevice, h->stream));
    if (H.p.interp != 0 || H.p.wall_mid != 0 || H.p.cos_wet != 0.0) h->variants = true;
    if (varying_rho(H.p)) {
      h->vrho = true;
      CUB(cudaMalloc(&H.pcorr, sizeof(double) * (size_t)H.nx * H.ny));
    }
    if (H.p.dissip == 1) {
      h->dissip = true;
      CUB(cudaMalloc(&H.uvel, sizeof(double) * 2 * (size_t)H.nx * H.ny));
    }
    fill_desc(h, j, h->idev[j]);
    {
      const InstDev& D = h->idev[j];
      H.wdev.resize(4 * (size_t)H.nx);
      for (int x = 0; x < H.nx; x++) {
        H.wdev[x] = (float)(H.Tbot[x] - (D.hr0 + D.hr1 * 0));
        H.wdev[H.nx + x] = (float)(H.Ttop[x] - (D.hr0 + D.hr1 * (H.ny - 1)));
        H.wdev[2 * H.nx + x] = (float)(H.Tbot[x] - (D.hr0 + D.hr1 * -0.5));
        H.wdev[3 * H.nx + x] = (float)(H.Ttop[x] - (D.hr0 + D.hr1 * (H.ny - 0.5)));
      }
      CUB(cudaMemcpyAsync(H.walls + 2 * H.nx, H.wdev.data(), sizeof(float) * 4 * H.nx,
                          cudaMemcpyHostToDevice, h->stream));
    }
    h->max_cells = std::max<int64_t>(h->max_cells, (int64_t)H.nx * H.ny);
  }
  CUB(cudaMalloc(&h->d_inst, sizeof(InstDev) * n));
  CUB(cudaMalloc(&h->d_finst, sizeof(InstDev) * n));
  {
    std::vector<InstDev> f = h->idev;
    const TileShape ts = TILE_SHAPES[0];
    for (auto& D : f) {
      D.tiles_x = (D.nx + ts.tx - 1) / ts.tx;
      D.tiles_y = (D.ny + ts.ty - 1) / ts.ty;
      D.tile_begin = 0;
    }
    CUB(cudaMemcpyAsync(h->d_finst, f.data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice,
                        h->stream));
    if (h->vrho || h->dissip) {
      // the pre-pass (corrected p, u): shape-0 tiles of all instances in
      // one work list
      int64_t begin = 0;
      for (auto& D : f) {
        D.tile_begin = begin;
        begin += (int64_t)D.tiles_x * D.tiles_y;
      }
      h->p_tiles = begin;
      h->p_grid = (int)std::min<int64_t>(begin, (int64_t)2 * h->num_sms);
      CUB(cudaMalloc(&h->d_pinst, sizeof(InstDev) * n));
      CUB(cudaMemcpyAsync(h->d_pinst, f.data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice,
                          h->stream));
    }
    CUB(cudaStreamSynchronize(h->stream));
  }
  // initial state of each instance: the rest state of every cell (three
  // numbers) from c0 and T0, pushed into buffer 0; one scratch of 5 values
  // per cell of the largest instance serves them all, in stream order
  {
    double* work = nullptr;
    CUB(cudaMalloc(&work, sizeof(double) * 5 * (size_t)h->max_cells));
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < n && e == cudaSuccess; j++) {
      InstHost& H = h->inst[j];
      const size_t N = (size_t)H.nx * H.ny;
      e = cudaMemcpyAsync(work, init[j].c0, sizeof(double) * N, cudaMemcpyHostToDevice,
                          h->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(work + N, init[j].T0, sizeof(double) * N, cudaMemcpyHostToDevice,
                            h->stream);
      if (e == cudaSuccess)
        e = launch_rest_state(h->d_finst + j, H.nx, H.ny, work, work + N, work + 2 * N,
                              h->stream);
      if (e == cudaSuccess)
        e = launch_push(h->storage, h->d_finst + j, H.nx, H.ny, work + 2 * N, 0, 1, h->stream);
    }
    cudaError_t es = cudaStreamSynchronize(h->stream);
    cudaFree(work);
    CUB(e);
    CUB(es);
  }
  CUB(cudaMalloc(&h->d_err, sizeof(int)));
  CUB(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  CUB(cudaMalloc(&h->d_seed, sizeof(uint32_t)));
  CUB(cudaMemsetAsync(h->d_seed, 0, sizeof(uint32_t), h->stream));
  h->withhold = fault_withhold();
  if (h->withhold >= 0) h->poll_lim = STASH_POLLS_TEST;
  {
    // default kernel: the stash strip kernel where it applies (16/32-bit
    // storage, every instance at least XG columns wide), else the tile kernel
    int min_nx = 1 << 30;
    double cells = 0.0, strips = 0.0;  // cells-weighted mean strips per instance
    for (auto& H : h->inst) {
      min_nx = std::min(min_nx, H.nx);
      const double c = (double)H.nx * H.ny;
      cells += c;
      strips += c * ((H.nx + TILE_SHAPES[STASH_ID].tx - 1) / TILE_SHAPES[STASH_ID].tx);
    }
    // which kernel refreshes the periodic ghost columns: the step itself for
    // narrow instances (a batch of 64 drops 128 to 768 wide, FP32: 23.3
    // GLUPS against 23.0 with ghost_kernel, F16MIX 27.3 against 26.3),
    // ghost_kernel for wide ones (4096^2, FP32: 24.2 against 24.0 in the
    // step, F16MIX 27.3 against 26.9)
    const int stash = strips <= 8.0 * cells ? STASH_OWN_ID : STASH_ID;
    // (the dissipation term's velocity gradients: the tile kernel only)
    h->tile = (h->storage == LBE_F64 || min_nx < XG || h->dissip) ? 0 : stash;
  }
  lbe_status s2 = setup_tiles(h);
  if (s2) return bail(s2);
  *out = h;
  return LBE_OK;
#undef CUB
}

lbe_status check_handle(lbe_handle* h, int32_t instance) {
  if (!h) return fail(nullptr, LBE_EINVAL, "handle is NULL");
  if (instance < 0 || instance >= h->n) return fail(h, LBE_EINVAL, "instance %d out of range", instance);
  return LBE_OK;
}

// ------------------------------------------------------------------ adjoint
// Device allocation owned by a scope (freed on every return path).
struct DevBuf {
  char* p = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  double* d() const { return reinterpret_cast<double*>(p); }
};

lbe_status dalloc(lbe_handle* h, DevBuf& b, size_t bytes, const char* what) {
  if (fault_alloc() || cudaMalloc(&b.p, bytes ? bytes : 1) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(h, LBE_ENOMEM, "adjoint: cannot allocate %zu bytes for %s", bytes, what);
  }
  return LBE_OK;
}

lbe_status check_adjoint_handle(lbe_handle* h) {
  lbe_status st = check_handle(h, 0);
  if (st) return st;
  if (h->n != 1) return fail(h, LBE_EINVAL, "the adjoint needs a handle of one instance (has %d)", h->n);
  if (h->vrho) return fail(h, LBE_EINVAL, "the adjoint is of the uniform-density step (rho2 = rho)");
  {
    const lbe_params& p = h->inst[0].p;
    if (p.interp != 0 || p.wall_mid != 0 || p.cos_wet != 0.0 || p.dissip != 0)
      return fail(h, LBE_EINVAL,
                  "the adjoint is of the default variants (interp, wall_mid, cos_wet, dissip "
                  "all 0)");
  }
  if (h->bad) return fail(h, LBE_ESTATE, "handle is in an error state; set a state or load a checkpoint");
  return LBE_OK;
}

// Checkpointed forward + reverse sweep (see lbe_adjoint in lbe.h).
lbe_status adjoint_run(lbe_handle* h, const lbe_adjoint_spec& sp, double* loss, double* grad,
                       double* dT0, double* dQ0, bool on_device) {
  InstHost& H = h->inst[0];
  const int nx = H.nx, ny = H.ny;
  const size_t N = (size_t)nx * ny, S27 = 27 * N;
  const int64_t NS = sp.steps, W = sp.window, K = sp.ckpt_every;
  const int64_t nseg = (NS + K - 1) / K;
  const int64_t kk = K < NS ? K : NS;
  const InstDev* d1 = h->d_finst;
  // the reverse sweep's arithmetic follows the forward's: FP64 for an FP64
  // handle, FP32 otherwise (the trajectory is then an FP32 one anyway)
  const bool fp32 = h->storage != LBE_F64;
  lbe_status st;
  DevBuf ck, states, abuf, scr, small, fin;
  if ((st = dalloc(h, ck, (size_t)nseg * H.buf_bytes, "checkpoints"))) return st;
  if ((st = dalloc(h, states, sizeof(double) * (size_t)(kk + 1) * S27, "segment states"))) return st;
  if ((st = dalloc(h, abuf, sizeof(double) * 2 * S27, "adjoint states"))) return st;
  if ((st = dalloc(h, scr, sizeof(double) * (size_t)adjoint_scratch_doubles(nx, ny), "scratch")))
    return st;
  if ((st = dalloc(h, small, sizeof(double) * (size_t)(4 + 4 * W), "reductions"))) return st;
  if ((st = dalloc(h, fin, H.buf_bytes, "final state"))) return st;
  double* theta = small.d();
  double* obs = theta + 4;
  CU(h, cudaMemsetAsync(theta, 0, sizeof(double) * 4, h->stream));
  auto cur_buf = [&]() { return H.arena + (size_t)h->parity * H.buf_bytes; };

  // forward: raw checkpoint at the start of every segment
  const int64_t steps0 = h->steps;
  for (int64_t sg = 0; sg < nseg; sg++) {
    CU(h, cudaMemcpyAsync(ck.p + (size_t)sg * H.buf_bytes, cur_buf(), H.buf_bytes,
                          cudaMemcpyDeviceToDevice, h->stream));
    const int64_t len = std::min(K, NS - sg * K);
    if ((st = run_steps(h, len))) return st;
    if ((st = wait(h))) return st;
  }
  const int fin_parity = h->parity;
  CU(h, cudaMemcpyAsync(fin.p, cur_buf(), H.buf_bytes, cudaMemcpyDeviceToDevice, h->stream));

  // reverse sweep over the segments; a_nxt holds dL/dQ_{n+1}
  double* a_cur = abuf.d();
  double* a_nxt = abuf.d() + S27;
  bool have_next = false;
  const int64_t first_w = NS - W + 1;
  for (int64_t sg = nseg - 1; sg >= 0; sg--) {
    const int64_t n0 = sg * K;
    const int64_t n1 = (sg == nseg - 1) ? NS : n0 + K - 1;
    CU(h, cudaMemcpyAsync(cur_buf(), ck.p + (size_t)sg * H.buf_bytes, H.buf_bytes,
                          cudaMemcpyDeviceToDevice, h->stream));
    // the step counter as in the forward run, so that the stochastic
    // rounding of a 16-bit storage recomputes the same states
    CU(h, launch_seed_set(h->d_seed, (uint32_t)(steps0 + n0), h->stream));
    cudaError_t e = launch_pull(h->storage, d1, nx, ny, states.d(), h->parity, h->stream);
    for (int64_t t = 1; e == cudaSuccess && t <= n1 - n0; t++) {
      if ((st = launch_steps_direct(h, 1))) return st;
      e = launch_pull(h->storage, d1, nx, ny, states.d() + (size_t)t * S27, h->parity, h->stream);
    }
    for (int64_t n = n1; e == cudaSuccess && n >= n0; n--) {
      const double* Q = states.d() + (size_t)(n - n0) * S27;
      const double wl = n >= first_w ? 1.0 / (double)W : 0.0;
      double* o = n >= first_w ? obs + 4 * (n - first_w) : nullptr;
      if (o) e = launch_observable(d1, nx, ny, Q, scr.d(), o, h->stream);
      if (e == cudaSuccess)
        e = launch_adjoint_step(d1, nx, ny, Q, have_next ? a_nxt : nullptr, wl, o, a_cur, theta,
                                scr.d(), fp32, h->stream);
      std::swap(a_cur, a_nxt);
      have_next = true;
    }
    if (e != cudaSuccess) return fail(h, LBE_ECUDA, "adjoint sweep: %s", cudaGetErrorString(e));
    if ((st = wait(h))) return st;
  }
  // a_nxt = dL/dQ_0
  if (dT0) {
    double* dst = on_device ? dT0 : scr.d();
    cudaError_t e = launch_adjoint_dT0(d1, nx, ny, a_nxt, dst, h->stream);
    if (e != cudaSuccess) return fail(h, LBE_ECUDA, "dT0 kernel: %s", cudaGetErrorString(e));
    if (!on_device && (st = to_host(h, dT0, dst, sizeof(double) * N))) return st;
  }
  if (dQ0) {
    if (on_device)
      CU(h, cudaMemcpyAsync(dQ0, a_nxt, sizeof(double) * S27, cudaMemcpyDeviceToDevice,
                            h->stream));
    else if ((st = to_host(h, dQ0, a_nxt, sizeof(double) * S27)))
      return st;
  }
  std::vector<double> hobs(4 * (size_t)W), hth(4);
  if ((st = to_host(h, hobs.data(), obs, sizeof(double) * 4 * W))) return st;
  if ((st = to_host(h, hth.data(), theta, sizeof(double) * 4))) return st;
  // back to the state after the forward run
  h->parity = fin_parity;
  CU(h, cudaMemcpyAsync(cur_buf(), fin.p, H.buf_bytes, cudaMemcpyDeviceToDevice, h->stream));
  h->steps = steps0 + NS;
  CU(h, launch_seed_set(h->d_seed, (uint32_t)h->steps, h->stream));
  h->prev_valid = false;
  if ((st = wait(h))) return st;
  if (loss) {
    double L = 0.0;
    for (int64_t j = 0; j < W; j++) L += hobs[4 * j] / hobs[4 * j + 1];
    *loss = L / (double)W;
  }
  if (grad)
    for (int j = 0; j < 3; j++) grad[j] = hth[j];
  return LBE_OK;
}

}  // namespace

void lbe::set_thread_error(const char* msg) { g_thread_err = msg ? msg : ""; }

extern "C" {

int32_t lbe_abi_version(void) { return LBE_ABI_VERSION; }

lbe_status lbe_init(const lbe_params* params, const lbe_init_fields* init, void* stream,
                    lbe_handle** out) {
  return create(1, params, init, stream, out);
}

lbe_status lbe_init_batch(int32_t n, const lbe_params* params, const lbe_init_fields* init,
                          void* stream, lbe_handle** out) {
  return create(n, params, init, stream, out);
}

lbe_status lbe_step(lbe_handle* h, int64_t nsteps) {
  if (!h) return fail(nullptr, LBE_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(h, LBE_EINVAL, "nsteps must be >= 0");
  if (h->bad) return fail(h, LBE_ESTATE, "handle is in an error state; set a state or load a checkpoint");
  int ce = 0;
  for (auto& H : h->inst)
    if (H.p.check_every > 0 && (ce == 0 || H.p.check_every < ce)) ce = H.p.check_every;
  if (ce == 0) return run_steps(h, nsteps);
  int64_t left = nsteps;
  while (left > 0) {
    int64_t to_check = ce - (h->steps % ce);
    int64_t k = left < to_check ? left : to_check;
    lbe_status st = run_steps(h, k);
    if (st) return st;
    left -= k;
    if (h->steps % ce == 0) {
      for (int j = 0; j < h->n; j++) {
        double s6[6];
        if ((st = sums6(h, j, s6))) return st;
        if (s6[5] != 0)
          return fail(h, LBE_ENAN, "instance %d: %.0f non-finite field values at step %lld", j,
                      s6[5], (long long)h->steps);
      }
    }
  }
  return wait(h);
}

lbe_status lbe_synchronize(lbe_handle* h) {
  if (!h) return fail(nullptr, LBE_EINVAL, "handle is NULL");
  return wait(h);
}

lbe_status lbe_fields(lbe_handle* h, int32_t instance, uint32_t mask, void* const dst[5],
                      int32_t on_device, int32_t dtype) {
  lbe_status st = check_handle(h, instance);
  if (st) return st;
  if (!dst) return fail(h, LBE_EINVAL, "dst is NULL");
  if (dtype != 0 && dtype != 1) return fail(h, LBE_EINVAL, "dtype must be 0 (f64) or 1 (f32)");
  for (int k = 0; k < 5; k++)
    if ((mask >> k & 1u) && !dst[k]) return fail(h, LBE_EINVAL, "dst[%d] is NULL", k);
  if ((st = ensure_scratch(h))) return st;
  const InstHost& H = h->inst[instance];
  const int64_t N = (int64_t)H.nx * H.ny;
  double* cur = h->scratch;
  if ((st = compute_fields(h, instance, h->parity, cur))) return st;
  float* tmp32 = reinterpret_cast<float*>(h->scratch + 5 * (size_t)h->max_cells);
  for (int k = 0; k < 5; k++) {
    if (!(mask >> k & 1u)) continue;
    const double* src = cur + k * N;
    if (dtype == 0) {
      if (on_device)
        CU(h, cudaMemcpyAsync(dst[k], src, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                              h->stream));
      else if ((st = to_host(h, dst[k], src, sizeof(double) * N)))
        return st;
    } else if (on_device) {
      cudaError_t e = launch_f64_to_f32(src, reinterpret_cast<float*>(dst[k]), N, h->stream);
      if (e != cudaSuccess) return fail(h, LBE_ECUDA, "cast kernel: %s", cudaGetErrorString(e));
    } else {
      cudaError_t e = launch_f64_to_f32(src, tmp32, N, h->stream);
      if (e != cudaSuccess) return fail(h, LBE_ECUDA, "cast kernel: %s", cudaGetErrorString(e));
      if ((st = to_host(h, dst[k], tmp32, sizeof(float) * N))) return st;
      if ((st = wait(h))) return st;  // tmp32 is reused by the next field
    }
  }
  return wait(h);
}

lbe_status lbe_sums(lbe_handle* h, int32_t instance, double out[5]) {
  lbe_status st = check_handle(h, instance);
  if (st) return st;
  if (!out) return fail(h, LBE_EINVAL, "out is NULL");
  double s6[6];
  if ((st = sums6(h, instance, s6))) return st;
  const InstHost& H = h->inst[instance];
  out[0] = s6[0];
  out[1] = s6[1];
  out[2] = s6[2] * H.p.rho * H.p.cv;
  out[3] = (h->prev_valid && s6[4] > 0) ? std::sqrt(s6[3]) / std::sqrt(s6[4]) : 0.0;
  out[4] = s6[5];
  return LBE_OK;
}

lbe_status lbe_get_state(lbe_handle* h, int32_t instance, double* pops, int32_t on_device) {
  lbe_status st = check_handle(h, instance);
  if (st) return st;
  if (!pops) return fail(h, LBE_EINVAL, "pops is NULL");
  const InstHost& H = h->inst[instance];
  const size_t N = (size_t)H.nx * H.ny;
  double* d = pops;
  if (!on_device) CU(h, cudaMalloc(&d, sizeof(double) * 27 * N));
  cudaError_t e = launch_pull(h->storage, h->d_finst + instance, H.nx, H.ny, d, h->parity, h->stream);
  if (e == cudaSuccess && !on_device) {
    st = wait_stream(h);  // (a copy into pageable memory would block unboundedly)
    if (st == LBE_OK)
      e = cudaMemcpyAsync(pops, d, sizeof(double) * 27 * N, cudaMemcpyDeviceToHost, h->stream);
  }
  if (st == LBE_OK) st = wait(h);
  if (!on_device) cudaFree(d);
  if (e != cudaSuccess) return fail(h, LBE_ECUDA, "get_state: %s", cudaGetErrorString(e));
  return st;
}

lbe_status lbe_set_state(lbe_handle* h, int32_t instance, const double* pops, int32_t on_device) {
  lbe_status st = check_handle(h, instance);
  if (st) return st;
  if (!pops) return fail(h, LBE_EINVAL, "pops is NULL");
  const InstHost& H = h->inst[instance];
  const size_t N = (size_t)H.nx * H.ny;
  double* d = const_cast<double*>(pops);
  if (!on_device) {
    CU(h, cudaMalloc(&d, sizeof(double) * 27 * N));
    cudaError_t e = cudaMemcpyAsync(d, pops, sizeof(double) * 27 * N, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
      cudaFree(d);
      return fail(h, LBE_ECUDA, "set_state copy: %s", cudaGetErrorString(e));
    }
  }
  // a new state: clear the device error word of an earlier copy time-out
  cudaError_t e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
  if (e == cudaSuccess)
    e = launch_push(h->storage, h->d_finst + instance, H.nx, H.ny, d, h->parity, 0, h->stream);
  st = wait(h);
  if (!on_device) cudaFree(d);
  if (e != cudaSuccess) return fail(h, LBE_ECUDA, "set_state: %s", cudaGetErrorString(e));
  if (st) return st;
  h->bad = false;
  h->prev_valid = false;
  return LBE_OK;
}

// checkpoint format: "LBECKPT2", int32 n, int32 storage, int64 steps, then per
// instance: lbe_params, Tbot[nx], Ttop[nx], uint64 nbytes, the raw bytes of the
// buffer the next step reads (so a restart continues bit for bit)
lbe_status lbe_save(lbe_handle* h, const char* path) {
  if (!h || !path) return fail(h, LBE_EINVAL, "handle or path is NULL");
  lbe_status st = wait(h);
  if (st) return st;
  FILE* fp = fopen(path, "wb");
  if (!fp) return fail(h, LBE_EINVAL, "cannot open %s for writing", path);
  const char magic[8] = {'L', 'B', 'E', 'C', 'K', 'P', 'T', '2'};
  const int32_t hdr[2] = {h->n, h->storage};
  const int64_t steps = h->steps;
  bool ok = fwrite(magic, 1, 8, fp) == 8 && fwrite(hdr, sizeof hdr, 1, fp) == 1 &&
            fwrite(&steps, sizeof steps, 1, fp) == 1;
  for (int j = 0; ok && j < h->n; j++) {
    const InstHost& H = h->inst[j];
    std::vector<char> raw(H.buf_bytes);
    cudaError_t e = cudaMemcpy(raw.data(), H.arena + (size_t)h->parity * H.buf_bytes,
                               H.buf_bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      fclose(fp);
      return fail(h, LBE_ECUDA, "save copy: %s", cudaGetErrorString(e));
    }
    const uint64_t nb = H.buf_bytes;
    ok = fwrite(&H.p, sizeof H.p, 1, fp) == 1 &&
         fwrite(H.Tbot.data(), sizeof(double), H.nx, fp) == (size_t)H.nx &&
         fwrite(H.Ttop.data(), sizeof(double), H.nx, fp) == (size_t)H.nx &&
         fwrite(&nb, sizeof nb, 1, fp) == 1 && fwrite(raw.data(), 1, nb, fp) == nb;
  }
  if (fclose(fp) != 0) ok = false;
  return ok ? LBE_OK : fail(h, LBE_EINVAL, "short write to %s", path);
}

lbe_status lbe_load(lbe_handle* h, const char* path) {
  if (!h || !path) return fail(h, LBE_EINVAL, "handle or path is NULL");
  lbe_status st = wait_stream(h);  // the error word is cleared below
  if (st) return st;
  FILE* fp = fopen(path, "rb");
  if (!fp) return fail(h, LBE_EINVAL, "cannot open %s", path);
  char magic[8];
  int32_t hdr[2];
  int64_t steps;
  bool ok = fread(magic, 1, 8, fp) == 8 && memcmp(magic, "LBECKPT2", 8) == 0 &&
            fread(hdr, sizeof hdr, 1, fp) == 1 && fread(&steps, sizeof steps, 1, fp) == 1;
  if (!ok || hdr[0] != h->n || hdr[1] != h->storage) {
    fclose(fp);
    return fail(h, LBE_EINVAL, "%s: not a checkpoint of this handle's layout", path);
  }
  std::vector<std::vector<char>> raws(h->n);
  for (int j = 0; j < h->n; j++) {
    InstHost& H = h->inst[j];
    lbe_params p;
    uint64_t nb = 0;
    std::vector<double> tb(H.nx), tt(H.nx);
    ok = fread(&p, sizeof p, 1, fp) == 1 && p.nx == H.nx && p.ny == H.ny &&
         fread(tb.data(), sizeof(double), H.nx, fp) == (size_t)H.nx &&
         fread(tt.data(), sizeof(double), H.nx, fp) == (size_t)H.nx &&
         fread(&nb, sizeof nb, 1, fp) == 1 && nb == H.buf_bytes;
    if (ok) {
      raws[j].resize(nb);
      ok = fread(raws[j].data(), 1, nb, fp) == nb;
    }
    if (!ok) {
      fclose(fp);
      return fail(h, LBE_EINVAL, "%s: truncated or mismatched instance %d", path, j);
    }
    if (memcmp(&p, &H.p, sizeof p) != 0 || tb != H.Tbot || tt != H.Ttop) {
      fclose(fp);
      return fail(h, LBE_EINVAL, "%s: instance %d has other parameters or walls", path, j);
    }
  }
  fclose(fp);
  for (int j = 0; j < h->n; j++) {
    InstHost& H = h->inst[j];
    CU(h, cudaMemcpy(H.arena + (size_t)h->parity * H.buf_bytes, raws[j].data(), H.buf_bytes,
                     cudaMemcpyHostToDevice));
  }
  CU(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  // the random bits of the stochastic rounding follow the step count
  CU(h, launch_seed_set(h->d_seed, (uint32_t)steps, h->stream));
  if ((st = wait_stream(h))) return st;
  h->steps = steps;
  h->bad = false;
  h->prev_valid = false;
  return LBE_OK;
}

int32_t lbe_num_tiles(void) { return NUM_TILES; }

lbe_status lbe_tile_shape(int32_t tile_id, int32_t* tx, int32_t* ty) {
  if (tile_id < 0 || tile_id >= NUM_TILES || !tx || !ty)
    return fail(nullptr, LBE_EINVAL, "tile id %d out of range", tile_id);
  *tx = TILE_SHAPES[tile_id].tx;
  *ty = TILE_SHAPES[tile_id].ty;
  return LBE_OK;
}

lbe_status lbe_set_tile(lbe_handle* h, int32_t tile_id, int32_t grid_ctas, int32_t seg_rows) {
  if (!h) return fail(nullptr, LBE_EINVAL, "handle is NULL");
  if (!tile_available(h->storage, tile_id))
    return fail(h, LBE_EINVAL, "kernel %d is not built for this storage", tile_id);
  if (is_strip(tile_id)) {
    for (auto& H : h->inst)
      if (H.nx < XG) return fail(h, LBE_EINVAL, "the strip kernel needs nx >= %d", XG);
    if (h->dissip)
      return fail(h, LBE_EINVAL, "the dissipation term (dissip = 1) runs on the tile kernel");
  }
  if (grid_ctas < -1) return fail(h, LBE_EINVAL, "grid_ctas must be >= -1");
  if (seg_rows < 0 && !is_strip(tile_id))
    return fail(h, LBE_EINVAL, "seg_rows < 0 (balanced pieces) is for the strip kernel");
  lbe_status st = wait(h);
  if (st) return st;
  h->tile = tile_id;
  h->grid_req = grid_ctas;
  h->seg_req = seg_rows;
  return setup_tiles(h);
}

lbe_status lbe_get_tile(const lbe_handle* h, int32_t out[4]) {
  if (!h || !out) return fail(nullptr, LBE_EINVAL, "handle or out is NULL");
  out[0] = h->tile;
  out[1] = h->grid;
  out[2] = is_strip(h->tile) ? h->seg : 0;
  // work items: with balanced ranges (strip kernel, seg <= 0), one per CTA
  const int64_t items = (is_strip(h->tile) && h->seg <= 0)
                            ? std::min<int64_t>(h->total_tiles, h->grid)
                            : h->total_tiles;
  out[3] = (int32_t)std::min<int64_t>(items, 2147483647);
  return LBE_OK;
}

lbe_status lbe_adjoint(lbe_handle* h, const lbe_adjoint_spec* spec, double* loss,
                       double grad[3], double* dT0, double* dQ0, int32_t on_device) {
  lbe_status st = check_adjoint_handle(h);
  if (st) return st;
  if (!spec) return fail(h, LBE_EINVAL, "spec is NULL");
  if (spec->steps < 1) return fail(h, LBE_EINVAL, "spec.steps must be >= 1");
  if (spec->window < 1 || spec->window > spec->steps)
    return fail(h, LBE_EINVAL, "spec.window must be in [1, steps]");
  if (spec->ckpt_every < 1) return fail(h, LBE_EINVAL, "spec.ckpt_every must be >= 1");
  return adjoint_run(h, *spec, loss, grad, dT0, dQ0, on_device != 0);
}

lbe_status lbe_adjoint_step(lbe_handle* h, const double* Q, const double* a_next, double wl,
                            double* a_out, double grad[3]) {
  lbe_status st = check_adjoint_handle(h);
  if (st) return st;
  if (!Q || !a_out) return fail(h, LBE_EINVAL, "Q and a_out must be device pointers");
  const InstHost& H = h->inst[0];
  DevBuf scr, small;
  if ((st = dalloc(h, scr, sizeof(double) * (size_t)adjoint_scratch_doubles(H.nx, H.ny), "scratch")))
    return st;
  if ((st = dalloc(h, small, sizeof(double) * 8, "reductions"))) return st;
  double* theta = small.d();
  double* obs = theta + 4;
  CU(h, cudaMemsetAsync(theta, 0, sizeof(double) * 4, h->stream));
  cudaError_t e = cudaSuccess;
  if (wl != 0.0) e = launch_observable(h->d_finst, H.nx, H.ny, Q, scr.d(), obs, h->stream);
  if (e == cudaSuccess)
    e = launch_adjoint_step(h->d_finst, H.nx, H.ny, Q, a_next, wl, obs, a_out, theta, scr.d(),
                            false, h->stream);
  if (e != cudaSuccess) return fail(h, LBE_ECUDA, "adjoint step: %s", cudaGetErrorString(e));
  double th[4];
  if ((st = to_host(h, th, theta, sizeof th))) return st;
  if ((st = wait(h))) return st;
  if (grad)
    for (int j = 0; j < 3; j++) grad[j] += th[j];
  return LBE_OK;
}

lbe_status lbe_observable(lbe_handle* h, const double* Q, double* out) {
  lbe_status st = check_adjoint_handle(h);
  if (st) return st;
  if (!Q || !out) return fail(h, LBE_EINVAL, "Q (device) and out (host) must not be NULL");
  const InstHost& H = h->inst[0];
  DevBuf scr, small;
  if ((st = dalloc(h, scr, sizeof(double) * (size_t)adjoint_scratch_doubles(H.nx, H.ny), "scratch")))
    return st;
  if ((st = dalloc(h, small, sizeof(double) * 4, "reductions"))) return st;
  cudaError_t e = launch_observable(h->d_finst, H.nx, H.ny, Q, scr.d(), small.d(), h->stream);
  if (e != cudaSuccess) return fail(h, LBE_ECUDA, "observable: %s", cudaGetErrorString(e));
  double o[4];
  if ((st = to_host(h, o, small.d(), sizeof o))) return st;
  if ((st = wait(h))) return st;
  *out = o[0] / o[1];
  return LBE_OK;
}

int64_t lbe_steps_done(const lbe_handle* h) { return h ? h->steps : -1; }
void* lbe_stream(const lbe_handle* h) { return h ? (void*)h->stream : nullptr; }
int32_t lbe_num_instances(const lbe_handle* h) { return h ? h->n : 0; }
int64_t lbe_state_bytes(const lbe_handle* h) {
  if (!h) return 0;
  int64_t b = 0;
  for (auto& H : h->inst) b += 2 * (int64_t)H.buf_bytes;
  return b;
}

void lbe_destroy(lbe_handle* h) {
  if (!h) return;
  if (h->stream) wait_stream(h);  // bounded; the buffers are freed either way
  free_handle(h);
}

const char* lbe_last_error(const lbe_handle* h) {
  return h ? h->err.c_str() : g_thread_err.c_str();
}

}  // extern "C"
