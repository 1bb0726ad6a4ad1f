// C ABI of libpk (include/pk.h): argument validation, workspace layout, the cuFFT plan cache and the
// host-side sequencing of the kernels of each entry point.
#include <cufft.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <string>
#include <tuple>

#include "host.cuh"

namespace pk {

// ---- errors -------------------------------------------------------------------------------------------

static thread_local std::string t_err;

pk_status fail(pk_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return st;
}

pk_status cuda_fail(cudaError_t e, const char* where) {
  return fail(PK_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

void clear_err() { t_err.clear(); }

static std::atomic<long long> g_launches{0};
void count_launch(int k) { g_launches += k; }

// ---- stage timing ---------------------------------------------------------------------------------------

constexpr int kProfMarks = 6;
static thread_local bool t_prof = false;
static thread_local cudaEvent_t t_ev[kProfMarks] = {};
static thread_local bool t_ev_rec[kProfMarks] = {};

void prof_mark(int k, cudaStream_t s) {
  if (!t_prof || k < 0 || k >= kProfMarks) return;
  if (!t_ev[k] && cudaEventCreate(&t_ev[k]) != cudaSuccess) return;
  if (cudaEventRecord(t_ev[k], s) == cudaSuccess) t_ev_rec[k] = true;
}

cudaError_t ensure_dynamic_smem(const void* kernel, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = done[{kernel, dev}];
  if (have >= smem) return cudaSuccess;
  if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess) return e;
  have = smem;
  return cudaSuccess;
}

int num_sms() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 132;
  cache[dev] = n;
  return n;
}

// ---- validation -----------------------------------------------------------------------------------------

pk_status validate(const pk_config* c) {
  if (!c) return fail(PK_EINVAL, "cfg is NULL");
  if (c->ng < 8 || c->ng > 1024 || (c->ng & 1)) return fail(PK_EINVAL, "ng must be even and in [8, 1024] (got %d)", c->ng);
  if (c->order < 1 || c->order > 6) return fail(PK_EINVAL, "order must be 1..6 (got %d)", c->order);
  if (c->order > 4 && c->prec == PK_FIXED64) return fail(PK_EINVAL, "orders 5 and 6 need PK_FP64 or PK_FP32");
  if (c->interlace != 0 && c->interlace != 1) return fail(PK_EINVAL, "interlace must be 0 or 1");
  if (c->prec < PK_FP64 || c->prec > PK_FIXED64) return fail(PK_EINVAL, "prec must be PK_FP64, PK_FP32 or PK_FIXED64");
  if (!(c->box > 0.0) || !std::isfinite(c->box)) return fail(PK_EINVAL, "box must be finite and > 0");
  if (c->bin_lo2 < 0 || c->bin_w2 < 1 || c->nbins < 1 || c->nbins > 2048)
    return fail(PK_EINVAL, "bins: need bin_lo2 >= 0, bin_w2 >= 1, 1 <= nbins <= 2048");
  if (int64_t(c->bin_lo2) + int64_t(c->bin_w2) * c->nbins > (int64_t(1) << 30)) return fail(PK_EINVAL, "bin edges too large");
  if (c->subtract_shot != 0 && c->subtract_shot != 1) return fail(PK_EINVAL, "subtract_shot must be 0 or 1");
  if (c->tile_run != 0 && c->tile_run != 1 && c->tile_run != 2 && c->tile_run != 4)
    return fail(PK_EINVAL, "tile_run must be 0, 1, 2 or 4");
  return PK_OK;
}

// Measured on one GB300 (assignment of PCS + interlacing): a single catalogue of 170 or 512 particles
// per tile runs 9 % or 2 % faster with runs of two tiles (fewer region nodes to flush per particle,
// fuller buckets), runs of four are slower (two blocks per SM), and batches of 32 catalogues run
// fastest with single tiles (fewer blocks per catalogue at the lower occupancy of longer runs).
int scatter_run(const pk_config* c, int64_t n, int ncat) {
  if (c->tile_run > 0) return c->tile_run;
  const int nt = c->ng / kTileCells;
  const double mean = double(n) / (double(std::max(ncat, 1)) * nt * nt * nt);
  return mean >= 100.0 && mean <= 700.0 ? 2 : 1;
}

// ---- cuFFT plans ------------------------------------------------------------------------------------------

static std::mutex g_plan_mu;
static std::map<std::tuple<int, int, int, int>, PlanEntry> g_plans;  // (device, ng, type, batch)

// kind: 0 R2C, 1 D2Z, 2 C2R, 3 Z2D; in-place on the padded layout [ng][ng][ng+2] (reals).
pk_status get_plan(int ng, int kind, int batch, PlanEntry* out) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto key = std::make_tuple(dev, ng, kind, batch);
  auto it = g_plans.find(key);
  if (it != g_plans.end()) {
    *out = it->second;
    return PK_OK;
  }
  PlanEntry e;
  const long long per = (long long)ng * ng * (ng + 2);
  e.batch = batch;
  e.dist = per;
  {  // the largest divisor of batch whose grids stay within 2^31 - 1 reals (at least one grid)
    const long long lim = std::max<long long>(1, 2147483647LL / per);
    e.sub = 1;
    for (int d = 1; d <= batch; ++d)
      if (batch % d == 0 && d <= lim) e.sub = d;
  }
  cufftHandle h = 0;
  if (cufftCreate(&h) != CUFFT_SUCCESS) return fail(PK_ECUFFT, "cufftCreate failed");
  e.h = int(h);
  if (cufftSetAutoAllocation(h, 0) != CUFFT_SUCCESS) return fail(PK_ECUFFT, "cufftSetAutoAllocation failed");
  long long n[3] = {ng, ng, ng};
  long long rem[3] = {ng, ng, ng + 2};
  long long cem[3] = {ng, ng, ng / 2 + 1};
  const long long rdist = (long long)ng * ng * (ng + 2), cdist = (long long)ng * ng * (ng / 2 + 1);
  static const cufftType types[4] = {CUFFT_R2C, CUFFT_D2Z, CUFFT_C2R, CUFFT_Z2D};
  const bool fwd = kind < 2;
  size_t work = 0;
  cufftResult r = cufftMakePlanMany64(h, 3, n, fwd ? rem : cem, 1, fwd ? rdist : cdist, fwd ? cem : rem, 1,
                                      fwd ? cdist : rdist, types[kind], e.sub, &work);
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(h);
    return fail(PK_ECUFFT, "cufftMakePlanMany64 failed (%d) for ng=%d kind=%d batch=%d", int(r), ng, kind, batch);
  }
  e.work = work;
  g_plans[key] = e;
  *out = e;
  return PK_OK;
}

pk_status exec_plan(const PlanEntry& p, int kind, void* data, void* work, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  if (cufftSetStream(p.h, s) != CUFFT_SUCCESS) return fail(PK_ECUFFT, "cufftSetStream failed");
  if (cufftSetWorkArea(p.h, work) != CUFFT_SUCCESS) return fail(PK_ECUFFT, "cufftSetWorkArea failed");
  const size_t elem = (kind == 1 || kind == 3) ? 8 : 4;
  for (int g = 0; g < p.batch; g += p.sub) {
    void* gd = static_cast<char*>(data) + size_t(g) * size_t(p.dist) * elem;
    cufftResult r;
    switch (kind) {
      case 0: r = cufftExecR2C(p.h, static_cast<cufftReal*>(gd), static_cast<cufftComplex*>(gd)); break;
      case 1: r = cufftExecD2Z(p.h, static_cast<cufftDoubleReal*>(gd), static_cast<cufftDoubleComplex*>(gd)); break;
      case 2: r = cufftExecC2R(p.h, static_cast<cufftComplex*>(gd), static_cast<cufftReal*>(gd)); break;
      default: r = cufftExecZ2D(p.h, static_cast<cufftDoubleComplex*>(gd), static_cast<cufftDoubleReal*>(gd)); break;
    }
    if (r != CUFFT_SUCCESS) return fail(PK_ECUFFT, "cuFFT exec failed (%d)", int(r));
  }
  return PK_OK;
}

// ---- shared sequencing ----------------------------------------------------------------------------------


pk_status carve_grid_stage(const pk_config* c, Carver& cv, GridStage* g) {
  const bool dbl = c->prec != PK_FP32;
  const int ngrid = c->interlace ? 2 : 1;
  g->kind = dbl ? 1 : 0;
  g->grids = cv.take<char>(size_t(ngrid) * padded_count(c->ng) * (dbl ? 8 : 4));
  g->tables = cv.take<char>(estimate_table_bytes(c->ng, dbl));
  g->wsums = cv.take<double>(3);
  g->bin_sum = cv.take<double>(c->nbins);
  g->bin_k = cv.take<double>(c->nbins);
  g->bin_cnt = cv.take<unsigned long long>(c->nbins);
  g->bin_aux = cv.take<double>(c->nbins);
  pk_status st = get_plan(c->ng, g->kind, ngrid, &g->plan);
  if (st != PK_OK) return st;
  g->fft_work = cv.take<char>(std::max<size_t>(g->plan.work, 256));
  return PK_OK;
}

// FFT of the padded grids, then the fused estimate (and optional finalisation into pk outputs).
pk_status run_fft_estimate(const pk_config* c, GridStage& g, void* delta_out, double* pk_out, double* kmean, int64_t* nmodes,
                           cudaStream_t s) {
  prof_mark(3, s);
  pk_status st = exec_plan(g.plan, g.kind, g.grids, g.fft_work, s);
  if (st != PK_OK) return st;
  prof_mark(4, s);
  const bool dbl = c->prec != PK_FP32;
  EstimateArgs a;
  a.ng = c->ng;
  a.order = c->order;
  a.interlace = c->interlace;
  a.nbins = pk_out ? c->nbins : 0;
  a.bin_lo2 = c->bin_lo2;
  a.bin_w2 = c->bin_w2;
  a.box = c->box;
  a.wsums = g.wsums;
  a.bin_sum = g.bin_sum;
  a.bin_k = g.bin_k;
  a.bin_cnt = g.bin_cnt;
  a.delta_out = delta_out;
  a.det_pass = c->prec == PK_FIXED64 ? 1 : 0;
  a.det_scale = g.bin_aux;
  cudaError_t e;
  if (pk_out) {
    if ((e = cudaMemsetAsync(g.bin_sum, 0, sizeof(double) * c->nbins, s)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(g.bin_k, 0, sizeof(double) * c->nbins, s)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(g.bin_cnt, 0, sizeof(unsigned long long) * c->nbins, s)) != cudaSuccess) return cuda_fail(e, "memset");
  }
  const size_t gbytes = size_t(padded_count(c->ng)) * (dbl ? 8 : 4);
  const void* G1 = g.grids;
  const void* G2 = c->interlace ? static_cast<const char*>(g.grids) + gbytes : nullptr;
  e = dbl ? launch_estimate<double>(G1, G2, g.tables, a, s) : launch_estimate<float>(G1, G2, g.tables, a, s);
  if (e != cudaSuccess) return cuda_fail(e, "estimate");
  if (pk_out) {
    if ((e = launch_finalize(a, c->subtract_shot, pk_out, kmean, nmodes, s)) != cudaSuccess) return cuda_fail(e, "finalize");
  }
  prof_mark(5, s);
  return PK_OK;
}


void carve_bin_stage(const pk_config* c, int64_t n, bool need_cells, Carver& cv, BinStage* b) {
  const int nt = tiles_per_axis(c->ng);
  const int64_t ntiles = int64_t(nt) * nt * nt;
  b->cells = need_cells ? cv.take<pk_cellpos>(size_t(std::max<int64_t>(n, 1))) : nullptr;
  const int64_t nkeys = ntiles * kSlabs;
  b->counts = cv.take<unsigned long long>(size_t(nkeys));
  b->sub = cv.take<int64_t>(size_t(nkeys + 1));
  b->scan = cv.take<long long>(scan_scratch_bytes(nkeys) / sizeof(long long) + 1);
}

// Positions in either format -> binned layout (sorted, wsorted, offsets). FP64 positions are prepared
// and counted in one sweep; `pos` is device-accessible (device memory or mapped pinned host memory),
// or, with `stage`, pageable host memory copied through stage->buf in pieces of stage->cap particles.
pk_status run_bin(const pk_config* c, const void* pos, int fmt, const float* w, int64_t n, BinStage& b, pk_cellpos* sorted,
                  float* wsorted, int64_t* offsets, cudaStream_t s, const HostStage* stage) {
  const int nt = tiles_per_axis(c->ng);
  cudaError_t e;
  if (fmt != PK_POS_F64_XYZ) {
    if ((e = launch_bin(static_cast<const pk_cellpos*>(pos), w, n, c->ng, nt, sorted, wsorted, offsets, b.counts, b.sub,
                        b.scan, s)) != cudaSuccess)
      return cuda_fail(e, "bin");
    return PK_OK;
  }
  const size_t nkeys = size_t(nt) * nt * nt * kSlabs;
  if ((e = cudaMemsetAsync(b.counts, 0, nkeys * sizeof(unsigned long long), s)) != cudaSuccess) return cuda_fail(e, "memset");
  const double* p = static_cast<const double*>(pos);
  if (!stage) {
    if ((e = launch_prepare_hist(p, 0, n, c->ng, c->box, nt, b.cells, b.counts, s)) != cudaSuccess)
      return cuda_fail(e, "prepare");
  } else {
    for (int64_t i0 = 0; i0 < n; i0 += stage->cap) {
      const int64_t cnt = std::min<int64_t>(stage->cap, n - i0);
      if ((e = cudaMemcpyAsync(stage->buf, p + 3 * i0, size_t(cnt) * 3 * sizeof(double), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
        return cuda_fail(e, "copy positions");
      if ((e = launch_prepare_hist(stage->buf, i0, cnt, c->ng, c->box, nt, b.cells, b.counts, s)) != cudaSuccess)
        return cuda_fail(e, "prepare");
    }
  }
  if ((e = launch_bin_finish(b.cells, w, n, c->ng, nt, sorted, wsorted, offsets, b.counts, b.sub, b.scan, s)) != cudaSuccess)
    return cuda_fail(e, "bin");
  return PK_OK;
}

pk_status run_weight_sums(const float* w, int64_t n, double* sums, cudaStream_t s) {
  cudaError_t e = w ? launch_weight_sums(w, n, sums, s) : launch_set_sums(sums, double(n), double(n), s);
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "weight sums");
}

// Mass assignment into `grids` (two consecutive grids of ng*ng*ldz elements when interlaced):
// PK_FP64 from positions in any order (direct FP64 atomics); PK_FP32 / PK_FIXED64 from the binned
// layout (sorted, offsets). wsums (device) holds the weight sums (fixed-point scale).
pk_status run_assign_into(const pk_config* c, const void* pos, int fmt, const pk_cellpos* sorted, const float* w,
                          const int64_t* offsets, int64_t n, const double* wsums, void* grids, int ldz, cudaStream_t s,
                          bool clear) {
  const bool two = c->interlace != 0;
  const int64_t per = int64_t(c->ng) * c->ng * ldz;
  const size_t all = size_t(per) * (two ? 2 : 1);
  cudaError_t e;
  if (c->prec == PK_FP64) {
    double* g1 = static_cast<double*>(grids);
    if (clear && (e = cudaMemsetAsync(g1, 0, all * 8, s)) != cudaSuccess) return cuda_fail(e, "memset");
    prof_mark(2, s);
    e = launch_assign_direct_f64(c->order, pos, fmt, w, n, c->ng, c->box, two, g1, two ? g1 + per : nullptr, ldz, s);
    if (e != cudaSuccess) return cuda_fail(e, "assign (fp64)");
  } else if (c->prec == PK_FP32) {
    float* g1 = static_cast<float*>(grids);
    if (clear && (e = cudaMemsetAsync(g1, 0, all * 4, s)) != cudaSuccess) return cuda_fail(e, "memset");
    prof_mark(2, s);
    e = launch_assign_tiles_f32(c->order, sorted, w, offsets, n, c->ng, two, g1, two ? g1 + per : nullptr, ldz, s, 1, 0,
                                scatter_run(c, n, 1));
    if (e != cudaSuccess) return cuda_fail(e, "assign (fp32)");
  } else {
    unsigned long long* g1 = static_cast<unsigned long long*>(grids);
    if ((e = cudaMemsetAsync(g1, 0, all * 8, s)) != cudaSuccess) return cuda_fail(e, "memset");
    prof_mark(2, s);
    e = launch_assign_tiles_fixed(c->order, sorted, w, offsets, n, c->ng, two, wsums, g1, two ? g1 + per : nullptr, ldz, s);
    if (e != cudaSuccess) return cuda_fail(e, "assign (fixed)");
    if ((e = launch_fixed_to_double(g1, int64_t(all), wsums, s)) != cudaSuccess) return cuda_fail(e, "fixed->double");
  }
  return PK_OK;
}

pk_status carve_forward(const pk_config* c, int64_t n, Carver& cv, ForwardStage* f) {
  pk_status st = carve_grid_stage(c, cv, &f->g);
  if (st != PK_OK) return st;
  if (c->prec != PK_FP64) {
    carve_bin_stage(c, n, true, cv, &f->b);
    f->sorted = cv.take<pk_cellpos>(size_t(std::max<int64_t>(n, 1)));
    f->wsorted = cv.take<float>(size_t(std::max<int64_t>(n, 1)));
    const int nt = tiles_per_axis(c->ng);
    f->offsets = cv.take<int64_t>(size_t(int64_t(nt) * nt * nt + 1));
  }
  return PK_OK;
}

// Workspace of pk_power_host: the forward stage, device copies of the weights (and, in FP64 mode, of
// the positions), the staging buffer for pageable positions and the device outputs.
constexpr int64_t kHostStageParticles = int64_t(1) << 22;
// FP32 from FP64 host positions: the catalogue crosses the CPU-GPU link in about sixteen pieces of
// 2^20 .. 2^26 particles (up to 1.6 GB), each prepared, binned and assigned while the next one is
// being copied; only the last piece's processing is not hidden behind the link.
constexpr int64_t kHostPieceMin = int64_t(1) << 20, kHostPieceMax = int64_t(1) << 26;
pk_status carve_host(const pk_config* c, int64_t n, Carver& cv, HostLayout* h) {
  pk_status st = carve_forward(c, n, cv, &h->f);
  if (st != PK_OK) return st;
  h->w = cv.take<float>(size_t(std::max<int64_t>(n, 1)));
  h->stage_cap = std::max<int64_t>(1, std::min<int64_t>(n, kHostStageParticles));
  h->stage = cv.take<double>(size_t(3 * h->stage_cap));
  if (c->prec == PK_FP32) {
    h->piece_cap = std::min<int64_t>(std::max<int64_t>(n, 1),
                                     std::min(kHostPieceMax, std::max(kHostPieceMin, (n + 15) / 16)));
    h->piece[0] = cv.take<double>(size_t(3 * h->piece_cap));
    h->piece[1] = cv.take<double>(size_t(3 * h->piece_cap));
  }
  h->pos = c->prec == PK_FP64 ? cv.take<double>(size_t(3 * std::max<int64_t>(n, 1))) : nullptr;
  h->pk = cv.take<double>(size_t(c->nbins));
  h->kmean = cv.take<double>(size_t(c->nbins));
  h->nmodes = cv.take<int64_t>(size_t(c->nbins));
  return PK_OK;
}

// Weight sums, binning (FP32/FIXED64) and assignment into the padded grids of f.g (not transformed).
pk_status run_forward_grids(const pk_config* c, const void* pos, int fmt, const float* w, int64_t n, ForwardStage& f,
                            cudaStream_t s, const HostStage* stage) {
  prof_mark(0, s);
  pk_status st = run_weight_sums(w, n, f.g.wsums, s);
  if (st != PK_OK) return st;
  if (c->prec == PK_FP64) {
    prof_mark(1, s);
    return run_assign_into(c, pos, fmt, nullptr, w, nullptr, n, f.g.wsums, f.g.grids, c->ng + 2, s);
  }
  if ((st = run_bin(c, pos, fmt, w, n, f.b, f.sorted, w ? f.wsorted : nullptr, f.offsets, s, stage)) != PK_OK) return st;
  prof_mark(1, s);
  return run_assign_into(c, nullptr, PK_POS_CELL_F32OFF, f.sorted, w ? f.wsorted : nullptr, f.offsets, n, f.g.wsums,
                         f.g.grids, c->ng + 2, s);
}

}  // namespace pk

using namespace pk;

// ---- entry points -----------------------------------------------------------------------------------------

extern "C" {

void pk_default_config(pk_config* cfg, int32_t ng, double box) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->ng = ng;
  cfg->order = 4;
  cfg->interlace = 1;
  cfg->prec = PK_FP32;
  cfg->box = box;
  cfg->bin_lo2 = 1;
  cfg->bin_w2 = 2;
  cfg->nbins = ng / 2;
  cfg->subtract_shot = 0;
  cfg->tile_run = 0;
}

int32_t pk_tiles_per_axis(const pk_config* cfg, int32_t* tile_cells) {
  if (tile_cells) *tile_cells = kTileCells;
  if (!cfg || cfg->ng < 1) return 0;
  return tiles_per_axis(cfg->ng);
}

const char* pk_last_error(void) { return t_err.c_str(); }

int32_t pk_profile_enable(int32_t on) {
  const bool was = t_prof;
  t_prof = on != 0;
  for (int k = 0; k < kProfMarks; ++k) t_ev_rec[k] = false;
  return was ? 1 : 0;
}

int32_t pk_profile_read(double* ms, int32_t max_stages) {
  int got = 0;
  for (int k = 0; k + 1 < kProfMarks && got < max_stages; ++k) {
    float v = 0.0f;
    if (t_ev_rec[k] && t_ev_rec[k + 1] && cudaEventSynchronize(t_ev[k + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&v, t_ev[k], t_ev[k + 1]) == cudaSuccess)
      ms[got] = double(v);
    else
      ms[got] = -1.0;
    ++got;
  }
  for (int k = 0; k < kProfMarks; ++k) t_ev_rec[k] = false;
  return got;
}

int64_t pk_profile_launches(void) { return int64_t(g_launches.load()); }

int32_t pk_device_error(void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned v = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  if (take_err_prepare(&v) != 0 || take_err_assign(&v) != 0 || take_err_tiles(&v) != 0 || take_err_direct(&v) != 0)
    return -1;
  return int32_t(v);
}

static size_t assign_ws(const pk_config* c, int64_t n) {
  Carver cv(nullptr);
  cv.take<double>(3);
  if (c->prec != PK_FP64) {
    BinStage b;
    carve_bin_stage(c, n, true, cv, &b);
    cv.take<pk_cellpos>(size_t(std::max<int64_t>(n, 1)));
    cv.take<float>(size_t(std::max<int64_t>(n, 1)));
    const int nt = tiles_per_axis(c->ng);
    cv.take<int64_t>(size_t(int64_t(nt) * nt * nt + 1));
  }
  return cv.size();
}

size_t pk_workspace_size(const pk_config* cfg, int64_t n, int32_t kind) {
  clear_err();
  if (validate(cfg) != PK_OK) return 0;
  if (n < 0) {
    fail(PK_EINVAL, "n < 0");
    return 0;
  }
  Carver cv(nullptr);
  size_t out = 0;
  switch (kind) {
    case PK_WS_ASSIGN:
      return assign_ws(cfg, n);
    case PK_WS_FFT_ESTIMATE:
    case PK_WS_POWER_BINNED: {
      GridStage g;
      if (carve_grid_stage(cfg, cv, &g) != PK_OK) return 0;
      return cv.size();
    }
    case PK_WS_POWER: {
      ForwardStage f;
      if (carve_forward(cfg, n, cv, &f) != PK_OK) return 0;
      return cv.size();
    }
    case PK_WS_BIN: {
      BinStage b;
      carve_bin_stage(cfg, n, true, cv, &b);
      return cv.size();
    }
    case PK_WS_POWER_HOST: {
      HostLayout h;
      if (carve_host(cfg, n, cv, &h) != PK_OK) return 0;
      return cv.size();
    }
    case PK_WS_BACKWARD:
      return backward_ws(cfg, n, &out) == PK_OK ? out : 0;
    case PK_WS_DIRECT:
    case PK_WS_CROSS:
      return direct_ws(cfg, n, kind == PK_WS_CROSS, &out) == PK_OK ? out : 0;
    case PK_WS_ALIASING:
      return aliasing_ws(cfg, &out) == PK_OK ? out : 0;
    case PK_WS_BISPECTRUM:
    case PK_WS_BISPECTRUM_COUNTS:
      if (n < 1 || n > 64) {
        fail(PK_EINVAL, "nshells must be 1..64");
        return 0;
      }
      return bispectrum_ws(cfg, int(n), kind == PK_WS_BISPECTRUM_COUNTS, &out) == PK_OK ? out : 0;
    default:
      fail(PK_EINVAL, "unknown workspace kind %d", kind);
      return 0;
  }
}

pk_status pk_prepare(const pk_config* cfg, const double* pos_dev, int64_t n, pk_cellpos* out_dev, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (n < 0 || (n > 0 && (!pos_dev || !out_dev))) return fail(PK_EINVAL, "bad positions/output");
  cudaError_t e = launch_prepare(pos_dev, n, cfg->ng, cfg->box, out_dev, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "prepare");
}

pk_status pk_bin(const pk_config* cfg, const void* pos_dev, int32_t pos_format, const float* w_dev, int64_t n,
                 pk_cellpos* sorted_dev, float* w_sorted_dev, int64_t* tile_offsets_dev, void* ws, size_t ws_bytes,
                 void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (pos_format != PK_POS_F64_XYZ && pos_format != PK_POS_CELL_F32OFF) return fail(PK_EINVAL, "bad pos_format");
  if (n < 0 || (n > 0 && (!pos_dev || !sorted_dev)) || !tile_offsets_dev) return fail(PK_EINVAL, "bad pointers");
  if (w_dev && !w_sorted_dev) return fail(PK_EINVAL, "w_sorted_dev required when w_dev is given");
  const size_t need = pk_workspace_size(cfg, n, PK_WS_BIN);
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  Carver cv(ws);
  BinStage b;
  carve_bin_stage(cfg, n, true, cv, &b);
  return run_bin(cfg, pos_dev, pos_format, w_dev, n, b, sorted_dev, w_dev ? w_sorted_dev : nullptr, tile_offsets_dev,
                 static_cast<cudaStream_t>(stream));
}

pk_status pk_assign(const pk_config* cfg, const void* pos_dev, int32_t pos_format, const float* w_dev, int64_t n,
                    void* grid1_dev, void* grid2_dev, void* ws, size_t ws_bytes, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (pos_format != PK_POS_F64_XYZ && pos_format != PK_POS_CELL_F32OFF) return fail(PK_EINVAL, "bad pos_format");
  if (n < 0 || (n > 0 && !pos_dev) || !grid1_dev) return fail(PK_EINVAL, "bad pointers");
  const size_t need = pk_workspace_size(cfg, n, PK_WS_ASSIGN);
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  pk_config c = *cfg;
  if (!grid2_dev) c.interlace = 0;
  const int64_t per = int64_t(c.ng) * c.ng * c.ng;
  const size_t esz = c.prec == PK_FP32 ? 4 : 8;
  Carver cv(ws);
  double* sums = cv.take<double>(3);
  if ((st = run_weight_sums(w_dev, n, sums, s)) != PK_OK) return st;
  cudaError_t e = cudaMemsetAsync(grid1_dev, 0, size_t(per) * esz, s);
  if (e == cudaSuccess && c.interlace) e = cudaMemsetAsync(grid2_dev, 0, size_t(per) * esz, s);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  if (c.prec == PK_FP64) {
    e = launch_assign_direct_f64(c.order, pos_dev, pos_format, w_dev, n, c.ng, c.box, c.interlace != 0,
                                 static_cast<double*>(grid1_dev), static_cast<double*>(c.interlace ? grid2_dev : nullptr),
                                 c.ng, s);
    return e == cudaSuccess ? PK_OK : cuda_fail(e, "assign (fp64)");
  }
  BinStage b;
  carve_bin_stage(&c, n, true, cv, &b);
  pk_cellpos* sorted = cv.take<pk_cellpos>(size_t(std::max<int64_t>(n, 1)));
  float* wsorted = cv.take<float>(size_t(std::max<int64_t>(n, 1)));
  const int nt = tiles_per_axis(c.ng);
  int64_t* offsets = cv.take<int64_t>(size_t(int64_t(nt) * nt * nt + 1));
  if ((st = run_bin(&c, pos_dev, pos_format, w_dev, n, b, sorted, w_dev ? wsorted : nullptr, offsets, s)) != PK_OK) return st;
  const float* ws_w = w_dev ? wsorted : nullptr;
  if (c.prec == PK_FP32) {
    e = launch_assign_tiles_f32(c.order, sorted, ws_w, offsets, n, c.ng, c.interlace != 0, static_cast<float*>(grid1_dev),
                               static_cast<float*>(c.interlace ? grid2_dev : nullptr), c.ng, s, 1, 0, scatter_run(&c, n, 1));
    return e == cudaSuccess ? PK_OK : cuda_fail(e, "assign (fp32)");
  }
  // PK_FIXED64: integer sums in the 8-byte output arrays, converted to double in place.
  unsigned long long* g1 = static_cast<unsigned long long*>(grid1_dev);
  unsigned long long* g2 = static_cast<unsigned long long*>(c.interlace ? grid2_dev : nullptr);
  e = launch_assign_tiles_fixed(c.order, sorted, ws_w, offsets, n, c.ng, c.interlace != 0, sums, g1, g2, c.ng, s);
  if (e != cudaSuccess) return cuda_fail(e, "assign (fixed)");
  if ((e = launch_fixed_to_double(g1, per, sums, s)) != cudaSuccess) return cuda_fail(e, "fixed->double");
  if (g2 && (e = launch_fixed_to_double(g2, per, sums, s)) != cudaSuccess) return cuda_fail(e, "fixed->double");
  return PK_OK;
}

pk_status pk_fft_estimate(const pk_config* cfg, const void* grid1_dev, const void* grid2_dev, double wsum, void* delta_k_dev,
                          void* ws, size_t ws_bytes, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (!grid1_dev || !delta_k_dev || (cfg->interlace && !grid2_dev)) return fail(PK_EINVAL, "bad pointers");
  if (!(wsum > 0.0) || !std::isfinite(wsum)) return fail(PK_EINVAL, "wsum must be finite and > 0");
  const size_t need = pk_workspace_size(cfg, 0, PK_WS_FFT_ESTIMATE);
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  GridStage g;
  if ((st = carve_grid_stage(cfg, cv, &g)) != PK_OK) return st;
  const bool dbl = cfg->prec != PK_FP32;
  const int64_t rows = int64_t(cfg->ng) * cfg->ng;
  const int64_t per = padded_count(cfg->ng);
  cudaError_t e;
  if (dbl) {
    double* d = static_cast<double*>(g.grids);
    e = launch_copy_rows<double>(static_cast<const double*>(grid1_dev), cfg->ng, d, cfg->ng + 2, cfg->ng, rows, s);
    if (e == cudaSuccess && cfg->interlace)
      e = launch_copy_rows<double>(static_cast<const double*>(grid2_dev), cfg->ng, d + per, cfg->ng + 2, cfg->ng, rows, s);
  } else {
    float* d = static_cast<float*>(g.grids);
    e = launch_copy_rows<float>(static_cast<const float*>(grid1_dev), cfg->ng, d, cfg->ng + 2, cfg->ng, rows, s);
    if (e == cudaSuccess && cfg->interlace)
      e = launch_copy_rows<float>(static_cast<const float*>(grid2_dev), cfg->ng, d + per, cfg->ng + 2, cfg->ng, rows, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "copy grids");
  if ((e = launch_set_sums(g.wsums, wsum, wsum, s)) != cudaSuccess) return cuda_fail(e, "set sums");
  return run_fft_estimate(cfg, g, delta_k_dev, nullptr, nullptr, nullptr, s);
}

pk_status pk_power(const pk_config* cfg, const void* pos_dev, int32_t pos_format, const float* w_dev, int64_t n,
                   double* pk_dev, double* kmean_dev, int64_t* nmodes_dev, void* delta_k_dev, void* ws, size_t ws_bytes,
                   void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (pos_format != PK_POS_F64_XYZ && pos_format != PK_POS_CELL_F32OFF) return fail(PK_EINVAL, "bad pos_format");
  if (n < 1 || !pos_dev) return fail(PK_EINVAL, "need at least one particle");
  if (!pk_dev || !kmean_dev || !nmodes_dev) return fail(PK_EINVAL, "pk, kmean and nmodes outputs are required");
  const size_t need = pk_workspace_size(cfg, n, PK_WS_POWER);
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  ForwardStage f;
  if ((st = carve_forward(cfg, n, cv, &f)) != PK_OK) return st;
  if ((st = run_forward_grids(cfg, pos_dev, pos_format, w_dev, n, f, s)) != PK_OK) return st;
  return run_fft_estimate(cfg, f.g, delta_k_dev, pk_dev, kmean_dev, nmodes_dev, s);
}

// FP32 grids from FP64 host positions, piece by piece: on a copy stream of its own the copy engine
// moves piece j into device buffer j % 2 (after the processing of piece j - 2 has read it); the caller's
// stream prepares and counts it, bins it and adds its assignment to the grids, so the transfer of
// piece j + 1 overlaps the processing of piece j. The grids are cleared once.
static pk_status run_host_pieces(const pk_config* c, const double* pos_host, const float* w, int64_t n, HostLayout& h,
                                 cudaStream_t s) {
  cudaError_t e;
  pk_status st = run_weight_sums(w, n, h.f.g.wsums, s);
  if (st != PK_OK) return st;
  const int nt = tiles_per_axis(c->ng);
  const size_t nkeys = size_t(nt) * nt * nt * kSlabs;
  const size_t gbytes = size_t(c->interlace ? 2 : 1) * size_t(padded_count(c->ng)) * sizeof(float);
  if ((e = cudaMemsetAsync(h.f.g.grids, 0, gbytes, s)) != cudaSuccess) return cuda_fail(e, "memset");
  cudaStream_t cs = nullptr;
  cudaEvent_t ev[5] = {};  // start, ready[2], free[2]
  auto release = [&]() {
    for (cudaEvent_t& x : ev)
      if (x) cudaEventDestroy(x);
    if (cs) cudaStreamDestroy(cs);
  };
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "copy stream");
  for (cudaEvent_t& x : ev)
    if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess) {
      release();
      return cuda_fail(e, "events");
    }
  cudaEvent_t ev_start = ev[0], *ev_ready = ev + 1, *ev_free = ev + 3;
  st = PK_OK;
  if ((e = cudaEventRecord(ev_start, s)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, ev_start, 0)) != cudaSuccess)
    st = cuda_fail(e, "order copy stream");
  for (int64_t i0 = 0, j = 0; st == PK_OK && i0 < n; i0 += h.piece_cap, ++j) {
    const int b = int(j & 1);
    const int64_t cnt = std::min<int64_t>(h.piece_cap, n - i0);
    if (j >= 2 && (e = cudaStreamWaitEvent(cs, ev_free[b], 0)) != cudaSuccess) { st = cuda_fail(e, "wait"); break; }
    if ((e = cudaMemcpyAsync(h.piece[b], pos_host + 3 * i0, size_t(cnt) * 3 * sizeof(double), cudaMemcpyHostToDevice, cs)) !=
            cudaSuccess ||
        (e = cudaEventRecord(ev_ready[b], cs)) != cudaSuccess || (e = cudaStreamWaitEvent(s, ev_ready[b], 0)) != cudaSuccess) {
      st = cuda_fail(e, "copy positions");
      break;
    }
    if ((e = cudaMemsetAsync(h.f.b.counts, 0, nkeys * sizeof(unsigned long long), s)) != cudaSuccess ||
        (e = launch_prepare_hist(h.piece[b], 0, cnt, c->ng, c->box, nt, h.f.b.cells, h.f.b.counts, s)) != cudaSuccess ||
        (e = cudaEventRecord(ev_free[b], s)) != cudaSuccess) {
      st = cuda_fail(e, "prepare");
      break;
    }
    const float* wp = w ? w + i0 : nullptr;
    if ((e = launch_bin_finish(h.f.b.cells, wp, cnt, c->ng, nt, h.f.sorted, w ? h.f.wsorted : nullptr, h.f.offsets,
                               h.f.b.counts, h.f.b.sub, h.f.b.scan, s)) != cudaSuccess) {
      st = cuda_fail(e, "bin");
      break;
    }
    st = run_assign_into(c, nullptr, PK_POS_CELL_F32OFF, h.f.sorted, w ? h.f.wsorted : nullptr, h.f.offsets, cnt, h.f.g.wsums,
                         h.f.g.grids, c->ng + 2, s, false);
  }
  release();  // destruction is deferred by the runtime until the queued work is done
  return st;
}

pk_status pk_power_host(const pk_config* cfg, const void* pos_host, int32_t pos_format, const float* w_host, int64_t n,
                        double* pk_host, double* kmean_host, int64_t* nmodes_host, void* ws, size_t ws_bytes, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (pos_format != PK_POS_F64_XYZ && pos_format != PK_POS_CELL_F32OFF) return fail(PK_EINVAL, "bad pos_format");
  if (n < 1 || !pos_host) return fail(PK_EINVAL, "need at least one particle");
  if (!pk_host || !kmean_host || !nmodes_host) return fail(PK_EINVAL, "pk, kmean and nmodes outputs are required");
  const size_t need = pk_workspace_size(cfg, n, PK_WS_POWER_HOST);
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  // where the positions live: pinned host memory is read through its device mapping; device or
  // managed memory belongs to pk_power
  cudaPointerAttributes attr;
  const void* mapped = nullptr;
  if (cudaPointerGetAttributes(&attr, pos_host) == cudaSuccess) {
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged)
      return fail(PK_EINVAL, "pos_host is device memory: use pk_power");
    if (attr.type == cudaMemoryTypeHost) mapped = attr.devicePointer;
  } else {
    (void)cudaGetLastError();  // not known to CUDA: pageable host memory
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  HostLayout h;
  if ((st = carve_host(cfg, n, cv, &h)) != PK_OK) return st;
  cudaError_t e;
  const float* w = nullptr;
  if (w_host) {
    if ((e = cudaMemcpyAsync(h.w, w_host, size_t(n) * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "copy weights");
    w = h.w;
  }
  const size_t rec = pos_format == PK_POS_F64_XYZ ? 3 * sizeof(double) : sizeof(pk_cellpos);
  if (cfg->prec == PK_FP64 || pos_format != PK_POS_F64_XYZ) {  // copy the positions to the device first
    void* dst = cfg->prec == PK_FP64 ? static_cast<void*>(h.pos) : static_cast<void*>(h.f.b.cells);
    if ((e = cudaMemcpyAsync(dst, pos_host, size_t(n) * rec, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "copy positions");
    st = run_forward_grids(cfg, dst, pos_format, w, n, h.f, s);
  } else if (cfg->prec == PK_FP32) {  // pieces copied by the copy engine while the previous one is processed
    (void)mapped;
    st = run_host_pieces(cfg, static_cast<const double*>(pos_host), w, n, h, s);
  } else if (mapped) {  // read over the CPU-GPU link while being prepared and counted
    st = run_forward_grids(cfg, mapped, pos_format, w, n, h.f, s);
  } else {
    HostStage stage;
    stage.buf = h.stage;
    stage.cap = h.stage_cap;
    st = run_forward_grids(cfg, pos_host, pos_format, w, n, h.f, s, &stage);
  }
  if (st != PK_OK) return st;
  if ((st = run_fft_estimate(cfg, h.f.g, nullptr, h.pk, h.kmean, h.nmodes, s)) != PK_OK) return st;
  const size_t nb = size_t(cfg->nbins);
  if ((e = cudaMemcpyAsync(pk_host, h.pk, nb * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(kmean_host, h.kmean, nb * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(nmodes_host, h.nmodes, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "copy results");
  return PK_OK;
}

pk_status pk_power_binned(const pk_config* cfg, const pk_cellpos* sorted_dev, const float* w_sorted_dev,
                          const int64_t* tile_offsets_dev, int64_t n, double* pk_dev, double* kmean_dev, int64_t* nmodes_dev,
                          void* delta_k_dev, void* ws, size_t ws_bytes, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (n < 1 || !sorted_dev || !tile_offsets_dev) return fail(PK_EINVAL, "need at least one particle and tile offsets");
  if (!pk_dev || !kmean_dev || !nmodes_dev) return fail(PK_EINVAL, "pk, kmean and nmodes outputs are required");
  const size_t need = pk_workspace_size(cfg, n, PK_WS_POWER_BINNED);
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  GridStage g;
  if ((st = carve_grid_stage(cfg, cv, &g)) != PK_OK) return st;
  prof_mark(0, s);
  if ((st = run_weight_sums(w_sorted_dev, n, g.wsums, s)) != PK_OK) return st;
  prof_mark(1, s);
  if (cfg->prec == PK_FP64)
    st = run_assign_into(cfg, sorted_dev, PK_POS_CELL_F32OFF, nullptr, w_sorted_dev, nullptr, n, g.wsums, g.grids, cfg->ng + 2, s);
  else
    st = run_assign_into(cfg, nullptr, PK_POS_CELL_F32OFF, sorted_dev, w_sorted_dev, tile_offsets_dev, n, g.wsums, g.grids,
                         cfg->ng + 2, s);
  if (st != PK_OK) return st;
  return run_fft_estimate(cfg, g, delta_k_dev, pk_dev, kmean_dev, nmodes_dev, s);
}

}  // extern "C"
