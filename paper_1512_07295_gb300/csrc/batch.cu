// a9 batched power spectra of many independent catalogues (mock catalogues): per group of up to
// kMaxBatch catalogues, one batched counting sort (key = catalogue * ntiles + tile), one tiled
// assignment launch per kernel over all (catalogue, tile) pairs as one sequence (blocks take tiles of
// any catalogue, so catalogues of uneven sizes leave no tail), one batched cuFFT of all 2 x batch
// grids, one fused estimate launch and one finalisation launch. No host
// synchronisation and no allocation, so the sequence can be captured in a CUDA graph and replayed.
#include "host.cuh"

namespace pk {

struct BatchLayout {
  pk_cellpos* sorted = nullptr;
  unsigned long long* counts = nullptr;
  int64_t* sub = nullptr;
  int64_t* offsets = nullptr;
  long long* scan = nullptr;
  float* grids = nullptr;
  float* tables = nullptr;
  double* wsums = nullptr;
  double* bin_sum = nullptr;
  double* bin_k = nullptr;
  unsigned long long* bin_cnt = nullptr;
  void* work = nullptr;
  PlanEntry plan;
};

static pk_status carve_batch(const pk_config* c, int batch, int64_t maxp, Carver& cv, BatchLayout* L, bool plan) {
  const int nt = tiles_per_axis(c->ng);
  const int64_t ntiles = int64_t(nt) * nt * nt * batch;
  L->sorted = cv.take<pk_cellpos>(size_t(std::max<int64_t>(maxp, 1)));
  L->counts = cv.take<unsigned long long>(size_t(ntiles * kSlabs));
  L->sub = cv.take<int64_t>(size_t(ntiles * kSlabs + 1));
  L->offsets = cv.take<int64_t>(size_t(ntiles + 1));
  L->scan = cv.take<long long>(scan_scratch_bytes(ntiles * kSlabs) / sizeof(long long) + 1);
  L->grids = cv.take<float>(size_t(2) * batch * padded_count(c->ng));
  L->tables = cv.take<float>(estimate_table_bytes(c->ng, false) / sizeof(float));
  L->wsums = cv.take<double>(size_t(3) * batch);
  L->bin_sum = cv.take<double>(size_t(batch) * c->nbins);
  L->bin_k = cv.take<double>(size_t(batch) * c->nbins);
  L->bin_cnt = cv.take<unsigned long long>(size_t(batch) * c->nbins);
  size_t work = 0;
  for (int b = 1; b <= batch; ++b) {  // the last group of a call may be smaller: size for the largest plan work
    if (!plan && b != batch) continue;
    PlanEntry p;
    pk_status st = get_plan(c->ng, 0, 2 * b, &p);
    if (st != PK_OK) return st;
    work = std::max(work, p.work);
    if (b == batch) L->plan = p;
  }
  L->work = cv.take<char>(std::max<size_t>(work, 256));
  return PK_OK;
}

__global__ void k_batch_sums(double* wsums, CatRanges r) {
  const int c = threadIdx.x;
  if (c < r.nb) {
    const double n = double(r.off[c + 1] - r.off[c]);
    wsums[3 * c] = n > 0 ? n : 1.0;
    wsums[3 * c + 1] = n > 0 ? n : 1.0;
    wsums[3 * c + 2] = n > 0 ? n : 1.0;
  }
}

}  // namespace pk

using namespace pk;

extern "C" {

size_t pk_batch_workspace_size(const pk_config* cfg, int32_t batch, int64_t max_group_particles) {
  clear_err();
  if (validate(cfg) != PK_OK) return 0;
  if (batch < 1 || batch > kMaxBatch || max_group_particles < 0) {
    fail(PK_EINVAL, "batch must be 1..%d and max_group_particles >= 0", kMaxBatch);
    return 0;
  }
  Carver cv(nullptr);
  BatchLayout L;
  if (carve_batch(cfg, batch, max_group_particles, cv, &L, true) != PK_OK) return 0;
  return cv.size();
}

pk_status pk_batch_power(const pk_config* cfg, int32_t n_cat, const int64_t* offsets_host, const pk_cellpos* pos_dev,
                         double* pk_dev, int64_t* nmodes_dev, int32_t batch, void* ws, size_t ws_bytes, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (cfg->prec != PK_FP32 || !cfg->interlace) return fail(PK_EINVAL, "pk_batch_power supports PK_FP32 with interlacing");
  if (n_cat < 1 || !offsets_host || !pos_dev || !pk_dev || !nmodes_dev) return fail(PK_EINVAL, "bad arguments");
  if (batch < 1 || batch > kMaxBatch) return fail(PK_EINVAL, "batch must be 1..%d", kMaxBatch);
  int64_t maxp = 0;
  for (int g0 = 0; g0 < n_cat; g0 += batch) {
    const int nb = std::min<int>(batch, n_cat - g0);
    if (offsets_host[g0] < 0) return fail(PK_EINVAL, "negative offset");
    for (int c = 0; c < nb; ++c)
      if (offsets_host[g0 + c + 1] < offsets_host[g0 + c]) return fail(PK_EINVAL, "offsets must be non-decreasing");
    maxp = std::max<int64_t>(maxp, offsets_host[g0 + nb] - offsets_host[g0]);
  }
  const size_t need = pk_batch_workspace_size(cfg, batch, maxp);
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  BatchLayout L;
  if ((st = carve_batch(cfg, batch, maxp, cv, &L, false)) != PK_OK) return st;
  const int ng = cfg->ng;
  const int nt = tiles_per_axis(ng);
  const int64_t per = padded_count(ng);
  cudaError_t e;
  for (int g0 = 0; g0 < n_cat; g0 += batch) {
    const int nb = std::min<int>(batch, n_cat - g0);
    CatRanges r;
    r.nb = nb;
    r.ng = ng;
    for (int c = 0; c <= nb; ++c) r.off[c] = offsets_host[g0 + c];
    const pk_cellpos* base = pos_dev;
    // a2: batched counting sort (sorted indices relative to the group's first particle)
    CatRanges rel = r;
    for (int c = 0; c <= nb; ++c) rel.off[c] = r.off[c] - r.off[0];
    // the assignment needs no order inside a tile: tile-only binning through shared memory
    if (int64_t(nt) * nt * nt <= kSmemBinTiles)
      e = launch_bin_batch_tiles(base + r.off[0], rel, nt, L.sorted, L.offsets, L.counts, L.scan, s);
    else
      e = launch_bin_batch(base + r.off[0], rel, ng, nt, L.sorted, L.offsets, L.counts, L.sub, L.scan, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch bin");
    // a3: all catalogues' grid pairs
    if ((e = cudaMemsetAsync(L.grids, 0, size_t(2) * nb * per * sizeof(float), s)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = launch_assign_tiles_f32(cfg->order, L.sorted, nullptr, L.offsets, rel.off[nb], ng, true, L.grids, L.grids + per,
                                     ng + 2, s, nb, 2 * per, scatter_run(cfg, rel.off[nb], nb))) != cudaSuccess)
      return cuda_fail(e, "batch assign");
    k_batch_sums<<<1, kMaxBatch, 0, s>>>(L.wsums, rel); count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch sums");
    // a4: one batched transform of the 2 nb grids
    PlanEntry plan;
    if ((st = get_plan(ng, 0, 2 * nb, &plan)) != PK_OK) return st;
    if ((st = exec_plan(plan, 0, L.grids, L.work, s)) != PK_OK) return st;
    // a5, a6
    const size_t nbins_all = size_t(nb) * cfg->nbins;
    if ((e = cudaMemsetAsync(L.bin_sum, 0, nbins_all * sizeof(double), s)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(L.bin_k, 0, nbins_all * sizeof(double), s)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(L.bin_cnt, 0, nbins_all * sizeof(unsigned long long), s)) != cudaSuccess) return cuda_fail(e, "memset");
    EstimateArgs a;
    a.ng = ng;
    a.order = cfg->order;
    a.interlace = 1;
    a.nbins = cfg->nbins;
    a.bin_lo2 = cfg->bin_lo2;
    a.bin_w2 = cfg->bin_w2;
    a.box = cfg->box;
    a.wsums = L.wsums;
    a.bin_sum = L.bin_sum;
    a.bin_k = L.bin_k;
    a.bin_cnt = L.bin_cnt;
    a.delta_out = nullptr;
    a.ncat = nb;
    a.cat_stride = per;  // complex elements between catalogues (two padded real grids)
    if ((e = launch_estimate<float>(L.grids, L.grids + per, L.tables, a, s)) != cudaSuccess) return cuda_fail(e, "batch estimate");
    if ((e = launch_finalize(a, cfg->subtract_shot, pk_dev + size_t(g0) * cfg->nbins, nullptr,
                             nmodes_dev + size_t(g0) * cfg->nbins, s)) != cudaSuccess)
      return cuda_fail(e, "batch finalize");
  }
  return PK_OK;
}

}  // extern "C"
