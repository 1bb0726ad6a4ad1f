// Host-side declarations shared by the translation units of libpk.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"

namespace pk {

int num_sms();  // SM count of the current device (cached per device)
void count_launch(int k = 1);  // number of kernels this library launched (pk_profile_launches)

// Per-translation-unit device error words (see PK_ERR_ACCESSOR): OR into *acc and clear.
int take_err_prepare(unsigned* acc);
int take_err_assign(unsigned* acc);
int take_err_tiles(unsigned* acc);
int take_err_direct(unsigned* acc);
// Raises a kernel's dynamic shared-memory limit to at least smem bytes, once per (kernel, device) and
// size: calls captured in a CUDA graph after the first eager call then issue launches only.
cudaError_t ensure_dynamic_smem(const void* kernel, size_t smem);

// Tile edge (cells) of the binned layout for a grid of side ng, and tiles per axis.
constexpr int kTileCells = 8;
inline int tiles_per_axis(int ng) { return (ng + kTileCells - 1) / kTileCells; }
// Inside a tile the binned particles are ordered by half-cell slab along x, 2 (c_x mod T) + [f_x >= 1/2]:
// the sort key of a particle is tile * kSlabs + slab.
constexpr int kSlabs = 2 * kTileCells;

// prepare.cu
cudaError_t launch_prepare(const double* pos, int64_t n, int ng, double box, pk_cellpos* out, cudaStream_t s);
size_t scan_scratch_bytes(int64_t n);
cudaError_t launch_exclusive_scan(const unsigned long long* in, int64_t n, int64_t* out, long long* scratch, cudaStream_t s);
// counts: ntiles * kSlabs entries; sub: ntiles * kSlabs + 1 (slab offsets); scan_scratch for ntiles * kSlabs.
cudaError_t launch_bin(const pk_cellpos* cells, const float* w, int64_t n, int ng, int ntile, pk_cellpos* sorted,
                       float* wsorted, int64_t* offsets, unsigned long long* counts, int64_t* sub, long long* scan_scratch,
                       cudaStream_t s);
// FP64 positions pos[0 .. cnt) -> cells[i0 .. i0 + cnt), keys counted into counts (cleared by the caller).
cudaError_t launch_prepare_hist(const double* pos, int64_t i0, int64_t cnt, int ng, double box, int ntile, pk_cellpos* cells,
                                unsigned long long* counts, cudaStream_t s);
// Scan of the counted keys, tile offsets and scatter of cells (and weights) into the binned layout.
cudaError_t launch_bin_finish(const pk_cellpos* cells, const float* w, int64_t n, int ng, int ntile, pk_cellpos* sorted,
                              float* wsorted, int64_t* offsets, unsigned long long* counts, int64_t* sub,
                              long long* scan_scratch, cudaStream_t s);

constexpr int kMaxBatch = 512;
struct CatRanges {  // particle ranges of the catalogues of one batch group (absolute indices)
  int64_t off[kMaxBatch + 1];
  int nb;
  int ng;
};
// Batched binning by tile only (no slab order inside a tile), counted and
// placed through per-block shared-memory histograms: one global atomic per (block, tile) instead of
// one per particle. Needs ntile^3 <= kSmemBinTiles; counts: nb ntile^3 entries.
constexpr int kSmemBinTiles = 8192;
cudaError_t launch_bin_batch_tiles(const pk_cellpos* p, const CatRanges& r, int ntile, pk_cellpos* sorted, int64_t* offsets,
                                   unsigned long long* counts, long long* scan_scratch, cudaStream_t s);
cudaError_t launch_bin_batch(const pk_cellpos* p, const CatRanges& r, int ng, int ntile, pk_cellpos* sorted, int64_t* offsets,
                             unsigned long long* counts, int64_t* sub, long long* scan_scratch, cudaStream_t s);

// assign.cu -- grid layout: node (x, y, z) at element (x * ng + y) * ldz + z of each grid.
cudaError_t launch_assign_direct_f64(int order, const void* pos, int fmt, const float* w, int64_t n, int ng, double box,
                                     bool interlace, double* g1, double* g2, int ldz, cudaStream_t s);
// FP32 tile assignment (assign_tiles.cu: the scatter on sparse tiles, the key-cell kernel on dense
// ones, chosen per tile), same grid layout, records binned by tile (any particle order inside a tile);
// ncat > 1: catalogue c's tiles have offsets toff + c * ntiles (one array of ncat * ntiles + 1
// offsets) and grids g + c * cat_stride; the kernels take the tiles of all catalogues as one sequence.
cudaError_t launch_assign_tiles_f32(int order, const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                    bool interlace, float* g1, float* g2, int ldz, cudaStream_t s, int ncat = 1,
                                    int64_t cat_stride = 0, int run = 1);
// Tiles per scatter run along z for a configuration (pk_config.tile_run, 0: chosen from the mean
// tile population n / (ncat N_t^3)).
int scatter_run(const pk_config* c, int64_t n, int ncat);
// PK_FIXED64: int64 grids at the scale 2^F derived on the device from wsums[2] = sum |w|, converted in
// place to FP64.
cudaError_t launch_fixed_to_double(unsigned long long* g, int64_t count, const double* wsums, cudaStream_t s);
// The deterministic path (orders 1..4): every tile a 32-bit region at a scale 2^e <= the global
// 2^F = fixed_scale(wsums[2]), added to the int64 grids shifted by F - e; sparse tiles on the
// bank-ordered scatter, dense ones on the key cells (products rounded one by one, summed exactly).
cudaError_t launch_assign_tiles_fixed(int order, const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                      bool interlace, const double* wsums, unsigned long long* g1, unsigned long long* g2,
                                      int ldz, cudaStream_t s);
// wsums (3 doubles): [sum w, sum w^2, sum |w|]
cudaError_t launch_weight_sums(const float* w, int64_t n, double* sums, cudaStream_t s);
cudaError_t launch_set_sums(double* sums, double s1, double s2, cudaStream_t s);
template <typename T>
cudaError_t launch_copy_rows(const T* src, int src_ld, T* dst, int dst_ld, int ng, int64_t rows, cudaStream_t s);

// estimate.cu
struct EstimateArgs {
  int ng, order, interlace, nbins, bin_lo2, bin_w2;
  double box;
  const double* wsums;  // device: [sum w, sum w^2, sum |w|]
  double* bin_sum;      // device accumulators (nbins each), zeroed by the caller
  double* bin_k;
  unsigned long long* bin_cnt;
  void* delta_out;      // optional half-complex delta(n)
  // batches (blockIdx.y = catalogue c): G1, G2 advance by c * cat_stride complex elements, wsums by 3c,
  // the bin accumulators and outputs by c * nbins
  int ncat = 1;
  int64_t cat_stride = 0;
  // deterministic mode (PK_FIXED64): 1 = the two-pass exact int64 bin sums are used; det_scale
  // (nbins doubles, device) holds the per-bin fixed-point scales between the passes
  int det_pass = 0;
  double* det_scale = nullptr;
  // set by the launcher: 1 = k_estimate_rows (private bins per row of a warp, no atomics), 0 = k_estimate
  // (32-slot items, shared atomics: the deterministic passes and bins beyond the private copies' room)
  int priv = 0;
  // set by the launcher for the row kernel: rows a warp takes at once (a private bin copy each)
  int rows_per_warp = 1;
};
size_t estimate_table_bytes(int ng, bool dbl);
template <typename R>
cudaError_t launch_estimate(const void* G1, const void* G2, void* tables, const EstimateArgs& a, cudaStream_t s);
cudaError_t launch_finalize(const EstimateArgs& a, int subtract_shot, double* pk, double* kmean, int64_t* nmodes,
                            cudaStream_t s);

}  // namespace pk
