// Host-side helpers shared by the entry-point translation units (api.cu, bispec.cu, adjoint.cu,
// batch.cu): error reporting, validation, workspace carving, the cuFFT plan cache and the common
// grid -> FFT -> estimate stage.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace pk {

pk_status fail(pk_status st, const char* fmt, ...);
pk_status cuda_fail(cudaError_t e, const char* where);
void clear_err();
pk_status validate(const pk_config* c);

// Carves 256-byte aligned regions from a workspace; with a NULL base it only counts bytes.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t size() const { return (off + 255) & ~size_t(255); }
};

// cuFFT plans over the padded in-place layout [ng][ng][ng+2] (reals) / [ng][ng][ng/2+1] (complex),
// `batch` grids spaced by the padded grid size. kind: 0 R2C, 1 D2Z, 2 C2R, 3 Z2D. A batch whose
// padded reals exceed 2^31 - 1 elements runs as several calls of `sub` grids each: on this GPU cuFFT
// takes a slower 64-bit-index path past that size (two 1024^3 grids: 18.7 ms in one call, 11.1 ms in
// two, and no 8 GB work area).
struct PlanEntry {
  int h = 0;
  size_t work = 0;
  int batch = 1, sub = 1;
  int64_t dist = 0;  // reals between consecutive grids
};
pk_status get_plan(int ng, int kind, int batch, PlanEntry* out);
pk_status exec_plan(const PlanEntry& p, int kind, void* data, void* work, cudaStream_t s);

inline int64_t padded_count(int ng) { return int64_t(ng) * ng * (ng + 2); }
inline int64_t half_count(int ng) { return int64_t(ng) * ng * (ng / 2 + 1); }

struct GridStage {
  void* grids = nullptr;  // [ngrid][ng][ng][ng+2] of float or double
  void* tables = nullptr;
  double* wsums = nullptr;  // [sum w, sum w^2, sum |w|]
  double* bin_sum = nullptr;
  double* bin_k = nullptr;
  unsigned long long* bin_cnt = nullptr;
  double* bin_aux = nullptr;  // per-bin fixed-point scales of the deterministic mode
  void* fft_work = nullptr;
  PlanEntry plan;
  int kind = 0;
};
pk_status carve_grid_stage(const pk_config* c, Carver& cv, GridStage* g);
pk_status run_fft_estimate(const pk_config* c, GridStage& g, void* delta_out, double* pk_out, double* kmean, int64_t* nmodes,
                           cudaStream_t s);

struct BinStage {
  pk_cellpos* cells = nullptr;
  unsigned long long* counts = nullptr;  // per (tile, slab) key
  int64_t* sub = nullptr;                // slab offsets
  long long* scan = nullptr;
};
void carve_bin_stage(const pk_config* c, int64_t n, bool need_cells, Carver& cv, BinStage* b);
// Pageable host FP64 positions are copied through buf (cap particles at a time).
struct HostStage {
  double* buf = nullptr;
  int64_t cap = 0;
};
pk_status run_bin(const pk_config* c, const void* pos, int fmt, const float* w, int64_t n, BinStage& b, pk_cellpos* sorted,
                  float* wsorted, int64_t* offsets, cudaStream_t s, const HostStage* stage = nullptr);
pk_status run_weight_sums(const float* w, int64_t n, double* sums, cudaStream_t s);
// clear = false adds to the grids instead of overwriting them (FP64 and FP32; the pieces of a catalogue).
pk_status run_assign_into(const pk_config* c, const void* pos, int fmt, const pk_cellpos* sorted, const float* w,
                          const int64_t* offsets, int64_t n, const double* wsums, void* grids, int ldz, cudaStream_t s,
                          bool clear = true);

// Workspace of the forward "positions -> padded transformed grids" stage (used by pk_power and
// recomputed by pk_power_backward).
struct ForwardStage {
  GridStage g;
  BinStage b;
  pk_cellpos* sorted = nullptr;
  float* wsorted = nullptr;
  int64_t* offsets = nullptr;
};
pk_status carve_forward(const pk_config* c, int64_t n, Carver& cv, ForwardStage* f);
pk_status run_forward_grids(const pk_config* c, const void* pos, int fmt, const float* w, int64_t n, ForwardStage& f,
                            cudaStream_t s, const HostStage* stage = nullptr);

struct HostLayout {
  ForwardStage f;
  float* w = nullptr;
  double* stage = nullptr;
  int64_t stage_cap = 0;
  double* piece[2] = {nullptr, nullptr};  // FP32 from FP64 positions: device copies of two pieces
  int64_t piece_cap = 0;
  double* pos = nullptr;
  double* pk = nullptr;
  double* kmean = nullptr;
  int64_t* nmodes = nullptr;
};
pk_status carve_host(const pk_config* c, int64_t n, Carver& cv, HostLayout* h);

// Optional stage timing (pk_profile_enable / pk_profile_read): prof_mark(k, s) records event k on s
// when profiling is on. Marks: 0 start, 1 before the grid clear, 2 before the assignment kernel,
// 3 before the FFT, 4 after the FFT, 5 end.
void prof_mark(int k, cudaStream_t s);

// Entry points implemented outside api.cu report their workspace sizes here.
pk_status bispectrum_ws(const pk_config* c, int nshells, bool counts, size_t* out);
pk_status backward_ws(const pk_config* c, int64_t n, size_t* out);
pk_status batch_ws(const pk_config* c, int64_t nmax, size_t* out);
pk_status direct_ws(const pk_config* c, int64_t n, bool cross, size_t* out);
pk_status aliasing_ws(const pk_config* c, size_t* out);
pk_status multigrid_ws(const pk_config* c, int ngrids, int64_t n, size_t* out);

}  // namespace pk
