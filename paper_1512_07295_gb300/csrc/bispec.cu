// a7 FFT bispectrum (Sec. 4.1, eq:Best2 and eq:IntI) and the exact triangle counts (eq:VBest).
//
// Shells s = 0..S-1 hold the modes n != 0 with (lo + s w) <= |n| < (lo + (s+1) w) (units of k_f).
// pk_bispectrum: every shell's filtered copy of delta(n) is inverse real-FFT'd (one batched C2R) into
// I_s(x) = sum_{n in s} delta(n) e^{+2 pi i n.x/N}; one pass over x-tiles staged in shared memory
// then accumulates S_t = sum_x I_a I_b I_c for all triangles t = (a, b, c) at once (FP32 products
// within a tile of 128 points, FP64 across tiles), and B_t = V^2 S_t / (N_c N_tri,t).
// pk_bispectrum_counts: N_tri,t = #{(q1, q2, q3): q_i in shell, q1 + q2 + q3 = 0} exactly. With
// F_s(x) = sum_{n in s} e^{+2 pi i n.x/N} (inverse FFT of the indicator), the number of pairs
// (q1 in a, q2 in b) with q1 + q2 = m is C_ab(m) = (1/N_c) sum_x F_a F_b e^{-2 pi i m.x/N}, an
// integer computed in FP64 (error far below 1/2) and rounded; N_tri = sum_{m in c} C_ab(m) in int64.
#include <cmath>
#include <vector>

#include "host.cuh"

namespace pk {

static std::vector<int> make_triangles(int nshells) {
  std::vector<int> t;
  for (int a = 0; a < nshells; ++a)
    for (int b = 0; b <= a; ++b)
      for (int c = 0; c <= b; ++c)
        if (a <= b + c + 1) {
          t.push_back(a);
          t.push_back(b);
          t.push_back(c);
        }
  return t;
}

__device__ __forceinline__ int shell_of(long long n2, int lo, int w, int nshells) {
  if (n2 == 0) return -1;
  int s = int(floorf((sqrtf(float(n2)) - float(lo)) / float(w)));
  if (s < 0) s = 0;
  long long e = (long long)lo + (long long)s * w;
  while (s > 0 && e * e > n2) { --s; e -= w; }
  if (e * e > n2) return -1;
  long long e1 = e + w;
  while (e1 * e1 <= n2) { ++s; e1 += w; if (s >= nshells) return -1; }
  return s < nshells ? s : -1;
}

__device__ __forceinline__ long long mode_n2(int64_t idx, int ng, int* iz_out) {
  const int lz = ng / 2 + 1;
  const int iz = int(idx % lz);
  const int64_t row = idx / lz;
  const int iy = int(row % ng), ix = int(row / ng);
  const int nx = signed_mode(ix, ng), ny = signed_mode(iy, ng);
  const int nz = iz == ng / 2 ? -(ng / 2) : iz;
  *iz_out = iz;
  return (long long)nx * nx + (long long)ny * ny + (long long)nz * nz;
}

// Writes the shell-filtered copies of delta (R2 = float2/double2) into the nshells complex buffers.
template <typename R2>
__global__ void k_shell_filter(const R2* __restrict__ delta, R2* __restrict__ out, int ng, int lo, int w, int nshells,
                               int64_t buf_stride) {
  const int64_t nh = int64_t(ng) * ng * (ng / 2 + 1);
  for (int64_t i = gtid(); i < nh; i += gstride()) {
    int iz;
    const int s = shell_of(mode_n2(i, ng, &iz), lo, w, nshells);
    const R2 d = delta[i];
    R2 z;
    z.x = 0;
    z.y = 0;
    for (int t = 0; t < nshells; ++t) out[t * buf_stride + i] = (t == s) ? d : z;
  }
}

// Indicator of each shell (1 on the shell's modes) for the counts.
__global__ void k_shell_indicator(double2* __restrict__ out, int ng, int lo, int w, int nshells, int64_t buf_stride) {
  const int64_t nh = int64_t(ng) * ng * (ng / 2 + 1);
  for (int64_t i = gtid(); i < nh; i += gstride()) {
    int iz;
    const int s = shell_of(mode_n2(i, ng, &iz), lo, w, nshells);
    for (int t = 0; t < nshells; ++t) out[t * buf_stride + i] = make_double2(t == s ? 1.0 : 0.0, 0.0);
  }
}

constexpr int kTX = 128;       // x points per staged tile
constexpr int kRow = kTX + 1;  // padded row of a staged field: shells in different banks

// Stages the tile's values of every field: vals[s][k] = I_s(tile * kTX + k) (0 past the grid).
template <typename R>
__device__ __forceinline__ void stage_fields(R* vals, const R* __restrict__ fields, int ng, int nshells, int64_t buf_stride,
                                             int64_t tile, int64_t npts) {
  for (int i = threadIdx.x; i < nshells * kTX; i += blockDim.x) {
    const int s = i / kTX, k = i - s * kTX;
    const int64_t x = tile * kTX + k;
    R v = R(0);
    if (x < npts) {
      const int64_t row = x / ng;
      v = fields[s * buf_stride + row * (ng + 2) + (x - row * ng)];
    }
    vals[s * kRow + k] = v;
  }
}

// The triple product with lanes over points: warp w owns a contiguous run of at most kWarpTri
// triangles (a, b, c) for the whole kernel and keeps one running sum per triangle in each lane. Per
// staged tile, lane l takes the points l, l + 32, l + 64, l + 96; the products I_a I_b of those points
// are reloaded only when the pair (a, b) changes (consecutive triangles share it), and every load is a
// conflict-free row segment. Every kFlushTiles tiles the lane sums are reduced across the warp (FP32,
// 32 lanes x kFlushTiles x 4 points) and added to a compensated FP32 pair per triangle (Neumaier's
// summation), which is added to S in FP64 at the end; the loop itself uses no FP64 arithmetic, which
// this GPU executes at a small fraction of the FP32 rate. The next tile's field values are loaded
// into registers while the current tile is processed.
constexpr int kWarpTri = 32;
constexpr int kTriWarps = 16;
constexpr int kFlushTiles = 16;
constexpr int kTriMaxShells = 16;                                                    // ntri <= 512 implies this
constexpr int kStagePer = (kTriMaxShells * kTX + kTriWarps * 32 - 1) / (kTriWarps * 32);  // staged values per thread

template <typename R>
__device__ __forceinline__ void comp_add(R* hi, R* lo, R v) {
  const R t = *hi + v;
  *lo += (fabs(*hi) >= fabs(v)) ? (*hi - t) + v : (v - t) + *hi;
  *hi = t;
}

template <typename R>
__global__ void __launch_bounds__(kTriWarps * 32) k_triple_warp(const R* __restrict__ fields, int ng, int nshells,
                                                               int64_t buf_stride, const int* __restrict__ tri_g, int ntri,
                                                               double* __restrict__ S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* shi = reinterpret_cast<R*>(smem_raw);  // [ntri] compensated per-block sums
  R* slo = shi + ntri;
  int* tri = reinterpret_cast<int*>(slo + ntri);                 // [ntri] packed a | b << 8 | c << 16
  R* vals = reinterpret_cast<R*>(tri + ((ntri + 3) / 4) * 4);      // [nshells][kRow]
  for (int t = threadIdx.x; t < ntri; t += blockDim.x) {
    shi[t] = R(0);
    slo[t] = R(0);
    tri[t] = tri_g[3 * t] | (tri_g[3 * t + 1] << 8) | (tri_g[3 * t + 2] << 16);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (ntri + kTriWarps - 1) / kTriWarps;  // <= kWarpTri (checked by the launcher)
  const int t_beg = warp * per, t_cnt = max(0, min(per, ntri - t_beg));
  R acc[kWarpTri];
#pragma unroll
  for (int j = 0; j < kWarpTri; ++j) acc[j] = R(0);
  const int64_t npts = int64_t(ng) * ng * ng;
  const int64_t ntiles = (npts + kTX - 1) / kTX;
  const int nval = nshells * kTX;
  // values of the first tile, then of the next one while the current one is processed
  R pre[kStagePer];
  auto load_tile = [&](int64_t tile) {
#pragma unroll
    for (int u = 0; u < kStagePer; ++u) {
      const int i = threadIdx.x + u * kTriWarps * 32;
      R v = R(0);
      if (i < nval) {
        const int sh = i / kTX, k = i - sh * kTX;
        const int64_t x = tile * kTX + k;
        if (x < npts) {
          const int64_t row = x / ng;
          v = fields[sh * buf_stride + row * (ng + 2) + (x - row * ng)];
        }
      }
      pre[u] = v;
    }
  };
  if (blockIdx.x < ntiles) load_tile(blockIdx.x);
  int since_flush = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kStagePer; ++u) {
      const int i = threadIdx.x + u * kTriWarps * 32;
      if (i < nval) {
        const int sh = i / kTX;
        vals[sh * kRow + (i - sh * kTX)] = pre[u];
      }
    }
    __syncthreads();
    if (tile + gridDim.x < ntiles) load_tile(tile + gridDim.x);
    int pab_key = -1;
    R pab[kTX / 32];
#pragma unroll
    for (int j = 0; j < kWarpTri; ++j) {
      if (j < t_cnt) {
        const int code = tri[t_beg + j];
        const int key = code & 0xffff, c = code >> 16;
        if (key != pab_key) {  // warp-uniform
          pab_key = key;
          const R* ra = vals + (key & 0xff) * kRow + lane;
          const R* rb = vals + (key >> 8) * kRow + lane;
#pragma unroll
          for (int i = 0; i < kTX / 32; ++i) pab[i] = ra[32 * i] * rb[32 * i];
        }
        const R* rc = vals + c * kRow + lane;
        R sum = acc[j];
#pragma unroll
        for (int i = 0; i < kTX / 32; ++i) sum += pab[i] * rc[32 * i];
        acc[j] = sum;
      }
    }
    if (++since_flush == kFlushTiles || tile + gridDim.x >= ntiles) {
      since_flush = 0;
#pragma unroll
      for (int j = 0; j < kWarpTri; ++j) {
        if (j < t_cnt) {
          R v = acc[j];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) comp_add(&shi[t_beg + j], &slo[t_beg + j], v);
        }
        acc[j] = R(0);
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntri; t += blockDim.x) atomicAdd(&S[t], double(shi[t]) + double(slo[t]));
}

template <typename R>
__global__ void __launch_bounds__(512) k_triple(const R* __restrict__ fields, int ng, int nshells, int64_t buf_stride,
                                               const int* __restrict__ tri, int ntri, double* __restrict__ S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sblk = reinterpret_cast<double*>(smem_raw);  // [ntri]
  R* vals = reinterpret_cast<R*>(smem_raw + size_t(ntri) * sizeof(double));  // [nshells][kRow]
  for (int t = threadIdx.x; t < ntri; t += blockDim.x) sblk[t] = 0.0;
  const int64_t npts = int64_t(ng) * ng * ng;
  const int64_t ntiles = (npts + kTX - 1) / kTX;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();
    stage_fields(vals, fields, ng, nshells, buf_stride, tile, npts);
    __syncthreads();
    for (int t = threadIdx.x; t < ntri; t += blockDim.x) {
      const R* va = vals + tri[3 * t] * kRow;
      const R* vb = vals + tri[3 * t + 1] * kRow;
      const R* vc = vals + tri[3 * t + 2] * kRow;
      R acc = R(0);
#pragma unroll 8
      for (int k = 0; k < kTX; ++k) acc += va[k] * vb[k] * vc[k];
      sblk[t] += double(acc);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntri; t += blockDim.x) atomicAdd(&S[t], sblk[t]);
}

__global__ void k_bisp_final(const double* __restrict__ S, const long long* __restrict__ counts, int ntri, double scale,
                             double* __restrict__ B) {
  for (int t = threadIdx.x + blockIdx.x * blockDim.x; t < ntri; t += blockDim.x * gridDim.x) {
    const long long c = counts[t];
    B[t] = c > 0 ? scale * S[t] / double(c) : __longlong_as_double(0x7ff8000000000000ll);
  }
}

__global__ void k_triangles(int* tri, int nshells) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int k = 0;
  for (int a = 0; a < nshells; ++a)
    for (int b = 0; b <= a; ++b)
      for (int c = 0; c <= b; ++c)
        if (a <= b + c + 1) {
          tri[k++] = a;
          tri[k++] = b;
          tri[k++] = c;
        }
}

// prod = F_a * F_b on the valid points of the padded real layout.
__global__ void k_pair_product(const double* __restrict__ fa, const double* __restrict__ fb, double* __restrict__ prod, int ng) {
  const int64_t npts = int64_t(ng) * ng * ng;
  for (int64_t x = gtid(); x < npts; x += gstride()) {
    const int64_t row = x / ng;
    const int64_t p = row * (ng + 2) + (x - row * ng);
    prod[p] = fa[p] * fb[p];
  }
}

struct TriOfC {  // for a pair (a, b): triangle index of (a, b, c) for each c, or -1
  int t[64];
};

// counts[t(a,b,c)] += sum_{m in shell c} round(Re C_ab(m) N_c / N_c), weighting stored modes by their
// Hermitian multiplicity (2 for 0 < i_z < N/2).
__global__ void k_pair_counts(const double2* __restrict__ cf, int ng, int lo, int w, int nshells, TriOfC map,
                              unsigned long long* __restrict__ counts) {
  __shared__ unsigned long long sc[64];
  for (int i = threadIdx.x; i < nshells; i += blockDim.x) sc[i] = 0;
  __syncthreads();
  const int64_t nh = int64_t(ng) * ng * (ng / 2 + 1);
  const double inv_nc = 1.0 / (double(ng) * ng * ng);
  for (int64_t i = gtid(); i < nh; i += gstride()) {
    int iz;
    const int s = shell_of(mode_n2(i, ng, &iz), lo, w, nshells);
    if (s < 0 || map.t[s] < 0) continue;
    const long long v = llrint(cf[i].x * inv_nc);
    if (v == 0) continue;
    const long long mult = (iz > 0 && iz < ng / 2) ? 2 : 1;
    atomicAdd(&sc[s], (unsigned long long)(v * mult));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nshells; i += blockDim.x)
    if (sc[i] && map.t[i] >= 0) atomicAdd(&counts[map.t[i]], sc[i]);
}

// ---- workspace layouts ----------------------------------------------------------------------------------

struct BispLayout {
  void* fields = nullptr;  // nshells padded grids (R)
  int* tri = nullptr;
  double* S = nullptr;
  void* work = nullptr;
  PlanEntry plan;
  int kind = 0;
};

static pk_status carve_bisp(const pk_config* c, int nshells, Carver& cv, BispLayout* L) {
  const bool dbl = c->prec != PK_FP32;
  const int ntri = int(make_triangles(nshells).size() / 3);
  L->kind = dbl ? 3 : 2;
  L->fields = cv.take<char>(size_t(nshells) * padded_count(c->ng) * (dbl ? 8 : 4));
  L->tri = cv.take<int>(size_t(3 * std::max(ntri, 1)));
  L->S = cv.take<double>(size_t(std::max(ntri, 1)));
  pk_status st = get_plan(c->ng, L->kind, nshells, &L->plan);
  if (st != PK_OK) return st;
  L->work = cv.take<char>(std::max<size_t>(L->plan.work, 256));
  return PK_OK;
}

struct CountLayout {
  double* fields = nullptr;  // nshells padded FP64 grids
  double* prod = nullptr;    // one padded FP64 grid
  unsigned long long* counts = nullptr;
  void* work = nullptr;
  PlanEntry inv, fwd;
};

static pk_status carve_counts(const pk_config* c, int nshells, Carver& cv, CountLayout* L) {
  const int ntri = int(make_triangles(nshells).size() / 3);
  L->fields = cv.take<double>(size_t(nshells) * padded_count(c->ng));
  L->prod = cv.take<double>(size_t(padded_count(c->ng)));
  L->counts = cv.take<unsigned long long>(size_t(std::max(ntri, 1)));
  pk_status st = get_plan(c->ng, 3, nshells, &L->inv);
  if (st != PK_OK) return st;
  if ((st = get_plan(c->ng, 1, 1, &L->fwd)) != PK_OK) return st;
  L->work = cv.take<char>(std::max<size_t>(std::max(L->inv.work, L->fwd.work), 256));
  return PK_OK;
}

pk_status bispectrum_ws(const pk_config* c, int nshells, bool counts, size_t* out) {
  Carver cv(nullptr);
  pk_status st;
  if (counts) {
    CountLayout L;
    st = carve_counts(c, nshells, cv, &L);
  } else {
    BispLayout L;
    st = carve_bisp(c, nshells, cv, &L);
  }
  if (st != PK_OK) return st;
  *out = cv.size();
  return PK_OK;
}

static pk_status check_shells(const pk_config* c, int lo, int w, int nshells) {
  if (nshells < 1 || nshells > 64) return fail(PK_EINVAL, "nshells must be 1..64");
  if (lo < 0 || w < 1) return fail(PK_EINVAL, "shells need shell_lo >= 0 and shell_w >= 1");
  const int64_t kmax = int64_t(lo) + int64_t(nshells) * w;
  if (3 * (kmax - 1) >= c->ng)
    return fail(PK_EINVAL, "shells reach |n| = %lld; the estimator needs 3 (kmax - 1) < N = %d (k_max = k_f N/3)",
                (long long)kmax - 1, c->ng);
  return PK_OK;
}

}  // namespace pk

using namespace pk;

extern "C" {

int32_t pk_bispectrum_ntri(int32_t nshells) {
  if (nshells < 1 || nshells > 64) return 0;
  return int32_t(make_triangles(nshells).size() / 3);
}

pk_status pk_bispectrum_counts(const pk_config* cfg, int32_t shell_lo, int32_t shell_w, int32_t nshells, int64_t* counts_dev,
                               void* ws, size_t ws_bytes, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if ((st = check_shells(cfg, shell_lo, shell_w, nshells)) != PK_OK) return st;
  if (!counts_dev) return fail(PK_EINVAL, "counts_dev is NULL");
  size_t need = 0;
  if ((st = bispectrum_ws(cfg, nshells, true, &need)) != PK_OK) return st;
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  CountLayout L;
  if ((st = carve_counts(cfg, nshells, cv, &L)) != PK_OK) return st;
  const std::vector<int> tri = make_triangles(nshells);
  const int ntri = int(tri.size() / 3);
  const int ng = cfg->ng;
  const int64_t pc = padded_count(ng);
  const int64_t hstride = pc / 2;  // complex elements per padded grid
  cudaError_t e;
  const int blocks = num_sms() * 8;
  k_shell_indicator<<<blocks, 256, 0, s>>>(reinterpret_cast<double2*>(L.fields), ng, shell_lo, shell_w, nshells, hstride); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "indicator");
  if ((st = exec_plan(L.inv, 3, L.fields, L.work, s)) != PK_OK) return st;
  if ((e = cudaMemsetAsync(L.counts, 0, sizeof(unsigned long long) * ntri, s)) != cudaSuccess) return cuda_fail(e, "memset");
  for (int a = 0; a < nshells; ++a) {
    for (int b = 0; b <= a; ++b) {
      TriOfC map;
      bool any = false;
      for (int c = 0; c < 64; ++c) map.t[c] = -1;
      for (int t = 0; t < ntri; ++t)
        if (tri[3 * t] == a && tri[3 * t + 1] == b) {
          map.t[tri[3 * t + 2]] = t;
          any = true;
        }
      if (!any) continue;
      k_pair_product<<<blocks, 256, 0, s>>>(L.fields + a * pc, L.fields + b * pc, L.prod, ng); count_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "pair product");
      if ((st = exec_plan(L.fwd, 1, L.prod, L.work, s)) != PK_OK) return st;
      k_pair_counts<<<blocks, 256, 0, s>>>(reinterpret_cast<const double2*>(L.prod), ng, shell_lo, shell_w, nshells, map,
                                            L.counts); count_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "pair counts");
    }
  }
  e = cudaMemcpyAsync(counts_dev, L.counts, sizeof(int64_t) * ntri, cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "copy counts");
}

pk_status pk_bispectrum(const pk_config* cfg, const void* delta_k_dev, int32_t shell_lo, int32_t shell_w, int32_t nshells,
                        const int64_t* counts_dev, double* B_dev, void* ws, size_t ws_bytes, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if ((st = check_shells(cfg, shell_lo, shell_w, nshells)) != PK_OK) return st;
  if (!delta_k_dev || !counts_dev || !B_dev) return fail(PK_EINVAL, "bad pointers");
  size_t need = 0;
  if ((st = bispectrum_ws(cfg, nshells, false, &need)) != PK_OK) return st;
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  BispLayout L;
  if ((st = carve_bisp(cfg, nshells, cv, &L)) != PK_OK) return st;
  const int ntri = pk_bispectrum_ntri(nshells);
  const int ng = cfg->ng;
  const int64_t pc = padded_count(ng);
  const bool dbl = cfg->prec != PK_FP32;
  const int blocks = num_sms() * 8;
  cudaError_t e;
  k_triangles<<<1, 32, 0, s>>>(L.tri, nshells); count_launch();
  if (dbl)
    k_shell_filter<double2><<<blocks, 256, 0, s>>>(static_cast<const double2*>(delta_k_dev), static_cast<double2*>(L.fields),
                                                  ng, shell_lo, shell_w, nshells, pc / 2);
  else
    k_shell_filter<float2><<<blocks, 256, 0, s>>>(static_cast<const float2*>(delta_k_dev), static_cast<float2*>(L.fields), ng,
                                                 shell_lo, shell_w, nshells, pc / 2); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "shell filter");
  if ((st = exec_plan(L.plan, L.kind, L.fields, L.work, s)) != PK_OK) return st;
  if ((e = cudaMemsetAsync(L.S, 0, sizeof(double) * ntri, s)) != cudaSuccess) return cuda_fail(e, "memset");
  if (ntri <= kTriWarps * kWarpTri && nshells <= kTriMaxShells) {  // lanes over points, warps over triangles
    const size_t wsmem = size_t(2 * ntri) * (dbl ? 8 : 4) + size_t((ntri + 3) / 4) * 16 + size_t(nshells) * kRow * (dbl ? 8 : 4);
    int per_sm = 1;
    if (dbl) {
      if ((e = ensure_dynamic_smem(reinterpret_cast<const void*>(k_triple_warp<double>), wsmem)) != cudaSuccess)
        return cuda_fail(e, "triple smem");
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_triple_warp<double>, kTriWarps * 32, wsmem) != cudaSuccess)
        per_sm = 1;
      k_triple_warp<double><<<num_sms() * std::max(per_sm, 1), kTriWarps * 32, wsmem, s>>>(
          static_cast<const double*>(L.fields), ng, nshells, pc, L.tri, ntri, L.S);
    } else {
      if ((e = ensure_dynamic_smem(reinterpret_cast<const void*>(k_triple_warp<float>), wsmem)) != cudaSuccess)
        return cuda_fail(e, "triple smem");
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_triple_warp<float>, kTriWarps * 32, wsmem) != cudaSuccess)
        per_sm = 1;
      k_triple_warp<float><<<num_sms() * std::max(per_sm, 1), kTriWarps * 32, wsmem, s>>>(
          static_cast<const float*>(L.fields), ng, nshells, pc, L.tri, ntri, L.S);
    }
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "triple product");
    const double vol = cfg->box * cfg->box * cfg->box;
    const double scale = vol * vol / (double(ng) * ng * ng);
    k_bisp_final<<<(ntri + 255) / 256, 256, 0, s>>>(L.S, reinterpret_cast<const long long*>(counts_dev), ntri, scale, B_dev);
    count_launch();
    e = cudaGetLastError();
    return e == cudaSuccess ? PK_OK : cuda_fail(e, "bispectrum final");
  }
  const size_t smem = size_t(nshells) * kRow * (dbl ? 8 : 4) + size_t(ntri) * 8;
  if (smem > 48 * 1024) {
    e = dbl ? ensure_dynamic_smem(reinterpret_cast<const void*>(k_triple<double>), smem)
            : ensure_dynamic_smem(reinterpret_cast<const void*>(k_triple<float>), smem);
    if (e != cudaSuccess) return cuda_fail(e, "triple smem");
  }
  const int tblocks = num_sms() * 2;
  if (dbl)
    k_triple<double><<<tblocks, 512, smem, s>>>(static_cast<const double*>(L.fields), ng, nshells, pc, L.tri, ntri, L.S);
  else
    k_triple<float><<<tblocks, 512, smem, s>>>(static_cast<const float*>(L.fields), ng, nshells, pc, L.tri, ntri, L.S); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "triple product");
  const double vol = cfg->box * cfg->box * cfg->box;
  const double scale = vol * vol / (double(ng) * ng * ng);
  k_bisp_final<<<(ntri + 255) / 256, 256, 0, s>>>(L.S, reinterpret_cast<const long long*>(counts_dev), ntri, scale, B_dev); count_launch();
  e = cudaGetLastError();
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "bispectrum final");
}

}  // extern "C"
