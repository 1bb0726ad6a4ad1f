// Interlacing with more than two grids (the extension Sec. 3.1 points to): J = 1, 2, 4 or 8 mass grids,
// grid j holding the particles shifted by d_j H with d_j in {0, 1/2}^3, each transformed, multiplied by
// e^{+i k.d_j H} = e^{+2 pi i n.d_j/N} and averaged:
//   delta(n) = sum_j e^{+2 pi i n.d_j/N} G_j(n) / (J sum(w) W(n)).
// By the shift theorem, image m of grid j then carries e^{+2 pi i m.d_j}, so the average keeps image m
// with the weight theta_m = (1/J) sum_j (-1)^{m.(2 d_j)}:
//   J = 2, d = {0, (1,1,1)/2}:                                 theta = 1 for m_x+m_y+m_z even (eq:intdelta);
//   J = 4, d = {0, (1,1,0)/2, (1,0,1)/2, (0,1,1)/2}:           theta = 1 when m_x, m_y, m_z have one parity;
//   J = 8, d = {0, 1/2}^3:                                      theta = 1 when every m_i is even.
// The first images left are |m|^2 = 2 (J = 2), 3 (J = 4) and 4 (J = 8). The grids come from the
// existing assignment: J = 2 and J = 8 as interlaced pairs (d, d + (1,1,1)/2) of the shifted
// particles, J = 4 as single grids. Every mode of the full N^3 grid is binned once, the stored mode
// and, for 0 < i_z < N/2, its partner -n with its own signed index (the phases of a Nyquist slot are
// not conjugate), as in the two-grid estimate.
#include "host.cuh"

namespace pk {

namespace {

// Shift pattern of grid j in half cells (h = 2 d, components 0, 1 or 2).
struct Shifts {
  int h[8][3];
  int bases;      // particle shifts to assign
  bool pairs;     // each base gives an interlaced pair (d, d + (1,1,1)/2)
};

bool make_shifts(int J, Shifts* s) {
  static const int base4[4][3] = {{0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
  switch (J) {
    case 1: s->bases = 1; s->pairs = false; break;
    case 2: s->bases = 1; s->pairs = true; break;
    case 4: s->bases = 4; s->pairs = false; break;
    case 8: s->bases = 4; s->pairs = true; break;
    default: return false;
  }
  int j = 0;
  for (int b = 0; b < s->bases; ++b) {
    for (int a = 0; a < 3; ++a) s->h[j][a] = base4[b][a];
    ++j;
    if (s->pairs) {
      for (int a = 0; a < 3; ++a) s->h[j][a] = base4[b][a] + 1;
      ++j;
    }
  }
  return true;
}

}  // namespace

// Copies of the positions shifted by h H/2 (h in {0, 1} per axis).
__global__ void k_shift_f64(const double* __restrict__ in, int64_t n, double hx, double hy, double hz, double* __restrict__ out) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    out[3 * i] = in[3 * i] + hx;
    out[3 * i + 1] = in[3 * i + 1] + hy;
    out[3 * i + 2] = in[3 * i + 2] + hz;
  }
}

__global__ void k_shift_cells(const pk_cellpos* __restrict__ in, int64_t n, int ng, int hx, int hy, int hz,
                              pk_cellpos* __restrict__ out) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const pk_cellpos r = in[i];
    int c[3] = {cell_x(r.cell), cell_y(r.cell), cell_z(r.cell)};
    float f[3] = {r.fx, r.fy, r.fz};
    const int h[3] = {hx, hy, hz};
    for (int a = 0; a < 3; ++a) {
      if (!h[a]) continue;
      float g;
      c[a] += half_shift(f[a], &g);
      if (g >= 1.0f) {  // f = 0.5 - 2^-25: f + 1/2 rounds to 1 in FP32, which is the next cell's 0
        g = 0.0f;
        c[a] += 1;
      }
      f[a] = g;
      if (c[a] >= ng) c[a] -= ng;
    }
    pk_cellpos o;
    o.cell = pack_cell(c[0], c[1], c[2]);
    o.fx = f[0];
    o.fy = f[1];
    o.fz = f[2];
    out[i] = o;
  }
}

// Per-slot tables (n the signed index of the slot), FP64: 1/W_1d(n), then e^{i pi n h/N} for h = 1 and
// h = 2 (cosine row, sine row each).
constexpr int kMultiTabRows = 5;
__global__ void k_multi_tables(double* __restrict__ tab, int ng, int order) {
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < ng; i += blockDim.x * gridDim.x) {
    const int n = signed_mode(i, ng);
    const double x = double(n) / double(ng);
    const double s = n == 0 ? 1.0 : sinpi(x) / (3.14159265358979323846 * x);
    double w = 1.0;
    for (int k = 0; k < order; ++k) w *= s;
    double sn, cs, sn2, cs2;
    sincospi(x, &sn, &cs);
    sincospi(2.0 * x, &sn2, &cs2);
    tab[i] = 1.0 / w;
    tab[ng + i] = cs;
    tab[2 * ng + i] = sn;
    tab[3 * ng + i] = cs2;
    tab[4 * ng + i] = sn2;
  }
}

struct MultiArgs {
  int ng, J, nbins, lo2, w2;
  int h[8][3];
  int64_t grid_stride;  // complex elements between transformed grids
  double vol;
  const double* wsums;
  double* bin_sum;
  double* bin_k;
  unsigned long long* bin_cnt;
  void* delta_out;
};

template <typename R>
struct Cx {
  R x, y;
};
template <typename R>
__device__ __forceinline__ Cx<R> cmr(Cx<R> a, Cx<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// Shifted-grid combine of J transformed grids and k-shell sums (eq:intdelta generalised to the shift
// set h_j, Sec. 3.1). Per stored mode n (and its partner -n on the half-complex layout):
//   delta(n) = sum_j e^{i pi n.h_j / N} G_j(n) / (J sum(w) W(n)),
// the per-axis phases e^{i pi n h/N} (h = 0, 1, 2) read from tables; the arithmetic runs in the grids'
// precision (FP32 grids: FP32 combine), the shell sums in FP64 (|k| sums from an FP64 square root).
// Consecutive lanes hold consecutive i_z, so a warp's modes fall in few shells: runs of equal shell
// are summed with a segmented warp scan and one lane per run adds them to shared memory.
template <typename V>
__global__ void __launch_bounds__(256) k_estimate_multi(const V* __restrict__ G, const double* __restrict__ tab_g, MultiArgs a) {
  using R = decltype(V{}.x);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ng = a.ng;
  double* s_sum = reinterpret_cast<double*>(smem_raw);
  double* s_k = s_sum + a.nbins;
  unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(s_k + a.nbins);
  R* tab = reinterpret_cast<R*>(s_cnt + a.nbins);  // [kMultiTabRows][ng], the grids' precision
  for (int i = threadIdx.x; i < kMultiTabRows * ng; i += blockDim.x) tab[i] = R(tab_g[i]);
  for (int i = threadIdx.x; i < a.nbins; i += blockDim.x) {
    s_sum[i] = 0.0;
    s_k[i] = 0.0;
    s_cnt[i] = 0ull;
  }
  __syncthreads();
  const R norm = R(1.0 / (double(a.J) * a.wsums[0]));
  const R vol = R(a.vol);
  const int H = ng / 2 + 1;
  const int64_t count = int64_t(ng) * ng * H;
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  // whole warps step together (the shell sums are warp-collective)
  for (int64_t m0 = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); m0 < count; m0 += stride) {
    const int64_t m = m0 + lane;
    int b = -1, mult = 0;
    R pv = R(0);
    double kv = 0.0;
    if (m < count) {
      const int iz = int(m % H);
      const int64_t xy = m / H;
      const int iy = int(xy % ng), ix = int(xy / ng);
      const int slot[3] = {ix, iy, iz};
      int pslot[3];  // slots of the partner -n
#pragma unroll
      for (int d = 0; d < 3; ++d) pslot[d] = slot[d] == 0 ? 0 : ng - slot[d];
      const R iw = tab[ix] * tab[iy] * tab[iz] * norm;
      // per-axis phase factors for h = 1, 2 at n and at -n
      Cx<R> e[3][2], q[3][2];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          e[d][h] = {tab[(1 + 2 * h) * ng + slot[d]], tab[(2 + 2 * h) * ng + slot[d]]};
          q[d][h] = {tab[(1 + 2 * h) * ng + pslot[d]], tab[(2 + 2 * h) * ng + pslot[d]]};
        }
      Cx<R> dn = {R(0), R(0)}, dp = {R(0), R(0)};
      for (int j = 0; j < a.J; ++j) {
        const V g = G[j * a.grid_stride + m];
        Cx<R> ph = {R(1), R(0)}, pp = {R(1), R(0)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int h = a.h[j][d];  // uniform across the block
          if (h != 0) {
            ph = cmr(ph, h == 1 ? e[d][0] : e[d][1]);
            pp = cmr(pp, h == 1 ? q[d][0] : q[d][1]);
          }
        }
        const Cx<R> t = cmr(Cx<R>{g.x, g.y}, ph);
        const Cx<R> u = cmr(Cx<R>{g.x, -g.y}, pp);  // G(-n) = conj G(n)
        dn.x += t.x;
        dn.y += t.y;
        dp.x += u.x;
        dp.y += u.y;
      }
      dn.x *= iw;
      dn.y *= iw;
      dp.x *= iw;
      dp.y *= iw;
      if (m == 0) dn = {R(0), R(0)};
      if (a.delta_out) {
        V o;
        o.x = dn.x;
        o.y = dn.y;
        static_cast<V*>(a.delta_out)[m] = o;
      }
      if (a.nbins > 0) {
        const long long nx = signed_mode(ix, ng), ny = signed_mode(iy, ng), nz = signed_mode(iz, ng);
        const long long n2 = nx * nx + ny * ny + nz * nz;
        b = bin_of(4 * n2, a.lo2, a.w2, a.nbins);
        if (b >= 0) {
          const bool partner = iz != 0 && iz != ng / 2;
          pv = vol * (dn.x * dn.x + dn.y * dn.y);
          if (partner) pv += vol * (dp.x * dp.x + dp.y * dp.y);
          mult = partner ? 2 : 1;
          kv = double(mult) * sqrt(double(n2));
        }
      }
    }
    if (a.nbins == 0) continue;
    // segmented inclusive scan over runs of equal b; the last lane of each run adds the run's sums
    const int bprev = __shfl_up_sync(0xffffffffu, b, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || bprev != b);
    const int start = 31 - __clz(heads & ((2u << lane) - 1u));
    const int bnext = __shfl_down_sync(0xffffffffu, b, 1);
    const bool end = lane == 31 || bnext != b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const R tv = __shfl_up_sync(0xffffffffu, pv, o);
      const double tk = __shfl_up_sync(0xffffffffu, kv, o);
      const int tc = __shfl_up_sync(0xffffffffu, mult, o);
      if (lane - o >= start) {
        pv += tv;
        kv += tk;
        mult += tc;
      }
    }
    if (end && b >= 0) {
      atomicAdd(&s_sum[b], double(pv));
      atomicAdd(&s_k[b], kv);
      atomicAdd(&s_cnt[b], (unsigned long long)mult);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.nbins; i += blockDim.x) {
    if (s_cnt[i] == 0ull) continue;
    atomicAdd(&a.bin_sum[i], s_sum[i]);
    atomicAdd(&a.bin_k[i], s_k[i]);
    atomicAdd(&a.bin_cnt[i], s_cnt[i]);
  }
}

namespace {

struct MultiLayout {
  void* grids = nullptr;  // [J] padded grids (real) = half-complex after the in-place R2C
  void* shifted = nullptr;
  BinStage b;
  pk_cellpos* sorted = nullptr;
  float* wsorted = nullptr;
  int64_t* offsets = nullptr;
  double* wsums = nullptr;
  double* tab = nullptr;
  double* bin_sum = nullptr;
  double* bin_k = nullptr;
  unsigned long long* bin_cnt = nullptr;
  void* fft_work = nullptr;
  PlanEntry plan;
  int kind = 0;
};

pk_status carve_multi(const pk_config* c, int J, int64_t n, Carver& cv, MultiLayout* L) {
  const bool dbl = c->prec != PK_FP32;
  L->kind = dbl ? 1 : 0;
  L->grids = cv.take<char>(size_t(J) * padded_count(c->ng) * (dbl ? 8 : 4));
  // shifted copies in the input's format (the larger of the two)
  L->shifted = cv.take<char>(size_t(std::max<int64_t>(n, 1)) * 24);
  if (c->prec != PK_FP64) {
    carve_bin_stage(c, n, true, cv, &L->b);
    L->sorted = cv.take<pk_cellpos>(size_t(std::max<int64_t>(n, 1)));
    L->wsorted = cv.take<float>(size_t(std::max<int64_t>(n, 1)));
    const int nt = tiles_per_axis(c->ng);
    L->offsets = cv.take<int64_t>(size_t(int64_t(nt) * nt * nt + 1));
  }
  L->wsums = cv.take<double>(3);
  L->tab = cv.take<double>(size_t(kMultiTabRows) * c->ng);
  L->bin_sum = cv.take<double>(c->nbins);
  L->bin_k = cv.take<double>(c->nbins);
  L->bin_cnt = cv.take<unsigned long long>(c->nbins);
  pk_status st = get_plan(c->ng, L->kind, J, &L->plan);
  if (st != PK_OK) return st;
  L->fft_work = cv.take<char>(std::max<size_t>(L->plan.work, 256));
  return PK_OK;
}

}  // namespace

pk_status multigrid_ws(const pk_config* c, int J, int64_t n, size_t* out) {
  Shifts sh;
  if (!make_shifts(J, &sh)) return fail(PK_EINVAL, "ngrids must be 1, 2, 4 or 8 (got %d)", J);
  Carver cv(nullptr);
  MultiLayout L;
  pk_status st = carve_multi(c, J, n, cv, &L);
  if (st != PK_OK) return st;
  *out = cv.size();
  return PK_OK;
}

}  // namespace pk

using namespace pk;

extern "C" {

size_t pk_multigrid_workspace_size(const pk_config* cfg, int32_t ngrids, int64_t n) {
  clear_err();
  if (validate(cfg) != PK_OK) return 0;
  if (n < 0) {
    fail(PK_EINVAL, "n < 0");
    return 0;
  }
  size_t out = 0;
  return multigrid_ws(cfg, ngrids, n, &out) == PK_OK ? out : 0;
}

pk_status pk_power_multigrid(const pk_config* cfg, int32_t ngrids, const void* pos_dev, int32_t pos_format,
                             const float* w_dev, int64_t n, double* pk_dev, double* kmean_dev, int64_t* nmodes_dev,
                             void* delta_k_dev, void* ws, size_t ws_bytes, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  Shifts sh;
  if (!make_shifts(ngrids, &sh)) return fail(PK_EINVAL, "ngrids must be 1, 2, 4 or 8 (got %d)", ngrids);
  if (pos_format != PK_POS_F64_XYZ && pos_format != PK_POS_CELL_F32OFF) return fail(PK_EINVAL, "bad pos_format");
  if (n < 1 || !pos_dev) return fail(PK_EINVAL, "need at least one particle");
  if (!pk_dev || !nmodes_dev) return fail(PK_EINVAL, "bad output pointers");
  size_t need = 0;
  if ((st = multigrid_ws(cfg, ngrids, n, &need)) != PK_OK) return st;
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  MultiLayout L;
  if ((st = carve_multi(cfg, ngrids, n, cv, &L)) != PK_OK) return st;
  const int ng = cfg->ng;
  const bool dbl = cfg->prec != PK_FP32;
  const int64_t per = padded_count(ng);
  const size_t gbytes = size_t(per) * (dbl ? 8 : 4);
  cudaError_t e;
  if ((st = run_weight_sums(w_dev, n, L.wsums, s)) != PK_OK) return st;
  pk_config sub = *cfg;
  sub.interlace = sh.pairs ? 1 : 0;
  const int blocks = int(std::min<int64_t>(int64_t(num_sms()) * 8, (n + 255) / 256));
  const double half = 0.5 * cfg->box / ng;
  // FP32 from FP64 positions: the first (unshifted) base prepares the packed records once; later bases
  // shift those records instead of preparing shifted FP64 positions again
  const bool reuse_prepared = cfg->prec == PK_FP32 && pos_format == PK_POS_F64_XYZ;
  for (int b = 0; b < sh.bases; ++b) {
    const int* hb = sh.h[sh.pairs ? 2 * b : b];
    const void* pos = pos_dev;
    int fmt = pos_format;
    if (hb[0] | hb[1] | hb[2]) {
      if (reuse_prepared) {  // base 0 is unshifted, so L.b.cells holds the prepared records
        k_shift_cells<<<blocks, 256, 0, s>>>(L.b.cells, n, ng, hb[0], hb[1], hb[2], static_cast<pk_cellpos*>(L.shifted));
        fmt = PK_POS_CELL_F32OFF;
      } else if (pos_format == PK_POS_F64_XYZ) {
        k_shift_f64<<<blocks, 256, 0, s>>>(static_cast<const double*>(pos_dev), n, hb[0] * half, hb[1] * half, hb[2] * half,
                                           static_cast<double*>(L.shifted));
      } else {
        k_shift_cells<<<blocks, 256, 0, s>>>(static_cast<const pk_cellpos*>(pos_dev), n, ng, hb[0], hb[1], hb[2],
                                             static_cast<pk_cellpos*>(L.shifted));
      }
      count_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "shift");
      pos = L.shifted;
    }
    void* grids = static_cast<char*>(L.grids) + gbytes * size_t(sh.pairs ? 2 * b : b);
    if (cfg->prec == PK_FP64) {
      st = run_assign_into(&sub, pos, fmt, nullptr, w_dev, nullptr, n, L.wsums, grids, ng + 2, s);
    } else {
      if ((st = run_bin(&sub, pos, fmt, w_dev, n, L.b, L.sorted, w_dev ? L.wsorted : nullptr, L.offsets, s)) != PK_OK)
        return st;
      st = run_assign_into(&sub, nullptr, PK_POS_CELL_F32OFF, L.sorted, w_dev ? L.wsorted : nullptr, L.offsets, n, L.wsums,
                           grids, ng + 2, s);
    }
    if (st != PK_OK) return st;
  }
  if ((st = exec_plan(L.plan, L.kind, L.grids, L.fft_work, s)) != PK_OK) return st;
  k_multi_tables<<<(ng + 127) / 128, 128, 0, s>>>(L.tab, ng, cfg->order); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "tables");
  const size_t nb = size_t(cfg->nbins);
  if ((e = cudaMemsetAsync(L.bin_sum, 0, sizeof(double) * nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(L.bin_k, 0, sizeof(double) * nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(L.bin_cnt, 0, sizeof(unsigned long long) * nb, s)) != cudaSuccess)
    return cuda_fail(e, "memset");
  MultiArgs a{};
  a.ng = ng;
  a.J = ngrids;
  a.nbins = cfg->nbins;
  a.lo2 = cfg->bin_lo2;
  a.w2 = cfg->bin_w2;
  for (int j = 0; j < ngrids; ++j)
    for (int d = 0; d < 3; ++d) a.h[j][d] = sh.h[j][d];
  a.grid_stride = per / 2;
  a.vol = cfg->box * cfg->box * cfg->box;
  a.wsums = L.wsums;
  a.bin_sum = L.bin_sum;
  a.bin_k = L.bin_k;
  a.bin_cnt = L.bin_cnt;
  a.delta_out = delta_k_dev;
  const int64_t hc = half_count(ng);
  const int eblocks = int(std::min<int64_t>(int64_t(num_sms()) * 4, (hc + 255) / 256));
  // bins first (8-byte entries), then the tables in the grids' precision
  const size_t smem = nb * (2 * sizeof(double) + sizeof(unsigned long long)) + (dbl ? 8 : 4) * size_t(kMultiTabRows) * ng;
  if (dbl) {
    if ((e = ensure_dynamic_smem(reinterpret_cast<const void*>(k_estimate_multi<double2>), smem)) != cudaSuccess)
      return cuda_fail(e, "estimate smem");
    k_estimate_multi<double2><<<eblocks, 256, smem, s>>>(static_cast<const double2*>(L.grids), L.tab, a);
  } else {
    if ((e = ensure_dynamic_smem(reinterpret_cast<const void*>(k_estimate_multi<float2>), smem)) != cudaSuccess)
      return cuda_fail(e, "estimate smem");
    k_estimate_multi<float2><<<eblocks, 256, smem, s>>>(static_cast<const float2*>(L.grids), L.tab, a);
  }
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "estimate");
  EstimateArgs f{};
  f.ng = ng;
  f.nbins = cfg->nbins;
  f.bin_lo2 = cfg->bin_lo2;
  f.bin_w2 = cfg->bin_w2;
  f.box = cfg->box;
  f.wsums = L.wsums;
  f.bin_sum = L.bin_sum;
  f.bin_k = L.bin_k;
  f.bin_cnt = L.bin_cnt;
  if ((e = launch_finalize(f, cfg->subtract_shot, pk_dev, kmean_dev, nmodes_dev, s)) != cudaSuccess)
    return cuda_fail(e, "finalize");
  return PK_OK;
}

}  // extern "C"
