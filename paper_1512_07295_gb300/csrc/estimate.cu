// a5 window deconvolution + interlacing combine + |delta|^2 shell binning, fused in one pass over the
// half-complex transforms of the two grids; a6 finalisation of P(k).
//
// For a stored mode n (slots i_x, i_y, i_z <= N/2) with G_g the DFT of mass grid g:
//   delta(n)  = [G_1(n) + e^{+i pi (n_x+n_y+n_z)/N} G_2(n)] / (2 sum(w) W(n))       (eq:intdelta, eq:windowcorrection)
//   W(n)      = prod_i sinc^p(pi n_i/N)                                               (eq:intkerFT)
// The Hermitian partner -n (not stored when 0 < i_z < N/2) has G_g(-n) = conj G_g(n) but its own
// phase: on a Nyquist slot (i = N/2, n_i = -N/2) the partner index is again -N/2, so its phase is
// e^{-i pi/2}, not the conjugate. Both are evaluated from the same loads, so every mode of the full
// N^3 grid is binned exactly once. P(n) = V |delta(n)|^2 (Sec. 2.2 estimator); bins by the exact
// integer test e_b^2 <= 4|n|^2 < e_{b+1}^2. Two kernels sum the shells:
//  - k_estimate_rows (the single pass, whenever its private bins fit): warps take whole rows and lanes
//    runs of consecutive slots, whose equal-bin runs are summed in registers into per-row private
//    shared-memory bins without atomics;
//  - k_estimate (the deterministic two-pass mode, and bins too many for private copies): warps take 32
//    consecutive slots of the flattened [i_x][i_y][i_z] array, reduce runs of equal bins with a
//    shuffle scan and add the run sums to per-block FP64 (or int64) shared bins.
// Both flush their bins once per block.
#include "internal.cuh"

namespace pk {

template <typename R>
struct C2 {
  R x, y;
};

template <typename R>
__device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R>
__device__ __forceinline__ C2<R> conj(C2<R> a) {
  return {a.x, -a.y};
}

// Per-slot tables: 1/W_1d(n), cos and sin of pi n/N (n the signed index of the slot).
template <typename R>
__global__ void k_tables(R* tab, int ng, int order) {
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < ng; i += blockDim.x * gridDim.x) {
    const int n = signed_mode(i, ng);
    const double x = 3.14159265358979323846 * double(n) / double(ng);
    const double s = n == 0 ? 1.0 : sin(x) / x;
    double w = 1.0;
    for (int k = 0; k < order; ++k) w *= s;
    tab[i] = R(1.0 / w);
    tab[ng + i] = R(cos(x));
    tab[2 * ng + i] = R(sin(x));
  }
}

size_t estimate_table_bytes(int ng, bool dbl) { return size_t(3) * ng * (dbl ? 8 : 4); }

// Shared-memory tables of k_estimate: the three global tables, the normalised i_z window and V.
__host__ __device__ inline size_t estimate_smem_table_bytes(int ng, size_t elem) { return ((size_t(4) * ng + 1) * elem + 15) / 16 * 16; }

// Private bin accumulators of k_estimate_rows (single pass, non-deterministic mode), one copy per row
// of a warp, updated without atomics: FP32 mode keeps each sum as an FP32 pair (value, compensation;
// Neumaier's summation, every term is >= 0), FP64 mode as one double.
template <typename R>
struct PrivBin;
template <>
struct PrivBin<float> {
  float2 sum, k;
  __device__ __forceinline__ static void add(float2& acc, float v) {
    const float t = acc.x + v;
    acc.y += (fmaxf(acc.x, v) - t) + fminf(acc.x, v);
    acc.x = t;
  }
  __device__ __forceinline__ static double value(float2 acc) { return double(acc.x) + double(acc.y); }
  __device__ __forceinline__ static float2 zero() { return make_float2(0.0f, 0.0f); }
  __device__ __forceinline__ static void merge(float2& acc, float2 o) {
    add(acc, o.x);
    acc.y += o.y;
  }
};
template <>
struct PrivBin<double> {
  double sum, k;
  __device__ __forceinline__ static void add(double& acc, double v) { acc += v; }
  __device__ __forceinline__ static double value(double acc) { return acc; }
  __device__ __forceinline__ static double zero() { return 0.0; }
  __device__ __forceinline__ static void merge(double& acc, double o) { acc += o; }
};
constexpr int kEstWarps = 8;  // 256 threads (k_estimate; k_estimate_rows at most)

template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 3) k_estimate(const C2<R>* __restrict__ G1, const C2<R>* __restrict__ G2,
                                                  const R* __restrict__ tab_g, EstimateArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {
    const int cat = blockIdx.y;
    G1 += cat * a.cat_stride;
    if (G2) G2 += cat * a.cat_stride;
    a.wsums += 3 * cat;
    a.bin_sum += int64_t(cat) * a.nbins;
    a.bin_k += int64_t(cat) * a.nbins;
    a.bin_cnt += int64_t(cat) * a.nbins;
  }
  const int ng = a.ng;
  R* tab = reinterpret_cast<R*>(smem_raw);  // 1/W, cos, sin (3 ng); 1/W times the norm (ng); V
  unsigned char* bins_raw = smem_raw + estimate_smem_table_bytes(ng, sizeof(R));
  double* s_sum = reinterpret_cast<double*>(bins_raw);
  double* s_k = s_sum + a.nbins;
  unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(s_k + a.nbins);
  {
    // the normalisation 1 / (2 sum w) (1 / sum w without interlacing) rides on the i_z window, and V
    // is kept beside the tables: both are read from shared memory in the loop, not recomputed
    const R wsum0 = R(a.wsums[0]);
    const R norm0 = a.interlace ? R(0.5) / wsum0 : R(1) / wsum0;
    for (int i = threadIdx.x; i < 3 * ng; i += blockDim.x) tab[i] = tab_g[i];
    for (int i = threadIdx.x; i < ng; i += blockDim.x) tab[3 * ng + i] = tab_g[i] * norm0;
    if (threadIdx.x == 0) tab[4 * ng] = R(a.box * a.box * a.box);
  }
  for (int i = threadIdx.x; i < a.nbins; i += blockDim.x) {
    s_sum[i] = 0.0;
    s_k[i] = 0.0;
    s_cnt[i] = 0ull;
  }
  __syncthreads();
  const R* winv = tab;
  const R* pc = tab + ng;
  const R* ps = tab + 2 * ng;
  const int lane = threadIdx.x & 31;
  const int half = ng / 2;
  const int lz = half + 1;
  // bin edges whose squares fit 32 bits take the 32-bit bin test
  const bool small_bins = int64_t(a.bin_lo2) + int64_t(a.nbins + 1) * a.bin_w2 <= 46340;
  const float inv_w2 = 1.0f / float(a.bin_w2);
  const R* winvz = tab + 3 * ng;
  const R* vol = tab + 4 * ng;
  const int64_t rows = int64_t(ng) * ng;
  const int64_t warp_g = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  C2<R>* dout = static_cast<C2<R>*>(a.delta_out);
  // work items: 32 consecutive slots of the flattened [row][i_z] half-complex array (an item may span
  // a row boundary, so no lane idles at the end of a row); the next item's loads are issued before the
  // current item is processed so that two loads per lane are in flight
  const int nslots = int(rows) * lz;  // <= 1024^2 * 513 < 2^31
  const int items = (nslots + 31) / 32;
  // the item's first slot as (i_x, i_y, i_z), advanced by the grid stride of 32 nwarps slots per item
  const int stride_slots = 32 * int(nwarps);
  const int srow = stride_slots / lz, siz = stride_slots - srow * lz;
  const int srow_x = srow / ng, srow_y = srow - srow_x * ng;
  int iz0, iy0, ix0;
  {
    const int b0 = int(warp_g) * 32;
    const int r0 = b0 / lz;
    iz0 = b0 - r0 * lz;
    ix0 = r0 / ng;
    iy0 = r0 - ix0 * ng;
  }
  C2<R> g1n = {R(0), R(0)}, g2n = {R(0), R(0)};
  if (warp_g < items) {
    const int sl = int(warp_g) * 32 + lane;
    if (sl < nslots) {
      g1n = G1[sl];
      if (a.interlace) g2n = G2[sl];
    }
  }
  for (int item = int(warp_g); item < items; item += int(nwarps)) {
    const C2<R> g1c = g1n, g2c = g2n;
    {
      const int nxt = item + int(nwarps);
      if (nxt < items) {
        const int sl = nxt * 32 + lane;
        if (sl < nslots) {
          g1n = G1[sl];
          if (a.interlace) g2n = G2[sl];
        }
      }
    }
    // this lane's slot: row (i_x, i_y) and i_z, from the item's first slot by carrying along the rows
    const int base = item * 32;
    int iz = iz0 + lane, rseg = 0;
    while (iz >= lz) {
      iz -= lz;
      ++rseg;
    }
    int ix = ix0, iy = iy0 + rseg;
    while (iy >= ng) {
      iy -= ng;
      ++ix;
    }
    const int row = ix * ng + iy;
    ix = min(ix, ng - 1);  // lanes past the last slot read a valid table entry and are not used
    {  // the next item's first slot
      iz0 += siz;
      int carry = 0;
      if (iz0 >= lz) {
        iz0 -= lz;
        carry = 1;
      }
      iy0 += srow_y + carry;
      ix0 += srow_x;
      while (iy0 >= ng) {
        iy0 -= ng;
        ++ix0;
      }
    }
    const int nx = signed_mode(ix, ng), ny = signed_mode(iy, ng);  // |n|^2 <= 3 (N/2)^2 < 2^20
    const R wxy = winv[ix] * winv[iy];
    const C2<R> phx = {pc[ix], ps[ix]}, phy = {pc[iy], ps[iy]};
    const C2<R> phxy = cmul(phx, phy);
    // partner phase per axis: conjugate except on the Nyquist slot
    const C2<R> phxy_p = cmul(ix == half ? phx : conj(phx), iy == half ? phy : conj(phy));
    const int nxy2 = nx * nx + ny * ny;
    {
      const bool live = base + lane < nslots;
      int b = -1;
      R val = R(0), ks = R(0);
      int cnt = 0;
      if (live) {
        const int nz = iz == half ? -half : iz;
        const int n2 = nxy2 + nz * nz;
        const int64_t idx = int64_t(row) * lz + iz;
        C2<R> d = {R(0), R(0)};
        if (n2 != 0) {
          const R c = wxy * winvz[iz];
          const C2<R> g1 = g1c;
          const bool partner = iz > 0 && iz < half;
          C2<R> dp;
          if (a.interlace) {
            const C2<R> g2 = g2c;
            const C2<R> phz = {pc[iz], ps[iz]};
            const C2<R> t = cmul(cmul(phxy, phz), g2);
            d = {(g1.x + t.x) * c, (g1.y + t.y) * c};
            if (ix == half || iy == half) {  // the partner's phase is not the conjugate on the Nyquist rows
              const C2<R> tp = cmul(cmul(phxy_p, conj(phz)), conj(g2));
              dp = {(g1.x + tp.x) * c, (-g1.y + tp.y) * c};
            } else {
              dp = conj(d);
            }
          } else {
            d = {g1.x * c, g1.y * c};
            dp = conj(d);
          }
          const float rn = sqrtf(float(n2));
          b = small_bins ? bin_of32(4 * n2, 2.0f * rn, a.bin_lo2, a.bin_w2, inv_w2, a.nbins)
                         : bin_of(4 * (long long)n2, a.bin_lo2, a.bin_w2, a.nbins);
          if (b >= 0) {
            val = d.x * d.x + d.y * d.y;
            cnt = 1;
            if (partner) {
              val += dp.x * dp.x + dp.y * dp.y;
              cnt = 2;
            }
            val *= *vol;
            // |n| sums are not used by the deterministic mode's first pass
            if (a.det_pass != 1) ks = R(cnt) * (sizeof(R) == 4 ? R(rn) : sqrt(R(n2)));
          }
        }
        if (dout) dout[idx] = d;
      }
      if (a.nbins == 0) continue;
      // segmented inclusive scan over runs of equal b (each lane combines only within its own run, so
      // a run's result never passes through another run's partial sums)
      const int bprev = __shfl_up_sync(0xffffffffu, b, 1);
      const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || bprev != b);
      const int start = 31 - __clz(heads & ((2u << lane) - 1u));
      const int bnext = __shfl_down_sync(0xffffffffu, b, 1);
      const bool end = lane == 31 || bnext != b;
      if (a.det_pass == 0) {
        R sv = val, sk = ks;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const R tv = __shfl_up_sync(0xffffffffu, sv, o);
          const R tk = __shfl_up_sync(0xffffffffu, sk, o);
          if (lane - o >= start) {
            sv += tv;
            sk += tk;
          }
        }
        // the run's mode count: its lanes with one mode plus its lanes with two
        const unsigned run = ((2u << lane) - 1u) & ~((1u << start) - 1u);
        const int sc = __popc(__ballot_sync(0xffffffffu, cnt >= 1) & run) + __popc(__ballot_sync(0xffffffffu, cnt == 2) & run);
        if (end && b >= 0) {
          atomicAdd(&s_sum[b], double(sv));
          atomicAdd(&s_k[b], double(sk));
          atomicAdd(&s_cnt[b], (unsigned long long)sc);
        }
      } else if (a.det_pass == 1) {  // deterministic mode, pass 1: per-bin maximum and mode count
        double sv = double(val);
        int sc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const double tv = __shfl_up_sync(0xffffffffu, sv, o);
          const int tc = __shfl_up_sync(0xffffffffu, sc, o);
          if (lane - o >= start) {
            sv = fmax(sv, tv);
            sc += tc;
          }
        }
        if (end && b >= 0) {
          atomicMax(reinterpret_cast<unsigned long long*>(&s_sum[b]), (unsigned long long)__double_as_longlong(sv));
          atomicAdd(&s_cnt[b], (unsigned long long)sc);
        }
      } else {  // pass 2: exact int64 sums of the values quantised at the bin's scale, and of |n| at 2^20
        long long q = b >= 0 ? llrint(double(val) * a.det_scale[b]) : 0ll;
        long long kq = b >= 0 ? llrint(double(ks) * 1048576.0) : 0ll;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const long long tq = __shfl_up_sync(0xffffffffu, q, o);
          const long long tk = __shfl_up_sync(0xffffffffu, kq, o);
          if (lane - o >= start) {
            q += tq;
            kq += tk;
          }
        }
        if (end && b >= 0) {
          atomicAdd(reinterpret_cast<unsigned long long*>(&s_sum[b]), (unsigned long long)q);
          atomicAdd(reinterpret_cast<unsigned long long*>(&s_k[b]), (unsigned long long)kq);
        }
      }
    }
  }
  __syncthreads();
  if (a.nbins == 0) return;
  for (int i = threadIdx.x; i < a.nbins; i += blockDim.x) {
    if (a.det_pass == 0) {
      if (s_cnt[i]) {
        atomicAdd(&a.bin_sum[i], s_sum[i]);
        atomicAdd(&a.bin_k[i], s_k[i]);
        atomicAdd(&a.bin_cnt[i], s_cnt[i]);
      }
    } else if (a.det_pass == 1) {
      if (s_cnt[i]) {
        atomicMax(reinterpret_cast<unsigned long long*>(&a.bin_sum[i]), (unsigned long long)__double_as_longlong(s_sum[i]));
        atomicAdd(&a.bin_cnt[i], s_cnt[i]);
      }
    } else {
      const unsigned long long v = __double_as_longlong(s_sum[i]), k = __double_as_longlong(s_k[i]);
      if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&a.bin_sum[i]), v);
      if (k) atomicAdd(reinterpret_cast<unsigned long long*>(&a.bin_k[i]), k);
    }
  }
}

// Loads of the half-complex transforms through the read-only path: L1 keeps the lines that a lane's
// consecutive slots share with its neighbours' (k_estimate_rows reads 8 or 16 bytes per lane and slot).
__device__ __forceinline__ C2<float> ld_nc(const C2<float>* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ C2<double> ld_nc(const C2<double>* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

// One run of equal bins being summed by a lane: bin (-2: none yet), sum of P, sum of |n|, modes.
template <typename R>
struct Run {
  int b;
  R v, k;
  int c;
};

template <typename R>
__device__ __forceinline__ void priv_add(PrivBin<R>* pw, unsigned* cw, int b, R v, R k, int c) {
  PrivBin<R>::add(pw[b].sum, v);
  PrivBin<R>::add(pw[b].k, k);
  cw[b] += unsigned(c);
}

// The single-pass estimate with private bins, by rows: a warp takes whole rows (i_x, i_y) of the
// half-complex grids, RW rows at a time (RW = 1 for N >= 256; short rows share a warp), and lane s of
// a row's L = 32 / RW lanes takes the J = ceil((N/2 + 1) / L) consecutive slots i_z = s J .. s J + J - 1.
// Along a row |n| grows with i_z (|n_z| = i_z on every stored slot), so the bins of a row's modes are
// non-decreasing (the out-of-range modes, bin -1, lie at its two ends) and a lane's slots form runs
// of equal bins, summed in registers. A run that starts and ends inside one lane holds a bin that no
// other lane of the row holds: it goes to the row's private bins at once (one copy per row of the
// warp, so rows never meet). The lane's first run (head) and last run (tail) may continue in the
// neighbouring lanes of the row; one segmented shuffle scan per row joins them: a tail carried on
// through lanes that hold a single run ends in the next lane's head, or at a lane boundary. Those run
// ends hold distinct bins too, so no update needs an atomic. Per mode the work is that of k_estimate
// (the stored mode and its Hermitian partner, the window division, the interlacing combine, the exact
// bin test); the row's phases, windows and |n_xy|^2 are taken once per lane and row, and the scan
// once per row instead of once per 32 slots. Blocks of 2 to 8 warps (fewer when the bins are many).
// SMALL: every bin edge squared fits 32 bits (bin_lo2 + (nbins + 1) bin_w2 <= 46340), the 32-bit bin test.
template <typename R, bool SMALL>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_estimate_rows(const C2<R>* __restrict__ G1,
                                                                              const C2<R>* __restrict__ G2,
                                                                              const R* __restrict__ tab_g, EstimateArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {
    const int cat = blockIdx.y;
    G1 += cat * a.cat_stride;
    if (G2) G2 += cat * a.cat_stride;
    a.wsums += 3 * cat;
    a.bin_sum += int64_t(cat) * a.nbins;
    a.bin_k += int64_t(cat) * a.nbins;
    a.bin_cnt += int64_t(cat) * a.nbins;
  }
  const int ng = a.ng;
  const int RW = a.rows_per_warp, ncopy = int(blockDim.x >> 5) * RW;  // private bin copies of the block
  R* tab = reinterpret_cast<R*>(smem_raw);  // 1/W, cos, sin (3 ng); 1/W times the norm (ng); V
  PrivBin<R>* pbin = reinterpret_cast<PrivBin<R>*>(smem_raw + estimate_smem_table_bytes(ng, sizeof(R)));
  unsigned* pcnt = reinterpret_cast<unsigned*>(pbin + size_t(ncopy) * a.nbins);
  {
    const R wsum0 = R(a.wsums[0]);
    const R norm0 = a.interlace ? R(0.5) / wsum0 : R(1) / wsum0;
    for (int i = threadIdx.x; i < 3 * ng; i += blockDim.x) tab[i] = tab_g[i];
    for (int i = threadIdx.x; i < ng; i += blockDim.x) tab[3 * ng + i] = tab_g[i] * norm0;
    if (threadIdx.x == 0) tab[4 * ng] = R(a.box * a.box * a.box);
    for (int i = threadIdx.x; i < ncopy * a.nbins; i += blockDim.x) {
      pbin[i].sum = PrivBin<R>::zero();
      pbin[i].k = PrivBin<R>::zero();
      pcnt[i] = 0u;
    }
  }
  __syncthreads();
  const R* winv = tab;
  const R* pc = tab + ng;
  const R* ps = tab + 2 * ng;
  const R* winvz = tab + 3 * ng;
  const R vol = tab[4 * ng];
  const int lane = threadIdx.x & 31;
  const int half = ng / 2, lz = half + 1;
  const int L = 32 / RW, grp = lane / L, sub = lane - grp * L;  // the lane's row of the warp, its place in it
  const int J = (lz + L - 1) / L;
  const int zb = min(sub * J, lz), ze = min(zb + J, lz);  // this lane's slots (none for the last lanes of a row)
  PrivBin<R>* pw = pbin + ((threadIdx.x >> 5) * RW + grp) * a.nbins;
  unsigned* cw = pcnt + ((threadIdx.x >> 5) * RW + grp) * a.nbins;
  const float inv_w2 = 1.0f / float(a.bin_w2);
  const int rows = ng * ng;
  const int nwarps = int((int64_t(gridDim.x) * blockDim.x) >> 5);
  C2<R>* dout = static_cast<C2<R>*>(a.delta_out);
  const C2<R> zero2 = {R(0), R(0)};
  for (int row0 = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * RW; row0 < rows; row0 += nwarps * RW) {
    const int row = min(row0 + grp, rows - 1);
    const int z0 = row0 + grp < rows ? zb : lz, z1 = row0 + grp < rows ? ze : lz;  // rows past the last: no slots
    const int ix = row / ng, iy = row - ix * ng;
    const int nx = signed_mode(ix, ng), ny = signed_mode(iy, ng);
    const R wxy = winv[ix] * winv[iy];
    const C2<R> phx = {pc[ix], ps[ix]}, phy = {pc[iy], ps[iy]};
    const C2<R> phxy = cmul(phx, phy);
    // partner phase per axis: conjugate except on the Nyquist slot
    const C2<R> phxy_p = cmul(ix == half ? phx : conj(phx), iy == half ? phy : conj(phy));
    const int nxy2 = nx * nx + ny * ny;  // |n|^2 <= 3 (N/2)^2 < 2^20
    const bool nyq_row = ix == half || iy == half;  // the partner's phase is not the conjugate there
    const int64_t rbase = int64_t(row) * lz;
    // the next two slots' loads are in flight while a slot is evaluated
    constexpr int PF = 2;
    C2<R> q1[PF], q2[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      q1[u] = zero2;
      q2[u] = zero2;
      if (z0 + u < z1) {
        q1[u] = ld_nc(G1 + rbase + z0 + u);
        if (a.interlace) q2[u] = ld_nc(G2 + rbase + z0 + u);
      }
    }
    Run<R> head = {-2, R(0), R(0), 0}, cur = {-2, R(0), R(0), 0};
    for (int iz = z0; iz < z1; ++iz) {
      const C2<R> g1 = q1[0], g2 = q2[0];
#pragma unroll
      for (int u = 0; u + 1 < PF; ++u) {
        q1[u] = q1[u + 1];
        q2[u] = q2[u + 1];
      }
      if (iz + PF < z1) {
        q1[PF - 1] = ld_nc(G1 + rbase + iz + PF);
        if (a.interlace) q2[PF - 1] = ld_nc(G2 + rbase + iz + PF);
      }
      const int nz = iz == half ? -half : iz;
      const int n2 = nxy2 + nz * nz;
      int b = -1;
      R val = R(0), ks = R(0);
      int cnt = 0;
      C2<R> d = zero2;
      if (n2 != 0) {
        const R c = wxy * winvz[iz];
        const bool partner = iz > 0 && iz < half;
        R vp;  // |delta(-n)|^2
        if (a.interlace) {
          const C2<R> phz = {pc[iz], ps[iz]};
          const C2<R> t = cmul(cmul(phxy, phz), g2);
          d = {(g1.x + t.x) * c, (g1.y + t.y) * c};
          if (nyq_row) {
            const C2<R> tp = cmul(cmul(phxy_p, conj(phz)), conj(g2));
            const C2<R> dp = {(g1.x + tp.x) * c, (-g1.y + tp.y) * c};
            vp = dp.x * dp.x + dp.y * dp.y;
          }
        } else {
          d = {g1.x * c, g1.y * c};
        }
        const R vd = d.x * d.x + d.y * d.y;
        if (!(a.interlace && nyq_row)) vp = vd;  // delta(-n) = conj delta(n) off the Nyquist rows
        // |n| = sqrt(n2): n2 < 2^20 converts exactly through the float 2^23 + n2
        const float rn = sqrtf(__int_as_float(0x4B000000 | n2) - 8388608.0f);
        if constexpr (SMALL)
          b = bin_of32(4 * n2, 2.0f * rn, a.bin_lo2, a.bin_w2, inv_w2, a.nbins);
        else
          b = bin_of(4 * (long long)n2, a.bin_lo2, a.bin_w2, a.nbins);
        if (b >= 0) {
          val = (partner ? vd + vp : vd) * vol;
          cnt = partner ? 2 : 1;
          const R r = sizeof(R) == 4 ? R(rn) : sqrt(R(n2));
          ks = partner ? r + r : r;
        }
      }
      if (dout) dout[rbase + iz] = d;
      if (b == cur.b) {
        cur.v += val;
        cur.k += ks;
        cur.c += cnt;
      } else {
        if (cur.b != -2) {  // the run cur.b ended inside this lane
          if (head.b == -2)
            head = cur;
          else if (cur.b >= 0)
            priv_add(pw, cw, cur.b, cur.v, cur.k, cur.c);
        }
        cur = {b, val, ks, cnt};
      }
    }
    if (a.nbins == 0) continue;
    // the lane's runs at its two ends: one run only (pass) or a head and a tail (cur)
    const bool pass = head.b == -2;
    const int first = pass ? cur.b : head.b;
    const int next_first = __shfl_down_sync(0xffffffffu, first, 1);
    const bool cont = sub < L - 1 && cur.b >= 0 && next_first == cur.b;  // the tail goes on in the next lane
    const bool prev_cont = __shfl_up_sync(0xffffffffu, cont ? 1 : 0, 1) != 0 && sub > 0;
    // segmented inclusive scan of the tails: a segment is a tail and the single-run lanes it goes on through
    const unsigned starts = __ballot_sync(0xffffffffu, sub == 0 || !(prev_cont && pass));
    const int start = 31 - __clz(starts & ((2u << lane) - 1u));
    R sv = cur.v, sk = cur.k;
    int sc = cur.c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const R tv = __shfl_up_sync(0xffffffffu, sv, o);
      const R tk = __shfl_up_sync(0xffffffffu, sk, o);
      const int tc = __shfl_up_sync(0xffffffffu, sc, o);
      if (lane - o >= start) {
        sv += tv;
        sk += tk;
        sc += tc;
      }
    }
    // a head ends the run carried in from the previous lanes
    const R iv = __shfl_up_sync(0xffffffffu, sv, 1), ik = __shfl_up_sync(0xffffffffu, sk, 1);
    const int ic = __shfl_up_sync(0xffffffffu, sc, 1);
    if (!pass && head.b >= 0) {
      if (prev_cont)
        priv_add(pw, cw, head.b, head.v + iv, head.k + ik, head.c + ic);
      else
        priv_add(pw, cw, head.b, head.v, head.k, head.c);
    }
    __syncwarp();
    if (cur.b >= 0 && !cont) priv_add(pw, cw, cur.b, sv, sk, sc);
    __syncwarp();
  }
  __syncthreads();
  if (a.nbins == 0) return;
  for (int i = threadIdx.x; i < a.nbins; i += blockDim.x) {
    // the warps' pairs combined in their own precision, converted to FP64 once
    auto vs = PrivBin<R>::zero(), ks = PrivBin<R>::zero();
    unsigned long long c = 0;
    for (int q = 0; q < ncopy; ++q) {
      const PrivBin<R>& pb = pbin[q * a.nbins + i];
      PrivBin<R>::merge(vs, pb.sum);
      PrivBin<R>::merge(ks, pb.k);
      c += pcnt[q * a.nbins + i];
    }
    if (c) {
      atomicAdd(&a.bin_sum[i], PrivBin<R>::value(vs));
      atomicAdd(&a.bin_k[i], PrivBin<R>::value(ks));
      atomicAdd(&a.bin_cnt[i], c);
    }
  }
}

// Deterministic mode, between the passes: scale_b = 2^F_b with F_b = 62 - ceil(log2(max_b M_b)), so
// that the int64 sum of a bin's quantised values cannot overflow; then clears the sum accumulators.
__global__ void k_det_scale(EstimateArgs a) {
  for (int b = threadIdx.x + blockIdx.x * blockDim.x; b < a.nbins; b += blockDim.x * gridDim.x) {
    const double mx = __longlong_as_double((long long)reinterpret_cast<unsigned long long*>(a.bin_sum)[b]);
    const double m = double(a.bin_cnt[b]);
    int f = 0;
    if (mx > 0.0 && m > 0.0) f = 62 - int(ceil(log2(mx * m)));
    a.det_scale[b] = ldexp(1.0, f);
    a.bin_sum[b] = 0.0;
    a.bin_k[b] = 0.0;
  }
}

template <typename R>
cudaError_t launch_estimate_pass(const void* G1, const void* G2, void* tables, const EstimateArgs& a, cudaStream_t s);

template <typename R>
cudaError_t launch_estimate(const void* G1, const void* G2, void* tables, const EstimateArgs& a, cudaStream_t s) {
  if (a.det_pass == 0 || a.nbins == 0) {
    EstimateArgs b = a;
    b.det_pass = 0;
    return launch_estimate_pass<R>(G1, G2, tables, b, s);
  }
  EstimateArgs b = a;
  b.det_pass = 1;
  cudaError_t e = launch_estimate_pass<R>(G1, G2, tables, b, s);
  if (e != cudaSuccess) return e;
  k_det_scale<<<dim3((a.nbins + 255) / 256, a.ncat), 256, 0, s>>>(b); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  b.det_pass = 2;
  b.delta_out = nullptr;
  return launch_estimate_pass<R>(G1, G2, tables, b, s);
}

template <typename R>
cudaError_t launch_estimate_pass(const void* G1, const void* G2, void* tables, const EstimateArgs& a, cudaStream_t s) {
  k_tables<R><<<(a.ng + 255) / 256, 256, 0, s>>>(static_cast<R*>(tables), a.ng, a.order); count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  EstimateArgs b = a;
  const size_t tab_bytes = estimate_smem_table_bytes(a.ng, sizeof(R));
  const size_t bin_bytes = size_t(a.nbins) * (sizeof(PrivBin<R>) + sizeof(unsigned));
  // The single pass runs by rows (k_estimate_rows) with private bins in at most 96 KB, so that two
  // blocks still fit an SM (N = 1024: 512 bins, eight copies, 80 KB): RW rows per warp, the fewest that leave at most a fifth of the lane slots idle
  // (RW = 1 from N = 256 on), and blocks of 8 warps, else 4 or 2 when the bins are many. The
  // deterministic passes, and bins beyond that room, take k_estimate's 32-slot items with shared
  // atomics.
  int wpb = 0;
  if (a.det_pass == 0) {
    const int lz = a.ng / 2 + 1;
    for (int rw = 1; rw <= 32 && !wpb; rw *= 2) {
      const int L = 32 / rw, J = (lz + L - 1) / L;
      if (rw < 32 && 5 * lz < 4 * L * J) continue;  // more than a fifth of the slots idle
      b.rows_per_warp = rw;
      for (int w = kEstWarps; w >= 2 && !wpb; w /= 2)
        if (size_t(w) * rw * bin_bytes <= 96 * 1024) wpb = w;
    }
  }
  b.priv = wpb ? 1 : 0;
  const int threads = wpb ? 32 * wpb : kEstWarps * 32;
  const size_t smem = tab_bytes + (wpb ? size_t(wpb) * b.rows_per_warp * bin_bytes : size_t(a.nbins) * 24);
  const bool small = int64_t(a.bin_lo2) + int64_t(a.nbins + 1) * a.bin_w2 <= 46340;
  const void* kern = !wpb ? reinterpret_cast<const void*>(k_estimate<R>)
                     : small ? reinterpret_cast<const void*>(k_estimate_rows<R, true>)
                             : reinterpret_cast<const void*>(k_estimate_rows<R, false>);
  if ((e = ensure_dynamic_smem(kern, smem)) != cudaSuccess) return e;
  const int64_t rows = int64_t(a.ng) * a.ng;
  // every block resident at once (the loop is grid-stride; a second partial wave would idle SMs)
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int bx = int(std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, std::max<int64_t>(1, int64_t(num_sms()) * per_sm / a.ncat))));
  const dim3 blocks(bx, a.ncat);
  if (b.priv && small)
    k_estimate_rows<R, true><<<blocks, threads, smem, s>>>(static_cast<const C2<R>*>(G1), static_cast<const C2<R>*>(G2),
                                                           static_cast<const R*>(tables), b);
  else if (b.priv)
    k_estimate_rows<R, false><<<blocks, threads, smem, s>>>(static_cast<const C2<R>*>(G1), static_cast<const C2<R>*>(G2),
                                                            static_cast<const R*>(tables), b);
  else
    k_estimate<R><<<blocks, kEstWarps * 32, smem, s>>>(static_cast<const C2<R>*>(G1), static_cast<const C2<R>*>(G2),
                                                       static_cast<const R*>(tables), b);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_estimate<float>(const void*, const void*, void*, const EstimateArgs&, cudaStream_t);
template cudaError_t launch_estimate<double>(const void*, const void*, void*, const EstimateArgs&, cudaStream_t);

__global__ void k_finalize(EstimateArgs a, int subtract_shot, double* pk, double* kmean, int64_t* nmodes) {
  {
    const int cat = blockIdx.y;
    a.wsums += 3 * cat;
    a.bin_sum += int64_t(cat) * a.nbins;
    a.bin_k += int64_t(cat) * a.nbins;
    a.bin_cnt += int64_t(cat) * a.nbins;
    pk += int64_t(cat) * a.nbins;
    if (kmean) kmean += int64_t(cat) * a.nbins;
    nmodes += int64_t(cat) * a.nbins;
  }
  const double kf = 2.0 * 3.14159265358979323846 / a.box;
  const double vol = a.box * a.box * a.box;
  const double shot = vol * a.wsums[1] / (a.wsums[0] * a.wsums[0]);
  for (int b = threadIdx.x + blockIdx.x * blockDim.x; b < a.nbins; b += blockDim.x * gridDim.x) {
    const unsigned long long m = a.bin_cnt[b];
    nmodes[b] = int64_t(m);
    if (m == 0) {
      pk[b] = __longlong_as_double(0x7ff8000000000000ll);
      if (kmean) kmean[b] = __longlong_as_double(0x7ff8000000000000ll);
    } else {
      double sum = a.bin_sum[b], ksum = a.bin_k[b];
      if (a.det_pass) {  // exact integer sums of the deterministic mode
        sum = double((long long)reinterpret_cast<const unsigned long long*>(a.bin_sum)[b]) / a.det_scale[b];
        ksum = double((long long)reinterpret_cast<const unsigned long long*>(a.bin_k)[b]) / 1048576.0;
      }
      pk[b] = sum / double(m) - (subtract_shot ? shot : 0.0);
      if (kmean) kmean[b] = kf * ksum / double(m);
    }
  }
}

cudaError_t launch_finalize(const EstimateArgs& a, int subtract_shot, double* pk, double* kmean, int64_t* nmodes,
                            cudaStream_t s) {
  k_finalize<<<dim3((a.nbins + 255) / 256, a.ncat), 256, 0, s>>>(a, subtract_shot, pk, kmean, nmodes); count_launch();
  return cudaGetLastError();
}

}  // namespace pk
