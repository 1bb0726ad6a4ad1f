// Direct summation of the Fourier coefficients of a particle set (eq:deltaDS, Sec. 2.2): the
// alias-free, window-free reference against which grid estimators are compared (Sec. 3.2), at cost
// N_P x (number of modes); and the binned cross power of two half-complex fields.
//
// For every stored mode of the half-complex layout [N][N][N/2+1] (signed n as in pk_fft_estimate):
//   delta(n) = (1/sum w) sum_i w_i exp(-2 pi i n.x_i/L),   delta(0) = 0.
// The sum is separable: with rows r = (i_x, i_z) and columns c = i_y,
//   delta[r][c] = sum_i a_i(r) b_i(c),  a_i(r) = w_i e^{-2 pi i (n_x x + n_z z)/L},  b_i(c) = e^{-2 pi i n_y y/L},
// a complex matrix product over the particles. Phases are exact integer products n * Phi of a
// fixed-point position fraction Phi = x/L mod 1 (32 bits in FP32, 64 in FP64) before the sine and
// cosine are taken, so no large argument is ever reduced in floating point.
//   FP32: k_ds_modes_tc, the product on the tensor cores (tcgen05, TF32 operands split in two).
//   FP64: k_ds_modes, FP64 FMAs on the CUDA cores in 256 x 32 mode tiles, each thread a 4 x 8
//         register tile, operands built in shared memory from per-particle, per-axis phase tables.
// Partial sums of particle slices meet in FP64 atomics.
#include "host.cuh"
#include "tc.cuh"

namespace pk {

PK_ERR_ACCESSOR(take_err_direct)

constexpr int kDsRows = 256;  // rows (i_x, i_z) per block
constexpr int kDsCols = 32;   // columns i_y per block
constexpr int kDsThreads = 256;

template <typename R>
struct DsT;
template <>
struct DsT<float> {
  using Phase = uint32_t;
  static constexpr int K = 56;  // particles per chunk
  static constexpr bool kCompensated = true;
  struct Rec {
    uint32_t px, py, pz;
    float w;
  };
  __device__ __forceinline__ static Phase from_frac(double t) { return uint32_t((unsigned long long)rint(t * 4294967296.0)); }
  // e^{-2 pi i T/2^32}
  __device__ __forceinline__ static void expi(Phase t, float w, float& re, float& im) {
    float s, c;
    sincospif(float(int32_t(t)) * 4.656612873077392578125e-10f, &s, &c);  // 2^-31
    re = w * c;
    im = -(w * s);
  }
};
template <>
struct DsT<double> {
  using Phase = uint64_t;
  static constexpr int K = 32;
  static constexpr bool kCompensated = false;
  struct Rec {
    uint64_t px, py, pz;
    double w;
  };
  __device__ __forceinline__ static Phase from_frac(double t) {
    const double th = t * 4294967296.0;
    const double hi = floor(th);
    const double lo = rint((th - hi) * 4294967296.0);
    return ((unsigned long long)hi << 32) + (unsigned long long)lo;
  }
  __device__ __forceinline__ static void expi(Phase t, double w, double& re, double& im) {
    double s, c;
    sincospi(double(int64_t(t)) * 1.0842021724855044340e-19, &s, &c);  // 2^-63
    re = w * c;
    im = -(w * s);
  }
};


// Positions -> fixed-point phase fractions and weights; per-block partial sums of the weights.
template <typename R>
__global__ void __launch_bounds__(256) k_ds_prep(const void* __restrict__ pos, int fmt, const float* __restrict__ w,
                                                 int64_t n, int ng, double box, typename DsT<R>::Rec* __restrict__ out,
                                                 double* __restrict__ wpart) {
  double local = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    double t[3];
    if (fmt == PK_POS_F64_XYZ) {
      const double* p = static_cast<const double*>(pos) + 3 * i;
      bool bad = false;
      for (int a = 0; a < 3; ++a) {
        double x = p[a];
        if (!isfinite(x)) bad = true;
        const double q = x / box;
        t[a] = q - floor(q);
      }
      if (bad) {
        raise_err(PK_DERR_NONFINITE);
        t[0] = t[1] = t[2] = 0.0;
      }
    } else {
      const pk_cellpos r = static_cast<const pk_cellpos*>(pos)[i];
      const int c[3] = {cell_x(r.cell), cell_y(r.cell), cell_z(r.cell)};
      const float f[3] = {r.fx, r.fy, r.fz};
      bool bad = false;
      for (int a = 0; a < 3; ++a) {
        if (c[a] >= ng || !(f[a] >= 0.0f && f[a] < 1.0f)) bad = true;
        t[a] = (double(c[a]) + double(f[a])) / double(ng);
      }
      if (bad) {
        raise_err(PK_DERR_CELLRANGE);
        t[0] = t[1] = t[2] = 0.0;
      }
    }
    const double wi = w ? double(w[i]) : 1.0;
    typename DsT<R>::Rec rec;
    rec.px = DsT<R>::from_frac(t[0]);
    rec.py = DsT<R>::from_frac(t[1]);
    rec.pz = DsT<R>::from_frac(t[2]);
    rec.w = R(wi);
    out[i] = rec;
    local += double(rec.w);
  }
  __shared__ double red[256];
  red[threadIdx.x] = local;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) wpart[blockIdx.x] = red[0];
}

// sum w from the per-block partials, in a fixed order.
__global__ void k_ds_wsum(const double* __restrict__ wpart, int nblk, double* __restrict__ wsum) {
  __shared__ double red[256];
  double v = 0.0;
  for (int i = threadIdx.x; i < nblk; i += 256) v += wpart[i];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *wsum = red[0];
}

template <typename R>
struct DsV2;
template <>
struct DsV2<float> {
  using T = float2;
};
template <>
struct DsV2<double> {
  using T = double2;
};

// Mode tiles. A block owns 256 rows r = (i_x, i_z) x 32 columns i_y of the mode matrix. Rows with
// i_z < N/2 come in rectangles of 8 i_x x 32 i_z, so a row operand is the product of two per-particle
// tables, w e^{-2 pi i n_x x/L} (8 entries) and e^{-2 pi i n_z z/L} (32 entries); the rows of the
// Nyquist plane i_z = N/2 (n_z = -N/2) come 256 i_x at a time and take their operands directly.
constexpr int kDsTx = 8, kDsTz = 32;
__host__ __device__ inline int ds_main_x_tiles(int ng) { return (ng + kDsTx - 1) / kDsTx; }
__host__ __device__ inline int ds_main_z_tiles(int ng) { return (ng / 2 + kDsTz - 1) / kDsTz; }
__host__ __device__ inline int ds_row_tiles(int ng) {
  return ds_main_x_tiles(ng) * ds_main_z_tiles(ng) + (ng + kDsRows - 1) / kDsRows;
}

// Shared-memory order of the operands, chosen so that the 16-byte loads of the register tiles take one
// wavefront: in each 32-row warp block, row 4 rg + q sits at (q/2) 16 + 2 rg + q%2; column 8 cg + j
// at (j/2) 8 + 2 cg + j%2.
__device__ __forceinline__ int ds_row_slot(int l) {
  const int w = l >> 5, rg = (l >> 2) & 7, q = l & 3;
  return 32 * w + (q >> 1) * 16 + 2 * rg + (q & 1);
}
__device__ __forceinline__ int ds_col_slot(int c) {
  const int cg = c >> 3, j = c & 7;
  return (j >> 1) * 8 + 2 * cg + (j & 1);
}

// One block: a row tile x 32 columns of the mode matrix, the particles of one slice. acc_out: FP64 sums
// on the half-complex layout [N][N][N/2+1], added to with atomics. Each thread accumulates a 4 x 8
// register tile of complex sums with four scalar FMAs per product; FP32 adds each chunk's totals to
// TwoSum pairs (hi in registers, lo in shared memory), FP64 accumulates in the registers directly.
template <typename R>
__global__ void __launch_bounds__(kDsThreads, 1) k_ds_modes(const typename DsT<R>::Rec* __restrict__ recs, int64_t n,
                                                             int ng, int64_t slice_len, double2* __restrict__ acc_out) {
  using Rec = typename DsT<R>::Rec;
  using Phase = typename DsT<R>::Phase;
  using V2 = typename DsV2<R>::T;
  constexpr int K = DsT<R>::K;
  constexpr bool kF32 = DsT<R>::kCompensated;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V2* sA = reinterpret_cast<V2*>(smem_raw);  // [K][kDsRows], row slots
  V2* sB = sA + K * kDsRows;                 // [K][kDsCols], column slots
  V2* sEx = sB + K * kDsCols;                // [K][kDsTx]
  V2* sEz = sEx + K * kDsTx;                 // [K][kDsTz]
  float* sLo = reinterpret_cast<float*>(sEz + K * kDsTz);  // FP32: [64][kDsThreads] compensation terms

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int H = ng / 2 + 1;
  const int col0 = blockIdx.y * kDsCols;
  const int64_t k_beg = int64_t(blockIdx.z) * slice_len;
  const int64_t k_end = min(n, k_beg + slice_len);

  // this block's rows: tile origin, and for row l the mode (i_x, i_z) = (ix0 + l / tz, iz0 + l % tz)
  const int tmain = ds_main_x_tiles(ng) * ds_main_z_tiles(ng);
  const bool nyq = int(blockIdx.x) >= tmain;
  int ix0, iz0;
  if (!nyq) {
    ix0 = (int(blockIdx.x) / ds_main_z_tiles(ng)) * kDsTx;
    iz0 = (int(blockIdx.x) % ds_main_z_tiles(ng)) * kDsTz;
  } else {
    ix0 = (int(blockIdx.x) - tmain) * kDsRows;
    iz0 = ng / 2;
  }
  // operand generation: the row of thread tid is l = tid (main: i_x = ix0 + warp, i_z = iz0 + lane)
  const int my_ix = nyq ? ix0 + tid : ix0 + warp;
  const int my_iz = nyq ? iz0 : iz0 + lane;
  const bool row_ok = my_ix < ng && (nyq || my_iz < ng / 2);
  const Phase nx_row = Phase(int64_t(signed_mode(min(my_ix, ng - 1), ng)));
  const Phase nz_nyq = Phase(int64_t(-(ng / 2)));
  const int a_slot = ds_row_slot(tid);
  // table entries of thread tid: Ex[k][x] for x = tid & 7; Ez[k][lane] and B[k][lane] for k = warp + 8 j
  const int tx_ix = ix0 + (tid & 7);
  const Phase nx_tab = Phase(int64_t(signed_mode(min(tx_ix, ng - 1), ng)));
  const bool tx_ok = tx_ix < ng;
  const Phase nz_tab = Phase(int64_t(iz0 + lane));
  const bool tz_ok = iz0 + lane < ng / 2;
  const int gen_col = col0 + lane;
  const bool col_ok = gen_col < ng;
  const Phase ny = Phase(int64_t(signed_mode(min(gen_col, ng - 1), ng)));
  const int b_slot = ds_col_slot(lane);

  // register tile: rows 32 warp + 4 rg + (0..3), columns 8 cg + (0..7)
  const int rg = lane >> 2, cg = lane & 3;
  R acc[64];
  float hi[kF32 ? 64 : 1];
#pragma unroll
  for (int i = 0; i < 64; ++i) acc[i] = R(0);
  if constexpr (kF32) {
#pragma unroll
    for (int i = 0; i < 64; ++i) {
      hi[i] = 0.0f;
      sLo[i * kDsThreads + tid] = 0.0f;
    }
  }

  for (int64_t k0 = k_beg; k0 < k_end; k0 += K) {
    const int cnt = int(min(int64_t(K), k_end - k0));
    __syncthreads();  // the previous chunk's operands are consumed
    // per-particle tables (Ex carries the weight) and the column operands
    for (int e = tid; e < K * kDsTx; e += kDsThreads) {
      const int k = e >> 3;
      R re = R(0), im = R(0);
      if (k < cnt && tx_ok && !nyq) {
        const Rec r = recs[k0 + k];
        DsT<R>::expi(Phase(nx_tab * r.px), r.w, re, im);
      }
      sEx[e] = V2{re, im};
    }
#pragma unroll
    for (int j = 0; j < K / 8; ++j) {
      const int k = warp + 8 * j;
      R bre = R(0), bim = R(0), zre = R(0), zim = R(0);
      if (k < cnt) {
        const Rec r = recs[k0 + k];
        if (col_ok) DsT<R>::expi(Phase(ny * r.py), R(1), bre, bim);
        if (tz_ok && !nyq) DsT<R>::expi(Phase(nz_tab * r.pz), R(1), zre, zim);
      }
      sB[k * kDsCols + b_slot] = V2{bre, bim};
      sEz[k * kDsTz + lane] = V2{zre, zim};
    }
    __syncthreads();
    if (!nyq) {
#pragma unroll 4
      for (int k = 0; k < K; ++k) {
        const V2 x = sEx[k * kDsTx + warp], z = sEz[k * kDsTz + lane];
        V2 a;
        a.x = row_ok ? x.x * z.x - x.y * z.y : R(0);
        a.y = row_ok ? x.x * z.y + x.y * z.x : R(0);
        sA[k * kDsRows + a_slot] = a;
      }
    } else {
#pragma unroll 4
      for (int k = 0; k < K; ++k) {
        R re = R(0), im = R(0);
        if (row_ok && k < cnt) {
          const Rec r = recs[k0 + k];
          DsT<R>::expi(Phase(nx_row * r.px + nz_nyq * r.pz), r.w, re, im);
        }
        sA[k * kDsRows + a_slot] = V2{re, im};
      }
    }
    __syncthreads();
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
      V2 a[4], b[8];
      const V2* pa = sA + k * kDsRows + 32 * warp + 2 * rg;
      const V2* pb = sB + k * kDsCols + 2 * cg;
      a[0] = pa[0];
      a[1] = pa[1];
      a[2] = pa[16];
      a[3] = pa[17];
#pragma unroll
      for (int j2 = 0; j2 < 4; ++j2) {
        b[2 * j2] = pb[8 * j2];
        b[2 * j2 + 1] = pb[8 * j2 + 1];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          R& re = acc[2 * (8 * i + j)];
          R& im = acc[2 * (8 * i + j) + 1];
          re = fma(a[i].x, b[j].x, re);
          re = fma(-a[i].y, b[j].y, re);
          im = fma(a[i].x, b[j].y, im);
          im = fma(a[i].y, b[j].x, im);
        }
      }
    }
    if constexpr (kF32) {  // TwoSum of the chunk totals into (hi, lo)
#pragma unroll
      for (int i = 0; i < 64; ++i) {
        const float v = acc[i];
        const float sum = __fadd_rn(hi[i], v);
        const float bb = __fsub_rn(sum, hi[i]);
        const float err = __fadd_rn(__fsub_rn(hi[i], __fsub_rn(sum, bb)), __fsub_rn(v, bb));
        sLo[i * kDsThreads + tid] = __fadd_rn(sLo[i * kDsThreads + tid], err);
        hi[i] = sum;
        acc[i] = 0.0f;
      }
    }
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int l = 32 * warp + 4 * rg + i;
    const int ix = nyq ? ix0 + l : ix0 + (l >> 5);
    const int iz = nyq ? iz0 : iz0 + (l & 31);
    if (ix >= ng || (!nyq && iz >= ng / 2)) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = col0 + 8 * cg + j;
      if (c >= ng) continue;
      double2* dst = acc_out + (int64_t(ix) * ng + c) * H + iz;
      const int q = 2 * (8 * i + j);
      if constexpr (kF32) {
        atomicAdd(&dst->x, double(hi[q]) + double(sLo[q * kDsThreads + tid]));
        atomicAdd(&dst->y, double(hi[q + 1]) + double(sLo[(q + 1) * kDsThreads + tid]));
      } else {
        atomicAdd(&dst->x, double(acc[q]));
        atomicAdd(&dst->y, double(acc[q + 1]));
      }
    }
  }
}

// delta = sums / sum w in the output precision; delta(0) = 0.
template <typename V>
__global__ void k_ds_finish(const double2* __restrict__ sums, const double* __restrict__ wsum, int64_t count,
                            V* __restrict__ out) {
  const double inv = 1.0 / *wsum;
  for (int64_t m = gtid(); m < count; m += gstride()) {
    const double2 v = sums[m];
    V o;
    o.x = m == 0 ? 0.0 : v.x * inv;
    o.y = m == 0 ? 0.0 : v.y * inv;
    out[m] = o;
  }
}

// Binned V Re[a(n) conj b(n)] over the stored modes, each with its multiplicity (2 for
// 0 < i_z < N/2, where the unstored partner -n adds the conjugate product; 1 on the i_z = 0 and
// i_z = N/2 planes); sums of the multiplicity and of multiplicity x |n| for the counts and mean |k|.
template <typename V>
__global__ void __launch_bounds__(256) k_cross_bins(const V* __restrict__ da, const V* __restrict__ db, int ng,
                                                    double vol, int lo2, int w2, int nbins, double* __restrict__ bin_sum,
                                                    double* __restrict__ bin_k, unsigned long long* __restrict__ bin_cnt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* s_sum = reinterpret_cast<double*>(smem_raw);
  double* s_k = s_sum + nbins;
  unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(s_k + nbins);
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
    s_sum[i] = 0.0;
    s_k[i] = 0.0;
    s_cnt[i] = 0ull;
  }
  __syncthreads();
  const int H = ng / 2 + 1;
  const int64_t count = int64_t(ng) * ng * H;
  for (int64_t m = gtid(); m < count; m += gstride()) {
    const int iz = int(m % H);
    const int64_t xy = m / H;
    const int iy = int(xy % ng), ix = int(xy / ng);
    const long long nx = signed_mode(ix, ng), ny = signed_mode(iy, ng);
    const long long nz = iz == ng / 2 ? -(ng / 2) : iz;
    const long long n2 = nx * nx + ny * ny + nz * nz;
    const int b = bin_of(4 * n2, lo2, w2, nbins);
    if (b < 0) continue;
    const int mult = (iz == 0 || iz == ng / 2) ? 1 : 2;
    const V a = da[m], c = db[m];
    const double re = double(a.x) * double(c.x) + double(a.y) * double(c.y);
    atomicAdd(&s_sum[b], double(mult) * vol * re);
    atomicAdd(&s_k[b], double(mult) * sqrt(double(n2)));
    atomicAdd(&s_cnt[b], (unsigned long long)mult);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
    if (s_cnt[i] == 0ull) continue;
    atomicAdd(&bin_sum[i], s_sum[i]);
    atomicAdd(&bin_k[i], s_k[i]);
    atomicAdd(&bin_cnt[i], s_cnt[i]);
  }
}

// ---- FP32 on the tensor cores (tcgen05, kind::tf32) -----------------------------------------------------
//
// The same product as a real matrix product D = A B per block: M = 128 rows (i_x, i_z), N = 64 real
// columns (the real parts of 32 complex columns i_y, then their imaginary parts), K = 2 per particle:
//   A[r][2k] = Re a_k(r), A[r][2k+1] = Im a_k(r),
//   B[c][2k] = Re b_k(c), B[c][2k+1] = -Im b_k(c)   (c < 32: real part of column c),
//   B[32+c][2k] = Im b_k(c), B[32+c][2k+1] = Re b_k(c) (imaginary part).
// TF32 keeps 10 mantissa bits, so each operand x is split into big = x rounded to TF32 and small =
// x - big (exact in FP32), and D accumulates big.big + big.small + small.big (three MMAs per k-step):
// each product then errs by about 2^-21 of its size.
//
// Pipeline, per chunk c of 32 particles: the operands go to stage c % 2 of shared memory and the
// chunk's MMAs (one issuing thread) to accumulator (c / 2) % 2 in TMEM (128 lanes x 64 FP32 columns,
// restarted every second chunk, so each total covers 64 particles), completion signalled on mbarrier
// c % 2 by tcgen05.commit. While they run, the block (16 warps) reads the accumulator of the previous
// pair (warp w: lanes 32 (w % 4).., columns 16 (w / 4)..) into TwoSum pairs in registers, then builds
// the next chunk's operands. Operands are K-major without
// swizzle: 8-row x 16-byte core matrices, K-adjacent cores 128 B apart (LBO), 8-row groups 2048 B
// apart (SBO). Every mbarrier wait is bounded in time.
constexpr int kTcRows = 128, kTcCols = 32, kTcK = 32, kTcThreads = 512;
constexpr int kTcTx = 8, kTcTz = 16;  // main row tiles: 8 i_x x 16 i_z
constexpr int kTcKr = 2 * kTcK;       // real K per chunk
constexpr uint32_t kTcTmemCols = 128; // two accumulators of 64 columns
constexpr uint64_t kTcWaitNs = 1000000000ull;  // bound of every mbarrier wait
constexpr uint32_t kTcSbo = (kTcKr / 4) * 128;   // 8-row groups of an operand
constexpr uint32_t kTcIdesc = tc::idesc_tf32(64, 128);

__host__ __device__ inline int tc_main_x_tiles(int ng) { return (ng + kTcTx - 1) / kTcTx; }
__host__ __device__ inline int tc_main_z_tiles(int ng) { return (ng / 2 + kTcTz - 1) / kTcTz; }
__host__ __device__ inline int tc_row_tiles(int ng) { return tc_main_x_tiles(ng) * tc_main_z_tiles(ng) + (ng + kTcRows - 1) / kTcRows; }

struct TcSmem {  // byte offsets in the dynamic shared memory (base aligned to 128)
  static constexpr uint32_t a_part = kTcRows * kTcKr * 4, b_part = 2 * kTcCols * kTcKr * 4;
  static constexpr uint32_t stage = 2 * a_part + 2 * b_part;  // A big, A small, B big, B small
  static constexpr uint32_t rec = 2 * stage, bar = rec + kTcK * 16, tmem = bar + 16, total = tmem + 16;
};

// w e^{-2 pi i T / 2^32}: the phase T (a fraction of a turn, exact in integers) becomes an angle in
// [-pi, pi) and the hardware sine and cosine (__sincosf, absolute error about 2^-21.4 there) take it.
__device__ __forceinline__ void tc_expi(uint32_t t, float w, float& re, float& im) {
  float s, c;
  __sincosf(float(int32_t(t)) * 1.46291807926715968e-9f, &s, &c);  // pi / 2^31
  re = w * c;
  im = -(w * s);
}

__global__ void __launch_bounds__(kTcThreads, 1) k_ds_modes_tc(const DsT<float>::Rec* __restrict__ recs, int64_t n, int ng,
                                                               int64_t slice_len, double2* __restrict__ acc_out) {
  using Rec = DsT<float>::Rec;
  extern __shared__ __align__(128) unsigned char smem_tc[];
  unsigned char* sm = smem_tc;
  const uint32_t sbase = uint32_t(__cvta_generic_to_shared(sm));
  Rec* sRec = reinterpret_cast<Rec*>(sm + TcSmem::rec);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + TcSmem::tmem);
  volatile int* s_bad = reinterpret_cast<volatile int*>(sm + TcSmem::tmem + 4);  // a wait ran out

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int H = ng / 2 + 1;
  const int col0 = blockIdx.y * kTcCols;
  const int64_t k_beg = int64_t(blockIdx.z) * slice_len;
  const int64_t k_end = min(n, k_beg + slice_len);
  const int nchunks = k_end > k_beg ? int((k_end - k_beg + kTcK - 1) / kTcK) : 0;
  const int tmain = tc_main_x_tiles(ng) * tc_main_z_tiles(ng);
  const bool nyq = int(blockIdx.x) >= tmain;
  int ix0, iz0;
  if (!nyq) {
    ix0 = (int(blockIdx.x) / tc_main_z_tiles(ng)) * kTcTx;
    iz0 = (int(blockIdx.x) % tc_main_z_tiles(ng)) * kTcTz;
  } else {
    ix0 = (int(blockIdx.x) - tmain) * kTcRows;
    iz0 = ng / 2;
  }

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sbase + TcSmem::tmem),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    *s_bad = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbase + TcSmem::bar) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbase + TcSmem::bar + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // operand roles, chosen so that a warp's 8-byte stores cover 8 rows x 4 consecutive particles (two
  // core matrices, 256 contiguous bytes): A row 8 warp + lane % 8, particles lane / 8 + 4 j (j < 8);
  // B row 8 (warp % 8) + lane % 8, particles lane / 8 + 4 j + 16 (warp / 8) (j < 4)
  const int ar = 8 * warp + (lane & 7), ak0 = lane >> 3;
  const int a_ix = nyq ? ix0 + ar : ix0 + (ar >> 4), a_iz = nyq ? iz0 : iz0 + (ar & 15);
  const bool a_ok = a_ix < ng && (nyq || a_iz < ng / 2);
  const uint32_t nx_row = uint32_t(int64_t(signed_mode(min(a_ix, ng - 1), ng)));
  const uint32_t nz_row = uint32_t(int64_t(nyq ? -(ng / 2) : a_iz));
  const int br = 8 * (warp & 7) + (lane & 7), bk0 = (lane >> 3) + 16 * (warp >> 3), bc = br & 31;
  const bool b_ok = col0 + bc < ng;
  const uint32_t ny = uint32_t(int64_t(signed_mode(min(col0 + bc, ng - 1), ng)));
  // epilogue: TMEM lanes 32 (warp % 4) + lane, columns 16 (warp / 4) .. + 15 of the accumulator
  const int er = 32 * (warp & 3) + lane, ecol = 16 * (warp >> 2);
  const uint32_t tlane = uint32_t(32 * (warp & 3)) << 16;
  float hi[16], lo[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) hi[j] = lo[j] = 0.0f;
  bool timed_out = false;
  uint32_t phase0 = 0u, phase1 = 0u;  // parity to wait for on mbarrier 0 / 1
  Rec next_rec;  // threads < kTcK: the record of the next chunk (zero weight past the slice)
  next_rec.px = next_rec.py = next_rec.pz = 0u;
  next_rec.w = 0.0f;
  if (tid < kTcK && k_beg + tid < k_end) next_rec = recs[k_beg + tid];
  int outstanding = -1;  // chunk whose MMAs may still be in flight

  for (int c = 0; c <= nchunks; ++c) {
    if (c < nchunks) {
      const int64_t k0 = k_beg + int64_t(c) * kTcK;
      const int st = c & 1;
      if (tid < kTcK) {  // this chunk's record (loaded one chunk ahead), then the next one's load
        sRec[tid] = next_rec;
        const int64_t kn = k0 + kTcK + tid;
        if (kn < k_end) {
          next_rec = recs[kn];
        } else {
          next_rec.px = next_rec.py = next_rec.pz = 0u;
          next_rec.w = 0.0f;
        }
      }
      __syncthreads();
      if (*s_bad) break;  // a wait of the previous chunk ran out (one value for the whole block here)
      unsigned char* stg = sm + st * TcSmem::stage;
#pragma unroll
      for (int kk = 0; kk < kTcK / 4; ++kk) {  // A: row ar, particles ak0 + 4 kk: w e^{-2 pi i (n_x x + n_z z)/L}
        const int k = ak0 + 4 * kk;
        const Rec r = sRec[k];
        float re = 0.0f, im = 0.0f;
        if (a_ok) tc_expi(nx_row * r.px + nz_row * r.pz, r.w, re, im);
        float2 big, small;
        tc::split(re, big.x, small.x);
        tc::split(im, big.y, small.y);
        const uint32_t off = tc::off(ar, 2 * k, kTcKr);
        *reinterpret_cast<float2*>(stg + off) = big;
        *reinterpret_cast<float2*>(stg + TcSmem::a_part + off) = small;
      }
#pragma unroll
      for (int kk = 0; kk < kTcK / 8; ++kk) {  // B: row br, particles bk0 + 4 kk: e^{-2 pi i n_y y/L}
        const int k = bk0 + 4 * kk;
        float yr = 0.0f, yi = 0.0f;
        if (b_ok) tc_expi(ny * sRec[k].py, 1.0f, yr, yi);
        const float v0 = br < 32 ? yr : yi, v1 = br < 32 ? -yi : yr;
        float2 big, small;
        tc::split(v0, big.x, small.x);
        tc::split(v1, big.y, small.y);
        const uint32_t off = tc::off(br, 2 * k, kTcKr);
        *reinterpret_cast<float2*>(stg + 2 * TcSmem::a_part + off) = big;
        *reinterpret_cast<float2*>(stg + 2 * TcSmem::a_part + TcSmem::b_part + off) = small;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = sbase + st * TcSmem::stage, sb = sa + 2 * TcSmem::a_part;
        const uint32_t d = tmem + uint32_t(64 * ((c >> 1) & 1));  // chunks 2p, 2p + 1 share accumulator p % 2
        // a k-step advances each operand by two core matrices (256 B): 16 in the address field
        const uint64_t ab0 = tc::desc(sa, kTcSbo), as0 = tc::desc(sa + TcSmem::a_part, kTcSbo);
        const uint64_t bb0 = tc::desc(sb, kTcSbo), bs0 = tc::desc(sb + TcSmem::b_part, kTcSbo);
#pragma unroll
        for (int ks = 0; ks < kTcKr / 8; ++ks) {
          const uint64_t ab = ab0 + 16u * ks, as = as0 + 16u * ks, bb = bb0 + 16u * ks, bs = bs0 + 16u * ks;
          const uint32_t acc0 = (ks > 0 || (c & 1)) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
              "l"(ab), "l"(bb), "r"(kTcIdesc), "r"(acc0)
              : "memory");
          asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(d), "l"(ab), "l"(bs), "r"(kTcIdesc)
                       : "memory");
          asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(d), "l"(as), "l"(bb), "r"(kTcIdesc)
                       : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         sbase + TcSmem::bar + 8 * st)
                     : "memory");
      }
      outstanding = c;
    }
    if (c >= 1) {  // the previous chunk's MMAs; after the second chunk of a pair (or the last), its accumulator
      const int pb = (c - 1) & 1;
      // no block barrier here (the MMA-issuing thread would hold every warp): each warp decides alone,
      // and a timeout reaches the whole block through s_bad at the next chunk's first barrier
      const bool ok = __all_sync(0xffffffffu, tc::wait(sbase + TcSmem::bar + 8 * pb, pb ? phase1 : phase0, kTcWaitNs));
      if (ok) {
        if (pb) phase1 ^= 1u; else phase0 ^= 1u;
        if (outstanding == c - 1) outstanding = -1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (((c - 1) & 1) || c == nchunks) tc::read_acc16(tmem + tlane + uint32_t(64 * (((c - 1) >> 1) & 1) + ecol), hi, lo);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      } else if (lane == 0) {
        *s_bad = 1;
      }
    }
  }
  __syncthreads();
  timed_out = *s_bad != 0;
  if (timed_out && tid == 0) raise_err(PK_DERR_TIMEOUT);

  if (!timed_out) {  // this thread's accumulator lane is row (i_x, i_z); its 16 columns are real or imaginary parts
    const int ix = nyq ? ix0 + er : ix0 + (er >> 4), iz = nyq ? iz0 : iz0 + (er & 15);
    if (ix < ng && (nyq || iz < ng / 2)) {
#pragma unroll 4
      for (int j = 0; j < 16; ++j) {
        const int col = col0 + (ecol & 31) + j;
        if (col >= ng) break;
        double2* dst = acc_out + (int64_t(ix) * ng + col) * H + iz;
        atomicAdd(ecol < 32 ? &dst->x : &dst->y, double(hi[j]) + double(lo[j]));
      }
    }
  } else {  // give the MMAs still in flight a bounded wait before the TMEM is freed
    if (outstanding >= 0) tc::wait(sbase + TcSmem::bar + 8 * (outstanding & 1), (outstanding & 1) ? phase1 : phase0, kTcWaitNs);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
  }
}

// ---- host side --------------------------------------------------------------------------------------------

namespace {

constexpr int kPrepBlocks = 1024;

struct DsLayout {
  void* recs = nullptr;
  double* wpart = nullptr;
  double* wsum = nullptr;
  double2* sums = nullptr;
};

void carve_ds(const pk_config* c, int64_t n, Carver& cv, DsLayout* L) {
  const size_t rec = c->prec == PK_FP32 ? sizeof(DsT<float>::Rec) : sizeof(DsT<double>::Rec);
  L->recs = cv.take<char>(rec * size_t(std::max<int64_t>(n, 1)));
  L->wpart = cv.take<double>(kPrepBlocks);
  L->wsum = cv.take<double>(1);
  L->sums = cv.take<double2>(size_t(half_count(c->ng)));
}

struct CrossLayout {
  double* bin_sum = nullptr;
  double* bin_k = nullptr;
  unsigned long long* bin_cnt = nullptr;
  double* wsums = nullptr;
};

void carve_cross(const pk_config* c, Carver& cv, CrossLayout* L) {
  L->bin_sum = cv.take<double>(c->nbins);
  L->bin_k = cv.take<double>(c->nbins);
  L->bin_cnt = cv.take<unsigned long long>(c->nbins);
  L->wsums = cv.take<double>(3);
}

// Particle slices per column of mode tiles: enough blocks for whole waves of one block per SM.
int ds_slices(int64_t tiles, int64_t n, int K) {
  const int64_t sms = num_sms();
  const int64_t chunks = (n + K - 1) / K;
  int best = 1;
  double best_eff = 0.0;
  for (int s = 1; s <= 64 && s <= chunks; ++s) {
    const int64_t blocks = tiles * s;
    const int64_t waves = (blocks + sms - 1) / sms;
    // particles per slice rounded up to whole chunks: the longest slice sets the time
    const double eff = double(blocks) / double(waves * sms);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = s;
    }
    if (blocks >= 4 * sms) break;
  }
  return best;
}

template <typename R>
pk_status run_direct(const pk_config* c, const void* pos, int fmt, const float* w, int64_t n, void* delta_out, DsLayout& L,
                     cudaStream_t s) {
  using Rec = typename DsT<R>::Rec;
  constexpr int K = DsT<R>::K;
  const int ng = c->ng;
  cudaError_t e;
  const int prep_blocks = int(std::min<int64_t>(kPrepBlocks, std::max<int64_t>(1, (n + 255) / 256)));
  k_ds_prep<R><<<prep_blocks, 256, 0, s>>>(pos, fmt, w, n, ng, c->box, static_cast<Rec*>(L.recs), L.wpart); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "direct prep");
  k_ds_wsum<<<1, 256, 0, s>>>(L.wpart, prep_blocks, L.wsum); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "direct wsum");
  const int64_t hc = half_count(ng);
  if ((e = cudaMemsetAsync(L.sums, 0, sizeof(double2) * size_t(hc), s)) != cudaSuccess) return cuda_fail(e, "memset");
  if constexpr (DsT<R>::kCompensated) {  // FP32: the tensor-core kernel
    const int64_t row_tiles = tc_row_tiles(ng);
    const int col_tiles = (ng + kTcCols - 1) / kTcCols;
    const int slices = ds_slices(row_tiles * col_tiles, n, kTcK);
    const int64_t chunks = (n + kTcK - 1) / kTcK;
    const int64_t slice_len = ((chunks + slices - 1) / slices) * kTcK;
    const size_t smem = TcSmem::total;
    if ((e = ensure_dynamic_smem(reinterpret_cast<const void*>(k_ds_modes_tc), smem)) != cudaSuccess)
      return cuda_fail(e, "direct smem");
    if (row_tiles > 2147483647) return fail(PK_EINVAL, "too many rows");
    k_ds_modes_tc<<<dim3(unsigned(row_tiles), col_tiles, slices), kTcThreads, smem, s>>>(
        reinterpret_cast<const DsT<float>::Rec*>(L.recs), n, ng, slice_len, L.sums);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "direct modes");
    const int fblocks = int(std::min<int64_t>(int64_t(num_sms()) * 8, (hc + 255) / 256));
    k_ds_finish<float2><<<fblocks, 256, 0, s>>>(L.sums, L.wsum, hc, static_cast<float2*>(delta_out));
    count_launch();
    e = cudaGetLastError();
    return e == cudaSuccess ? PK_OK : cuda_fail(e, "direct finish");
  } else {  // FP64: the CUDA-core kernel
  const int64_t row_tiles = ds_row_tiles(ng);
  const int col_tiles = (ng + kDsCols - 1) / kDsCols;
  const int slices = ds_slices(row_tiles * col_tiles, n, K);
  const int64_t chunks = (n + K - 1) / K;
  const int64_t slice_len = ((chunks + slices - 1) / slices) * K;
  const size_t smem = sizeof(typename DsV2<R>::T) * size_t(K) * (kDsRows + kDsCols + kDsTx + kDsTz) +
                      (DsT<R>::kCompensated ? sizeof(float) * 64 * kDsThreads : 0);
  if ((e = ensure_dynamic_smem(reinterpret_cast<const void*>(k_ds_modes<R>), smem)) != cudaSuccess)
    return cuda_fail(e, "direct smem");
  if (row_tiles > 2147483647) return fail(PK_EINVAL, "too many rows");
  k_ds_modes<R><<<dim3(unsigned(row_tiles), col_tiles, slices), kDsThreads, smem, s>>>(static_cast<const Rec*>(L.recs), n, ng,
                                                                                    slice_len, L.sums); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "direct modes");
  const int fblocks = int(std::min<int64_t>(int64_t(num_sms()) * 8, (hc + 255) / 256));
  k_ds_finish<double2><<<fblocks, 256, 0, s>>>(L.sums, L.wsum, hc, static_cast<double2*>(delta_out));
  count_launch();
  e = cudaGetLastError();
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "direct finish");
  }
}

}  // namespace

pk_status direct_ws(const pk_config* c, int64_t n, bool cross, size_t* out) {
  Carver cv(nullptr);
  if (cross) {
    CrossLayout L;
    carve_cross(c, cv, &L);
  } else {
    DsLayout L;
    carve_ds(c, n, cv, &L);
  }
  *out = cv.size();
  return PK_OK;
}

}  // namespace pk

using namespace pk;

extern "C" {

pk_status pk_direct_modes(const pk_config* cfg, const void* pos_dev, int32_t pos_format, const float* w_dev, int64_t n,
                          void* delta_k_dev, void* ws, size_t ws_bytes, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (pos_format != PK_POS_F64_XYZ && pos_format != PK_POS_CELL_F32OFF) return fail(PK_EINVAL, "bad pos_format");
  if (n < 1 || !pos_dev) return fail(PK_EINVAL, "need at least one particle");
  if (!delta_k_dev) return fail(PK_EINVAL, "delta_k_dev is NULL");
  const size_t need = pk_workspace_size(cfg, n, PK_WS_DIRECT);
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  DsLayout L;
  carve_ds(cfg, n, cv, &L);
  return cfg->prec == PK_FP32 ? run_direct<float>(cfg, pos_dev, pos_format, w_dev, n, delta_k_dev, L, s)
                              : run_direct<double>(cfg, pos_dev, pos_format, w_dev, n, delta_k_dev, L, s);
}

pk_status pk_cross_power(const pk_config* cfg, const void* delta_a_dev, const void* delta_b_dev, double* pk_dev,
                         double* kmean_dev, int64_t* nmodes_dev, void* ws, size_t ws_bytes, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (!delta_a_dev || !delta_b_dev || !pk_dev || !nmodes_dev) return fail(PK_EINVAL, "bad pointers");
  const size_t need = pk_workspace_size(cfg, 0, PK_WS_CROSS);
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  CrossLayout L;
  carve_cross(cfg, cv, &L);
  cudaError_t e;
  const size_t nb = size_t(cfg->nbins);
  if ((e = cudaMemsetAsync(L.bin_sum, 0, sizeof(double) * nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(L.bin_k, 0, sizeof(double) * nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(L.bin_cnt, 0, sizeof(unsigned long long) * nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(L.wsums, 0, sizeof(double) * 3, s)) != cudaSuccess)
    return cuda_fail(e, "memset");
  const int ng = cfg->ng;
  const double vol = cfg->box * cfg->box * cfg->box;
  const int64_t hc = half_count(ng);
  const int blocks = int(std::min<int64_t>(int64_t(num_sms()) * 4, (hc + 255) / 256));
  const size_t smem = nb * (2 * sizeof(double) + sizeof(unsigned long long));
  if (cfg->prec == PK_FP32) {
    if ((e = ensure_dynamic_smem(reinterpret_cast<const void*>(k_cross_bins<float2>), smem)) != cudaSuccess)
      return cuda_fail(e, "cross smem");
    k_cross_bins<float2><<<blocks, 256, smem, s>>>(static_cast<const float2*>(delta_a_dev),
                                                   static_cast<const float2*>(delta_b_dev), ng, vol, cfg->bin_lo2,
                                                   cfg->bin_w2, cfg->nbins, L.bin_sum, L.bin_k, L.bin_cnt);
  } else {
    if ((e = ensure_dynamic_smem(reinterpret_cast<const void*>(k_cross_bins<double2>), smem)) != cudaSuccess)
      return cuda_fail(e, "cross smem");
    k_cross_bins<double2><<<blocks, 256, smem, s>>>(static_cast<const double2*>(delta_a_dev),
                                                    static_cast<const double2*>(delta_b_dev), ng, vol, cfg->bin_lo2,
                                                    cfg->bin_w2, cfg->nbins, L.bin_sum, L.bin_k, L.bin_cnt);
  }
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "cross bins");
  EstimateArgs a{};
  a.ng = ng;
  a.nbins = cfg->nbins;
  a.bin_lo2 = cfg->bin_lo2;
  a.bin_w2 = cfg->bin_w2;
  a.box = cfg->box;
  a.wsums = L.wsums;  // zeros: no shot noise is subtracted
  a.bin_sum = L.bin_sum;
  a.bin_k = L.bin_k;
  a.bin_cnt = L.bin_cnt;
  if ((e = launch_finalize(a, 0, pk_dev, kmean_dev, nmodes_dev, s)) != cudaSuccess) return cuda_fail(e, "finalize");
  return PK_OK;
}

}  // extern "C"
