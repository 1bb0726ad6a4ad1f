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
#include <utility>
#include <vector>

#include "host.cuh"

namespace pk {

// The grid of the triple sums: the shells reach |n_i| <= k - 1 with k = lo + nshells w, so the product
// of three shell fields holds wavevectors with components up to 3 (k - 1) and sums over any grid of
// M > 3 (k - 1) points per side without aliasing: S_M / M^3 = S_N / N^3 = sum over closed triangles
// of delta delta delta. The smallest even M with prime factors 2, 3, 5, 7 (and at most N) is taken;
// 16 shells of 4 k_f need M = 192 instead of N = 256 (2.4 times fewer points to transform and sum).
static int bisp_grid(int ng, int lo, int w, int nshells) {
  const int64_t need = 3 * (int64_t(lo) + int64_t(nshells) * w - 1) + 1;
  for (int64_t m = std::max<int64_t>(8, need + (need & 1)); m < ng; m += 2) {
    int64_t r = m;
    for (int f : {2, 3, 5, 7})
      while (r % f == 0) r /= f;
    if (r == 1) return int(m);
  }
  return ng;
}

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

// Writes the shell-filtered copies of delta (R2 = float2/double2; half-complex on the N grid) into the
// nshells complex buffers of the bispectrum grid M <= N: slot (i_x, i_y, i_z) of M takes the mode
// n = (signed i_x, signed i_y, i_z) of delta when n lies in a shell (every shell mode has |n_i| < M/2).
template <typename R2>
__global__ void k_shell_filter(const R2* __restrict__ delta, R2* __restrict__ out, int ng, int mg, int lo, int w, int nshells,
                               int64_t buf_stride) {
  const int64_t nh = int64_t(mg) * mg * (mg / 2 + 1);
  const int lzm = mg / 2 + 1, lzn = ng / 2 + 1;
  for (int64_t i = gtid(); i < nh; i += gstride()) {
    int iz;
    const int s = shell_of(mode_n2(i, mg, &iz), lo, w, nshells);
    R2 d;
    d.x = 0;
    d.y = 0;
    if (s >= 0) {
      const int64_t row = i / lzm;
      const int iy = int(row % mg), ix = int(row / mg);
      const int sx = signed_mode(ix, mg), sy = signed_mode(iy, mg);
      const int jx = sx < 0 ? sx + ng : sx, jy = sy < 0 ? sy + ng : sy;
      d = delta[(int64_t(jx) * ng + jy) * lzn + iz];
    }
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

// The FP32 triple product for up to kRegShells shells with the triangles in registers. The triangle
// list of kRegShells shells is fixed at compile time (kTri, the order of make_triangles; the list of
// fewer shells is its first ntri entries), warp w of a block owns its triangles w kRegWarpTri ..
// (w + 1) kRegWarpTri - 1, and the code of each warp is instantiated for its own triangles, so that the
// shell indices are constants and the values of a point live in registers. Lane l takes the points l,
// l + 32, l + 64, l + 96 of each staged tile and, per point, reads each shell its triangles use once from
// shared memory (about 104 reads per point over the 8 warps, against one or more per triangle in
// k_triple_warp), forms I_a I_b once per shell pair and adds I_a I_b I_c to the triangle's running sum.
// Every kFlushTiles tiles the lane sums are added across the warp by a transposing butterfly (five
// exchange steps leave lane l with the sums of the warp's triangles 2 l and 2 l + 1) and added to the
// block's compensated FP32 pair of those triangles, as in k_triple_warp.
constexpr int kRegShells = 16;
constexpr int kRegWarpTri = 64;
constexpr int kRegWarps = 8;
constexpr int kRegTri = kRegWarps * kRegWarpTri;

struct TriTable {
  int n = 0;
  int a[kRegTri] = {};
  int b[kRegTri] = {};
  int c[kRegTri] = {};
  constexpr TriTable() {
    for (int x = 0; x < kRegShells; ++x)
      for (int y = 0; y <= x; ++y)
        for (int z = 0; z <= y; ++z)
          if (x <= y + z + 1) {
            a[n] = x;
            b[n] = y;
            c[n] = z;
            ++n;
          }
  }
};
constexpr TriTable kTri{};
static_assert(kTri.n <= kRegTri, "the triangles of kRegShells shells must fit the warps' registers");

template <int W, int J>
__device__ __forceinline__ void reg_tri(const float (&v)[kRegShells], float& pab, float (&acc)[kRegWarpTri]) {
  constexpr int t = W * kRegWarpTri + J;
  if constexpr (t < kTri.n) {
    constexpr int a = kTri.a[t], b = kTri.b[t], c = kTri.c[t];
    if constexpr (J == 0 || a != kTri.a[t - 1] || b != kTri.b[t - 1]) pab = v[a] * v[b];
    acc[J] = fmaf(pab, v[c], acc[J]);
  }
}

template <int W, int... J>
__device__ __forceinline__ void reg_tris(const float (&v)[kRegShells], float& pab, float (&acc)[kRegWarpTri],
                                         std::integer_sequence<int, J...>) {
  (reg_tri<W, J>(v, pab, acc), ...);
}

// The four points of lane l in the staged tile: col = vals + l, shell s of point l + 32 i at
// col[s kRow + 32 i]. Reads of shells that warp W's triangles do not use are dead and dropped.
template <int W>
__device__ __forceinline__ void reg_tile(const float* col, float (&acc)[kRegWarpTri]) {
#pragma unroll 1
  for (int i = 0; i < kTX / 32; ++i) {
    float v[kRegShells];
#pragma unroll
    for (int s = 0; s < kRegShells; ++s) v[s] = col[s * kRow + 32 * i];
    float pab = 0.f;
    reg_tris<W>(v, pab, acc, std::make_integer_sequence<int, kRegWarpTri>{});
  }
}

// One exchange step of the transposing butterfly over n running sums: the lane with bit o clear keeps
// the first half (adding its partner's first half), the other the second half.
template <int N>
__device__ __forceinline__ void fold_half(float (&acc)[kRegWarpTri], int lane, int o) {
  const bool up = (lane & o) != 0;
#pragma unroll
  for (int j = 0; j < N / 2; ++j) {
    const float lo = acc[j], hi = acc[j + N / 2];
    const float send = up ? lo : hi;
    const float keep = up ? hi : lo;
    acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
  }
}

// cp.async groups: the 4-byte copies of a tile are one group (a copy of 0 source bytes writes a zero).
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__global__ void __launch_bounds__(kRegWarps * 32, 2) k_triple_reg(const float* __restrict__ fields, int ng, int nshells,
                                                                  int64_t buf_stride, int ntri, double* __restrict__ S) {
  static_assert(kRegWarps * 32 == 2 * kTX, "two threads per staged point");
  __shared__ float shi[kRegTri], slo[kRegTri];
  __shared__ __align__(16) float vals[2][kRegShells * kRow];  // tile i in vals[i & 1], tile i + 1 arriving in the other
  for (int t = threadIdx.x; t < kRegTri; t += blockDim.x) {
    shi[t] = 0.f;
    slo[t] = 0.f;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float acc[kRegWarpTri];
#pragma unroll
  for (int j = 0; j < kRegWarpTri; ++j) acc[j] = 0.f;
  const int64_t npts = int64_t(ng) * ng * ng;
  const int64_t ntiles = (npts + kTX - 1) / kTX;
  // staging: thread t copies point t mod kTX of the tile for the shells t / kTX + 2 u. The point's
  // row (y, z plane index x / N) and column advance by a fixed step per tile of the block.
  const int k = threadIdx.x % kTX, s0 = threadIdx.x / kTX;
  const int64_t rows = int64_t(ng) * ng;
  int64_t row = (int64_t(blockIdx.x) * kTX + k) / ng;
  int col = int((int64_t(blockIdx.x) * kTX + k) - row * ng);
  const int64_t step = int64_t(gridDim.x) * kTX;
  const int64_t step_row = step / ng;
  const int step_col = int(step - step_row * ng);
  const float* fbase = fields + int64_t(s0) * buf_stride;
  const int64_t fstride = 2 * buf_stride;
  const unsigned sbase = static_cast<unsigned>(__cvta_generic_to_shared(&vals[0][s0 * kRow + k]));
  constexpr unsigned kBufBytes = kRegShells * kRow * sizeof(float);
  auto stage = [&](unsigned dst) {
    const bool in_pt = row < rows;
    const float* src = fbase + row * (ng + 2) + col;
#pragma unroll
    for (int u = 0; u < kRegShells / 2; ++u) {
      const bool in = in_pt && s0 + 2 * u < nshells;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst + u * 2 * kRow * 4), "l"(in ? src : fields),
                   "r"(in ? 4 : 0)
                   : "memory");
      src += fstride;
    }
    cp_async_commit();
    row += step_row;
    col += step_col;
    if (col >= ng) {
      col -= ng;
      ++row;
    }
  };
  if (blockIdx.x < ntiles) stage(sbase);
  const bool busy = warp * kRegWarpTri < ntri;  // warp-uniform
  int since_flush = 0, buf = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, buf ^= 1) {
    cp_async_wait_all();
    __syncthreads();  // tile in vals[buf] for every thread; every warp done with vals[buf ^ 1]
    if (tile + gridDim.x < ntiles) stage(sbase + (buf ^ 1) * kBufBytes);
    if (busy) {
      const float* col = vals[buf] + lane;
      switch (warp) {
        case 0: reg_tile<0>(col, acc); break;
        case 1: reg_tile<1>(col, acc); break;
        case 2: reg_tile<2>(col, acc); break;
        case 3: reg_tile<3>(col, acc); break;
        case 4: reg_tile<4>(col, acc); break;
        case 5: reg_tile<5>(col, acc); break;
        case 6: reg_tile<6>(col, acc); break;
        default: reg_tile<7>(col, acc); break;
      }
    }
    if (++since_flush == kFlushTiles || tile + gridDim.x >= ntiles) {
      // every warp folds (an idle warp's sums are zero): a fold under the warp's condition costs
      // the compiler dozens of registers
      since_flush = 0;
      fold_half<64>(acc, lane, 16);
      fold_half<32>(acc, lane, 8);
      fold_half<16>(acc, lane, 4);
      fold_half<8>(acc, lane, 2);
      fold_half<4>(acc, lane, 1);
      const int t0 = warp * kRegWarpTri + 2 * lane;
      comp_add(&shi[t0], &slo[t0], acc[0]);
      comp_add(&shi[t0 + 1], &slo[t0 + 1], acc[1]);
#pragma unroll
      for (int j = 0; j < kRegWarpTri; ++j) acc[j] = 0.f;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntri; t += blockDim.x) atomicAdd(&S[t], double(shi[t]) + double(slo[t]));
}
static_assert(kRegWarps == 8, "k_triple_reg dispatches eight warps");

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

// mg: the grid of the triple sums (bisp_grid; the workspace query sizes for mg = N, the largest).
static pk_status carve_bisp(const pk_config* c, int mg, int nshells, Carver& cv, BispLayout* L) {
  const bool dbl = c->prec != PK_FP32;
  const int ntri = int(make_triangles(nshells).size() / 3);
  L->kind = dbl ? 3 : 2;
  L->fields = cv.take<char>(size_t(nshells) * padded_count(mg) * (dbl ? 8 : 4));
  L->tri = cv.take<int>(size_t(3 * std::max(ntri, 1)));
  L->S = cv.take<double>(size_t(std::max(ntri, 1)));
  pk_status st = get_plan(mg, L->kind, nshells, &L->plan);
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

static pk_status carve_counts(const pk_config* c, int mg, int nshells, Carver& cv, CountLayout* L) {
  const int ntri = int(make_triangles(nshells).size() / 3);
  L->fields = cv.take<double>(size_t(nshells) * padded_count(mg));
  L->prod = cv.take<double>(size_t(padded_count(mg)));
  L->counts = cv.take<unsigned long long>(size_t(std::max(ntri, 1)));
  pk_status st = get_plan(mg, 3, nshells, &L->inv);
  if (st != PK_OK) return st;
  if ((st = get_plan(mg, 1, 1, &L->fwd)) != PK_OK) return st;
  L->work = cv.take<char>(std::max<size_t>(std::max(L->inv.work, L->fwd.work), 256));
  return PK_OK;
}

pk_status bispectrum_ws(const pk_config* c, int nshells, bool counts, size_t* out) {
  Carver cv(nullptr);
  pk_status st;
  if (counts) {
    CountLayout L;
    st = carve_counts(c, c->ng, nshells, cv, &L);
  } else {
    BispLayout L;
    st = carve_bisp(c, c->ng, nshells, cv, &L);
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

int32_t pk_bispectrum_triangles(int32_t nshells, int32_t* tri_host) {
  if (nshells < 1 || nshells > 64 || !tri_host) return 0;
  const std::vector<int> t = make_triangles(nshells);
  for (size_t i = 0; i < t.size(); ++i) tri_host[i] = int32_t(t[i]);
  return int32_t(t.size() / 3);
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
  const int ng = bisp_grid(cfg->ng, shell_lo, shell_w, nshells);  // pair counts on the triple-sum grid
  Carver cv(ws);
  CountLayout L;
  if ((st = carve_counts(cfg, ng, nshells, cv, &L)) != PK_OK) return st;
  if (cv.size() > ws_bytes) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, cv.size());
  const std::vector<int> tri = make_triangles(nshells);
  const int ntri = int(tri.size() / 3);
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
  const int ng = bisp_grid(cfg->ng, shell_lo, shell_w, nshells);  // the triple sums' grid M <= N
  Carver cv(ws);
  BispLayout L;
  if ((st = carve_bisp(cfg, ng, nshells, cv, &L)) != PK_OK) return st;
  if (cv.size() > ws_bytes) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, cv.size());
  const int ntri = pk_bispectrum_ntri(nshells);
  const int64_t pc = padded_count(ng);
  const bool dbl = cfg->prec != PK_FP32;
  const int blocks = num_sms() * 8;
  cudaError_t e;
  k_triangles<<<1, 32, 0, s>>>(L.tri, nshells); count_launch();
  if (dbl)
    k_shell_filter<double2><<<blocks, 256, 0, s>>>(static_cast<const double2*>(delta_k_dev), static_cast<double2*>(L.fields),
                                                  cfg->ng, ng, shell_lo, shell_w, nshells, pc / 2);
  else
    k_shell_filter<float2><<<blocks, 256, 0, s>>>(static_cast<const float2*>(delta_k_dev), static_cast<float2*>(L.fields),
                                                 cfg->ng, ng, shell_lo, shell_w, nshells, pc / 2);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "shell filter");
  if ((st = exec_plan(L.plan, L.kind, L.fields, L.work, s)) != PK_OK) return st;
  if ((e = cudaMemsetAsync(L.S, 0, sizeof(double) * ntri, s)) != cudaSuccess) return cuda_fail(e, "memset");
  if (!dbl && nshells <= kRegShells) {  // triangles in registers
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_triple_reg, kRegWarps * 32, 0) != cudaSuccess) per_sm = 1;
    k_triple_reg<<<num_sms() * std::max(per_sm, 1), kRegWarps * 32, 0, s>>>(static_cast<const float*>(L.fields), ng, nshells,
                                                                             pc, ntri, L.S);
  } else if (ntri <= kTriWarps * kWarpTri && nshells <= kTriMaxShells) {  // lanes over points, warps over triangles
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
  } else {  // one thread per triangle
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
      k_triple<float><<<tblocks, 512, smem, s>>>(static_cast<const float*>(L.fields), ng, nshells, pc, L.tri, ntri, L.S);
  }
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "triple product");
  const double vol = cfg->box * cfg->box * cfg->box;
  const double scale = vol * vol / (double(ng) * ng * ng);
  k_bisp_final<<<(ntri + 255) / 256, 256, 0, s>>>(L.S, reinterpret_cast<const long long*>(counts_dev), ntri, scale, B_dev); count_launch();
  e = cudaGetLastError();
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "bispectrum final");
}

}  // extern "C"
