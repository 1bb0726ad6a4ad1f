// a3 mass assignment, FP32, column walk with register windows (eq:delgrid on both grids of Sec. 3.1).
//
// A particle adds p^3 products to each grid. Accumulating them one by one in shared memory
// (k_assign_tile) serialises on shared atomics; here the products are summed in registers and only
// completed planes leave the thread:
//  - one block per tile of T^3 cells at a time; the tile's particles (binned by tile and, inside
//    the tile, by half-cell slab along x: pk_bin) are staged in shared memory in pieces and sorted
//    there by "key cell" with a counting sort; the key cell is the cell whose fixed stencil (nodes
//    key + S0 .. key + S0 + p - 1 per axis) covers the particle on that grid, key = cell + delta,
//    delta in {0, 1};
//  - each lane owns one key column (k_y, k_z) of one grid and walks it in x with a window of
//    p x p x p register accumulators (planes key+S0 .. key+S0+p-1); after each x step the oldest
//    plane is complete, is summed along z across the lanes of the key row with shuffles and is
//    added to a shared-memory region of (T+4)^3 nodes per grid (32-bit fixed point); the walk of a
//    tile resumes across its pieces, which the slab order makes possible;
//  - after the tile, the region is added to the grids in global memory.
// Per particle and grid: p weights per axis, p^2 products w_x w_y and p^3 multiply-adds, issued as
// packed two-lane FP32 FMAs (fma.rn.f32x2) over pairs of y rows for PCS and CIC.
#include <map>
#include <mutex>
#include <utility>

#include "internal.cuh"

namespace pk {

PK_ERR_ACCESSOR(take_err_walk)

namespace walk {

constexpr int T = kTileCells;  // tile edge (cells)
constexpr int K = T + 1;       // key cells per axis and grid
constexpr int NKEY = K * K * K;
constexpr int RS = T + 4;  // region edge (nodes -1 .. T+2)
constexpr int RVOL = RS * RS * RS;
constexpr int MAXWARP = 6;

// Key columns per row (and key cells per axis) that grid G uses: the unshifted grid of an even
// order keys on floor(u), so its keys stay inside the tile's T cells; the shifted grid, and odd
// orders (nearest-node keys), reach one cell further.
template <int P, int G>
__host__ __device__ constexpr int kspan() {
  return (G == 0 && P % 2 == 0) ? T : K;
}
// Walker lanes: lane = KZ r + kz for key row r of the warp and key column kz (KZ = kspan); 8-column
// rows give four rows per warp (all 32 lanes hold a column), 9-column rows three (lanes 27..31 hold
// none). Neighbouring key columns of a row are neighbouring lanes, so a completed plane is summed
// along z with shuffles before it is added to shared memory.
template <int P, int G>
__host__ __device__ constexpr int rows_per_warp() {
  return 32 / kspan<P, G>();
}
template <int P, int G>
__host__ __device__ constexpr int warps_of_grid() {
  return kspan<P, G>() / rows_per_warp<P, G>();
}
template <int P>
__host__ __device__ constexpr int threads() {
  return 32 * (warps_of_grid<P, 0>() + warps_of_grid<P, 1>());
}
static_assert(T == 8 && K == 9, "the lane layout assumes 8-cell tiles");

template <bool W>
__host__ __device__ constexpr int chunk() {
  return W ? 1024 : 2048;
}

template <bool W>
struct Smem {
  int4 sp[chunk<W>()];
  unsigned short perm[2][chunk<W>()];
  int hist[2][NKEY + 1];  // counts -> exclusive offsets -> bucket ends
  int reg[2][RVOL];  // the tile's node region, fixed point at the tile's scale
  float red[MAXWARP];
  int kmin[2], kmax[2];  // range of key x per grid over the staged chunk
  int scan[2][MAXWARP];
  unsigned long long mbar;  // completion barrier of the bulk copy that stages a chunk
  float sw[W ? chunk<W>() : 1];
};

// Stencil start relative to the key cell: PCS and TSC start one node below it.
template <int P>
__host__ __device__ constexpr int s0() {
  return (P == 3 || P == 4) ? -1 : 0;
}

// Key-cell shift and offset on one axis for a particle at u = c + f on a grid: key = c + delta,
// t = u - key. CIC/PCS key on floor(u); TSC and NGP key on the nearest node (NGP cell half-open).
template <int P>
__device__ __forceinline__ int key_delta(float f, float* t) {
  if constexpr (P == 3) {
    const int d = f >= 0.5f ? 1 : 0;
    *t = f - float(d);
    return d;
  } else if constexpr (P == 1) {
    const int d = f > 0.5f ? 1 : 0;
    *t = f - float(d);
    return d;
  } else {
    *t = f;
    return 0;
  }
}

// Grid G's key delta and offset for in-cell offset f (grid 2 samples the particle shifted by H/2).
template <int P, int G>
__device__ __forceinline__ int grid_key(float f, float* t) {
  if constexpr (G == 0) {
    return key_delta<P>(f, t);
  } else {
    float f2;
    const int d2 = half_shift(f, &f2);
    return d2 + key_delta<P>(f2, t);
  }
}

// Weights of the p stencil nodes from the offset t (PCS returned times 6: the 1/216 of the three
// axes is folded into the particle weight).
template <int P>
__device__ __forceinline__ void weights(float t, float* w) {
  if constexpr (P == 4) {
    const float g = 1.0f - t;
    const float t2 = t * t, g2 = g * g;
    const float t3 = t2 * t, g3 = g2 * g;
    w[0] = g3;
    w[1] = fmaf(3.0f, t3, fmaf(-6.0f, t2, 4.0f));
    w[2] = fmaf(3.0f, g3, fmaf(-6.0f, g2, 4.0f));
    w[3] = t3;
  } else if constexpr (P == 3) {
    const float a = 0.5f - t, b = 0.5f + t;
    w[0] = 0.5f * a * a;
    w[1] = 0.75f - t * t;
    w[2] = 0.5f * b * b;
  } else if constexpr (P == 2) {
    w[0] = 1.0f - t;
    w[1] = t;
  } else {
    w[0] = 1.0f;
  }
}

template <int P>
__host__ __device__ constexpr float weight_scale() {
  return P == 4 ? 1.0f / 216.0f : 1.0f;
}

// Integer reduction into shared memory at a 32-bit shared-window address: the regions are plain
// shared arrays, and naming the state space keeps the address arithmetic 32-bit (constant offsets
// fold into the instruction) instead of generic 64-bit atomics.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void red_shared(unsigned addr, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr), "r"(v));
}

// Packed pairs of FP32 values in one 64-bit register (PTX .f32x2 arithmetic, sm_100 family).
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pack2(float a, float b) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 unpack2(f2x v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  f2x r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ void fma2(f2x& d, f2x a, f2x b) { asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b)); }

// Per-particle operands of the window update. Even p: the y weights as P/2 packed pairs and the x
// and z weights broadcast into both halves of a pair; odd p: scalar weights.
template <int P, bool PACK = (P % 2 == 0)>
struct Operands;
template <int P>
struct Operands<P, true> {
  f2x xa[P], y2[P / 2], z2[P];
};
template <int P>
struct Operands<P, false> {
  float wx[P], wy[P], wz[P];
};

// Where stencil row b sits among the packed pairs of an even order: pair b / 2, high half if b is odd.
template <int P>
__host__ __device__ constexpr int ypair(int b) {
  return b / 2;
}
template <int P>
__host__ __device__ constexpr bool yhigh(int b) {
  return (b & 1) != 0;
}
__device__ __forceinline__ float half2x(f2x v, bool high) {
  const float2 q = unpack2(v);
  return high ? q.y : q.x;
}

// Register window of one walker: plane a (x node key+S0+a) x row b (y) x column c (z).
// Even p: y pairs packed in 64-bit registers; odd p: scalars.
template <int P, bool PACK = (P % 2 == 0)>
struct Window;

template <int P>
struct Window<P, true> {
  f2x v[P][P / 2][P];  // plane a, y pair bp, z column c
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int a = 0; a < P; ++a)
#pragma unroll
      for (int bp = 0; bp < P / 2; ++bp)
#pragma unroll
        for (int c = 0; c < P; ++c) v[a][bp][c] = 0ull;
  }
  // v[a][bp][c] += (w_x[a] y-pair bp) * w_z[c]: p^2/2 packed products, p^3/2 packed FMAs
  __device__ __forceinline__ void add(const Operands<P>& o) {
#pragma unroll
    for (int a = 0; a < P; ++a) {
#pragma unroll
      for (int bp = 0; bp < P / 2; ++bp) {
        const f2x xy = mul2(o.xa[a], o.y2[bp]);
#pragma unroll
        for (int c = 0; c < P; ++c) fma2(v[a][bp][c], xy, o.z2[c]);
      }
    }
  }
  __device__ __forceinline__ void row(int a, int b, float* out) const {
#pragma unroll
    for (int c = 0; c < P; ++c) out[c] = half2x(v[a][ypair<P>(b)][c], yhigh<P>(b));
  }
  __device__ __forceinline__ void shift() {
#pragma unroll
    for (int a = 0; a + 1 < P; ++a)
#pragma unroll
      for (int bp = 0; bp < P / 2; ++bp)
#pragma unroll
        for (int c = 0; c < P; ++c) v[a][bp][c] = v[a + 1][bp][c];
#pragma unroll
    for (int bp = 0; bp < P / 2; ++bp)
#pragma unroll
      for (int c = 0; c < P; ++c) v[P - 1][bp][c] = 0ull;
  }
};

template <int P>
struct Window<P, false> {
  float v[P][P][P];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int a = 0; a < P; ++a)
#pragma unroll
      for (int b = 0; b < P; ++b)
#pragma unroll
        for (int c = 0; c < P; ++c) v[a][b][c] = 0.0f;
  }
  __device__ __forceinline__ void add(const Operands<P>& o) {
#pragma unroll
    for (int a = 0; a < P; ++a)
#pragma unroll
      for (int b = 0; b < P; ++b) {
        const float xy = o.wx[a] * o.wy[b];
#pragma unroll
        for (int c = 0; c < P; ++c) v[a][b][c] = fmaf(xy, o.wz[c], v[a][b][c]);
      }
  }
  __device__ __forceinline__ void row(int a, int b, float* out) const {
#pragma unroll
    for (int c = 0; c < P; ++c) out[c] = v[a][b][c];
  }
  __device__ __forceinline__ void shift() {
#pragma unroll
    for (int a = 0; a + 1 < P; ++a)
#pragma unroll
      for (int b = 0; b < P; ++b)
#pragma unroll
        for (int c = 0; c < P; ++c) v[a][b][c] = v[a + 1][b][c];
#pragma unroll
    for (int b = 0; b < P; ++b)
#pragma unroll
      for (int c = 0; c < P; ++c) v[P - 1][b][c] = 0.0f;
  }
};

// Weights of an even order on one axis as P/2 packed pairs (nodes 2bp, 2bp + 1). (Evaluating the
// PCS pieces on (t, 1 - t) as packed pairs takes fewer instructions but a longer dependency chain,
// and measured slower.)
template <int P>
__device__ __forceinline__ void packed_weights(float t, f2x* pr) {
  float w[P];
  weights<P>(t, w);
#pragma unroll
  for (int bp = 0; bp < P / 2; ++bp) pr[bp] = pack2(w[2 * bp], w[2 * bp + 1]);
}

// Window operands of one particle on grid G (x weights scaled by the particle weight wgt).
template <int P, int G>
__device__ __forceinline__ Operands<P> particle_operands(const int4 r, float wgt) {
  float tx, ty, tz;
  grid_key<P, G>(__int_as_float(r.y), &tx);
  grid_key<P, G>(__int_as_float(r.z), &ty);
  grid_key<P, G>(__int_as_float(r.w), &tz);
  Operands<P> o;
  if constexpr (P % 2 == 0) {
    f2x px[P / 2], pz[P / 2];
    packed_weights<P>(tx, px);
    packed_weights<P>(ty, o.y2);
    packed_weights<P>(tz, pz);
    const f2x wg = pack2(wgt, wgt);
#pragma unroll
    for (int bp = 0; bp < P / 2; ++bp) px[bp] = mul2(px[bp], wg);
#pragma unroll
    for (int a = 0; a < P; ++a) {
      const float x = half2x(px[ypair<P>(a)], yhigh<P>(a));
      const float z = half2x(pz[ypair<P>(a)], yhigh<P>(a));
      o.xa[a] = pack2(x, x);
      o.z2[a] = pack2(z, z);
    }
  } else {
    weights<P>(tx, o.wx);
    weights<P>(ty, o.wy);
    weights<P>(tz, o.wz);
#pragma unroll
    for (int a = 0; a < P; ++a) o.wx[a] *= wgt;
  }
  return o;
}

// Plane a of every lane's window, summed over the key columns of each row with shuffles: node z of
// the row receives column kz's offset c = z - kz - S0 for kz = z - S0 - c; the lane of column kz
// collects the sum for node kz + S0 and adds it to the region; nodes past the row's last column are
// added by the columns that reach them. The region holds fixed-point integers (value x scale, rounded
// to nearest): integer shared-memory atomics run about three times faster than FP32 ones.
template <int P, int KZ>
__device__ __forceinline__ void flush_plane(const Window<P>& win, int a, int* reg, int rx, int ry0, int kz, bool valid,
                                            float scale) {
#pragma unroll
  for (int b = 0; b < P; ++b) {
    float v[P];
    win.row(a, b, v);
    float sum = v[0];
#pragma unroll
    for (int d = 1; d < P; ++d) {
      const float t = __shfl_up_sync(0xffffffffu, v[d], d);
      if (kz >= d) sum += t;
    }
    if (valid) {
      const unsigned r = smem_u32(reg + (rx * RS + ry0 + b) * RS + kz + s0<P>() + 1);
      red_shared(r, __float2int_rn(sum * scale));
#pragma unroll
      for (int c = 1; c < P; ++c)
        if (kz + c >= KZ) red_shared(r + 4u * c, __float2int_rn(v[c] * scale));
    }
  }
}

// State of one warp of walkers across the chunks of a tile: the register window, the next x step to
// process (xo) and the number of window shifts since a particle was last added (zs; the window is all
// zero once zs >= P).
template <int P>
struct Walker {
  Window<P> win;
  int xo, zs;
  __device__ __forceinline__ void reset() {
    win.zero();
    xo = 0;
    zs = P;
  }
};

// One warp of walkers of grid G (warp-in-grid q) over the staged chunk: lane -> key column (ky, kz);
// each walks its column in x with its register window; bucket (col, x) holds perm[hist[key-1] ..
// hist[key]) after the scatter (hist = bucket ends). All 32 lanes run the x loop together (the
// flush shuffles). A tile's particles arrive ordered by half-cell slab along x, and every grid's key
// x is a non-decreasing function of that slab, so the chunk's keys lie in [xo, kmax]: steps below
// kmax are complete after this chunk and are flushed; step kmax stays open for the next chunk (its
// partial sums stay in the window), unless this is the tile's last chunk, which walks to the end of
// the span and flushes the remaining planes. Buckets past the grid's key span are empty by
// construction.
template <int P, int G, bool W>
__device__ __forceinline__ void walk_range(Smem<W>& S, Walker<P>& wk, bool last, int q, int lane, float scale) {
  constexpr int KZ = kspan<P, G>(), R = rows_per_warp<P, G>();
  const int* ends = S.hist[G];
  const int r = lane / KZ, kz = lane - r * KZ;
  const bool valid = r < R;
  const int ky = R * q + (valid ? r : 0);
  const int kbase = (ky * K + kz) * K;
  if (S.kmin[G] < wk.xo && lane == 0) raise_err(PK_DERR_ORDER);  // keys behind the walk: not in slab order
  const int xe = last ? KZ - 1 : max(wk.xo, S.kmax[G]);
  int jb = valid ? (kbase + wk.xo == 0 ? 0 : ends[kbase + wk.xo - 1]) : 0;
  const int ry0 = ky + s0<P>() + 1;  // region row of stencil offset 0
  int* reg = S.reg[G];
  const unsigned short* perm = S.perm[G];
  Window<P>& win = wk.win;
#pragma unroll 1
  for (int x = wk.xo; x <= xe; ++x) {
    const int je = valid ? ends[kbase + x] : 0;
    if (__any_sync(0xffffffffu, jb < je)) {
      wk.zs = 0;
      // one particle per iteration; the next record is loaded before the current one is accumulated
      int j = jb;
      int4 r0 = make_int4(0, 0, 0, 0);
      float s0w = 1.0f;
      if (j < je) {
        const int i0 = perm[j];
        r0 = S.sp[i0];
        if (W) s0w = S.sw[i0];
      }
      for (; j < je; ++j) {
        const int4 c0 = r0;
        const float c0w = s0w;
        if (j + 1 < je) {
          const int i0 = perm[j + 1];
          r0 = S.sp[i0];
          if (W) s0w = S.sw[i0];
        }
        win.add(particle_operands<P, G>(c0, c0w * weight_scale<P>()));
      }
    }
    if (valid) jb = je;
    if (x < xe || last) {  // node plane x + s0 is complete: add it to the region and shift the window
      if (wk.zs < P) flush_plane<P, KZ>(win, 0, reg, x + s0<P>() + 1, ry0, kz, valid, scale);
      win.shift();
      ++wk.zs;
    }
  }
  if (last) {  // the remaining planes KZ + s0 .. KZ + s0 + P - 2 (plane a is non-zero while a < P - zs)
#pragma unroll
    for (int a = 0; a + 1 < P; ++a)
      if (a < P - wk.zs) flush_plane<P, KZ>(win, a, reg, KZ + a + s0<P>() + 1, ry0, kz, valid, scale);
    wk.reset();
  } else {
    wk.xo = xe;
  }
}

// Bulk copy (TMA) of `bytes` from global to shared memory, completing on the mbarrier at bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  const unsigned b = static_cast<unsigned>(__cvta_generic_to_shared(bar));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d), "l"(src),
               "r"(bytes), "r"(b)
               : "memory");
}

// Waits for phase `parity` of the mbarrier, giving up after a bounded number of polls.
__device__ __forceinline__ bool bulk_wait(unsigned long long* bar, unsigned parity) {
  const unsigned b = static_cast<unsigned>(__cvta_generic_to_shared(bar));
  for (int it = 0; it < (1 << 22); ++it) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok)
                 : "r"(b), "r"(parity)
                 : "memory");
    if (ok) return true;
  }
  return false;
}

// Adds a tile's node regions (origin: node (cx0-1, cy0-1, cz0-1); grid gi at reg + gi RVOL),
// converted back from fixed point, to the grids. A thread owns one of 8 slots along z for its whole
// share of the rows: slot 0 is node 0 of a row, slots 1..5 the node pairs (1,2)..(9,10), whose global
// z index is even so each pair is one 8-byte vector reduction, slot 6 node 11, slot 7 idle. The
// slot's z indices are computed once, outside the row loop.
__device__ __forceinline__ void flush_region(const int* reg, int ngrid, int cx0, int cy0, int cz0, int ng, int ldz,
                                             float inv_scale, float* g1, float* g2, int tid, int nthreads) {
  const int slot = tid & 7;
  if (slot == 7) return;
  const bool pair = slot >= 1 && slot <= 5;
  const int rz = slot == 0 ? 0 : (slot == 6 ? RS - 1 : 2 * slot - 1);
  const int z = wrap(cz0 - 1 + rz, ng);
  const bool vec = pair && z + 1 < ng;  // z even, row bases 8-byte aligned (ldz even)
  const int z1 = pair ? wrap(z + 1, ng) : 0;
  const int nrows = ngrid * RS * RS;
  for (int row = tid >> 3; row < nrows; row += nthreads >> 3) {
    const int gi = row / (RS * RS), rr = row - gi * (RS * RS);
    const int rx = rr / RS, ry = rr - rx * RS;
    const int* src = reg + gi * RVOL + rr * RS + rz;
    float* gg = (gi == 0 ? g1 : g2) + (int64_t(wrap(cx0 - 1 + rx, ng)) * ng + wrap(cy0 - 1 + ry, ng)) * ldz;
    const float v0 = float(src[0]) * inv_scale;
    if (!pair) {
      if (v0 != 0.0f) atomicAdd(gg + z, v0);
    } else {
      const float v1 = float(src[1]) * inv_scale;
      if (v0 != 0.0f || v1 != 0.0f) {
        if (vec) {
          asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(gg + z), "f"(v0), "f"(v1) : "memory");
        } else {
          atomicAdd(gg + z, v0);
          atomicAdd(gg + z1, v1);
        }
      }
    }
  }
}

// Fixed-point scale 2^e of a tile's region: no node (nor any partial sum of one) exceeds the tile's
// total |weight| B, and B 2^e < 2^30 leaves room for the rounding of every addition. With weights,
// B is summed by the block (red: one float per warp); the caller synchronises before the first use.
template <bool W>
__device__ __forceinline__ void tile_scale(const float* w, int64_t beg, int64_t end, float* red, int nwarp, int tid,
                                           int nthreads, float* scale, float* inv_scale) {
  float bound = float(end - beg);
  if (W) {
    float a = 0.0f;
    for (int64_t i = beg + tid; i < end; i += nthreads) a += fabsf(w[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((tid & 31) == 0) red[tid >> 5] = a;
    __syncthreads();
    bound = 0.0f;
    for (int q = 0; q < nwarp; ++q) bound += red[q];
    bound *= 1.0001f;  // the FP32 sum's rounding
  }
  int ex;
  frexpf(fmaxf(bound, 1.0f), &ex);  // bound < 2^ex
  *scale = ldexpf(1.0f, 30 - ex);
  *inv_scale = ldexpf(1.0f, ex - 30);
}

// ---- direct scatter (sparse tiles) ------------------------------------------------------------------
// A walk pays for every x step of every key column of a tile whether or not its buckets hold
// particles; on sparse tiles that fixed cost dominates. There, each thread adds its particles' p^3
// weights per grid straight into the fixed-point region with integer shared atomics instead.
constexpr int SCATTER_THREADS = 256;

// Pieces of the scatter are staged in two buffers: the next piece is copied while this one is used.
template <bool W>
__host__ __device__ constexpr int scatter_chunk() {
  return W ? 512 : 1024;
}

template <bool W>
struct ScatterSmem {
  int4 sp[2][scatter_chunk<W>()];
  int reg[2][RVOL];
  float red[SCATTER_THREADS / 32];
  unsigned long long mbar[2];
  float sw[2][W ? scatter_chunk<W>() : 1];
};

// Adds one particle's p^3 weights on grid G to that grid's region (scale: the weight times the
// region's fixed-point scale). Region nodes of the stencil: key + S0 + 1 .. key + S0 + p per axis.
// (Rounding by adding 1.5 2^23 instead of a conversion would cap the scale at 2^21 per unit weight,
// too coarse on sparse tiles: their nodes then miss the FP32 grid tolerance.)
template <int P, int G>
__device__ __forceinline__ void scatter_particle(int* reg, int lx, int ly, int lz, float fx, float fy, float fz, float sc) {
  float tx, ty, tz;
  const int kx = lx + grid_key<P, G>(fx, &tx), ky = ly + grid_key<P, G>(fy, &ty), kz = lz + grid_key<P, G>(fz, &tz);
  float wx[P], wy[P], wz[P];
  weights<P>(tx, wx);
  weights<P>(ty, wy);
  weights<P>(tz, wz);
#pragma unroll
  for (int a = 0; a < P; ++a) wx[a] *= sc;
  const unsigned base = smem_u32(reg + ((kx + s0<P>() + 1) * RS + ky + s0<P>() + 1) * RS + kz + s0<P>() + 1);
#pragma unroll
  for (int a = 0; a < P; ++a)
#pragma unroll
    for (int b = 0; b < P; ++b) {
      const float xy = wx[a] * wy[b];
#pragma unroll
      for (int c = 0; c < P; ++c) red_shared(base + 4u * ((a * RS + b) * RS + c), __float2int_rn(xy * wz[c]));
    }
}

}  // namespace walk

template <int P, bool W>
__global__ void __launch_bounds__(walk::threads<P>(), 3)
    k_assign_walk(const pk_cellpos* __restrict__ p, const float* __restrict__ w, const int64_t* __restrict__ toff, int64_t n,
                  int ng, int ntile, int interlace, float* __restrict__ g1, float* __restrict__ g2, int ldz,
                  int64_t cat_stride) {
  using namespace walk;
  constexpr int CH = chunk<W>();
  constexpr int THREADS = threads<P>(), NWARP = THREADS / 32, NW0 = warps_of_grid<P, 0>();
  constexpr int SCAN_PER_THREAD = (NKEY + 1 + THREADS - 1) / THREADS;
  {  // blockIdx.y selects a catalogue of a batch: its grids and its tile offsets
    const int cat = blockIdx.y;
    g1 += cat * cat_stride;
    if (g2) g2 += cat * cat_stride;
    toff += int64_t(cat) * ntile * ntile * ntile;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<W>& S = *reinterpret_cast<Smem<W>*>(smem_raw);
  const int ngrid = interlace ? 2 : 1;
  const int ntiles = ntile * ntile * ntile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    const unsigned b = static_cast<unsigned>(__cvta_generic_to_shared(&S.mbar));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  }
  __syncthreads();
  unsigned parity = 0;
  Walker<P> wk;
  wk.reset();
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t beg = max(toff[tile], int64_t(0)), end = min(toff[tile + 1], n);
    if (beg >= end) continue;
    const int tz = tile % ntile, ty = (tile / ntile) % ntile, tx = tile / (ntile * ntile);
    const int cx0 = tx * T, cy0 = ty * T, cz0 = tz * T;  // first cell of the tile
    for (int i = tid; i < ngrid * RVOL; i += THREADS) (&S.reg[0][0])[i] = 0;
    float scale, inv_scale;
    tile_scale<W>(w, beg, end, S.red, NWARP, tid, THREADS, &scale, &inv_scale);
    for (int64_t c0 = beg; c0 < end; c0 += CH) {
      const int m = int(min(int64_t(CH), end - c0));
      // stage the chunk with one bulk copy (16-byte records, 16-byte aligned)
      if (tid == 0) bulk_load(S.sp, p + c0, unsigned(m) * 16u, &S.mbar);
      if (W)
        for (int i = tid; i < m; i += THREADS) S.sw[i] = w[c0 + i];
      for (int i = tid; i < 2 * (NKEY + 1); i += THREADS) (&S.hist[0][0])[i] = 0;
      if (tid < 2) {
        S.kmin[tid] = K;
        S.kmax[tid] = -1;
      }
      const bool arrived = bulk_wait(&S.mbar, parity);
      parity ^= 1u;
      if (__syncthreads_or(!arrived)) {  // the copy did not complete: report, drain, stop
        if (tid == 0) {
          raise_err(PK_DERR_TIMEOUT);
          bulk_wait(&S.mbar, parity ^ 1u);
        }
        return;
      }
      // count the key cells of both grids; the record's cell word is replaced by the two keys
      // (grid 1 in the low half, grid 2 in the high half), or by -1 for a particle that is skipped;
      // the range of key x per grid is gathered for the walk
      int lo0 = K, hi0 = -1, lo1 = K, hi1 = -1;
      for (int i = tid; i < m; i += THREADS) {
        const int4 r = S.sp[i];
        const uint32_t cell = uint32_t(r.x);
        const int lx = cell_x(cell) - cx0, ly = cell_y(cell) - cy0, lz = cell_z(cell) - cz0;
        if ((cell >> 30) == 0 && unsigned(lx) < unsigned(T) && unsigned(ly) < unsigned(T) && unsigned(lz) < unsigned(T)) {
          float t;
          const float fx = __int_as_float(r.y), fy = __int_as_float(r.z), fz = __int_as_float(r.w);
          const int kx1 = lx + grid_key<P, 0>(fx, &t);
          const int k1 = ((ly + grid_key<P, 0>(fy, &t)) * K + (lz + grid_key<P, 0>(fz, &t))) * K + kx1;
          atomicAdd(&S.hist[0][k1], 1);
          lo0 = min(lo0, kx1);
          hi0 = max(hi0, kx1);
          int k2 = 0;
          if (interlace) {
            const int kx2 = lx + grid_key<P, 1>(fx, &t);
            k2 = ((ly + grid_key<P, 1>(fy, &t)) * K + (lz + grid_key<P, 1>(fz, &t))) * K + kx2;
            atomicAdd(&S.hist[1][k2], 1);
            lo1 = min(lo1, kx2);
            hi1 = max(hi1, kx2);
          }
          S.sp[i].x = k1 | (k2 << 16);
        } else {
          raise_err(PK_DERR_CELLRANGE);
          S.sp[i].x = -1;
        }
      }
      lo0 = __reduce_min_sync(0xffffffffu, lo0);
      hi0 = __reduce_max_sync(0xffffffffu, hi0);
      lo1 = __reduce_min_sync(0xffffffffu, lo1);
      hi1 = __reduce_max_sync(0xffffffffu, hi1);
      if (lane == 0) {
        atomicMin(&S.kmin[0], lo0);
        atomicMax(&S.kmax[0], hi0);
        atomicMin(&S.kmin[1], lo1);
        atomicMax(&S.kmax[1], hi1);
      }
      __syncthreads();
      // block-wide exclusive scan of both histograms (NKEY + 1 entries each)
      {
        int v0[SCAN_PER_THREAD], v1[SCAN_PER_THREAD];
        int s0v = 0, s1v = 0;
#pragma unroll
        for (int k = 0; k < SCAN_PER_THREAD; ++k) {
          const int idx = tid * SCAN_PER_THREAD + k;
          v0[k] = idx <= NKEY ? S.hist[0][idx] : 0;
          v1[k] = idx <= NKEY ? S.hist[1][idx] : 0;
          s0v += v0[k];
          s1v += v1[k];
        }
        int x0 = s0v, x1 = s1v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y0 = __shfl_up_sync(0xffffffffu, x0, o), y1 = __shfl_up_sync(0xffffffffu, x1, o);
          if (lane >= o) {
            x0 += y0;
            x1 += y1;
          }
        }
        if (lane == 31) {
          S.scan[0][warp] = x0;
          S.scan[1][warp] = x1;
        }
        __syncthreads();
        int e0 = x0 - s0v, e1 = x1 - s1v;
        for (int q = 0; q < warp; ++q) {
          e0 += S.scan[0][q];
          e1 += S.scan[1][q];
        }
#pragma unroll
        for (int k = 0; k < SCAN_PER_THREAD; ++k) {
          const int idx = tid * SCAN_PER_THREAD + k;
          if (idx <= NKEY) {
            S.hist[0][idx] = e0;
            S.hist[1][idx] = e1;
          }
          e0 += v0[k];
          e1 += v1[k];
        }
      }
      __syncthreads();
      // scatter particle indices into key order; hist[key] advances to the bucket's end
      for (int i = tid; i < m; i += THREADS) {
        const int keys = S.sp[i].x;
        if (keys < 0) continue;
        S.perm[0][atomicAdd(&S.hist[0][keys & 0xffff], 1)] = (unsigned short)i;
        if (interlace) S.perm[1][atomicAdd(&S.hist[1][keys >> 16], 1)] = (unsigned short)i;
      }
      __syncthreads();
      // walk: the first NW0 warps grid 1, the others grid 2 (warp-uniform grid)
      const bool last = c0 + CH >= end;
      if (warp < NW0)
        walk_range<P, 0, W>(S, wk, last, warp, lane, scale);
      else if (interlace)
        walk_range<P, 1, W>(S, wk, last, warp - NW0, lane, scale);
      __syncthreads();
    }
    flush_region(&S.reg[0][0], ngrid, cx0, cy0, cz0, ng, ldz, inv_scale, g1, g2, tid, THREADS);
    __syncthreads();
  }
}

// a3, FP32, direct scatter: a block takes tiles in a grid-stride sequence and their pieces in
// order, the copy of the next piece overlapping the use of the current one; particles are spread over
// the lanes of a warp q = ceil(m / 32) records apart (different cells, so a warp's atomics seldom meet
// on one node); fixed-point regions are flushed to the grids as in k_assign_walk.
template <int P, bool W>
__global__ void __launch_bounds__(walk::SCATTER_THREADS, 4)
    k_assign_scatter(const pk_cellpos* __restrict__ p, const float* __restrict__ w, const int64_t* __restrict__ toff,
                     int64_t n, int ng, int ntile, int interlace, float* __restrict__ g1, float* __restrict__ g2, int ldz,
                     int64_t cat_stride) {
  using namespace walk;
  constexpr int CH = scatter_chunk<W>(), THREADS = SCATTER_THREADS, NWARP = THREADS / 32;
  {
    const int cat = blockIdx.y;
    g1 += cat * cat_stride;
    if (g2) g2 += cat * cat_stride;
    toff += int64_t(cat) * ntile * ntile * ntile;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem<W>& S = *reinterpret_cast<ScatterSmem<W>*>(smem_raw);
  const int ngrid = interlace ? 2 : 1;
  const int ntiles = ntile * ntile * ntile;
  const int tid = threadIdx.x;
  if (tid < 2) {
    const unsigned b = static_cast<unsigned>(__cvta_generic_to_shared(&S.mbar[tid]));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  }
  __syncthreads();
  // the block's pieces: (tile, first record c0, tile's records [beg, end))
  struct Piece {
    int tile;
    int64_t beg, end, c0;
  };
  auto advance = [&](Piece& c) -> bool {  // next piece of this tile, else the first of the next non-empty tile
    c.c0 += CH;
    while (c.c0 >= c.end) {
      c.tile += gridDim.x;
      if (c.tile >= ntiles) return false;
      c.beg = max(toff[c.tile], int64_t(0));
      c.end = min(toff[c.tile + 1], n);
      c.c0 = c.beg;
    }
    return true;
  };
  Piece cur;
  cur.tile = int(blockIdx.x) - int(gridDim.x);
  cur.beg = cur.end = 0;
  cur.c0 = -CH;
  if (!advance(cur)) return;
  if (tid == 0) bulk_load(S.sp[0], p + cur.c0, unsigned(min(int64_t(CH), cur.end - cur.c0)) * 16u, &S.mbar[0]);
  Piece nxt = cur;
  bool has_next = advance(nxt);
  unsigned parity = 0u;  // bit b: the phase buffer b waits for next
  int buf = 0;
  float scale = 1.0f, inv_scale = 1.0f;
  int cx0 = 0, cy0 = 0, cz0 = 0;
  while (true) {
    const int m = int(min(int64_t(CH), cur.end - cur.c0));
    if (cur.c0 == cur.beg) {  // first piece of a tile: clear the region, take the tile's scale
      const int tz = cur.tile % ntile, ty = (cur.tile / ntile) % ntile, tx = cur.tile / (ntile * ntile);
      cx0 = tx * T;
      cy0 = ty * T;
      cz0 = tz * T;
      for (int i = tid; i < ngrid * RVOL; i += THREADS) (&S.reg[0][0])[i] = 0;
      tile_scale<W>(w, cur.beg, cur.end, S.red, NWARP, tid, THREADS, &scale, &inv_scale);
    }
    // the other buffer was released by the synchronisation that ended the previous piece
    if (has_next && tid == 0)
      bulk_load(S.sp[buf ^ 1], p + nxt.c0, unsigned(min(int64_t(CH), nxt.end - nxt.c0)) * 16u, &S.mbar[buf ^ 1]);
    if (W)
      for (int i = tid; i < m; i += THREADS) S.sw[buf][i] = w[cur.c0 + i];
    const bool arrived = bulk_wait(&S.mbar[buf], (parity >> buf) & 1u);
    parity ^= 1u << buf;
    if (__syncthreads_or(!arrived)) {  // a copy did not complete: report, drain what is in flight, stop
      if (tid == 0) {
        raise_err(PK_DERR_TIMEOUT);
        bulk_wait(&S.mbar[buf], ((parity >> buf) & 1u) ^ 1u);
        if (has_next) bulk_wait(&S.mbar[buf ^ 1], (parity >> (buf ^ 1)) & 1u);
      }
      return;
    }
    const int4* sp = S.sp[buf];
    const float* sw = S.sw[buf];
    const int q = (m + 31) / 32;
    for (int i = tid; i < 32 * q; i += THREADS) {
      const int j = (i & 31) * q + (i >> 5);
      if (j >= m) continue;
      const int4 r = sp[j];
      const uint32_t cell = uint32_t(r.x);
      const int lx = cell_x(cell) - cx0, ly = cell_y(cell) - cy0, lz = cell_z(cell) - cz0;
      if ((cell >> 30) != 0 || unsigned(lx) >= unsigned(T) || unsigned(ly) >= unsigned(T) || unsigned(lz) >= unsigned(T)) {
        raise_err(PK_DERR_CELLRANGE);
        continue;
      }
      const float fx = __int_as_float(r.y), fy = __int_as_float(r.z), fz = __int_as_float(r.w);
      const float sc = (W ? sw[j] : 1.0f) * weight_scale<P>() * scale;
      scatter_particle<P, 0>(S.reg[0], lx, ly, lz, fx, fy, fz, sc);
      if (interlace) scatter_particle<P, 1>(S.reg[1], lx, ly, lz, fx, fy, fz, sc);
    }
    __syncthreads();
    if (cur.c0 + CH >= cur.end) {  // last piece of the tile
      flush_region(&S.reg[0][0], ngrid, cx0, cy0, cz0, ng, ldz, inv_scale, g1, g2, tid, THREADS);
      __syncthreads();
    }
    if (!has_next) break;
    cur = nxt;
    buf ^= 1;
    has_next = advance(nxt);
  }
}

// Shared-memory opt-in and resident blocks per SM of a kernel, set up once per (kernel, device): later
// launches make no attribute or occupancy calls, so a call captured in a CUDA graph holds launches only.
static cudaError_t kernel_setup(const void* kernel, int threads, size_t smem, int* per_sm) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find({kernel, dev});
  if (it != cache.end()) {
    *per_sm = it->second;
    return cudaSuccess;
  }
  if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess) return e;
  int n = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
  cache[{kernel, dev}] = n;
  *per_sm = n;
  return cudaSuccess;
}

// Mean particles per tile below which the direct scatter replaces the walk. Measured per tile on one
// GB300: the walk costs about 73 ns + 0.018 ns per particle of block time, the scatter 19 ns + 0.048 ns,
// so they cross near 1800 particles per tile (8^3 cells).
constexpr int64_t kScatterMaxMean = 1536;

template <int P, bool W>
static cudaError_t launch_scatter_pw(const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                     bool interlace, float* g1, float* g2, int ldz, cudaStream_t s, int ncat,
                                     int64_t cat_stride) {
  const int ntile = tiles_per_axis(ng);
  const int ntiles = ntile * ntile * ntile;
  const size_t smem = sizeof(walk::ScatterSmem<W>);
  int per_sm = 1;
  cudaError_t e = kernel_setup(reinterpret_cast<const void*>(k_assign_scatter<P, W>), walk::SCATTER_THREADS, smem, &per_sm);
  if (e != cudaSuccess) return e;
  const dim3 blocks(std::max(1, std::min(ntiles, std::max(1, num_sms() * per_sm / ncat))), ncat);
  k_assign_scatter<P, W><<<blocks, walk::SCATTER_THREADS, smem, s>>>(p, w, toff, n, ng, ntile, interlace ? 1 : 0, g1, g2, ldz,
                                                                     cat_stride);
  count_launch();
  return cudaGetLastError();
}

bool assign_uses_scatter(int64_t n, int ng, int ncat) {
  const int64_t nt = tiles_per_axis(ng);
  return n < kScatterMaxMean * nt * nt * nt * ncat;
}

template <int P, bool W>
static cudaError_t launch_walk_pw(const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng, bool interlace,
                                  float* g1, float* g2, int ldz, cudaStream_t s, int ncat, int64_t cat_stride) {
  const int ntile = tiles_per_axis(ng);
  const int ntiles = ntile * ntile * ntile;
  if (assign_uses_scatter(n, ng, ncat))  // sparse tiles: the direct scatter
    return launch_scatter_pw<P, W>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride);
  const size_t smem = sizeof(walk::Smem<W>);
  int per_sm = 1;
  cudaError_t e = kernel_setup(reinterpret_cast<const void*>(k_assign_walk<P, W>), walk::threads<P>(), smem, &per_sm);
  if (e != cudaSuccess) return e;
  const dim3 blocks(std::max(1, std::min(ntiles, std::max(1, num_sms() * per_sm / ncat))), ncat);
  k_assign_walk<P, W><<<blocks, walk::threads<P>(), smem, s>>>(p, w, toff, n, ng, ntile, interlace ? 1 : 0, g1, g2, ldz, cat_stride);
  count_launch();
  return cudaGetLastError();
}

template <int P>
static cudaError_t launch_walk_p(const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng, bool interlace,
                                 float* g1, float* g2, int ldz, cudaStream_t s, int ncat, int64_t cat_stride) {
  return w ? launch_walk_pw<P, true>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride)
           : launch_walk_pw<P, false>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride);
}

cudaError_t launch_assign_walk_f32(int order, const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                   bool interlace, float* g1, float* g2, int ldz, cudaStream_t s, int ncat,
                                   int64_t cat_stride) {
  switch (order) {
    case 1: return launch_walk_p<1>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride);
    case 2: return launch_walk_p<2>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride);
    case 3: return launch_walk_p<3>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride);
    case 4: return launch_walk_p<4>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride);
    case 5:
    case 6:  // orders beyond PCS: the direct scatter of the records (box unused for packed records)
      if (ncat != 1) return cudaErrorInvalidValue;
      return launch_assign_direct_f32(order, p, PK_POS_CELL_F32OFF, w, n, ng, 1.0, interlace, g1, g2, ldz, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pk
