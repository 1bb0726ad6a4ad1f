// a3 mass assignment, FP32, on tiles of binned particles (eq:delgrid on both grids of Sec. 3.1).
//
// A particle adds p^3 products to each grid. The particles arrive binned by tile of T^3 cells (pk_bin);
// a block takes one tile at a time, stages its particles in shared memory in pieces (bulk copies) and
// accumulates the tile's nodes in a shared region of (T+4)^3 nodes per grid held in 32-bit fixed
// point, which is added to the grids in global memory after the tile. Two kernels fill the region:
//  - k_assign_scatter (sparse tiles): each thread adds its particles' p^3 weights per grid with
//    integer shared atomics;
//  - k_assign_cells (dense tiles): a piece is counting-sorted by "key cell" (the cell whose fixed
//    stencil, nodes key + S0 .. key + S0 + p - 1 per axis, covers the particle on that grid); each
//    lane sums one key cell's particles into a p x p x p register window and adds the window to the
//    region once, so a node receives one addition per key cell instead of one per particle.
// Per particle and grid: p weights per axis, p^2 products w_x w_y and p^3 multiply-adds, issued as
// packed two-lane FP32 FMAs (fma.rn.f32x2) over pairs of y rows for PCS and CIC.
#include <map>
#include <mutex>
#include <utility>

#include "internal.cuh"

namespace pk {

PK_ERR_ACCESSOR(take_err_tiles)

namespace tiles {

constexpr int T = kTileCells;  // tile edge (cells)
constexpr int K = T + 1;       // key cells per axis and grid
constexpr int NKEY = K * K * K;
constexpr int RS = T + 4;  // region edge (nodes -1 .. T+2)
constexpr int RVOL = RS * RS * RS;
constexpr int kDetRun = 32;  // deterministic mode: rounded particles summed per window (det_tile_scale)
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
// 64-bit two's-complement reduction (the region of the heavy tiles, below).
__device__ __forceinline__ void red_shared(unsigned addr, long long v) {
  asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(addr), "l"(v));
}
// Window value (already at the region's fixed-point scale) to the region's integer type, to nearest.
__device__ __forceinline__ int to_fixed(float v, int*) { return __float2int_rn(v); }
__device__ __forceinline__ long long to_fixed(float v, long long*) { return __float2ll_rn(v); }

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
__device__ __forceinline__ f2x fma2c(f2x a, f2x b, f2x c) {
  f2x r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  f2x r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

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

// Register window of one key cell: plane a (x node key+S0+a) x row b (y) x column c (z).
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
  // The deterministic mode: every product rounded to an integer by the FMA that adds 1.5 2^23 (exact
  // for |product| <= 2^22), the integers summed exactly (the caller keeps every partial sum below 2^24).
  __device__ __forceinline__ void add_rounded(const Operands<P>& o) {
    const f2x m = pack2(12582912.0f, 12582912.0f), mn = pack2(-12582912.0f, -12582912.0f);
#pragma unroll
    for (int a = 0; a < P; ++a) {
#pragma unroll
      for (int bp = 0; bp < P / 2; ++bp) {
        const f2x xy = mul2(o.xa[a], o.y2[bp]);
#pragma unroll
        for (int c = 0; c < P; ++c) v[a][bp][c] = add2(v[a][bp][c], add2(fma2c(xy, o.z2[c], m), mn));
      }
    }
  }
  __device__ __forceinline__ void row(int a, int b, float* out) const {
#pragma unroll
    for (int c = 0; c < P; ++c) out[c] = half2x(v[a][ypair<P>(b)][c], yhigh<P>(b));
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
  __device__ __forceinline__ void add_rounded(const Operands<P>& o) {
#pragma unroll
    for (int a = 0; a < P; ++a)
#pragma unroll
      for (int b = 0; b < P; ++b) {
        const float xy = o.wx[a] * o.wy[b];
#pragma unroll
        for (int c = 0; c < P; ++c) v[a][b][c] += fmaf(xy, o.wz[c], 12582912.0f) - 12582912.0f;
      }
  }
  __device__ __forceinline__ void row(int a, int b, float* out) const {
#pragma unroll
    for (int c = 0; c < P; ++c) out[c] = v[a][b][c];
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

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned source) from global memory into L2.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
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
// converted back from fixed point, to the grids, and clears them for the next tile. A thread takes
// whole z rows of RS = 12 nodes: three 16-byte shared loads and stores, then the nodes into the grid
// row. The tile's first z index cz0 is a multiple of 8 (even), so away from the periodic seam nodes
// 1..10 of a row form five pairs at even z, one 8-byte vector reduction each (row bases are 8-byte
// aligned: ldz even), and nodes 0 and 11 go alone; rows that wrap in z take one node at a time.
// Zero nodes are skipped.
template <int RZ>
__device__ __forceinline__ void flush_rows(int* reg, int ngrid, int cx0, int cy0, int cz0, int ng, int ldz,
                                           float inv_scale, float* g1, float* g2, int tid, int nthreads) {
  static_assert(RZ % 8 == 4, "rows of 8 k + 4 nodes: 16-byte aligned, pairs at even z inside");
  constexpr int Q = RZ / 4, VOL = RS * RS * RZ;
  const bool seam = cz0 == 0 || cz0 + RZ - 1 > ng;  // some node of a row wraps in z
  const int z0 = cz0 - 1;
  const int nrows = ngrid * RS * RS;
  for (int row = tid; row < nrows; row += nthreads) {
    const int gi = row >= RS * RS ? 1 : 0, rr = row - gi * (RS * RS);
    const int rx = rr / RS, ry = rr - rx * RS;
    int4* src = reinterpret_cast<int4*>(reg + gi * VOL + rr * RZ);
    int iv[RZ];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int4 v = src[q];
      src[q] = make_int4(0, 0, 0, 0);
      iv[4 * q] = v.x;
      iv[4 * q + 1] = v.y;
      iv[4 * q + 2] = v.z;
      iv[4 * q + 3] = v.w;
    }
    float* gg = (gi == 0 ? g1 : g2) + (int64_t(wrap(cx0 - 1 + rx, ng)) * ng + wrap(cy0 - 1 + ry, ng)) * ldz;
    if (!seam) {
      if (iv[0] != 0) atomicAdd(gg + z0, float(iv[0]) * inv_scale);
#pragma unroll
      for (int k = 1; k < RZ - 1; k += 2)
        if ((iv[k] | iv[k + 1]) != 0)
          asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(gg + z0 + k), "f"(float(iv[k]) * inv_scale),
                       "f"(float(iv[k + 1]) * inv_scale)
                       : "memory");
      if (iv[RZ - 1] != 0) atomicAdd(gg + z0 + RZ - 1, float(iv[RZ - 1]) * inv_scale);
    } else {
#pragma unroll
      for (int k = 0; k < RZ; ++k)
        if (iv[k] != 0) atomicAdd(gg + wrap(z0 + k, ng), float(iv[k]) * inv_scale);
    }
  }
}

__device__ __forceinline__ void flush_region(int* reg, int ngrid, int cx0, int cy0, int cz0, int ng, int ldz,
                                             float inv_scale, float* g1, float* g2, int tid, int nthreads) {
  static_assert(RS == 12 && (RVOL * 4) % 16 == 0, "rows of 12 nodes, 16-byte aligned");
  flush_rows<RS>(reg, ngrid, cx0, cy0, cz0, ng, ldz, inv_scale, g1, g2, tid, nthreads);
}

// The same for 64-bit regions (heavy tiles): rows of RS nodes, each node converted and added on its
// own (these tiles are few).
__device__ __forceinline__ void flush_region(long long* reg, int ngrid, int cx0, int cy0, int cz0, int ng, int ldz,
                                             float inv_scale, float* g1, float* g2, int tid, int nthreads) {
  const int nrows = ngrid * RS * RS;
  for (int row = tid; row < nrows; row += nthreads) {
    const int gi = row >= RS * RS ? 1 : 0, rr = row - gi * (RS * RS);
    const int rx = rr / RS, ry = rr - rx * RS;
    long long* src = reg + gi * RVOL + rr * RS;
    float* gg = (gi == 0 ? g1 : g2) + (int64_t(wrap(cx0 - 1 + rx, ng)) * ng + wrap(cy0 - 1 + ry, ng)) * ldz;
#pragma unroll
    for (int k = 0; k < RS; ++k) {
      const long long v = src[k];
      src[k] = 0;
      if (v != 0) atomicAdd(gg + wrap(cz0 - 1 + k, ng), float(v) * inv_scale);
    }
  }
}

// Any region (edge E, first node O below the tile) added to the grids node by node and cleared: the
// regions of orders 5 and 6 (rows of 14 nodes).
template <int E, int O, typename R>
__device__ __forceinline__ void flush_region_edge(R* reg, int ngrid, int cx0, int cy0, int cz0, int ng, int ldz,
                                                  float inv_scale, float* g1, float* g2, int tid, int nthreads) {
  constexpr int VOL = E * E * E;
  const int nrows = ngrid * E * E;
  for (int row = tid; row < nrows; row += nthreads) {
    const int gi = row >= E * E ? 1 : 0, rr = row - gi * (E * E);
    const int rx = rr / E, ry = rr - rx * E;
    R* src = reg + gi * VOL + rr * E;
    float* gg = (gi == 0 ? g1 : g2) + (int64_t(wrap(cx0 - O + rx, ng)) * ng + wrap(cy0 - O + ry, ng)) * ldz;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const R v = src[k];
      src[k] = 0;
      if (v != 0) atomicAdd(gg + wrap(cz0 - O + k, ng), float(v) * inv_scale);
    }
  }
}

// A region of the deterministic path added to its int64 grids node by node (integer additions in any
// order give the same sums) and cleared: edge RS in x and y, EZ along z, first node one below.
// A run's 32-bit region (scale 2^e) added to the int64 grids at the global scale 2^F, shift = F - e >= 0:
// integer sums of integers, so the result does not depend on the order of the additions.
template <int EZ>
__device__ __forceinline__ void flush_region_fixed(int* reg, int ngrid, int cx0, int cy0, int cz0, int ng, int ldz, int shift,
                                                   unsigned long long* g1, unsigned long long* g2, int tid, int nthreads) {
  constexpr int VOL = RS * RS * EZ;
  const int nrows = ngrid * RS * RS;
  for (int row = tid; row < nrows; row += nthreads) {
    const int gi = row >= RS * RS ? 1 : 0, rr = row - gi * (RS * RS);
    const int rx = rr / RS, ry = rr - rx * RS;
    int* src = reg + gi * VOL + rr * EZ;
    unsigned long long* gg = (gi == 0 ? g1 : g2) + (int64_t(wrap(cx0 - 1 + rx, ng)) * ng + wrap(cy0 - 1 + ry, ng)) * ldz;
#pragma unroll
    for (int k = 0; k < EZ; ++k) {
      const int v = src[k];
      src[k] = 0;
      if (v != 0) atomicAdd(gg + wrap(cz0 - 1 + k, ng), (unsigned long long)((long long)v * (1ll << shift)));
    }
  }
}

// Largest share of a particle's weight that one node receives: the peak of the one-dimensional
// window cubed (CIC and NGP 1, TSC 3/4 per axis, PCS 2/3 per axis).
template <int P>
__host__ __device__ constexpr float node_share() {
  // orders 5 and 6: centre values 115/192 and 11/20 of the one-dimensional B-spline, cubed, rounded up
  return P == 4 ? 8.0f / 27.0f : (P == 3 ? 27.0f / 64.0f : (P == 5 ? 0.2149f : (P == 6 ? 0.1664f : 1.0f)));
}

// Fixed-point scale 2^e of a tile's region: no node (nor any partial sum of one) exceeds
// node_share x the tile's total |weight| B, and that bound x 2^e < 2^30 leaves room for the rounding
// of every addition. With weights, B is summed by the block (red: one float per warp); the caller
// synchronises before the first use.
template <int P, bool W, int BITS = 30>
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
  frexpf(fmaxf(bound * node_share<P>(), 1.0f), &ex);  // node bound < 2^ex
  *scale = ldexpf(1.0f, BITS - ex);
  *inv_scale = ldexpf(1.0f, ex - BITS);
}

// Deterministic mode (k_assign_cells with int64 grids): the tile's scale 2^e with
//  - node share x count x max |w| x 2^e < 2^30: no node of the 32-bit region can overflow (a count and
//    a maximum, not a floating-point sum, so the scale does not depend on the order of the records);
//  - 32 products of at most node share x max |w| x 2^e < 2^(ex1 + e) each below 2^24: a window's
//    partial sums of kDetRun = 32 rounded products stay exact in FP32 (e <= 19 - ex1);
//  - e <= F, the global scale 2^F = fixed_scale(qsrc[2]); shift = F - e carries the tile's integers to it.
template <int P, bool W>
__device__ __forceinline__ void det_tile_scale(const float* w, int64_t beg, int64_t end, const double* qsrc, float* red,
                                               int nwarp, int tid, int nthreads, float* scale, int* shift) {
  float wmax = 1.0f;
  if (W) {
    float m = 0.0f;
    for (int64_t i = beg + tid; i < end; i += nthreads) m = fmaxf(m, fabsf(w[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    wmax = 0.0f;
    for (int q = 0; q < nwarp; ++q) wmax = fmaxf(wmax, red[q]);
  }
  int ex, ex1, fx;
  frexpf(fmaxf(float(end - beg) * wmax * node_share<P>(), 1.0f), &ex);  // node bound < 2^ex
  frexpf(fmaxf(wmax * node_share<P>(), 1e-30f), &ex1);                  // one product < 2^ex1
  frexpf(fixed_scale(qsrc[2]), &fx);                                     // 2^F = 2^(fx - 1)
  static_assert(kDetRun == 32, "the window bound below is for 32 products");
  const int e = min(min(30 - ex, 19 - ex1), fx - 1);
  *scale = ldexpf(1.0f, e);
  *shift = fx - 1 - e;
}

// The first tile t + k stride (k >= 0) below ntiles whose population end - beg lies in [lo, hi], else
// ntiles. Warp-parallel: 32 candidates per round of loads and a ballot; every lane of a full warp
// calls it with the same arguments and gets the same answer, so all warps of a block agree.
__device__ __forceinline__ int next_tile(const int64_t* toff, int64_t n, int t, int stride, int ntiles, int64_t lo,
                                         int64_t hi) {
  const int lane = threadIdx.x & 31;
  for (; t < ntiles; t += 32 * stride) {
    const int c = t + lane * stride;
    bool ok = false;
    if (c < ntiles) {
      const int64_t cnt = min(toff[c + 1], n) - max(toff[c], int64_t(0));
      ok = cnt >= lo && cnt <= hi;
    }
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if (m) return t + (__ffs(m) - 1) * stride;
  }
  return ntiles;
}

// ---- direct scatter (sparse tiles) ------------------------------------------------------------------
// Sorting a piece by key cell costs a fixed amount per piece (histograms, scans, the count order);
// on sparse tiles that fixed cost dominates. There, each thread adds its particles' p^3 weights per
// grid straight into the fixed-point region with integer shared atomics instead.
//
// Bank order. The region's rows are RS = 12 nodes and its planes 144 = 16 (mod 32) nodes, so the
// stencil node (a, b, c) of a particle whose first node has index q lies in bank
// (q + 16 a + 12 b + c) mod 32: two particles' additions meet in one bank at every step exactly when
// their q agree mod 32, and never otherwise. A piece's particles are therefore bucketed per grid by
// q mod 32, and round k gives lane l the k-th particle of bucket l, so the 32 additions of every
// warp instruction go to 32 different banks. For even p the stencil's planes pair up (a, a ^ 1), and
// a lane that adds plane a ^ 1 at step a moves all its additions by 16 banks: buckets are then taken
// mod 16, lanes l and l + 16 share bucket l mod 16 (its particles 2 k and 2 k + 1 in round k), and
// the lane whose bank half differs from its particle's flips the planes. Rounds then number the
// largest bucket's size over two instead of over one.
constexpr int SCATTER_THREADS = 256;

// Pieces of the scatter are staged in two buffers: the next piece is copied while this one is used.
// 768 records for runs of two or four tiles without weights (fewer barriers and bucket phases per
// record, fuller last rounds; the blocks per SM of the launch bounds still fit); 512 otherwise: with
// weights the buffers would not fit, and single tiles (four blocks per SM, 64 registers) would spill.
template <int P, bool W, typename R = int, int S = 1>
__host__ __device__ constexpr int scatter_chunk() {
  return (W || S == 1 || (P >= 5 && sizeof(R) == 8)) ? 512 : 768;
}

// Scatter region per order: nodes -1 .. T+2 of the tile (edge RS, first node one below the tile) up to
// PCS; orders 5 and 6 reach two nodes below and four above a cell on either grid: nodes -2 .. T+3.
template <int P>
__host__ __device__ constexpr int region_edge() {
  return P >= 5 ? T + 6 : RS;
}
template <int P>
__host__ __device__ constexpr int region_off() {
  return P >= 5 ? 2 : 1;
}
// Runs of S tiles along z share one region: its rows along z hold 8 S + 4 nodes.
template <int P, int S = 1>
__host__ __device__ constexpr int region_z() {
  return P >= 5 ? region_edge<P>() : T * S + 4;
}
template <int P, int S = 1>
__host__ __device__ constexpr int region_vol() {
  return region_edge<P>() * region_edge<P>() * region_z<P, S>();
}

// A finished scatter tile's region into the grids: rows of 12 nodes up to PCS, node by node beyond.
template <int P, int S, typename R>
__device__ __forceinline__ void flush_scatter_region(R* reg, int ngrid, int cx0, int cy0, int cz0, int ng, int ldz,
                                                     float inv_scale, float* g1, float* g2, int tid, int nthreads) {
  if constexpr (P >= 5 || sizeof(R) == 8) {
    static_assert(S == 1, "orders 5, 6 and 64-bit regions take single tiles");
    flush_region_edge<region_edge<P>(), region_off<P>()>(reg, ngrid, cx0, cy0, cz0, ng, ldz, inv_scale, g1, g2, tid, nthreads);
  } else {
    flush_rows<region_z<P, S>()>(reg, ngrid, cx0, cy0, cz0, ng, ldz, inv_scale, g1, g2, tid, nthreads);
  }
}

template <int P, bool W, typename R = int, int S = 1>
struct ScatterSmem {
  int4 sp[2][scatter_chunk<P, W, R, S>()];
  alignas(16) R reg[2][2][region_vol<P, S>()];  // two runs' regions in turn: one is flushed while the next is filled
  float red[2][SCATTER_THREADS / 32];
  unsigned long long mbar[2];
  float sw[2][W ? scatter_chunk<P, W, R, S>() : 1];
  // the piece's buckets per grid: counts (then cleared), sizes and offsets, the records in bucket order
  int cnt[2][32];
  int nr[2][32];
  int off[2][32];
  int rounds[2];
  unsigned short list[2][scatter_chunk<P, W, R, S>()];
};

// First stencil node on one axis of grid G, relative to the tile origin, for orders 5 and 6 (from the
// B-spline's own stencil start), with the weights.
template <int P, int G>
__device__ __forceinline__ int high_start(int l, float f, float* w) {
  float f2 = f;
  int d = 0;
  if constexpr (G == 1) d = half_shift(f, &f2);
  return l + d + bspline<P>(f2, w);
}

// Index of the region node where grid G's stencil of a particle at local cell (lx, ly, lz) + f starts.
template <int P, int G, int S = 1>
__device__ __forceinline__ int stencil_origin(int lx, int ly, int lz, float fx, float fy, float fz) {
  constexpr int E = region_edge<P>(), O = region_off<P>(), EZ = region_z<P, S>();
  if constexpr (P >= 5) {
    float w[P];
    const int sx = high_start<P, G>(lx, fx, w), sy = high_start<P, G>(ly, fy, w), sz = high_start<P, G>(lz, fz, w);
    return ((sx + O) * E + sy + O) * EZ + sz + O;
  } else {
    float t;
    const int kx = lx + grid_key<P, G>(fx, &t), ky = ly + grid_key<P, G>(fy, &t), kz = lz + grid_key<P, G>(fz, &t);
    return ((kx + s0<P>() + O) * E + ky + s0<P>() + O) * EZ + kz + s0<P>() + O;
  }
}

// Fixed-point value of one addition. For PCS and TSC the product is rounded to an integer by the FMA
// that adds 1.5 2^23 (the sum then lies in [2^23, 2^24], where the float's unit is 1, so its low
// mantissa bits hold the integer; exact for |v| <= 2^22, which scatter_scale guarantees), which runs
// on the FMA pipe instead of the conversion unit's quarter rate.
// float -> int64 rounded to nearest (ties away from zero) from the float's bits, in integer
// instructions: |v| = m 2^e with the 24-bit significand m. On this GPU the float -> int64 conversion
// runs on the FP64 pipe, a small fraction of the integer rate.
__device__ __forceinline__ long long float_to_ll(float v) {
  const int b = __float_as_int(v);
  const int e = ((b >> 23) & 0xff) - 150;  // v = m 2^e
  const long long m = (b & 0x7fffff) | 0x800000;
  long long r;
  if (e >= 0)
    r = m << min(e, 39);  // |v| < 2^63 for every value a region holds
  else if (e > -25)
    r = (m + (1ll << (-e - 1))) >> (-e);
  else
    r = 0;  // |v| < 1/2 (zero and subnormals included)
  return b < 0 ? -r : r;
}

template <int P, typename R>
__device__ __forceinline__ R fixed_product(float x, float y) {
  if constexpr (sizeof(R) == 8) {
    return float_to_ll(x * y);
  } else if constexpr (P >= 3) {
    return __float_as_int(fmaf(x, y, 12582912.0f)) - 0x4B400000;
  } else {
    return __float2int_rn(x * y);
  }
}

// Fixed-point value of one addition: through fixed_product, or (SUB) the bits of the subnormal product
// (mul.rn.f32 without .ftz keeps subnormal results whatever the compiler's flush-to-zero setting).
template <int P, typename R, bool SUB>
__device__ __forceinline__ R node_value(float xy, float z) {
  if constexpr (SUB) {
    float r;
    asm("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(xy), "f"(z));
    return __float_as_int(r);
  } else {
    return fixed_product<P, R>(xy, z);
  }
}

// Buckets of the bank order: 16 for even p on the 12-node region (plane pairs 16 banks apart), 32
// otherwise; lanes per bucket.
template <int P, typename R = int>
__host__ __device__ constexpr bool flip_planes() {
  return sizeof(R) == 4 && P % 2 == 0 && region_edge<P>() == 12;  // 12 (8 S + 4) = 16 (mod 32) for every S
}
// 64-bit regions: a node spans two banks, so the bank pair of node q is q mod 16, and the two halves of
// a warp (served in turn) each take one record of every bucket mod 16.
template <int P, typename R = int>
__host__ __device__ constexpr int bank_buckets() {
  return sizeof(R) == 8 ? 16 : (flip_planes<P, R>() ? 16 : 32);
}

// Adds one particle's p^3 weights on grid G to that grid's region (scale: the weight times the
// region's fixed-point scale). Region nodes of the stencil: key + S0 + 1 .. key + S0 + p per axis.
// lane: the caller's lane; for even p the planes are taken in pairs swapped when the lane's bank half
// differs from the stencil origin's (the bank order above).
// NN (unit weights: every product >= 0) with orders 3..6 and 32-bit regions: the products are rounded
// to integers by the multiply itself. With the x weights scaled by 2^-100 and the z weights by 2^-49
// (both exact, the operands stay normal), x y z 2^-149 falls in the subnormal range, whose spacing
// is 2^-149: the multiply rounds it (to nearest, ties to even) to m 2^-149 with m = round(x y z), and
// the float's bits are m itself (every addition stays below 2^22 < 2^23, scatter_scale's cap). The
// same integers as the 1.5 2^23 addition of fixed_product, without its bias subtraction.
template <int P, typename R, bool NN>
__host__ __device__ constexpr bool subnormal_rounding() {
  return NN && P >= 3 && sizeof(R) == 4;
}

template <int P, int G, int S, typename R, bool NN = false>
__device__ __forceinline__ void scatter_particle(R* reg, int lx, int ly, int lz, float fx, float fy, float fz, float sc,
                                                 int lane) {
  constexpr bool SUB = subnormal_rounding<P, R, NN>();
  if constexpr (P >= 5) {  // orders 5 and 6: the B-spline weights and stencil start per axis
    constexpr int E = region_edge<P>(), O = region_off<P>();
    float wx[P], wy[P], wz[P];
    const int sx = high_start<P, G>(lx, fx, wx), sy = high_start<P, G>(ly, fy, wy), sz = high_start<P, G>(lz, fz, wz);
#pragma unroll
    for (int a = 0; a < P; ++a) wx[a] *= SUB ? sc * 0x1p-100f : sc;
    if constexpr (SUB)
#pragma unroll
      for (int c = 0; c < P; ++c) wz[c] *= 0x1p-49f;
    static_assert(S == 1, "orders 5 and 6 take single tiles");
    const unsigned base = smem_u32(reg + ((sx + O) * E + sy + O) * E + sz + O);
#pragma unroll
    for (int a = 0; a < P; ++a)
#pragma unroll
      for (int b = 0; b < P; ++b) {
        const float xy = wx[a] * wy[b];
#pragma unroll
        for (int c = 0; c < P; ++c)
          red_shared(base + unsigned(sizeof(R)) * ((a * E + b) * E + c), node_value<P, R, SUB>(xy, wz[c]));
      }
  } else {
    float tx, ty, tz;
    const int kx = lx + grid_key<P, G>(fx, &tx), ky = ly + grid_key<P, G>(fy, &ty), kz = lz + grid_key<P, G>(fz, &tz);
    float wx[P], wy[P], wz[P];
    weights<P>(tx, wx);
    weights<P>(ty, wy);
    weights<P>(tz, wz);
#pragma unroll
    for (int a = 0; a < P; ++a) wx[a] *= SUB ? sc * 0x1p-100f : sc;
    if constexpr (SUB)
#pragma unroll
      for (int c = 0; c < P; ++c) wz[c] *= 0x1p-49f;
    constexpr int EZ = region_z<P, S>();  // rows along z; planes RS EZ nodes apart (16 mod 32)
    const int q = ((kx + s0<P>() + 1) * RS + ky + s0<P>() + 1) * EZ + kz + s0<P>() + 1;
    unsigned base_even = smem_u32(reg + q), base_odd = base_even;
    if constexpr (flip_planes<P, R>()) {
      if ((q ^ lane) & 16) {  // step a adds plane a ^ 1
#pragma unroll
        for (int a = 0; a < P; a += 2) {
          const float t = wx[a];
          wx[a] = wx[a + 1];
          wx[a + 1] = t;
        }
        base_even += unsigned(sizeof(R)) * RS * EZ;
        base_odd -= unsigned(sizeof(R)) * RS * EZ;
      }
    }
#pragma unroll
    for (int a = 0; a < P; ++a) {
      const unsigned base = (a & 1) ? base_odd : base_even;
#pragma unroll
      for (int b = 0; b < P; ++b) {
        const float xy = wx[a] * wy[b];
#pragma unroll
        for (int c = 0; c < P; ++c)
          red_shared(base + unsigned(sizeof(R)) * ((a * RS + b) * EZ + c), node_value<P, R, SUB>(xy, wz[c]));
      }
    }
  }
}

// Fixed-point scale 2^e of a sparse tile's region: tile_scale's bound (node share x total |weight| x
// 2^e < 2^30) and, where fixed_product rounds by the 1.5 2^23 addition, node share x max |weight| x
// 2^e <= 2^22 for every single addition. With weights the block reduces the sum and the maximum
// (red: two floats per warp); the caller synchronises before the first use.
// DET (the deterministic path): the bound is the particle count times max |w| (a maximum does not
// depend on the order of the records, a floating-point sum may), and the exponent is capped at emax
// (the global scale's), so that every run's scale divides the global one.
template <int P, bool W, typename R, int S, bool DET = false>
__device__ __forceinline__ void scatter_scale(const float* w, const int64_t (&beg)[S], const int64_t (&end)[S],
                                              float (*red)[SCATTER_THREADS / 32], int tid, float* scale, float* inv_scale,
                                              int emax = 127) {
  constexpr int NW = SCATTER_THREADS / 32;
  float bound = 0.0f, wmax = 1.0f;
#pragma unroll
  for (int q = 0; q < S; ++q) bound += float(end[q] - beg[q]);
  const float count = bound;
  if (W) {
    float a = 0.0f, m = 0.0f;
#pragma unroll
    for (int q = 0; q < S; ++q)
      for (int64_t i = beg[q] + tid; i < end[q]; i += SCATTER_THREADS) {
        a += fabsf(w[i]);
        m = fmaxf(m, fabsf(w[i]));
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = a;
      red[1][tid >> 5] = m;
    }
    __syncthreads();
    bound = 0.0f;
    wmax = 0.0f;
    for (int q = 0; q < NW; ++q) {
      bound += red[0][q];
      wmax = fmaxf(wmax, red[1][q]);
    }
    bound = DET ? count * wmax : bound * 1.0001f;  // (the FP32 sum's rounding)
  }
  int ex;
  frexpf(fmaxf(bound * node_share<P>(), 1.0f), &ex);  // node bound < 2^ex
  int e = (sizeof(R) == 8 ? 62 : 30) - ex;
  if (P >= 3 && sizeof(R) == 4) {
    int ex1;
    frexpf(fmaxf(wmax * node_share<P>(), 1e-30f), &ex1);  // one addition < 2^ex1
    e = min(e, 22 - ex1);
  }
  e = min(e, emax);
  *scale = ldexpf(1.0f, e);
  *inv_scale = ldexpf(1.0f, -e);
}

}  // namespace tiles

// The first run r + k stride (k >= 0) below nruns holding a tile of lo .. hi particles, else nruns. A
// run is S tiles consecutive along z (tile index (t_x N_t + t_y) N_t + t_z, so its tiles are
// consecutive indices). Warp-parallel as next_tile.
template <int S>
__device__ __forceinline__ int next_run(const int64_t* toff, int64_t n, int r, int stride, int nruns, int64_t lo, int64_t hi) {
  const int lane = threadIdx.x & 31;
  for (; r < nruns; r += 32 * stride) {
    const int c = r + lane * stride;
    bool ok = false;
    if (c < nruns)
#pragma unroll
      for (int q = 0; q < S; ++q) {
        const int64_t cnt = min(toff[c * S + q + 1], n) - max(toff[c * S + q], int64_t(0));
        ok |= cnt >= lo && cnt <= hi;
      }
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if (m) return r + (__ffs(m) - 1) * stride;
  }
  return nruns;
}

// Blocks per SM of the scatter's launch bounds.
template <int P, typename R, int S>
__host__ __device__ constexpr int scatter_blocks() {
  return (P >= 5 || sizeof(R) == 8 || S >= 4) ? 2 : (S == 2 ? 3 : 4);
}

// a3, FP32, direct scatter: a block takes runs of S tiles along z (one region per run) in a
// grid-stride sequence, and the runs' pieces in order, the copy of the next piece overlapping the use
// of the current one. A piece is up to CH consecutive records of the run's tiles of min_count ..
// max_count particles (tiles of the run outside that range, taken by the key-cell kernel, split the
// run into segments; a piece never spans two). Per piece: each record's stencil origin on each grid
// is bucketed by bank (counts with shared atomics, which also give the record's place in its bucket);
// one warp per grid turns the counts into offsets; the records are listed in bucket order; then the
// warps take rounds (grid 1's, then grid 2's), lane l of round k scattering the k-th record of
// bucket l (even p: record 2 k + l / 16 of bucket l mod 16). Runs use two regions in turn: a finished
// run's region is added to the grids (and cleared) in the bucket phase of the next piece. The block
// barrier at the top of each piece separates every use of the staging buffers, buckets and regions.
// (The tiles of a run are consecutive along z, so the tile index is (t_x N_t + t_y) N_t + t_z and a
// run is S consecutive indices; S divides N_t.)
// GT: the grids' element type. float: FP32 grids, the region's fixed-point scale per run; unsigned
// long long (PK_FIXED64, R = long long): int64 grids at the one scale 2^F from qsrc[2] = sum |w|
// (fixed_scale), every contribution rounded on its own, so the sums do not depend on the order.
template <int P, bool W, typename R, int S, typename GT = float>
__global__ void __launch_bounds__(tiles::SCATTER_THREADS, scatter_blocks<P, R, S>())
    k_assign_scatter(const pk_cellpos* __restrict__ p, const float* __restrict__ w, const int64_t* __restrict__ toff,
                     int64_t n, int ng, int ntile, int interlace, GT* __restrict__ g1, GT* __restrict__ g2, int ldz,
                     int64_t cat_stride, int64_t min_count, int64_t max_count, int ncat, const double* __restrict__ qsrc = nullptr) {
  constexpr bool FX = sizeof(GT) == 8;
  static_assert(!FX || (sizeof(R) == 4 && S == 1 && P <= 4), "the deterministic path: 32-bit regions, single tiles");
  using namespace tiles;
  constexpr int CH = scatter_chunk<P, W, R, S>(), THREADS = SCATTER_THREADS, NWARP = THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem<P, W, R, S>& Sm = *reinterpret_cast<ScatterSmem<P, W, R, S>*>(smem_raw);
  const int ngrid = interlace ? 2 : 1;
  // runs of all catalogues of a batch in one sequence: run R of catalogue R / nruns_cat covers the tiles
  // R S .. R S + S - 1 of the catalogues' consecutive tile offsets, so the blocks share every catalogue
  const int nruns_cat = ntile * ntile * (ntile / S), nruns = ncat * nruns_cat;
  const int tid = threadIdx.x;
  if (tid < 2) {
    const unsigned b = static_cast<unsigned>(__cvta_generic_to_shared(&Sm.mbar[tid]));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  }
  for (int i = tid; i < 2 * 2 * region_vol<P, S>(); i += THREADS) (&Sm.reg[0][0][0])[i] = 0;
  if (tid < 64) (&Sm.cnt[0][0])[tid] = 0;
  __syncthreads();
  auto in_range = [&](int t) {
    const int64_t c = min(toff[t + 1], n) - max(toff[t], int64_t(0));
    return c >= min_count && c <= max_count;
  };
  // the block's pieces: run, next tile of the run after the current segment, the segment's records
  // [c0 ..., end), and whether the piece is the run's first (called by every thread alike)
  struct Piece {
    int run, snext;
    int64_t end, c0;
    bool first;
  };
  auto advance = [&](Piece& c) -> bool {
    c.c0 += CH;
    c.first = false;
    if (c.c0 < c.end) return true;
    int q = c.snext;
    while (true) {
      while (q < S && !in_range(c.run * S + q)) ++q;
      if (q < S) break;
      c.run = next_run<S>(toff, n, c.run + int(gridDim.x), int(gridDim.x), nruns, min_count, max_count);
      if (c.run >= nruns) return false;
      q = 0;
      c.first = true;
    }
    int e = q;
    while (e + 1 < S && in_range(c.run * S + e + 1)) ++e;
    c.c0 = max(toff[c.run * S + q], int64_t(0));
    c.end = min(toff[c.run * S + e + 1], n);
    c.snext = e + 1;
    return true;
  };
  Piece cur;
  cur.run = int(blockIdx.x) - int(gridDim.x);
  cur.snext = S;
  cur.end = 0;
  cur.c0 = -CH;
  cur.first = false;
  if (!advance(cur)) return;
  if (tid == 0) bulk_load(Sm.sp[0], p + cur.c0, unsigned(min(int64_t(CH), cur.end - cur.c0)) * 16u, &Sm.mbar[0]);
  if (W)
    for (int i = tid; i < int(min(int64_t(CH), cur.end - cur.c0)); i += THREADS) Sm.sw[0][i] = w[cur.c0 + i];
  Piece nxt = cur;
  bool has_next = advance(nxt);
  unsigned parity = 0u;  // bit b: the phase buffer b waits for next
  int buf = 0;
  int rb = 1;  // region of the current run (switched at each run's first piece)
  float scale = 1.0f, inv_scale = 1.0f;
  int cx0 = 0, cy0 = 0, cz0 = 0;
  bool pending = false;  // the previous run's region (rb ^ 1) is still to be flushed
  int pcx0 = 0, pcy0 = 0, pcz0 = 0;
  int ccat = 0, pcat = 0;  // catalogues of the current and of the pending run
  float pinv = 1.0f;
  while (true) {
    const int m = int(min(int64_t(CH), cur.end - cur.c0));
    const bool arrived = bulk_wait(&Sm.mbar[buf], (parity >> buf) & 1u);
    parity ^= 1u << buf;
    if (__syncthreads_or(!arrived)) {  // a copy did not complete: report, drain what is in flight, stop
      if (tid == 0) {
        raise_err(PK_DERR_TIMEOUT);
        bulk_wait(&Sm.mbar[buf], ((parity >> buf) & 1u) ^ 1u);
      }
      return;
    }
    // every use of the other buffer and of the flushed region ended before the barrier above
    if (has_next) {
      const int mn = int(min(int64_t(CH), nxt.end - nxt.c0));
      if (tid == 0) bulk_load(Sm.sp[buf ^ 1], p + nxt.c0, unsigned(mn) * 16u, &Sm.mbar[buf ^ 1]);
      if (W)
        for (int i = tid; i < mn; i += THREADS) Sm.sw[buf ^ 1][i] = w[nxt.c0 + i];
    }
    if (cur.first) {  // first piece of a run: the other region, the run's origin and scale
      rb ^= 1;
      const int cat = cur.run / nruns_cat, run = cur.run - cat * nruns_cat;
      ccat = cat;
      const int rz = run % (ntile / S), ty = (run / (ntile / S)) % ntile, tx = run / ((ntile / S) * ntile);
      cx0 = tx * T;
      cy0 = ty * T;
      cz0 = rz * S * T;
      int64_t rbeg[S], rend[S];
#pragma unroll
      for (int q = 0; q < S; ++q) {
        const int t = cur.run * S + q;
        const bool on = in_range(t);
        rbeg[q] = on ? max(toff[t], int64_t(0)) : 0;
        rend[q] = on ? min(toff[t + 1], n) : 0;
      }
      if constexpr (FX) {  // the run's scale 2^e (e <= F) and the shift F - e to the global scale 2^F
        int fx;
        frexpf(fixed_scale(qsrc[2]), &fx);
        scatter_scale<P, W, R, S, true>(w, rbeg, rend, Sm.red, tid, &scale, &inv_scale, fx - 1);
        int es;
        frexpf(scale, &es);
        inv_scale = __int_as_float(fx - es);  // the shift F - e, carried in the float's bits
      } else {
        scatter_scale<P, W, R, S>(w, rbeg, rend, Sm.red, tid, &scale, &inv_scale);
      }
    }
    if (pending) {
      if constexpr (FX)
        flush_region_fixed<region_z<P, S>()>(&Sm.reg[rb ^ 1][0][0], ngrid, pcx0, pcy0, pcz0, ng, ldz, __float_as_int(pinv),
                                             g1 + pcat * cat_stride, g2 ? g2 + pcat * cat_stride : nullptr, tid, THREADS);
      else
        flush_scatter_region<P, S>(&Sm.reg[rb ^ 1][0][0], ngrid, pcx0, pcy0, pcz0, ng, ldz, pinv, g1 + pcat * cat_stride,
                                   g2 ? g2 + pcat * cat_stride : nullptr, tid, THREADS);
      pending = false;
    }
    const int4* sp = Sm.sp[buf];
    const float* sw = Sm.sw[buf];
    // buckets: stencil origin mod NB per grid, and the record's place in its bucket
    constexpr int PER = (CH + THREADS - 1) / THREADS, NB = bank_buckets<P, R>(), LPB = 32 / NB;
    int qb[PER][2], rk[PER][2];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int j = tid + u * THREADS;
      qb[u][0] = -1;
      if (j < m) {
        const int4 r = sp[j];
        const uint32_t cell = uint32_t(r.x);
        const int lx = cell_x(cell) - cx0, ly = cell_y(cell) - cy0, lz = cell_z(cell) - cz0;
        if ((cell >> 30) != 0 || unsigned(lx) >= unsigned(T) || unsigned(ly) >= unsigned(T) || unsigned(lz) >= unsigned(S * T)) {
          raise_err(PK_DERR_CELLRANGE);
          continue;
        }
        const float fx = __int_as_float(r.y), fy = __int_as_float(r.z), fz = __int_as_float(r.w);
        qb[u][0] = stencil_origin<P, 0, S>(lx, ly, lz, fx, fy, fz) & (NB - 1);
        rk[u][0] = atomicAdd(&Sm.cnt[0][qb[u][0]], 1);
        if (interlace) {  // both grids' records share the buckets (one pool, one set of rounds)
          qb[u][1] = stencil_origin<P, 1, S>(lx, ly, lz, fx, fy, fz) & (NB - 1);
          rk[u][1] = atomicAdd(&Sm.cnt[0][qb[u][1]], 1);
        }
      }
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {  // the pool's bucket offsets, sizes and round count; counts cleared
      const int c = lane < NB ? Sm.cnt[warp][lane] : 0;
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      int mx = (c + LPB - 1) / LPB;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane < NB) {
        Sm.off[warp][lane] = incl - c;
        Sm.nr[warp][lane] = c;
        Sm.cnt[warp][lane] = 0;
      }
      if (lane == 0) Sm.rounds[warp] = mx;
    }
    __syncthreads();
    unsigned short* list = &Sm.list[0][0];  // the pool: record index, grid in bit 15
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      if (qb[u][0] < 0) continue;
      const unsigned short j = static_cast<unsigned short>(tid + u * THREADS);
      list[Sm.off[0][qb[u][0]] + rk[u][0]] = j;
      if (interlace) list[Sm.off[0][qb[u][1]] + rk[u][1]] = static_cast<unsigned short>(j | 0x8000u);
    }
    __syncthreads();
    // rounds of the pool, dealt to the warps in turn; a lane's grid is that of its record
    const int rtot = Sm.rounds[0];
    for (int item = warp; item < rtot; item += NWARP) {
      const int k = item * LPB + lane / NB, bkt = lane % NB;
      if (k >= Sm.nr[0][bkt]) continue;
      const int e = list[Sm.off[0][bkt] + k];
      const int j = e & 0x7fff, g = e >> 15;
      const int4 r = sp[j];
      const uint32_t cell = uint32_t(r.x);
      int lx = cell_x(cell) - cx0, ly = cell_y(cell) - cy0, lz = cell_z(cell) - cz0;
      float fx = __int_as_float(r.y), fy = __int_as_float(r.z), fz = __int_as_float(r.w);
      const float sc = (W ? sw[j] : 1.0f) * weight_scale<P>() * scale;
      if (g) {  // grid 2 samples the particle shifted by H/2: grid 1's stencil of the shifted position
        float f2;
        lx += half_shift(fx, &f2);
        fx = f2;
        ly += half_shift(fy, &f2);
        fy = f2;
        lz += half_shift(fz, &f2);
        fz = f2;
      }
      scatter_particle<P, 0, S, R, !W>(Sm.reg[rb][g], lx, ly, lz, fx, fy, fz, sc, lane);
    }
    if (!has_next || nxt.first) {  // last piece of the run: its region is flushed with the next piece
      pending = true;
      pcx0 = cx0;
      pcat = ccat;
      pcy0 = cy0;
      pcz0 = cz0;
      pinv = inv_scale;
    }
    if (!has_next) break;
    cur = nxt;
    buf ^= 1;
    has_next = advance(nxt);
  }
  __syncthreads();
  if (pending) {
    if constexpr (FX)
      flush_region_fixed<region_z<P, S>()>(&Sm.reg[rb][0][0], ngrid, pcx0, pcy0, pcz0, ng, ldz, __float_as_int(pinv),
                                           g1 + pcat * cat_stride, g2 ? g2 + pcat * cat_stride : nullptr, tid, THREADS);
    else
      flush_scatter_region<P, S>(&Sm.reg[rb][0][0], ngrid, pcx0, pcy0, pcz0, ng, ldz, pinv, g1 + pcat * cat_stride,
                                 g2 ? g2 + pcat * cat_stride : nullptr, tid, THREADS);
  }
}

// ---- cells (dense tiles) ---------------------------------------------------------------------------
// Per staged piece of a tile the particles are counting-sorted by key cell on each grid; each grid's
// non-empty key cells then form a list ordered by particle count, largest first. Even warps take grid
// 1's list and odd warps grid 2's (all warps grid 1's without interlacing); thread t of a grid's nt
// threads takes item t of each round of nt items in even rounds and item nt - 1 - t in odd ones, so
// the 32 lanes of a warp hold cells of nearly equal load and the warps' totals even out. A lane sums
// its cell's particles into a register window of p^3 node values (the cell's whole stencil) and adds
// the window to the tile's fixed-point region once. Pieces need no order inside the tile.
namespace tiles {
constexpr int CELL_THREADS = 256;
constexpr int CNT_BINS = 64;  // particle counts above 63 share the first place of the ordering

// Records per piece: a key cell's window is added to the region once per piece, so larger pieces
// mean fewer (and fuller) additions and fewer per-piece sorts. 32-bit regions: the largest piece at
// which two blocks still fit an SM's 228 KB (20 B per record, 24 with weights, beside ~23 KB of
// histograms, lists and regions): 4608 records, so that a tile of the mean population 8^3 x 8 = 4096
// and most of the Poisson and clustering spread above it take one piece. 64-bit regions (heavy tiles,
// one block per SM): 8192.
template <bool W, typename R = int>
__host__ __device__ constexpr int cell_chunk() {
  return sizeof(R) == 8 ? (W ? 4096 : 8192) : (W ? 3840 : 4608);
}

// R: the region's integer type, int (32-bit fixed point) or long long (64-bit, the heavy tiles).
template <bool W, typename R = int>
struct CellSmem {
  int4 sp[cell_chunk<W, R>()];
  unsigned short perm[2][cell_chunk<W, R>()];
  int hist[2][NKEY + 1];  // counts -> exclusive offsets -> bucket ends
  alignas(16) R reg[2][RVOL];
  unsigned short order[2][NKEY];  // non-empty key cells per grid, largest bucket first
  int cbin[2][CNT_BINS];
  int nitems[2];
  float red[CELL_THREADS / 32];
  int scan[2][CELL_THREADS / 32];
  unsigned long long mbar;
  float sw[W ? cell_chunk<W, R>() : 1];
};

// One key cell of grid G: its bucket of particles into a register window, then the window into the
// region (nodes key + S0 + 1 .. key + S0 + p per axis). The fixed-point scale (a power of two) rides
// on the particle weight, so the window already holds fixed-point values; the next record is loaded
// before the current one is accumulated.
template <int P, bool W, typename R, int G>
__device__ __forceinline__ void add_window(const CellSmem<W, R>& S, const Window<P>& win, unsigned base) {
#pragma unroll
  for (int a = 0; a < P; ++a)
#pragma unroll
    for (int b = 0; b < P; ++b) {
      float v[P];
      win.row(a, b, v);
#pragma unroll
      for (int c = 0; c < P; ++c)
        red_shared(base + unsigned(sizeof(R)) * ((a * RS + b) * RS + c), to_fixed(v[c], static_cast<R*>(nullptr)));
    }
}

template <int P, bool W, typename R, int G, bool DET = false>
__device__ __forceinline__ void cell_key(const CellSmem<W, R>& S, int key, float wscale) {
  const int* ends = S.hist[G];
  const unsigned short* perm = S.perm[G];
  const int jb = key == 0 ? 0 : ends[key - 1], je = ends[key];
  const int kx = key % K, kz = (key / K) % K, ky = key / (K * K);
  const unsigned base =
      smem_u32(&S.reg[G][0] + ((kx + s0<P>() + 1) * RS + ky + s0<P>() + 1) * RS + kz + s0<P>() + 1);
  if constexpr (DET) {
    // every product rounded to an integer, at most kDetRun particles per window (partial sums < 2^24,
    // exact in FP32), so the region receives the same integers in any order
    for (int j0 = jb; j0 < je; j0 += kDetRun) {
      const int j1 = min(je, j0 + kDetRun);
      Window<P> win;
      win.zero();
      for (int j = j0; j < j1; ++j) {
        const int i = perm[j];
        win.add_rounded(particle_operands<P, G>(S.sp[i], (W ? S.sw[i] : 1.0f) * wscale));
      }
      add_window<P, W, R, G>(S, win, base);
    }
  } else {
    Window<P> win;
    win.zero();
    int4 r = make_int4(0, 0, 0, 0);
    float rw = 1.0f;
    if (jb < je) {
      const int i = perm[jb];
      r = S.sp[i];
      if (W) rw = S.sw[i];
    }
    for (int j = jb; j < je; ++j) {
      const int4 c = r;
      const float cw = rw;
      if (j + 1 < je) {
        const int i = perm[j + 1];
        r = S.sp[i];
        if (W) rw = S.sw[i];
      }
      win.add(particle_operands<P, G>(c, cw * wscale));
    }
    add_window<P, W, R, G>(S, win, base);
  }
}
}  // namespace tiles

static_assert(2 * (sizeof(tiles::CellSmem<false, int>) + 1024) <= 233472 &&
                  2 * (sizeof(tiles::CellSmem<true, int>) + 1024) <= 233472,
              "two key-cell blocks (32-bit regions) per SM");

// GT: the grids' element type. float: FP32 grids. unsigned long long (PK_FIXED64, R = int): int64 grids
// at the one scale 2^F from qsrc[2] = sum |w|; every product is rounded to an integer at the tile's
// scale 2^e <= 2^F (det_tile_scale) and the integers are summed exactly, so the grids do not depend on
// the order of the records or of the additions.
template <int P, bool W, typename R, typename GT = float>
__global__ void __launch_bounds__(tiles::CELL_THREADS, 2)
    k_assign_cells(const pk_cellpos* __restrict__ p, const float* __restrict__ w, const int64_t* __restrict__ toff, int64_t n,
                   int ng, int ntile, int interlace, GT* __restrict__ g1, GT* __restrict__ g2, int ldz,
                   int64_t cat_stride, int64_t min_count, int64_t max_count, int ncat, const double* __restrict__ qsrc = nullptr) {
  using namespace tiles;
  constexpr bool DET = sizeof(GT) == 8;
  static_assert(!DET || sizeof(R) == 4, "the deterministic mode: 32-bit regions");
  constexpr int CH = cell_chunk<W, R>(), THREADS = CELL_THREADS, NWARP = THREADS / 32;
  constexpr int SCAN_PER_THREAD = (NKEY + 1 + THREADS - 1) / THREADS;
  static_assert(CNT_BINS == 64, "count bins: two per lane of one warp");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CellSmem<W, R>& S = *reinterpret_cast<CellSmem<W, R>*>(smem_raw);
  constexpr int BITS = sizeof(R) == 8 ? 62 : 30;  // node bound x scale < 2^BITS
  const int ngrid = interlace ? 2 : 1;
  // the tiles of all catalogues of a batch in one sequence (catalogue t / ntiles_cat, consecutive offsets)
  const int ntiles_cat = ntile * ntile * ntile, ntiles = ncat * ntiles_cat;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    const unsigned b = static_cast<unsigned>(__cvta_generic_to_shared(&S.mbar));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  }
  for (int i = tid; i < 2 * RVOL; i += THREADS) (&S.reg[0][0])[i] = 0;  // flush_region clears it after each tile
  __syncthreads();
  unsigned parity = 0;
  // the block's tiles of min_count .. max_count particles (the scatter takes the sparser ones, the 64-bit
  // instance of this kernel the heavier ones)
  for (int tile = next_tile(toff, n, blockIdx.x, gridDim.x, ntiles, min_count, max_count), nt = 0; tile < ntiles; tile = nt) {
    nt = next_tile(toff, n, tile + int(gridDim.x), int(gridDim.x), ntiles, min_count, max_count);
    const int64_t beg = max(toff[tile], int64_t(0)), end = min(toff[tile + 1], n);
    const int cat = tile / ntiles_cat, lt = tile - cat * ntiles_cat;
    GT* const cg1 = g1 + cat * cat_stride;
    GT* const cg2 = g2 ? g2 + cat * cat_stride : nullptr;
    const int tz = lt % ntile, ty = (lt / ntile) % ntile, tx = lt / (ntile * ntile);
    const int cx0 = tx * T, cy0 = ty * T, cz0 = tz * T;  // first cell of the tile
    float scale, inv_scale;
    int shift = 0;  // deterministic mode: F - e
    if constexpr (DET)
      det_tile_scale<P, W>(w, beg, end, qsrc, S.red, NWARP, tid, THREADS, &scale, &shift);
    else
      tile_scale<P, W, BITS>(w, beg, end, S.red, NWARP, tid, THREADS, &scale, &inv_scale);
    const float wscale = scale * weight_scale<P>();
    for (int64_t c0 = beg; c0 < end; c0 += CH) {
      const int m = int(min(int64_t(CH), end - c0));
      if (tid == 0) {
        bulk_load(S.sp, p + c0, unsigned(m) * 16u, &S.mbar);
        // the block's next piece (of this tile, else of its next tile) moves to L2 meanwhile
        int64_t nb = c0 + CH, ne = end;
        if (nb >= ne && nt < ntiles) {
          nb = max(toff[nt], int64_t(0));
          ne = min(toff[nt + 1], n);
        }
        if (nb < ne) bulk_prefetch_l2(p + nb, unsigned(min(int64_t(CH), ne - nb)) * 16u);
      }
      if (W)
        for (int i = tid; i < m; i += THREADS) S.sw[i] = w[c0 + i];
      for (int i = tid; i < 2 * (NKEY + 1); i += THREADS) (&S.hist[0][0])[i] = 0;
      if (tid < 2 * CNT_BINS) (&S.cbin[0][0])[tid] = 0;
      const bool arrived = bulk_wait(&S.mbar, parity);
      parity ^= 1u;
      if (__syncthreads_or(!arrived)) {  // the copy did not complete: report, drain, stop
        if (tid == 0) {
          raise_err(PK_DERR_TIMEOUT);
          bulk_wait(&S.mbar, parity ^ 1u);
        }
        return;
      }
      // key cells of both grids (the record's cell word becomes the two keys, or -1 when skipped);
      // four records per thread and pass, loaded before any is used
      for (int i0 = tid; i0 < m; i0 += 4 * THREADS) {
        int4 r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) r[u] = i0 + u * THREADS < m ? S.sp[i0 + u * THREADS] : make_int4(-1, 0, 0, 0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * THREADS;
          if (i >= m) break;
          const uint32_t cell = uint32_t(r[u].x);
          const int lx = cell_x(cell) - cx0, ly = cell_y(cell) - cy0, lz = cell_z(cell) - cz0;
          if ((cell >> 30) == 0 && unsigned(lx) < unsigned(T) && unsigned(ly) < unsigned(T) && unsigned(lz) < unsigned(T)) {
            float t;
            const float fx = __int_as_float(r[u].y), fy = __int_as_float(r[u].z), fz = __int_as_float(r[u].w);
            const int k1 =
                ((ly + grid_key<P, 0>(fy, &t)) * K + (lz + grid_key<P, 0>(fz, &t))) * K + lx + grid_key<P, 0>(fx, &t);
            atomicAdd(&S.hist[0][k1], 1);
            int k2 = 0;
            if (interlace) {
              k2 = ((ly + grid_key<P, 1>(fy, &t)) * K + (lz + grid_key<P, 1>(fz, &t))) * K + lx + grid_key<P, 1>(fx, &t);
              atomicAdd(&S.hist[1][k2], 1);
            }
            S.sp[i].x = k1 | (k2 << 16);
          } else {
            raise_err(PK_DERR_CELLRANGE);
            S.sp[i].x = -1;
          }
        }
      }
      __syncthreads();
      // Counts of both histograms, read once: the non-empty key cells are counted by bucket size
      // (bin 0: the largest) and the warps scan the counts.
      int v0[SCAN_PER_THREAD], v1[SCAN_PER_THREAD];
      int x0, x1, s0v = 0, s1v = 0;
#pragma unroll
      for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        const int idx = tid * SCAN_PER_THREAD + k;
        v0[k] = idx <= NKEY ? S.hist[0][idx] : 0;
        v1[k] = idx <= NKEY ? S.hist[1][idx] : 0;
        if (v0[k] > 0) atomicAdd(&S.cbin[0][CNT_BINS - 1 - min(v0[k], CNT_BINS - 1)], 1);  // entry NKEY is 0
        if (v1[k] > 0) atomicAdd(&S.cbin[1][CNT_BINS - 1 - min(v1[k], CNT_BINS - 1)], 1);
        s0v += v0[k];
        s1v += v1[k];
      }
      x0 = s0v;
      x1 = s1v;
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
      // exclusive offsets of both histograms; warp g scans grid g's count bins (64 bins, two per lane)
      if (warp < 2) {
        int* cb = S.cbin[warp];
        const int a0 = cb[2 * lane], a1 = cb[2 * lane + 1];
        int x = a0 + a1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        const int ex = x - a0 - a1;
        cb[2 * lane] = ex;
        cb[2 * lane + 1] = ex + a0;
        if (lane == 31) S.nitems[warp] = x;
      }
      {
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
      // each non-empty key cell takes its place in the count order (its count still at hand), and
      // the particle indices go into key order: hist[key] advances to the bucket's end. Four records
      // per thread and pass, so that eight atomics are in flight before their slots are written.
#pragma unroll
      for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        const int idx = tid * SCAN_PER_THREAD + k;
        if (v0[k] > 0) S.order[0][atomicAdd(&S.cbin[0][CNT_BINS - 1 - min(v0[k], CNT_BINS - 1)], 1)] = (unsigned short)idx;
        if (v1[k] > 0) S.order[1][atomicAdd(&S.cbin[1][CNT_BINS - 1 - min(v1[k], CNT_BINS - 1)], 1)] = (unsigned short)idx;
      }
      for (int i0 = tid; i0 < m; i0 += 4 * THREADS) {
        int keys[4], at0[4], at1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) keys[u] = i0 + u * THREADS < m ? S.sp[i0 + u * THREADS].x : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          at0[u] = keys[u] >= 0 ? atomicAdd(&S.hist[0][keys[u] & 0xffff], 1) : 0;
          at1[u] = keys[u] >= 0 && interlace ? atomicAdd(&S.hist[1][keys[u] >> 16], 1) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (keys[u] < 0) continue;
          S.perm[0][at0[u]] = (unsigned short)(i0 + u * THREADS);
          if (interlace) S.perm[1][at1[u]] = (unsigned short)(i0 + u * THREADS);
        }
      }
      __syncthreads();
      // interlaced: even warps take grid 1's key cells and odd warps grid 2's (the grid is then a
      // compile-time constant of the inner loop); otherwise all warps take grid 1's. Within a grid,
      // thread t of the grid's nt threads takes item t of each round of nt in even rounds and item
      // nt - 1 - t in odd ones.
      {
        const int gsel = interlace ? (warp & 1) : 0;
        const int nt = interlace ? THREADS / 2 : THREADS;
        const int t = interlace ? (warp >> 1) * 32 + lane : tid;
        const int nitems = S.nitems[gsel];
        const unsigned short* order = S.order[gsel];
        for (int r0 = 0; r0 < nitems; r0 += 2 * nt) {  // two rounds: ascending, then descending
          const int i0 = r0 + t, i1 = r0 + 2 * nt - 1 - t;
          if (gsel == 0) {
            if (i0 < nitems) cell_key<P, W, R, 0, DET>(S, order[i0], wscale);
            if (i1 < nitems) cell_key<P, W, R, 0, DET>(S, order[i1], wscale);
          } else {
            if (i0 < nitems) cell_key<P, W, R, 1, DET>(S, order[i0], wscale);
            if (i1 < nitems) cell_key<P, W, R, 1, DET>(S, order[i1], wscale);
          }
        }
      }
      __syncthreads();
    }
    if constexpr (DET)
      flush_region_fixed<RS>(&S.reg[0][0], ngrid, cx0, cy0, cz0, ng, ldz, shift, cg1, cg2, tid, THREADS);
    else
      flush_region(&S.reg[0][0], ngrid, cx0, cy0, cz0, ng, ldz, inv_scale, cg1, cg2, tid, THREADS);
    __syncthreads();
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

// Tile population from which the key-cell kernel takes a tile instead of the scatter, per order. Speed
// alone (uniform catalogues of 256 .. 8192 particles per tile, both grids, one GB300) puts the crossover
// near 750 for PCS, 1400 for TSC and 7000 for CIC. Accuracy caps it lower: the scatter rounds every
// particle's contribution to a node, so its error grows as the square root of the tile's population
// (CIC at 5500 per tile: 4.6e-6 of the largest node; PCS in a 3250-particle tile: 2.1e-6), while the
// key-cell kernel rounds once per key cell. NGP stays on the scatter: its unit contributions at a
// power-of-two scale are exact.
static int cells_min_count(int order) {
  switch (order) {
    case 4: return 768;
    case 3: return 1024;
    case 2: return 512;
    default: return INT_MAX;
  }
}

template <int P, bool W, typename R = int, int S = 1>
static cudaError_t launch_scatter_pw(const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                     bool interlace, float* g1, float* g2, int ldz, cudaStream_t s, int ncat,
                                     int64_t cat_stride, int64_t lo, int64_t hi) {
  const int ntile = tiles_per_axis(ng);
  const int nruns = ntile * ntile * (ntile / S);
  const size_t smem = sizeof(tiles::ScatterSmem<P, W, R, S>);
  static_assert(scatter_blocks<P, R, S>() * (sizeof(tiles::ScatterSmem<P, W, R, S>) + 1024) <= 233472,
                "the launch bounds' blocks per SM fit the SM's shared memory");
  int per_sm = 1;
  cudaError_t e = kernel_setup(reinterpret_cast<const void*>(k_assign_scatter<P, W, R, S>), tiles::SCATTER_THREADS, smem, &per_sm);
  if (e != cudaSuccess) return e;
  // one sequence of runs over all catalogues (blocks take runs of any catalogue, so uneven catalogues
  // leave no tail of idle blocks)
  const dim3 blocks(unsigned(std::max<int64_t>(1, std::min<int64_t>(int64_t(nruns) * ncat, int64_t(num_sms()) * per_sm))), 1);
  k_assign_scatter<P, W, R, S><<<blocks, tiles::SCATTER_THREADS, smem, s>>>(p, w, toff, n, ng, ntile, interlace ? 1 : 0, g1,
                                                                           g2, ldz, cat_stride, lo, hi, ncat);
  count_launch();
  return cudaGetLastError();
}

// The key-cell kernel over the tiles of lo .. hi particles (defined below).
template <int P, bool W, typename R, typename GT = float>
static cudaError_t launch_cells_one(const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                    bool interlace, GT* g1, GT* g2, int ldz, cudaStream_t s, int ncat,
                                    int64_t cat_stride, int64_t lo, int64_t hi, const double* qsrc = nullptr);

// PK_FIXED64, int64 grids: the sparse tiles on the bank-ordered scatter (32-bit regions at a scale 2^e
// per tile that divides the global 2^F), the dense ones (orders 2..4) on the key cells summing rounded
// products exactly (the same regions and scales).
template <int P, bool W>
static cudaError_t launch_scatter_fixed(const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                        bool interlace, const double* wsums, unsigned long long* g1, unsigned long long* g2,
                                        int ldz, cudaStream_t s) {
  const int ntile = tiles_per_axis(ng);
  const int nruns = ntile * ntile * ntile;
  const size_t smem = sizeof(tiles::ScatterSmem<P, W, int, 1>);
  auto* kern = k_assign_scatter<P, W, int, 1, unsigned long long>;
  int per_sm = 1;
  cudaError_t e = kernel_setup(reinterpret_cast<const void*>(kern), tiles::SCATTER_THREADS, smem, &per_sm);
  if (e != cudaSuccess) return e;
  const dim3 blocks(std::max(1, std::min(nruns, num_sms() * per_sm)), 1);
  kern<<<blocks, tiles::SCATTER_THREADS, smem, s>>>(p, w, toff, n, ng, ntile, interlace ? 1 : 0, g1, g2, ldz, 0, 1,
                                                   int64_t(cells_min_count(P)) - 1, 1, wsums);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if constexpr (P >= 2 && P <= 4)  // the dense tiles: key cells summing rounded products exactly
    return launch_cells_one<P, W, int, unsigned long long>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, 1, 0,
                                                           cells_min_count(P), INT64_MAX, wsums);
  return cudaSuccess;
}

cudaError_t launch_assign_tiles_fixed(int order, const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                      bool interlace, const double* wsums, unsigned long long* g1, unsigned long long* g2,
                                      int ldz, cudaStream_t s) {
  switch (order) {
#define PK_FX_CASE(P)                                                                              \
  case P:                                                                                          \
    return w ? launch_scatter_fixed<P, true>(p, w, toff, n, ng, interlace, wsums, g1, g2, ldz, s)  \
             : launch_scatter_fixed<P, false>(p, w, toff, n, ng, interlace, wsums, g1, g2, ldz, s);
    PK_FX_CASE(1)
    PK_FX_CASE(2)
    PK_FX_CASE(3)
    PK_FX_CASE(4)
#undef PK_FX_CASE
    default: return cudaErrorInvalidValue;
  }
}

// Tiles of at least this many particles accumulate their region in 64-bit fixed point. A 32-bit region
// rounds each window at 2^-30 of the tile's node bound (node share x total weight), so a node much
// lighter than the tile's heaviest possible node keeps fewer significant bits: in a tile that holds a
// dense clump (10^5 particles in a few cells) the background nodes would keep ~1e-4 relative accuracy.
// With 62 bits every node keeps the accuracy of the FP32 window sums. The heavy tiles are few (the
// 1024^3 Zel'dovich benchmark catalogue averages 4096 particles per tile), and their kernel instance,
// with twice the region memory, runs one block per SM.
constexpr int64_t kHeavyTile = 16384;

template <int P, bool W, typename R, typename GT>
static cudaError_t launch_cells_one(const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                    bool interlace, GT* g1, GT* g2, int ldz, cudaStream_t s, int ncat,
                                    int64_t cat_stride, int64_t lo, int64_t hi, const double* qsrc) {
  const int ntile = tiles_per_axis(ng);
  const int ntiles = ntile * ntile * ntile;
  const size_t smem = sizeof(tiles::CellSmem<W, R>);
  int per_sm = 1;
  cudaError_t e = kernel_setup(reinterpret_cast<const void*>(k_assign_cells<P, W, R, GT>), tiles::CELL_THREADS, smem, &per_sm);
  if (e != cudaSuccess) return e;
  const dim3 blocks(unsigned(std::max<int64_t>(1, std::min<int64_t>(int64_t(ntiles) * ncat, int64_t(num_sms()) * per_sm))), 1);
  k_assign_cells<P, W, R, GT><<<blocks, tiles::CELL_THREADS, smem, s>>>(p, w, toff, n, ng, ntile, interlace ? 1 : 0, g1, g2,
                                                                        ldz, cat_stride, lo, hi, ncat, qsrc);
  count_launch();
  return cudaGetLastError();
}

// The key-cell kernel over the tiles of at least cells_min_count(P) particles: 32-bit regions below
// kHeavyTile particles, 64-bit regions from there on.
template <int P, bool W>
static cudaError_t launch_cells_pw(const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                   bool interlace, float* g1, float* g2, int ldz, cudaStream_t s, int ncat,
                                   int64_t cat_stride) {
  cudaError_t e = launch_cells_one<P, W, int>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride,
                                              cells_min_count(P), kHeavyTile - 1);
  if (e != cudaSuccess) return e;
  return launch_cells_one<P, W, long long>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, kHeavyTile,
                                           INT64_MAX);
}

// Tiles of fewer than cells_min_count(P) particles: the scatter; the others: the key cells (NGP: all
// on the scatter). Orders 5 and 6 take every tile on the scatter (a register window of p^3 = 125 or
// 216 nodes does not fit), with 64-bit regions from kHeavyTile particles on. Each kernel skips the
// other's tiles, so all launch whatever the populations.
template <int P>
static cudaError_t launch_tiles_p(const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng, bool interlace,
                                  float* g1, float* g2, int ldz, cudaStream_t s, int ncat, int64_t cat_stride, int run) {
  if constexpr (P >= 5) {
    cudaError_t e = w ? launch_scatter_pw<P, true>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, 1, kHeavyTile - 1)
                      : launch_scatter_pw<P, false>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, 1, kHeavyTile - 1);
    if (e != cudaSuccess) return e;
    return w ? launch_scatter_pw<P, true, long long>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, kHeavyTile,
                                                     INT64_MAX)
             : launch_scatter_pw<P, false, long long>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, kHeavyTile,
                                                      INT64_MAX);
  } else {
    const int64_t hi = int64_t(cells_min_count(P)) - 1;
    const int ntile = tiles_per_axis(ng);
    if (run != 2 && run != 4) run = 1;
    if (ntile % run != 0) run = 1;
    cudaError_t e;
    if (run == 4)
      e = w ? launch_scatter_pw<P, true, int, 4>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, 1, hi)
            : launch_scatter_pw<P, false, int, 4>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, 1, hi);
    else if (run == 2)
      e = w ? launch_scatter_pw<P, true, int, 2>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, 1, hi)
            : launch_scatter_pw<P, false, int, 2>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, 1, hi);
    else
      e = w ? launch_scatter_pw<P, true>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, 1, hi)
            : launch_scatter_pw<P, false>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, 1, hi);
    if (e != cudaSuccess) return e;
    if constexpr (P > 1)
      e = w ? launch_cells_pw<P, true>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride)
            : launch_cells_pw<P, false>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride);
    return e;
  }
}

cudaError_t launch_assign_tiles_f32(int order, const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                    bool interlace, float* g1, float* g2, int ldz, cudaStream_t s, int ncat,
                                    int64_t cat_stride, int run) {
  switch (order) {
    case 1: return launch_tiles_p<1>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, run);
    case 2: return launch_tiles_p<2>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, run);
    case 3: return launch_tiles_p<3>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, run);
    case 4: return launch_tiles_p<4>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, run);
    case 5: return launch_tiles_p<5>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, 1);
    case 6: return launch_tiles_p<6>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride, 1);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pk
