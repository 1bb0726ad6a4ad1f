// a3 mass assignment, FP32, column walk with register windows (eq:delgrid on both grids of Sec. 3.1).
//
// The scatter is FP32-FMA bound: a particle adds p^3 products to each grid. Accumulating them one by
// one in shared memory (k_assign_tile) serialises on shared atomics; here the products are summed in
// registers and only completed planes leave the thread:
//  - one block per tile of T^3 cells (particles binned by tile, pk_bin), staged in shared memory in
//    chunks and sorted there by "key cell" (a counting sort): the key cell is the cell whose fixed
//    stencil (nodes key + S0 .. key + S0 + p - 1 on each axis) covers the particle on that grid;
//    key = cell + delta with delta in {0, 1}, so each grid has (T+1)^2 key columns of T+1 key cells;
//  - one thread per (grid, key column) walks its column in x with a window of p x p x p register
//    accumulators (planes key+S0 .. key+S0+p-1); after each x step the oldest plane is complete and
//    is added (16 shared atomics for PCS) to a shared-memory region of (T+4)^3 nodes per grid;
//  - after the tile, the region is added to the grid in global memory.
// Per particle and grid: p weights per axis, p^2 products w_y w_z and p^3 FMAs, all in registers.
#include "internal.cuh"

namespace pk {

namespace walk {

constexpr int T = kTileCells;  // tile edge (cells)
constexpr int K = T + 1;       // key cells per axis and grid
constexpr int NCOL = K * K;    // key columns per grid
constexpr int NKEY = K * K * K;
constexpr int RS = T + 4;  // region edge (nodes -1 .. T+2)
constexpr int RVOL = RS * RS * RS;
constexpr int CHUNK = 2048;  // particles staged per pass
constexpr int THREADS = 192;

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

// Grid g's key delta and offset for in-cell offset f (grid 2 samples the particle shifted by H/2).
template <int P>
__device__ __forceinline__ int grid_key(int g, float f, float* t) {
  if (g == 0) return key_delta<P>(f, t);
  float f2;
  const int d2 = half_shift(f, &f2);
  return d2 + key_delta<P>(f2, t);
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

struct Smem {
  int4 sp[CHUNK];
  unsigned short rank[2][CHUNK];
  unsigned short perm[2][CHUNK];
  int hist[2][NKEY + 1];
  float reg[2][RVOL];
  float sw[CHUNK];  // staged weights (only when weights are given)
};

}  // namespace walk

template <int P>
__global__ void __launch_bounds__(walk::THREADS) k_assign_walk(const pk_cellpos* __restrict__ p, const float* __restrict__ w,
                                                               const int64_t* __restrict__ toff, int64_t n, int ng, int ntile,
                                                               int interlace, float* __restrict__ g1, float* __restrict__ g2,
                                                               int ldz, int64_t cat_stride) {
  using namespace walk;
  {  // blockIdx.y selects a catalogue of a batch: its grids and its tile offsets
    const int cat = blockIdx.y;
    g1 += cat * cat_stride;
    if (g2) g2 += cat * cat_stride;
    toff += int64_t(cat) * ntile * ntile * ntile;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const int ngrid = interlace ? 2 : 1;
  const int ntiles = ntile * ntile * ntile;
  const int tid = threadIdx.x;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t beg = max(toff[tile], int64_t(0)), end = min(toff[tile + 1], n);
    if (beg >= end) continue;
    const int tz = tile % ntile, ty = (tile / ntile) % ntile, tx = tile / (ntile * ntile);
    const int cx0 = tx * T, cy0 = ty * T, cz0 = tz * T;  // first cell of the tile
    for (int i = tid; i < ngrid * RVOL; i += THREADS) (&S.reg[0][0])[i] = 0.0f;
    for (int64_t c0 = beg; c0 < end; c0 += CHUNK) {
      const int m = int(min(int64_t(CHUNK), end - c0));
      for (int i = tid; i < ngrid * (NKEY + 1); i += THREADS) (&S.hist[0][0])[i] = 0;
      __syncthreads();
      // stage the chunk and histogram the key cells of both grids
      for (int i = tid; i < m; i += THREADS) {
        const int4 r = reinterpret_cast<const int4*>(p)[c0 + i];
        S.sp[i] = r;
        if (w) S.sw[i] = w[c0 + i];
        const uint32_t cell = uint32_t(r.x);
        const int lx = cell_x(cell) - cx0, ly = cell_y(cell) - cy0, lz = cell_z(cell) - cz0;
        const float f[3] = {__int_as_float(r.y), __int_as_float(r.z), __int_as_float(r.w)};
        const bool ok = lx >= 0 && lx < T && ly >= 0 && ly < T && lz >= 0 && lz < T;
        if (!ok) raise_err(PK_DERR_CELLRANGE);
        for (int g = 0; g < ngrid; ++g) {
          unsigned short rk = 0xffff;
          if (ok) {
            float t;
            const int dx = grid_key<P>(g, f[0], &t), dy = grid_key<P>(g, f[1], &t), dz = grid_key<P>(g, f[2], &t);
            const int key = ((ly + dy) * K + (lz + dz)) * K + (lx + dx);
            rk = (unsigned short)atomicAdd(&S.hist[g][key], 1);
          }
          S.rank[g][i] = rk;
        }
      }
      __syncthreads();
      // exclusive scan of each grid's key histogram (one warp per grid); hist[g][NKEY] becomes the total
      {
        const int warp = tid >> 5, lane = tid & 31;
        if (warp < ngrid) {
          int carry = 0;
          for (int base = 0; base < NKEY + 1; base += 32) {
            const int idx = base + lane;
            const int v = idx < NKEY + 1 ? S.hist[warp][idx] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int y = __shfl_up_sync(0xffffffffu, x, o);
              if (lane >= o) x += y;
            }
            if (idx < NKEY + 1) S.hist[warp][idx] = carry + x - v;
            carry += __shfl_sync(0xffffffffu, x, 31);
          }
        }
      }
      __syncthreads();
      // scatter particle indices into key order
      for (int i = tid; i < m; i += THREADS) {
        const int4 r = S.sp[i];
        const uint32_t cell = uint32_t(r.x);
        const int lx = cell_x(cell) - cx0, ly = cell_y(cell) - cy0, lz = cell_z(cell) - cz0;
        const float f[3] = {__int_as_float(r.y), __int_as_float(r.z), __int_as_float(r.w)};
        for (int g = 0; g < ngrid; ++g) {
          const unsigned short rk = S.rank[g][i];
          if (rk == 0xffff) continue;
          float t;
          const int dx = grid_key<P>(g, f[0], &t), dy = grid_key<P>(g, f[1], &t), dz = grid_key<P>(g, f[2], &t);
          const int key = ((ly + dy) * K + (lz + dz)) * K + (lx + dx);
          S.perm[g][S.hist[g][key] + rk] = (unsigned short)i;
        }
      }
      __syncthreads();
      // walk: one thread per (grid, key column)
      if (tid < ngrid * NCOL) {
        const int g = tid / NCOL, col = tid - g * NCOL;
        const int ky = col / K, kz = col - ky * K;
        const int* hist = S.hist[g] + col * K;
        if (hist[0] != hist[K]) {
          float acc[P][P][P];
#pragma unroll
          for (int a = 0; a < P; ++a)
#pragma unroll
            for (int b = 0; b < P; ++b)
#pragma unroll
              for (int c = 0; c < P; ++c) acc[a][b][c] = 0.0f;
          float* reg = S.reg[g];
          const int ry0 = ky + s0<P>() + 1, rz0 = kz + s0<P>() + 1;  // region row/col of stencil offset 0
          const unsigned short* perm = S.perm[g];
#pragma unroll
          for (int x = 0; x < K; ++x) {
            const int jb = hist[x], je = hist[x + 1];
            for (int j = jb; j < je; ++j) {
              const int i = perm[j];
              const int4 r = S.sp[i];
              float tx, ty, tz;
              grid_key<P>(g, __int_as_float(r.y), &tx);
              grid_key<P>(g, __int_as_float(r.z), &ty);
              grid_key<P>(g, __int_as_float(r.w), &tz);
              float wx[P], wy[P], wz[P];
              weights<P>(tx, wx);
              weights<P>(ty, wy);
              weights<P>(tz, wz);
              const float wgt = (w ? S.sw[i] : 1.0f) * weight_scale<P>();
#pragma unroll
              for (int a = 0; a < P; ++a) wx[a] *= wgt;
#pragma unroll
              for (int b = 0; b < P; ++b)
#pragma unroll
                for (int c = 0; c < P; ++c) {
                  const float yz = wy[b] * wz[c];
#pragma unroll
                  for (int a = 0; a < P; ++a) acc[a][b][c] = fmaf(wx[a], yz, acc[a][b][c]);
                }
            }
            // node plane x + s0 is complete: add it to the region and shift the window
            const int rx = x + s0<P>() + 1;
#pragma unroll
            for (int b = 0; b < P; ++b)
#pragma unroll
              for (int c = 0; c < P; ++c) {
                const float v = acc[0][b][c];
                if (v != 0.0f) atomicAdd(&reg[(rx * RS + ry0 + b) * RS + rz0 + c], v);
              }
#pragma unroll
            for (int a = 0; a + 1 < P; ++a)
#pragma unroll
              for (int b = 0; b < P; ++b)
#pragma unroll
                for (int c = 0; c < P; ++c) acc[a][b][c] = acc[a + 1][b][c];
#pragma unroll
            for (int b = 0; b < P; ++b)
#pragma unroll
              for (int c = 0; c < P; ++c) acc[P - 1][b][c] = 0.0f;
          }
          // the remaining planes K + s0 .. K + s0 + P - 2
#pragma unroll
          for (int a = 0; a + 1 < P; ++a) {
            const int rx = K + a + s0<P>() + 1;
#pragma unroll
            for (int b = 0; b < P; ++b)
#pragma unroll
              for (int c = 0; c < P; ++c) {
                const float v = acc[a][b][c];
                if (v != 0.0f) atomicAdd(&reg[(rx * RS + ry0 + b) * RS + rz0 + c], v);
              }
          }
        }
      }
      __syncthreads();
    }
    // add the tile's region (origin: node (cx0-1, cy0-1, cz0-1)) to the grids
    for (int i = tid; i < ngrid * RVOL; i += THREADS) {
      const float v = (&S.reg[0][0])[i];
      if (v != 0.0f) {
        const int gi = i / RVOL, k = i - gi * RVOL;
        const int rx = k / (RS * RS), ry = (k / RS) % RS, rz = k % RS;
        float* gg = gi == 0 ? g1 : g2;
        atomicAdd(gg + (int64_t(wrap(cx0 - 1 + rx, ng)) * ng + wrap(cy0 - 1 + ry, ng)) * ldz + wrap(cz0 - 1 + rz, ng), v);
      }
    }
    __syncthreads();
  }
}

template <int P>
static cudaError_t launch_walk_p(const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng, bool interlace,
                                 float* g1, float* g2, int ldz, cudaStream_t s, int ncat, int64_t cat_stride) {
  const int ntile = tiles_per_axis(ng);
  const int ntiles = ntile * ntile * ntile;
  size_t smem = sizeof(walk::Smem);
  if (!w) smem -= sizeof(float) * walk::CHUNK;  // the weights stage is the last member
  cudaError_t e = cudaFuncSetAttribute(k_assign_walk<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_assign_walk<P>, walk::THREADS, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const dim3 blocks(std::max(1, std::min(ntiles, std::max(1, num_sms() * per_sm / ncat))), ncat);
  k_assign_walk<P><<<blocks, walk::THREADS, smem, s>>>(p, w, toff, n, ng, ntile, interlace ? 1 : 0, g1, g2, ldz, cat_stride);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_assign_walk_f32(int order, const pk_cellpos* p, const float* w, const int64_t* toff, int64_t n, int ng,
                                   bool interlace, float* g1, float* g2, int ldz, cudaStream_t s, int ncat,
                                   int64_t cat_stride) {
  switch (order) {
    case 1: return launch_walk_p<1>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride);
    case 2: return launch_walk_p<2>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride);
    case 3: return launch_walk_p<3>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride);
    default: return launch_walk_p<4>(p, w, toff, n, ng, interlace, g1, g2, ldz, s, ncat, cat_stride);
  }
}

}  // namespace pk
