// a1 position preparation and a2 counting sort of particles by cell tile.
//
// a1 (Sec. 2.3, s = (x_j - x)/H): an FP64 position is wrapped into [0, L) (periodic box) and split
// into the integer cell c = floor(x/H) and the offset f = x/H - c in [0, 1), stored as FP32.
// a2: particles are grouped by tile of T^3 cells with a counting sort (histogram, exclusive scan,
// scatter), and inside a tile by half-cell slab along x (key tile * 2T + 2 (c_x mod T) + [f_x >= 1/2]),
// which keeps neighbouring cells' particles together in a staged piece; the assignment itself
// accepts any order inside a tile.
// Histogram and scatter use warp-aggregated atomics: consecutive particles of a spatially ordered
// catalogue share a key, and one atomic per distinct key per warp replaces 32. Particles are
// validated on the way (an invalid record is reported and binned as cell 0, offset 0).
#include "internal.cuh"

namespace pk {

PK_ERR_ACCESSOR(take_err_prepare)

// floor(u) and the fraction u - floor(u) rounded to FP32 (to nearest, ties to even) for 0 <= u < 2^20,
// read from u's bits with integer operations: FP64 arithmetic is scarce on this GPU, and the fraction
// of a double is exact in its significand, so this equals float(u - floor(u)) bit for bit.
__device__ __forceinline__ void split_units(double u, int* c, float* f) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(u));
  const int e = int((b >> 52) & 0x7ff) - 1023;
  if (e < 0) {  // u in [0, 1), or -0: floor 0 (+ 0.0f makes -0 the +0 that u - floor(u) gives)
    *c = 0;
    *f = __double2float_rn(u) + 0.0f;
    return;
  }
  const int sh = 52 - e;  // fraction bits of the significand (32 < sh <= 52 for u < 2^20)
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  *c = int(m >> sh);
  const unsigned long long fr = m & ((1ull << sh) - 1);  // u - floor(u) = fr 2^-sh exactly
  if (fr == 0) {
    *f = 0.0f;
    return;
  }
  const int top = 63 - __clzll(static_cast<long long>(fr));  // fr in [2^top, 2^(top+1)), top < sh
  unsigned long long m24;  // 24-bit significand, rounded; 2^24 when the rounding carries
  if (top >= 24) {
    const int d = top - 23;
    m24 = fr >> d;
    const unsigned long long rem = fr & ((1ull << d) - 1), half = 1ull << (d - 1);
    if (rem > half || (rem == half && (m24 & 1ull))) ++m24;
  } else {
    m24 = fr << (23 - top);
  }
  const int ex = top - sh + 127;  // biased exponent of 2^(top - sh), >= 75
  *f = __int_as_float(int((unsigned(ex - 1) << 23) + unsigned(m24)));
}

__device__ __forceinline__ pk_cellpos prepare_one(const double* p, int ng, double box, double scale) {
  pk_cellpos r;
  int c[3];
  float fo[3];
  bool bad = false;
  const unsigned long long box_bits = static_cast<unsigned long long>(__double_as_longlong(box));
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double x = p[a];
    const unsigned long long xb = static_cast<unsigned long long>(__double_as_longlong(x));
    if (((xb >> 52) & 0x7ff) == 0x7ff) {  // NaN or infinite
      bad = true;
      x = 0.0;
    } else if (xb >= box_bits) {  // negative (sign bit) or >= L: another periodic image
      x = fmod(x, box);
      if (x < 0.0) x += box;
    }
    int ci;
    float ff;
    split_units(x * scale, &ci, &ff);
    if (ci >= ng) { ci -= ng; }
    if (ff >= 1.0f) {  // f rounded up to 1 in FP32: the particle sits on the next node
      ff = 0.0f;
      ci = ci + 1 == ng ? 0 : ci + 1;
    }
    c[a] = ci;
    fo[a] = ff;
  }
  if (bad) {
    raise_err(PK_DERR_NONFINITE);
    c[0] = c[1] = c[2] = 0;
    fo[0] = fo[1] = fo[2] = 0.0f;
  }
  r.cell = pack_cell(c[0], c[1], c[2]);
  r.fx = fo[0];
  r.fy = fo[1];
  r.fz = fo[2];
  return r;
}

__global__ void k_prepare(const double* __restrict__ pos, int64_t n, int ng, double box, pk_cellpos* __restrict__ out) {
  const double scale = double(ng) / box;
  for (int64_t i = gtid(); i < n; i += gstride()) out[i] = prepare_one(pos + 3 * i, ng, box, scale);
}

// Sort key of a (validated) particle: tile and half-cell slab along x.
__device__ __forceinline__ int bin_key(const pk_cellpos& r, int ntile) {
  const int cx = cell_x(r.cell), tx = cx / kTileCells, ty = cell_y(r.cell) / kTileCells, tz = cell_z(r.cell) / kTileCells;
  const int slab = 2 * (cx - tx * kTileCells) + (r.fx >= 0.5f ? 1 : 0);
  return ((tx * ntile + ty) * ntile + tz) * kSlabs + slab;
}

// Validates a packed particle (coordinates < N, offsets in [0,1)); invalid ones are reported and
// mapped to cell 0 so that every later index stays in bounds.
__device__ __forceinline__ pk_cellpos checked(pk_cellpos r, int ng) {
  const bool ok = cell_x(r.cell) < ng && cell_y(r.cell) < ng && cell_z(r.cell) < ng && (r.cell >> 30) == 0 &&
                  r.fx >= 0.0f && r.fx < 1.0f && r.fy >= 0.0f && r.fy < 1.0f && r.fz >= 0.0f && r.fz < 1.0f;
  if (!ok) {
    raise_err(PK_DERR_CELLRANGE);
    r.cell = 0;
    r.fx = r.fy = r.fz = 0.0f;
  }
  return r;
}

// Warp-aggregated increment of ctr[key]; returns the value this lane would have seen alone.
__device__ __forceinline__ unsigned long long agg_inc(unsigned long long* ctr, int key, unsigned active) {
  const unsigned peers = __match_any_sync(active, key);
  const int leader = __ffs(peers) - 1;
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(ctr + key, (unsigned long long)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

__global__ void k_tile_hist(const pk_cellpos* __restrict__ p, int64_t n, int ng, int ntile,
                            unsigned long long* __restrict__ counts) {
  const int64_t stride = gstride();
  const int64_t nround = (n + 31) / 32 * 32;
  for (int64_t i = gtid(); i < nround; i += stride) {
    const bool live = i < n;
    const unsigned active = __ballot_sync(0xffffffffu, live);
    if (live) agg_inc(counts, bin_key(checked(p[i], ng), ntile), active);
  }
}

__global__ void k_tile_scatter(const pk_cellpos* __restrict__ p, const float* __restrict__ w, int64_t n, int ng, int ntile,
                               const int64_t* __restrict__ sub, unsigned long long* __restrict__ cursor,
                               pk_cellpos* __restrict__ out, float* __restrict__ wout) {
  const int64_t stride = gstride();
  const int64_t nround = (n + 31) / 32 * 32;
  for (int64_t i = gtid(); i < nround; i += stride) {
    const bool live = i < n;
    const unsigned active = __ballot_sync(0xffffffffu, live);
    if (live) {
      const pk_cellpos r = checked(p[i], ng);
      const int key = bin_key(r, ntile);
      const int64_t dst = sub[key] + int64_t(agg_inc(cursor, key, active));
      out[dst] = r;
      if (wout) wout[dst] = w[i];
    }
  }
}

// a1 and the counting pass of a2 in one sweep over FP64 positions pos[0 .. cnt) (device memory, or
// pinned host memory read over the CPU-GPU link): each particle is prepared, written to out[i0 + k]
// and its sort key counted. A block stages its 256 particles' 6 KB of coordinates in shared memory
// with 16-byte loads (when pos is 16-byte aligned), so every byte crosses the link once, in full lines.
constexpr int kPrepBlock = 256;
__global__ void __launch_bounds__(kPrepBlock) k_prepare_hist(const double* __restrict__ pos, int64_t i0, int64_t cnt, int ng,
                                                             double box, int ntile, int vec, pk_cellpos* __restrict__ out,
                                                             unsigned long long* __restrict__ counts) {
  __shared__ double2 s_pos[kPrepBlock * 3 / 2];
  double* sp = reinterpret_cast<double*>(s_pos);
  const double scale = double(ng) / box;
  for (int64_t base = int64_t(blockIdx.x) * kPrepBlock; base < cnt; base += int64_t(gridDim.x) * kPrepBlock) {
    const int m = int(min(int64_t(kPrepBlock), cnt - base));
    const double* src = pos + 3 * base;
    if (vec) {
      const int nv = (3 * m) / 2;
      for (int v = threadIdx.x; v < nv; v += kPrepBlock) s_pos[v] = reinterpret_cast<const double2*>(src)[v];
      if (((3 * m) & 1) && threadIdx.x == 0) sp[3 * m - 1] = src[3 * m - 1];
    } else {
      for (int v = threadIdx.x; v < 3 * m; v += kPrepBlock) sp[v] = src[v];
    }
    __syncthreads();
    const int k = threadIdx.x;
    const bool live = k < m;
    const unsigned active = __ballot_sync(0xffffffffu, live);
    if (live) {
      const pk_cellpos r = prepare_one(sp + 3 * k, ng, box, scale);
      out[i0 + base + k] = r;
      agg_inc(counts, bin_key(r, ntile), active);
    }
    __syncthreads();
  }
}

// Tile offsets from the slab offsets: offsets[t] = sub[t * kSlabs], t = 0 .. ntiles.
__global__ void k_tile_offsets(const int64_t* __restrict__ sub, int64_t ntiles, int64_t* __restrict__ offsets) {
  for (int64_t t = gtid(); t <= ntiles; t += gstride()) offsets[t] = sub[t * kSlabs];
}

// Batched binning: blockIdx.y = catalogue c of the group, particles r.off[c] .. r.off[c+1]-1 of p,
// key c * ntiles + tile. Sorted output indices count from the group's first particle.
__global__ void k_tile_hist_batch(const pk_cellpos* __restrict__ p, CatRanges r, int ntile,
                                  unsigned long long* __restrict__ counts) {
  const int c = blockIdx.y;
  const int64_t beg = r.off[c], cnt = r.off[c + 1] - beg;
  const int base = c * ntile * ntile * ntile * kSlabs;
  const int64_t nround = (cnt + 31) / 32 * 32;
  for (int64_t k = gtid(); k < nround; k += gstride()) {
    const bool live = k < cnt;
    const unsigned active = __ballot_sync(0xffffffffu, live);
    if (live) agg_inc(counts, base + bin_key(checked(p[beg + k], r.ng), ntile), active);
  }
}

__global__ void k_tile_scatter_batch(const pk_cellpos* __restrict__ p, CatRanges r, int ntile,
                                     const int64_t* __restrict__ sub, unsigned long long* __restrict__ cursor,
                                     pk_cellpos* __restrict__ out) {
  const int c = blockIdx.y;
  const int64_t beg = r.off[c], cnt = r.off[c + 1] - beg;
  const int base = c * ntile * ntile * ntile * kSlabs;
  const int64_t nround = (cnt + 31) / 32 * 32;
  for (int64_t k = gtid(); k < nround; k += gstride()) {
    const bool live = k < cnt;
    const unsigned active = __ballot_sync(0xffffffffu, live);
    if (live) {
      const pk_cellpos rec = checked(p[beg + k], r.ng);
      const int key = base + bin_key(rec, ntile);
      out[sub[key] + int64_t(agg_inc(cursor, key, active))] = rec;
    }
  }
}

// Batched binning by tile with shared-memory histograms. Block (x, c) takes particles
// [off[c] + x kBinChunk, ..) of catalogue c: it counts their tiles in shared memory, then adds one
// count per non-empty tile to the global counters (count pass), or reserves one range per non-empty
// tile with a global atomic and places its particles there through shared-memory cursors (place
// pass). Output indices count from the group's first particle, as k_tile_scatter_batch's.
constexpr int kBinChunk = 32768;

__device__ __forceinline__ int tile_of(const pk_cellpos& r, int ntile) {
  return ((cell_x(r.cell) / kTileCells) * ntile + cell_y(r.cell) / kTileCells) * ntile + cell_z(r.cell) / kTileCells;
}

// Records per thread and round of the chunk loops: their loads are issued together, so each thread
// keeps several in flight (one at a time left the kernels waiting on memory at 8 % issue).
constexpr int kBinUnroll = 4;

__global__ void k_tile_count_smem(const pk_cellpos* __restrict__ p, CatRanges r, int ntile,
                                  unsigned long long* __restrict__ counts) {
  extern __shared__ int s_cnt[];  // [ntiles]
  const int c = blockIdx.y, ntiles = ntile * ntile * ntile;
  const int64_t beg = r.off[c] + int64_t(blockIdx.x) * kBinChunk, end = min(r.off[c + 1], beg + kBinChunk);
  if (beg >= end) return;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) s_cnt[t] = 0;
  __syncthreads();
  for (int64_t i0 = beg + threadIdx.x; i0 < end; i0 += int64_t(kBinUnroll) * blockDim.x) {
    pk_cellpos rec[kBinUnroll];
#pragma unroll
    for (int u = 0; u < kBinUnroll; ++u) {
      const int64_t i = i0 + int64_t(u) * blockDim.x;
      if (i < end) rec[u] = p[i];
    }
#pragma unroll
    for (int u = 0; u < kBinUnroll; ++u)
      if (i0 + int64_t(u) * blockDim.x < end) atomicAdd(&s_cnt[tile_of(checked(rec[u], r.ng), ntile)], 1);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
    if (s_cnt[t]) atomicAdd(&counts[int64_t(c) * ntiles + t], (unsigned long long)s_cnt[t]);
}

__global__ void k_tile_place_smem(const pk_cellpos* __restrict__ p, CatRanges r, int ntile, const int64_t* __restrict__ offsets,
                                  unsigned long long* __restrict__ cursor, pk_cellpos* __restrict__ out) {
  extern __shared__ long long s_base[];  // [ntiles] range start, then int cursors [ntiles]
  const int c = blockIdx.y, ntiles = ntile * ntile * ntile;
  int* s_cnt = reinterpret_cast<int*>(s_base + ntiles);
  const int64_t beg = r.off[c] + int64_t(blockIdx.x) * kBinChunk, end = min(r.off[c + 1], beg + kBinChunk);
  if (beg >= end) return;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) s_cnt[t] = 0;
  __syncthreads();
  for (int64_t i0 = beg + threadIdx.x; i0 < end; i0 += int64_t(kBinUnroll) * blockDim.x) {
    pk_cellpos rec[kBinUnroll];
#pragma unroll
    for (int u = 0; u < kBinUnroll; ++u) {
      const int64_t i = i0 + int64_t(u) * blockDim.x;
      if (i < end) rec[u] = p[i];
    }
#pragma unroll
    for (int u = 0; u < kBinUnroll; ++u)
      if (i0 + int64_t(u) * blockDim.x < end) atomicAdd(&s_cnt[tile_of(checked(rec[u], r.ng), ntile)], 1);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    const int k = s_cnt[t];
    if (k) {
      const int64_t key = int64_t(c) * ntiles + t;
      s_base[t] = offsets[key] + (long long)atomicAdd(&cursor[key], (unsigned long long)k);
    }
    s_cnt[t] = 0;
  }
  __syncthreads();
  for (int64_t i0 = beg + threadIdx.x; i0 < end; i0 += int64_t(kBinUnroll) * blockDim.x) {
    pk_cellpos rec[kBinUnroll];
#pragma unroll
    for (int u = 0; u < kBinUnroll; ++u) {
      const int64_t i = i0 + int64_t(u) * blockDim.x;
      if (i < end) rec[u] = p[i];
    }
    int64_t dst[kBinUnroll];
#pragma unroll
    for (int u = 0; u < kBinUnroll; ++u) {
      if (i0 + int64_t(u) * blockDim.x < end) {
        rec[u] = checked(rec[u], r.ng);
        const int t = tile_of(rec[u], ntile);
        dst[u] = s_base[t] + atomicAdd(&s_cnt[t], 1);
      }
    }
#pragma unroll
    for (int u = 0; u < kBinUnroll; ++u)
      if (i0 + int64_t(u) * blockDim.x < end) out[dst[u]] = rec[u];
  }
}

// Exclusive scan of int64 counts, three phases over blocks of kScanBlock elements.
constexpr int kScanBlock = 1024;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* total) {
  __shared__ long long warp_sums[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    long long s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    if (lane < nw) warp_sums[lane] = s;
  }
  __syncthreads();
  const long long before = wid > 0 ? warp_sums[wid - 1] : 0;
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void k_scan_blocks(const unsigned long long* __restrict__ in, int64_t n, long long* __restrict__ block_sums) {
  const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
  long long v = i < n ? (long long)in[i] : 0;
  long long tot;
  block_exclusive_scan(v, &tot);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(long long* __restrict__ block_sums, int nblocks) {
  // one block: sequential chunks of kScanBlock
  long long carry = 0;
  for (int base = 0; base < nblocks; base += kScanBlock) {
    const int i = base + threadIdx.x;
    const long long v = i < nblocks ? block_sums[i] : 0;
    long long tot;
    const long long ex = block_exclusive_scan(v, &tot);
    if (i < nblocks) block_sums[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
}

__global__ void k_scan_apply(const unsigned long long* __restrict__ in, int64_t n, const long long* __restrict__ block_sums,
                             int64_t* __restrict__ out, int64_t total_slot) {
  const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
  const long long v = i < n ? (long long)in[i] : 0;
  const long long ex = block_exclusive_scan(v, nullptr);
  if (i < n) out[i] = block_sums[blockIdx.x] + ex;
  if (i == n - 1) out[total_slot] = block_sums[blockIdx.x] + ex + v;
}

// ---- host launchers -----------------------------------------------------------------------------

cudaError_t launch_prepare(const double* pos, int64_t n, int ng, double box, pk_cellpos* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, int64_t(num_sms()) * 16);
  k_prepare<<<int(blocks), threads, 0, s>>>(pos, n, ng, box, out); count_launch();
  return cudaGetLastError();
}

size_t scan_scratch_bytes(int64_t n) { return size_t((n + kScanBlock - 1) / kScanBlock) * sizeof(long long); }

cudaError_t launch_exclusive_scan(const unsigned long long* in, int64_t n, int64_t* out, long long* scratch, cudaStream_t s) {
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  k_scan_blocks<<<int(nb), kScanBlock, 0, s>>>(in, n, scratch); count_launch();
  k_scan_sums<<<1, kScanBlock, 0, s>>>(scratch, int(nb)); count_launch();
  k_scan_apply<<<int(nb), kScanBlock, 0, s>>>(in, n, scratch, out, n); count_launch();
  return cudaGetLastError();
}

static cudaError_t launch_tile_offsets(const int64_t* sub, int64_t ntiles, int64_t* offsets, cudaStream_t s) {
  const int threads = 256;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((ntiles + threads) / threads, int64_t(num_sms()) * 8));
  k_tile_offsets<<<int(blocks), threads, 0, s>>>(sub, ntiles, offsets); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_prepare_hist(const double* pos, int64_t i0, int64_t cnt, int ng, double box, int ntile, pk_cellpos* cells,
                                unsigned long long* counts, cudaStream_t s) {
  if (cnt == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((cnt + kPrepBlock - 1) / kPrepBlock, int64_t(num_sms()) * 16);
  const int vec = (reinterpret_cast<uintptr_t>(pos) & 15u) == 0 ? 1 : 0;
  k_prepare_hist<<<int(blocks), kPrepBlock, 0, s>>>(pos, i0, cnt, ng, box, ntile, vec, cells, counts); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bin(const pk_cellpos* cells, const float* w, int64_t n, int ng, int ntile, pk_cellpos* sorted,
                       float* wsorted, int64_t* offsets, unsigned long long* counts, int64_t* sub, long long* scan_scratch,
                       cudaStream_t s) {
  const int64_t nkeys = int64_t(ntile) * ntile * ntile * kSlabs;
  cudaError_t e = cudaMemsetAsync(counts, 0, size_t(nkeys) * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int threads = 256;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, int64_t(num_sms()) * 16));
  if (n > 0) {
    k_tile_hist<<<int(blocks), threads, 0, s>>>(cells, n, ng, ntile, counts); count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return launch_bin_finish(cells, w, n, ng, ntile, sorted, wsorted, offsets, counts, sub, scan_scratch, s);
}

cudaError_t launch_bin_finish(const pk_cellpos* cells, const float* w, int64_t n, int ng, int ntile, pk_cellpos* sorted,
                              float* wsorted, int64_t* offsets, unsigned long long* counts, int64_t* sub,
                              long long* scan_scratch, cudaStream_t s) {
  const int64_t ntiles = int64_t(ntile) * ntile * ntile, nkeys = ntiles * kSlabs;
  const int threads = 256;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, int64_t(num_sms()) * 16));
  cudaError_t e;
  if ((e = launch_exclusive_scan(counts, nkeys, sub, scan_scratch, s)) != cudaSuccess) return e;
  if ((e = launch_tile_offsets(sub, ntiles, offsets, s)) != cudaSuccess) return e;
  if (n > 0) {
    if ((e = cudaMemsetAsync(counts, 0, size_t(nkeys) * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    k_tile_scatter<<<int(blocks), threads, 0, s>>>(cells, w, n, ng, ntile, sub, counts, sorted, wsorted); count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_bin_batch_tiles(const pk_cellpos* p, const CatRanges& r, int ntile, pk_cellpos* sorted, int64_t* offsets,
                                   unsigned long long* counts, long long* scan_scratch, cudaStream_t s) {
  const int ntiles = ntile * ntile * ntile;
  const int64_t nkeys = int64_t(ntiles) * r.nb;
  cudaError_t e = cudaMemsetAsync(counts, 0, size_t(nkeys) * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  int64_t maxc = 1;
  for (int c = 0; c < r.nb; ++c) maxc = std::max<int64_t>(maxc, r.off[c + 1] - r.off[c]);
  const dim3 blocks(unsigned((maxc + kBinChunk - 1) / kBinChunk), unsigned(r.nb));
  const size_t smem_count = size_t(ntiles) * sizeof(int), smem_place = size_t(ntiles) * (sizeof(long long) + sizeof(int));
  if ((e = ensure_dynamic_smem(reinterpret_cast<const void*>(k_tile_count_smem), smem_count)) != cudaSuccess) return e;
  if ((e = ensure_dynamic_smem(reinterpret_cast<const void*>(k_tile_place_smem), smem_place)) != cudaSuccess) return e;
  k_tile_count_smem<<<blocks, 512, smem_count, s>>>(p, r, ntile, counts); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_exclusive_scan(counts, nkeys, offsets, scan_scratch, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(counts, 0, size_t(nkeys) * sizeof(unsigned long long), s)) != cudaSuccess) return e;
  k_tile_place_smem<<<blocks, 512, smem_place, s>>>(p, r, ntile, offsets, counts, sorted); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bin_batch(const pk_cellpos* p, const CatRanges& r, int ng, int ntile, pk_cellpos* sorted, int64_t* offsets,
                             unsigned long long* counts, int64_t* sub, long long* scan_scratch, cudaStream_t s) {
  const int64_t ntiles = int64_t(ntile) * ntile * ntile * r.nb, nkeys = ntiles * kSlabs;
  cudaError_t e = cudaMemsetAsync(counts, 0, size_t(nkeys) * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  int64_t maxc = 1;
  for (int c = 0; c < r.nb; ++c) maxc = std::max<int64_t>(maxc, r.off[c + 1] - r.off[c]);
  const dim3 blocks(unsigned(std::max<int64_t>(1, std::min<int64_t>((maxc + 255) / 256, std::max(1, num_sms() * 16 / r.nb)))),
                    unsigned(r.nb));
  (void)ng;
  k_tile_hist_batch<<<blocks, 256, 0, s>>>(p, r, ntile, counts); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_exclusive_scan(counts, nkeys, sub, scan_scratch, s)) != cudaSuccess) return e;
  if ((e = launch_tile_offsets(sub, ntiles, offsets, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(counts, 0, size_t(nkeys) * sizeof(unsigned long long), s)) != cudaSuccess) return e;
  k_tile_scatter_batch<<<blocks, 256, 0, s>>>(p, r, ntile, sub, counts, sorted); count_launch();
  return cudaGetLastError();
}

}  // namespace pk
