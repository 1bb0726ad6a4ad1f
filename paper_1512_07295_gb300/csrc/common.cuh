// Shared device-side definitions of libpk (sm_103a): the B-spline weights of Sec. 2.3 written as
// polynomials of the in-cell offset, packed-cell helpers, the device error word and small utilities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pk.h"

namespace pk {

constexpr int kMaxOrder = 6;

// Device error word (PK_DERR_* bits). Without relocatable device code a __device__ variable is local to
// its translation unit, so each unit that raises errors has its own word and a host accessor defined
// with PK_ERR_ACCESSOR; pk_device_error reads and clears all of them.
static __device__ unsigned int g_err = 0;

__device__ __forceinline__ void raise_err(unsigned bits) { atomicOr(&g_err, bits); }

#define PK_ERR_ACCESSOR(fn)                                                          \
  int fn(unsigned* acc) {                                                            \
    unsigned v = 0, z = 0;                                                           \
    if (cudaMemcpyFromSymbol(&v, g_err, sizeof(v)) != cudaSuccess) return -1;       \
    if (cudaMemcpyToSymbol(g_err, &z, sizeof(z)) != cudaSuccess) return -1;         \
    *acc |= v;                                                                       \
    return 0;                                                                        \
  }

// Packed cell: cx << 20 | cy << 10 | cz.
__host__ __device__ __forceinline__ uint32_t pack_cell(int cx, int cy, int cz) {
  return (uint32_t(cx) << 20) | (uint32_t(cy) << 10) | uint32_t(cz);
}
__host__ __device__ __forceinline__ int cell_x(uint32_t c) { return int(c >> 20) & 1023; }
__host__ __device__ __forceinline__ int cell_y(uint32_t c) { return int(c >> 10) & 1023; }
__host__ __device__ __forceinline__ int cell_z(uint32_t c) { return int(c) & 1023; }

// Values N_P(f + k), k = 0..P-1, of the cardinal B-spline of order P on integer knots (support [0, P])
// at an offset f in [0, 1), by the recurrence N_q(x) = [x N_{q-1}(x) + (q - x) N_{q-1}(x - 1)] / (q - 1)
// (every term non-negative, so no cancellation), updated in place from the top index down.
template <int P, typename T>
__device__ __forceinline__ void cardinal_bspline(T f, T* b) {
  b[0] = T(1);
#pragma unroll
  for (int q = 2; q <= P; ++q) {
    const T inv = T(1) / T(q - 1);
    b[q - 1] = (T(1) - f) * b[q - 2] * inv;
#pragma unroll
    for (int k = q - 2; k >= 1; --k) b[k] = ((f + T(k)) * b[k] + (T(q) - f - T(k)) * b[k - 1]) * inv;
    b[0] = f * b[0] * inv;
  }
}

// The centred B-spline of order P >= 5 (beyond PCS): the weight of the k-th stencil node is
// N_P(m - g) = N_P(g + P - m) with m = k + 1, i.e. b[P - 1 - k]; g is the offset from floor(u) (even P)
// or floor(u + 1/2) (odd P). Returns the first node relative to c = floor(u).
template <int P, typename T>
__device__ __forceinline__ int bspline_high(T f, T* w, T* g_out) {
  T g = f;
  int start;
  if constexpr (P % 2 == 0) {
    start = 1 - P / 2;
  } else {
    const bool up = f >= T(0.5);
    g = up ? f - T(0.5) : f + T(0.5);
    start = (up ? 1 : 0) - (P - 1) / 2;
  }
  T b[P];
  cardinal_bspline<P>(g, b);
#pragma unroll
  for (int k = 0; k < P; ++k) w[k] = b[P - 1 - k];
  *g_out = g;
  return start;
}

// Order-P B-spline weights of Sec. 2.3 for a particle at u = c + f (c integer, 0 <= f < 1) on one
// axis. Returns the first node of the stencil relative to c and writes the P weights of nodes
// start .. start+P-1, W^(P)(s) with s = node - u:
//   NGP  (P=1): the node with -1/2 <= s < 1/2 (half-open cell).
//   CIC  (P=2): nodes c, c+1: 1-f, f.
//   TSC  (P=3): nearest node m = floor(u + 1/2), t = u - m in [-1/2, 1/2): nodes m-1, m, m+1:
//               (1/2 - t)^2/2, 3/4 - t^2, (1/2 + t)^2/2.
//   PCS  (P=4): nodes c-1..c+2, g = 1-f: g^3/6, (4 - 6 f^2 + 3 f^3)/6, (4 - 6 g^2 + 3 g^3)/6, f^3/6.
template <int P, typename T>
__device__ __forceinline__ int bspline(T f, T* w) {
  if constexpr (P == 1) {
    w[0] = T(1);
    return f > T(0.5) ? 1 : 0;
  } else if constexpr (P == 2) {
    w[0] = T(1) - f;
    w[1] = f;
    return 0;
  } else if constexpr (P == 3) {
    const bool up = f >= T(0.5);
    const T t = up ? f - T(1) : f;
    const T a = T(0.5) - t, b = T(0.5) + t;
    w[0] = T(0.5) * a * a;
    w[1] = T(0.75) - t * t;
    w[2] = T(0.5) * b * b;
    return up ? 0 : -1;
  } else if constexpr (P == 4) {
    const T g = T(1) - f;
    const T f2 = f * f, g2 = g * g;
    const T sixth = T(1) / T(6);
    w[0] = g2 * g * sixth;
    w[1] = (T(4) - T(6) * f2 + T(3) * f2 * f) * sixth;
    w[2] = (T(4) - T(6) * g2 + T(3) * g2 * g) * sixth;
    w[3] = f2 * f * sixth;
    return -1;
  } else {
    T g;
    return bspline_high<P>(f, w, &g);
  }
}

// Same stencil as bspline<P>, returning d/du of each node weight W(node - u) (u = c + f).
template <int P, typename T>
__device__ __forceinline__ int bspline_deriv(T f, T* w, T* dw) {
  if constexpr (P == 2) {
    w[0] = T(1) - f; w[1] = f;
    dw[0] = T(-1); dw[1] = T(1);
    return 0;
  } else if constexpr (P == 3) {
    const bool up = f >= T(0.5);
    const T t = up ? f - T(1) : f;
    const T a = T(0.5) - t, b = T(0.5) + t;
    w[0] = T(0.5) * a * a; w[1] = T(0.75) - t * t; w[2] = T(0.5) * b * b;
    dw[0] = -a; dw[1] = T(-2) * t; dw[2] = b;
    return up ? 0 : -1;
  } else if constexpr (P == 4) {
    const T g = T(1) - f;
    const T f2 = f * f, g2 = g * g;
    const T sixth = T(1) / T(6);
    w[0] = g2 * g * sixth;
    w[1] = (T(4) - T(6) * f2 + T(3) * f2 * f) * sixth;
    w[2] = (T(4) - T(6) * g2 + T(3) * g2 * g) * sixth;
    w[3] = f2 * f * sixth;
    dw[0] = T(-0.5) * g2;
    dw[1] = T(-2) * f + T(1.5) * f2;
    dw[2] = T(2) * g - T(1.5) * g2;
    dw[3] = T(0.5) * f2;
    return -1;
  } else {
    // d/du N_P(m - g) = N_{P-1}(m - 1 - g) - N_{P-1}(m - g), and N_{P-1}(m - g) = c[P - 1 - m] for
    // 1 <= m <= P - 1 (zero outside), c the order P - 1 values at g
    T g;
    const int start = bspline_high<P>(f, w, &g);
    T c[P - 1];
    cardinal_bspline<P - 1>(g, c);
#pragma unroll
    for (int k = 0; k < P; ++k) dw[k] = (k >= 1 ? c[P - 1 - k] : T(0)) - (k <= P - 2 ? c[P - 2 - k] : T(0));
    return start;
  }
}

// Shift of the interlaced grid: u + 1/2 = c' + f' with c' = c + (f >= 1/2).
template <typename T>
__device__ __forceinline__ int half_shift(T f, T* f2) {
  const bool up = f >= T(0.5);
  *f2 = up ? f - T(0.5) : f + T(0.5);
  return up ? 1 : 0;
}

// Periodic index for i in [-n, 2n): every caller is a stencil node or a tile region node within a
// few cells of the grid (N >= 8), so one conditional correction replaces the integer remainder.
__device__ __forceinline__ int wrap(int i, int n) {
  i += i < 0 ? n : 0;
  return i >= n ? i - n : i;
}

// Signed mode index of FFT slot i (slot N/2 is -N/2).
__device__ __forceinline__ int signed_mode(int i, int n) { return i < n / 2 ? i : i - n; }

// Bin of a mode with 4|n|^2 = v4 for the edges e_b = lo2 + b w2 (units of k_f/2): e_b^2 <= v4 <
// e_{b+1}^2, decided exactly in integers after a floating-point guess; -1 outside the bins and for n = 0.
__device__ __forceinline__ int bin_of(long long v4, int lo2, int w2, int nbins) {
  if (v4 == 0) return -1;
  const float r = sqrtf(float(v4));
  int b = int(floorf((r - float(lo2)) / float(w2)));
  if (b < 0) b = 0;
  long long e = (long long)lo2 + (long long)b * w2;
  while (b > 0 && e * e > v4) { --b; e -= w2; }
  if (e * e > v4) return -1;
  long long e1 = e + w2;
  while (e1 * e1 <= v4) { ++b; e1 += w2; if (b >= nbins) return -1; }
  return b < nbins ? b : -1;
}

// bin_of in 32-bit integers, for 4|n|^2 < 2^31 (N <= 1024) and bin edges whose squares fit 32 bits
// (bin_lo2 + (nbins + 1) bin_w2 <= 46340); r = sqrt(v4) from the caller, inv_w2 = 1 / bin_w2.
__device__ __forceinline__ int bin_of32(int v4, float r, int lo2, int w2, float inv_w2, int nbins) {
  if (v4 == 0) return -1;
  int b = int(floorf((r - float(lo2)) * inv_w2));
  if (b < 0) b = 0;
  int e = lo2 + b * w2;
  while (b > 0 && e * e > v4) { --b; e -= w2; }
  if (e * e > v4) return -1;
  int e1 = e + w2;
  while (e1 * e1 <= v4) { ++b; e1 += w2; if (b >= nbins) return -1; }
  return b < nbins ? b : -1;
}

// Fixed-point scale 2^F of the deterministic grids, F = 62 - ceil(log2(sum |w|)): no node can hold
// more than the total mass, so the int64 sums cannot overflow.
__device__ __forceinline__ float fixed_scale(double total) {
  if (!(total > 1.0)) total = 1.0;
  int f = 62 - int(ceil(log2(total)));
  f = f < 0 ? 0 : (f > 62 ? 62 : f);
  return ldexpf(1.0f, f);
}

// Grid-stride helpers over int64 ranges.
__device__ __forceinline__ int64_t gtid() { return int64_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }

}  // namespace pk
