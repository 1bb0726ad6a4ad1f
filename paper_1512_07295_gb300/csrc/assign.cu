// a3 mass assignment (eq:delgrid, Sec. 2.3) on the grid and on the grid shifted by H/2 (Sec. 3.1).
//
// k_assign_direct: one thread per particle, FP64 weights, FP64 global atomics straight into the grid.
// This is the plain FP64 path (oracle-parity mode and the baseline the fast path is measured
// against): it accepts particles in any order. The FP32 and PK_FIXED64 paths run on the tiled kernels
// of assign_tiles.cu; this file also holds the conversions and weight sums they share.
#include "internal.cuh"

namespace pk {

PK_ERR_ACCESSOR(take_err_assign)

// ---- plain FP64 path ------------------------------------------------------------------------------

template <int P, typename G>
__device__ __forceinline__ void scatter_direct(G* __restrict__ g, const int* c, const double* f, double wgt, int ng,
                                               int ldz) {
  double wx[P], wy[P], wz[P];
  const int sx = bspline<P>(f[0], wx), sy = bspline<P>(f[1], wy), sz = bspline<P>(f[2], wz);
#pragma unroll
  for (int a = 0; a < P; ++a) {
    const int gx = wrap(c[0] + sx + a, ng);
#pragma unroll
    for (int b = 0; b < P; ++b) {
      const int gy = wrap(c[1] + sy + b, ng);
      const double wxy = wgt * wx[a] * wy[b];
      G* row = g + (int64_t(gx) * ng + gy) * ldz;
#pragma unroll
      for (int d = 0; d < P; ++d) atomicAdd(row + wrap(c[2] + sz + d, ng), G(wxy * wz[d]));
    }
  }
}

template <int P, typename G>
__global__ void k_assign_direct(const void* __restrict__ pos, int fmt, const float* __restrict__ w, int64_t n, int ng,
                                double box, int interlace, G* __restrict__ g1, G* __restrict__ g2, int ldz) {
  const double scale = double(ng) / box;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    int c[3];
    double f[3];
    if (fmt == PK_POS_F64_XYZ) {
      const double* p = static_cast<const double*>(pos) + 3 * i;
      bool bad = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double x = p[a];
        if (!isfinite(x)) { bad = true; x = 0.0; }
        if (!(x >= 0.0 && x < box)) {  // another periodic image (fmod is the identity on [0, L))
          x = fmod(x, box);
          if (x < 0.0) x += box;
        }
        const double u = x * scale;
        const double fl = floor(u);
        int ci = int(fl);
        f[a] = u - fl;
        if (ci >= ng) ci -= ng;
        c[a] = ci;
      }
      if (bad) { raise_err(PK_DERR_NONFINITE); continue; }
    } else {
      const pk_cellpos r = static_cast<const pk_cellpos*>(pos)[i];
      c[0] = cell_x(r.cell); c[1] = cell_y(r.cell); c[2] = cell_z(r.cell);
      f[0] = r.fx; f[1] = r.fy; f[2] = r.fz;
      if (c[0] >= ng || c[1] >= ng || c[2] >= ng || !(f[0] >= 0.0 && f[0] < 1.0 && f[1] >= 0.0 && f[1] < 1.0 &&
                                                      f[2] >= 0.0 && f[2] < 1.0)) {
        raise_err(PK_DERR_CELLRANGE);
        continue;
      }
    }
    const double wgt = w ? double(w[i]) : 1.0;
    scatter_direct<P>(g1, c, f, wgt, ng, ldz);
    if (interlace) {
      int c2[3];
      double f2[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) c2[a] = c[a] + half_shift(f[a], &f2[a]);
      scatter_direct<P>(g2, c2, f2, wgt, ng, ldz);
    }
  }
}

template <typename G>
static cudaError_t launch_direct(int order, const void* pos, int fmt, const float* w, int64_t n, int ng, double box,
                                 bool interlace, G* g1, G* g2, int ldz, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = int(std::min<int64_t>((n + threads - 1) / threads, int64_t(num_sms()) * 16));
  switch (order) {
    case 1: k_assign_direct<1, G><<<blocks, threads, 0, s>>>(pos, fmt, w, n, ng, box, interlace, g1, g2, ldz); break;
    case 2: k_assign_direct<2, G><<<blocks, threads, 0, s>>>(pos, fmt, w, n, ng, box, interlace, g1, g2, ldz); break;
    case 3: k_assign_direct<3, G><<<blocks, threads, 0, s>>>(pos, fmt, w, n, ng, box, interlace, g1, g2, ldz); break;
    case 4: k_assign_direct<4, G><<<blocks, threads, 0, s>>>(pos, fmt, w, n, ng, box, interlace, g1, g2, ldz); break;
    case 5: k_assign_direct<5, G><<<blocks, threads, 0, s>>>(pos, fmt, w, n, ng, box, interlace, g1, g2, ldz); break;
    case 6: k_assign_direct<6, G><<<blocks, threads, 0, s>>>(pos, fmt, w, n, ng, box, interlace, g1, g2, ldz); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_assign_direct_f64(int order, const void* pos, int fmt, const float* w, int64_t n, int ng, double box,
                                     bool interlace, double* g1, double* g2, int ldz, cudaStream_t s) {
  return launch_direct<double>(order, pos, fmt, w, n, ng, box, interlace, g1, g2, ldz, s);
}

// ---- small helpers ---------------------------------------------------------------------------------

__global__ void k_fixed_to_double(unsigned long long* g, int64_t count, const double* __restrict__ wsums) {
  const double inv_scale = 1.0 / double(fixed_scale(wsums[2]));
  for (int64_t i = gtid(); i < count; i += gstride()) {
    const long long v = (long long)g[i];
    reinterpret_cast<double*>(g)[i] = double(v) * inv_scale;
  }
}

cudaError_t launch_fixed_to_double(unsigned long long* g, int64_t count, const double* wsums, cudaStream_t s) {
  const int blocks = num_sms() * 8;
  k_fixed_to_double<<<blocks, 256, 0, s>>>(g, count, wsums); count_launch();
  return cudaGetLastError();
}

__global__ void k_weight_sums(const float* __restrict__ w, int64_t n, double* __restrict__ sums) {
  double a = 0.0, b = 0.0, c = 0.0;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    const double v = w[i];
    a += v;
    b += v * v;
    c += fabs(v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(sums, a);
    atomicAdd(sums + 1, b);
    atomicAdd(sums + 2, c);
  }
}

__global__ void k_set_sums(double* sums, double s1, double s2) {
  sums[0] = s1;
  sums[1] = s2;
  sums[2] = s1;
}

cudaError_t launch_weight_sums(const float* w, int64_t n, double* sums, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(sums, 0, 3 * sizeof(double), s);
  if (e != cudaSuccess || n == 0) return e;
  k_weight_sums<<<num_sms() * 4, 256, 0, s>>>(w, n, sums); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_set_sums(double* sums, double s1, double s2, cudaStream_t s) {
  k_set_sums<<<1, 1, 0, s>>>(sums, s1, s2); count_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void k_copy_rows(const T* __restrict__ src, int src_ld, T* __restrict__ dst, int dst_ld, int ng, int64_t rows) {
  const int64_t total = rows * ng;
  for (int64_t i = gtid(); i < total; i += gstride()) {
    const int64_t r = i / ng;
    const int z = int(i - r * ng);
    dst[r * dst_ld + z] = src[r * src_ld + z];
  }
}

template <typename T>
cudaError_t launch_copy_rows(const T* src, int src_ld, T* dst, int dst_ld, int ng, int64_t rows, cudaStream_t s) {
  k_copy_rows<T><<<num_sms() * 8, 256, 0, s>>>(src, src_ld, dst, dst_ld, ng, rows); count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_copy_rows<float>(const float*, int, float*, int, int, int64_t, cudaStream_t);
template cudaError_t launch_copy_rows<double>(const double*, int, double*, int, int, int64_t, cudaStream_t);

}  // namespace pk
