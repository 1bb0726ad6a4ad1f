// Residual aliasing factor of the window-corrected (and optionally interlaced) grid estimate,
// F_res(k) = sum_{m != 0} theta_m |w_m(k)|^2 (eq:res, with |w_m(k)|^2 = |W(k - m k_s)|^2 / |W(k)|^2),
// evaluated on every mode of the grid and averaged per k-bin: the analytic prediction of the aliasing
// left in P(k) (Sec. 3.2), e.g. a Poisson catalogue's window-corrected power is (1 + F_res) / nbar.
//
// With x = n / N and |W| = sinc^p, |w_m|^2 = prod_i (x_i / (x_i - m_i))^{2p}, so the image sum factorises
// per axis into the one-dimensional forms of eq:res1Dnoi and eq:res1Di:
//   f(x)  = sum_{m != 0} (x/(x-m))^{2p} = x^{2p} [zeta(2p, 1-x) + zeta(2p, 1+x)],
//   F_int(x) = f(x/2) (even images only),   f'(x) = sum_{m != 0} (-1)^m (x/(x-m))^{2p} = 2 F_int(x) - f(x),
//   F_res = prod(1 + f_i) - 1                              (no interlacing, theta_m = 1),
//   F_res = [prod(1 + f_i) + prod(1 + f'_i)] / 2 - 1       (interlacing, theta_m = [1 + (-1)^{sum m}]/2),
// the products expanded so that nothing close to 1 is subtracted from 1. The Hurwitz zeta function is
// summed directly for 16 terms and completed with the Euler-Maclaurin tail (six Bernoulli terms).
#include "host.cuh"

namespace pk {

// zeta(s, q) = sum_{k >= 0} (k + q)^{-s}, integer s >= 2, q > 0.
__device__ double hurwitz_zeta(int s, double q) {
  constexpr int M = 16;
  double sum = 0.0;
  for (int k = 0; k < M; ++k) sum += pow(k + q, -double(s));
  const double a = M + q;
  // tail: int_M^inf + g(M)/2 - sum_j B_2j/(2j)! g^(2j-1)(M), g(t) = (t + q)^{-s}
  double tail = pow(a, 1.0 - s) / (s - 1) + 0.5 * pow(a, -double(s));
  const double b2j[6] = {1.0 / 6.0, -1.0 / 30.0, 1.0 / 42.0, -1.0 / 30.0, 5.0 / 66.0, -691.0 / 2730.0};
  double fact = 1.0;   // (2j)!
  double rising = s;   // s (s+1) ... (s + 2j - 2)
  double pw = pow(a, -double(s) - 1.0);
  for (int j = 1; j <= 6; ++j) {
    fact *= double(2 * j - 1) * double(2 * j);
    tail += b2j[j - 1] / fact * rising * pw;
    rising *= double(s + 2 * j - 1) * double(s + 2 * j);
    pw /= a * a;
  }
  return sum + tail;
}

__device__ double fres_axis(double x, int p) {  // f(x), eq:res1Dnoi
  if (x == 0.0) return 0.0;
  return pow(x, 2.0 * p) * (hurwitz_zeta(2 * p, 1.0 - x) + hurwitz_zeta(2 * p, 1.0 + x));
}

// tab[i] = f(x_i), tab[N + i] = f'(x_i) for slot i (x_i = signed(i) / N).
__global__ void k_alias_tables(double* __restrict__ tab, int ng, int order) {
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < ng; i += blockDim.x * gridDim.x) {
    const double x = double(signed_mode(i, ng)) / double(ng);
    const double f = fres_axis(x, order);
    tab[i] = f;
    tab[ng + i] = 2.0 * fres_axis(0.5 * x, order) - f;
  }
}

__device__ __forceinline__ double excess3(double a, double b, double c) {  // (1+a)(1+b)(1+c) - 1
  return a + b + c + a * b + a * c + b * c + a * b * c;
}

// Per bin: sum of multiplicity x F_res, of multiplicity x |n|, the mode count (the multiplicities of the
// half-complex layout: 2 for 0 < i_z < N/2; F_res is even in n) and the largest F_res (non-negative
// doubles order like their bit patterns).
__global__ void __launch_bounds__(256) k_alias_bins(const double* __restrict__ tab_g, int ng, int interlace, int lo2,
                                                    int w2, int nbins, double* __restrict__ bin_sum,
                                                    double* __restrict__ bin_k, unsigned long long* __restrict__ bin_cnt,
                                                    unsigned long long* __restrict__ bin_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* tab = reinterpret_cast<double*>(smem_raw);  // [2][ng]
  double* s_sum = tab + 2 * ng;
  double* s_k = s_sum + nbins;
  unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(s_k + nbins);
  unsigned long long* s_max = s_cnt + nbins;
  for (int i = threadIdx.x; i < 2 * ng; i += blockDim.x) tab[i] = tab_g[i];
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
    s_sum[i] = 0.0;
    s_k[i] = 0.0;
    s_cnt[i] = 0ull;
    s_max[i] = 0ull;
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
    double f = excess3(tab[ix], tab[iy], tab[iz]);  // slot i_z = N/2 holds n_z = -N/2
    if (interlace) f = 0.5 * (f + excess3(tab[ng + ix], tab[ng + iy], tab[ng + iz]));
    const int mult = (iz == 0 || iz == ng / 2) ? 1 : 2;
    atomicAdd(&s_sum[b], double(mult) * f);
    atomicAdd(&s_k[b], double(mult) * sqrt(double(n2)));
    atomicAdd(&s_cnt[b], (unsigned long long)mult);
    atomicMax(&s_max[b], (unsigned long long)__double_as_longlong(fmax(f, 0.0)));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
    if (s_cnt[i] == 0ull) continue;
    atomicAdd(&bin_sum[i], s_sum[i]);
    atomicAdd(&bin_k[i], s_k[i]);
    atomicAdd(&bin_cnt[i], s_cnt[i]);
    atomicMax(&bin_max[i], s_max[i]);
  }
}

__global__ void k_alias_final(const double* __restrict__ bin_sum, const double* __restrict__ bin_k,
                              const unsigned long long* __restrict__ bin_cnt, const unsigned long long* __restrict__ bin_max,
                              int nbins, double kf, double* __restrict__ mean, double* __restrict__ mx,
                              double* __restrict__ kmean, int64_t* __restrict__ nmodes) {
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  for (int b = threadIdx.x + blockIdx.x * blockDim.x; b < nbins; b += blockDim.x * gridDim.x) {
    const unsigned long long m = bin_cnt[b];
    nmodes[b] = int64_t(m);
    mean[b] = m ? bin_sum[b] / double(m) : nan;
    if (mx) mx[b] = m ? __longlong_as_double((long long)bin_max[b]) : nan;
    if (kmean) kmean[b] = m ? kf * bin_k[b] / double(m) : nan;
  }
}

namespace {

struct AliasLayout {
  double* tab = nullptr;
  double* bin_sum = nullptr;
  double* bin_k = nullptr;
  unsigned long long* bin_cnt = nullptr;
  unsigned long long* bin_max = nullptr;
};

void carve_alias(const pk_config* c, Carver& cv, AliasLayout* L) {
  L->tab = cv.take<double>(size_t(2) * c->ng);
  L->bin_sum = cv.take<double>(c->nbins);
  L->bin_k = cv.take<double>(c->nbins);
  L->bin_cnt = cv.take<unsigned long long>(c->nbins);
  L->bin_max = cv.take<unsigned long long>(c->nbins);
}

}  // namespace

pk_status aliasing_ws(const pk_config* c, size_t* out) {
  Carver cv(nullptr);
  AliasLayout L;
  carve_alias(c, cv, &L);
  *out = cv.size();
  return PK_OK;
}

}  // namespace pk

using namespace pk;

extern "C" {

pk_status pk_aliasing_residual(const pk_config* cfg, double* fres_mean_dev, double* fres_max_dev, double* kmean_dev,
                               int64_t* nmodes_dev, void* ws, size_t ws_bytes, void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (!fres_mean_dev || !nmodes_dev) return fail(PK_EINVAL, "bad pointers");
  const size_t need = pk_workspace_size(cfg, 0, PK_WS_ALIASING);
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  AliasLayout L;
  carve_alias(cfg, cv, &L);
  const size_t nb = size_t(cfg->nbins);
  cudaError_t e;
  if ((e = cudaMemsetAsync(L.bin_sum, 0, sizeof(double) * nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(L.bin_k, 0, sizeof(double) * nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(L.bin_cnt, 0, sizeof(unsigned long long) * nb, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(L.bin_max, 0, sizeof(unsigned long long) * nb, s)) != cudaSuccess)
    return cuda_fail(e, "memset");
  const int ng = cfg->ng;
  k_alias_tables<<<(ng + 127) / 128, 128, 0, s>>>(L.tab, ng, cfg->order); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "aliasing tables");
  const int64_t hc = half_count(ng);
  const int blocks = int(std::min<int64_t>(int64_t(num_sms()) * 4, (hc + 255) / 256));
  const size_t smem = sizeof(double) * 2 * size_t(ng) + nb * (2 * sizeof(double) + 2 * sizeof(unsigned long long));
  if ((e = ensure_dynamic_smem(reinterpret_cast<const void*>(k_alias_bins), smem)) != cudaSuccess)
    return cuda_fail(e, "aliasing smem");
  k_alias_bins<<<blocks, 256, smem, s>>>(L.tab, ng, cfg->interlace, cfg->bin_lo2, cfg->bin_w2, cfg->nbins, L.bin_sum, L.bin_k,
                                         L.bin_cnt, L.bin_max); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "aliasing bins");
  const double kf = 2.0 * 3.14159265358979323846 / cfg->box;
  k_alias_final<<<(cfg->nbins + 255) / 256, 256, 0, s>>>(L.bin_sum, L.bin_k, L.bin_cnt, L.bin_max, cfg->nbins, kf,
                                                          fres_mean_dev, fres_max_dev, kmean_dev, nmodes_dev); count_launch();
  e = cudaGetLastError();
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "aliasing final");
}

}  // extern "C"
