// a8 adjoint of the power spectrum with respect to particle positions (the paper has no adjoint; this
// is the chain rule through a3..a6).
//
// With P_b = (V/M_b) sum_{n in b} |delta(n)|^2, delta(n) = [G_1(n) + phi(n) G_2(n)] c(n),
// c(n) = a / (sum(w) W(n)) (a = 1/2 interlaced, 1 otherwise), phi(n) = e^{+i pi (n_x+n_y+n_z)/N}:
//   A(n)       = 2 kappa(n) c(n) conj(delta(n)),   kappa(n) = (dL/dP_b) V / M_b for n in bin b
//   dL/drho_1[j] = Re sum_n A(n) e^{-2 pi i n.j/N},   dL/drho_2[j] = Re sum_n A(n) phi(n) e^{-2 pi i n.j/N}.
// Re sum_n B(n) e^{-i theta_n} = sum_n X(n) e^{+i theta_n} with X(n) = [conj B(n) + B(-n)] / 2 Hermitian,
// i.e. one inverse real FFT per grid. B(-n) uses delta(-n) = [conj G_1(n) + phi(-n) conj G_2(n)] c(n),
// with the Nyquist-slot phase rule of the forward estimate. Finally
//   dL/dx_{i,a} = w_i (N/L) sum_g sum_{j in stencil} dL/drho_g[j] dW(j_a - u_a)/du_a prod_{b != a} W(j_b - u_b).
#include "host.cuh"

namespace pk {

template <typename R>
struct CC {
  R x, y;
};
template <typename R>
__device__ __forceinline__ CC<R> mul(CC<R> a, CC<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R>
__device__ __forceinline__ CC<R> cj(CC<R> a) {
  return {a.x, -a.y};
}

// In place: (G_1, G_2) at every stored slot -> (X_1, X_2); window and phases evaluated in FP64.
template <typename R>
__global__ void k_adjoint_modes(CC<R>* __restrict__ G1, CC<R>* __restrict__ G2, int ng, int order, int interlace,
                                int lo2, int w2, int nbins, double box, const double* __restrict__ wsums,
                                const double* __restrict__ dl_dpk, const unsigned long long* __restrict__ counts) {
  const int half = ng / 2, lz = half + 1;
  const int64_t nh = int64_t(ng) * ng * lz;
  const double vol = box * box * box;
  const double a = interlace ? 0.5 : 1.0;
  const double wsum = wsums[0];
  for (int64_t i = gtid(); i < nh; i += gstride()) {
    const int iz = int(i % lz);
    const int64_t row = i / lz;
    const int iy = int(row % ng), ix = int(row / ng);
    const int n[3] = {signed_mode(ix, ng), signed_mode(iy, ng), iz == half ? -half : iz};
    const long long n2 = (long long)n[0] * n[0] + (long long)n[1] * n[1] + (long long)n[2] * n[2];
    const int b = bin_of(4 * n2, lo2, w2, nbins);
    CC<R> x1 = {R(0), R(0)}, x2 = {R(0), R(0)};
    if (b >= 0 && counts[b] > 0) {
      // window, phases (signed index of the mode and of its partner on each axis)
      double w = 1.0;
      double ph = 0.0, php = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double t = 3.14159265358979323846 * double(n[k]) / double(ng);
        const double s = n[k] == 0 ? 1.0 : sin(t) / t;
        double wk = 1.0;
        for (int q = 0; q < order; ++q) wk *= s;
        w *= wk;
        ph += t;
        const int slot = k == 0 ? ix : (k == 1 ? iy : iz);
        php += (slot == half) ? t : -t;  // the partner of a Nyquist slot keeps n = -N/2
      }
      const R c = R(a / (wsum * w));
      const R kap2c = R(2.0 * dl_dpk[b] * vol / double(counts[b])) * c;
      const CC<R> phi = {R(cos(ph)), R(sin(ph))}, phip = {R(cos(php)), R(sin(php))};
      const CC<R> g1 = G1[i];
      const CC<R> g2 = interlace ? G2[i] : CC<R>{R(0), R(0)};
      CC<R> d, dm;
      if (interlace) {
        const CC<R> t = mul(phi, g2), tp = mul(phip, cj(g2));
        d = {(g1.x + t.x) * c, (g1.y + t.y) * c};
        dm = {(g1.x + tp.x) * c, (-g1.y + tp.y) * c};
      } else {
        d = {g1.x * c, g1.y * c};
        dm = cj(d);
      }
      const CC<R> A = {kap2c * d.x, -kap2c * d.y};     // 2 kappa c conj(delta(n))
      const CC<R> Am = {kap2c * dm.x, -kap2c * dm.y};  // 2 kappa c conj(delta(-n))
      // X_1 = [conj A(n) + A(-n)] / 2
      x1 = {R(0.5) * (A.x + Am.x), R(0.5) * (-A.y + Am.y)};
      if (interlace) {
        const CC<R> B = mul(A, phi), Bm = mul(Am, phip);
        x2 = {R(0.5) * (B.x + Bm.x), R(0.5) * (-B.y + Bm.y)};
      }
    }
    G1[i] = x1;
    if (interlace) G2[i] = x2;
  }
}

template <int P, typename R>
__device__ __forceinline__ void gather_grid(const R* __restrict__ g, const int* c, const R* f, int ng, R* grad) {
  R w[3][P], dw[3][P];
  int st[3];
  for (int a = 0; a < 3; ++a) st[a] = bspline_deriv<P>(f[a], w[a], dw[a]);
  const int ldz = ng + 2;
  for (int i = 0; i < P; ++i) {
    const int gx = wrap(c[0] + st[0] + i, ng);
    for (int j = 0; j < P; ++j) {
      const int gy = wrap(c[1] + st[1] + j, ng);
      const R* row = g + (int64_t(gx) * ng + gy) * ldz;
      for (int k = 0; k < P; ++k) {
        const R v = row[wrap(c[2] + st[2] + k, ng)];
        grad[0] += v * dw[0][i] * w[1][j] * w[2][k];
        grad[1] += v * w[0][i] * dw[1][j] * w[2][k];
        grad[2] += v * w[0][i] * w[1][j] * dw[2][k];
      }
    }
  }
}

template <int P, typename R>
__global__ void k_gather(const void* __restrict__ pos, int fmt, const float* __restrict__ wts, int64_t n, int ng, double box,
                         int interlace, int f32pos, const R* __restrict__ g1, const R* __restrict__ g2, R* __restrict__ out) {
  const double scale = double(ng) / box;
  for (int64_t i = gtid(); i < n; i += gstride()) {
    int c[3];
    R f[3];
    bool ok = true;
    if (fmt == PK_POS_F64_XYZ) {
      const double* p = static_cast<const double*>(pos) + 3 * i;
      for (int a = 0; a < 3; ++a) {
        double x = p[a];
        if (!isfinite(x)) { ok = false; x = 0.0; }
        if (!(x >= 0.0 && x < box)) {  // another periodic image (fmod is the identity on [0, L))
          x = fmod(x, box);
          if (x < 0.0) x += box;
        }
        const double u = x * scale;
        const double fl = floor(u);
        int ci = int(fl);
        if (ci >= ng) ci -= ng;
        double fr = u - fl;
        if (f32pos) {  // same rounding as the forward's position preparation (PK_FP32, PK_FIXED64)
          float ff = float(fr);
          if (ff >= 1.0f) { ff = 0.0f; ci = ci + 1 == ng ? 0 : ci + 1; }
          fr = ff;
        }
        c[a] = ci;
        f[a] = R(fr);
      }
    } else {
      const pk_cellpos r = static_cast<const pk_cellpos*>(pos)[i];
      c[0] = cell_x(r.cell); c[1] = cell_y(r.cell); c[2] = cell_z(r.cell);
      f[0] = R(r.fx); f[1] = R(r.fy); f[2] = R(r.fz);
      ok = c[0] < ng && c[1] < ng && c[2] < ng;
    }
    R grad[3] = {R(0), R(0), R(0)};
    if (ok) {
      gather_grid<P, R>(g1, c, f, ng, grad);
      if (interlace) {
        int c2[3];
        R f2[3];
        for (int a = 0; a < 3; ++a) c2[a] = c[a] + half_shift(f[a], &f2[a]);
        gather_grid<P, R>(g2, c2, f2, ng, grad);
      }
    }
    const R s = R(scale) * (wts ? R(wts[i]) : R(1));
    out[3 * i] = grad[0] * s;
    out[3 * i + 1] = grad[1] * s;
    out[3 * i + 2] = grad[2] * s;
  }
}

template <typename R>
static cudaError_t launch_gather(int order, const void* pos, int fmt, const float* w, int64_t n, int ng, double box, int interlace,
                                 int f32pos, const R* g1, const R* g2, R* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int blocks = int(std::min<int64_t>((n + 255) / 256, int64_t(num_sms()) * 16));
  switch (order) {
    case 2: k_gather<2, R><<<blocks, 256, 0, s>>>(pos, fmt, w, n, ng, box, interlace, f32pos, g1, g2, out); count_launch(); break;
    case 3: k_gather<3, R><<<blocks, 256, 0, s>>>(pos, fmt, w, n, ng, box, interlace, f32pos, g1, g2, out); count_launch(); break;
    case 4: k_gather<4, R><<<blocks, 256, 0, s>>>(pos, fmt, w, n, ng, box, interlace, f32pos, g1, g2, out); count_launch(); break;
    case 5: k_gather<5, R><<<blocks, 256, 0, s>>>(pos, fmt, w, n, ng, box, interlace, f32pos, g1, g2, out); count_launch(); break;
    default: k_gather<6, R><<<blocks, 256, 0, s>>>(pos, fmt, w, n, ng, box, interlace, f32pos, g1, g2, out); count_launch(); break;
  }
  return cudaGetLastError();
}

struct BackLayout {
  ForwardStage f;
  PlanEntry inv;
  void* inv_work = nullptr;
};

static pk_status carve_back(const pk_config* c, int64_t n, Carver& cv, BackLayout* L) {
  pk_status st = carve_forward(c, n, cv, &L->f);
  if (st != PK_OK) return st;
  const bool dbl = c->prec != PK_FP32;
  if ((st = get_plan(c->ng, dbl ? 3 : 2, c->interlace ? 2 : 1, &L->inv)) != PK_OK) return st;
  L->inv_work = cv.take<char>(std::max<size_t>(L->inv.work, 256));
  return PK_OK;
}

pk_status backward_ws(const pk_config* c, int64_t n, size_t* out) {
  Carver cv(nullptr);
  BackLayout L;
  pk_status st = carve_back(c, n, cv, &L);
  if (st != PK_OK) return st;
  *out = cv.size();
  return PK_OK;
}

}  // namespace pk

using namespace pk;

extern "C" pk_status pk_power_backward(const pk_config* cfg, const void* pos_dev, int32_t pos_format, const float* w_dev,
                                       int64_t n, const double* dl_dpk_dev, void* dl_dx_dev, void* ws, size_t ws_bytes,
                                       void* stream) {
  clear_err();
  pk_status st = validate(cfg);
  if (st != PK_OK) return st;
  if (cfg->order < 2) return fail(PK_EINVAL, "the adjoint needs order 2..6 (NGP has no derivative)");
  if (pos_format != PK_POS_F64_XYZ && pos_format != PK_POS_CELL_F32OFF) return fail(PK_EINVAL, "bad pos_format");
  if (n < 1 || !pos_dev || !dl_dpk_dev || !dl_dx_dev) return fail(PK_EINVAL, "bad pointers");
  size_t need = 0;
  if ((st = backward_ws(cfg, n, &need)) != PK_OK) return st;
  if (!ws || ws_bytes < need) return fail(PK_ESIZE, "workspace %zu < %zu bytes", ws_bytes, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver cv(ws);
  BackLayout L;
  if ((st = carve_back(cfg, n, cv, &L)) != PK_OK) return st;
  GridStage& g = L.f.g;
  // forward grids and their transforms (recomputed), then the exact mode counts of the bins
  if ((st = run_forward_grids(cfg, pos_dev, pos_format, w_dev, n, L.f, s)) != PK_OK) return st;
  if ((st = exec_plan(g.plan, g.kind, g.grids, g.fft_work, s)) != PK_OK) return st;
  const bool dbl = cfg->prec != PK_FP32;
  EstimateArgs a;
  a.ng = cfg->ng;
  a.order = cfg->order;
  a.interlace = cfg->interlace;
  a.nbins = cfg->nbins;
  a.bin_lo2 = cfg->bin_lo2;
  a.bin_w2 = cfg->bin_w2;
  a.box = cfg->box;
  a.wsums = g.wsums;
  a.bin_sum = g.bin_sum;
  a.bin_k = g.bin_k;
  a.bin_cnt = g.bin_cnt;
  a.delta_out = nullptr;
  cudaError_t e;
  if ((e = cudaMemsetAsync(g.bin_sum, 0, sizeof(double) * cfg->nbins, s)) != cudaSuccess) return cuda_fail(e, "memset");
  if ((e = cudaMemsetAsync(g.bin_k, 0, sizeof(double) * cfg->nbins, s)) != cudaSuccess) return cuda_fail(e, "memset");
  if ((e = cudaMemsetAsync(g.bin_cnt, 0, sizeof(unsigned long long) * cfg->nbins, s)) != cudaSuccess) return cuda_fail(e, "memset");
  const int64_t per = padded_count(cfg->ng);
  const size_t gbytes = size_t(per) * (dbl ? 8 : 4);
  void* G1 = g.grids;
  void* G2 = cfg->interlace ? static_cast<char*>(g.grids) + gbytes : nullptr;
  e = dbl ? launch_estimate<double>(G1, G2, g.tables, a, s) : launch_estimate<float>(G1, G2, g.tables, a, s);
  if (e != cudaSuccess) return cuda_fail(e, "mode counts");
  const int blocks = num_sms() * 8;
  if (dbl)
    k_adjoint_modes<double><<<blocks, 256, 0, s>>>(static_cast<CC<double>*>(G1), static_cast<CC<double>*>(G2), cfg->ng,
                                                   cfg->order, cfg->interlace, cfg->bin_lo2, cfg->bin_w2, cfg->nbins, cfg->box,
                                                   g.wsums, dl_dpk_dev, g.bin_cnt);
  else
    k_adjoint_modes<float><<<blocks, 256, 0, s>>>(static_cast<CC<float>*>(G1), static_cast<CC<float>*>(G2), cfg->ng,
                                                  cfg->order, cfg->interlace, cfg->bin_lo2, cfg->bin_w2, cfg->nbins, cfg->box,
                                                  g.wsums, dl_dpk_dev, g.bin_cnt); count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "adjoint modes");
  if ((st = exec_plan(L.inv, dbl ? 3 : 2, g.grids, L.inv_work, s)) != PK_OK) return st;
  if (dbl)
    e = launch_gather<double>(cfg->order, pos_dev, pos_format, w_dev, n, cfg->ng, cfg->box, cfg->interlace,
                              cfg->prec != PK_FP64, static_cast<const double*>(G1), static_cast<const double*>(G2), static_cast<double*>(dl_dx_dev), s);
  else
    e = launch_gather<float>(cfg->order, pos_dev, pos_format, w_dev, n, cfg->ng, cfg->box, cfg->interlace, 1,
                             static_cast<const float*>(G1), static_cast<const float*>(G2), static_cast<float*>(dl_dx_dev), s);
  return e == cudaSuccess ? PK_OK : cuda_fail(e, "gather");
}
