/*
 * pk.h -- C ABI of the GB300 (sm_103a) Fourier-space estimator library (libpk.so).
 *
 * Method: Sefusatti, Crocce, Scoccimarro & Couchman, "Accurate Estimators of Correlation Functions
 * in Fourier Space" (arXiv:1512.07295). Particles are assigned to a periodic grid with the order-p
 * B-spline kernels of Sec. 2.3 (eq:delgrid), both on the grid and on a second grid offset by H/2
 * (interlacing, Sec. 3.1); each grid is Fourier transformed, divided by the window
 * W(k) = prod_i sinc^p(pi k_i / k_s) (eq:windowcorrection, eq:intkerFT) and the two are averaged with
 * the phase exp(+i k.(H/2)(1,1,1)) that cancels the odd alias images (eq:intdelta). |delta(k)|^2 is
 * binned in k-shells (power spectrum, Sec. 2.2) and the shell-filtered fields give the bispectrum
 * (eq:Best2, eq:IntI).
 *
 * Conventions used by every entry point:
 *   - N = cfg->ng grid points per side, H = L/N, V = L^3, k_f = 2 pi / L, N_c = N^3.
 *   - delta(n) = (1/N_c) sum_j (rho_j/rhobar - 1) exp(-2 pi i n.j/N); P(n) = V |delta(n)|^2, i.e. the
 *     paper's P times (2 pi)^3. Signed mode index n_i in [-N/2, N/2).
 *   - Grid 2 holds the particles shifted by +H/2 on every axis; it is combined as
 *     delta = [G1 + exp(+i pi (n_x+n_y+n_z)/N) G2] / (2 sum(w) W(n)), G_g the DFT of mass grid g.
 *   - Power-spectrum bins: edges e_b = bin_lo2 + b*bin_w2 (b = 0..nbins) in units of k_f/2; mode
 *     n != 0 is in bin b when e_b^2 <= 4|n|^2 < e_{b+1}^2 (exact integer test).
 *
 * Memory and ownership: every pointer argument named *_dev, and every output array, is device
 * memory owned by the caller (for example a torch tensor). Host pointers are named *_host. The
 * library allocates no device memory of its own: each call that needs scratch takes a workspace
 * (ws, ws_bytes) of at least pk_workspace_size() bytes, 256-byte aligned. The one exception is the
 * internal state cuFFT keeps in a plan (twiddle tables), created once per (device, N, precision,
 * batch) and cached for the life of the process; its work area is taken from the workspace.
 *
 * Streams and errors: every call is asynchronous on the caller's stream (a cudaStream_t passed as
 * void*, NULL = legacy default stream); nothing synchronises the device. Arguments are validated on
 * the host before any launch: an invalid configuration returns PK_EINVAL, a workspace or buffer that
 * is too small PK_ESIZE, and no work is queued. Launch and cuFFT failures return PK_ECUDA/PK_ECUFFT.
 * Conditions found on the device (a non-finite position, a particle outside the packed-cell range,
 * a bounded wait that ran out) set a device error word that pk_device_error() reads and clears.
 * On any error the contents of the outputs are undefined. pk_last_error() returns a thread-local
 * message describing the last failure.
 */
#ifndef PK_H
#define PK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PK_OK = 0,
  PK_EINVAL = 1,   /* invalid configuration or argument; nothing was launched */
  PK_ESIZE = 2,    /* workspace or output buffer too small; nothing was launched */
  PK_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
  PK_ECUFFT = 4,   /* a cuFFT call failed */
  PK_ETIMEOUT = 5, /* a bounded device-side wait ran out (reported through pk_device_error) */
  PK_EDEVICE = 6   /* the device error word was set (see pk_device_error) */
} pk_status;

typedef enum {
  PK_FP64 = 0,   /* FP64 positions arithmetic, FP64 grids, FP64 FFT: the oracle-parity mode */
  PK_FP32 = 1,   /* cell index + FP32 offset arithmetic, FP32 grids and FFT, FP64 shell sums */
  PK_FIXED64 = 2 /* as PK_FP32, but grids accumulated in 64-bit fixed point: bit-reproducible */
} pk_precision;

typedef enum {
  PK_POS_F64_XYZ = 0,    /* double[n][3], length units, any value (wrapped into [0, L)) */
  PK_POS_CELL_F32OFF = 1 /* pk_cellpos[n] (below), relative to the grid of cfg->ng */
} pk_pos_format;

/* Device error word bits (pk_device_error). */
#define PK_DERR_NONFINITE 1u  /* a position was NaN or infinite; the particle was skipped */
#define PK_DERR_CELLRANGE 2u  /* a packed cell coordinate was >= N or an offset outside [0,1) */
#define PK_DERR_TIMEOUT 4u    /* a bounded device-side wait ran out */

/* A particle on the grid of side N: cell = cx << 20 | cy << 10 | cz (each coordinate < N <= 1024),
 * and the offset of the particle inside that cell in units of H, each in [0, 1). 16 bytes. */
typedef struct {
  uint32_t cell;
  float fx, fy, fz;
} pk_cellpos;

typedef struct {
  int32_t ng;            /* N: even, 8 <= N <= 1024 */
  int32_t order;         /* p: 1 NGP, 2 CIC, 3 TSC, 4 PCS (Sec. 2.3); 5, 6 the next B-splines
                            (PK_FP64 and PK_FP32, pk_batch_power included) */
  int32_t interlace;     /* 1: add the H/2-shifted grid (Sec. 3.1); 0: single grid */
  int32_t prec;          /* pk_precision */
  double box;            /* L > 0 */
  int32_t bin_lo2;       /* first bin edge in units of k_f/2 (>= 0) */
  int32_t bin_w2;        /* bin width in units of k_f/2 (>= 1) */
  int32_t nbins;         /* number of bins (1..2048) */
  int32_t subtract_shot; /* 1: subtract the shot noise V sum(w^2)/sum(w)^2 from every bin */
  int32_t tile_run;      /* PK_FP32 sparse tiles: tiles per scatter region along z (1, 2, 4; 0 = chosen
                            from the mean tile population). A run of S tiles shares one shared-memory
                            region of 12 x 12 x (8 S + 4) nodes per grid. */
} pk_config;

/* Which call pk_workspace_size sizes. */
typedef enum {
  PK_WS_ASSIGN = 0,
  PK_WS_FFT_ESTIMATE = 1,
  PK_WS_POWER = 2,
  PK_WS_POWER_BINNED = 3,
  PK_WS_BIN = 4,
  PK_WS_BACKWARD = 5,
  PK_WS_BISPECTRUM = 6,
  PK_WS_BISPECTRUM_COUNTS = 7,
  PK_WS_POWER_HOST = 8,
  PK_WS_DIRECT = 9,
  PK_WS_CROSS = 10,
  PK_WS_ALIASING = 11
} pk_ws_kind;

/* Fills cfg with the paper's default binning for an N grid: bins centred on b k_f, b = 1..N/2
 * (bin_lo2 = 1, bin_w2 = 2, nbins = N/2), PCS with interlacing, FP32, no shot-noise subtraction. */
void pk_default_config(pk_config* cfg, int32_t ng, double box);

/* Bytes of workspace the call `kind` needs for this configuration and n particles (for
 * PK_WS_BISPECTRUM / _COUNTS, n is the number of shells). Returns 0 for an invalid configuration
 * (see pk_last_error). */
size_t pk_workspace_size(const pk_config* cfg, int64_t n, int32_t kind);

/* Workspace of pk_batch_power for groups of `batch` catalogues holding at most
 * max_group_particles particles in total. Returns 0 for invalid arguments. */
size_t pk_batch_workspace_size(const pk_config* cfg, int32_t batch, int64_t max_group_particles);

/* Number of tiles per axis used by the binned layout: ceil(N / tile_cells(N)). The tile edge in
 * cells is written to *tile_cells. */
int32_t pk_tiles_per_axis(const pk_config* cfg, int32_t* tile_cells);

/* a1 -- Position preparation (Sec. 2.3, s = (x_j - x)/H): wraps FP64 positions into [0, L) and
 * converts them to the packed cell + FP32 offset form of the grid cfg->ng.
 *   pos_dev: double[n][3] (device); out_dev: pk_cellpos[n] (device).
 * Non-finite positions set PK_DERR_NONFINITE and are written as cell 0, offset 0 (weight them out). */
pk_status pk_prepare(const pk_config* cfg, const double* pos_dev, int64_t n, pk_cellpos* out_dev,
                     void* stream);

/* a2 -- Counting sort of particles by cell tile (T^3 cells, T from pk_tiles_per_axis): the
 * "binned" layout the fast assignment reads. Input positions in either format (and optional
 * weights w_dev, float[n], NULL for unit weights); outputs sorted_dev (pk_cellpos[n]),
 * w_sorted_dev (float[n], or NULL when w_dev is NULL) and tile_offsets_dev (int64[ntiles + 1],
 * ntiles = tiles_per_axis^3, the start of each tile's particles; the last entry is n).
 * Inside a tile, particles are ordered by half-cell slab along x, 2 (c_x mod T) + [f_x >= 1/2]
 * (no defined order within a slab); the assignment of pk_power_binned accepts any order inside a
 * tile, so a binned layout made elsewhere only has to keep each tile's particles together. Invalid
 * packed records (a coordinate >= N or an offset outside [0, 1)) set PK_DERR_CELLRANGE and are
 * written as cell 0, offset 0. */
pk_status pk_bin(const pk_config* cfg, const void* pos_dev, int32_t pos_format, const float* w_dev,
                 int64_t n, pk_cellpos* sorted_dev, float* w_sorted_dev, int64_t* tile_offsets_dev,
                 void* ws, size_t ws_bytes, void* stream);

/* a3 -- Mass assignment (eq:delgrid; interlaced grid of Sec. 3.1): grid1[j] = sum_i w_i
 * prod_axis W^(p)(j_axis - u_i,axis), grid2 the same with u + 1/2 (skipped when grid2_dev is NULL
 * or cfg->interlace is 0). Outputs are unpadded N^3 C-order arrays (x slowest) of double (PK_FP64,
 * PK_FIXED64) or float (PK_FP32), overwritten. w_dev: float[n] weights or NULL (unit weights). */
pk_status pk_assign(const pk_config* cfg, const void* pos_dev, int32_t pos_format, const float* w_dev,
                    int64_t n, void* grid1_dev, void* grid2_dev, void* ws, size_t ws_bytes, void* stream);

/* a4+a5 -- FFT and window-corrected, interlaced density (eq:windowcorrection, eq:intdelta).
 * grid1_dev / grid2_dev: unpadded N^3 mass grids as written by pk_assign (grid2 ignored unless
 * cfg->interlace); wsum: sum of the particle weights. delta_k_dev receives delta(n) on the
 * half-complex layout [N][N][N/2+1] (complex double for PK_FP64/PK_FIXED64, complex float for
 * PK_FP32), index (i_x, i_y, i_z) <-> n = (signed(i_x), signed(i_y), i_z) with i_z = N/2 meaning
 * n_z = -N/2; delta(0) = 0. The grids are not modified. */
pk_status pk_fft_estimate(const pk_config* cfg, const void* grid1_dev, const void* grid2_dev, double wsum,
                          void* delta_k_dev, void* ws, size_t ws_bytes, void* stream);

/* a1..a6 -- Power spectrum of a catalogue in any order (Sec. 2.2 estimator on the interlaced,
 * window-corrected grid). Outputs (device, length nbins): pk_dev (mean V|delta|^2 per bin, shot noise
 * subtracted if cfg->subtract_shot; NaN for an empty bin), kmean_dev (mean |k| of the bin's modes),
 * nmodes_dev (int64 mode count, exact). delta_k_dev (optional, layout of pk_fft_estimate) receives
 * delta(n) for a later pk_bispectrum or pk_power_backward. */
pk_status pk_power(const pk_config* cfg, const void* pos_dev, int32_t pos_format, const float* w_dev,
                   int64_t n, double* pk_dev, double* kmean_dev, int64_t* nmodes_dev, void* delta_k_dev,
                   void* ws, size_t ws_bytes, void* stream);

/* a1..a6 end to end from host memory: pk_power for positions pos_host (and optional weights w_host,
 * float[n]) in HOST memory, with P(k), kmean and the mode counts written to host memory (length
 * nbins each). PK_FP32 with FP64 positions: the positions cross the CPU-GPU link in about sixteen
 * pieces, copied by the copy engine on a stream the call creates (and releases) for itself, each
 * piece prepared, binned and added to the grids while the next one is in flight. PK_FIXED64: pinned
 * positions are read by the GPU directly while being prepared and counted, pageable ones copied
 * through the workspace in pieces. Weights, and positions in the FP64 mode or the packed format, are
 * copied to the workspace first. Asynchronous on `stream` like every call: the host
 * outputs are valid once the stream has synchronised. Device or managed pos_host: PK_EINVAL.
 * Workspace: pk_workspace_size(cfg, n, PK_WS_POWER_HOST). */
pk_status pk_power_host(const pk_config* cfg, const void* pos_host, int32_t pos_format, const float* w_host,
                        int64_t n, double* pk_host, double* kmean_host, int64_t* nmodes_host, void* ws,
                        size_t ws_bytes, void* stream);

/* Same as pk_power for a catalogue already in the binned layout of pk_bin (sorted_dev,
 * w_sorted_dev or NULL, tile_offsets_dev): the steady-state hot path when one catalogue is measured
 * more than once or arrives sorted. */
pk_status pk_power_binned(const pk_config* cfg, const pk_cellpos* sorted_dev, const float* w_sorted_dev,
                          const int64_t* tile_offsets_dev, int64_t n, double* pk_dev, double* kmean_dev,
                          int64_t* nmodes_dev, void* delta_k_dev, void* ws, size_t ws_bytes, void* stream);

/* a7 -- Exact triangle counts N_tri (the V_B of eq:VBest as a number of mode triplets) for shells
 * s = 0..nshells-1 covering (shell_lo + s shell_w) <= |n| < (shell_lo + (s+1) shell_w) (units of
 * k_f, n != 0), over the triangles s1 >= s2 >= s3 with s1 <= s2 + s3 + 1, s1 slowest.
 * Requires 3 (kmax - 1) < N, kmax = shell_lo + nshells shell_w (Sec. 4.1: k_max = k_f N/3).
 * counts_dev: int64[ntri], ntri = pk_bispectrum_ntri(nshells). Depends only on N and the shells;
 * callers cache it. Computed by an FP64 convolution of shell indicators, rounded, summed in int64,
 * on the same grid M as pk_bispectrum. */
int32_t pk_bispectrum_ntri(int32_t nshells);
/* a7 -- The triangles of pk_bispectrum_counts and pk_bispectrum in their output order: tri_host (HOST
 * memory, int32[3 ntri], caller-owned) receives (s1, s2, s3) per triangle. Returns ntri, or 0 (and
 * writes nothing) for nshells outside 1..64 or a NULL tri_host. Host work only. */
int32_t pk_bispectrum_triangles(int32_t nshells, int32_t* tri_host);
pk_status pk_bispectrum_counts(const pk_config* cfg, int32_t shell_lo, int32_t shell_w, int32_t nshells,
                               int64_t* counts_dev, void* ws, size_t ws_bytes, void* stream);

/* a7 -- FFT bispectrum (eq:Best2, eq:IntI): for each shell I_s(x) = sum_{n in s} delta(n)
 * exp(+2 pi i n.x/N) (inverse FFT of the shell-filtered delta), then for every triangle
 * B = V^2 sum_x I_1 I_2 I_3 / (N_c N_tri) with FP64 sums (NaN where N_tri = 0). The sums run on
 * the smallest grid M <= N of even side with factors 2, 3, 5, 7 and M > 3 (kmax - 1) (the product
 * of three shell fields then has no alias at n = 0), with N_c = M^3: the same B as on N.
 * The workspace query sizes for M = N, the largest.
 * delta_k_dev: as written by pk_power / pk_fft_estimate with the same cfg; counts_dev from
 * pk_bispectrum_counts; B_dev: double[ntri]. */
pk_status pk_bispectrum(const pk_config* cfg, const void* delta_k_dev, int32_t shell_lo, int32_t shell_w,
                        int32_t nshells, const int64_t* counts_dev, double* B_dev, void* ws, size_t ws_bytes,
                        void* stream);

/* a8 -- Adjoint of pk_power (not in the paper): given dL/dP_b (double[nbins], device) for the
 * same cfg, positions and weights as the forward call, writes dL/dx (float[n][3] for PK_FP32,
 * double[n][3] for PK_FP64 and PK_FIXED64; length units, input particle order). The grid transforms G_1, G_2 are recomputed from the
 * positions (one assignment and FFT, the memory-for-time trade of not saving them); the gradient is
 * back-propagated through the binning, the window division and the interlacing phase to each grid
 * (dL/drho_g[j] = Re sum_n A_g(n) e^{-2 pi i n.j/N}, an inverse real FFT of a Hermitian array), and
 * gathered at every particle with the kernel derivative dW^(p)/du. Orders 2..4 (NGP has no
 * derivative). */
pk_status pk_power_backward(const pk_config* cfg, const void* pos_dev, int32_t pos_format, const float* w_dev,
                            int64_t n, const double* dl_dpk_dev, void* dl_dx_dev, void* ws, size_t ws_bytes,
                            void* stream);

/* a9 -- Batched power spectra of n_cat independent catalogues (PK_FP32 only, unit weights):
 * catalogue c holds particles offsets_host[c] .. offsets_host[c+1]-1 of pos_dev (pk_cellpos, any
 * order within a catalogue, offsets non-decreasing). Outputs pk_dev / nmodes_dev: [n_cat][nbins].
 * Groups of `batch` catalogues (1..512) are binned, assigned, transformed (one batched cuFFT) and
 * estimated together with a fixed number of launches per group and no host synchronisation, so the
 * whole call can be captured in a CUDA graph. ws sized by pk_batch_workspace_size. */
pk_status pk_batch_power(const pk_config* cfg, int32_t n_cat, const int64_t* offsets_host,
                         const pk_cellpos* pos_dev, double* pk_dev, int64_t* nmodes_dev, int32_t batch,
                         void* ws, size_t ws_bytes, void* stream);

/* Direct summation (eq:deltaDS, Sec. 2.2; the alias-free benchmark of Sec. 3.2): for every stored
 * mode of the half-complex layout of pk_fft_estimate (index (i_x, i_y, i_z) <-> signed n, i_z = N/2
 * meaning n_z = -N/2),
 *   delta(n) = (1/sum_i w_i) sum_i w_i exp(-2 pi i n.x_i/L),  delta(0) = 0,
 * with no grid, no window and no aliasing; cfg->order and cfg->interlace are ignored. Unlike a grid
 * transform the sum is not periodic in n: the stored n_i = -N/2 is that vector, not +N/2. Cost
 * N_P x N^2 (N/2+1) complex multiply-adds. Positions in either format (FP64 wrapped into [0, L), or
 * pk_cellpos of the grid cfg->ng), w_dev float[n] or NULL for unit weights; n >= 1.
 * Output delta_k_dev: complex float (PK_FP32) or complex double (PK_FP64, PK_FIXED64), overwritten.
 * Arithmetic: each phase is the exact integer product of n with a fixed-point fraction x/L mod 1
 * (32 bits in PK_FP32, 64 bits otherwise) before its sine and cosine are taken. PK_FP32 runs the sum
 * as a matrix product on the tensor cores (TF32 operands split in two, three products per term,
 * hardware sine/cosine, FP32 sums over runs of 64 particles with compensated totals): error below
 * about 6e-6 of sum |w| / sum w. PK_FP64 / PK_FIXED64 compute in FP64 on the CUDA cores. Partial sums
 * of particle slices are added in FP64 with atomics, so the last bits may differ between runs.
 * Invalid positions set PK_DERR_NONFINITE / PK_DERR_CELLRANGE and count at x = 0 with their weight.
 * Workspace: pk_workspace_size(cfg, n, PK_WS_DIRECT). */
pk_status pk_direct_modes(const pk_config* cfg, const void* pos_dev, int32_t pos_format, const float* w_dev,
                          int64_t n, void* delta_k_dev, void* ws, size_t ws_bytes, void* stream);

/* Binned cross power of two fields on the half-complex layout (Sec. 3.2 compares the grid estimate
 * delta^G with the direct sum through P_{G-DS} ~ <delta^G(k) delta(-k)> and the auto spectra): for
 * each bin of cfg, pk_dev[b] = mean over the modes of V Re[a(n) conj(b(n))], where a stored mode with
 * 0 < i_z < N/2 counts twice (its partner -n, not stored, contributes the conjugate product) and the
 * planes i_z = 0 and i_z = N/2 count once; nmodes_dev[b] the number of modes so counted (equal to
 * the full-grid count of pk_power), kmean_dev[b] their mean |k| (may be NULL). With a = b this is
 * the auto power of a field that is Hermitian in n, such as the direct sum. No shot noise is
 * subtracted; empty bins give NaN. delta_a_dev / delta_b_dev: complex float (PK_FP32) or complex
 * double. Workspace: pk_workspace_size(cfg, 0, PK_WS_CROSS). */
pk_status pk_cross_power(const pk_config* cfg, const void* delta_a_dev, const void* delta_b_dev, double* pk_dev,
                         double* kmean_dev, int64_t* nmodes_dev, void* ws, size_t ws_bytes, void* stream);

/* Multi-grid interlacing (the extension of Sec. 3.1 to more than two grids): P(k) from J = ngrids
 * mass grids, grid j holding the particles shifted by d_j H, each transformed, multiplied by
 * e^{+2 pi i n.d_j/N} and averaged, delta(n) = sum_j e^{+2 pi i n.d_j/N} G_j(n) / (J sum(w) W(n)).
 * Shift sets: J = 1 {0}; J = 2 {0, (1,1,1)/2} (the pk_power interlacing); J = 4 {0, (1,1,0)/2,
 * (1,0,1)/2, (0,1,1)/2}, which keeps only the alias images m whose components share one parity
 * (first left: |m|^2 = 3, against 2 for J = 2); J = 8 {0, 1/2}^3, which keeps only images with every
 * m_i even (first left: |m|^2 = 4). cfg->interlace is ignored; positions, weights, precision modes
 * and outputs as pk_power (delta_k_dev optional, the half-complex layout). Cost: J assignments (J/2
 * interlaced pairs for J = 2, 8) and one batched transform of J grids.
 * Workspace: pk_multigrid_workspace_size(cfg, ngrids, n) bytes (0 for invalid arguments). */
size_t pk_multigrid_workspace_size(const pk_config* cfg, int32_t ngrids, int64_t n);
pk_status pk_power_multigrid(const pk_config* cfg, int32_t ngrids, const void* pos_dev, int32_t pos_format,
                             const float* w_dev, int64_t n, double* pk_dev, double* kmean_dev, int64_t* nmodes_dev,
                             void* delta_k_dev, void* ws, size_t ws_bytes, void* stream);

/* Residual aliasing factor (eq:res, Sec. 3.2): for every mode n of the full N^3 grid,
 *   F_res(n) = sum_{m != 0} theta_m |W(k - m k_s)|^2 / |W(k)|^2,  |W| = sinc^p (p = cfg->order),
 * with theta_m = 1, or [1 + (-1)^{m_x+m_y+m_z}]/2 when cfg->interlace (the images the interlacing
 * cancels). It factorises per axis into the one-dimensional forms of eq:res1Dnoi / eq:res1Di
 * (Hurwitz zeta functions, evaluated in FP64). Per bin of cfg: fres_mean_dev[b] the mean of F_res
 * over the bin's modes, fres_max_dev[b] its largest value (may be NULL), kmean_dev[b] the mean |k|
 * (may be NULL), nmodes_dev[b] the mode count (as pk_power); NaN for empty bins. The window-corrected
 * power of a Poisson catalogue has expectation (1 + F_res(n)) / nbar at every mode (eq:Pknoint with
 * P = 0). Workspace: pk_workspace_size(cfg, 0, PK_WS_ALIASING). */
pk_status pk_aliasing_residual(const pk_config* cfg, double* fres_mean_dev, double* fres_max_dev, double* kmean_dev,
                               int64_t* nmodes_dev, void* ws, size_t ws_bytes, void* stream);

/* No-allocation variant of the fused estimate (a5+a6), for callers that cannot allocate device
 * memory or pass a workspace: code running inside a framework that owns all device memory and
 * forbids allocation while its kernels run (plugins, custom operators of a graph runtime), services
 * with a fixed pre-reserved memory budget, host callbacks that must not enter the allocator. The
 * paper has no counterpart; this is a deployment variant of the same computation as the estimate
 * stage of pk_power.
 * Inputs: g1_dev / g2_dev, the DFTs of the two mass grids (as written by any forward real-to-complex
 * 3-D FFT of the pk_assign grids, unnormalised, sign -i) on the half-complex layout [N][N][N/2+1]
 * (complex float for PK_FP32, complex double otherwise; g2 ignored without interlacing); wsum and
 * w2sum, the sums of the weights and of their squares. Outputs as pk_power (pk_dev, kmean_dev,
 * nmodes_dev, nbins entries each).
 * Scratch: a fixed file-scope device array of about 56 KB in the library (held by every GPU that
 * loads the library until the process exits); N above 1024 or nbins above 1024 is rejected with
 * PK_ESIZE (and N above 1024 fails validation first, PK_EINVAL). A call outside stream capture looks
 * up that array's device address (with the device current), which also follows a device reset; a
 * call under capture uses the address of the device's last call outside capture, so make one call
 * on each device before capturing (a capture that starts with the device's first call returns
 * PK_EINVAL). All calls share the array: calls that overlap on the GPU (other streams, other host
 * threads) race and give wrong results; serialise them. Nothing is allocated. */
pk_status pk_estimate_noalloc(const pk_config* cfg, const void* g1_dev, const void* g2_dev, double wsum, double w2sum,
                              double* pk_dev, double* kmean_dev, int64_t* nmodes_dev, void* stream);

/* Stage timing for profiling (not part of the method). pk_profile_enable(1) makes the following
 * pk_power / pk_power_binned / pk_power_backward calls on this host thread record CUDA events on
 * their stream at the stage boundaries; pk_profile_read waits for the last recorded event and writes
 * up to max_stages durations in milliseconds of the most recent call: [0] position preparation and
 * binning (weight sums only for pk_power_binned), [1] clearing the grids, [2] the mass-assignment
 * kernel, [3] FFT, [4] estimate and finalisation (-1 for a stage that was not recorded). Returns the previous enable state / the number
 * of values written. */
int32_t pk_profile_enable(int32_t on);
int32_t pk_profile_read(double* ms_host, int32_t max_stages);

/* Number of kernels this library has launched in the process so far (cuFFT's own kernels excluded). */
int64_t pk_profile_launches(void);

/* Message describing the last failure of a pk_* call on this host thread ("" if none). */
const char* pk_last_error(void);

/* Reads and clears the device error word (PK_DERR_* bits) after synchronising `stream`.
 * Returns -1 if the read itself failed. */
int32_t pk_device_error(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PK_H */
