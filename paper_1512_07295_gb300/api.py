"""PyTorch-facing wrappers of the C ABI (include/pk.h). Tensors supply device memory and the current
CUDA stream; every step of the computation runs in libpk's kernels (and cuFFT for the transforms).

Positions: an (n, 3) float64 CUDA tensor (length units), or an (n, 4) int32 CUDA tensor holding
pk_cellpos records (packed cell, then the three FP32 offsets as raw bits) as produced by ``prepare``.
"""

import ctypes
from dataclasses import dataclass

import torch

from . import ffi
from .ffi import check

_PREC = {"fp64": ffi.PK_FP64, "fp32": ffi.PK_FP32, "fixed64": ffi.PK_FIXED64}


@dataclass
class Config:
    """Mirror of pk_config. Bins default to b k_f, b = 1..ng/2 (edges in units of k_f/2)."""

    ng: int
    box: float
    order: int = 4
    interlace: bool = True
    prec: str = "fp32"
    bin_lo2: int = 1
    bin_w2: int = 2
    nbins: int = 0
    subtract_shot: bool = False
    tile_run: int = 0

    def c(self):
        nb = self.nbins if self.nbins > 0 else self.ng // 2
        return ffi.PkConfig(int(self.ng), int(self.order), int(bool(self.interlace)), _PREC[self.prec], float(self.box),
                            int(self.bin_lo2), int(self.bin_w2), int(nb), int(bool(self.subtract_shot)), int(self.tile_run))

    @property
    def nb(self):
        return self.nbins if self.nbins > 0 else self.ng // 2

    @property
    def real_dtype(self):
        return torch.float32 if self.prec == "fp32" else torch.float64


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _pos_format(pos, on_device=True):
    if pos.is_cuda != on_device or not pos.is_contiguous():
        raise ValueError(f"positions must be a contiguous {'CUDA' if on_device else 'CPU'} tensor")
    if pos.dtype == torch.float64 and pos.dim() == 2 and pos.shape[1] == 3:
        return ffi.PK_POS_F64_XYZ
    if pos.dtype == torch.int32 and pos.dim() == 2 and pos.shape[1] == 4:
        return ffi.PK_POS_CELL_F32OFF
    raise ValueError("positions: (n,3) float64 or (n,4) int32 pk_cellpos records")


def _weights(w, n, device):
    if w is None:
        return None
    if w.dtype != torch.float32 or w.device != device or not w.is_contiguous() or w.numel() != n:
        raise ValueError("weights: contiguous float32 tensor of n entries on the positions' device")
    return w


def workspace(cfg, n, kind, device):
    size = ffi.lib().pk_workspace_size(ctypes.byref(cfg.c()), int(n), int(kind))
    if size == 0:
        raise ffi.PkError(ffi.PK_EINVAL, ffi.last_error())
    return torch.empty(size, dtype=torch.uint8, device=device)


def half_shape(ng):
    return (ng, ng, ng // 2 + 1)


def prepare(pos, cfg):
    """FP64 positions -> (n, 4) int32 pk_cellpos records (a1)."""
    if _pos_format(pos) != ffi.PK_POS_F64_XYZ:
        raise ValueError("prepare takes (n,3) float64 positions")
    out = torch.empty((pos.shape[0], 4), dtype=torch.int32, device=pos.device)
    check(ffi.lib().pk_prepare(ctypes.byref(cfg.c()), _p(pos), pos.shape[0], _p(out), _stream(pos.device)))
    return out


def cellpos_split(cells):
    """(packed cell int32, offsets float32 (n,3)) views of pk_cellpos records."""
    return cells[:, 0], cells[:, 1:].view(torch.float32)


def bin_particles(pos, cfg, weights=None):
    """Counting sort by tile (a2): returns (sorted (n,4) int32, sorted weights or None, tile offsets int64)."""
    fmt = _pos_format(pos)
    n = pos.shape[0]
    w = _weights(weights, n, pos.device)
    ntile = ffi.lib().pk_tiles_per_axis(ctypes.byref(cfg.c()), None)
    sorted_ = torch.empty((n, 4), dtype=torch.int32, device=pos.device)
    wsorted = torch.empty(n, dtype=torch.float32, device=pos.device) if w is not None else None
    offsets = torch.empty(ntile ** 3 + 1, dtype=torch.int64, device=pos.device)
    ws = workspace(cfg, n, ffi.PK_WS_BIN, pos.device)
    check(ffi.lib().pk_bin(ctypes.byref(cfg.c()), _p(pos), fmt, _p(w), n, _p(sorted_), _p(wsorted), _p(offsets), _p(ws),
                           ws.numel(), _stream(pos.device)))
    return sorted_, wsorted, offsets


def assign(pos, cfg, weights=None):
    """Mass grids (a3): (grid1, grid2 or None), each (ng, ng, ng) of the precision's real type."""
    fmt = _pos_format(pos)
    n = pos.shape[0]
    w = _weights(weights, n, pos.device)
    dt = cfg.real_dtype
    g1 = torch.empty((cfg.ng,) * 3, dtype=dt, device=pos.device)
    g2 = torch.empty((cfg.ng,) * 3, dtype=dt, device=pos.device) if cfg.interlace else None
    ws = workspace(cfg, n, ffi.PK_WS_ASSIGN, pos.device)
    check(ffi.lib().pk_assign(ctypes.byref(cfg.c()), _p(pos), fmt, _p(w), n, _p(g1), _p(g2), _p(ws), ws.numel(),
                              _stream(pos.device)))
    return g1, g2


def fft_estimate(grid1, grid2, cfg, wsum):
    """delta(n) on the half-complex layout (ng, ng, ng/2+1) from mass grids (a4+a5)."""
    ctype = torch.complex64 if cfg.prec == "fp32" else torch.complex128
    delta = torch.empty(half_shape(cfg.ng), dtype=ctype, device=grid1.device)
    ws = workspace(cfg, 0, ffi.PK_WS_FFT_ESTIMATE, grid1.device)
    check(ffi.lib().pk_fft_estimate(ctypes.byref(cfg.c()), _p(grid1), _p(grid2), float(wsum), _p(delta), _p(ws), ws.numel(),
                                    _stream(grid1.device)))
    return delta


def _outputs(cfg, device):
    nb = cfg.nb
    return (torch.empty(nb, dtype=torch.float64, device=device), torch.empty(nb, dtype=torch.float64, device=device),
            torch.empty(nb, dtype=torch.int64, device=device))


def power(pos, cfg, weights=None, return_delta=False, ws=None):
    """P(k) of a catalogue in any order (a1..a6): (pk, kmean, nmodes[, delta])."""
    fmt = _pos_format(pos)
    n = pos.shape[0]
    w = _weights(weights, n, pos.device)
    pk, km, nm = _outputs(cfg, pos.device)
    delta = None
    if return_delta:
        ctype = torch.complex64 if cfg.prec == "fp32" else torch.complex128
        delta = torch.empty(half_shape(cfg.ng), dtype=ctype, device=pos.device)
    if ws is None:
        ws = workspace(cfg, n, ffi.PK_WS_POWER, pos.device)
    check(ffi.lib().pk_power(ctypes.byref(cfg.c()), _p(pos), fmt, _p(w), n, _p(pk), _p(km), _p(nm), _p(delta), _p(ws),
                             ws.numel(), _stream(pos.device)))
    return (pk, km, nm, delta) if return_delta else (pk, km, nm)


def power_host(pos, cfg, weights=None, ws=None, out=None, device=None):
    """P(k) end to end from host memory (pk_power_host): pos is an (n, 3) float64 or packed (n, 4)
    int32 CPU tensor (pinned tensors are read by the GPU directly), weights an optional float32 CPU
    tensor; returns CPU tensors (pk, kmean, nmodes), valid after the stream has synchronised
    (``out`` may hold pinned tensors to fill). The workspace lives on ``device``."""
    fmt = _pos_format(pos, on_device=False)
    device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    n = pos.shape[0]
    if weights is not None:
        weights = weights.to(torch.float32).contiguous()
        if weights.is_cuda or weights.shape[0] != n:
            raise ValueError("weights must be a CPU tensor of length n")
    if ws is None:
        ws = workspace(cfg, n, ffi.PK_WS_POWER_HOST, device)
    if out is None:
        out = (torch.empty(cfg.nb, dtype=torch.float64), torch.empty(cfg.nb, dtype=torch.float64),
               torch.empty(cfg.nb, dtype=torch.int64))
    pk, km, cnt = out
    check(ffi.lib().pk_power_host(ctypes.byref(cfg.c()), _p(pos), fmt, _p(weights), n, _p(pk), _p(km), _p(cnt), _p(ws),
                                  ws.numel(), _stream(device)))
    return pk, km, cnt


def power_binned(binned, cfg, return_delta=False, ws=None, out=None):
    """P(k) from the binned layout of ``bin_particles``: (pk, kmean, nmodes[, delta])."""
    sorted_, wsorted, offsets = binned
    n = sorted_.shape[0]
    pk, km, nm = out if out is not None else _outputs(cfg, sorted_.device)
    delta = None
    if return_delta:
        ctype = torch.complex64 if cfg.prec == "fp32" else torch.complex128
        delta = torch.empty(half_shape(cfg.ng), dtype=ctype, device=sorted_.device)
    if ws is None:
        ws = workspace(cfg, n, ffi.PK_WS_POWER_BINNED, sorted_.device)
    check(ffi.lib().pk_power_binned(ctypes.byref(cfg.c()), _p(sorted_), _p(wsorted), _p(offsets), n, _p(pk), _p(km), _p(nm),
                                    _p(delta), _p(ws), ws.numel(), _stream(sorted_.device)))
    return (pk, km, nm, delta) if return_delta else (pk, km, nm)


def direct_modes(pos, cfg, weights=None, ws=None):
    """delta(n) by direct summation (eq:deltaDS) on the half-complex layout (ng, ng, ng/2+1), no window
    and no aliasing; cfg.order and cfg.interlace are ignored."""
    fmt = _pos_format(pos)
    n = pos.shape[0]
    w = _weights(weights, n, pos.device)
    ctype = torch.complex64 if cfg.prec == "fp32" else torch.complex128
    delta = torch.empty(half_shape(cfg.ng), dtype=ctype, device=pos.device)
    if ws is None:
        ws = workspace(cfg, n, ffi.PK_WS_DIRECT, pos.device)
    check(ffi.lib().pk_direct_modes(ctypes.byref(cfg.c()), _p(pos), fmt, _p(w), n, _p(delta), _p(ws), ws.numel(),
                                    _stream(pos.device)))
    return delta


def cross_power(delta_a, delta_b, cfg, ws=None):
    """Binned V Re[delta_a conj(delta_b)] of two half-complex fields (pk_cross_power): (pk, kmean, nmodes)."""
    ctype = torch.complex64 if cfg.prec == "fp32" else torch.complex128
    for d in (delta_a, delta_b):
        if d.dtype != ctype or tuple(d.shape) != half_shape(cfg.ng) or not d.is_contiguous() or not d.is_cuda:
            raise ValueError(f"fields: contiguous {ctype} CUDA tensors of shape {half_shape(cfg.ng)}")
    pk, km, nm = _outputs(cfg, delta_a.device)
    if ws is None:
        ws = workspace(cfg, 0, ffi.PK_WS_CROSS, delta_a.device)
    check(ffi.lib().pk_cross_power(ctypes.byref(cfg.c()), _p(delta_a), _p(delta_b), _p(pk), _p(km), _p(nm), _p(ws),
                                   ws.numel(), _stream(delta_a.device)))
    return pk, km, nm


def power_multigrid(pos, cfg, ngrids, weights=None, return_delta=False, ws=None):
    """P(k) with multi-grid interlacing over ngrids = 1, 2, 4 or 8 half-cell-shifted grids
    (pk_power_multigrid): (pk, kmean, nmodes[, delta])."""
    fmt = _pos_format(pos)
    n = pos.shape[0]
    w = _weights(weights, n, pos.device)
    pk, km, nm = _outputs(cfg, pos.device)
    delta = None
    if return_delta:
        ctype = torch.complex64 if cfg.prec == "fp32" else torch.complex128
        delta = torch.empty(half_shape(cfg.ng), dtype=ctype, device=pos.device)
    if ws is None:
        size = ffi.lib().pk_multigrid_workspace_size(ctypes.byref(cfg.c()), int(ngrids), int(n))
        if size == 0:
            raise ffi.PkError(ffi.PK_EINVAL, ffi.last_error())
        ws = torch.empty(size, dtype=torch.uint8, device=pos.device)
    check(ffi.lib().pk_power_multigrid(ctypes.byref(cfg.c()), int(ngrids), _p(pos), fmt, _p(w), n, _p(pk), _p(km), _p(nm),
                                       _p(delta), _p(ws), ws.numel(), _stream(pos.device)))
    return (pk, km, nm, delta) if return_delta else (pk, km, nm)


def aliasing_residual(cfg, device="cuda"):
    """Per-bin mean and maximum of the residual aliasing factor F_res (eq:res) for cfg's order and
    interlacing, with the mean |k| and mode counts (pk_aliasing_residual): (mean, max, kmean, nmodes)."""
    nb = cfg.nb
    mean, mx, km = (torch.empty(nb, dtype=torch.float64, device=device) for _ in range(3))
    nm = torch.empty(nb, dtype=torch.int64, device=device)
    ws = workspace(cfg, 0, ffi.PK_WS_ALIASING, device)
    check(ffi.lib().pk_aliasing_residual(ctypes.byref(cfg.c()), _p(mean), _p(mx), _p(km), _p(nm), _p(ws), ws.numel(),
                                         _stream(torch.device(device))))
    return mean, mx, km, nm


def bispectrum_ntri(nshells):
    return int(ffi.lib().pk_bispectrum_ntri(int(nshells)))


def triangles(nshells):
    """Shell triples (s1, s2, s3) of pk_bispectrum's outputs, in order (pk_bispectrum_triangles)."""
    import numpy as np

    tri = np.zeros(3 * max(bispectrum_ntri(nshells), 1), dtype=np.int32)
    m = int(ffi.lib().pk_bispectrum_triangles(int(nshells), tri.ctypes.data_as(ctypes.c_void_p)))
    return [tuple(int(v) for v in tri[3 * i:3 * i + 3]) for i in range(m)]


def bispectrum_counts(cfg, shell_lo, shell_w, nshells, device="cuda"):
    """Exact N_tri per triangle (int64, device)."""
    counts = torch.empty(bispectrum_ntri(nshells), dtype=torch.int64, device=device)
    ws = workspace(cfg, nshells, ffi.PK_WS_BISPECTRUM_COUNTS, device)
    check(ffi.lib().pk_bispectrum_counts(ctypes.byref(cfg.c()), int(shell_lo), int(shell_w), int(nshells), _p(counts), _p(ws),
                                         ws.numel(), _stream(torch.device(device))))
    return counts


def bispectrum(delta, cfg, shell_lo, shell_w, nshells, counts=None):
    """FFT bispectrum per triangle (float64, device); counts from ``bispectrum_counts``."""
    if counts is None:
        counts = bispectrum_counts(cfg, shell_lo, shell_w, nshells, delta.device)
    out = torch.empty(bispectrum_ntri(nshells), dtype=torch.float64, device=delta.device)
    ws = workspace(cfg, nshells, ffi.PK_WS_BISPECTRUM, delta.device)
    check(ffi.lib().pk_bispectrum(ctypes.byref(cfg.c()), _p(delta), int(shell_lo), int(shell_w), int(nshells), _p(counts),
                                  _p(out), _p(ws), ws.numel(), _stream(delta.device)))
    return out, counts


def power_backward(pos, cfg, dl_dpk, weights=None):
    """dL/dx for dL/dP_b (a8): (n, 3) float32 (fp32) or float64 (fp64, fixed64)."""
    fmt = _pos_format(pos)
    n = pos.shape[0]
    w = _weights(weights, n, pos.device)
    dl = dl_dpk.to(device=pos.device, dtype=torch.float64).contiguous()
    out = torch.empty((n, 3), dtype=torch.float32 if cfg.prec == "fp32" else torch.float64, device=pos.device)
    ws = workspace(cfg, n, ffi.PK_WS_BACKWARD, pos.device)
    check(ffi.lib().pk_power_backward(ctypes.byref(cfg.c()), _p(pos), fmt, _p(w), n, _p(dl), _p(out), _p(ws), ws.numel(),
                                      _stream(pos.device)))
    return out


def batch_workspace(cfg, batch, max_group_particles, device):
    size = ffi.lib().pk_batch_workspace_size(ctypes.byref(cfg.c()), int(batch), int(max_group_particles))
    if size == 0:
        raise ffi.PkError(ffi.PK_EINVAL, ffi.last_error())
    return torch.empty(size, dtype=torch.uint8, device=device)


def max_group_particles(offsets, batch):
    offs = [int(v) for v in offsets]
    return max(offs[min(g + batch, len(offs) - 1)] - offs[g] for g in range(0, len(offs) - 1, batch))


def batch_power(cells, offsets, cfg, batch=64, ws=None, out=None):
    """P(k) of many catalogues (a9). cells: (n,4) int32 pk_cellpos; offsets: host int64 sequence of
    n_cat + 1 catalogue boundaries. Returns (pk, nmodes) of shape (n_cat, nbins)."""
    if _pos_format(cells) != ffi.PK_POS_CELL_F32OFF:
        raise ValueError("batch_power takes pk_cellpos records")
    import numpy as np

    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    ncat = len(offs) - 1
    if out is None:
        pk = torch.empty((ncat, cfg.nb), dtype=torch.float64, device=cells.device)
        nm = torch.empty((ncat, cfg.nb), dtype=torch.int64, device=cells.device)
    else:
        pk, nm = out
    if ws is None:
        ws = batch_workspace(cfg, batch, max_group_particles(offs, batch), cells.device)
    check(ffi.lib().pk_batch_power(ctypes.byref(cfg.c()), ncat, offs.ctypes.data_as(ctypes.c_void_p), _p(cells), _p(pk), _p(nm),
                                   int(batch), _p(ws), ws.numel(), _stream(cells.device)))
    return pk, nm


def autotune_batch(cells, offsets, cfg, candidates=(32, 64, 128, 256, 512), reps=3, runs=None):
    """Chooses the group size of batch_power for these catalogues by timing each candidate (CUDA
    events, after one warm-up call each). Returns (best, {candidate: ms}). The group size sets how
    many catalogues share each batched launch: larger groups fill the GPU with fewer launches but
    need a larger workspace. runs: also try these scatter run lengths (tiles per region along z,
    cfg.tile_run); the best run length is then written to cfg.tile_run and the keys are
    "group/run"."""
    if runs:
        best, table = None, {}
        base = cfg.tile_run
        for r in runs:
            cfg.tile_run = int(r)
            b, t = autotune_batch(cells, offsets, cfg, candidates, reps)
            for k, v in t.items():
                table[f"{k}/{r}"] = v
            if best is None or t[b] < table[f"{best[0]}/{best[1]}"]:
                best = (b, int(r))
        cfg.tile_run = best[1] if best else base
        return best[0], table
    import numpy as np

    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    ncat = len(offs) - 1
    pk = torch.empty((ncat, cfg.nb), dtype=torch.float64, device=cells.device)
    nm = torch.empty((ncat, cfg.nb), dtype=torch.int64, device=cells.device)
    times = {}
    for b in candidates:
        b = int(min(max(b, 1), 512))
        ws = batch_workspace(cfg, b, max_group_particles(offs, b), cells.device)
        batch_power(cells, offs, cfg, batch=b, ws=ws, out=(pk, nm))
        torch.cuda.synchronize()  # the warm-up call (plans, attributes) ends before the timed calls start
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            batch_power(cells, offs, cfg, batch=b, ws=ws, out=(pk, nm))
        e1.record()
        torch.cuda.synchronize()
        times[b] = e0.elapsed_time(e1) / reps
        del ws
    best = min(times, key=times.get)
    return best, times


def estimate_noalloc(g1_hat, g2_hat, cfg, wsum, w2sum):
    """P(k) from the transforms of the two mass grids without any device allocation by the library
    (pk_estimate_noalloc). g*_hat: (ng, ng, ng/2+1) complex tensors. Returns (pk, kmean, nmodes)."""
    pk, km, nm = _outputs(cfg, g1_hat.device)
    check(ffi.lib().pk_estimate_noalloc(ctypes.byref(cfg.c()), _p(g1_hat), _p(g2_hat), float(wsum), float(w2sum), _p(pk),
                                        _p(km), _p(nm), _stream(g1_hat.device)))
    return pk, km, nm


def device_error(device=None):
    """Reads and clears the device error word (PK_DERR_* bits) after synchronising the stream."""
    return int(ffi.lib().pk_device_error(_stream(device)))


class PowerSpectrum(torch.autograd.Function):
    """P(k) (pk_power) with the hand-written adjoint (pk_power_backward) as its backward."""

    @staticmethod
    def forward(ctx, pos, cfg, weights=None):
        pk, _, _ = power(pos, cfg, weights)
        ctx.save_for_backward(pos, weights if weights is not None else torch.empty(0, device=pos.device))
        ctx.cfg = cfg
        ctx.has_w = weights is not None
        return pk

    @staticmethod
    def backward(ctx, grad_pk):
        pos, w = ctx.saved_tensors
        g = power_backward(pos, ctx.cfg, torch.nan_to_num(grad_pk, nan=0.0), w if ctx.has_w else None)
        return g.to(pos.dtype), None, None


def power_spectrum(pos, cfg, weights=None):
    """Differentiable P(k) of FP64 positions."""
    return PowerSpectrum.apply(pos, cfg, weights)
