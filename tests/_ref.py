"""Oracle-side helpers shared by the GPU parity tests (they call only ``oracle``)."""

import numpy as np

import oracle


def grids(pos, box, ng, p, weights=None, interlace=True):
    u = oracle.assign.grid_units(pos, box, ng)
    r1 = oracle.assign.assign_units(u, ng, p, weights)
    r2 = oracle.assign.assign_units(u, ng, p, weights, shift=True) if interlace else None
    return r1, r2


def power(pos, box, ng, p, interlace=True, weights=None, edges=None, subtract=False):
    r1, r2 = grids(pos, box, ng, p, weights, interlace)
    delta = oracle.fourier.density_modes(r1, p, r2)
    shot = oracle.power.shot_noise(box, weights, len(pos)) if subtract else 0.0
    pk, keff, cnt = oracle.power.power_spectrum(delta, box, edges, subtract=shot)
    return pk, keff, cnt, delta


def half_complex(full):
    """The stored half (i_z <= N/2) of a full-grid array, matching the library's delta layout."""
    ng = full.shape[0]
    return full[:, :, : ng // 2 + 1]


def cellpos_to_units(cells_np, ng):
    """Grid-unit positions (FP64) of pk_cellpos records (int32 (n,4)): u = c + f exactly."""
    c = cells_np[:, 0].astype(np.uint32)
    f = cells_np[:, 1:].copy().view(np.float32).astype(np.float64)
    cx = ((c >> 20) & 1023).astype(np.float64)
    cy = ((c >> 10) & 1023).astype(np.float64)
    cz = (c & 1023).astype(np.float64)
    return np.stack([cx + f[:, 0], cy + f[:, 1], cz + f[:, 2]], axis=1)


def power_units(u, box, ng, p, interlace=True):
    r1 = oracle.assign.assign_units(u, ng, p)
    r2 = oracle.assign.assign_units(u, ng, p, shift=True) if interlace else None
    delta = oracle.fourier.density_modes(r1, p, r2)
    return oracle.power.power_spectrum(delta, box)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def pack_cellpos(u, ng):
    """pk_cellpos records (int32 (n,4)) of grid-unit positions u (FP64), made on the host: cell index
    floor(u) mod N on each axis, FP32 offset u - floor(u) (an offset that rounds up to 1 moves to the
    next cell with offset 0). cellpos_to_units gives back the exact positions of the records."""
    u = np.mod(np.asarray(u, dtype=np.float64), ng)
    c = np.floor(u).astype(np.int64)
    f = (u - c).astype(np.float32)
    up = f >= np.float32(1.0)
    c = np.where(up, c + 1, c) % ng
    f = np.where(up, np.float32(0.0), f).astype(np.float32)
    out = np.empty((len(u), 4), dtype=np.int32)
    out[:, 0] = ((c[:, 0] << 20) | (c[:, 1] << 10) | c[:, 2]).astype(np.uint32).view(np.int32)
    out[:, 1:] = f.view(np.int32)
    return out
