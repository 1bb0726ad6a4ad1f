#!/usr/bin/env python
"""Throughput of the PCS + interlacing power-spectrum path on one GB300 (or N independent replicas).

Workload (one step): P(k) of a 1024^3-particle Zel'dovich-displaced catalogue in a periodic box of
L = 2000 Mpc/h on an N_G = 512 grid, PCS assignment with interlacing, FP32 cell + offset positions
(binned by tile, resident in HBM), FP32 grids and FFT, FP64 shell sums: assignment of both grids,
two real FFTs, the fused deconvolution / interlacing / shell reduction and the finalisation.

Printed: one JSON line (rank 0). ``value`` = particles/s (P(k)/s in ``pk_per_s``); ``e2e`` = the same
metric through pk_power_host from pinned host FP64 positions (the GPU reads them over the CPU-GPU link
while preparing them; binning, assignment, FFT, estimate and the D2H of the results inside the timed
region); ``roofline`` for the assignment kernel;
``cpu_baseline`` = the FP64 CPU oracle on a bounded sample; ``fp64_plain`` = the plain FP64 GPU path
(global FP64 atomics, FP64 FFT) on the same catalogue.

``--impl reference`` times the FP64 CPU oracle (the reference arm) on a bounded
sample of the same workload and prints the same metric.
"""

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particles/s & P(k)/s (PCS+interlace, N_g=512), % HBM roofline vs plain FP64 path"

# DRAM bytes (read + write) per particle of one k_assign_cells<4,false> launch, from an ncu capture of
# the 256^3-particle / N_G = 128 case (8 particles per cell, as in the 1024^3 / N_G = 512 workload, so
# the per-particle traffic carries over). None when the kernel has changed since the capture.
ASSIGN_TRAFFIC_PER_PARTICLE = 299.68e6 / 256 ** 3
ASSIGN_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on 256^3 particles / N_G=128 "
                         "(profiles/k_assign_cells_pcs_interlace_256cube_ng128.md), scaled by the particle count")
RMS_DISP = 4.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nside", type=int, default=1024)
    ap.add_argument("--ng", type=int, default=512)
    ap.add_argument("--box", type=float, default=2000.0)
    ap.add_argument("--quick", action="store_true", help="small catalogue (128^3, N_G=128) for smoke runs")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, fp64 baseline and cpu baseline")
    ap.add_argument("--only-row", choices=["adjoint", "batch", "bispectrum", "direct", "multigrid", "e2e", "ng1024", "c1"],
                    default=None,
                    help="time one secondary row on its own workload and print it (no P(k) step)")
    ap.add_argument("--ds-nside", type=int, default=128, help="--only-row direct: particles per side")
    ap.add_argument("--ds-ng", type=int, default=128, help="--only-row direct: grid size")
    ap.add_argument("--batch-cats", type=int, default=512, help="--only-row batch: catalogues in the batch")
    ap.add_argument("--row-ng", type=int, default=1024, help="--only-row ng1024: grid size (1024 for the row itself)")
    ap.add_argument("--no-oracle", action="store_true", help="skip the measured CPU oracle rows (c1 and c2 configurations)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return ap.parse_args()


def replica_seed(rank):
    """Seed of the catalogue a rank generates: every replica times its own independent realisation."""
    return 3 + rank


def max_over_ranks(ms, device):
    """The job's time: the largest per-rank time over all ranks (identity on a single process)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, steps, ms_total):
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world * units_per_rank * steps / (ms_total * 1e-3)


def workload_name(a):
    return (f"ZA clustered catalogue {a.nside}^3 particles, L={a.box:g} Mpc/h, N_G={a.ng}, PCS+interlacing P(k), "
            f"FP32 cell+offset positions binned by tile")


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def oracle_sample_rate(pos_sample, n_full, box, ng, with_fft=True):
    """Times the FP64 oracle: assignment of a particle sample (both grids) and, once, the FFT,
    deconvolution, interlacing and binning at N_G; returns (particles/s of the full workload, detail)."""
    import oracle

    t0 = time.perf_counter()
    u = oracle.assign.grid_units(pos_sample, box, ng)
    r1 = oracle.assign.assign_units(u, ng, 4)
    r2 = oracle.assign.assign_units(u, ng, 4, shift=True)
    t_assign = time.perf_counter() - t0
    t_fft = 0.0
    if with_fft:
        t0 = time.perf_counter()
        delta = oracle.fourier.density_modes(r1, 4, r2)
        oracle.power.power_spectrum(delta, box)
        t_fft = time.perf_counter() - t0
        del delta
    t_full = t_assign * (n_full / len(pos_sample)) + t_fft
    return n_full / t_full, {"t_assign_s": t_assign, "t_fft_estimate_s": t_fft, "sample_particles": len(pos_sample),
                             "t_full_extrapolated_s": t_full}


def _oracle_assign_chunk(args):
    """One worker's share of the oracle's assignment (both grids): u in grid units."""
    import oracle

    u, ng, p = args
    return oracle.assign.assign_units(u, ng, p), oracle.assign.assign_units(u, ng, p, shift=True)


def oracle_power_parallel(pos, box, ng, p, workers):
    """The FP64 oracle's P(k) (PCS + interlacing at p = 4) with its assignment split over worker
    processes by particle chunk (the oracle's own function on each chunk, the chunk grids summed); the
    FFT, deconvolution and binning run in this process (scipy.fft with every core). Returns
    (pk, t_assign_s, t_rest_s)."""
    import concurrent.futures
    import multiprocessing

    import oracle

    t0 = time.perf_counter()
    u = oracle.assign.grid_units(pos, box, ng)
    chunks = np.array_split(u, workers)
    with concurrent.futures.ProcessPoolExecutor(workers, mp_context=multiprocessing.get_context("spawn")) as ex:
        r1 = r2 = None
        for a, b in ex.map(_oracle_assign_chunk, [(c, ng, p) for c in chunks]):
            r1 = a if r1 is None else r1 + a
            r2 = b if r2 is None else r2 + b
    t_assign = time.perf_counter() - t0
    t0 = time.perf_counter()
    pk, _, _ = oracle.power.power_spectrum(oracle.fourier.density_modes(r1, p, r2), box)
    return pk, t_assign, time.perf_counter() - t0


def measured_oracle_rows(steps=3):
    """The FP64 CPU oracle timed end to end (assignment of both grids, FFT, deconvolution, interlacing,
    binning) on the two smaller benchmark configurations, median of `steps` runs, assignment over a
    process pool of every host core: c1, 64^3 Poisson particles in L = 1000 Mpc/h on N_G = 64; c2,
    256^3 Zel'dovich particles in L = 1500 Mpc/h on N_G = 256 (PCS + interlacing both)."""
    from paper_1512_07295_gb300 import catalogs

    cores = len(os.sched_getaffinity(0))
    out = {"cores": cores, "kind": "oracle", "runs": steps}
    cases = {"c1_poisson_64cube_ng64": (catalogs.poisson(64 ** 3, 1000.0, seed=1), 1000.0, 64),
             "c2_zeldovich_256cube_ng256": (catalogs.zeldovich(256, 1500.0, rms=RMS_DISP, seed=2), 1500.0, 256)}
    for name, (pos, box, ng) in cases.items():
        walls, parts = [], []
        for _ in range(steps):
            t0 = time.perf_counter()
            _, ta, tr = oracle_power_parallel(pos, box, ng, 4, cores)
            walls.append(time.perf_counter() - t0)
            parts.append((ta, tr))
        i = int(np.argsort(walls)[len(walls) // 2])
        out[name] = {"particles": int(len(pos)), "s_per_pk_median": float(walls[i]),
                     "particles_per_s": float(len(pos) / walls[i]), "t_assign_s": float(parts[i][0]),
                     "t_fft_estimate_s": float(parts[i][1]), "all_s": [float(x) for x in walls]}
    return out


def _rel_per_bin(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.abs(a / b - 1.0)


def _sig(x, digits=3):
    return [float(f"{v:.{digits}g}") for v in np.asarray(x, dtype=np.float64)]


def row_accuracy_c2(dev):
    """FP32 against FP64, per k-bin, on the 256^3 Zel'dovich catalogue (L = 1500 Mpc/h, N_G = 256):
    CIC, TSC, PCS, each with and without interlacing. FP64: pk_power from the FP64 positions (the
    oracle-parity mode); FP32: pk_power on the same positions, which splits them into cell + FP32
    offset records (a1) and runs the FP32 grids and transforms with FP64 shell sums. The difference is
    the whole FP32 path's error: positions, assignment, FFT and estimate."""
    import torch

    from paper_1512_07295_gb300 import api, catalogs

    pos = catalogs.zeldovich_torch(256, 1500.0, RMS_DISP, seed=2, device=dev)
    out = {"workload": "256^3 ZA particles, L=1500 Mpc/h, N_G=256: FP32 (cell + FP32 offset) vs FP64 positions and "
                       "grids, |P32/P64 - 1| per k-bin", "cases": {}}
    for p, name in ((2, "CIC"), (3, "TSC"), (4, "PCS")):
        for inter in (False, True):
            c64 = api.Config(ng=256, box=1500.0, order=p, interlace=inter, prec="fp64")
            c32 = api.Config(ng=256, box=1500.0, order=p, interlace=inter, prec="fp32")
            pk64, _, n64 = api.power(pos, c64)
            ws = api.workspace(c32, pos.shape[0], api.ffi.PK_WS_POWER, dev)
            pk32, _, n32 = api.power(pos, c32, ws=ws)
            ms = _time_cuda(lambda: api.power(pos, c32, ws=ws), 3)
            rel = _rel_per_bin(pk32, pk64)
            out["cases"][f"{name}{'+interlace' if inter else ''}"] = {
                "max_rel": float(rel.max()), "median_rel": float(np.median(rel)),
                "counts_equal": bool(torch.equal(n32, n64)), "fp32_ms_per_pk": ms, "per_bin": _sig(rel, 2)}
            del ws
    del pos
    torch.cuda.empty_cache()
    return out


def numa_report(host_tensor, dev_index):
    """Where a pinned host buffer's pages live and which NUMA node the GPU hangs off (Linux sysfs and
    /proc/self/numa_maps), to explain the CPU-GPU link rate of the end-to-end call."""
    rep = {}
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(dev_index), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip().lower()
        dom, rest = out.split(":", 1)
        sysfs = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}/numa_node"
        rep["gpu_pci"] = out
        rep["gpu_numa_node"] = int(open(sysfs).read().strip()) if os.path.exists(sysfs) else None
    except Exception as e:  # pragma: no cover - depends on the host
        rep["gpu_numa_node_error"] = type(e).__name__
    try:
        addr = host_tensor.data_ptr()
        end = addr + host_tensor.numel() * host_tensor.element_size()
        pages = {}
        for line in open("/proc/self/numa_maps"):
            parts = line.split()
            start = int(parts[0], 16)
            if addr <= start < end or start <= addr < start + (1 << 32):
                for f in parts[1:]:
                    if f.startswith("N") and "=" in f:
                        k, v = f.split("=")
                        pages[k] = pages.get(k, 0) + int(v)
        rep["buffer_pages_per_node"] = pages
    except Exception as e:  # pragma: no cover
        rep["numa_maps_error"] = type(e).__name__
    try:
        rep["cpus"] = len(os.sched_getaffinity(0))
        rep["host_nodes"] = sorted(int(d[4:]) for d in os.listdir("/sys/devices/system/node")
                                   if d.startswith("node") and d[4:].isdigit())
    except Exception:  # pragma: no cover
        pass
    return rep


def _time_cuda(fn, reps, warm=1):
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def alu_peak(dev):
    """Derived FP32 FMA peak (TFLOP/s): SMs x 128 FP32 lanes x 2 flop x the measured maximum SM clock."""
    import torch

    peaks = measured_peaks() or {}
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    return nsm * 128 * 2 * sm_max * 1e6 / 1e12


def row_bispectrum(dev, host64, big_box, profile_range=False):
    import torch

    from paper_1512_07295_gb300 import api, ffi

    rows = {}
    # a7: FFT bispectrum, 16 shells of width 4 k_f (up to k_N/2) on N_G = 256, delta of the large catalogue
    cfg = api.Config(ng=256, box=big_box, prec="fp32")
    n = host64.shape[0]
    dpos = host64.to(dev)
    _, _, _, delta = api.power(dpos, cfg, return_delta=True)
    del dpos
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    counts = api.bispectrum_counts(cfg, 0, 4, 16, dev)
    torch.cuda.synchronize()
    t_counts = time.perf_counter() - t0
    ws = api.workspace(cfg, 16, ffi.PK_WS_BISPECTRUM, dev)
    out = torch.empty(api.bispectrum_ntri(16), dtype=torch.float64, device=dev)

    def bisp():
        check = ffi.lib().pk_bispectrum(api.ctypes.byref(cfg.c()), api._p(delta), 0, 4, 16, api._p(counts), api._p(out),
                                        api._p(ws), ws.numel(), api._stream(dev))
        ffi.check(check)

    ms = _time_cuda(bisp, 5)
    if profile_range:  # one call bracketed for ncu --profile-from-start off
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        bisp()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    rows["bispectrum"] = {"workload": f"delta of the {n}-particle catalogue on N_G=256, 16 shells of 4 k_f, 508 triangles",
                          "ms_per_call": ms, "bispectra_per_s": 1e3 / ms, "triangles": int(out.numel()),
                          "counts_once_s": t_counts}
    del ws, delta, counts, out
    torch.cuda.empty_cache()
    return rows["bispectrum"]


def row_bispectrum_only(dev, a):
    """The bispectrum row on its own: the catalogue generated on the GPU, then row_bispectrum."""
    import torch

    from paper_1512_07295_gb300 import catalogs

    pos = catalogs.zeldovich_torch(a.nside, a.box, RMS_DISP, seed=replica_seed(0), device=dev).cpu()
    torch.cuda.empty_cache()
    return row_bispectrum(dev, pos, a.box, a.profile_range)


def row_adjoint(dev):
    import torch

    from paper_1512_07295_gb300 import api, catalogs, ffi

    rows = {}
    # a8: adjoint, 128^3 Zel'dovich particles, L = 500, N_G = 128, PCS + interlacing, FP32
    cfg = api.Config(ng=128, box=500.0, prec="fp32")
    pos = catalogs.zeldovich_torch(128, 500.0, 4.0, seed=6, device=dev)
    dl = torch.randn(cfg.nb, dtype=torch.float64, device=dev)
    wsb = api.workspace(cfg, pos.shape[0], ffi.PK_WS_BACKWARD, dev)
    g = torch.empty((pos.shape[0], 3), dtype=torch.float32, device=dev)

    def back():
        ffi.check(ffi.lib().pk_power_backward(api.ctypes.byref(cfg.c()), api._p(pos), ffi.PK_POS_F64_XYZ, None, pos.shape[0],
                                              api._p(dl), api._p(g), api._p(wsb), wsb.numel(), api._stream(dev)))

    ms = _time_cuda(back, 10, 2)
    rows["adjoint"] = {"workload": "dL/dx of P(k), 128^3 ZA particles, L=500, N_G=128, PCS+interlacing, FP32 (forward grids "
                                   "recomputed inside)", "ms_per_call": ms, "particles_per_s": pos.shape[0] / (ms * 1e-3)}
    del wsb, g, pos
    torch.cuda.empty_cache()
    return rows["adjoint"]


def row_batch(dev, profile_range=False, ncats=512):
    import torch

    from paper_1512_07295_gb300 import api, catalogs

    rows = {}
    # a9: 512 mock catalogues, N_P log-uniform in [1e5, 2e6], L = 1000, N_G = 128, PCS + interlacing, FP32
    # (fewer with --batch-cats, for profiling captures)
    cfg = api.Config(ng=128, box=1000.0, prec="fp32")
    sizes = catalogs.batch_sizes(ncats, 1e5, 2e6, seed=4)
    gen = torch.Generator(device=dev)
    gen.manual_seed(4)
    parts = []
    for i, m in enumerate(sizes):
        m = int(m)
        if i % 2 == 0:
            p64 = torch.rand((m, 3), generator=gen, device=dev, dtype=torch.float64) * 1000.0
        else:
            side = int(np.ceil(m ** (1.0 / 3.0)))
            p64 = catalogs.zeldovich_torch(side, 1000.0, 4.0, seed=1000 + i, device=dev)[:m].contiguous()
        parts.append(api.prepare(p64, cfg))
        del p64
    cells = torch.cat(parts)
    del parts
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    # group size chosen by the library's autotuner, then the call timed eagerly and as a CUDA graph replay
    batch, tune_ms = api.autotune_batch(cells, offs, cfg, candidates=(64, 128, 256, 512), reps=2, runs=(1, 2, 4))
    wsc = api.batch_workspace(cfg, batch, api.max_group_particles(offs, batch), dev)
    pkb = torch.empty((ncats, cfg.nb), dtype=torch.float64, device=dev)
    nmb = torch.empty((ncats, cfg.nb), dtype=torch.int64, device=dev)
    ms = _time_cuda(lambda: api.batch_power(cells, offs, cfg, batch=batch, ws=wsc, out=(pkb, nmb)), 3)
    if profile_range:  # one call bracketed for ncu --profile-from-start off
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        api.batch_power(cells, offs, cfg, batch=batch, ws=wsc, out=(pkb, nmb))
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(dev)
    cap.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(cap):
        with torch.cuda.graph(graph, stream=cap):
            api.batch_power(cells, offs, cfg, batch=batch, ws=wsc, out=(pkb, nmb))
    torch.cuda.current_stream(dev).wait_stream(cap)
    ms_graph = _time_cuda(graph.replay, 3)
    rows["batch"] = {"workload": f"{ncats} catalogues, {int(sizes.sum())} particles, N_P log-uniform in [1e5, 2e6], L=1000, "
                                 f"N_G=128, PCS+interlacing, FP32, groups of {batch}, scatter runs of {cfg.tile_run} "
                                 f"tile(s) (autotuned)",
                     "ms_per_call": ms, "pk_per_s": ncats / (ms * 1e-3), "particles_per_s": float(sizes.sum()) / (ms * 1e-3),
                     "graph_ms_per_call": ms_graph, "autotune_ms": {str(k): v for k, v in tune_ms.items()}}
    del graph
    del wsc, cells
    torch.cuda.empty_cache()
    return rows["batch"]


def row_direct(dev, alu_peak_tflops, nside=128, ng=128):
    import torch

    from paper_1512_07295_gb300 import api, catalogs, ffi

    rows = {}
    # direct summation (eq:deltaDS): 128^3 Zel'dovich particles, L = 50, every stored mode of N_G = 128,
    # then the Sec. 3.2 comparison of the PCS + interlacing grid estimate with it
    cfg = api.Config(ng=ng, box=50.0, order=4, interlace=True, prec="fp32")
    pos = catalogs.zeldovich_torch(nside, 50.0, 1.0, seed=7, device=dev)
    n = pos.shape[0]
    wsd = api.workspace(cfg, n, ffi.PK_WS_DIRECT, dev)
    ds = torch.empty((ng, ng, ng // 2 + 1), dtype=torch.complex64, device=dev)

    def direct():
        ffi.check(ffi.lib().pk_direct_modes(api.ctypes.byref(cfg.c()), api._p(pos), ffi.PK_POS_F64_XYZ, None, n, api._p(ds),
                                            api._p(wsd), wsd.numel(), api._stream(dev)))

    ms = _time_cuda(direct, 3)
    pairs = float(n) * ng * ng * (ng // 2 + 1)
    tflops = 8.0 * pairs / (ms * 1e-3) / 1e12
    # the FP32 path runs on the tensor cores with three TF32 products per complex multiply-add; its
    # peak is the measured dense bf16 rate times the nominal TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s)
    peaks = measured_peaks() or {}
    tf32_peak = float(peaks.get("bf16_tflops", 1900.0)) * (1.1 / 2.25)
    p_ds, _, _ = api.cross_power(ds, ds, cfg)
    _, _, _, dg = api.power(pos, cfg, return_delta=True)
    p_g, _, _ = api.cross_power(dg, dg, cfg)
    p_x, _, _ = api.cross_power(dg, ds, cfg)
    shot = 50.0 ** 3 / n  # auto and cross spectra corrected by 1/nbar as in Sec. 3.2
    rel_auto = torch.abs((p_g - shot) / (p_ds - shot) - 1.0)
    rel_cross = torch.abs((p_x - shot) / (p_ds - shot) - 1.0)
    half = ng // 4 - 1  # the bin at k_N / 2
    rows["direct"] = {"workload": f"direct summation of delta(k) (eq:deltaDS): {nside}^3 ZA particles, L=50, all "
                                  f"{ng * ng * (ng // 2 + 1)} stored modes of N_G={ng}, FP32 terms with compensated sums",
                      "ms_per_call": ms, "pairs_per_s": pairs / (ms * 1e-3),
                      "roofline": {"bound": "tensor", "achieved": 3.0 * tflops, "peak": tf32_peak, "unit": "TFLOP/s",
                                   "frac": 3.0 * tflops / tf32_peak, "flop_per_pair": 24,
                                   "peak_source": "MEASURED_PEAKS.json bf16_tflops (of measured) x nominal TF32/BF16 1.1/2.25",
                                   "note": "three TF32 products per complex multiply-add; operand generation on the CUDA "
                                           "cores bounds the kernel"},
                      "fp32_equivalent": {"achieved": tflops, "peak": alu_peak_tflops, "unit": "TFLOP/s",
                                          "frac": tflops / alu_peak_tflops, "flop_per_pair": 8,
                                          "peak_source": "derived: SMs x 128 FP32 lanes x 2 flop x max SM clock"},
                      "pcs_interlace_vs_ds": {"max_rel_auto": rel_auto.max().item(), "max_rel_cross": rel_cross.max().item(),
                                              "rel_auto_at_half_kN": rel_auto[half].item(),
                                              "rel_cross_at_half_kN": rel_cross[half].item()}}
    del wsd, ds, dg, pos
    torch.cuda.empty_cache()
    return rows["direct"]


def row_multigrid(dev):
    import torch

    from paper_1512_07295_gb300 import api, catalogs

    # multi-grid interlacing: P(k) of 256^3 ZA particles (L = 500, N_G = 256, PCS, FP32) from J = 2, 4, 8
    # shifted grids; accuracy against the direct sum on 64^3 particles / N_G = 64 (L = 50, Sec. 3.2 style,
    # shot noise subtracted from both), in FP64 so that the aliasing left, not FP32 rounding, is measured
    out = {"workload": "P(k) from J half-cell-shifted grids, 256^3 ZA particles, L=500, N_G=256, PCS, FP32; accuracy "
                       "(FP64) vs direct summation on 64^3 ZA particles, L=50, N_G=64", "ms_per_call": {},
           "max_rel_vs_ds": {}, "rel_vs_ds_at_kN": {}}
    cfg = api.Config(ng=256, box=500.0, order=4, prec="fp32")
    pos = catalogs.zeldovich_torch(256, 500.0, 4.0, seed=8, device=dev)
    for J in (2, 4, 8):
        out["ms_per_call"][str(J)] = _time_cuda(lambda: api.power_multigrid(pos, cfg, J), 3)
    del pos
    torch.cuda.empty_cache()
    small = api.Config(ng=64, box=50.0, order=4, prec="fp64")
    pos = catalogs.zeldovich_torch(64, 50.0, 1.0, seed=7, device=dev)
    ds = api.direct_modes(pos, small)
    p_ds, _, _ = api.cross_power(ds, ds, small)
    shot = 50.0 ** 3 / pos.shape[0]
    for J in (1, 2, 4, 8):
        pk, _, _ = api.power_multigrid(pos, small, J)
        rel = torch.abs((pk - shot) / (p_ds - shot) - 1.0)
        out["max_rel_vs_ds"][str(J)] = rel.max().item()
        out["rel_vs_ds_at_kN"][str(J)] = rel[-1].item()
    del pos, ds
    torch.cuda.empty_cache()
    return out


def row_e2e(dev, nside, ng, box, profile_range=False):
    """pk_power_host alone on the benchmark's catalogue (pinned host FP64 positions), for profiling."""
    import torch

    from paper_1512_07295_gb300 import api, catalogs, ffi

    cfg = api.Config(ng=ng, box=box, order=4, interlace=True, prec="fp32")
    n = nside ** 3
    host64 = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
    host64.copy_(catalogs.zeldovich_torch(nside, box, RMS_DISP, seed=replica_seed(0), device=dev))
    torch.cuda.empty_cache()
    wsp = api.workspace(cfg, n, ffi.PK_WS_POWER_HOST, dev)
    host_out = (torch.empty(cfg.nb, dtype=torch.float64, pin_memory=True),
                torch.empty(cfg.nb, dtype=torch.float64, pin_memory=True),
                torch.empty(cfg.nb, dtype=torch.int64, pin_memory=True))
    ms = _time_cuda(lambda: api.power_host(host64, cfg, ws=wsp, out=host_out, device=dev), 3)
    if profile_range:  # one call bracketed for ncu --profile-from-start off
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        api.power_host(host64, cfg, ws=wsp, out=host_out, device=dev)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    return {"workload": f"pk_power_host, {n} particles from pinned host FP64 positions, N_G={ng}", "ms_per_call": ms}


def row_ng1024(dev, pos64, box, hbm_peak, ng=1024, profile_range=False):
    """The benchmark catalogue on an N_G = 1024 grid (PCS + interlacing, FP32, binned records resident):
    one particle per cell, so every tile goes to the per-particle scatter. (ng: another grid size for
    a smaller case of the same kind, e.g. 256^3 particles on N_G = 256 for a profile.)"""
    import torch

    from paper_1512_07295_gb300 import api, ffi

    cfg = api.Config(ng=ng, box=box, order=4, interlace=True, prec="fp32")
    n = pos64.shape[0]
    cells = api.prepare(pos64, cfg)
    binned = api.bin_particles(cells, cfg)
    del cells
    torch.cuda.empty_cache()
    ws = api.workspace(cfg, n, ffi.PK_WS_POWER_BINNED, dev)
    out = (torch.empty(cfg.nb, dtype=torch.float64, device=dev), torch.empty(cfg.nb, dtype=torch.float64, device=dev),
           torch.empty(cfg.nb, dtype=torch.int64, device=dev))
    ms = _time_cuda(lambda: api.power_binned(binned, cfg, ws=ws, out=out), 5, 2)
    if profile_range:  # one call bracketed for ncu --profile-from-start off
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        api.power_binned(binned, cfg, ws=ws, out=out)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    lib = ffi.lib()
    lib.pk_profile_enable(1)
    stages = np.zeros(5)
    buf = (ctypes.c_double * 5)()
    for _ in range(3):
        api.power_binned(binned, cfg, ws=ws, out=out)
        lib.pk_profile_read(ctypes.cast(buf, ctypes.c_void_p), 5)
        stages += np.array(list(buf)) / 3
    lib.pk_profile_enable(0)
    nh = ng * ng * (ng // 2 + 1)
    path_bytes = 16.0 * n + 2 * (4.0 * ng ** 3 + (4.0 * ng ** 3 + 8.0 * nh) + 8.0 * nh)
    del ws, binned
    torch.cuda.empty_cache()
    return {"workload": f"{n} ZA particles, L={box:g} Mpc/h, N_G={ng}, PCS+interlacing, FP32 binned records",
            "ms_per_call": ms, "particles_per_s": n / (ms * 1e-3), "pk_per_s": 1e3 / ms,
            "stages_ms": {"grid_clear": float(stages[1]), "assign": float(stages[2]), "fft": float(stages[3]),
                          "estimate": float(stages[4])},
            "path_hbm_roofline": {"algorithmic_bytes": path_bytes, "achieved_gbs": path_bytes / (ms * 1e-3) / 1e9,
                                  "peak_gbs": hbm_peak, "frac": path_bytes / (ms * 1e-3) / 1e9 / hbm_peak}}


def row_c1(dev):
    """Config 1: 64^3 Poisson particles, L = 1000 Mpc/h, N_G = 64, PCS + interlacing, from device FP64
    positions: ms per P(k) in FP64 and FP32, their difference per bin, and P(k) against the shot noise
    V/N at the lowest 8 bins (the aliased shot noise of PCS + interlacing stays near 1 there)."""
    import torch

    from paper_1512_07295_gb300 import api, catalogs, ffi

    box, ng = 1000.0, 64
    pos = torch.from_numpy(catalogs.poisson(64 ** 3, box, seed=5)).to(dev)
    res = {}
    pks = {}
    for prec in ("fp64", "fp32"):
        cfg = api.Config(ng=ng, box=box, prec=prec)
        ws = api.workspace(cfg, pos.shape[0], ffi.PK_WS_POWER, dev)
        res[f"{prec}_ms_per_pk"] = _time_cuda(lambda: api.power(pos, cfg, ws=ws), 10, 3)
        pks[prec] = api.power(pos, cfg, ws=ws)[0].cpu().numpy()
    rel = np.abs(pks["fp32"] / pks["fp64"] - 1.0)
    shot = box ** 3 / pos.shape[0]
    res.update({"workload": "64^3 Poisson particles, L=1000 Mpc/h, N_G=64, PCS+interlacing, FP64 device positions",
                "fp32_vs_fp64_max_rel": float(rel.max()), "fp32_vs_fp64_median_rel": float(np.median(rel)),
                "p_over_shot_noise_first_8_bins": _sig(pks["fp64"][:8] / shot, 4)})
    # the single-particle check: one particle at (123.4, 567.8, 901.2), FP64 grids: its mass and the
    # p^3 nodes of each stencil
    cfg64 = api.Config(ng=ng, box=box, prec="fp64")
    one = torch.tensor([[123.4, 567.8, 901.2]], dtype=torch.float64, device=dev)
    g1, g2 = api.assign(one, cfg64)
    res["single_particle"] = {"grid_sums_minus_1": [float(g1.sum().item() - 1.0), float(g2.sum().item() - 1.0)],
                              "nonzero_nodes": [int(torch.count_nonzero(g1).item()), int(torch.count_nonzero(g2).item())]}
    # the lattice check: one particle on every node, so every mode n != 0 of either grid vanishes
    ax = (torch.arange(ng, dtype=torch.float64, device=dev) + 0.0) * (box / ng)
    lat = torch.stack(torch.meshgrid(ax, ax, ax, indexing="ij"), dim=-1).reshape(-1, 3).contiguous()
    plat = api.power(lat, cfg64)[0].cpu().numpy()
    res["lattice_max_p_over_shot_noise"] = float(np.max(np.abs(plat)) / (box ** 3 / lat.shape[0]))
    return res


def row_ng1024_only(dev, a):
    """The N_G = 1024 row on its own: the catalogue generated on the GPU, then row_ng1024."""
    from paper_1512_07295_gb300 import catalogs

    pos = catalogs.zeldovich_torch(a.nside, a.box, RMS_DISP, seed=replica_seed(0), device=dev)
    return row_ng1024(dev, pos, a.box, float((measured_peaks() or {}).get("hbm_gbs", 6800.0)), a.row_ng, a.profile_range)


def measure_rows(dev, host64, big_box, alu_peak_tflops):
    """Times the other hot-path rows on their own workloads (one GB300)."""
    return {"bispectrum": row_bispectrum(dev, host64, big_box), "adjoint": row_adjoint(dev), "batch": row_batch(dev),
            "direct": row_direct(dev, alu_peak_tflops), "multigrid": row_multigrid(dev)}


def run_reference(a):
    """The reference arm: the FP64 CPU oracle on the host cores, one bounded sample of the workload per
    step: the oracle's assignment (both grids) of 2^20 particles over a process pool of every core,
    scaled linearly to the full catalogue, plus the oracle's FFT, deconvolution, interlacing and binning
    of one full N_G grid pair (timed once, added to every step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import concurrent.futures
    import multiprocessing

    import oracle
    from paper_1512_07295_gb300 import catalogs

    n_full = a.nside ** 3
    cores = len(os.sched_getaffinity(0))
    # a Zel'dovich catalogue of the same box and displacement recipe, 128^3 particles: the oracle's cost
    # per particle does not depend on the clustering, so it stands in as the sample source
    src = catalogs.zeldovich(128, a.box, rms=RMS_DISP, seed=3)
    rng = np.random.default_rng(5)
    sample = 1 << 20
    t0 = time.perf_counter()
    r1 = oracle.assign.assign_units(oracle.assign.grid_units(src[:4096], a.box, a.ng), a.ng, 4)
    r2 = oracle.assign.assign_units(oracle.assign.grid_units(src[:4096], a.box, a.ng), a.ng, 4, shift=True)
    t1 = time.perf_counter()
    oracle.power.power_spectrum(oracle.fourier.density_modes(r1, 4, r2), a.box)
    t_fft = time.perf_counter() - t1
    del r1, r2
    rates = []
    with concurrent.futures.ProcessPoolExecutor(cores, mp_context=multiprocessing.get_context("spawn")) as ex:
        for step in range(a.warmup + a.steps):
            pos = src[rng.choice(len(src), size=sample, replace=False)]
            u = oracle.assign.grid_units(pos, a.box, a.ng)
            ts = time.perf_counter()
            for _ in ex.map(_oracle_assign_chunk, [(c, a.ng, 4) for c in np.array_split(u, cores)]):
                pass
            t_assign = time.perf_counter() - ts
            if step >= a.warmup:
                rates.append(n_full / (t_assign * n_full / sample + t_fft))
    wall = time.perf_counter() - t0
    value = float(np.median(rates))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * n_full / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "timed": "FP64 CPU oracle per step: 2^20-particle assignment of both grids "
                   f"over {cores} worker processes, scaled to {n_full} particles, + one N_G={a.ng} FFT/deconvolution/"
                   "binning (timed once)"},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle",
                         "sample": f"2^20 particles per step of a 128^3 Zel'dovich catalogue of the same recipe (assignment, "
                                   f"both grids, {cores} processes) + one full N_G={a.ng} FFT (scipy, {cores} workers) and "
                                   "binning; extrapolated linearly in N_P"},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall, "t_fft_estimate_s": t_fft,
    }
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.quick:
        a.nside, a.ng, a.box = 128, 128, 500.0
    if a.impl == "reference":
        run_reference(a)
        return

    import torch
    import torch.distributed as dist

    from paper_1512_07295_gb300 import api, catalogs, ffi

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = ffi.lib()
    if a.only_row:
        row = {"adjoint": lambda: row_adjoint(dev), "batch": lambda: row_batch(dev, a.profile_range, a.batch_cats),
               "bispectrum": lambda: row_bispectrum_only(dev, a),
               "direct": lambda: row_direct(dev, alu_peak(dev), a.ds_nside, a.ds_ng),
               "multigrid": lambda: row_multigrid(dev),
               "e2e": lambda: row_e2e(dev, a.nside, a.ng, a.box, a.profile_range),
               "ng1024": lambda: row_ng1024_only(dev, a),
               "c1": lambda: row_c1(dev)}[a.only_row]()
        if rank == 0:
            print(json.dumps({"row": a.only_row, **row}), flush=True)
        return

    n = a.nside ** 3
    cfg = api.Config(ng=a.ng, box=a.box, order=4, interlace=True, prec="fp32")

    # ---- input: seeded Zel'dovich catalogue (one independent realisation per rank) ----------------
    pos64 = catalogs.zeldovich_torch(a.nside, a.box, RMS_DISP, seed=replica_seed(rank), device=dev)
    host64 = None
    if not a.no_extras:
        host64 = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
        host64.copy_(pos64)
    cells = api.prepare(pos64, cfg)
    del pos64
    torch.cuda.empty_cache()
    binned = api.bin_particles(cells, cfg)
    del cells
    torch.cuda.empty_cache()
    sorted_, _, offsets = binned
    ws = api.workspace(cfg, n, ffi.PK_WS_POWER_BINNED, dev)
    out = (torch.empty(cfg.nb, dtype=torch.float64, device=dev), torch.empty(cfg.nb, dtype=torch.float64, device=dev),
           torch.empty(cfg.nb, dtype=torch.int64, device=dev))
    torch.cuda.synchronize()

    def step():
        api.power_binned(binned, cfg, ws=ws, out=out)

    # ---- timed region ------------------------------------------------------------------------------
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    launches0 = lib.pk_profile_launches()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.profile_range:
        torch.cuda.profiler.start()
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if a.profile_range:
        torch.cuda.profiler.stop()
    launches = lib.pk_profile_launches() - launches0
    clk = clocks.stop()
    ms_total = max_over_ranks(e0.elapsed_time(e1), dev)
    ms_step = ms_total / a.steps
    value = job_rate(world, n, a.steps, ms_total)
    pk_per_s = job_rate(world, 1, a.steps, ms_total)

    # ---- per-stage times (same calls, CUDA events at the stage boundaries) ----------------------------
    lib.pk_profile_enable(1)
    stages = np.zeros(5)
    nprof = max(3, min(a.steps, 10))
    buf = (ctypes.c_double * 5)()
    for _ in range(nprof):
        step()
        lib.pk_profile_read(ctypes.cast(buf, ctypes.c_void_p), 5)
        stages += np.array(list(buf))
    lib.pk_profile_enable(0)
    stages /= nprof
    t_assign_ms = float(stages[2])

    peaks = measured_peaks() or {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    alu_peak_tflops = alu_peak(dev)  # FP32 FMA lanes x 2 flop x max clock
    p3 = cfg.order ** 3
    assign_flop = 2.0 * 2 * p3 * n  # two grids, p^3 multiply-adds per particle each
    assign_bytes = 16.0 * n + 2 * 4.0 * a.ng ** 3  # particle records read once, two grids written once
    achieved_tflops = assign_flop / (t_assign_ms * 1e-3) / 1e12
    achieved_gbs = assign_bytes / (t_assign_ms * 1e-3) / 1e9
    same_density = a.nside ** 3 == 8 * a.ng ** 3
    traffic = ASSIGN_TRAFFIC_PER_PARTICLE * n if (ASSIGN_TRAFFIC_PER_PARTICLE and same_density) else None
    nh = a.ng * a.ng * (a.ng // 2 + 1)
    path_bytes = 16.0 * n + 2 * (4.0 * a.ng ** 3 + (4.0 * a.ng ** 3 + 8.0 * nh) + 8.0 * nh)
    result = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(a), "particles": n, "ng": a.ng, "box": a.box, "order": 4, "interlace": True,
                   "l2": "inputs (16 B x 1024^3 particles = 17.2 GB) far exceed the 129 MB L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "pk_per_s": pk_per_s,
        # the dominant kernel against the HBM roofline (algorithmic bytes / CUDA-event time of the stage)
        "roofline": {"kernel": "k_assign_cells<4,false>", "bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak,
                     "unit": "GB/s", "frac": achieved_gbs / hbm_peak, "traffic": traffic,
                     "traffic_source": ASSIGN_TRAFFIC_SOURCE if traffic else None, "algorithmic_bytes": assign_bytes,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                     "timing": "CUDA events on the library's stream around the assignment stage (scatter pass + key-cell "
                               f"kernel), mean over {nprof} steps",
                     "note": "bound by shared-memory and instruction issue, not DRAM: see alu",
                     "alu": {"achieved": achieved_tflops, "peak": alu_peak_tflops, "unit": "TFLOP/s",
                             "frac": achieved_tflops / alu_peak_tflops,
                             "peak_source": "derived: SMs x 128 FP32 lanes x 2 flop x the maximum SM clock"}},
        "path_hbm_roofline": {"algorithmic_bytes": path_bytes, "achieved_gbs": path_bytes / (ms_step * 1e-3) / 1e9,
                              "peak_gbs": hbm_peak, "frac": path_bytes / (ms_step * 1e-3) / 1e9 / hbm_peak},
        "stages_ms": {"weights": stages[0], "grid_clear": stages[1], "assign": stages[2], "fft": stages[3],
                      "estimate": stages[4]},
        "clocks": clk,
        "gpu_launches": int(launches),
    }
    pk32_step = out[0].clone()

    if rank == 0 and not a.no_extras:
        # ---- plain FP64 GPU path on the same binned catalogue ---------------------------------------
        del ws
        torch.cuda.empty_cache()
        cfg64 = api.Config(ng=a.ng, box=a.box, order=4, interlace=True, prec="fp64")
        ws64 = api.workspace(cfg64, n, ffi.PK_WS_POWER_BINNED, dev)
        api.power_binned(binned, cfg64, ws=ws64)
        torch.cuda.synchronize()
        k64 = 2
        e0.record(stream)
        for _ in range(k64):
            api.power_binned(binned, cfg64, ws=ws64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / k64
        result["fp64_plain"] = {"ms_per_step": ms64, "value": n / (ms64 * 1e-3), "unit": "particles/s",
                                "speedup_of_fast_path": ms64 / ms_step}
        del ws64
        torch.cuda.empty_cache()
        # ---- the deterministic path (PK_FIXED64: 64-bit fixed-point grids) on the same catalogue ----
        cfgfx = api.Config(ng=a.ng, box=a.box, order=4, interlace=True, prec="fixed64")
        wsfx = api.workspace(cfgfx, n, ffi.PK_WS_POWER_BINNED, dev)
        pa = api.power_binned(binned, cfgfx, ws=wsfx)[0].clone()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k64):
            pb = api.power_binned(binned, cfgfx, ws=wsfx)[0]
        e1.record(stream)
        torch.cuda.synchronize()
        msfx = e0.elapsed_time(e1) / k64
        result["fixed64"] = {"ms_per_step": msfx, "value": n / (msfx * 1e-3), "unit": "particles/s",
                             "bitwise_repeatable": bool(torch.equal(pa, pb)),
                             "path": "PK_FIXED64: FP32 contributions summed exactly in 64-bit fixed point (grids and "
                                     "bin sums), binned records resident"}
        del wsfx, binned, sorted_, offsets
        torch.cuda.empty_cache()

        # ---- the FP32 step's error per k-bin against FP64 from the FP64 positions ------------------
        # (positions, assignment, transforms and estimate together), and pk_power from the unsorted
        # device FP64 positions (a1 + a2 + the step: preparation and binning inside the timed call)
        pos64 = catalogs.zeldovich_torch(a.nside, a.box, RMS_DISP, seed=replica_seed(rank), device=dev)
        pk64, _, n64 = api.power(pos64, cfg64)
        rel = _rel_per_bin(pk32_step, pk64)
        result["fp32_vs_fp64_per_bin"] = {
            "reference": "pk_power in PK_FP64 from the FP64 positions (FP64 grids and transforms; oracle parity 1e-10)",
            "max_rel": float(rel.max()), "median_rel": float(np.median(rel)), "per_bin": _sig(rel, 2)}
        torch.cuda.empty_cache()
        wsu = api.workspace(cfg, n, ffi.PK_WS_POWER, dev)
        out_u = (torch.empty(cfg.nb, dtype=torch.float64, device=dev), torch.empty(cfg.nb, dtype=torch.float64, device=dev),
                 torch.empty(cfg.nb, dtype=torch.int64, device=dev))

        def unsorted_step():
            ffi.check(ffi.lib().pk_power(api.ctypes.byref(cfg.c()), api._p(pos64), ffi.PK_POS_F64_XYZ, None, n,
                                         api._p(out_u[0]), api._p(out_u[1]), api._p(out_u[2]), None, api._p(wsu),
                                         wsu.numel(), api._stream(dev)))

        ms_u = _time_cuda(unsorted_step, 3)
        result["from_unsorted_device_positions"] = {
            "ms_per_step": ms_u, "value": n / (ms_u * 1e-3), "unit": "particles/s",
            "path": "pk_power from device FP64 xyz: a1 prepare + a2 counting sort by tile + the timed step's a3..a6"}
        del wsu
        torch.cuda.empty_cache()
        ng1024 = row_ng1024(dev, pos64, a.box, hbm_peak) if a.nside ** 3 >= 1024 ** 3 else None

        # ---- e2e through pk_power_host from pinned host FP64 positions ------------------------------
        # the positions cross the CPU-GPU link in pieces while the previous piece is processed; P(k),
        # kmean and the mode counts come back to pinned host memory, all inside the timed region
        wsp = api.workspace(cfg, n, ffi.PK_WS_POWER_HOST, dev)
        host_out = (torch.empty(cfg.nb, dtype=torch.float64, pin_memory=True),
                    torch.empty(cfg.nb, dtype=torch.float64, pin_memory=True),
                    torch.empty(cfg.nb, dtype=torch.int64, pin_memory=True))

        def e2e_step():
            api.power_host(host64, cfg, ws=wsp, out=host_out, device=dev)

        # context for e2e: the link's rate for the whole catalogue in one copy, just before it, and where
        # the pinned buffer's pages and the GPU sit
        pos64.copy_(host64, non_blocking=True)
        torch.cuda.synchronize()
        e0.record(stream)
        pos64.copy_(host64, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        link_gbs = 24.0 * n / (e0.elapsed_time(e1) * 1e-3) / 1e9
        del pos64
        torch.cuda.empty_cache()

        e2e_step()
        torch.cuda.synchronize()
        ke = 3
        e0.record(stream)
        for _ in range(ke):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = e0.elapsed_time(e1) / ke
        result["e2e"] = {"value": n / (ms_e2e * 1e-3), "unit": "particles/s", "h2d_bytes_per_step": 24 * n,
                         "d2h_bytes_per_step": 24 * cfg.nb, "ms_per_step": ms_e2e,
                         "link_h2d_gbs_one_copy": link_gbs,
                         "one_copy_ms": 24.0 * n / (link_gbs * 1e9) * 1e3,
                         "gpu_work_ms": ms_u, "numa": numa_report(host64, local),
                         "path": "pk_power_host: pinned host FP64 xyz copied over the CPU-GPU link in 16 pieces by the "
                                 "copy engine, each prepared, binned and assigned while the next is in flight -> FFT -> "
                                 "estimate -> D2H of P(k), kmean, counts"}
        del wsp
        torch.cuda.empty_cache()

        # ---- other hot-path rows and the 256^3 accuracy table ---------------------------------------
        result["rows"] = measure_rows(dev, host64, a.box, alu_peak_tflops)
        result["rows"]["accuracy_c2"] = row_accuracy_c2(dev)
        result["rows"]["c1"] = row_c1(dev)
        if ng1024 is not None:
            result["rows"]["ng1024"] = ng1024

        # ---- FP64 CPU oracle ----------------------------------------------------------------------
        cores = len(os.sched_getaffinity(0))
        rng = np.random.default_rng(11)
        idx = np.sort(rng.choice(n, size=1 << 20, replace=False))
        sample = host64[torch.from_numpy(idx)].numpy()
        t0 = time.perf_counter()
        _, t_assign, t_rest = oracle_power_parallel(sample, a.box, a.ng, 4, cores)
        t_full = t_assign * (n / len(sample)) + t_rest
        result["cpu_baseline"] = {"value": n / t_full, "unit": "particles/s", "cores": cores, "kind": "oracle",
                                  "sample": f"2^20 random particles of the catalogue assigned to both grids (the oracle's "
                                            f"assignment over {cores} worker processes) + one full N_G={a.ng} FFT, "
                                            "deconvolution and binning; assignment time scaled linearly to the full "
                                            "catalogue (extrapolated)",
                                  "t_assign_s": t_assign, "t_fft_estimate_s": t_rest, "sample_particles": len(sample),
                                  "t_full_extrapolated_s": t_full, "wall_s": time.perf_counter() - t0}
        if not a.no_oracle:
            result["cpu_oracle_measured"] = measured_oracle_rows()
    elif not a.no_extras:
        result["e2e"] = None
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
