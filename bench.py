#!/usr/bin/env python
"""Benchmark of the Monte-Carlo snakuscule hot path on GB300.

One step = the whole path over one synthetic image: ingest the voxels into the
library's volume (a1), seed the lattice (a2), evolve every contour for T
iterations (a3-a8: Philox samples, trilinear gathers from TMA-staged bricks,
compensated warp reductions, gradient steps) and localize (a9: energy cull and
overlap competition, cells copied to the host).

Metric: MC contour samples per second (contours x samples x iterations per step /
step time), the default workload being the 1024x1024x256 uint16 brain-like volume
with ~100k nuclei (spacing 1:1:2, stride-6 lattice of 2,456,500 contours, 512
samples, 100 iterations); `--workload large-2d` runs the 4096x4096 2D image.  `value` is measured with the
input already in HBM; `e2e` repeats the step through the same C ABI from pinned
host memory (host-to-device copy of the image and device-to-host copy of the cells
inside the timed region).  The roofline entry covers the evolution kernel (plain
ALU issue bound), `cpu_baseline` times the FP64 oracle on the host cores on a
bounded sample of the same workload.  On one GPU the default line also records,
under `forms`, short runs of the batching form (64 uneven volumes in one
autotuned, graph-replayed plan) and the serving form (the request loop's
throughput and tile latencies), each in a child process after the timed steps.

With torchrun (N > 1) every rank processes its own image (weak scaling, replicas:
contours never interact across images); the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# Algorithmic ALU work per sample, in issue slots: the lean instruction count of
# one sample -- Philox4x32-10 (10 rounds of two wide multiplies and two three-input
# XORs per block), word-to-float conversions, radius and direction (hardware
# sqrt / lg2+ex2 / sin / cos), index offsets, floor and fraction per axis, the
# gather and multilinear interpolation, the two weight bands, and the sums (one
# product and one pairwise addition per sum, and a four-operation compensated step
# per block of B samples), with each pair of independent FP32 operations that the
# packed two-lane instructions can take counted as one slot.  2D: 52.75 (a Philox
# block serves two samples; one quad load of row values and x-differences per
# bilinear gather; B = 8); 3D: 102.25 (counted when a 3D sample took three whole
# words; eight 8/16-bit taps, each one operation from exact biased floats; B = 4).
# The per-iteration reduction and update are excluded.  These counts are frozen as
# the definition of the work; the two-word 3D samples of the current kernel (one
# block per two samples) have a leaner count of their own, 95.25, reported beside.
ALG_SLOTS_PER_SAMPLE = {2: 52.75, 3: 102.25}
ALG_SLOTS_CURRENT = {2: 52.75, 3: 95.25}
# dram__bytes_read.sum + dram__bytes_write.sum of the evolve kernel per launch, from
# ncu captures of the current kernel (to be removed when the kernel changes): brain-3d
# at full size (one pass: 759.12 MB read + 54.86 MB written); large-2d from its
# 2048^2 instance (7.42 MB read + 0.04 MB written) scaled with the image (x 4).
DRAM_BYTES_PER_LAUNCH = {
    ("brain-3d", "brick", 0, "native"): (814.0e6, "ncu capture of the full-size launch"),
    ("large-2d", "brick", 0, "native"): (29.9e6, "ncu capture of the 2048^2 instance scaled with the image (x 4)"),
}
SM_COUNT = 152
LANES_PER_SM_CLOCK = 128          # 4 schedulers x 32 lanes, one instruction per clock
SM_MAX_MHZ = 2070.0

WORKLOADS = {
    "large-2d": dict(ndim=2, stride=6.0, N=128, T=100, seed=1,
                     desc="4096x4096 uint8, ~12k disks r 5-10, blur 1.5 + Poisson; stride-6 lattice (465,124 "
                          "contours), 128 samples, 100 iterations"),
    "brain-3d": dict(ndim=3, stride=6.0, N=512, T=100, seed=2,
                     desc="1024x1024x256 uint16 spacing 1:1:2, ~100k ellipsoids, log-normal brightness, ramp + "
                          "noise; stride-6 lattice (2,456,500 contours), 512 samples, 100 iterations"),
    "small-3d": dict(ndim=3, stride=4.0, N=256, T=50, seed=0,
                     desc="64x64x32 uint8, 20 balls r 4-6, noise 15; stride-4 lattice (2048 contours), 256 samples, "
                          "50 iterations"),
    "batch-3d": dict(ndim=3, stride=4.0, N=256, T=80, seed=3, count=64,
                     desc="64 uint8 volumes 64^3..512x512x128 (log-uniform voxel count), 1 nucleus per 2000 voxels, "
                          "r 3-8; stride-4 lattices; one autotuned plan over all volumes replayed as a CUDA graph; "
                          "256 samples, 80 iterations"),
    "serve-3d": dict(ndim=3, stride=6.0, N=512, T=100, seed=4, tiles=8, requests=32, load=0.7, ipr=10,
                     budget_gb=120, contour_cap=262144, bound_budget_gb=0.4,
                     desc="request loop over uint16 tiles 128^3..1024x1024x64 (log-uniform voxel count, brain-3d "
                          "nucleus model, 8 distinct tiles cycled with distinct Philox streams), 32 requests; "
                          "saturated (all submitted at once) and Poisson arrivals at 0.7x the saturated rate; "
                          "HBM budget 120 GB, at most 262,144 resident contours, 10 iterations per round (up "
                          "to 8x for small tiles); 512 samples, 100 iterations; also saturated under a 0.4 GB "
                          "budget without the contour cap"),
}


def make_input(name: str, seed: int, dtype: str, size: int = 0):
    from paper_1804_06304_gb300 import synth
    if name == "large-2d":
        side = size or 4096
        s = synth.large_2d(seed, shape=(side, side), n_nuclei=int(round(12_000 * side * side / 4096**2)))
    elif name in ("batch-3d", "serve-3d"):
        raise ValueError(f"{name} has no single input")
    elif name == "brain-3d":
        side = size or 1024
        s = synth.brain_3d(seed, shape=(side, side, side // 4), n_nuclei=int(round(100_000 * (side / 1024) ** 3)),
                           with_f16=(dtype == "f16"))
    else:
        s = synth.small_3d(seed)
    vol = s.volume_f16 if dtype == "f16" else s.volume
    return s, np.ascontiguousarray(vol)


def lattice_count(shape_xyz, spacing, stride, ndim):
    c = 1
    for d in range(ndim):
        c *= max(1, int(math.floor(shape_xyz[d] * spacing[d] / stride)))
    return c


# ------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        self.out = None
        self.uuid = uuid

    def start(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [l.strip().split(",") for l in self.out.read().splitlines() if l.strip()]
        os.unlink(self.out.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------ oracle leg
def oracle_sample(s, vol, wl, spacing, seconds: float, rng_seed: int = 0, threads: int = 0, seed: int = 7,
                  states: bool = False):
    """Time the FP64 oracle (all host cores, or `threads`) on a random subset of the
    workload's contours, sized to take about `seconds`, with Philox key `seed`;
    returns (samples/s, threads, sample text), and with ``states`` also the contour
    indices of the subset and the oracle's final cR (m x 4) and E (m,)."""
    from oracle import oracle
    ndim = wl["ndim"]
    seeds = oracle.seed_lattice(ndim, s.shape_xyz, spacing, wl["stride"])
    R0 = seeds[0, 3]
    op = oracle.make_params(ndim, wl["N"], wl["T"], eps0=8 * R0 * R0 / s.contrast, dR=1.0,
                            Rmin=max(0.5, 0.5 * R0), Rmax=3 * R0, max_step=0.5, seed=seed)
    img = oracle.VolumeImage(vol, spacing)
    threads = threads or oracle.max_threads()
    rng = np.random.default_rng(rng_seed)
    pilot = min(len(seeds), max(threads * 2, 16))
    idx = rng.choice(len(seeds), pilot, replace=False)
    t0 = time.perf_counter()
    oracle.evolve(img, op, seeds[idx], ids=idx, nthreads=threads)
    dt = time.perf_counter() - t0
    per = dt / pilot
    m = int(min(len(seeds), max(pilot, seconds / max(per, 1e-9))))
    idx = rng.choice(len(seeds), m, replace=False)
    t0 = time.perf_counter()
    cR, E, _ = oracle.evolve(img, op, seeds[idx], ids=idx, nthreads=threads)
    dt = time.perf_counter() - t0
    samples = m * wl["N"] * wl["T"]
    desc = f"{m} of {len(seeds)} contours (random, seed {rng_seed}), all {wl['T']} iterations"
    if states:
        return samples / dt, threads, desc, idx, cR, E
    return samples / dt, threads, desc


def oracle_params_of(oracle, ndim: int, p):
    """The oracle's parameters for the library's evolve parameters ``p``, every real
    rounded to FP32 as the library receives it, so that both sides start from the
    same numbers."""
    f = lambda x: float(np.float32(x))  # noqa: E731
    return oracle.make_params(ndim, p.N, p.T, eps0=f(p.eps0), dR=f(p.dR), Rmin=f(p.Rmin), Rmax=f(p.Rmax),
                              max_step=f(p.max_step), seed=p.seed, stream_id=p.stream_id)


def lattice_shape(shape_xyz, spacing, stride, ndim):
    return [max(1, int(math.floor(shape_xyz[d] * spacing[d] / stride))) for d in range(ndim)]


def window_ids(L, m: int) -> np.ndarray:
    """Contour indices (x fastest, as the lattice numbers them) of a centred box of
    about ``m`` lattice cells."""
    ndim = len(L)
    side = max(1, int(round(m ** (1.0 / ndim))))
    ranges = []
    for d in range(ndim):
        w = min(L[d], side)
        lo = (L[d] - w) // 2
        ranges.append(np.arange(lo, lo + w, dtype=np.int64))
    k = np.zeros([len(r) for r in ranges], np.int64)
    mul = 1
    for d in range(ndim):
        shape = [1] * ndim
        shape[d] = len(ranges[d])
        k = k + ranges[d].reshape(shape) * mul
        mul *= L[d]
    return np.sort(k.ravel())


def oracle_window(s, vol, wl, spacing, init_state, p, seconds: float, threads: int = 0):
    """The FP64 oracle on every contour of a centred window of the lattice, sized to
    take about ``seconds`` on ``threads`` host threads (all by default), started from
    the GPU run's own initial FP32 state with its FP32 parameters and Philox key.
    Returns (samples/s, threads, sample text, window ids, final cR (m x 4), E (m,))."""
    from oracle import oracle
    ndim = wl["ndim"]
    L = lattice_shape(s.shape_xyz, spacing, wl["stride"], ndim)
    op = oracle_params_of(oracle, ndim, p)
    img = oracle.VolumeImage(vol, tuple(float(np.float32(v)) for v in spacing))
    threads = threads or oracle.max_threads()
    seeds = init_state[:4].T.astype(np.float64)
    pilot = window_ids(L, max(threads * 8, 64))
    t0 = time.perf_counter()
    oracle.evolve(img, op, seeds[pilot], ids=pilot, nthreads=threads)
    per = (time.perf_counter() - t0) / len(pilot)
    ids = window_ids(L, int(max(len(pilot), seconds / max(per, 1e-9))))
    t0 = time.perf_counter()
    cR, E, _ = oracle.evolve(img, op, seeds[ids], ids=ids, nthreads=threads)
    dt = time.perf_counter() - t0
    box = "x".join(str(len(np.unique((ids // int(np.prod(L[:d]))) % L[d]))) for d in range(ndim))
    desc = (f"every contour of a centred {box} window of the {'x'.join(map(str, L))} lattice ({len(ids)} of "
            f"{int(np.prod(L))}), all {wl['T']} iterations")
    return len(ids) * wl["N"] * wl["T"] / dt, threads, desc, ids, cR, E


def match_points(a: np.ndarray, b: np.ndarray, tol: float) -> int:
    """One-to-one greedy matching of two point sets within ``tol``, closest pairs
    first; returns the number of matched pairs."""
    if len(a) == 0 or len(b) == 0:
        return 0
    from scipy.spatial import cKDTree
    pairs = cKDTree(a).query_ball_tree(cKDTree(b), tol)
    cand = [(float(np.linalg.norm(a[i] - b[j])), i, j) for i, js in enumerate(pairs) for j in js]
    cand.sort()
    ua, ub, m = set(), set(), 0
    for _, i, j in cand:
        if i not in ua and j not in ub:
            ua.add(i)
            ub.add(j)
            m += 1
    return m


def window_cells(ac, V, gpu_state: np.ndarray, idx: np.ndarray, E0: float) -> np.ndarray:
    """The library's localization (ac_localize) of the window's contours alone, with
    the GPU run's final states: the cells the oracle's localization is compared with."""
    sub = ac.ac_seed(V, explicit=np.ascontiguousarray(gpu_state[:4, idx].T))
    ac.ac_set_state(sub, np.ascontiguousarray(gpu_state[:, idx]))
    return ac.ac_localize(sub, float(np.float32(E0)))


def oracle_check(gpu_state: np.ndarray, idx: np.ndarray, cR: np.ndarray, E: np.ndarray, spacing, ndim: int,
                 E0: float = 0.0, gpu_cells=None) -> dict:
    """Final states of the FP32 GPU run against the FP64 oracle's on the oracle's
    contours, both free-running from the same FP32 seeds, parameters and Philox
    streams: centre error in voxels (the 0.25-voxel bar), over all contours and over
    the converged ones (oracle energy below E0), radius and energy errors; with
    ``gpu_cells`` (the library's localization of the same contours, centres in
    physical units) also the detection-set agreement 2 |matched| / (|D_gpu| +
    |D_oracle|) against the oracle's own overlap competition (one-to-one matches
    within 0.5 voxel)."""
    g = gpu_state[:, idx].astype(np.float64)
    sp = np.asarray(spacing[:ndim], np.float64)
    dc = np.linalg.norm((g[:ndim].T - cR[:, :ndim]) / sp, axis=1)
    dR = np.abs(g[3] - cR[:, 3])
    dE = np.abs(g[4] - E)
    conv = E < E0
    out = {"contours": int(len(idx)), "centre_err_voxels": {"median": float(np.median(dc)),
                                                            "p99": float(np.quantile(dc, 0.99)),
                                                            "max": float(dc.max())},
           "frac_centre_within_0.25_voxel": float(np.mean(dc <= 0.25)),
           "converged": {"contours": int(np.sum(conv)),
                         "frac_centre_within_0.25_voxel": float(np.mean(dc[conv] <= 0.25)) if np.any(conv)
                         else None},
           "radius_err_max": float(dR.max()),
           "energy_abs_err_median": float(np.median(dE)), "energy_abs_median": float(np.median(np.abs(E))),
           "note": "free-running final states after all iterations from the same FP32 seeds, FP32 "
                   "parameters and Philox streams; a last-bit difference can send a contour near a saddle "
                   "between touching nuclei, or on background noise, to another end point; per-iteration "
                   "agreement is the teacher-forced parity of the tests"}
    if gpu_cells is not None:
        from oracle import oracle
        ids_o = oracle.localize(ndim, cR, E, float(np.float32(E0)))
        dg = np.asarray(gpu_cells, np.float64).reshape(-1, 3)[:, :ndim] / sp
        do = cR[ids_o, :ndim] / sp
        m = match_points(dg, do, 0.5)
        out["detections"] = {"gpu": int(len(dg)), "oracle": int(len(do)), "matched": int(m),
                             "agreement": 2.0 * m / max(len(dg) + len(do), 1)}
    return out


def oracle_sample_batch(vols, wl, seconds: float, rng_seed: int = 0):
    """The oracle on random volumes of a batch, each through ``oracle_sample``, until
    about `seconds` of evolution have run; returns (samples/s, threads, sample text)."""
    rng = np.random.default_rng(rng_seed)
    samples, spent, picked, threads = 0.0, 0.0, [], 0
    while spent < seconds and len(picked) < 4 * len(vols):
        i = int(rng.integers(len(vols)))
        sv = vols[i]
        t0 = time.perf_counter()
        rate, threads, desc = oracle_sample(sv, sv.volume, wl, sv.spacing, max(0.5, seconds - spent),
                                            rng_seed=int(rng.integers(1 << 30)))
        wall = time.perf_counter() - t0
        m = int(desc.split(" of ")[0])
        samples += m * wl["N"] * wl["T"]
        spent += m * wl["N"] * wl["T"] / rate
        picked.append(f"volume {i}: {desc.split(' (')[0]}")
        if wall > 2 * seconds:
            break
    return samples / spent, threads, "; ".join(picked) + f"; all {wl['T']} iterations"


# ------------------------------------------------------------------------ ranks
def aggregate_ranks(local_ms: list, samples_per_rank: int, world: int, reduce_max=None) -> tuple:
    """Whole-job throughput of independent replicas: each rank's mean step time,
    the maximum over ranks (``reduce_max`` all-reduces a float with MAX; None on a
    single rank), and value = world x samples per rank / that time."""
    t = float(np.mean(local_ms))
    if reduce_max is not None:
        t = reduce_max(t)
    return t, world * samples_per_rank / (t * 1e-3)


def torch_max_reducer(device):
    import torch
    import torch.distributed as dist

    def f(x: float) -> float:
        v = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        return float(v[0])
    return f


def image_config(args, wl, contours: int, world: int) -> dict:
    """The ``config`` of a single-image workload, identical in both arms."""
    rules = {k: v for k, v in (("freeze", args.freeze), ("cull", args.cull)) if v}
    return {"workload": args.workload + (f"@{args.size}" if args.size else ""), "desc": wl["desc"],
            "contours": int(contours), "samples": wl["N"], "iterations": wl["T"], "path": args.path,
            "dtype": args.dtype, "stopping_rules": rules or None,
            "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"}


# ------------------------------------------------------------------------ main
def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="brain-3d", choices=sorted(WORKLOADS))
    ap.add_argument("--dtype", default="native", choices=["native", "f16"])
    ap.add_argument("--path", default="brick", choices=["brick", "plain", "grid"],
                    help="grid: the voxel-grid form of Eq. 5 instead of Monte-Carlo samples")
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--compensated", type=int, default=1)
    ap.add_argument("--brick", type=str, default="0,0,0")
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--halo", type=float, default=0.0, help="halo factor (0 = library default)")
    ap.add_argument("--size", type=int, default=0, help="image side (smaller instances for profiling captures)")
    ap.add_argument("--freeze", type=str, default="", help="TOL,ITERS: convergence freeze rule (off by default)")
    ap.add_argument("--cull", type=str, default="", help="ITER,FRAC: stop contours with E > FRAC x E0 at ITER")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 reference measurement")
    ap.add_argument("--count", type=int, default=0, help="batch-3d: number of volumes (profiling captures)")
    ap.add_argument("--no-forms", action="store_true",
                    help="brain-3d: skip the short batching and serving runs recorded under `forms`")
    args = ap.parse_args(argv)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]
    if args.steps < 1 or args.warmup < 0:
        raise SystemExit("need --steps >= 1 and --warmup >= 0")

    if args.impl == "reference":
        return reference_arm(args, wl, rank, world)

    import torch
    import torch.distributed as dist
    from paper_1804_06304_gb300 import ac

    dist_on = world > 1
    if dist_on:
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.workload == "batch-3d":
        return batch_arm(args, wl, rank, world, dev)
    if args.workload == "serve-3d":
        return serve_arm(args, wl, rank, world, dev)

    s, vol = make_input(args.workload, wl["seed"] + rank, args.dtype, args.size)
    spacing = s.spacing
    ndim = wl["ndim"]
    C_expected = lattice_count(s.shape_xyz, spacing, wl["stride"], ndim)
    vol_dev = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).to(dev)
    vol_pin = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).pin_memory()
    dcode = {np.dtype(np.uint8): ac.AC_U8, np.dtype(np.uint16): ac.AC_U16, np.dtype(np.float16): ac.AC_F16}[vol.dtype]

    V = ac.ac_create_volume(vol_dev, spacing, dtype=dcode)
    C = ac.ac_seed(V, stride=wl["stride"])
    assert C.count == C_expected, (C.count, C_expected)
    init_state = ac.ac_get_state(C)    # the lattice every step re-seeds (the oracle check starts from it)
    R0 = wl["stride"] / math.sqrt(1.5)
    params = ac.default_params(ndim, R0, s.contrast, N=wl["N"], T=wl["T"], seed=1000 + rank,
                               path={"brick": ac.AC_PATH_BRICK, "plain": ac.AC_PATH_PLAIN,
                                     "grid": ac.AC_PATH_GRID}[args.path],
                               lanes_per_contour=args.lanes, compensated=args.compensated,
                               brick=tuple(int(x) for x in args.brick.split(",")), warps_per_block=args.warps,
                               halo_factor=args.halo)
    E0 = ac.default_E0(ndim, s.contrast)
    rules = {}
    if args.freeze:
        tol, its = args.freeze.split(",")
        rules.update(freeze_tol=float(tol), freeze_iters=int(its))
    if args.cull:
        it, frac = args.cull.split(",")
        rules.update(cull_iter=int(it), cull_E=float(frac) * E0)
    params = dataclasses.replace(params, **rules)

    def step(src):
        ac.ac_load_volume(V, src)
        ac.ac_reseed(C)
        ac.ac_evolve(C, params)
        return ac.ac_localize(C, E0)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    for _ in range(args.warmup):
        step(vol_dev)
    torch.cuda.synchronize()
    if dist_on:
        dist.barrier()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    clocks.start()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kernel_ms = []
    launches0 = ac.ac_kernel_launches()
    n_cells = 0
    for i in range(args.steps):
        flush.zero_()                      # L2 flush between timed steps (outside the events)
        ev0[i].record()
        cells = step(vol_dev)
        ev1[i].record()
        kernel_ms.append(ac.ac_evolve_kernel_ms(C))
        n_cells = len(cells)
    from paper_1804_06304_gb300.evaluate import detection_prf
    detection = detection_prf(cells["c"][:, :ndim], s.centres[:, :ndim], s.radii)
    torch.cuda.synchronize()
    launches = ac.ac_kernel_launches() - launches0
    paths = ac.ac_evolve_stats(C)
    final_state = ac.ac_get_state(C) if rank == 0 and not args.no_cpu_baseline else None
    if dist_on:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    # with stopping rules only the evaluated contour-iterations count (the speed-up
    # of stopping shows in voxels/s)
    samples = (int(sum(paths)) if rules else C.count * wl["T"]) * wl["N"]
    reducer = torch_max_reducer(dev) if dist_on else None
    t_ms, value = aggregate_ranks(step_ms, samples, world, reducer)
    k_ms, _ = aggregate_ranks(kernel_ms, samples, world, reducer)

    # end to end through the C ABI from pinned host memory: every step uploads its
    # image and reads its cells back.  Pipelined (the default, as an application
    # would run it): two volume buffers, the next step's upload on a copy stream
    # overlapping this step's evolution; serial: upload, then evolve, in turn.
    e2e = None
    if not args.no_e2e:
        up = torch.cuda.Stream(device=dev, priority=-1)   # its repack kernels get SMs as evolve blocks retire
        V2 = ac.ac_create_volume(vol_dev, spacing, dtype=dcode)
        C2 = ac.ac_seed(V2, stride=wl["stride"])
        vols, ctrs = (V, V2), (C, C2)
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        eclocks = ClockSampler(uuid)
        eclocks.start()
        torch.cuda.synchronize()
        flush.zero_()
        b0.record()
        ac.ac_load_volume(vols[0], vol_pin, stream=up)
        ready[0].record(up)
        e2e_kms = []
        for i in range(args.steps):
            cur = i % 2
            if i + 1 < args.steps:      # the other buffer's last user (step i - 1) has finished
                ac.ac_load_volume(vols[1 - cur], vol_pin, stream=up)
                ready[1 - cur].record(up)
            torch.cuda.current_stream().wait_event(ready[cur])
            ac.ac_reseed(ctrs[cur])
            ac.ac_evolve(ctrs[cur], params)
            cells = ac.ac_localize(ctrs[cur], E0)
            e2e_kms.append(ac.ac_evolve_kernel_ms(ctrs[cur]))
        b1.record()
        b1.synchronize()
        eclk = eclocks.stop()
        pipe_ms = b0.elapsed_time(b1) / args.steps
        e_ms, e_val = aggregate_ranks([pipe_ms], samples, world, reducer)
        # serial, for comparison: each step's upload before its evolution
        ser_ms = []
        for i in range(max(3, min(args.steps, 5))):
            flush.zero_()
            b0.record()
            step(vol_pin)
            b1.record()
            b1.synchronize()
            ser_ms.append(b0.elapsed_time(b1))
        s_ms, s_val = aggregate_ranks(ser_ms, samples, world, reducer)
        e2e = {"value": e_val, "unit": "samples/s", "ms_per_step": e_ms,
               "h2d_bytes_per_step": int(vol.nbytes), "d2h_bytes_per_step": int(len(cells) * 24 + 4 * 6),
               "evolve_kernel_ms": float(np.mean(e2e_kms)), "clocks": eclk,
               "mode": "pipelined: two volume buffers, the next step's host-to-device upload on a copy stream "
                       "during this step's evolution; every step's upload and cell read-back inside the timed region",
               "serial": {"value": s_val, "ms_per_step": s_ms}}

    achieved = ALG_SLOTS_PER_SAMPLE[ndim] * samples / (k_ms * 1e-3) / 1e12
    peak = SM_COUNT * LANES_PER_SM_CLOCK * SM_MAX_MHZ * 1e6 / 1e12
    traffic, traffic_src = DRAM_BYTES_PER_LAUNCH.get((args.workload, args.path, args.size, args.dtype), (None, None))
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tslot/s", "frac": achieved / peak,
            "frac_current_formulation": ALG_SLOTS_CURRENT[ndim] * samples / (k_ms * 1e-3) / 1e12 / peak,
            "traffic": traffic,
            "traffic_note": None if traffic is None else "DRAM bytes per evolve launch: " + traffic_src,
            "kernel": "evolve_brick_kernel" if args.path == "brick" else "evolve_plain_kernel",
            "kernel_ms": k_ms, "alg_slots_per_sample": ALG_SLOTS_PER_SAMPLE[ndim],
            "alg_slots_per_sample_current": ALG_SLOTS_CURRENT[ndim],
            "peak_basis": f"{SM_COUNT} SMs x {LANES_PER_SM_CLOCK} lanes x {SM_MAX_MHZ:.0f} MHz (max SM clock)"}

    # the other roofs the path touches: HBM (the volume and the contour state per
    # launch, measured copy bandwidth) and the shared-memory gathers (2D: one 8- or
    # 16-byte quad per sample; 3D: eight taps), each as a fraction of its peak
    other = None
    if args.path != "grid":
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        hbm_alg = vol.nbytes + C.count * 20 * 2   # volume read once, state read and written
        tap = 8 if (ndim == 2 and vol.dtype.itemsize <= 2 and vol.dtype != np.uint16) else \
            16 if ndim == 2 else 8 * vol.dtype.itemsize
        smem_peak = SM_COUNT * 128 * SM_MAX_MHZ * 1e6 / 1e9   # 32 banks x 4 B per clock per SM, GB/s
        gb = tap * samples / (k_ms * 1e-3) / 1e9
        other = {"hbm": {"achieved": hbm_alg / (k_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                         "frac": hbm_alg / (k_ms * 1e-3) / 1e9 / hbm_peak,
                         "note": "algorithmic bytes: volume once + contour state in and out, per evolve launch"},
                 "smem_gather": {"achieved": gb, "peak": smem_peak, "unit": "GB/s", "frac": gb / smem_peak,
                                 "bytes_per_sample": tap}}

    # the reference point the metric names: the plain FP32 path (one launch per
    # iteration, global gathers, plain FP32 sums) on the same workload
    plain = None
    if args.path == "brick" and not args.no_plain and not rules:
        pp = dataclasses.replace(params, path=ac.AC_PATH_PLAIN, compensated=0, lanes_per_contour=0,
                                 warps_per_block=0, brick=(0, 0, 0))
        ac.ac_reseed(C)
        ac.ac_evolve(C, pp)
        torch.cuda.synchronize()
        pms = []
        for _ in range(max(3, min(args.steps, 5))):
            flush.zero_()
            ac.ac_reseed(C)
            ac.ac_evolve(C, pp)
            pms.append(ac.ac_evolve_kernel_ms(C))
        p_ms, p_val = aggregate_ranks(pms, samples, world, reducer)
        plain = {"value": p_val, "unit": "samples/s", "kernel_ms": p_ms,
                 "speedup": (world * samples / (k_ms * 1e-3)) / p_val,
                 "note": "evolve kernels only, both arms; plain path with plain FP32 sums"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.path != "grid":
        v, thr, desc, idx, o_cR, o_E = oracle_window(s, vol, wl, spacing, init_state, params, args.cpu_seconds)
        v1, _, desc1 = oracle_sample(s, vol, wl, spacing, min(3.0, args.cpu_seconds), rng_seed=1, threads=1)
        cpu = {"value": v, "unit": "samples/s", "cores": thr, "kind": "oracle", "sample": desc,
               "one_thread": {"value": v1, "sample": desc1}}
        if not rules:
            cells_w = window_cells(ac, V, final_state, idx, E0)
            cpu["oracle_check"] = oracle_check(final_state, idx, o_cR, o_E, spacing, ndim, E0, cells_w["c"])
    citers = C.count * wl["T"]

    if rank == 0 and args.path == "grid":
        # the grid form has no samples: throughput in contour-iterations
        _, gval = aggregate_ranks(step_ms, citers, world, reducer)
        print(json.dumps({
            "metric": "contour-iterations/s (voxel-grid form of Eq. 5; whole path: ingest, seed, evolve, localize)",
            "value": gval, "unit": "contour-iterations/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 arithmetic on " + str(vol.dtype) + " voxels", "data": "synthetic",
            "config": {"workload": args.workload + (f"@{args.size}" if args.size else ""), "desc": wl["desc"],
                       "contours": C.count, "iterations": wl["T"], "path": "grid",
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "contour_iterations_per_s": gval, "evolve_kernel_ms": k_ms,
            "evolve_contour_iterations_per_s": world * citers / (k_ms * 1e-3), "cells": n_cells,
            "detection": detection,
            "gpu_launches": int(launches), "roofline": None, "cpu_baseline": None,
            "e2e": None if e2e is None else dict(e2e, value=e2e["value"] / wl["N"], unit="contour-iterations/s"),
            "clocks": clk}))
    elif rank == 0:
        line = {
            "metric": "MC contour samples/s (whole path: ingest, seed, evolve, localize)",
            "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "step_ms": {"median": float(np.median(step_ms)), "p99": float(np.percentile(step_ms, 99)),
                        "min": float(np.min(step_ms)), "max": float(np.max(step_ms))},
            "dtype": "f32 arithmetic on " + str(vol.dtype) + " voxels", "data": "synthetic",
            "config": image_config(args, wl, C.count, world),
            "voxels_per_s": world * int(np.prod(vol.shape)) / (t_ms * 1e-3),
            "evolve_samples_per_s": world * samples / (k_ms * 1e-3),
            "contour_iterations_per_s": world * citers / (t_ms * 1e-3),
            "evaluated_contour_iterations": int(sum(paths)),
            "stopped": dict(zip(("freeze", "cull"), ac.ac_evolve_stops(C))) if rules else None,
            "cells": n_cells,
            "detection": detection,
            "gather_paths": {"fast": paths[0], "clamped": paths[1], "global": paths[2]},
            "gpu_launches": int(launches),
            "roofline": roof, "other_roofs": other, "vs_plain_fp32": plain,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
        }
        if args.workload == "brain-3d" and world == 1 and not args.no_forms and not args.size:
            line["forms"] = run_forms()
        print(json.dumps(line))
    if dist_on:
        dist.destroy_process_group()


def run_forms(timeout_s: float = 900.0) -> dict:
    """The batching and serving forms, each run briefly in a child process of this
    script after the timed steps (batch-3d: 3 warm-up and 3 timed steps; serve-3d:
    its 32 requests saturated, under Poisson arrivals and under a binding HBM
    budget; no CPU baseline), summarized for the default bench line."""
    out = {}
    for name, extra in (("batch-3d", ["--steps", "3", "--warmup", "3"]), ("serve-3d", [])):
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", name, "--no-cpu-baseline", *extra]
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
            d = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
        except (subprocess.TimeoutExpired, OSError, ValueError, IndexError) as e:
            r, d = None, None
            out[name] = {"error": type(e).__name__}
            continue
        if d is None:
            out[name] = {"error": f"exit {r.returncode}: " + r.stderr.strip()[-300:]}
            continue
        try:
            out[name] = _form_summary(name, extra, d)
        except (KeyError, TypeError) as e:   # a side run never takes the headline line down with it
            out[name] = {"error": f"unexpected output ({type(e).__name__}: {e})"}
    return out


def _form_summary(name: str, extra: list, d: dict) -> dict:
    f = {"command": " ".join(["python bench.py", "--workload", name, "--no-cpu-baseline", *extra]),
         "value": d["value"], "unit": d["unit"], "ms_per_step": d["ms_per_step"], "steps": d["steps"],
         "e2e": {k: (d.get("e2e") or {}).get(k) for k in ("value", "ms_per_step")},
         "roofline_frac": d["roofline"]["frac"], "gpu_launches": d.get("gpu_launches"), "clocks": d.get("clocks"),
         "autotuned": d["config"].get("autotuned")}
    if name == "batch-3d":
        f["evolve_kernel_ms"] = d["roofline"].get("kernel_ms")
        f["detection_f"] = (d.get("detection") or {}).get("f")
    else:
        sv = d["serving"]
        f["latency_ms"] = {"saturated_p50": sv["saturated_latency_ms_p50"], "poisson_p50": sv["latency_ms_p50"],
                           "poisson_p99": sv["latency_ms_p99"], "poisson_lambda_hz": sv["poisson_lambda_hz"]}
        f["saturated_tiles_per_s"] = sv["saturated_tiles_per_s"]
        f["budget_bound"] = sv.get("budget_bound_saturated")
    return f


def batch_arm(args, wl, rank, world, dev):
    """Batching form: every step re-seeds the 64 volumes' lattices, replays one
    CUDA graph holding the binning, sort and single evolution launch over all of
    them, and localizes each volume."""
    import torch
    import torch.distributed as dist
    from paper_1804_06304_gb300 import ac, synth

    dist_on = world > 1
    vols = synth.batch_3d(wl["seed"] + rank, count=args.count or wl["count"])
    V, C = [], []
    pinned = []
    for sv in vols:
        V.append(ac.ac_create_volume(sv.volume, sv.spacing))
        C.append(ac.ac_seed(V[-1], stride=wl["stride"]))
        pinned.append(torch.from_numpy(sv.volume).pin_memory())
    R0 = wl["stride"] / math.sqrt(1.5)
    params = ac.default_params(3, R0, 170.0, N=wl["N"], T=wl["T"], seed=1000 + rank, compensated=args.compensated)
    t0 = time.perf_counter()
    fixed = tuple(int(x) for x in args.brick.split(","))
    if args.lanes or args.warps or any(fixed):   # an explicit configuration skips the autotuner
        params = dataclasses.replace(params, lanes_per_contour=args.lanes, warps_per_block=args.warps, brick=fixed)
    else:
        params = ac.ac_autotune(C, params)
    tune_s = time.perf_counter() - t0
    items = [(i, 1, wl["T"], 0) for i in range(len(C))]
    plan = ac.ac_plan_create(C, params, items=items)
    E0 = ac.default_E0(3, 170.0)
    total = sum(c.count for c in C)
    samples = total * wl["N"] * wl["T"]

    def step(from_host=False, keep=None):
        if from_host:
            for v, src in zip(V, pinned):
                ac.ac_load_volume(v, src)
        for c in C:
            ac.ac_reseed(c)
        ac.ac_plan_launch(plan, use_graph=True)
        cells = ac.ac_localize_batch(C, E0)   # every set in one pass
        if keep is not None:
            keep.extend(cells)
        return sum(len(c) for c in cells)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist_on:
        dist.barrier()
    clocks = ClockSampler(None)
    clocks.start()
    ms, kms = [], []
    launches0 = ac.ac_kernel_launches()
    cells = 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        cells = step()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        kms.append(ac.ac_evolve_kernel_ms(C[0]))
    launches = ac.ac_kernel_launches() - launches0
    torch.cuda.synchronize()
    if dist_on:
        dist.barrier()
    clk = clocks.stop()
    reducer = torch_max_reducer(dev) if dist_on else None
    t_ms, value = aggregate_ranks(ms, samples, world, reducer)
    k_ms, _ = aggregate_ranks(kms, samples, world, reducer)
    from paper_1804_06304_gb300.evaluate import match_inside
    kept = []
    step(keep=kept)
    tp = sum(match_inside(c["c"], sv.centres, sv.radii) for c, sv in zip(kept, vols))
    n_det, n_true = sum(len(c) for c in kept), sum(len(sv.centres) for sv in vols)
    pr, rc = tp / max(n_det, 1), tp / max(n_true, 1)
    detection = {"tp": tp, "fp": n_det - tp, "fn": n_true - tp, "precision": pr, "recall": rc,
                 "f": 2 * pr * rc / (pr + rc) if pr + rc > 0 else 0.0}
    e2e = None
    if not args.no_e2e:
        # end to end from pinned host memory, pipelined as an application would run
        # it: a second set of volumes, contours and plan, the next step's 64 uploads
        # on a copy stream during this step's evolution; every step's uploads and
        # cell read-back inside the timed region.  Serial (upload, then evolve) for
        # comparison.
        up = torch.cuda.Stream(device=dev, priority=-1)   # its repack kernels get SMs as evolve blocks retire
        V2 = [ac.ac_create_volume(sv.volume, sv.spacing) for sv in vols]
        C2 = [ac.ac_seed(v, stride=wl["stride"]) for v in V2]
        plan2 = ac.ac_plan_create(C2, params, items=items)
        bufs = ((V, C, plan), (V2, C2, plan2))
        ready = [torch.cuda.Event(), torch.cuda.Event()]

        def upload(vs):
            for v, src in zip(vs, pinned):
                ac.ac_load_volume(v, src, stream=up)

        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ac.ac_plan_launch(plan2, use_graph=True)   # capture the second plan's graph, fill the staging buffers
        upload(V)
        upload(V2)
        torch.cuda.synchronize()
        flush.zero_()
        b0.record()
        upload(bufs[0][0])
        ready[0].record(up)
        for i in range(args.steps):
            cur = i % 2
            if i + 1 < args.steps:
                upload(bufs[1 - cur][0])
                ready[1 - cur].record(up)
            torch.cuda.current_stream().wait_event(ready[cur])
            for c in bufs[cur][1]:
                ac.ac_reseed(c)
            ac.ac_plan_launch(bufs[cur][2], use_graph=True)
            ecells = ac.ac_localize_batch(bufs[cur][1], E0)
        b1.record()
        b1.synchronize()
        e_ms, e_val = aggregate_ranks([b0.elapsed_time(b1) / args.steps], samples, world, reducer)
        ems = []
        for _ in range(max(3, min(args.steps, 5))):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step(from_host=True)
            e1.record()
            e1.synchronize()
            ems.append(e0.elapsed_time(e1))
        s_ms, s_val = aggregate_ranks(ems, samples, world, reducer)
        e2e = {"value": e_val, "unit": "samples/s", "ms_per_step": e_ms,
               "h2d_bytes_per_step": int(sum(sv.volume.nbytes for sv in vols)),
               "d2h_bytes_per_step": int(sum(len(c) for c in ecells) * 24 + len(C) * 24),
               "mode": "pipelined: two sets of volumes, contours and plans, the next step's uploads on a copy "
                       "stream during this step's evolution; every step's uploads and cell read-back inside "
                       "the timed region",
               "serial": {"value": s_val, "ms_per_step": s_ms}}
    paths = ac.ac_evolve_stats(C[0])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, thr, desc = oracle_sample_batch(vols, wl, args.cpu_seconds)
        cpu = {"value": v, "unit": "samples/s", "cores": thr, "kind": "oracle", "sample": desc}
    achieved = ALG_SLOTS_PER_SAMPLE[3] * samples / (k_ms * 1e-3) / 1e12
    peak = SM_COUNT * LANES_PER_SM_CLOCK * SM_MAX_MHZ * 1e6 / 1e12
    if rank == 0:
        print(json.dumps({
            "metric": "MC contour samples/s (whole path: seed, evolve, localize; batching form)",
            "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 arithmetic on uint8 voxels", "data": "synthetic",
            "config": {"workload": "batch-3d", "desc": wl["desc"], "volumes": len(C), "contours": total,
                       "voxels": int(sum(sv.volume.size for sv in vols)), "samples": wl["N"], "iterations": wl["T"],
                       "autotuned": {"lanes_per_contour": params.lanes_per_contour, "brick": list(params.brick),
                                     "warps_per_block": params.warps_per_block, "seconds": tune_s},
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "cells": cells, "detection": detection,
            "gather_paths": {"fast": paths[0], "clamped": paths[1], "global": paths[2]},
            "gpu_launches": int(launches),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tslot/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "evolve_brick_kernel (plan, graph)",
                         "kernel_ms": k_ms, "alg_slots_per_sample": ALG_SLOTS_PER_SAMPLE[3]},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk}))
    if dist_on:
        dist.destroy_process_group()


def serve_arm(args, wl, rank, world, dev):
    """Serving form: tiles submitted to the library's request loop (ac_server_*),
    first all at once (saturated throughput), then as Poisson arrivals at a fraction
    of that rate (tile latency p50 / p99, host clock from submit to cells ready).
    Tiles come from pinned host memory, so every request includes its upload."""
    import torch
    import torch.distributed as dist
    from paper_1804_06304_gb300 import ac, synth

    dist_on = world > 1
    tiles = [t for _, t in synth.tile_stream(wl["seed"] + rank, count=wl["tiles"])]
    pinned = [torch.from_numpy(t.volume).pin_memory().numpy() for t in tiles]
    R0 = wl["stride"] / math.sqrt(1.5)
    contrast = tiles[0].contrast
    params = ac.default_params(3, R0, contrast, N=wl["N"], T=wl["T"], seed=2000 + rank,
                               compensated=args.compensated)
    # brick shape and lane grouping tuned once on two tiles of the stream
    probe = [ac.ac_seed(ac.ac_create_volume(pinned[i], tiles[i].spacing), stride=wl["stride"]) for i in (0, 1)]
    params = ac.ac_autotune(probe, params)
    del probe
    E0 = ac.default_E0(3, contrast)
    n_req = wl["requests"]

    def contours(t):
        return int(np.prod([max(1, int(math.floor(n * sp / wl["stride"]))) for n, sp in
                            zip(t.shape_xyz, t.spacing)]))

    def run(arrivals, cap=wl["contour_cap"], balance=True, budget_gb=wl["budget_gb"]):
        srv = ac.Server(params, ac.AC_U16, 3, wl["stride"], E0, hbm_budget_bytes=int(budget_gb * 1e9),
                        iters_per_round=wl["ipr"], max_resident_contours=cap, balance_rounds=balance)
        t0 = time.perf_counter()
        tickets = []
        for i, a in enumerate(arrivals):
            delay = t0 + a - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            j = i % len(tiles)
            tickets.append((j, srv.submit(pinned[j], tiles[j].spacing, stream_id=i)))
        res = [srv.wait(tk, timeout=600)[1] for _, tk in tickets]
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        samples = sum(contours(tiles[j]) for j, _ in tickets) * wl["N"] * wl["T"]
        voxels = sum(tiles[j].volume.size for j, _ in tickets)
        return wall, samples, voxels, res, st

    run([0.0] * max(args.warmup, 1))                      # warm-up requests
    torch.cuda.synchronize()
    if dist_on:
        dist.barrier()
    clocks = ClockSampler(None)
    clocks.start()
    launches0 = ac.ac_kernel_launches()
    wall, samples, voxels, res_sat, st_sat = run([0.0] * n_req)
    launches = ac.ac_kernel_launches() - launches0
    rate = n_req / wall
    lam = wl["load"] * rate
    rng = np.random.default_rng(wl["seed"])
    arrivals = list(np.cumsum(rng.exponential(1.0 / lam, size=n_req)) - 0.0)
    arrivals = [a - arrivals[0] for a in arrivals]
    wall_p, samples_p, voxels_p, res_p, st_p = run(arrivals)
    clk = clocks.stop()
    # the same saturated stream without the contour cap: every tile resident at once
    wall_u, samples_u, _, res_u, _ = run([0.0] * n_req, cap=0)
    lat_u = np.array([r["total_ms"] for r in res_u])
    # the same Poisson stream with every tile advancing iters_per_round per round
    _, _, _, res_nb, _ = run(arrivals, balance=False)
    lat_nb = np.array([r["total_ms"] for r in res_nb])
    # the saturated stream under a budget below its working set (no contour cap):
    # admission by device bytes alone
    wall_b, samples_b, _, res_b, st_b = run([0.0] * n_req, cap=0, budget_gb=wl["bound_budget_gb"])
    lat_b = np.array([r["total_ms"] for r in res_b])
    reducer = torch_max_reducer(dev) if dist_on else None
    t_ms, value = aggregate_ranks([wall * 1e3], samples, world, reducer)
    lat = np.array([r["total_ms"] for r in res_p])
    lat_sat = np.array([r["total_ms"] for r in res_sat])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, thr, desc = oracle_sample_batch(tiles, wl, args.cpu_seconds)
        cpu = {"value": v, "unit": "samples/s", "cores": thr, "kind": "oracle", "sample": desc}
    achieved = ALG_SLOTS_PER_SAMPLE[3] * samples / wall / 1e12
    peak = SM_COUNT * LANES_PER_SM_CLOCK * SM_MAX_MHZ * 1e6 / 1e12
    if rank == 0:
        print(json.dumps({
            "metric": "MC contour samples/s (serving form: upload, seed, evolve, localize per tile)",
            "value": value, "unit": "samples/s", "n_gpus": world, "steps": n_req, "warmup": max(args.warmup, 1),
            "ms_per_step": t_ms / n_req, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 arithmetic on uint16 voxels", "data": "synthetic",
            "config": {"workload": "serve-3d", "desc": wl["desc"], "requests": n_req,
                       "autotuned": {"lanes_per_contour": params.lanes_per_contour, "brick": list(params.brick),
                                     "warps_per_block": params.warps_per_block},
                       "timing": "host clock around the request loop (submit to the last cells)",
                       "l2": "inputs larger than L2 in total; each request uploads its tile",
                       "parallelism": f"replicas x{world}"},
            "voxels_per_s": voxels / wall,
            "serving": {"saturated_tiles_per_s": rate, "saturated_latency_ms_p50": float(np.median(lat_sat)),
                        "poisson_lambda_hz": lam, "poisson_tiles_per_s": n_req / wall_p,
                        "poisson_voxels_per_s": voxels_p / wall_p, "poisson_samples_per_s": samples_p / wall_p,
                        "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
                        "queue_ms_p50": float(np.median([r["queue_ms"] for r in res_p])),
                        "rounds_saturated": st_sat["rounds"], "rounds_poisson": st_p["rounds"],
                        "peak_resident_gb": st_sat["peak_resident_bytes"] / 1e9,
                        "poisson_unbalanced_rounds": {"latency_ms_p50": float(np.percentile(lat_nb, 50)),
                                                      "latency_ms_p99": float(np.percentile(lat_nb, 99))},
                        "uncapped_saturated": {"samples_per_s": samples_u / wall_u,
                                               "latency_ms_p50": float(np.percentile(lat_u, 50)),
                                               "latency_ms_p99": float(np.percentile(lat_u, 99))},
                        "budget_bound_saturated": {"budget_gb": wl["bound_budget_gb"],
                                                   "peak_resident_gb": st_b["peak_resident_bytes"] / 1e9,
                                                   "working_set_gb": sum(r["est_bytes"] for r in res_b) / 1e9,
                                                   "samples_per_s": samples_b / wall_b,
                                                   "latency_ms_p50": float(np.percentile(lat_b, 50)),
                                                   "latency_ms_p99": float(np.percentile(lat_b, 99))}},
            "gpu_launches": int(launches),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tslot/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "whole request loop (host clock; uploads, seeding and localization included)",
                         "alg_slots_per_sample": ALG_SLOTS_PER_SAMPLE[3]},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "samples/s", "ms_per_step": t_ms / n_req,
                    "h2d_bytes_per_step": int(voxels * 2 / n_req),
                    "d2h_bytes_per_step": int(sum(r["n_cells"] for r in res_sat) * 24 / n_req),
                    "note": "the serving value is end to end: host tiles in, cells out"},
            "clocks": clk}))
    if dist_on:
        dist.destroy_process_group()


def reference_arm(args, wl, rank, world):
    """The FP64 oracle timed on the host cores: each step a bounded random sample of
    the same workload's contours (all iterations)."""
    if rank != 0:
        return
    per_step = max(2.0, min(15.0, 120.0 / max(1, args.steps + args.warmup)))
    if args.workload in ("batch-3d", "serve-3d"):
        from paper_1804_06304_gb300 import synth
        vols = synth.batch_3d(wl["seed"], count=wl["count"]) if args.workload == "batch-3d" else \
            [t for _, t in synth.tile_stream(wl["seed"], count=wl["tiles"])]
        run = lambda seed: oracle_sample_batch(vols, wl, per_step, rng_seed=seed)  # noqa: E731
        C = sum(lattice_count(sv.shape_xyz, sv.spacing, wl["stride"], 3) for sv in vols)
    else:
        s, vol = make_input(args.workload, wl["seed"], args.dtype, args.size)
        run = lambda seed: oracle_sample(s, vol, wl, s.spacing, per_step, rng_seed=seed)  # noqa: E731
        C = lattice_count(s.shape_xyz, s.spacing, wl["stride"], wl["ndim"])
    for i in range(args.warmup):
        run(100 + i)
    vals, thr, desc = [], 0, ""
    t0 = time.perf_counter()
    for i in range(args.steps):
        v, thr, desc = run(i)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": "MC contour samples/s (whole path: ingest, seed, evolve, localize)",
            "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": image_config(args, wl, C, world) if args.workload not in ("batch-3d", "serve-3d") else
            {"workload": args.workload, "desc": wl["desc"], "contours": C, "samples": wl["N"], "iterations": wl["T"]},
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": thr, "kind": "oracle",
                             "sample": f"per step: {desc}"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
