"""Cases that reach every gather of the evolution kernels (shared-memory quads and
raw taps on the fast and clamped paths, global-memory fallback, the plain and grid
paths, tiny volumes with balls far outside, batches, the request loop).  Run once
with the normal build and once with the bounds-checked build (AC_BUILD=checked);
tests/test_gpu_checked.py compares the two.

Usable as a script: ``python -m tests._checked_cases OUT.npz``.
"""
from __future__ import annotations

import dataclasses
import math
import sys

import numpy as np


def run_cases() -> dict:
    from paper_1804_06304_gb300 import ac, synth
    out = {}
    s3 = synth.small_3d(0)
    R3 = 4.0 / math.sqrt(1.5)
    base3 = ac.default_params(3, R3, s3.contrast, N=64, T=8, seed=11)
    for name, kw in [("b3_g32", dict(lanes_per_contour=32)), ("b3_g8", dict(lanes_per_contour=8)),
                     ("plain3", dict(path=ac.AC_PATH_PLAIN)), ("grid3", dict(path=ac.AC_PATH_GRID)),
                     ("b3_rules", dict(freeze_tol=0.05, freeze_iters=2, cull_iter=4, cull_E=-1.0))]:
        V = ac.ac_create_volume(s3.volume, s3.spacing)
        C = ac.ac_seed(V, stride=4.0)
        ac.ac_evolve(C, dataclasses.replace(base3, **kw))
        out[name] = ac.ac_get_state(C)
    # global fallback: radii far beyond the staged halo
    V = ac.ac_create_volume(s3.volume, s3.spacing)
    C = ac.ac_seed(V, stride=4.0, R0=1.0)
    st = ac.ac_get_state(C)
    st[3, ::5] = 7.0
    ac.ac_set_state(C, st)
    ac.ac_evolve(C, dataclasses.replace(base3, Rmin=0.5, Rmax=9.0))
    out["b3_global"] = ac.ac_get_state(C)
    out["b3_global_paths"] = np.array(ac.ac_evolve_stats(C))
    # the full-size brick layouts of a brain-like volume: 8 lanes on 4x4x4-cell bricks in
    # one 16-warp CTA per SM (a 209.7 KB region whose 128-byte rows are padded to 144),
    # and 16 lanes on 4x2x2-cell bricks (padded rows, two CTAs per SM); four and two
    # contours per warp share a gather path
    sb = synth.brain_3d(4, shape=(256, 256, 64), n_nuclei=1563, with_f16=False)
    Rb = 6.0 / math.sqrt(1.5)
    baseb = ac.default_params(3, Rb, sb.contrast, N=512, T=4, seed=13)
    for name, kw in [("brain_g8", dict(lanes_per_contour=8, brick=(24, 24, 12), warps_per_block=16)),
                     ("brain_g16", dict(lanes_per_contour=16, brick=(24, 12, 6)))]:
        V = ac.ac_create_volume(sb.volume, sb.spacing)
        C = ac.ac_seed(V, stride=6.0)
        ac.ac_evolve(C, dataclasses.replace(baseb, **kw))
        out[name] = ac.ac_get_state(C)
        out[name + "_paths"] = np.array(ac.ac_evolve_stats(C))
    # 2D: half-precision quads (u8), float quads (u16, f32)
    s2 = synth.large_2d(1, shape=(256, 256), n_nuclei=47)
    R2 = 6.0 / math.sqrt(1.5)
    base2 = ac.default_params(2, R2, s2.contrast, N=128, T=8, seed=12)
    for name, vol, kw in [("b2_u8_g4", s2.volume, dict(lanes_per_contour=4)),
                          ("b2_u8_g16", s2.volume, dict(lanes_per_contour=16, sampling=1)),
                          ("b2_u16", (s2.volume.astype(np.uint16) * 100), {}),
                          ("b2_f32", s2.volume.astype(np.float32), {}),
                          ("plain2", s2.volume, dict(path=ac.AC_PATH_PLAIN)),
                          ("grid2", s2.volume, dict(path=ac.AC_PATH_GRID))]:
        V = ac.ac_create_volume(vol, s2.spacing)
        C = ac.ac_seed(V, stride=6.0)
        ac.ac_evolve(C, dataclasses.replace(base2, **kw))
        out[name] = ac.ac_get_state(C)
    # tiny volumes, balls far outside
    rng = np.random.default_rng(5)
    t3 = rng.integers(0, 255, size=(2, 2, 3), dtype=np.uint8)
    V = ac.ac_create_volume(t3)
    C = ac.ac_seed(V, explicit=np.array([[1.0, 0.5, 0.5, 2.0], [0.0, 0.0, 1.0, 5.0]], np.float32))
    ac.ac_evolve(C, ac.default_params(3, 2.0, 100.0, N=33, T=5, seed=2))
    out["tiny3"] = ac.ac_get_state(C)
    t2 = rng.integers(0, 255, size=(5, 2), dtype=np.uint8)
    V = ac.ac_create_volume(t2)
    C = ac.ac_seed(V, explicit=np.array([[0.5, 2.0, 0.0, 3.0]], np.float32))
    ac.ac_evolve(C, ac.default_params(2, 3.0, 100.0, N=7, T=5, seed=3))
    out["tiny2"] = ac.ac_get_state(C)
    # batch over two volumes of different sizes
    vols = synth.batch_3d(2, count=2, max_scale=0.2)
    sets = []
    keep = []
    for sv in vols:
        V = ac.ac_create_volume(sv.volume, sv.spacing)
        keep.append(V)
        sets.append(ac.ac_seed(V, stride=4.0))
    ac.ac_evolve_batch(sets, base3, items=[(1, 1, 8, 0), (2, 1, 5, 0)])
    for i, c in enumerate(sets):
        out[f"batch{i}"] = ac.ac_get_state(c)
    # request loop
    srv = ac.Server(base3, ac.AC_U8, 3, 4.0, ac.default_E0(3, s3.contrast), hbm_budget_bytes=1 << 30,
                    iters_per_round=3)
    tickets = [srv.submit(sv.volume, sv.spacing, stream_id=i) for i, sv in enumerate(vols)]
    for i, t in enumerate(tickets):
        cells, _ = srv.wait(t, timeout=300)
        out[f"served{i}"] = np.stack([cells["c"][:, 0], cells["c"][:, 1], cells["c"][:, 2], cells["r"], cells["E"],
                                      cells["id"].astype(np.float32)]) if len(cells) else np.zeros((6, 0), np.float32)
    srv.close()
    return out


if __name__ == "__main__":
    np.savez(sys.argv[1], **run_cases())
