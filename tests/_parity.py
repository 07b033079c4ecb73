"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and
compare with the FP64 oracle on the same seeded inputs.

Tolerance (per-iteration, teacher-forced): |x_gpu - x_oracle| <= 1e-5 *
max(|x_oracle|, M_x), M_x a magnitude sum of the oracle for that quantity, because
a relative error alone is meaningless for background contours whose energy is
zero plus noise.  The magnitudes follow where FP32 errors are absolute rather
than relative:
  E      M = V/N sum |I| / (2R)^d   -- the weight S is a ramp in r, and r carries
         an absolute rounding error, so a sample with S near 0 has an S error of
         order 1e-6 on S's natural scale 1 (the intensity mass bounds it);
  dE/dR  M = d/R * (the E magnitude) + V/N sum |dS/dR I| / (2R)^d;
  dE/dc  M = V/N sum |S'(r)| I / (2R)^d, direction-free, since the error of a
         sample direction is absolute.  Evaluations with a sample
within 1e-5 of a band edge are excluded (FP32 and FP64 may put that sample on
different sides of a kink of S).
"""
from __future__ import annotations

import numpy as np

REL = 1e-5


def oracle_params(oracle, ndim, p, edge_tol=1e-5):
    f = lambda x: float(np.float32(x))
    return oracle.make_params(ndim, p.N, p.T, eps0=f(p.eps0), dR=f(p.dR), Rmin=f(p.Rmin), Rmax=f(p.Rmax),
                              max_step=f(p.max_step), seed=p.seed, stream_id=p.stream_id, edge_tol=edge_tol,
                              integration=1 if p.path == 2 else 0, freeze_tol=f(p.freeze_tol),
                              freeze_iters=p.freeze_iters, cull_iter=p.cull_iter, cull_E=f(p.cull_E))


def oracle_image(oracle, volume, spacing, scale=1.0):
    sp = tuple(float(np.float32(s)) for s in spacing)
    return oracle.VolumeImage(volume, sp, scale=float(np.float32(scale)))


def gpu_run(ac, volume, spacing, params, stride=None, explicit=None, trace_k=None, trace_t=None, scale=1.0,
            device_volume=False):
    import torch
    data = torch.from_numpy(volume).cuda() if device_volume else volume
    V = ac.ac_create_volume(data, spacing, intensity_scale=scale)
    Cn = ac.ac_seed(V, stride=stride, explicit=explicit)
    init = ac.ac_get_state(Cn)
    tr = None
    if trace_k is not None:
        t0, t1 = trace_t if trace_t is not None else (1, params.T + 1)
        k0, k1 = trace_k
        buf = torch.full(((t1 - t0) * (k1 - k0) * 9,), float("nan"), device="cuda", dtype=torch.float32)
        ac.ac_evolve(Cn, params, trace=(buf, k0, k1, t0, t1))
        tr = buf.view(t1 - t0, k1 - k0, 9).cpu().numpy()
    else:
        ac.ac_evolve(Cn, params)
    final = ac.ac_get_state(Cn)
    return {"vol": V, "ctr": Cn, "init": init, "final": final, "trace": tr}


def teacher_forced(oracle, img, op, trace, k0, t0, nthreads=0):
    """Re-evaluate every traced (iteration, contour) with the oracle at the GPU's
    recorded state.  Returns (pass fraction over unflagged rows, number of flagged
    rows, details of failures)."""
    T, K, _ = trace.shape
    rows = trace.reshape(-1, 9).astype(np.float64)
    iters = np.repeat(np.arange(t0, t0 + T), K)
    ks = np.tile(np.arange(k0, k0 + K), T)
    # rows the kernel never wrote (after a contour stopped) stay NaN and are skipped
    valid = ~np.isnan(rows[:, :4]).any(axis=1)
    res = np.full((len(rows), oracle.RES_LEN), np.nan)
    res[valid] = oracle.eval_many(img, op, rows[valid, :4], iters[valid], ks[valid], nthreads=nthreads)
    res[~valid, oracle.FLAGS] = 1.0   # excluded like flagged rows
    ok = np.ones(len(rows), bool)
    d = 3 if op.ndim == 3 else 2
    mag_e = res[:, oracle.MAG_I]
    mag_r = d / rows[:, 3] * mag_e + (res[:, oracle.MAG_R] - d / rows[:, 3] * res[:, oracle.MAG_E])
    pairs = [(4, oracle.E, mag_e), (5, oracle.DEDR, mag_r)]
    pairs += [(6 + a, oracle.DEDC + a, res[:, oracle.MAG_G]) for a in range(3)]
    worst = 0.0
    for gc, oc, mag in pairs:
        tol = REL * np.maximum(np.abs(res[:, oc]), mag) + 1e-30
        err = np.abs(rows[:, gc] - res[:, oc])
        ok &= (err <= tol) | ~valid
        worst = max(worst, float(np.max(np.where((res[:, oracle.FLAGS] > 0) | ~valid, 0, err / tol))))
    flagged = (res[:, oracle.FLAGS] > 0) & valid
    good = ok[~flagged & valid]
    frac = float(good.mean()) if len(good) else 1.0
    bad = np.nonzero(~ok & ~flagged & valid)[0][:10]
    details = [(int(iters[i]), int(ks[i]), rows[i, 4:].tolist(), res[i, [0, 7, 8, 9, 10]].tolist()) for i in bad]
    return frac, int(flagged.sum()), worst, details, res


def match_sets(a, b, tol):
    """One-to-one greedy matching of two point sets within `tol` (closest first)."""
    if len(a) == 0 or len(b) == 0:
        return 0
    d = np.linalg.norm(a[:, None, :] - b[None, :, :], axis=2)
    pairs = np.argwhere(d < tol)
    order = np.argsort(d[pairs[:, 0], pairs[:, 1]])
    ua, ub = set(), set()
    m = 0
    for i, j in pairs[order]:
        if i not in ua and j not in ub:
            ua.add(i)
            ub.add(j)
            m += 1
    return m
