"""Precision form: the brain-like 3D workload stored as uint16, FP16 and FP32, with
compensated and plain FP32 sums, against the FP64 oracle.

For every storage and summation mode a stripe of contours is traced over every
iteration; the oracle re-evaluates each traced state (teacher-forced) and the
errors of E, dE/dR and dE/dc are reported relative to their magnitude sums (see
tests/_parity.py).  Final centres and radii are compared with a free-running oracle
on the same contours.  The report prints one JSON line per case (run pytest with
-s to see it); the assertions are the parity bar for the compensated sums and a
looser bound, stated below, for plain sums.
"""
import json
import math

import numpy as np
import pytest

from tests import _parity as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ac():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06304_gb300 import ac as lib
    lib.load()
    return lib


@pytest.fixture(scope="module")
def brain():
    from paper_1804_06304_gb300 import synth
    # 1/64 of the 1024x1024x256 volume, same spacing and nucleus density
    return synth.brain_3d(2, shape=(256, 256, 64), n_nuclei=1563)


def _normalised_errors(oracle, trace, res, ndim):
    rows = trace.reshape(-1, 9).astype(np.float64)
    mag_e = res[:, oracle.MAG_I]
    mag_r = ndim / rows[:, 3] * mag_e + (res[:, oracle.MAG_R] - ndim / rows[:, 3] * res[:, oracle.MAG_E])
    out = {}
    for name, gc, oc, mag in [("E", 4, oracle.E, mag_e), ("dEdR", 5, oracle.DEDR, mag_r)] + \
            [(f"dEdc{a}", 6 + a, oracle.DEDC + a, res[:, oracle.MAG_G]) for a in range(ndim)]:
        err = np.abs(rows[:, gc] - res[:, oc]) / np.maximum(np.maximum(np.abs(res[:, oc]), mag), 1e-30)
        keep = res[:, oracle.FLAGS] == 0
        out[name] = {"max": float(err[keep].max()), "median": float(np.median(err[keep])),
                     "p99.99": float(np.quantile(err[keep], 0.9999))}
    return out


@pytest.mark.parametrize("storage", ["u16", "f16", "f32"])
@pytest.mark.parametrize("comp", [1, 0])
def test_precision_brain_like(ac, oracle, brain, storage, comp):
    s = brain
    vol = {"u16": s.volume, "f16": s.volume_f16, "f32": s.volume.astype(np.float32)}[storage]
    R0 = 6.0 / math.sqrt(1.5)
    p = ac.default_params(3, R0, s.contrast, N=512, T=20, seed=17, compensated=comp, sampling=2)
    C = 42 * 42 * 21
    k0 = C // 2
    r = P.gpu_run(ac, vol, s.spacing, p, stride=6.0, trace_k=(k0, k0 + 256))
    img = P.oracle_image(oracle, vol, s.spacing)
    op = P.oracle_params(oracle, 3, p)
    frac, nflag, worst, bad, res = P.teacher_forced(oracle, img, op, r["trace"], k0, 1)
    errs = _normalised_errors(oracle, r["trace"], res, 3)
    cR, E, _ = oracle.evolve(img, op, r["init"][:4, k0:k0 + 256].T.astype(np.float64), ids=np.arange(k0, k0 + 256))
    dc = np.linalg.norm(r["final"][:3, k0:k0 + 256].T - cR[:, :3], axis=1)
    dR = np.abs(r["final"][3, k0:k0 + 256] - cR[:, 3])
    report = {"storage": storage, "sums": "compensated" if comp else "plain", "contours": 256, "iterations": 20,
              "samples": 512, "pass_fraction_1e-5": frac, "flagged": nflag, "errors": errs,
              "final_centre_err_max": float(dc.max()), "final_centre_err_median": float(np.median(dc)),
              "final_radius_err_max": float(dR.max())}
    print("PRECISION " + json.dumps(report))
    if comp:
        assert frac >= 0.9999, report
    else:
        # plain FP32 sums of 16 terms per lane and a 32-lane tree: relative error
        # bound about (16 + 5) x 2^-24 of the magnitude, well inside 1e-4
        assert max(v["max"] for v in errs.values()) < 1e-4, report
    assert np.median(dc) < 0.25
