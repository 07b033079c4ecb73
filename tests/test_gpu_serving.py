"""Serving form: tiles of different sizes submitted over time to the request loop
(include/ac_serve.h) give exactly the cells each gives when evolved alone through
ac_create_volume / ac_seed / ac_evolve / ac_localize, whatever tiles share its
rounds, under a tight memory budget, and with one tile that fails."""
import dataclasses
import math
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

STRIDE = 6.0
CONTRAST = 1700.0
T = 20


@pytest.fixture(scope="module")
def ac():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06304_gb300 import ac as lib
    lib.load()
    return lib


@pytest.fixture(scope="module")
def tiles():
    from paper_1804_06304_gb300 import synth
    return [s for _, s in synth.tile_stream(21, count=6, max_scale=0.3)]


def _params(ac):
    return ac.default_params(3, STRIDE / math.sqrt(1.5), CONTRAST, N=128, T=T, seed=5)


def _alone(ac, volume, spacing, params, stream_id):
    V = ac.ac_create_volume(volume, spacing)
    C = ac.ac_seed(V, stride=STRIDE)
    ac.ac_evolve(C, dataclasses.replace(params, stream_id=stream_id))
    return ac.ac_localize(C, ac.default_E0(3, CONTRAST))


def _same_cells(a, b):
    assert len(a) == len(b)
    for f in a.dtype.names:
        np.testing.assert_array_equal(a[f], b[f])


def _est_bytes(volume, elem):
    nz, ny, nx = volume.shape
    pitch = (nx * elem + 15) // 16 * 16
    C = max(1, int(nx // STRIDE)) * max(1, int(ny // STRIDE)) * max(1, int(nz // STRIDE))
    return pitch * ny * nz + 100 * C + (1 << 20)


@pytest.mark.parametrize("balance", [False, True])
def test_alone_equals_mix(ac, tiles, balance):
    p = _params(ac)
    vols = [(t.volume, t.spacing) for t in tiles]
    if balance:   # a small crop beside the large tiles, all submitted together
        vols.append((np.ascontiguousarray(tiles[0].volume[:48, :48, :48]), tiles[0].spacing))
    want = [_alone(ac, v, sp, p, 100 + i) for i, (v, sp) in enumerate(vols)]
    srv = ac.Server(p, ac.AC_U16, 3, STRIDE, ac.default_E0(3, CONTRAST), hbm_budget_bytes=120 << 30,
                    iters_per_round=7, balance_rounds=balance)
    tickets = []
    for i, (v, sp) in enumerate(vols):
        tickets.append(srv.submit(v, sp, stream_id=100 + i))
        if not balance:
            time.sleep(0.003 * i)          # staggered arrivals: tiles join at different rounds
    rounds = []
    for tk, w in zip(tickets, want):
        cells, res = srv.wait(tk, timeout=300)
        assert res["status"] == 0 and res["rounds"] <= math.ceil(T / 7)
        assert res["total_ms"] >= res["run_ms"] > 0 and res["n_cells"] == len(cells)
        rounds.append(res["rounds"])
        _same_cells(cells, w)
    if balance:
        assert rounds[-1] == 1                 # the crop: 8 x 7 iterations per round cover all 20
    else:
        assert rounds == [math.ceil(T / 7)] * len(vols)
    st = srv.stats()
    assert st["completed"] == len(vols) and st["resident"] == 0 and st["pending"] == 0 and st["finished"] == 0
    assert st["rounds"] < len(vols) * math.ceil(T / 7)    # rounds were shared
    with pytest.raises(ac.ACError):
        srv.wait(tickets[0], timeout=0)                   # collected already
    srv.close()


def _lattice(volume):
    nz, ny, nx = volume.shape
    return max(1, int(nx // STRIDE)) * max(1, int(ny // STRIDE)) * max(1, int(nz // STRIDE))


@pytest.mark.parametrize("mode", ["budget", "one_at_a_time", "contours"])
def test_admission_limits(ac, tiles, mode):
    p = _params(ac)
    want = [_alone(ac, t.volume, t.spacing, p, 7 + i) for i, t in enumerate(tiles)]
    est = [_est_bytes(t.volume, 2) for t in tiles]
    budget = int(1.2 * max(est)) if mode == "budget" else 120 << 30
    cap = max(_lattice(t.volume) for t in tiles) if mode == "contours" else 0
    srv = ac.Server(p, ac.AC_U16, 3, STRIDE, ac.default_E0(3, CONTRAST), hbm_budget_bytes=budget,
                    iters_per_round=5, max_resident=1 if mode == "one_at_a_time" else 0,
                    max_resident_contours=cap, balance_rounds=False)
    tickets = [srv.submit(t.volume, t.spacing, stream_id=7 + i) for i, t in enumerate(tiles)]
    for tk, w, e in zip(tickets, want, est):
        cells, res = srv.wait(tk, timeout=300)
        assert res["est_bytes"] == e
        _same_cells(cells, w)
    st = srv.stats()
    assert st["peak_resident_bytes"] <= budget
    if mode == "one_at_a_time":
        assert st["peak_resident_bytes"] == max(est)
        assert st["rounds"] == len(tiles) * math.ceil(T / 5)
    elif mode == "contours":
        assert st["rounds"] > math.ceil(T / 5) and st["peak_resident_bytes"] < sum(est)
    else:
        assert st["peak_resident_bytes"] < sum(est)       # the budget held tiles back
        big = np.zeros((budget // (2 * 64 * 64) + 8, 64, 64), np.uint16)
        with pytest.raises(ac.ACError) as e:
            srv.submit(big, (1.0, 1.0, 1.0))
        assert e.value.status == ac.AC_ERR_BUDGET
    srv.close()


def test_failing_tile_is_reported_alone(ac, tiles):
    """A tile with non-finite voxels ends with AC_ERR_NUMERIC; the tiles that
    shared its rounds are unaffected (each set keeps its own status word)."""
    p = _params(ac)
    vols = [t.volume[:40, :96, :96].astype(np.float32) for t in tiles[:3]]
    bad = vols[1].copy()
    bad[18:21, 40:43, 40:43] = np.nan
    vols[1] = bad
    want = {i: _alone(ac, vols[i], tiles[i].spacing, p, 50 + i) for i in (0, 2)}
    srv = ac.Server(p, ac.AC_F32, 3, STRIDE, ac.default_E0(3, CONTRAST), hbm_budget_bytes=1 << 30,
                    iters_per_round=10)
    tickets = [srv.submit(v, tiles[i].spacing, stream_id=50 + i) for i, v in enumerate(vols)]
    for i, tk in enumerate(tickets):
        if i == 1:
            with pytest.raises(ac.ACError) as e:
                srv.wait(tk, timeout=300)
            assert e.value.status == ac.AC_ERR_NUMERIC
        else:
            cells, _ = srv.wait(tk, timeout=300)
            _same_cells(cells, want[i])
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 2
    srv.close()


def test_destroy_with_tiles_in_flight(ac, tiles):
    p = _params(ac)
    srv = ac.Server(p, ac.AC_U16, 3, STRIDE, ac.default_E0(3, CONTRAST), hbm_budget_bytes=120 << 30,
                    iters_per_round=2)
    for i, t in enumerate(tiles):
        srv.submit(t.volume, t.spacing, stream_id=i)
    srv.close()                                           # stops after the current round, frees everything


def test_served_tiles_match_the_oracle(ac, oracle, tiles):
    """Served tiles against the FP64 oracle, not only against the CUDA path alone:
    four tiles share the request loop's rounds; one of them records a stripe of
    its evaluations (ac_server_submit_traced), which the oracle re-evaluates at the
    recorded states (1e-5 of the magnitude, pass fraction >= 0.9999); for two tiles
    the oracle evolves every contour from the lattice with the server's parameters
    and the tile's stream id and localizes them: detection-set agreement with the
    served cells, with matching within 0.5 and within 0.25 voxel, at least 0.999,
    or three times closer to 1 than the oracle against itself after a one-ulp
    change of the seeds (tests/_parity.floor_bar)."""
    import torch
    from tests import _parity as P
    p = dataclasses.replace(_params(ac), T=30)
    E0 = ac.default_E0(3, CONTRAST)
    srv = ac.Server(p, ac.AC_U16, 3, STRIDE, E0, hbm_budget_bytes=120 << 30, iters_per_round=7)
    k0, k1 = 100, 356
    buf = torch.full(((k1 - k0) * p.T * 9,), float("nan"), device="cuda", dtype=torch.float32)
    tickets = []
    for i, t in enumerate(tiles[:4]):
        tr = (buf, k0, k1, 1, p.T + 1) if i == 1 else None
        tickets.append(srv.submit(t.volume, t.spacing, stream_id=200 + i, trace=tr))
    served = [srv.wait(tk, timeout=300)[0] for tk in tickets]
    srv.close()
    trace = buf.view(p.T, k1 - k0, 9).cpu().numpy()
    img = P.oracle_image(oracle, tiles[1].volume, tiles[1].spacing)
    op = P.oracle_params(oracle, 3, dataclasses.replace(p, stream_id=201))
    frac, nflag, worst, bad, _ = P.teacher_forced(oracle, img, op, trace, k0, 1)
    assert frac >= 0.9999, (frac, worst, bad)
    for i in (1, 2):
        t = tiles[i]
        V = ac.ac_create_volume(t.volume, t.spacing)
        seeds = ac.ac_get_state(ac.ac_seed(V, stride=STRIDE))       # the lattice the server seeds
        pi = dataclasses.replace(p, stream_id=200 + i)
        ids = np.arange(seeds.shape[1])
        _, _, cells_o, floor = P.oracle_with_floor(ac, oracle, t, t.volume, 3, pi, seeds[:4].T.astype(np.float64),
                                                   ids)
        dg = served[i]["c"].astype(np.float64) / np.asarray(t.spacing, np.float64)
        agree, agree_q = P.compare_cells(dg, cells_o)
        print("SERVED " + str({"tile": i, "cells": (len(dg), len(cells_o)), "agreement": agree,
                               "agreement_0.25": agree_q, "floor": floor}))
        assert len(cells_o) > 20
        assert agree >= P.floor_bar(floor["agreement"]), (i, agree, floor)
        assert agree_q >= P.floor_bar(floor["agreement_0.25"]), (i, agree_q, floor)
