"""The paper's variants through the C ABI against the FP64 oracle: the voxel-grid
form of Eq. 5 (AC_PATH_GRID) and the stopping rules (convergence freeze and
energy culling) on every path."""
import dataclasses
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
def small3d():
    from paper_1804_06304_gb300 import synth
    return synth.small_3d(0)


@pytest.fixture(scope="module")
def aniso3d():
    from paper_1804_06304_gb300 import synth
    return synth.brain_3d(5, shape=(96, 96, 24), n_nuclei=60)


@pytest.fixture(scope="module")
def crop2d():
    from paper_1804_06304_gb300 import synth
    return synth.large_2d(1, shape=(256, 256), n_nuclei=47)


def _p3(ac, s, **kw):
    R0 = 4.0 / math.sqrt(1.5)
    base = dict(N=256, T=30, seed=99)
    base.update(kw)
    return ac.default_params(3, R0, s.contrast, **base)


# ------------------------------------------------------------------ grid form of Eq. 5
@pytest.mark.parametrize("G,comp", [(8, 1), (16, 1), (8, 0)])
def test_grid_teacher_forced_small3d(ac, oracle, small3d, G, comp):
    s = small3d
    p = _p3(ac, s, path=ac.AC_PATH_GRID, lanes_per_contour=G, compensated=comp)
    r = P.gpu_run(ac, s.volume, s.spacing, p, stride=4.0, trace_k=(0, 2048))
    img = P.oracle_image(oracle, s.volume, s.spacing)
    frac, nflag, worst, bad, _ = P.teacher_forced(oracle, img, P.oracle_params(oracle, 3, p), r["trace"], 0, 1)
    assert frac >= 0.9999, (frac, nflag, worst, bad)
    np.testing.assert_array_equal(r["trace"][-1, :, :4].T, r["final"][:4])
    np.testing.assert_array_equal(r["trace"][-1, :, 4], r["final"][4])


def test_grid_teacher_forced_anisotropic_u16_f16(ac, oracle, aniso3d):
    s = aniso3d
    R0 = 6.0 / math.sqrt(1.5)
    for vol in (s.volume, s.volume_f16):
        p = ac.default_params(3, R0, s.contrast, N=1, T=12, seed=3, path=ac.AC_PATH_GRID)
        r = P.gpu_run(ac, vol, s.spacing, p, stride=6.0, trace_k=(0, 1000))
        img = P.oracle_image(oracle, vol, s.spacing)
        frac, nflag, worst, bad, _ = P.teacher_forced(oracle, img, P.oracle_params(oracle, 3, p), r["trace"], 0, 1)
        assert frac >= 0.9999, (vol.dtype, frac, nflag, worst, bad)


@pytest.mark.parametrize("G,comp", [(0, 1), (8, 1), (16, 0)])
def test_grid_teacher_forced_2d(ac, oracle, crop2d, G, comp):
    s = crop2d
    R0 = 6.0 / math.sqrt(1.5)
    p = ac.default_params(2, R0, s.contrast, N=1, T=20, seed=8, path=ac.AC_PATH_GRID, lanes_per_contour=G,
                          compensated=comp)
    r = P.gpu_run(ac, s.volume, s.spacing, p, stride=6.0, trace_k=(0, 1764))
    img = P.oracle_image(oracle, s.volume, s.spacing)
    frac, nflag, worst, bad, _ = P.teacher_forced(oracle, img, P.oracle_params(oracle, 2, p), r["trace"], 0, 1)
    assert frac >= 0.9999, (frac, nflag, worst, bad)


def test_grid_free_running_small3d(ac, oracle, small3d):
    """Deterministic descent on the grid energy: the FP32 path follows the FP64
    oracle to the same converged centres."""
    s = small3d
    p = _p3(ac, s, path=ac.AC_PATH_GRID)
    r = P.gpu_run(ac, s.volume, s.spacing, p, stride=4.0)
    img = P.oracle_image(oracle, s.volume, s.spacing)
    cR, E, _ = oracle.evolve(img, P.oracle_params(oracle, 3, p), r["init"][:4].T.astype(np.float64))
    dc = np.linalg.norm(r["final"][:3].T - cR[:, :3], axis=1)
    assert np.mean(dc < 0.25) >= 0.99, np.sort(dc)[-10:]
    E0 = ac.default_E0(3, s.contrast)
    cells = ac.ac_localize(r["ctr"], E0)
    ids_o = oracle.localize(3, cR, E, E0)
    m = P.match_sets(np.stack([c for c in cells["c"]]) if len(cells) else np.zeros((0, 3)), cR[ids_o, :3], 0.5)
    assert 2 * m / (len(cells) + len(ids_o)) >= 0.99, (m, len(cells), len(ids_o))
    assert len(cells) >= 18


def test_grid_batch_equals_single(ac, small3d):
    s = small3d
    p = _p3(ac, s, path=ac.AC_PATH_GRID, T=10)
    V = ac.ac_create_volume(s.volume, s.spacing)
    a, b = ac.ac_seed(V, stride=4.0), ac.ac_seed(V, stride=5.0)
    ac.ac_evolve_batch([a, b], p, items=[(3, 1, 10, 0), (4, 1, 10, 0)])
    a2, b2 = ac.ac_seed(V, stride=4.0), ac.ac_seed(V, stride=5.0)
    ac.ac_evolve(a2, dataclasses.replace(p, stream_id=3))
    ac.ac_evolve(b2, dataclasses.replace(p, stream_id=4))
    np.testing.assert_array_equal(ac.ac_get_state(a), ac.ac_get_state(a2))
    np.testing.assert_array_equal(ac.ac_get_state(b), ac.ac_get_state(b2))


def test_grid_radius_bounds(ac, small3d):
    s = small3d
    V = ac.ac_create_volume(s.volume, s.spacing)
    C = ac.ac_seed(V, stride=4.0)
    with pytest.raises(ac.ACError) as e:
        ac.ac_evolve(C, _p3(ac, s, path=ac.AC_PATH_GRID, Rmax=400.0))
    assert e.value.status == ac.AC_ERR_ARG
    # a radius set beyond the bound: the contour stops and the status reports it
    st = ac.ac_get_state(C)
    st[3, 5] = 300.0
    ac.ac_set_state(C, st)
    ac.ac_evolve(C, _p3(ac, s, path=ac.AC_PATH_GRID, T=2, Rmax=200.0, Rmin=0.5))
    with pytest.raises(ac.ACError) as e:
        ac.ac_get_state(C)
    assert e.value.status == ac.AC_ERR_ARG


# ------------------------------------------------------------------ stopping rules
def _runs(trace):
    """Per contour: the number of evaluated (written) trace rows."""
    return (~np.isnan(trace[:, :, 0])).sum(axis=0)


def _check_rules(ac, oracle, r, p, img, ndim):
    tr = r["trace"]
    T, K, _ = tr.shape
    ne = _runs(tr)
    # rows are a prefix: nothing written after the last evaluation
    for k in range(K):
        assert not np.isnan(tr[:ne[k], k, 0]).any() and np.isnan(tr[ne[k]:, k, 0]).all()
    frozen = culled = 0
    tol = np.float32(p.freeze_tol)
    for k in range(K):
        n = int(ne[k])
        rows = tr[:n, k]
        # observed steps (float32, the kernel's arithmetic): max |c' - c|, |R' - R|
        d = np.abs(rows[1:, :4] - rows[:-1, :4])
        step = np.maximum(d[:, 3], d[:, :ndim].max(axis=1)) if n > 1 else np.zeros(0, np.float32)
        small = step < tol
        run = 0
        for sflag in small:   # no run of freeze_iters applied small steps
            run = run + 1 if sflag else 0
            assert run < p.freeze_iters
        is_culled = p.cull_iter > 0 and n == p.cull_iter and rows[-1, 4] > np.float32(p.cull_E)
        if n < T and is_culled:
            culled += 1
        elif n < T:
            frozen += 1
            # the last freeze_iters - 1 applied steps were small, and the unapplied one too
            assert run == p.freeze_iters - 1, (k, n, small[-p.freeze_iters:])
            last = rows[-1].astype(np.float64)
            res = oracle.eval_many(img, P.oracle_params(oracle, ndim, p), last[None, :4], [n], [k])
            pp = np.array([last[0] - last[3], last[1], last[2]])
            qq = np.array([last[0] + last[3], last[1], last[2]])
            p1, q1 = oracle.update_pq(img, P.oracle_params(oracle, ndim, p), n, res[0], pp, qq)
            c1, R1 = (p1 + q1) / 2, (q1[0] - p1[0]) / 2
            est = max(abs(R1 - rows[-1, 3]), np.abs(c1[:ndim] - rows[-1, :ndim]).max())
            assert est < tol * (1 + 1e-3) + 1e-5, (k, est)
        elif p.cull_iter > 0 and n >= p.cull_iter:
            assert rows[p.cull_iter - 1, 4] <= np.float32(p.cull_E)
        # the final state is the last evaluated state and its energy
        np.testing.assert_array_equal(r["final"][:4, k], rows[-1, :4])
        assert r["final"][4, k] == rows[-1, 4]
    assert ac.ac_evolve_stops(r["ctr"]) == (frozen, culled)
    return frozen, culled


@pytest.mark.parametrize("path", [0, 1, 2])
def test_stopping_rules_follow_their_definition(ac, oracle, small3d, path):
    s = small3d
    E0 = ac.default_E0(3, s.contrast)
    p = _p3(ac, s, path=path, T=60, freeze_tol=0.08, freeze_iters=3, cull_iter=15, cull_E=0.3 * E0)
    r = P.gpu_run(ac, s.volume, s.spacing, p, stride=4.0, trace_k=(0, 2048))
    img = P.oracle_image(oracle, s.volume, s.spacing)
    frozen, culled = _check_rules(ac, oracle, r, p, img, 3)
    assert frozen > 0 and culled > 0
    frac, nflag, worst, bad, _ = P.teacher_forced(oracle, img, P.oracle_params(oracle, 3, p), r["trace"], 0, 1)
    assert frac >= 0.9999, (frac, worst, bad)


def test_stopping_rules_resume_and_paths_agree(ac, small3d):
    """Two calls (update_last, first_iter) equal one; brick and plain paths give the
    same bits with the rules on; stopped contours stay stopped; ac_set_state clears
    the rule state."""
    s = small3d
    E0 = ac.default_E0(3, s.contrast)
    p = _p3(ac, s, T=40, freeze_tol=0.08, freeze_iters=3, cull_iter=15, cull_E=0.3 * E0)
    V = ac.ac_create_volume(s.volume, s.spacing)
    one = ac.ac_seed(V, stride=4.0)
    ac.ac_evolve(one, p)
    two = ac.ac_seed(V, stride=4.0)
    ac.ac_evolve(two, dataclasses.replace(p, T=17, update_last=1))
    ac.ac_evolve(two, dataclasses.replace(p, T=23, first_iter=18))
    np.testing.assert_array_equal(ac.ac_get_state(one), ac.ac_get_state(two))
    assert ac.ac_evolve_stops(one) == ac.ac_evolve_stops(two)
    plain = ac.ac_seed(V, stride=4.0)
    ac.ac_evolve(plain, dataclasses.replace(p, path=ac.AC_PATH_PLAIN))
    np.testing.assert_array_equal(ac.ac_get_state(one), ac.ac_get_state(plain))
    before = ac.ac_get_state(one)
    stopped = sum(ac.ac_evolve_stops(one))
    assert stopped > 0
    ac.ac_evolve(one, dataclasses.replace(p, T=5, first_iter=41))
    after = ac.ac_get_state(one)
    moved = np.any(after != before, axis=0)
    assert moved.sum() <= after.shape[1] - stopped   # stopped contours did not move
    ac.ac_set_state(one, after)
    assert ac.ac_evolve_stops(one) == (0, 0)


def test_stopping_rules_off_is_unchanged(ac, small3d):
    """Rules disabled (the defaults) give the same bits as limits that never fire."""
    s = small3d
    p = _p3(ac, s, T=20)
    V = ac.ac_create_volume(s.volume, s.spacing)
    a = ac.ac_seed(V, stride=4.0)
    ac.ac_evolve(a, p)
    b = ac.ac_seed(V, stride=4.0)
    ac.ac_evolve(b, dataclasses.replace(p, freeze_tol=0.0, freeze_iters=3, cull_iter=5, cull_E=float("inf")))
    np.testing.assert_array_equal(ac.ac_get_state(a), ac.ac_get_state(b))
    assert ac.ac_evolve_stops(b) == (0, 0)


def test_stopping_rules_against_free_running_oracle(ac, oracle, small3d):
    """The FP64 oracle with the same rules stops the same contours for the same
    reasons (decisions near a threshold may differ between FP32 and FP64)."""
    s = small3d
    E0 = ac.default_E0(3, s.contrast)
    p = _p3(ac, s, T=60, freeze_tol=0.08, freeze_iters=3, cull_iter=15, cull_E=0.3 * E0)
    r = P.gpu_run(ac, s.volume, s.spacing, p, stride=4.0, trace_k=(0, 2048))
    img = P.oracle_image(oracle, s.volume, s.spacing)
    cR, E, _, stops, ne = oracle.evolve(img, P.oracle_params(oracle, 3, p), r["init"][:4].T.astype(np.float64),
                                        stops=True)
    n_gpu = _runs(r["trace"])
    culled_gpu = (n_gpu == p.cull_iter) & (r["final"][4] > np.float32(p.cull_E))
    stop_gpu = np.where(n_gpu == p.T, 0, np.where(culled_gpu, 2, 1))
    agree = np.mean(stop_gpu == stops)
    print("STOP_AGREEMENT", agree, np.bincount(stop_gpu, minlength=3), np.bincount(stops, minlength=3))
    assert agree >= 0.8, agree
    same = (stop_gpu == stops) & (n_gpu == ne)
    dc = np.linalg.norm(r["final"][:3].T - cR[:, :3], axis=1)
    assert np.mean(dc[same] < 0.25) >= 0.99


def test_split_launch_with_items_equals_plain(ac, small3d):
    """An energy rule inside a brick launch splits it (brick kernel up to cull_iter,
    then the plain kernel over the compacted survivors); per-set windows that
    straddle, precede or follow cull_iter give exactly the plain path's results."""
    s = small3d
    E0 = ac.default_E0(3, s.contrast)
    p = _p3(ac, s, T=10, cull_iter=6, cull_E=0.3 * E0)
    items = [(1, 1, 10, 0), (2, 1, 5, 1), (3, 7, 4, 0)]   # straddles 6; ends before it; starts after it
    V = ac.ac_create_volume(s.volume, s.spacing)
    res = {}
    for path in (ac.AC_PATH_BRICK, ac.AC_PATH_PLAIN):
        sets = [ac.ac_seed(V, stride=st) for st in (4.0, 4.0, 5.0)]
        ac.ac_evolve_batch(sets, dataclasses.replace(p, path=path), items=items)
        res[path] = [ac.ac_get_state(c) for c in sets] + [np.array(ac.ac_evolve_stops(c)) for c in sets]
    for x, y in zip(res[ac.AC_PATH_BRICK], res[ac.AC_PATH_PLAIN]):
        np.testing.assert_array_equal(x, y)
    assert res[ac.AC_PATH_BRICK][3][1] > 0   # the first set had contours culled
