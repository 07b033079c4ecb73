"""Batching form: plans over several uneven volumes, CUDA-graph replay, per-set
iteration windows advanced round by round, and the autotuner -- all checked
against single-set runs (bit-identical) or the FP64 oracle."""
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
def vols():
    from paper_1804_06304_gb300 import synth
    return synth.batch_3d(11, count=5, max_scale=0.35)


def _sets(ac, vols, keep):
    out = []
    for s in vols:
        V = ac.ac_create_volume(s.volume)
        keep.append(V)
        out.append(ac.ac_seed(V, stride=4.0))
    return out


def _params(ac, **kw):
    return ac.default_params(3, 4.0 / math.sqrt(1.5), 170.0, **{**dict(N=128, T=8, seed=77), **kw})


@pytest.mark.parametrize("use_graph", [False, True])
def test_plan_matches_batch_and_replays(ac, vols, use_graph):
    keep = []
    p = _params(ac)
    a = _sets(ac, vols, keep)
    items = [(40 + i, 1, 8, 1) for i in range(len(vols))]
    ac.ac_evolve_batch(a, p, items=items)
    ac.ac_evolve_batch(a, p, items=[(40 + i, 9, 8, 0) for i in range(len(vols))])
    b = _sets(ac, vols, keep)
    plan = ac.ac_plan_create(b, p, items=items)
    ac.ac_plan_launch(plan, use_graph=use_graph)
    ac.ac_plan_set_items(plan, [(40 + i, 9, 8, 0) for i in range(len(vols))])
    ac.ac_plan_launch(plan, use_graph=use_graph)   # a graph launch is a replay of the first capture
    assert ac.ac_evolve_kernel_ms(b[0]) > 0.0        # kernel-time events are recorded by the replay too
    for x, y in zip(a, b):
        np.testing.assert_array_equal(ac.ac_get_state(y), ac.ac_get_state(x))


@pytest.mark.parametrize("path", [0, 1])
def test_rounds_equal_uninterrupted(ac, vols, path):
    """Serving-style rounds: every set advances 5 iterations a round through one
    plan (sets start at different rounds); each ends where an uninterrupted run of
    its 20 iterations ends."""
    keep = []
    p = _params(ac, T=20, path=path)
    ref = _sets(ac, vols, keep)
    for i, c in enumerate(ref):
        ac.ac_evolve(c, ac.EvolveParams(**{**p.__dict__, "stream_id": i}))
    want = [ac.ac_get_state(c) for c in ref]
    sets = _sets(ac, vols, keep)
    start = [0, 1, 1, 2, 3]           # round in which each set joins
    progress = [0] * len(sets)
    plan = ac.ac_plan_create(sets, p, items=[(i, 1, 0, 0) for i in range(len(sets))])
    for rnd in range(8):
        items = []
        for i in range(len(sets)):
            if rnd < start[i] or progress[i] >= 20:
                items.append((i, max(1, progress[i] + 1), 0, 0))
                continue
            n = min(5, 20 - progress[i])
            items.append((i, progress[i] + 1, n, 1 if progress[i] + n < 20 else 0))
            progress[i] += n
        ac.ac_plan_set_items(plan, items)
        ac.ac_plan_launch(plan, use_graph=True)
    assert progress == [20] * len(sets)
    for c, w in zip(sets, want):
        np.testing.assert_array_equal(ac.ac_get_state(c), w)


def test_autotune_leaves_sets_and_passes_parity(ac, oracle, vols):
    keep = []
    sets = _sets(ac, vols[:3], keep)
    before = [ac.ac_get_state(c) for c in sets]
    p = _params(ac, T=6)
    tuned = ac.ac_autotune(sets, p)
    assert tuned.lanes_per_contour in (4, 8, 16, 32) and tuned.warps_per_block >= 1
    assert all(b > 0 for b in tuned.brick)
    for c, b in zip(sets, before):
        np.testing.assert_array_equal(ac.ac_get_state(c), b)
    assert ac.ac_autotune(sets, p) == tuned          # cached
    s = vols[0]
    r = P.gpu_run(ac, s.volume, s.spacing, tuned, stride=4.0, trace_k=(0, min(600, sets[0].count)))
    img = P.oracle_image(oracle, s.volume, s.spacing)
    frac, nflag, worst, bad, _ = P.teacher_forced(oracle, img, P.oracle_params(oracle, 3, tuned), r["trace"], 0, 1)
    assert frac >= 0.9999, (frac, worst, bad)


def test_localize_batch_equals_each_set_and_the_oracle(ac, oracle, vols):
    """One ac_localize_batch over uneven 3D sets, a 2D set, a set that the energy
    cull empties, an explicitly empty set and a cap below the accepted count gives
    every set exactly the cells of ac_localize alone, which are the oracle's."""
    from paper_1804_06304_gb300 import synth
    keep = []
    sets = _sets(ac, vols, keep)
    ac.ac_evolve_batch(sets, _params(ac, T=20))
    s2 = synth.large_2d(4, shape=(256, 256), n_nuclei=60)
    V2 = ac.ac_create_volume(s2.volume, s2.spacing)
    C2 = ac.ac_seed(V2, stride=6.0)
    ac.ac_evolve(C2, ac.default_params(2, 6.0 / math.sqrt(1.5), s2.contrast, N=128, T=20, seed=3))
    V0 = ac.ac_create_volume(np.zeros((8, 8, 8), np.uint8))
    C0 = ac.ac_seed(V0, explicit=np.zeros((0, 4), np.float32))
    Ecut = ac.ac_seed(ac.ac_create_volume(vols[0].volume), stride=4.0)   # E = 0 at seeding: culled by E0 < 0
    all_sets = sets + [C2, C0, Ecut]
    E0 = [ac.default_E0(3, 170.0)] * len(sets) + [ac.default_E0(2, s2.contrast), -1.0, -1.0]
    alone = [ac.ac_localize(c, e) for c, e in zip(all_sets, E0)]
    assert len(alone[0]) > 3 and len(alone[-2]) == 0 and len(alone[-1]) == 0
    got = ac.ac_localize_batch(all_sets, E0)
    for a, b in zip(alone, got):
        np.testing.assert_array_equal(a, b)
    for c, e, cells in zip(all_sets[:len(sets) + 1], E0, got):
        st = ac.ac_get_state(c).astype(np.float64)
        nd = 2 if c is C2 else 3
        assert list(cells["id"]) == list(oracle.localize(nd, st[:4].T, st[4], float(np.float32(e))))
    caps = [2] + [c.count for c in all_sets[1:]]
    part = ac.ac_localize_batch(all_sets, E0, caps=caps)
    np.testing.assert_array_equal(part[0], alone[0][:2])
    for a, b in zip(alone[1:], part[1:]):
        np.testing.assert_array_equal(a, b)
    assert ac.ac_localize_batch([], 0.0) == []


def test_localize_batch_rejects_bad_arguments(ac, vols):
    keep = []
    sets = _sets(ac, vols[:2], keep)
    with pytest.raises(ac.ACError) as e:
        ac.ac_localize_batch([sets[0], sets[1], sets[0]], 0.0)
    assert e.value.status == ac.AC_ERR_ARG
    with pytest.raises(ac.ACError) as e:
        ac.ac_localize_batch(sets, [0.0, float("nan")])
    assert e.value.status == ac.AC_ERR_ARG
    with pytest.raises(ac.ACError) as e:
        ac.ac_localize_batch(sets, 0.0, caps=[5, -1])
    assert e.value.status == ac.AC_ERR_ARG
