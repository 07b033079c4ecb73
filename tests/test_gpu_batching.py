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
