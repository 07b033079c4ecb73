"""Handles release what they allocate: repeated create / seed / evolve / batch /
plan / localize / destroy cycles and request loops leave device memory where it
started."""
import gc
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ac():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06304_gb300 import ac as lib
    lib.load()
    return lib


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _cycle(ac, s, i):
    R0 = 4.0 / math.sqrt(1.5)
    p = ac.default_params(3, R0, s.contrast, N=64, T=4, seed=i, cull_iter=2, cull_E=0.0)
    V = ac.ac_create_volume(s.volume, s.spacing)
    a, b = ac.ac_seed(V, stride=4.0), ac.ac_seed(V, stride=5.0)
    ac.ac_evolve(a, p)
    ac.ac_evolve_batch([a, b], p, items=[(1, 5, 4, 0), (2, 1, 4, 0)])
    plan = ac.ac_plan_create([a, b], p)
    ac.ac_plan_launch(plan, use_graph=True)
    ac.ac_plan_launch(plan, use_graph=True)
    ac.ac_localize(a, ac.default_E0(3, s.contrast))
    ac.ac_evolve_stops(b)
    ac.ac_destroy_plan(plan)
    ac.ac_destroy_contours(a)
    ac.ac_destroy_contours(b)
    ac.ac_destroy_volume(V)


def test_handles_release_device_memory(ac):
    from paper_1804_06304_gb300 import synth
    s = synth.small_3d(0)
    _cycle(ac, s, 0)                      # first use: lazily created library state
    gc.collect()
    before = _free_bytes()
    for i in range(30):
        _cycle(ac, s, i + 1)
    gc.collect()
    after = _free_bytes()
    assert before - after < (8 << 20), (before, after)


def test_server_releases_device_memory(ac):
    from paper_1804_06304_gb300 import synth
    tiles = [t for _, t in synth.tile_stream(31, count=3, max_scale=0.2)]
    p = ac.default_params(3, 6.0 / math.sqrt(1.5), 1700.0, N=64, T=6, seed=3)

    def serve():
        srv = ac.Server(p, ac.AC_U16, 3, 6.0, ac.default_E0(3, 1700.0), hbm_budget_bytes=1 << 30,
                        iters_per_round=2)
        ts = [srv.submit(t.volume, t.spacing, stream_id=i) for i, t in enumerate(tiles)]
        for t in ts:
            srv.wait(t, timeout=300)
        srv.close()

    serve()
    gc.collect()
    before = _free_bytes()
    for _ in range(5):
        serve()
    gc.collect()
    after = _free_bytes()
    assert before - after < (8 << 20), (before, after)
