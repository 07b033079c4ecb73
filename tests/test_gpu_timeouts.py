"""Bounded waits that run out, in the forms that fault nothing: the library's wait
bounds are lowered for the test (ac_set_wait_limits), so the brick kernel's wait
for its TMA load gives up at once (the copy in flight is still drained before the
CTA exits) and the overlap competition of the localization stops before its first
round; a request-loop ticket is polled before its tile can have finished.  Each
gives AC_ERR_TIMEOUT, and the library works normally afterwards.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ac():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_06304_gb300 import ac as lib
    lib.load()
    yield lib
    lib.ac_set_wait_limits(-1, -1)


@pytest.fixture(scope="module")
def small3d():
    from paper_1804_06304_gb300 import synth
    return synth.small_3d(0)


def _params(ac, s, **kw):
    return ac.default_params(3, 4.0 / math.sqrt(1.5), s.contrast, N=256, T=kw.pop("T", 8), seed=31, **kw)


def test_brick_load_wait_gives_up(ac, small3d):
    s = small3d
    p = _params(ac, s)
    V = ac.ac_create_volume(s.volume, s.spacing)
    ref = ac.ac_seed(V, stride=4.0)
    ac.ac_evolve(ref, p)
    want = ac.ac_get_state(ref)
    C = ac.ac_seed(V, stride=4.0)
    try:
        ac.ac_set_wait_limits(tma_polls=0)
        ac.ac_evolve(C, p)
        with pytest.raises(ac.ACError) as e:
            ac.ac_get_state(C)
        assert e.value.status == ac.AC_ERR_TIMEOUT and "brick load" in str(e.value)
        fast, clamped, glob = ac.ac_evolve_stats(C)
        assert fast + clamped + glob == 0          # every brick gave up before its contours
    finally:
        ac.ac_set_wait_limits(-1, -1)
    ac.ac_reseed(C)                                # clears the status word
    ac.ac_evolve(C, p)
    np.testing.assert_array_equal(ac.ac_get_state(C), want)


def test_localize_round_bound(ac, oracle, small3d):
    s = small3d
    p = _params(ac, s, T=20)
    V = ac.ac_create_volume(s.volume, s.spacing)
    C = ac.ac_seed(V, stride=4.0)
    ac.ac_evolve(C, p)
    st = ac.ac_get_state(C)
    E0 = 1e9                                       # every contour survives the energy cull
    C2 = ac.ac_seed(V, stride=4.0)
    ac.ac_evolve(C2, p)
    try:
        ac.ac_set_wait_limits(localize_rounds=0)
        with pytest.raises(ac.ACError) as e:
            ac.ac_localize(C, E0)
        assert e.value.status == ac.AC_ERR_TIMEOUT and "round bound" in str(e.value)
        with pytest.raises(ac.ACError) as e:          # the same bound in a batch
            ac.ac_localize_batch([C2], E0)
        assert e.value.status == ac.AC_ERR_TIMEOUT and "round bound" in str(e.value)
    finally:
        ac.ac_set_wait_limits(-1, -1)
    with pytest.raises(ac.ACError) as e:            # the status word keeps the failure
        ac.ac_get_state(C)
    assert e.value.status == ac.AC_ERR_TIMEOUT
    ac.ac_reseed(C)
    ac.ac_evolve(C, p)
    np.testing.assert_array_equal(ac.ac_get_state(C), st)
    cells = ac.ac_localize(C, E0)
    want = oracle.localize(3, st[:4].T.astype(np.float64), st[4].astype(np.float64), E0)
    assert list(cells["id"]) == list(want)
    with pytest.raises(ac.ACError) as e:            # the batch's set keeps its failure too
        ac.ac_get_state(C2)
    assert e.value.status == ac.AC_ERR_TIMEOUT
    ac.ac_reseed(C2)
    ac.ac_evolve(C2, p)
    assert list(ac.ac_localize_batch([C2], E0)[0]["id"]) == list(want)


def test_server_wait_times_out_on_an_unfinished_tile(ac):
    from paper_1804_06304_gb300 import synth
    tiles = [t for _, t in synth.tile_stream(11, count=2, max_scale=0.25)]
    R0 = 6.0 / math.sqrt(1.5)
    p = ac.default_params(3, R0, tiles[0].contrast, N=512, T=40, seed=5)
    srv = ac.Server(p, ac.AC_U16, 3, 6.0, ac.default_E0(3, tiles[0].contrast), hbm_budget_bytes=1 << 32,
                    iters_per_round=5)
    try:
        tk = srv.submit(tiles[0].volume, tiles[0].spacing, stream_id=1)
        with pytest.raises(ac.ACError) as e:
            srv.wait(tk, timeout=0.0)
        assert e.value.status == ac.AC_ERR_TIMEOUT
        cells, res = srv.wait(tk, timeout=600)     # the ticket stays valid
        assert res["status"] == ac.AC_OK and res["rounds"] >= 8
    finally:
        srv.close()
