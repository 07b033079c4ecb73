"""ac_evolve_static: the evolve entry point for callers that cannot allocate device
memory (their memory belongs to their own allocator, or they run in loops where an
allocation could block the device).  The caller owns the volume and the contour
state; the library's temporaries live in one fixed device array.

Checked through the C ABI against ac_evolve on the same seeded inputs, twice in a
row (the second call reuses the array the first one left behind), in 3D on the
brick path and in 2D on both paths, bit for bit; a repeated call leaves the
device's free memory unchanged; a padded volume runs on the plain path; arguments
the entry point cannot take are rejected before any device work.  This file is
collected last.
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
    return lib


def _reference_then_static(ac, volume, spacing, stride, params_list, ndim):
    import torch
    V = ac.ac_create_volume(volume, spacing)
    C = ac.ac_seed(V, stride=stride)
    init = ac.ac_get_state(C)
    refs = []
    for p in params_list:
        ac.ac_evolve(C, p)
        refs.append(ac.ac_get_state(C))
    vol_dev = torch.from_numpy(volume).cuda()
    state_dev = torch.from_numpy(init.copy()).cuda()
    R0 = stride / math.sqrt(1.5)
    outs = []
    for p in params_list:
        ac.ac_evolve_static(vol_dev, state_dev, p, R0, stride, spacing=spacing)
        outs.append(state_dev.cpu().numpy().copy())
    return refs, outs


def _assert_close(ref, out):
    # the same kernel on the same inputs and launch plan: identical bits (tighter
    # than the 1e-5 parity bar of the other GPU tests)
    np.testing.assert_array_equal(out, ref)


def test_static_3d_brick_two_calls(ac):
    from paper_1804_06304_gb300 import synth
    s = synth.small_3d(0)
    R0 = 4.0 / math.sqrt(1.5)
    p1 = ac.default_params(3, R0, s.contrast, N=256, T=12, seed=21, update_last=1)
    p2 = ac.default_params(3, R0, s.contrast, N=256, T=9, seed=21, first_iter=13)
    refs, outs = _reference_then_static(ac, s.volume, s.spacing, 4.0, [p1, p2], 3)
    for ref, out in zip(refs, outs):
        _assert_close(ref, out)


@pytest.mark.parametrize("path", [0, 1])
def test_static_2d_two_calls(ac, path):
    from paper_1804_06304_gb300 import synth
    s = synth.large_2d(1, shape=(512, 512), n_nuclei=188)
    R0 = 6.0 / math.sqrt(1.5)
    p1 = ac.default_params(2, R0, s.contrast, N=128, T=20, seed=5, path=path)
    p2 = ac.default_params(2, R0, s.contrast, N=64, T=7, seed=6, path=path, stream_id=3)
    refs, outs = _reference_then_static(ac, s.volume, s.spacing, 6.0, [p1, p2], 2)
    for ref, out in zip(refs, outs):
        _assert_close(ref, out)


def test_static_rejects_sizes_beyond_its_array(ac):
    import torch
    vol = torch.zeros((8, 16, 16), dtype=torch.uint8, device="cuda")
    state = torch.zeros((5, 4), dtype=torch.float32, device="cuda")
    p = ac.EvolveParams(N=8, T=1, eps0=0.1)
    with pytest.raises(ac.ACError) as e:
        ac.ac_evolve_static(vol, state, p, 2.0, 3.0, n_contours=ac.AC_STATIC_MAX_CONTOURS + 1)
    assert e.value.status == ac.AC_ERR_BUDGET and "AC_STATIC_MAX_CONTOURS" in str(e.value)


def test_static_call_allocates_nothing(ac):
    """After a first call (which looks up the array's address and loads the kernels),
    another call leaves the device's free memory exactly where it was."""
    import torch
    from paper_1804_06304_gb300 import synth
    s = synth.small_3d(0)
    R0 = 4.0 / math.sqrt(1.5)
    p = ac.default_params(3, R0, s.contrast, N=256, T=6, seed=4)
    V = ac.ac_create_volume(s.volume, s.spacing)
    C = ac.ac_seed(V, stride=4.0)
    init = ac.ac_get_state(C)
    vol_dev = torch.from_numpy(s.volume).cuda()
    state_dev = torch.from_numpy(init.copy()).cuda()
    ac.ac_evolve_static(vol_dev, state_dev, p, R0, 4.0, spacing=s.spacing)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    state_dev.copy_(torch.from_numpy(init))
    torch.cuda.synchronize()
    ac.ac_evolve_static(vol_dev, state_dev, p, R0, 4.0, spacing=s.spacing)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_padded_volume_on_the_plain_path(ac):
    """A row-padded view (row stride W + 5 voxels) runs on the plain path and gives
    the bits of ac_evolve on the same voxels; the brick path rejects that pitch
    (not a multiple of 16 bytes) with AC_ERR_ARG."""
    import torch
    from paper_1804_06304_gb300 import synth
    s = synth.large_2d(2, shape=(200, 160), n_nuclei=40)
    H, W = s.volume.shape
    R0 = 6.0 / math.sqrt(1.5)
    p = ac.default_params(2, R0, s.contrast, N=128, T=9, seed=12, path=ac.AC_PATH_PLAIN)
    V = ac.ac_create_volume(s.volume, s.spacing)
    C = ac.ac_seed(V, stride=6.0)
    init = ac.ac_get_state(C)
    ac.ac_evolve(C, p)
    ref = ac.ac_get_state(C)
    padded = torch.zeros((H, W + 5), dtype=torch.uint8, device="cuda")
    padded[:, :W] = torch.from_numpy(s.volume).cuda()
    view = padded[:, :W]
    assert view.stride() == (W + 5, 1)
    state_dev = torch.from_numpy(init.copy()).cuda()
    ac.ac_evolve_static(view, state_dev, p, R0, 6.0, spacing=s.spacing)
    np.testing.assert_array_equal(state_dev.cpu().numpy(), ref)
    pb = ac.default_params(2, R0, s.contrast, N=128, T=9, seed=12, path=ac.AC_PATH_BRICK)
    with pytest.raises(ac.ACError) as e:
        ac.ac_evolve_static(view, torch.from_numpy(init.copy()).cuda(), pb, R0, 6.0, spacing=s.spacing)
    assert e.value.status == ac.AC_ERR_ARG and "16" in str(e.value)


def test_static_rejects_unusable_tensors(ac):
    """The binding refuses, with AC_ERR_ARG and before any device work, a state that
    is not a contiguous CUDA float32 (5, C) tensor, a contour count above its
    columns, a volume with a non-unit x stride, of an unsupported dtype or in host
    memory."""
    import torch
    vol = torch.zeros((8, 32, 32), dtype=torch.uint8, device="cuda")
    state = torch.zeros((5, 4), dtype=torch.float32, device="cuda")
    p = ac.EvolveParams(N=8, T=1, eps0=0.1)
    bad = [dict(state=state.double()), dict(state=torch.zeros((4, 5), device="cuda").t()),
           dict(state=torch.zeros((4, 4), device="cuda")), dict(state=state.cpu()), dict(n_contours=5),
           dict(n_contours=0), dict(vol=vol[:, :, ::2]), dict(vol=vol.int()), dict(vol=vol.cpu())]
    for b in bad:
        with pytest.raises(ac.ACError) as e:
            ac.ac_evolve_static(b.get("vol", vol), b.get("state", state), p, 2.0, 3.0,
                                n_contours=b.get("n_contours"))
        assert e.value.status == ac.AC_ERR_ARG, b
