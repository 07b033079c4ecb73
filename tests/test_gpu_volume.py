"""Volume upload routes: dense and strided host arrays, dense and strided device
tensors, and reloads into an existing volume all give the same device copy (the
evolution's bits), including extents whose rows the library pads to 16 bytes."""
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


def _evolve(ac, vol, ndim):
    V = ac.ac_create_volume(vol)
    C = ac.ac_seed(V, stride=3.0)
    ac.ac_evolve(C, ac.default_params(ndim, 3.0 / math.sqrt(1.5), 100.0, N=64, T=4, seed=11))
    return V, ac.ac_get_state(C)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.float16, np.float32])
@pytest.mark.parametrize("ndim", [2, 3])
def test_upload_routes_agree(ac, dtype, ndim):
    import torch
    rng = np.random.default_rng(5)
    shape = (9, 23, 37) if ndim == 3 else (41, 37)        # 37 voxels per row: padded in every type
    outer = (9, 25, 44) if ndim == 3 else (41, 44)        # larger array: rows (and planes) of a view are strided
    base = (rng.random(outer) * 200).astype(dtype)
    view = base[:, :23, :37] if ndim == 3 else base[:, :37]
    dense = np.ascontiguousarray(view)
    pinned = torch.from_numpy(dense).pin_memory()
    dbase = torch.from_numpy(base).cuda()
    routes = {"host dense": dense, "host strided": view, "host pinned": pinned,
              "device dense": torch.from_numpy(dense).cuda(),
              "device strided": dbase[:, :23, :37] if ndim == 3 else dbase[:, :37]}
    states = {k: _evolve(ac, v, ndim)[1] for k, v in routes.items()}
    # an existing volume reloaded twice from dense host voxels (the kept staging
    # buffer reused), after holding other voxels
    V = ac.ac_create_volume(np.zeros_like(dense))
    ac.ac_load_volume(V, dense)
    ac.ac_load_volume(V, (dense[::-1] if ndim == 2 else dense[:, ::-1]).copy())
    ac.ac_load_volume(V, dense)
    C = ac.ac_seed(V, stride=3.0)
    ac.ac_evolve(C, ac.default_params(ndim, 3.0 / math.sqrt(1.5), 100.0, N=64, T=4, seed=11))
    states["reloaded"] = ac.ac_get_state(C)
    want = states["host dense"]
    assert np.any(want[4] != 0)
    for k, s in states.items():
        np.testing.assert_array_equal(s, want, err_msg=k)
