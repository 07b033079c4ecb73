"""The C ABI library builds for sm_103a, loads without a GPU, exports every entry
point include/*.h declares, and rejects invalid arguments before touching the
device.  No compute call runs here."""
import ctypes as ct
import shutil
import subprocess

import numpy as np
import pytest


@pytest.fixture(scope="module")
def ac():
    if shutil.which("nvcc") is None and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1804_06304_gb300 import ac
    ac.load()
    return ac


def test_exports_every_declared_symbol(ac):
    syms = ac.header_symbols()
    assert "ac_create_volume" in syms and "ac_localize" in syms and len(syms) >= 13
    out = subprocess.run(["nm", "-D", "--defined-only", ac.lib_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [s for s in syms if s not in exported]
    assert not missing, missing


def test_built_for_sm_103a(ac):
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", ac.lib_path()], capture_output=True,
                         text=True).stdout
    assert "sm_103a" in out


def test_argument_validation_without_device(ac):
    l = ac.load()
    out = ct.c_void_p()
    dims = (ct.c_int64 * 3)(4, 4, 4)
    sp = (ct.c_float * 3)(1, 1, 1)
    buf = np.zeros(64, np.uint8)
    ptr = ct.c_void_p(buf.ctypes.data)
    assert l.ac_create_volume(ptr, 0, 0, 4, dims, 0, 0, sp, 1.0, None, ct.byref(out)) == ac.AC_ERR_ARG
    assert l.ac_create_volume(ptr, 0, 9, 3, dims, 0, 0, sp, 1.0, None, ct.byref(out)) == ac.AC_ERR_ARG
    assert l.ac_create_volume(None, 0, 0, 3, dims, 0, 0, sp, 1.0, None, ct.byref(out)) == ac.AC_ERR_ARG
    bad = (ct.c_int64 * 3)(1, 4, 4)
    assert l.ac_create_volume(ptr, 0, 0, 3, bad, 0, 0, sp, 1.0, None, ct.byref(out)) == ac.AC_ERR_ARG
    neg = (ct.c_float * 3)(1, -1, 1)
    assert l.ac_create_volume(ptr, 0, 0, 3, dims, 0, 0, neg, 1.0, None, ct.byref(out)) == ac.AC_ERR_ARG
    assert l.ac_create_volume(ptr, 0, 0, 3, dims, 2, 0, sp, 1.0, None, ct.byref(out)) == ac.AC_ERR_ARG
    assert "stride" in ac.ac_last_error()
    assert l.ac_seed(None, None, None, 0, None, ct.byref(out)) == ac.AC_ERR_ARG
    assert l.ac_evolve(None, None, None, None) == ac.AC_ERR_ARG
    assert l.ac_evolve_batch(None, None, 0, None, None) == ac.AC_ERR_ARG
    n = ct.c_int64()
    assert l.ac_localize(None, None, None, 0, ct.byref(n), None) == ac.AC_ERR_ARG
    assert l.ac_get_state(None, None, None) == ac.AC_ERR_ARG
    assert l.ac_set_state(None, None, None) == ac.AC_ERR_ARG
    assert l.ac_philox4x32_10(None, 0, None, -1, None) == ac.AC_ERR_ARG
    assert l.ac_contour_count(None) == -1
    assert l.ac_set_wait_limits(-1, -1) == ac.AC_OK
    l.ac_destroy_volume(None)
    l.ac_destroy_contours(None)


def test_struct_layouts_match_header(ac, tmp_path):
    """The ctypes mirrors of the ABI structs match the C layout (gcc offsetof on include/ac.h)."""
    import os
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    checks = {
        "ac_evolve_params": ["N", "T", "eps0", "dR", "Rmin", "Rmax", "max_step", "seed", "stream_id", "path",
                             "lanes_per_contour", "compensated", "brick", "warps_per_block", "first_iter",
                             "update_last", "sampling", "halo_factor", "freeze_tol", "freeze_iters", "cull_iter",
                             "cull_E"],
        "ac_trace": ["device_buf", "k_begin", "k_end", "t_begin", "t_end"],
        "ac_cell": ["c", "r", "E", "id"],
        "ac_seed_params": ["stride", "R0"],
        "ac_localize_params": ["E0"],
        "ac_batch_item": ["stream_id", "first_iter", "n_iter", "update_last"],
        "ac_layout": ["lanes_per_contour", "warps_per_block", "brick", "halo", "region", "smem_bytes"],
        "ac_server_params": ["evolve", "dtype", "ndim", "stride", "R0", "E0", "iters_per_round", "max_resident",
                             "hbm_budget_bytes", "max_resident_contours", "balance_rounds"],
        "ac_tile_result": ["ticket", "status", "rounds", "n_cells", "contours", "voxels", "est_bytes", "queue_ms",
                           "run_ms", "total_ms"],
        "ac_server_stats": ["pending", "resident", "finished", "completed", "failed", "rounds", "resident_bytes",
                            "peak_resident_bytes", "budget_bytes"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ac_serve.h"', "int main(void){"]
    for st, fields in checks.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f in fields:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", inc, "-o", str(exe), str(src)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        st, f, v = line.split()
        got[(st, f)] = int(v)
    for st, fields in checks.items():
        cls = getattr(ac, st)
        assert ct.sizeof(cls) == got[(st, "size")], st
        for f in fields:
            assert getattr(cls, f).offset == got[(st, f)], (st, f)


def test_server_argument_validation_without_device(ac):
    """ac_server_create checks every parameter before touching the device."""
    l = ac.load()
    good = ac.default_params(3, 4.0, 170.0, N=64, T=4)

    def params(**kw):
        sp = ac.ac_server_params()
        sp.evolve = good.to_c()
        sp.dtype, sp.ndim, sp.stride, sp.R0, sp.E0 = ac.AC_U8, 3, 4.0, 0.0, -10.0
        sp.iters_per_round, sp.max_resident, sp.hbm_budget_bytes = 5, 0, 1 << 30
        for k, v in kw.items():
            if k == "N":
                sp.evolve.N = v
            else:
                setattr(sp, k, v)
        return sp

    out = ct.c_void_p()
    for bad in [dict(dtype=7), dict(ndim=4), dict(stride=0.0), dict(R0=-1.0), dict(E0=float("nan")),
                dict(iters_per_round=0), dict(max_resident=-1), dict(hbm_budget_bytes=0), dict(N=0),
                dict(max_resident_contours=-5), dict(balance_rounds=2)]:
        sp = params(**bad)
        assert l.ac_server_create(ct.byref(sp), ct.byref(out)) == ac.AC_ERR_ARG, bad
        assert not out.value
    assert l.ac_server_create(None, ct.byref(out)) == ac.AC_ERR_ARG
    t = ct.c_int64()
    dims = (ct.c_int64 * 3)(4, 4, 4)
    sp3 = (ct.c_float * 3)(1, 1, 1)
    assert l.ac_server_submit(None, None, dims, 0, 0, sp3, 1.0, 0, ct.byref(t)) == ac.AC_ERR_ARG
    r = ac.ac_tile_result()
    assert l.ac_server_wait(None, 1, 0.0, None, 0, ct.byref(r)) == ac.AC_ERR_ARG
    st = ac.ac_server_stats()
    assert l.ac_server_get_stats(None, ct.byref(st)) == ac.AC_ERR_ARG
    l.ac_server_destroy(None)
    assert l.ac_plan_rebind(None, None, None, 0, None) == ac.AC_ERR_ARG


def test_static_path_rejects_grid_and_rules_without_device(ac):
    l = ac.load()
    dims = (ct.c_int64 * 3)(8, 8, 8)
    sp = (ct.c_float * 3)(1, 1, 1)
    fake = ct.c_void_p(0x1000)   # never dereferenced: the arguments are refused first
    for kw in (dict(path=ac.AC_PATH_GRID), dict(freeze_iters=2, freeze_tol=0.1), dict(cull_iter=3)):
        p = ac.default_params(3, 3.0, 100.0, N=64, T=4, **kw).to_c()
        assert l.ac_evolve_static(fake, 0, 3, dims, 0, 0, sp, 1.0, fake, 8, 3.0, 4.0, ct.byref(p), None) == \
            ac.AC_ERR_ARG, kw
    for kw in (dict(freeze_tol=-1.0), dict(freeze_iters=-1), dict(cull_iter=-2), dict(cull_E=float("nan")),
               dict(path=3), dict(path=ac.AC_PATH_GRID, lanes_per_contour=32)):
        p = ac.default_params(3, 3.0, 100.0, N=64, T=4, **kw).to_c()
        assert l.ac_evolve_static(fake, 0, 3, dims, 0, 0, sp, 1.0, fake, 8, 3.0, 4.0, ct.byref(p), None) == \
            ac.AC_ERR_ARG, kw
