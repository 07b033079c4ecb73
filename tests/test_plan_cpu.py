"""Launch layout of the brick path, on the CPU (`ac_plan_layout`: host logic, no
device work).

The layout is the GB300 form of the "Parallel Contour Evaluation" section: lanes
of a warp share a contour's samples, the contours of a brick share the brick's
staged region.  Pinned here: the default brain-3d layout, worked out by hand from
the planner's stated rules (halo, alignment, padding, shared-memory budget); the
layout rules themselves as invariants over a seeded sweep of volumes, spacings,
lattices and parameters; and the argument errors.
"""
import math

import numpy as np
import pytest

from paper_1804_06304_gb300 import ac

ES = {ac.AC_U8: 1, ac.AC_U16: 2, ac.AC_F16: 2, ac.AC_F32: 4}
SMEM_PER_SM = 233472      # bytes of shared memory per SM (228 KB)
SMEM_RESERVED = 1024      # reserved per CTA by the runtime
SMEM_PER_CTA = 232448     # largest opt-in dynamic shared memory per CTA (227 KB)


def _params(ndim, R0, N, **kw):
    return ac.default_params(ndim, R0, 1000.0, N=N, T=100, seed=1, **kw)


def test_brain3d_default_layout_by_hand():
    """1024x1024x256 u16, spacing 1:1:2, stride 6, N = 512.  8 lanes per contour
    (four contours per warp); bricks of 4x4x4 lattice cells = 24x24x12 voxels (z:
    4 cells of 6 / 2 voxels); 64 contours x 8 lanes = 16 warps, so one CTA per SM
    and a budget of 215 KB.  Halo = ceil((2.5 R0 + dR/2) / spacing) + 2 = (15, 15,
    9): the region 24 + 2*15 + 7 (x alignment slack) = 61 -> 64 voxels = 128
    bytes, padded to 72; 54; 30 -> 233,280 bytes, over the budget, so the halo
    shrinks to (14, 14, 8): 72 x 52 x 28 x 2 = 209,664 bytes."""
    R0 = 6.0 / math.sqrt(1.5)
    L = ac.ac_plan_layout(3, ac.AC_U16, (1024, 1024, 256), (1.0, 1.0, 2.0), 6.0, R0, _params(3, R0, 512))
    assert L["lanes_per_contour"] == 8 and L["warps_per_block"] == 16
    assert L["brick"] == (24, 24, 12)
    assert L["halo"] == (14, 14, 8)
    assert L["region"] == (72, 52, 28)
    assert L["smem_bytes"] == 72 * 52 * 28 * 2 == 209664


def test_sixteen_lane_layouts_and_row_padding():
    """16 lanes: 2x4x2-cell bricks (12x24x6 voxels, 16 contours, 8 warps, two CTAs
    per SM at <= 110 KB): region 12 + 28 + 7 = 47 -> 48 (96-byte rows), 52, 22 after
    one halo step.  A 24x12x6 brick instead gives 64-voxel = 128-byte rows, which
    the planner pads to 72 voxels (144 bytes); its halo shrinks to (13, 13, 7)."""
    R0 = 6.0 / math.sqrt(1.5)
    dims, sp = (1024, 1024, 256), (1.0, 1.0, 2.0)
    a = ac.ac_plan_layout(3, ac.AC_U16, dims, sp, 6.0, R0, _params(3, R0, 512, lanes_per_contour=16))
    assert (a["brick"], a["warps_per_block"], a["region"], a["smem_bytes"]) == ((12, 24, 6), 8, (48, 52, 22), 109824)
    b = ac.ac_plan_layout(3, ac.AC_U16, dims, sp, 6.0, R0, _params(3, R0, 512, lanes_per_contour=16,
                                                                   brick=(24, 12, 6)))
    assert b["region"] == (72, 38, 20) and b["halo"] == (13, 13, 7)
    assert b["smem_bytes"] == 72 * 38 * 20 * 2 <= 110 * 1024


def test_lane_defaults():
    """Lanes per contour by N: 2D 4 at N = 128 (compensated, fast sampling); 3D 32
    at N = 256, 8 at 512 <= N < 1024, 32 at N = 1024, 8 at N = 64."""
    R0 = 6.0 / math.sqrt(1.5)
    g3 = lambda N: ac.ac_plan_layout(3, ac.AC_U8, (256, 256, 128), (1, 1, 1), 6.0, R0,
                                     _params(3, R0, N))["lanes_per_contour"]
    assert [g3(N) for N in (64, 256, 512, 1000, 1024)] == [8, 32, 8, 8, 32]
    g2 = ac.ac_plan_layout(2, ac.AC_U8, (4096, 4096), (1, 1), 6.0, R0, _params(2, R0, 128))
    assert g2["lanes_per_contour"] == 4 and g2["warps_per_block"] == 10


def test_plain_path_reports_lanes_only():
    R0 = 4.0 / math.sqrt(1.5)
    L = ac.ac_plan_layout(3, ac.AC_U8, (64, 64, 32), (1, 1, 1), 4.0, R0, _params(3, R0, 256, path=ac.AC_PATH_PLAIN))
    assert L["lanes_per_contour"] == 32 and L["warps_per_block"] == 8
    assert L["brick"] == (0, 0, 0) and L["region"] == (0, 0, 0) and L["smem_bytes"] == 0


def test_layout_rules_hold_over_a_sweep():
    """Over a seeded sweep of 3D and 2D volumes (extents 8..2048, spacings 0.5..3,
    every voxel type, lattice strides 3..10, N 16..1024, default and explicit lanes,
    bricks and halo factors), every layout the planner accepts obeys its rules:
    lanes in {4, 8, 16, 32}; 1..16 warps; the region starts 16-byte aligned in x
    (its x extent a multiple of 16 bytes) and is at most 256 voxels per axis (the
    TMA box limit); a 3D region holds brick + halo in every axis (up to the volume)
    and its rows are not a multiple of 128 bytes unless they span the volume's
    rows; 3D shared memory is the region's bytes, within 110 KB when two CTAs of at
    most 8 warps share an SM (and both fit its 228 KB) and within 215 KB for one
    CTA of more warps."""
    rng = np.random.default_rng(20260)
    accepted = 0
    for trial in range(600):
        ndim = 3 if trial % 3 else 2
        dtype = int(rng.integers(0, 4))
        es = ES[dtype]
        dims = [int(v) for v in np.exp(rng.uniform(np.log(8), np.log(2048), size=ndim))]
        if ndim == 3:
            dims[2] = max(2, dims[2] // 4)
        sp = [float(v) for v in rng.choice([0.5, 1.0, 1.0, 2.0, 3.0], size=ndim)]
        stride = float(rng.uniform(3.0, 10.0))
        R0 = stride / math.sqrt(1.5)
        N = int(rng.choice([16, 64, 128, 256, 512, 700, 1024]))
        kw = {}
        if rng.random() < 0.3:
            kw["lanes_per_contour"] = int(rng.choice([8, 16, 32]))
        if rng.random() < 0.2:
            kw["brick"] = tuple(int(v) for v in rng.integers(4, 40, size=3))
        if rng.random() < 0.2:
            kw["halo_factor"] = float(rng.uniform(1.0, 4.0))
        try:
            L = ac.ac_plan_layout(ndim, dtype, dims, sp, stride, R0, _params(ndim, R0, N, **kw))
        except ac.ACError as e:
            assert e.status == ac.AC_ERR_ARG and "shared-memory budget" in str(e)
            continue
        accepted += 1
        G, W = L["lanes_per_contour"], L["warps_per_block"]
        assert G in (4, 8, 16, 32) and 1 <= W <= 16
        reg, B, h = L["region"], L["brick"], L["halo"]
        assert (reg[0] * es) % 16 == 0
        assert all(1 <= r <= 256 for r in reg)
        if ndim == 3:
            al = 16 // es
            for d in range(3):
                need = B[d] + 2 * h[d]
                assert reg[d] >= min(need, dims[d]), (d, L, dims)
            assert (reg[0] * es) % 128 != 0 or reg[0] >= dims[0], (L, dims, es)
            assert L["smem_bytes"] == reg[0] * reg[1] * reg[2] * es
            if W <= 8:
                assert L["smem_bytes"] <= 110 * 1024
                assert 2 * (L["smem_bytes"] + SMEM_RESERVED + 64) <= SMEM_PER_SM
            else:
                assert L["smem_bytes"] <= 215 * 1024
                assert L["smem_bytes"] + 64 <= SMEM_PER_CTA
            assert reg[0] % al == 0
        else:
            assert L["smem_bytes"] <= 200 * 1024
    assert accepted >= 500


@pytest.mark.parametrize("bad", [dict(ndim=4), dict(dtype=9), dict(stride=0.0), dict(r0=-1.0),
                                 dict(dims=(1, 64, 64)), dict(spacing=(1.0, 0.0, 1.0))])
def test_layout_argument_errors(bad):
    args = dict(ndim=3, dtype=ac.AC_U8, dims=(64, 64, 64), spacing=(1.0, 1.0, 1.0), stride=4.0, r0=3.0)
    args.update(bad)
    with pytest.raises(ac.ACError) as e:
        ac.ac_plan_layout(args["ndim"], args["dtype"], args["dims"], args["spacing"], args["stride"], args["r0"],
                          _params(3, 3.0, 256))
    assert e.value.status == ac.AC_ERR_ARG
