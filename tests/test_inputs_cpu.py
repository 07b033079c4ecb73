"""Host-side pieces of the measurement, on CPU: the seeded input generators are
reproducible and follow their stated shapes, bench.py's lattice count agrees with
the oracle's lattice, and the clock sampler turns nvidia-smi rows into the clocks
record (median SM clock, max clock, throttle reasons)."""
import os
import sys
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_generators_are_seeded_and_shaped():
    from paper_1804_06304_gb300 import synth
    a, b, c = synth.small_3d(0), synth.small_3d(0), synth.small_3d(1)
    assert a.volume.shape == (32, 64, 64) and a.volume.dtype == np.uint8 and len(a.centres) == 20
    assert np.array_equal(a.volume, b.volume) and not np.array_equal(a.volume, c.volume)
    l2 = synth.large_2d(1, shape=(256, 192), n_nuclei=40)
    assert l2.volume.shape == (192, 256) and l2.volume.dtype == np.uint8 and l2.ndim == 2
    assert np.array_equal(l2.volume, synth.large_2d(1, shape=(256, 192), n_nuclei=40).volume)
    br = synth.brain_3d(2, shape=(64, 48, 16), n_nuclei=30)
    assert br.volume.shape == (16, 48, 64) and br.volume.dtype == np.uint16 and br.spacing == (1.0, 1.0, 2.0)
    assert br.volume_f16 is not None and br.volume_f16.dtype == np.float16
    vols = synth.batch_3d(3, count=4, max_scale=0.2)
    assert len(vols) == 4 and all(v.volume.dtype == np.uint8 for v in vols)
    assert all(64 <= v.volume.shape[2] <= 64 * 8 ** 0.2 + 1 for v in vols)
    tiles = synth.tile_stream(4, count=3, max_scale=0.1)
    times = [t for t, _ in tiles]
    assert times == sorted(times) and all(s.volume.dtype == np.uint16 for _, s in tiles)


@pytest.mark.parametrize("shape,spacing,stride,ndim", [((64, 64, 32), (1.0, 1.0, 1.0), 4.0, 3),
                                                        ((97, 53, 1), (1.0, 1.0, 1.0), 6.0, 2),
                                                        ((90, 70, 40), (1.0, 1.0, 2.0), 6.0, 3),
                                                        ((5, 3, 2), (0.5, 0.5, 1.0), 4.0, 3)])
def test_lattice_count_matches_oracle(shape, spacing, stride, ndim):
    import bench
    from oracle import oracle
    assert bench.lattice_count(shape, spacing, stride, ndim) == len(oracle.seed_lattice(ndim, shape, spacing, stride))


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler_with_rows(rows):
    import bench
    cs = bench.ClockSampler(None)
    cs.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    cs.out.write("\n".join(rows) + "\n")
    cs.proc = _FakeProc()
    return cs


def test_clock_sampler_summary():
    ok = _sampler_with_rows(["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
                             "0, 2055, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
                             "0, 2070, 2070, 1210.5, 0x0, Not Active, Not Active, Not Active, Not Active",
                             "garbage line"]).stop()
    assert ok == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = _sampler_with_rows(["0, 1500, 2070, 1300, 0x40, Not Active, Active, Not Active, Not Active"]).stop()
    assert hot["reasons"] == ["hw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert _sampler_with_rows([]).stop() is None
