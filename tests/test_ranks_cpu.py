"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): images are
independent replicas, so ranks exchange nothing but the step time, whose maximum
sets the whole-job throughput.  The reference arm under torchrun prints one line
from rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [10.0, 12.0] if rank == 0 else [30.0, 34.0]
    t, v = bench.aggregate_ranks(local, 1000, world, bench.torch_max_reducer("cpu"))
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 32.0                          # max over ranks of the mean step time
        assert abs(v - 2 * 1000 / 0.032) < 1e-6   # world x per-rank samples / max time


def test_single_rank_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    t, v = bench.aggregate_ranks([2.0, 4.0], 500, 1)
    assert t == 3.0 and abs(v - 500 / 0.003) < 1e-6


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_once():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", "29517", "bench.py", "--impl", "reference",
                        "--workload", "small-3d", "--steps", "1", "--warmup", "0", "--gpus", "2"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_oracle_check_measures_centre_error_in_voxels():
    """The bench's oracle check: identical states give zero error; a centre shifted
    by 0.5 physical units along an axis of spacing 2 is 0.25 voxel off."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(3)
    C = 50
    state = rng.uniform(1, 20, size=(5, C)).astype(np.float32)
    idx = np.array([3, 7, 11, 40])
    cR = state[:4, idx].T.astype(np.float64)
    E = state[4, idx].astype(np.float64)
    ok = bench.oracle_check(state, idx, cR, E, (1.0, 1.0, 2.0), 3)
    assert ok["contours"] == 4 and ok["centre_err_voxels"]["max"] == 0.0
    assert ok["frac_centre_within_0.25_voxel"] == 1.0 and ok["radius_err_max"] == 0.0
    moved = state.copy()
    moved[2, 11] += 0.5
    moved[0, 40] += 0.6
    chk = bench.oracle_check(moved, idx, cR, E, (1.0, 1.0, 2.0), 3)
    assert abs(chk["centre_err_voxels"]["max"] - 0.6) < 1e-5
    assert chk["frac_centre_within_0.25_voxel"] == 0.75      # 0.25 voxel passes, 0.6 does not
    conv = bench.oracle_check(moved, idx, cR, E, (1.0, 1.0, 2.0), 3, E0=float(np.sort(E)[2]))
    assert conv["converged"]["contours"] == 2


def test_oracle_check_detection_agreement():
    """The bench's detection-set agreement: the oracle's own localization of its
    states against given cells, one-to-one within 0.5 voxel (anisotropic spacing)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle
    # three well separated contours, all below E0; the GPU side finds two of them,
    # one shifted by 0.4 voxel along z (0.8 physical units at spacing 2)
    cR = np.array([[10.0, 10.0, 10.0, 3.0], [30.0, 10.0, 10.0, 3.0], [10.0, 30.0, 20.0, 3.0]])
    E = np.array([-5.0, -4.0, -3.0])
    state = np.vstack([cR.T, E]).astype(np.float32)
    idx = np.arange(3)
    cells = np.array([[10.0, 10.0, 10.8], [30.0, 10.0, 10.0]])
    chk = bench.oracle_check(state, idx, cR, E, (1.0, 1.0, 2.0), 3, E0=-1.0, gpu_cells=cells)
    assert list(oracle.localize(3, cR, E, -1.0)) == [0, 1, 2]
    assert chk["detections"] == {"gpu": 2, "oracle": 3, "matched": 2, "agreement": 0.8}
    far = np.array([[10.0, 10.0, 12.2], [30.0, 10.0, 10.0], [10.0, 30.0, 20.0]])   # 1.1 voxel off in z
    assert bench.oracle_check(state, idx, cR, E, (1.0, 1.0, 2.0), 3, E0=-1.0,
                              gpu_cells=far)["detections"]["matched"] == 2
