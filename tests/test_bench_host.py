"""Host-side logic of bench.py on CPU: argument defaults, the cross-rank
reduction (world_size 2, gloo) and the reference arm's JSON contract."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, n = bench.reduce_over_ranks(10.0 + 5.0 * rank, 3 + rank, world, "cpu")
    q.put((rank, ms, n))
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, n in got:
        assert ms == 15.0 and n == 7       # max of times, sum of launches


def test_defaults_finish_quickly():
    import bench
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.workload == "batch64"


def test_reference_arm_json_contract():
    """The reference arm times the oracle on the host; tiny run on CPU."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "cavity65", "--steps", "3", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_kernel_digest_changes_with_source(tmp_path):
    import bench
    d1 = bench.kernel_source_digest("fused")
    assert len(d1) == 16 and d1 == bench.kernel_source_digest("fused")
    assert d1 != bench.kernel_source_digest("collide")


def test_quad_workload_cavities_are_convex_and_seeded():
    import oracle as O
    from paper_2306_07603_gb300.workloads import quad257
    a, b = quad257(), quad257()
    assert a == b and len(a) == 10
    for sp in a:
        g = O.quad_grid(9, 9, sp.corners)      # raises unless J > 0 everywhere
        assert g.J.min() > 0.3


def test_oracle_pool_runs_every_cavity_on_several_processes():
    """The reference arm's oracle pool: spawned single-threaded processes, each
    advancing its group of cavities; whole-job throughput over all of them."""
    import bench
    from paper_2306_07603_gb300.workloads import CavitySpec
    specs = [CavitySpec(17, 17, 100.0, 0.75, 60.0), CavitySpec(21, 17, 400.0, 1.25, 45.0),
             CavitySpec(17, 23, 100.0, 1.0, 90.0)]
    mlups, wall, used = bench.oracle_pool_mlups(specs, 1, 3, 2)
    assert used == 2 and wall > 0 and mlups > 0
    assert mlups == pytest.approx(sum(sp.nodes for sp in specs) * 3 / wall / 1e6)
