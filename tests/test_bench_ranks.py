"""bench.py on CPU.  The replica path: two gloo ranks on 127.0.0.1, each
with its own time; the job's time is the slowest rank's and the value counts
the generations of every rank.  The reference arm: its JSON line."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    got = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (got, bench.replica_value(world, 100, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (20.0, 2 * 100 / 0.020)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.replica_value(1, 10, 2.0) == 5000.0


def test_reference_arm_json_line_on_cpu():
    """bench.py --impl reference (the FP64 oracle on the host cores) prints
    one JSON line with the contract's keys, here on the small workload."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "dtlz2_m3_d12_N105", "--steps", "3", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, check=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "steps", "warmup", "higher_is_better",
                "cpu_baseline", "e2e", "config"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["workload"] == "dtlz2_m3_d12_N105"


def test_operator_workloads_bytes_and_oracle_params():
    """The operator workloads' algorithmic bytes per generation (rows of d
    float32 read and written per offspring, as the kernels' definitions
    fix them) and the oracle parameters each maps to."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle as orc
    N, d, row = 9870, 5000, 5000 * 4
    W = bench.WORKLOADS
    assert bench.repro_bytes(W["dtlz1_m3_d5000_N9870"]) == (2 * 4935 + N) * row
    assert bench.repro_bytes(W["de_dtlz1_m3_d5000_N9870"]) == 5 * N * row
    assert bench.repro_bytes(W["random_dtlz1_m3_d5000_N9870"]) == N * row
    assert bench.repro_bytes(W["cso_dtlz1_m3_d5000_N9870"]) == 6 * N * row    # phi > 0: the centre
    assert bench.repro_bytes(dict(W["cso_dtlz1_m3_d5000_N9870"], cso_phi=0.0)) == 5 * N * row
    assert bench.repro_bytes(W["pso_dtlz1_m3_d5000_N9870"]) == 7 * N * row
    for name, op in (("dtlz1_m3_d5000_N9870", orc.OP_SBX_PM), ("de_dtlz1_m3_d5000_N9870", orc.OP_DE),
                     ("random_dtlz1_m3_d5000_N9870", orc.OP_RANDOM),
                     ("cso_dtlz1_m3_d5000_N9870", orc.OP_CSO), ("pso_dtlz1_m3_d5000_N9870", orc.OP_PSO)):
        p = bench.oracle_params(orc, W[name])
        assert p.op == op and (p.N, p.d, p.m, p.H, p.problem) == (N, d, 3, 139, 1)
    assert abs(bench.oracle_params(orc, W["cso_dtlz1_m3_d5000_N9870"]).cso_phi - 0.1) < 1e-12
    p = bench.oracle_params(orc, W["pso_dtlz1_m3_d5000_N9870"])
    assert (p.pso_w, p.pso_c1, p.pso_c2) == (0.7298, 1.49618, 1.49618)
    assert set(bench.OPS) == {0, 1, 2, 3, 4}
