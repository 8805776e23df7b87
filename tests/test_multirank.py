"""Multi-GPU form of the benchmark on CPU: replicas with no data-path
collective, reduced once after the timed region (max time over ranks, sum of
accepted tuples), exercised with two gloo ranks."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


_CHILD = textwrap.dedent("""
    import os, sys, json
    sys.path.insert(0, sys.argv[1])
    import torch.distributed as dist
    dist.init_process_group("gloo")
    import bench
    rank = dist.get_rank()
    times = [10.0 + 5 * rank, 1.5 - rank]      # rank 1 is slower on the first, faster on the second
    acc = [100 + rank, 7 * (rank + 1)]
    w, r, l = bench._dist()
    t, a = bench.reduce_over_ranks(times, acc)
    print(json.dumps({"rank": rank, "world": w, "t": t, "a": a}))
    dist.destroy_process_group()
""")


def test_two_gloo_ranks_reduce_max_time_and_sum_accepted():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=180)
        assert p.returncode == 0, e[-2000:]
        outs.append(o.strip().splitlines()[-1])
    import json
    res = [json.loads(o) for o in outs]
    for r in res:
        assert r["world"] == 2
        assert r["t"] == [15.0, 1.5]
        assert r["a"] == [201, 21]


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    t, a = bench.reduce_over_ranks([3.0, 4.0], [5, 6])
    assert t == [3.0, 4.0] and a == [5, 6]
