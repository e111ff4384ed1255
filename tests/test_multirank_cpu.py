"""The N > 1 launch of bench.py on CPU: two gloo ranks (world size 2, 127.0.0.1), no GPU.
The path does not shard (independent replicas), so what is checked is the host logic the
multi-GPU run relies on: the rendezvous, the barrier, the max-over-ranks timing, distinct
replica problems per rank, the whole-job aggregate, and that the reference arm runs on
rank 0 only."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    from paper_2305_09044_gb300 import synth
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    bench._init_dist(w)
    bench._barrier(w)
    # each rank reports a different time; every rank must see the maximum
    mx = bench._max_over_ranks(10.0 + 5.0 * rank, w)
    wl = bench.replica_workload(synth.WORKLOADS["tiny3"], r, w)
    # the reference arm returns at once on ranks other than 0 (no oracle work there)
    printed = None
    if r != 0:
        import contextlib
        import io
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            class A:
                steps, warmup = 1, 1
            bench.run_reference(A(), r, w)
        printed = buf.getvalue()
    bench._barrier(w)
    bench._pg.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"max": mx, "data_seed": wl.data_seed, "init_seed": wl.init_seed, "printed": printed}, f)


def test_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert res[0]["max"] == res[1]["max"] == 15.0
    assert res[0]["data_seed"] != res[1]["data_seed"] and res[0]["init_seed"] != res[1]["init_seed"]
    assert res[1]["printed"] == ""


def test_job_throughput_and_single_rank_workload():
    import bench
    from paper_2305_09044_gb300 import synth
    w = synth.WORKLOADS["tiny3"]
    assert bench.replica_workload(w, 0, 1) is w
    # two ranks of 4e8 slots per step, 3 steps, slowest rank 12 ms -> 2 * 4e8 * 3 / 0.012
    assert bench.job_throughput(2, 4e8, 3, 12.0) == pytest.approx(2e11)
