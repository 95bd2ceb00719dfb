"""The N-replica path of bench.py on CPU: two gloo ranks (world size 2) through the same
environment parsing, process-group setup, barrier and max-over-ranks timing the GPU run
uses under torchrun; the reference arm runs on rank 0 only."""
import json
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as td
    ws, r, local = bench.dist_env()
    bench.dist_init(ws)
    bench.barrier(ws)
    # rank 1 is the slow replica: the job's time is its time, the rate counts both ranks' units
    value, ms = bench.replica_rate(ws, 1000.0, 10.0 if r == 0 else 25.0)

    class Args:
        cpu_window, warmup, steps = 8, 0, 1

    ref = bench.run_reference(Args, ws, r) if r == 1 else "skipped"
    json.dump({"ws": ws, "rank": r, "local": local, "value": value, "ms": ms, "ref": ref},
              open(os.path.join(out_dir, f"rank{r}.json"), "w"))
    bench.barrier(ws)
    td.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    mp.spawn(_rank, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in (0, 1)]
    for r, d in enumerate(res):
        assert d["ws"] == 2 and d["rank"] == r and d["local"] == r
        assert d["ms"] == 25.0                          # max over ranks
        assert abs(d["value"] - 2 * 1000.0 / 0.025) < 1e-6
    assert res[1]["ref"] is None                        # only rank 0 runs the reference arm
