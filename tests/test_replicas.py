"""The multi-GPU path is replicas: every rank renders the same scene for its own
receivers, with no collective on the data path; ranks meet only to time the job (a
barrier, the slowest rank's time) and to add up the work.  These run that host logic as
two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from paper_2502_01826_gb300 import synthetic

    bench.barrier(ws)
    t = bench.max_over_ranks(1.5 + rank, ws)              # slowest rank's time
    w = bench.sum_over_ranks(100.0 * (rank + 1), ws)      # whole-job work
    cfg = bench.rank_receivers(synthetic.config_ble(K=64, n_rx=8), rank)
    out[rank] = (t, w, cfg["rx"].tobytes(), cfg["scene"]["means"].tobytes())
    dist.destroy_process_group()


def test_two_gloo_ranks_time_and_count_the_job():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        t, w, _, _ = res[r]
        assert t == 2.5          # max(1.5, 2.5) on every rank
        assert w == 300.0        # 100 + 200 on every rank
    rx0 = np.frombuffer(res[0][2], np.float32)
    rx1 = np.frombuffer(res[1][2], np.float32)
    assert not np.array_equal(rx0, rx1)            # each rank its own receivers
    assert res[0][3] == res[1][3]                  # the same scene on every rank
    from paper_2502_01826_gb300 import synthetic
    assert np.array_equal(rx0, synthetic.config_ble(K=64, n_rx=8)["rx"].ravel())  # rank 0 unchanged
    assert rx1.min() >= 0.0 and np.all(rx1.reshape(-1, 3) <= np.array(synthetic.BOX, np.float32))
