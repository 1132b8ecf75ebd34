"""The multi-rank path on CPU (gloo, world size 2): each rank takes its
event shard, computes its accumulators (with the oracle here, as there is no
GPU), and the one exchange -- a sum of the accumulators and histogram bins --
reproduces the single-process result over the whole range."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_per_rank, out_path):
    import torch.distributed as dist

    import oracle
    from paper_1002_3446_gb300 import dist as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    proc = oracle.process(6, hist_obs=1, hist_bins=12, hist_lo=100.0, hist_hi=1300.0)
    first, count = tdist.event_range(rank, world, n_per_rank, first=1000)
    r = oracle.generate(proc, 7, first, count, threads=1, per_event=False)
    acc = torch.zeros(8, dtype=torch.float64)
    acc[:4] = torch.tensor(r["acc"])
    hist = torch.tensor(np.concatenate([r["hist_w"], r["hist_w2"]]))
    tdist.reduce_sums(acc, hist)
    if rank == 0:
        np.save(out_path, np.concatenate([acc.numpy(), hist.numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_equals_single_process(tmp_path, orc):
    import torch.multiprocessing as mp
    world, n_per_rank = 2, 3000
    out = str(tmp_path / "r0.npy")
    mp.start_processes(_worker, args=(world, _free_port(), n_per_rank, out), nprocs=world, start_method="spawn")
    got = np.load(out)
    proc = orc.process(6, hist_obs=1, hist_bins=12, hist_lo=100.0, hist_hi=1300.0)
    ref = orc.generate(proc, 7, 1000, world * n_per_rank, threads=1, per_event=False)
    assert np.allclose(got[:4], ref["acc"], rtol=1e-13)
    assert np.allclose(got[8:], np.concatenate([ref["hist_w"], ref["hist_w2"]]), rtol=1e-12, atol=0)
    from paper_1002_3446_gb300 import dist as tdist
    assert np.isclose(tdist.sigma_from_acc(got[:8])[0], orc.sigma(ref["acc"])[0], rtol=1e-13)


def test_event_range():
    from paper_1002_3446_gb300 import dist as tdist
    assert tdist.event_range(0, 4, 100) == (0, 100)
    assert tdist.event_range(3, 4, 100, first=5) == (305, 100)
    with pytest.raises(ValueError):
        tdist.event_range(4, 4, 100)
