"""The multi-GPU path is replicas over disjoint trajectory-id ranges (no
collective on the data path); only the timing reduction crosses ranks.  Two
gloo ranks on CPU check (a) the bench's max/sum reductions and barrier and
(b) that per-rank id ranges reproduce the single-process ensemble exactly."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_per_rank, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    from paper_2605_00479_gb300 import presets as P

    class Args:
        gpus = world
    w, r, _ = bench.dist_setup(Args)
    assert (w, r) == (world, rank)
    bench.barrier(w)
    assert bench.max_over_ranks(w, float(rank + 1)) == float(world)
    assert bench.sum_over_ranks(w, 1.5) == 1.5 * world
    m = P.telegraph(0.3, 0.2, 10.0, 1.0)
    res = oracle.run(m, P.TELEGRAPH_X0, n_per_rank, 5.0, [2.5, 5.0], "uniform_bf16", "sr", seed=9,
                     g0=rank * n_per_rank)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), res["snapshots"])
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_trajectory_ids(tmp_path):
    world, n = 2, 24
    mp.start_processes(_worker, args=(world, _free_port(), n, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    import oracle
    from paper_2605_00479_gb300 import presets as P
    whole = oracle.run(P.telegraph(0.3, 0.2, 10.0, 1.0), P.TELEGRAPH_X0, world * n, 5.0, [2.5, 5.0],
                       "uniform_bf16", "sr", seed=9)["snapshots"]
    parts = np.concatenate([np.load(tmp_path / f"rank{r}.npy") for r in range(world)], axis=2)
    np.testing.assert_array_equal(parts, whole)


def _worker_ext(rank, world, port, n_per_rank, out_dir):
    """Tau-leaping and RDME ranks: disjoint id ranges, timing reductions only."""
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    from paper_2605_00479_gb300 import presets as P

    class Args:
        gpus = world
    w, r, _ = bench.dist_setup(Args)
    assert bench.max_over_ranks(w, 2.0 * rank) == 2.0 * (world - 1)
    tau = oracle.tau_run(P.dimer(), P.dimer_x0(300), n_per_rank, 5.0, 0.1, [2.5, 5.0], "mixed_bf16", "sr", seed=4,
                         g0=rank * n_per_rank)
    x0 = np.zeros((4, 2), np.int32)
    x0[0, 0] = 40
    rd = oracle.rdme_run(P.dimer(2e-2, 0.1), (2, 2), [0.5, 0.2], x0, n_per_rank, 2.0, [1.0, 2.0], "uniform_f16", "sr",
                         seed=4, g0=rank * n_per_rank)
    np.save(os.path.join(out_dir, f"tau{rank}.npy"), tau["snapshots"])
    np.save(os.path.join(out_dir, f"rdme{rank}.npy"), rd["snapshots"])
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_tau_and_rdme(tmp_path):
    world, n = 2, 20
    mp.start_processes(_worker_ext, args=(world, _free_port(), n, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    import oracle
    from paper_2605_00479_gb300 import presets as P
    tau = oracle.tau_run(P.dimer(), P.dimer_x0(300), world * n, 5.0, 0.1, [2.5, 5.0], "mixed_bf16", "sr",
                         seed=4)["snapshots"]
    x0 = np.zeros((4, 2), np.int32)
    x0[0, 0] = 40
    rd = oracle.rdme_run(P.dimer(2e-2, 0.1), (2, 2), [0.5, 0.2], x0, world * n, 2.0, [1.0, 2.0], "uniform_f16", "sr",
                         seed=4)["snapshots"]
    np.testing.assert_array_equal(np.concatenate([np.load(tmp_path / f"tau{r}.npy") for r in range(world)], axis=2),
                                  tau)
    np.testing.assert_array_equal(np.concatenate([np.load(tmp_path / f"rdme{r}.npy") for r in range(world)], axis=3),
                                  rd)
