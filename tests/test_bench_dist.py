"""The N > 1 plumbing of bench.py on CPU ranks (gloo, world size 2).

bench.py runs one independent replica per rank ("replicas only": the path
does not shard); ranks exchange nothing but a barrier and the max of their
timings. These tests run that plumbing on two CPU processes.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    from rve_inputs import neo_hookean_config

    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    m = bench.max_over_ranks(w, float(10 * rank + 1), torch.device("cpu"))
    phase, _, _ = neo_hookean_config(24, seed=rank)
    np.save(os.path.join(out_dir, f"phase{rank}.npy"), phase)
    with open(os.path.join(out_dir, f"max{rank}.txt"), "w") as f:
        f.write(repr(m))
    bench.barrier(w)
    dist.destroy_process_group()


def test_replicas_barrier_and_max_over_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    assert float(open(tmp_path / "max0.txt").read()) == 11.0
    assert float(open(tmp_path / "max1.txt").read()) == 11.0
    p0, p1 = np.load(tmp_path / "phase0.npy"), np.load(tmp_path / "phase1.npy")
    assert p0.shape == p1.shape and not np.array_equal(p0, p1)  # each replica its own microstructure


def _ref_worker(rank, world, port, out_dir):
    import contextlib
    import io
    import sys

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench

    buf = io.StringIO()
    sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
    counts_missing = bench.reference_counts() is None
    with contextlib.redirect_stdout(buf):
        if rank != 0 or counts_missing:
            bench.main()
    with open(os.path.join(out_dir, f"ref{rank}.txt"), "w") as f:
        f.write(buf.getvalue())


def test_reference_arm_prints_on_rank_zero_only(tmp_path):
    port = _free_port()
    mp.spawn(_ref_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    assert open(tmp_path / "ref1.txt").read() == ""
