"""The N > 1 host path of bench.py on CPU, as two gloo ranks (no GPU): the slowest rank's time
is taken on every rank, whole-job throughput counts every rank's slice, each rank gets its own
slice, and the reference arm runs on rank 0 only."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = bench.dist_info()
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, w)         # rank 1 is the slow one
        ms2 = bench.max_over_ranks(7.0 if rank == 0 else 3.0, w)  # called in the same order everywhere
        value = bench.weak_scaling_value(w, 2.0e9, 4, ms)
        from paper_2211_07532_gb300 import synth
        seed = synth.BASE_SEED + 1000 * 2 + r                     # slice_200(index=rank)'s seed
        q.put((r, w, loc, ms, ms2, value, seed))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, ms, ms2, value, seed) in enumerate(out):
        assert (rank, world, local) == (r, 2, r)
        assert ms == 150.0 and ms2 == 7.0                  # the max over both ranks, on both ranks
        assert value == pytest.approx(2 * 2.0e9 * 4 / 0.150 / 1e9)
    assert out[0][6] != out[1][6]                           # one slice per rank


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.weak_scaling_value(1, 1e9, 2, 1000.0) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, ref_seconds = 1, 0, 0.01
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""


def test_launch_count_matches_the_measured_launch_lists():
    """`gpu_launches` counts the kernels of one solve; the counts per form are those of the ncu
    launch lists of one 200^2 / J = 4 / 30 power + 50 FISTA solve (profiles/launches_slice200_*.md,
    without the simulation's forward): FP32 620, BF16 625, FP16 hi+lo 1028."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.launches_per_recon(4, 50, 30, "fp32", 200, 200) == 620
    assert bench.launches_per_recon(4, 50, 30, "bf16", 200, 200) == 625
    assert bench.launches_per_recon(4, 50, 30, "fp16x2", 200, 200) == 1028
    # images whose level-1 approximation exceeds the middle-level kernel: one launch per level each way
    assert (bench.launches_per_recon(4, 50, 30, "fp32", 512, 512)
            - bench.launches_per_recon(4, 50, 30, "fp32", 200, 200)) == 50 * (8 - 3)
