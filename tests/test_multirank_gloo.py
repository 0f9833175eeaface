"""The N > 1 host logic of bench.py on CPU: two gloo ranks (127.0.0.1), each with its own
seeded problem (weak scaling, no data-path exchange). Checks the per-rank seeds give
distinct inputs, that the slowest rank's time and the summed report counters come back to
every rank, and that the whole-job value counts the work of all ranks. Each rank also runs
the CPU oracle on its own small shard with one injected fault; the combined counters equal
the sum of the shards' reports."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as d

    import bench
    import oracle as O
    import synth as S
    d.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 24
        A, B, Cin = bench.gen_inputs(n, bench.rank_seed(rank))
        # rank-local oracle run of the shard with one accumulator flip in tile (rank, 0)
        inj = [dict(i=8 * rank + 1, j=2, site=O.SITE_ACCUM, mode=O.MODE_BITFLIP, bit=55)]
        _, rep = O.ft_gemm(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, n, n, n, 1.5, A, n, B, n, 0.5, Cin, n, 8, 8, 4,
                           injections=inj)
        local = dict(detected=int(rep.detected), corrected=int(rep.corrected), tiles_checked=int(rep.tiles_checked))
        summed = bench.sum_over_ranks(local, d)
        slowest = bench.max_over_ranks(10.0 + rank, d)
        status = bench.or_over_ranks(1 << rank, d)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([A[:5].tolist() + [summed["detected"], summed["corrected"], summed["tiles_checked"], slowest,
                                            status]], dtype=np.float64))
    finally:
        d.destroy_process_group()


def test_two_gloo_ranks_shard_and_combine(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "r0.npy")[0]
    r1 = np.load(tmp_path / "r1.npy")[0]
    assert not np.array_equal(r0[:5], r1[:5])          # distinct seeded problems per rank
    assert np.array_equal(r0[5:], r1[5:])              # every rank holds the combined values
    detected, corrected, tiles, slowest, status = r0[5:]
    assert (detected, corrected, tiles) == (2, 2, 2 * 9)  # one fault per shard, 3 x 3 tiles each
    assert slowest == 11.0 and status == 3
    import bench
    assert bench.job_tflops(2, 2.0e12, 3, 1000.0) == pytest.approx(12.0)  # 2 ranks x 3 steps x 2 TFLOP / 1 s


def test_collectives_in_the_gpu_arm_are_reached_by_every_rank():
    """Every call in bench.run_ours that synchronises the ranks (directly or through the
    timed helpers) must sit outside any branch that depends on the rank; a rank-0-only
    section that reached a barrier would leave the others gone and rank 0 waiting."""
    import ast
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py")).read()
    run_ours = next(n for n in ast.parse(src).body if isinstance(n, ast.FunctionDef) and n.name == "run_ours")
    syncing = {"barrier", "timed", "measure_e2e", "max_over_ranks", "sum_over_ranks", "or_over_ranks"}
    # nested helpers that synchronise must not be called under a rank test either
    bad = []

    def visit(node, under_rank):
        if isinstance(node, ast.If):
            names = {x.id for x in ast.walk(node.test) if isinstance(x, ast.Name)}
            for child in node.body + node.orelse:
                visit(child, under_rank or "rank" in names)
            return
        if isinstance(node, ast.Call) and isinstance(node.func, ast.Name) and node.func.id in syncing and under_rank:
            bad.append(node.lineno)
        for child in ast.iter_child_nodes(node):
            visit(child, under_rank)

    for stmt in run_ours.body:
        visit(stmt, False)
    assert not bad, f"rank-dependent synchronising calls at bench.py lines {bad}"
