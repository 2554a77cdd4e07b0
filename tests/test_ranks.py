"""The multi-rank host paths of bench.py on the CPU: how independent problems are split
between ranks, the reductions of timings and counts over a gloo process group of two
ranks, and a two-rank torchrun launch of the reference arm (only rank 0 reports)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n", [0, 1, 7, 256, 257])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shards_cover_every_item_once(n, world):
    parts = [list(bench.shard(n, r, world)) for r in range(world)]
    assert sorted(x for p in parts for x in p) == list(range(n))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1
    for p in parts:  # contiguous
        if p:
            assert p == list(range(p[0], p[0] + len(p)))
    rr = [bench.round_robin(n, r, world) for r in range(world)]
    assert sorted(x for p in rr for x in p) == list(range(n))
    assert all(x % world == r for r, p in enumerate(rr) for x in p)


def test_reductions_without_a_process_group():
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.sum_over_ranks(2, None, None) == 2.0
    assert bench.gather_lists([1, 2], None) == [1, 2]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = dict(
            mx=bench.max_over_ranks(1.5 + rank, dist, "cpu"),
            sm=bench.sum_over_ranks(10 * (rank + 1), dist, "cpu"),
            gl=bench.gather_lists([rank] * (rank + 1), dist),
            mine=list(bench.shard(5, rank, world)),
        )
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_reductions_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, g in enumerate(got):
        assert g["mx"] == 2.5                 # the slowest rank's time, on every rank
        assert g["sm"] == 30.0                # units summed over the ranks
        assert g["gl"] == [0, 1, 1]           # per-request values, rank order
    assert got[0]["mine"] + got[1]["mine"] == [0, 1, 2, 3, 4]


def test_reference_arm_under_torchrun_reports_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(line) for line in p.stdout.splitlines() if line.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_timeline_downsampling_keeps_the_ends():
    pts = [(0.01 * i, 10 * i) for i in range(100)]
    out = bench._downsample(pts, 5)
    assert len(out) == 5 and out[0] == [0.0, 0] and out[-1] == [0.99, 990]
    assert bench._downsample(pts[:3], 40) == [[0.0, 0], [0.01, 10], [0.02, 20]]
    assert bench._downsample([], 40) == []


def _slab_rank_main(rank, world, port, out_dir, ny):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2212_10680_gb300 import fmlbm
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        y0, rows = fmlbm.fmlbm_decomp_slab_rows(ny, world, rank)      # host-only: no GPU
        parts = [None] * world
        dist.all_gather_object(parts, (y0, rows))
        with open(os.path.join(out_dir, f"slab{rank}.json"), "w") as f:
            json.dump(dict(mine=[y0, rows], all=parts), f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,ny", [(2, 64), (2, 6), (3, 36)])
def test_slab_rows_over_gloo_ranks(tmp_path, world, ny):
    # one y-slab of a decomposed lattice per rank: the slabs cover the rows once, in rank
    # order, and the three ghost rows below and above a rank's slab are the boundary rows of
    # ranks r - 1 and r + 1 (periodic), which the halo exchange brings in
    import torch.multiprocessing as mp
    mp.start_processes(_slab_rank_main, args=(world, _free_port(), str(tmp_path), ny), nprocs=world, join=True,
                       start_method="spawn")
    got = [json.load(open(tmp_path / f"slab{r}.json")) for r in range(world)]
    parts = [tuple(p) for p in got[0]["all"]]
    assert all([tuple(p) for p in g["all"]] == parts for g in got)
    owner = {}
    for r, (y0, rows) in enumerate(parts):
        assert tuple(got[r]["mine"]) == (y0, rows)
        for y in range(y0, y0 + rows):
            assert y not in owner
            owner[y] = r
    assert sorted(owner) == list(range(ny))
    for r, (y0, rows) in enumerate(parts):
        below = [(y0 - k) % ny for k in (3, 2, 1)]
        above = [(y0 + rows + k) % ny for k in (0, 1, 2)]
        assert {owner[y] for y in below} == {(r - 1) % world}
        assert {owner[y] for y in above} == {(r + 1) % world}
