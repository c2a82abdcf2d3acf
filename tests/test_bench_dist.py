"""Multi-process paths of bench.py on CPU (gloo, world size 2): the max-over-ranks reduction
and the reference arm under torchrun (rank 0 prints one JSON line, the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out = bench.max_over_ranks(dist, [1.0 + rank, 10.0 - rank], "cpu")
    q.put((rank, out))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 10.0]


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--workload", "two_atom_24", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["value"] > 0


def test_probe_grids_and_pipe_flop_count():
    # host logic of the probe modes: --grid G or n1,n2,n3 keeps the cell and replaces the grid;
    # the tensor-pipe flop count of the BF16x3 GEMMs as the kernels tile them (three split
    # products; 128-row tiles; Gram column tiles rounded up to 16 and stacked [Y; HY], upper
    # triangle only; rotation blocks of at most 256 columns)
    import bench
    c = bench.cell_for("lattice216_120", "120,40,40")
    assert c.n == (120, 40, 40) and c.natom == 216
    assert bench.cell_for("lattice64_80", "40").n == (40, 40, 40)
    ng, ns = 4096, 128
    gram, rot = bench.gemm_pipe_flops(ng, ns)
    assert gram == 3 * 2 * 128 * (2 * 128) * ng      # one tile pair, N = 2 * 128
    assert rot == 3 * 2 * ng * 128 * 128             # one block of 128 (rounded to 16) columns, K = 128
    gram2, _ = bench.gemm_pipe_flops(ng, 130)       # two tiles: widths 128 and 16 (2 rounded up)
    assert gram2 == 3 * 2 * 128 * (2 * 128 + 2 * 16 + 2 * 16) * ng
