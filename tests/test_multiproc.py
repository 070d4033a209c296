"""The N > 1 paths on the CPU: gloo ranks, world size 2 and 3.

Under torchrun the bench shards the domain into spatial slabs, one per rank
(the paper's decomposition, Sec. 3.1): each rank's library plan forms its
slab's part of every Gram, the parts are all-gathered in rank order, and
every rank's plan sums them in that order and solves the same eigenproblems.
The library calls need a GPU and are tested on one GPU (two slab plans); here
the host side is tested: the rank-ordered gather of the parts, the
max-over-ranks job time, the torchrun launch of the reference arm (rank 0
prints the single JSON line, the other ranks exit 0), and the whole
decomposition carried out with the oracle on gloo ranks against the
single-process fit.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    v = bench.max_over_ranks(1.5 + rank, "cpu")
    with open(os.path.join(outdir, f"r{rank}.txt"), "w") as fh:
        fh.write(repr(v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    vals = [float(open(tmp_path / f"r{r}.txt").read()) for r in range(world)]
    assert vals == [2.5, 2.5]


def _gather_main(rank, world, port, outdir):
    import numpy as np
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    part = torch.arange(24, dtype=torch.float64).reshape(3, 2, 2, 2) + 100.0 * rank
    parts = torch.empty((world, 3, 2, 2, 2), dtype=torch.float64)
    bench.gather_slab_grams(part, parts)
    np.save(os.path.join(outdir, f"g{rank}.npy"), parts.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_gram_gather_is_in_rank_order_on_every_rank(tmp_path, world):
    import numpy as np
    mp.spawn(_gather_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [np.load(tmp_path / f"g{r}.npy") for r in range(world)]
    base = np.arange(24, dtype=np.float64).reshape(3, 2, 2, 2)
    for g in got:
        assert np.array_equal(g, got[0])
        for r in range(world):
            assert np.array_equal(g[r], base + 100.0 * r)


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--small"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "columns" in d["config"]["sample"] and d["cpu_baseline"]["sample"] == d["config"]["sample"]


# ---------------------------------------------------------------- slab partition
# The paper's spatial decomposition (Sec. 3.1): each rank owns a contiguous
# slab of the flattened points; mean, blocks, window, DFT and the partial Gram
# are local, one sum of the Grams (here in fixed rank order, for a result that
# is the same on every rank), the eigen-solve is redundant, the modes local.
# Run with the oracle on gloo ranks, against the single-process fit.
def _slab_main(rank, world, port, outdir):
    import numpy as np
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import oracle as O
    nt, M, nfft, nov = 512, 90, 64, 32
    rs = np.random.RandomState(7)
    X = rs.randn(nt, M) + 2.0 * np.sin(2 * np.pi * 5 * np.arange(nt) / nfft)[:, None] * rs.randn(M)[None, :]
    W = 0.5 + rs.rand(M)
    bounds = [M * r // world for r in range(world + 1)]        # uneven slabs when world does not divide M
    sl = slice(bounds[rank], bounds[rank + 1])
    d = O.Desc(nt=nt, M=bounds[rank + 1] - bounds[rank], nfft=nfft, noverlap=nov, weights=W[sl])
    Xs = X[:, sl]
    Q = O.block_dft(Xs, nfft, nov, d.w(), O.time_mean(Xs))
    G = torch.from_numpy(O.gram(Q, W[sl]))
    parts = [torch.zeros_like(G) for _ in range(world)]
    dist.all_gather(parts, G)
    Gsum = parts[0].clone()
    for p in parts[1:]:
        Gsum += p                                                # rank order on every rank
    lam, Psi, _, conv = O.jacobi_eigh(Gsum.numpy())
    Phi = O.modes(Q, lam, Psi, 3)
    np.savez(os.path.join(outdir, f"slab{rank}.npz"), G=Gsum.numpy(), lam=lam, Phi=Phi, conv=conv,
             lo=bounds[rank], hi=bounds[rank + 1])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_partition_matches_single_process(tmp_path, world):
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle as O
    mp.spawn(_slab_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [np.load(os.path.join(str(tmp_path), f"slab{r}.npz")) for r in range(world)]
    nt, M, nfft, nov = 512, 90, 64, 32
    rs = np.random.RandomState(7)
    X = rs.randn(nt, M) + 2.0 * np.sin(2 * np.pi * 5 * np.arange(nt) / nfft)[:, None] * rs.randn(M)[None, :]
    W = 0.5 + rs.rand(M)
    fit = O.spod_fit(X, O.Desc(nt=nt, M=M, nfft=nfft, noverlap=nov, weights=W))
    Phi = O.modes(fit.Qhat, fit.lam, fit.Psi, 3)
    for r in range(world):
        assert bool(res[r]["conv"])
        # the reduced Gram (hence the redundant eigen-solve) is identical on every rank
        assert np.array_equal(res[r]["G"], res[0]["G"]) and np.array_equal(res[r]["lam"], res[0]["lam"])
    assert np.abs(res[0]["G"] - fit.M).max() <= 1e-12 * np.abs(fit.M).max()
    np.testing.assert_allclose(res[0]["lam"], fit.lam, rtol=1e-10, atol=1e-12 * fit.lam.max())
    Phis = np.concatenate([res[r]["Phi"] for r in range(world)], axis=2)
    # modes of well-separated eigenvalues agree column by column (same phase rule)
    gap = (fit.lam[:, :3] - fit.lam[:, 1:4]) / fit.lam[:, :1]
    ok = gap > 1e-6
    err = np.abs(Phis - Phi).max(axis=2) / np.abs(Phi).max(axis=2)
    assert err[ok].max() <= 1e-8
