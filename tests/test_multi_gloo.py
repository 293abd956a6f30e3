"""Multi-rank host logic on CPU (gloo, world size 2): channel shards tile the
band, gathered per-rank images equal the whole, timings reduce to the max, and a
block split over time sums to the whole image."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1904_11422_gb300 import shard, synth


def test_channel_shard_partition():
    for n_chan in [0, 1, 5, 64, 67]:
        for world in [1, 2, 3, 8]:
            covered = []
            for r in range(world):
                lo, hi = shard.channel_shard(n_chan, r, world)
                assert 0 <= lo <= hi <= n_chan
                covered += list(range(lo, hi))
                assert abs((hi - lo) - n_chan / world) < 1
            assert covered == list(range(n_chan))
    with pytest.raises(ValueError):
        shard.channel_shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    w = synth.random_small(77, n_ant=5, n_pol=2, n_chan=5, grid_n=16, support=3, n_time=4)
    arr = oracle.OracleArray(w.ant_xy, w.freq_hz, 2, w.grid_n, w.support, w.cell_lambda, w.sigma_cells,
                             gains=w.gains, delays=w.delays_s)
    lo, hi = shard.channel_shard(w.n_chan, rank, world)
    local = oracle.image(arr, w.volts, subtract=True, c_lo=lo, c_hi=hi, n_threads=1)
    full = shard.gather_channels(torch.from_numpy(local), w.n_chan)
    slowest = shard.max_over_ranks(1.5 + rank)
    if rank == 0:
        np.save(os.path.join(out_dir, "full.npy"), full.numpy())
        np.save(os.path.join(out_dir, "slowest.npy"), np.array([slowest]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_images_equal_the_whole(tmp_path, oracle_lib):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import oracle
    w = synth.random_small(77, n_ant=5, n_pol=2, n_chan=5, grid_n=16, support=3, n_time=4)
    arr = oracle.OracleArray(w.ant_xy, w.freq_hz, 2, w.grid_n, w.support, w.cell_lambda, w.sigma_cells,
                             gains=w.gains, delays=w.delays_s)
    whole = oracle.image(arr, w.volts, subtract=True, n_threads=1)
    full = np.load(tmp_path / "full.npy")
    assert np.array_equal(full, whole)  # channels are independent: bit-identical
    assert np.load(tmp_path / "slowest.npy")[0] == 1.5 + world - 1


def _time_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    w = synth.random_small(78, n_ant=6, n_pol=2, n_chan=3, grid_n=16, support=3, n_time=9)
    arr = oracle.OracleArray(w.ant_xy, w.freq_hz, 2, w.grid_n, w.support, w.cell_lambda, w.sigma_cells,
                             gains=w.gains, delays=w.delays_s)
    lo, hi = shard.time_shard(w.n_time, rank, world)
    local = torch.from_numpy(oracle.image(arr, w.volts[lo:hi], subtract=True, n_threads=1))
    total = shard.sum_images(local)
    if rank == 0:
        np.save(os.path.join(out_dir, "total.npy"), total.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_time_split_block_sums_to_the_whole(tmp_path, oracle_lib):
    """Ranks image disjoint sample ranges of every channel (autocorrelations removed
    per rank); one sum all-reduce gives the whole block's image."""
    world = 2
    mp.spawn(_time_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    import oracle
    w = synth.random_small(78, n_ant=6, n_pol=2, n_chan=3, grid_n=16, support=3, n_time=9)
    arr = oracle.OracleArray(w.ant_xy, w.freq_hz, 2, w.grid_n, w.support, w.cell_lambda, w.sigma_cells,
                             gains=w.gains, delays=w.delays_s)
    whole = oracle.image(arr, w.volts, subtract=True, n_threads=1)
    total = np.load(tmp_path / "total.npy")
    assert np.abs(total - whole).max() <= 1e-12 * np.abs(whole).max()
    assert [shard.time_shard(9, r, 2) for r in range(2)] == [(0, 5), (5, 9)]


def _bench_worker(rank, world, port, out_dir, mode):
    """One rank of bench.py's multi-GPU plumbing: the rank's share of the band
    (shard.rank_channels), its slice of the block (synth.channel_slice), the
    slowest rank's time (shard.max_over_ranks) and the job's units
    (shard.job_units); the imaging call is the oracle's, on CPU."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    w = synth.random_small(79, n_ant=5, n_pol=2, n_chan=7, grid_n=16, support=3, n_time=3)
    lo, hi = shard.rank_channels(w.n_chan, rank, world, mode)
    wl = w if (lo, hi) == (0, w.n_chan) else synth.channel_slice(w, lo, hi)
    arr = oracle.OracleArray(wl.ant_xy, wl.freq_hz, 2, wl.grid_n, wl.support, wl.cell_lambda, wl.sigma_cells,
                             gains=wl.gains, delays=wl.delays_s)
    local = torch.from_numpy(oracle.image(arr, wl.volts, subtract=True, n_threads=1))
    slowest = shard.max_over_ranks(10.0 + rank)
    units = shard.job_units(w.units, world, mode)
    full = shard.gather_channels(local, w.n_chan) if mode == "channels" else local
    np.save(os.path.join(out_dir, f"{mode}_{rank}.npy"), full.numpy())
    np.save(os.path.join(out_dir, f"{mode}_{rank}_meta.npy"), np.array([slowest, units, lo, hi]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["channels", "replicate"])
def test_bench_shard_plumbing(tmp_path, oracle_lib, mode):
    world = 2
    mp.spawn(_bench_worker, args=(world, _free_port(), str(tmp_path), mode), nprocs=world, join=True)
    import oracle
    w = synth.random_small(79, n_ant=5, n_pol=2, n_chan=7, grid_n=16, support=3, n_time=3)
    arr = oracle.OracleArray(w.ant_xy, w.freq_hz, 2, w.grid_n, w.support, w.cell_lambda, w.sigma_cells,
                             gains=w.gains, delays=w.delays_s)
    whole = oracle.image(arr, w.volts, subtract=True, n_threads=1)
    ranges = []
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"{mode}_{r}.npy"), whole)  # bit-identical
        slowest, units, lo, hi = np.load(tmp_path / f"{mode}_{r}_meta.npy")
        assert slowest == 10.0 + world - 1
        assert units == (w.units if mode == "channels" else world * w.units)
        ranges.append((int(lo), int(hi)))
    assert ranges == ([(0, 4), (4, 7)] if mode == "channels" else [(0, 7), (0, 7)])
    assert shard.scaling(mode) == ("strong" if mode == "channels" else "weak")


def test_bench_starts_its_own_ranks():
    import bench
    cmd = bench.torchrun_command(["--gpus", "8", "--steps", "5"], 8, 29511)
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=8" in cmd and "--nnodes=1" in cmd
    assert cmd[cmd.index("--master-addr") + 1] == "127.0.0.1"
    assert cmd[cmd.index("--master-port") + 1] == "29511"
    assert cmd[-5].endswith("bench.py") and cmd[-4:] == ["--gpus", "8", "--steps", "5"]
