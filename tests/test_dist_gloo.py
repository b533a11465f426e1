"""Data-parallel step on CPU (gloo, 2 ranks): each rank renders its shard of
the view/light pairs (with the FP64 oracle, so no GPU is needed) and the
gradients are summed with the pipeline's all-reduce; the result must equal the
single-process sum over all pairs. Covers the sharding and exchange logic the
multi-GPU benchmark uses."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle as O
    import scenegen as sg
    from paper_2408_12282_gb300 import pipeline as PL
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = sg.make_workload("c4", N=400, res=32, n_pairs=5)
    dimg = sg.random_dimg(3, 32 * 32 * 5)
    keys = PL.SCENE_KEYS
    acc = {k: np.zeros_like(getattr(wl.scenes[0], k)) for k in keys}
    for p in PL.shard_pairs(len(wl.pairs), rank, world):
        r = O.render_pair(wl.scenes[0], wl.pairs[p], wl.mlp, dimg=dimg[p * 1024:(p + 1) * 1024])
        for k in keys:
            acc[k] += r["grads"][k]
    tensors = [torch.from_numpy(acc[k]) for k in keys]
    PL.allreduce_gradients(tensors)
    if rank == 0:
        np.savez(out_path, **{k: t.numpy() for k, t in zip(keys, tensors)})
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gradient_allreduce_equals_full_batch(tmp_path):
    import oracle as O
    import scenegen as sg
    from paper_2408_12282_gb300 import pipeline as PL
    out = str(tmp_path / "g.npz")
    mp.get_context("spawn")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    wl = sg.make_workload("c4", N=400, res=32, n_pairs=5)
    dimg = sg.random_dimg(3, 32 * 32 * 5)
    ref = {k: np.zeros_like(getattr(wl.scenes[0], k)) for k in PL.SCENE_KEYS}
    for p in range(5):
        r = O.render_pair(wl.scenes[0], wl.pairs[p], wl.mlp, dimg=dimg[p * 1024:(p + 1) * 1024])
        for k in PL.SCENE_KEYS:
            ref[k] += r["grads"][k]
    for k in PL.SCENE_KEYS:
        assert np.allclose(got[k], ref[k], rtol=1e-12, atol=1e-14 * np.abs(ref[k]).max()), k
    assert PL.shard_pairs(5, 0, 2) == [0, 2, 4] and PL.shard_pairs(5, 1, 2) == [1, 3]
