"""Data-parallel step on CPU (gloo, 2 ranks): each rank renders its shard of
the view/light pairs (with the FP64 oracle, so no GPU is needed), writes the
scene and network gradients into a Renderer's flat gradient buffer (built on
the CPU: host-side set-up only) and calls Renderer.exchange_gradients, the
one all-reduce the multi-GPU benchmark's step makes; the result must equal the
single-process sum over all pairs, for every scene tensor and every dW, db."""
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
    rend = PL.renderer_for_workload(wl, device="cpu")
    rend.zero_grads()
    for p in PL.shard_pairs(len(wl.pairs), rank, world):
        r = O.render_pair(wl.scenes[0], wl.pairs[p], wl.mlp, dimg=dimg[p * 1024:(p + 1) * 1024])
        for k in keys:
            rend.grads[k] += torch.from_numpy(r["grads"][k]).float()
        for l in range(len(rend.dW)):
            rend.dW[l] += torch.from_numpy(r["dW"][l]).float()
            rend.db[l] += torch.from_numpy(r["db"][l]).float()
    rend.exchange_gradients()
    if rank == 0:
        out = {k: rend.grads[k].numpy() for k in keys}
        out.update({f"W{l}": w.numpy() for l, w in enumerate(rend.dW)})
        out.update({f"b{l}": b.numpy() for l, b in enumerate(rend.db)})
        np.savez(out_path, **out)
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
            ref[k] = ref[k] + r["grads"][k]
        for l in range(len(r["dW"])):
            ref[f"W{l}"] = ref.get(f"W{l}", 0) + r["dW"][l]
            ref[f"b{l}"] = ref.get(f"b{l}", 0) + r["db"][l]
    assert len(ref) == len(PL.SCENE_KEYS) + 10
    for k, v in ref.items():       # float32 buffers: sums of two rank partials, each rounded once
        assert np.allclose(got[k], v, rtol=1e-5, atol=1e-6 * max(np.abs(v).max(), 1e-30)), k
    assert PL.shard_pairs(5, 0, 2) == [0, 2, 4] and PL.shard_pairs(5, 1, 2) == [1, 3]


def _worker_peer_dies(rank, world, port, out_path):
    import sys
    import time
    from datetime import timedelta
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2408_12282_gb300 import pipeline as PL
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=10))
    if rank == 1:
        os._exit(3)                      # dies between steps, before the gradient exchange
    t0 = time.time()
    try:
        PL.exchange_gradients(torch.ones(16))
        status = "completed"
    except Exception as ex:              # the exchange must fail, not hang
        status = f"error:{type(ex).__name__}"
    with open(out_path, "w") as fh:
        fh.write(f"{status} {time.time() - t0:.2f}")
    os._exit(0)


def test_a_dead_peer_fails_the_gradient_exchange_instead_of_hanging(tmp_path):
    """Failure detection on the host: a rank that exits before the exchange
    makes the survivor's all-reduce raise within the process group's timeout
    (10 s) rather than wait forever."""
    out = str(tmp_path / "status.txt")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker_peer_dies, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    alive = [p.is_alive() for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert not any(alive), "a rank did not finish"
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
    status, secs = open(out).read().split()
    assert status.startswith("error:"), status
    assert float(secs) < 60
