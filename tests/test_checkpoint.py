"""Checkpoint / resume of the trainable state (CPU tensors stand in for the
device buffers): round trip, in-place restore (buffers a captured graph reads
keep their storage), and refusal of a checkpoint that does not fit."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import scenegen as sg
from paper_2408_12282_gb300 import pipeline as PL


def _renderer(seed, with_sh=True):
    wl = sg.make_workload("c3", N=50, res=16, net="paper", seed_offset=seed)
    scene = {k: torch.from_numpy(np.ascontiguousarray(getattr(wl.scenes[0], k), np.float32)) for k in PL.SCENE_KEYS}
    mlp = PL.MLPParams(0, 0, [torch.from_numpy(np.asarray(w, np.float32)) for w in wl.mlp.weights],
                       [torch.from_numpy(np.asarray(b, np.float32)) for b in wl.mlp.biases])
    sh = torch.from_numpy(sg.vis_sh_coeffs(seed, 50).astype(np.float32)) if with_sh else None
    return SimpleNamespace(scene=scene, mlp=mlp, vis_sh=sh)


def _flat(r):
    return {k: v.clone() for k, v in PL.state_dict(r).items()}


def test_round_trip_restores_every_tensor_in_place(tmp_path):
    r = _renderer(0)
    saved = _flat(r)
    path = tmp_path / "ck.pt"
    rng = torch.get_rng_state()
    PL.save_checkpoint(path, r, step=1234, extra={"lr": 1e-3, "rng": rng})
    ptrs = {k: v.data_ptr() for k, v in r.scene.items()}
    other = _renderer(1)                       # different values, same shapes
    for k in PL.SCENE_KEYS:
        r.scene[k].copy_(other.scene[k])
    for a, b in zip(r.mlp.W + r.mlp.b, other.mlp.W + other.mlp.b):
        a.copy_(b)
    r.vis_sh.copy_(other.vis_sh)
    assert not all(torch.equal(saved[k], v) for k, v in PL.state_dict(r).items())
    info = PL.load_checkpoint(path, r)
    assert info["step"] == 1234 and info["extra"]["lr"] == 1e-3
    assert torch.equal(info["extra"]["rng"], rng)
    now = PL.state_dict(r)
    assert set(now) == set(saved)
    assert all(torch.equal(now[k], saved[k]) for k in saved)
    assert {k: v.data_ptr() for k, v in r.scene.items()} == ptrs     # restored in place


def test_mismatched_checkpoints_are_refused(tmp_path):
    r = _renderer(0)
    path = tmp_path / "ck.pt"
    PL.save_checkpoint(path, r)
    before = _flat(r)
    no_sh = _renderer(0, with_sh=False)
    with pytest.raises(ValueError, match="unexpected"):
        PL.load_checkpoint(path, no_sh)                # the file holds vis_sh, the renderer has none
    sd = PL.state_dict(r)
    sd["scene.mu"] = sd["scene.mu"][:-1]
    with pytest.raises(ValueError, match="shape"):
        PL.load_state_dict(r, sd)
    assert all(torch.equal(PL.state_dict(r)[k], v) for k, v in before.items())   # nothing copied
    torch.save({"format": "something-else"}, tmp_path / "bad.pt")
    with pytest.raises(ValueError, match="not a"):
        PL.load_checkpoint(tmp_path / "bad.pt", r)

