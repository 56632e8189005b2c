"""Checkpoint and resume (CPU): the voxel arrays and the caller-held training
state survive a save / load round trip bit for bit, in their dtypes, and a
pruning run resumed from a checkpoint takes the same decisions as one that
never stopped (the oracle's pruning stands in for the device calls)."""
import numpy as np
import pytest
import torch

from paper_2511_02510_gb300 import checkpoint, synth
from paper_2511_02510_gb300.raster import Scene


def tiny_scene(density_dtype=torch.float16, sh_dtype=torch.bfloat16):
    return Scene.from_numpy(synth.scene_tiny(), "cpu", density_dtype, sh_dtype)


def test_round_trip_keeps_bits_and_dtypes(tmp_path):
    scene = tiny_scene()
    n = scene.n
    g = torch.Generator().manual_seed(0)
    state = {"ema_m": torch.rand(n, generator=g), "state_s": torch.randint(0, 2, (n,), dtype=torch.uint8),
             "adam_m_density": torch.randn(n, 8, generator=g), "adam_v_sh": torch.rand(n, 48, generator=g),
             "pct_state": torch.tensor([float("nan"), 3.5])}
    path = str(tmp_path / "ck.pt")
    checkpoint.save(path, scene, state, step=1234, meta={"q_ppm": 50000, "note": "mid-ramp"})
    s2, st2, step, meta = checkpoint.load(path, device="cpu")
    assert step == 1234 and meta == {"q_ppm": 50000, "note": "mid-ramp"} and s2.sh_degree == scene.sh_degree
    for k in checkpoint.SCENE_ARRAYS:
        a, b = getattr(scene, k), getattr(s2, k)
        assert a.dtype == b.dtype and torch.equal(a.view(torch.uint8), b.view(torch.uint8)), k
    assert set(st2) == set(state)
    for k, v in state.items():
        assert v.dtype == st2[k].dtype and torch.equal(v.view(torch.uint8), st2[k].view(torch.uint8)), k
    assert not list(tmp_path.glob("*.tmp*"))            # the temporary file was renamed into place


def test_shapes_and_format_checked(tmp_path):
    scene = tiny_scene()
    path = str(tmp_path / "ck.pt")
    checkpoint.save(path, scene)
    blob = torch.load(path, weights_only=True)
    blob["format"] = 99
    torch.save(blob, path)
    with pytest.raises(ValueError, match="format"):
        checkpoint.load(path, device="cpu")
    bad = Scene(scene.geom, scene.level, scene.density[:, :4], scene.sh)
    with pytest.raises(ValueError, match="density"):
        checkpoint.save(str(tmp_path / "bad.pt"), bad)


def test_resumed_pruning_takes_the_same_decisions(ora, tmp_path):
    # Three pruning steps (Eq. 11-12, guard i EMA + hysteresis, guard iii cap) with drifting w_max, run straight
    # through and with a save / load of (m, s) after the first step.
    scene = tiny_scene(torch.float32, torch.float32)
    n = scene.n
    rng = np.random.default_rng(3)
    z = rng.uniform(1, 10, n).astype(np.float32)
    seen = (rng.uniform(size=n) < 0.9).astype(np.uint8)
    ws = [rng.uniform(0, 1, n).astype(np.float32) ** (1 + k) for k in range(3)]

    def run(m, s, steps):
        masks = []
        for w in steps:
            r = ora.prune(w, seen, z, m, s, cap_ppm=20000)
            m, s = r["m"], r["s"]
            masks.append(r["mask"])
        return m, s, masks

    m0 = rng.uniform(0.2, 0.6, n).astype(np.float32)      # near the hysteresis band, so states flip
    s0 = (rng.uniform(size=n) < 0.5).astype(np.uint8)
    m_a, s_a, masks_a = run(m0, s0, ws)
    m1, s1, masks_b = run(m0, s0, ws[:1])
    path = str(tmp_path / "ck.pt")
    checkpoint.save(path, scene, {"ema_m": torch.from_numpy(m1), "state_s": torch.from_numpy(s1)}, step=1)
    _, st, step, _ = checkpoint.load(path, device="cpu")
    assert step == 1
    m_b, s_b, more = run(st["ema_m"].numpy(), st["state_s"].numpy(), ws[1:])
    masks_b += more
    assert np.array_equal(m_a.view(np.uint32), m_b.view(np.uint32)) and np.array_equal(s_a, s_b)
    for a, b in zip(masks_a, masks_b):
        assert np.array_equal(a, b)
    assert sum(int(m.sum()) for m in masks_a) > 0          # the run did prune something
