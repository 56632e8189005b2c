"""Data-parallel training over views (paper_2511_02510_gb300/dp.py) on two gloo
ranks on the CPU: rank r renders view r of the tiny scene (the oracle stands
in for the GPU: FP64 render and reverse pass of Eq. 2-5, FP32 binning
statistics), packs w_max as the library does with its pixel-id base, and the
exchange step reduces gradients and statistics.  The reduced arrays, and the
pruning (Eq. 11-12) and subdivision (Eq. 13-16) decisions every rank then
takes from them, equal one process rendering both views: bit for bit for the
statistics and the decisions, to FP64 rounding for the gradient sums."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def cams():
    from paper_2511_02510_gb300 import synth
    return [synth.orbit_camera(40, 32, 60.0, 1.6, 30.0, 25.0, target=(0.5, 0.4, 0.5)),
            synth.orbit_camera(36, 28, 60.0, 1.6, 150.0, 30.0, target=(0.5, 0.4, 0.5))]


def pack(w, arg):
    """The library's packed w_max word: (f32 bits of w << 32) | (0xffffffff - pixel id), 0 if never hit."""
    bits = np.asarray(w, np.float32).view(np.uint32).astype(np.uint64)
    word = (bits << np.uint64(32)) | (np.uint64(0xffffffff) - np.asarray(arg).astype(np.uint64))
    return np.where(np.asarray(arg) >= 0, word, np.uint64(0)).view(np.int64)


def loss_grads(P, seed=3):
    return np.random.default_rng(seed).normal(size=(P, 3))


def adapt(O, sc, w_max, z_min, delta_min, seen):
    n = sc["geom"].shape[0]
    pr = O.prune(w_max, seen, z_min, np.full(n, 0.32, np.float32), np.ones(n, np.uint8), cap_ppm=20000)
    sd = O.subdivide(sc, delta_min, z_min, w_max, seen, prune_mask=pr["mask"], top_ppm=50000, l_max=8, kappa=0.1)
    return pr, sd


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_2511_02510_gb300 import dp, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = synth.scene_tiny()
    cs = cams()
    sizes = [c["width"] * c["height"] for c in cs]
    base = dp.pixel_id_bases(sizes)[rank]
    cam = cs[rank]
    # this rank's view: render, statistics, gradients of its slice of the loss
    r = O.render(sc, [cam])
    st = O.pairs(sc, [cam])
    g_all = loss_grads(sum(sizes))
    g = g_all[base:base + sizes[rank]]
    b = O.render_backward(sc, [cam], g)
    arg = np.where(r["w_arg"] >= 0, r["w_arg"] + base, -1)
    t = {"dd": torch.from_numpy(b["d_density"].copy()), "ds": torch.from_numpy(b["d_sh"].copy()),
         "wm": torch.from_numpy(pack(r["w_max"], arg)), "z": torch.from_numpy(st["z_min"].copy()),
         "dl": torch.from_numpy(st["delta_min"].copy()), "seen": torch.from_numpy(st["seen"].copy())}
    mine = {"w32": r["w_max"].astype(np.float32), "arg": arg}
    dp.allreduce_step(t["dd"], t["ds"], t["wm"], t["z"], t["dl"], t["seen"])
    # every rank decides from the reduced arrays
    word = t["wm"].numpy().view(np.uint64)
    w_red = (word >> np.uint64(32)).astype(np.uint32).view(np.float32)
    arg_red = np.where(word != 0, (np.uint64(0xffffffff) - (word & np.uint64(0xffffffff))).astype(np.int64), -1)
    pr, sd = adapt(O, sc, w_red, t["z"].numpy(), t["dl"].numpy(), t["seen"].numpy())
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, {"dd": t["dd"].numpy(), "ds": t["ds"].numpy(), "w": w_red, "arg": arg_red, "z": t["z"].numpy(),
                  "dl": t["dl"].numpy(), "seen": t["seen"].numpy(), "mask": pr["mask"], "m": pr["m"],
                  "selected": sd["selected"], "geom": sd["geom"], "density": sd["density"], "mine": mine}))


def test_two_ranks_equal_one_process_over_both_views(ora):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2511_02510_gb300 import synth
    sc = synth.scene_tiny()
    cs = cams()
    sizes = [c["width"] * c["height"] for c in cs]
    r = ora.render(sc, cs)
    st = ora.pairs(sc, cs)
    b = ora.render_backward(sc, cs, loss_grads(sum(sizes)))
    for a in res.values():
        # statistics: bit for bit
        np.testing.assert_array_equal(a["z"].view(np.uint32), st["z_min"].view(np.uint32))
        np.testing.assert_array_equal(a["dl"].view(np.uint32), st["delta_min"].view(np.uint32))
        np.testing.assert_array_equal(a["seen"], st["seen"])
        # w_max: the FP32 maximum, its argmax the two-view one (equal FP32 weights on the two ranks'
        # rays: the smaller global pixel id, the packed tie rule)
        np.testing.assert_array_equal(a["w"], r["w_max"].astype(np.float32))
        m0, m1 = res[0]["mine"], res[1]["mine"]
        tie = (m0["arg"] >= 0) & (m1["arg"] >= 0) & (m0["w32"] == m1["w32"])
        expect = np.where(tie, np.minimum(m0["arg"], m1["arg"]), r["w_arg"])
        np.testing.assert_array_equal(a["arg"], expect)
        # gradients: the sum over views, to FP64 rounding
        np.testing.assert_allclose(a["dd"], b["d_density"], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(a["ds"], b["d_sh"], rtol=1e-12, atol=1e-15)
    # both ranks take the decisions one process takes over both views
    pr, sd = adapt(ora, sc, r["w_max"].astype(np.float32), st["z_min"], st["delta_min"], st["seen"])
    assert pr["n_pruned"] > 0 and sd["k"] > 0
    for a in res.values():
        np.testing.assert_array_equal(a["mask"], pr["mask"])
        np.testing.assert_array_equal(a["m"].view(np.uint32), pr["m"].view(np.uint32))
        np.testing.assert_array_equal(a["selected"], sd["selected"])
        np.testing.assert_array_equal(a["geom"].view(np.uint32), sd["geom"].view(np.uint32))
        np.testing.assert_array_equal(a["density"].view(np.uint32), sd["density"].view(np.uint32))


def test_pixel_id_bases():
    sys.path.insert(0, ROOT)
    from paper_2511_02510_gb300 import dp
    assert dp.pixel_id_bases([10, 5, 7]) == [0, 10, 15]
    assert dp.pixel_id_bases([]) == []
    import pytest
    with pytest.raises(ValueError):
        dp.pixel_id_bases([1 << 31, 1 << 31])
