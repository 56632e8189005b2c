"""GPU parity of the in-place topology change (lv_subdivide_apply_inplace:
Sec. IV-D, Eq. 13-16 with the optimizer refresh, and the removal of the
voxels pruned by Sec. IV-C) against the oracle's placement
(oracle/inplace.py), bit for bit: every row below n' in every array, the
selection and n', in the growing and the shrinking case, without a split, in
FP32 and FP16/BF16 storage, with auxiliary arrays of 1-, 2- and 4-byte
elements, at the capacity limit, and on the 2M-voxel scene with its rendered
statistics."""
import numpy as np
import pytest
import torch

from gpu_helpers import gpu_forward, np_
from oracle import inplace as IP
from paper_2511_02510_gb300 import litevoxel as L
from paper_2511_02510_gb300 import synth
from test_gpu_adapt import cu, gpu_prune, rand_scene, sub_params

pytestmark = pytest.mark.gpu

SENTINEL = 0xA5


def gpu_subdivide_inplace(sc, delta, z, u, seen, pm=None, density_dtype=torch.float32, sh_dtype=torch.float32,
                          aux=(), capacity=None, **kw):
    """Select, then apply in place on arrays of `capacity` rows (rows beyond n hold a sentinel byte)."""
    p = sub_params(**kw)
    n = sc["geom"].shape[0]
    cap = capacity if capacity is not None else 8 * n + 8

    def grown(a, dtype=None):
        t = cu(a, dtype)
        out = torch.empty((cap,) + tuple(t.shape[1:]), dtype=t.dtype, device="cuda")
        out.view(torch.uint8).fill_(SENTINEL)
        out[:n] = t
        return out

    geom, level = grown(sc["geom"]), grown(sc["level"])
    dens, sh = grown(sc["density"], density_dtype), grown(sc["sh"], sh_dtype)
    vox = L.make_voxels(geom, dens, sh, level)
    vox.n = n
    auxs, keep = [], []
    for arr, fill in aux:
        t = grown(arr)
        a = L.lv_aux_array()
        a.in_, a.out = t.data_ptr(), t.data_ptr()
        a.width = 1 if t.dim() == 1 else t.shape[1]
        a.elem_bytes = t.element_size()
        a.fill = int(np.array([fill], arr.dtype).view({1: np.uint8, 2: np.uint16, 4: np.uint32}[arr.dtype.itemsize])[0])
        auxs.append(a)
        keep.append(t)
    sel = torch.zeros(max(n, 1), dtype=torch.uint8, device="cuda")
    nn = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(L.lv_subdivide_workspace_size(n, p), dtype=torch.uint8, device="cuda")
    L.lv_subdivide_select(vox, cu(delta), cu(z), cu(u), cu(seen), None if pm is None else cu(pm), p, cap, sel, nn,
                          ws, status)
    L.lv_subdivide_apply_inplace(vox, cap, p, auxs, ws)
    torch.cuda.synchronize()
    m = int(nn.item())
    return {"geom": np_(geom), "level": np_(level), "density": dens.cpu(), "sh": sh.cpu(), "selected": np_(sel)[:n],
            "n_new": m, "status": int(status.item()), "aux": [np_(t) for t in keep]}


def assert_matches(g, r, density_dtype=torch.float32):
    m = r["n_new"]
    assert g["status"] == 0 and g["n_new"] == m
    np.testing.assert_array_equal(g["selected"], r["selected"])
    np.testing.assert_array_equal(g["geom"][:m].view(np.uint32), r["geom"].view(np.uint32))
    np.testing.assert_array_equal(g["level"][:m], r["level"])
    if density_dtype == torch.float32:
        np.testing.assert_array_equal(g["density"][:m].numpy().view(np.uint32), r["density"].view(np.uint32))
    else:
        np.testing.assert_array_equal(g["density"][:m].numpy().view(np.uint16),
                                      r["density"].astype(np.float16).view(np.uint16))
    np.testing.assert_array_equal(g["sh"][:m].float().numpy(), r["sh"])
    for a, b in zip(g["aux"], r["aux"]):
        np.testing.assert_array_equal(a[:m], b)


def case(n, seed, p_prune, **kw):
    sc = rand_scene(n, 300 + seed)
    rng = np.random.default_rng(seed)
    delta = rng.uniform(0.0, 0.2, n).astype(np.float32)
    z = rng.uniform(1, 20, n).astype(np.float32)
    u = rng.uniform(0, 1, n).astype(np.float32)
    u[: n // 8] = np.float32(0.5)
    seen = (rng.uniform(size=n) < 0.8).astype(np.uint8)
    pm = (rng.uniform(size=n) < p_prune).astype(np.uint8)
    aux = [(rng.normal(size=(n, 8)).astype(np.float32), 0.0), (rng.uniform(size=n).astype(np.float32), 1.0),
           ((rng.uniform(size=n) < 0.5).astype(np.uint8), 1), (rng.integers(0, 60000, (n, 3)).astype(np.uint16), 7)]
    return sc, (delta, z, u, seen), pm, aux


@pytest.mark.parametrize("n,seed,p_prune,top_ppm", [
    (3000, 0, 0.02, 50000),       # growing: children fill every hole, the rest appended
    (20001, 1, 0.1, 200000),      # growing, ragged size, more holes
    (5000, 2, 0.3, 20000),        # shrinking: fewer children than holes, the tail moves
    (4097, 3, 0.05, 0),           # no split: compaction from the tail only
    (777, 4, 0.0, 100000),        # no hole: every child but child 0 appended
    (1, 5, 0.0, 1000000),         # a single voxel split
    (100003, 6, 0.01, 50000),     # several thousand warps
])
def test_inplace_bit_exact(ora, n, seed, p_prune, top_ppm):
    sc, args, pm, aux = case(n, seed, p_prune)
    g = gpu_subdivide_inplace(sc, *args, pm=pm, aux=aux, top_ppm=top_ppm)
    r = IP.subdivide_inplace(sc, *args, prune_mask=pm, aux=aux, top_ppm=top_ppm)
    assert_matches(g, r)
    # the rows beyond n' that were never written keep their sentinel
    m, cap = r["n_new"], 8 * n + 8
    tail = np.arange(max(m, n), cap)
    assert np.all(g["level"][tail] == SENTINEL)


def test_inplace_mixed_precision(ora):
    n = 6000
    sc, args, pm, aux = case(n, 11, 0.05)
    g = gpu_subdivide_inplace(sc, *args, pm=pm, aux=aux, density_dtype=torch.float16, sh_dtype=torch.bfloat16)
    ref = dict(sc)
    ref["density"] = torch.as_tensor(sc["density"]).half().float().numpy()
    ref["sh"] = torch.as_tensor(sc["sh"]).bfloat16().float().numpy()
    r = IP.subdivide_inplace(ref, *args, prune_mask=pm, aux=aux)
    assert_matches(g, r, torch.float16)


def test_inplace_everything_pruned_and_capacity(ora):
    n = 2000
    sc, args, pm, aux = case(n, 12, 0.0)
    # every voxel pruned: nothing remains
    g = gpu_subdivide_inplace(sc, *args, pm=np.ones(n, np.uint8), aux=aux)
    assert g["status"] == 0 and g["n_new"] == 0
    # capacity below n': LV_ERR_CAPACITY and no row changes
    r = IP.subdivide_inplace(sc, *args, prune_mask=pm, aux=aux, top_ppm=100000)
    g = gpu_subdivide_inplace(sc, *args, pm=pm, aux=aux, top_ppm=100000, capacity=r["n_new"] - 1)
    assert g["status"] == L.LV_ERR_CAPACITY
    np.testing.assert_array_equal(g["geom"][:n], sc["geom"])
    np.testing.assert_array_equal(g["density"][:n].numpy(), sc["density"])
    np.testing.assert_array_equal(g["aux"][0][:n], aux[0][0])


def test_inplace_refuses_bad_arguments():
    n = 100
    sc, args, pm, aux = case(n, 13, 0.0)
    p = sub_params()
    geom, dens, sh, level = cu(sc["geom"]), cu(sc["density"]), cu(sc["sh"]), cu(sc["level"])
    vox = L.make_voxels(geom, dens, sh, level)
    ws = torch.empty(L.lv_subdivide_workspace_size(n, p), dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LvError) as ei:
        L.lv_subdivide_apply_inplace(vox, n - 1, p, [], ws)           # capacity below the voxel count
    assert ei.value.status == L.LV_ERR_INVALID_ARG
    a = L.lv_aux_array()
    t_in, t_out = cu(aux[0][0]), cu(aux[0][0])
    a.in_, a.out, a.width, a.elem_bytes = t_in.data_ptr(), t_out.data_ptr(), 8, 4
    with pytest.raises(L.LvError) as ei:
        L.lv_subdivide_apply_inplace(vox, n, p, [a], ws)              # in place: in must equal out
    assert ei.value.status == L.LV_ERR_INVALID_ARG
    with pytest.raises(L.LvError) as ei:
        L.lv_subdivide_apply_inplace(vox, n, p, [], ws[:64])          # short workspace
    assert ei.value.status == L.LV_ERR_WORKSPACE


@pytest.mark.slow
def test_inplace_on_the_360_scene_step(ora):
    # The bench's adaptation on the 2M-voxel scene's rendered statistics: prune (16 bins, q 5 %, EMA 0.9,
    # cap 1 %) then subdivide (top 5 %) in place, with the six auxiliary arrays of a training step.
    sc = synth.scene_360()
    cam = synth.orbit_camera(1237, 822, 60.0, 3.0, 37.0, 15.0)
    scene, ctx, vox = gpu_forward(sc, [cam])
    w, _ = ctx.unpack_wmax()
    torch.cuda.synchronize()
    w, z, dl, seen = np_(w), np_(ctx.z_min), np_(ctx.delta_min), np_(ctx.seen)
    n = len(w)
    del ctx, scene
    mask, npr, m, s = gpu_prune(w, seen, z, np.full(n, 0.32, np.float32), np.ones(n, np.uint8), cap_ppm=10000)
    rng = np.random.default_rng(0)
    aux = [(rng.normal(size=(n, 8)).astype(np.float32), 0.0), (rng.normal(size=(n, 8)).astype(np.float32), 0.0),
           (rng.normal(size=(n, 48)).astype(np.float32), 0.0), (rng.normal(size=(n, 48)).astype(np.float32), 0.0),
           (m, 1.0), (s, 1)]
    g = gpu_subdivide_inplace(sc, dl, z, w, seen, pm=mask, aux=aux, capacity=int(1.35 * n))
    r = IP.subdivide_inplace(sc, dl, z, w, seen, prune_mask=mask, aux=aux)
    assert npr > 0 and r["k"] > 0
    assert_matches(g, r)
