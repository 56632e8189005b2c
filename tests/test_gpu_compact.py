"""GPU parity of the stable compaction (lv_compact) against the oracle:
every voxel and auxiliary array bit for bit, in both storage precisions, at
sizes that leave ragged warps, with the degenerate masks and the capacity
check; lv_check_status reads the device status word."""
import numpy as np
import pytest
import torch

from gpu_helpers import np_
from paper_2511_02510_gb300 import litevoxel as L
from test_gpu_adapt import cu, rand_scene

pytestmark = pytest.mark.gpu


def gpu_compact(sc, keep, aux=(), density_dtype=torch.float32, sh_dtype=torch.float32, capacity=None):
    n = sc["geom"].shape[0]
    geom, level = cu(sc["geom"]), cu(sc["level"])
    dens, sh = cu(sc["density"], density_dtype), cu(sc["sh"], sh_dtype)
    vin = L.make_voxels(geom, dens, sh, level)
    cap = n if capacity is None else capacity
    og = torch.full((cap, 4), -7.0, dtype=torch.float32, device="cuda")
    ol = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    od = torch.zeros((cap, 8), dtype=density_dtype, device="cuda")
    osh = torch.zeros((cap, 48), dtype=sh_dtype, device="cuda")
    vout = L.make_voxels(og, od, osh, ol)
    vout.n = cap
    auxs, held = [], []
    for arr in aux:
        ti = cu(arr)
        to = torch.zeros((cap,) + tuple(ti.shape[1:]), dtype=ti.dtype, device="cuda")
        a = L.lv_aux_array()
        a.in_, a.out = ti.data_ptr(), to.data_ptr()
        a.width = 1 if ti.dim() == 1 else ti.shape[1]
        a.elem_bytes = ti.element_size()
        auxs.append(a)
        held.append((ti, to))
    km = cu(keep)
    nn = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(L.lv_compact_workspace_size(n), dtype=torch.uint8, device="cuda")
    L.lv_compact(vin, km, auxs, vout, nn, ws, status)
    st = L.lv_check_status(status)
    m = int(nn.item())
    k = min(m, cap)
    return {"geom": np_(og)[:k], "level": np_(ol)[:k], "density": od[:k].cpu(), "sh": osh[:k].cpu(), "n_new": m,
            "status": st, "aux": [np_(t)[:k] for _, t in held], "geom_all": np_(og)}


@pytest.mark.parametrize("n,p_keep", [(1, 1.0), (33, 0.5), (5000, 0.9), (100003, 0.3)])
def test_compact_bit_exact(ora, n, p_keep):
    sc = rand_scene(n, n)
    rng = np.random.default_rng(n)
    keep = (rng.uniform(size=n) < p_keep).astype(np.uint8)
    aux = [rng.normal(size=(n, 48)).astype(np.float32), rng.uniform(size=n).astype(np.float32),
           rng.integers(0, 255, size=n).astype(np.uint8), rng.integers(0, 60000, size=(n, 3)).astype(np.uint16)]
    g = gpu_compact(sc, keep, aux)
    r = ora.compact(sc, keep, aux)
    assert g["status"] == L.LV_OK and g["n_new"] == r["n_new"]
    np.testing.assert_array_equal(g["geom"].view(np.uint32), r["geom"].view(np.uint32))
    np.testing.assert_array_equal(g["level"], r["level"])
    np.testing.assert_array_equal(g["density"].numpy().view(np.uint32), r["density"].view(np.uint32))
    np.testing.assert_array_equal(g["sh"].numpy().view(np.uint32), r["sh"].view(np.uint32))
    for a, b in zip(g["aux"], r["aux"]):
        np.testing.assert_array_equal(a, b)


def test_compact_mixed_precision_storage(ora):
    n = 4097
    sc = rand_scene(n, 3)
    keep = (np.arange(n) % 3 != 1).astype(np.uint8)
    g = gpu_compact(sc, keep, density_dtype=torch.float16, sh_dtype=torch.bfloat16)
    r = ora.compact(sc, keep)
    assert g["n_new"] == r["n_new"]
    np.testing.assert_array_equal(g["density"].numpy(), r["density"].astype(np.float16))
    np.testing.assert_array_equal(g["sh"].float().numpy(), torch.as_tensor(r["sh"]).bfloat16().float().numpy())


def test_compact_degenerate_masks_and_capacity(ora):
    n = 777
    sc = rand_scene(n, 9)
    g = gpu_compact(sc, np.zeros(n, np.uint8))
    assert g["n_new"] == 0 and g["status"] == L.LV_OK
    g = gpu_compact(sc, np.ones(n, np.uint8))
    np.testing.assert_array_equal(g["geom"], sc["geom"])
    # one row short: capacity error, the count is still reported, nothing is written
    keep = np.ones(n, np.uint8)
    keep[::2] = 0
    m = int(keep.sum())
    g = gpu_compact(sc, keep, capacity=m - 1)
    assert g["status"] == L.LV_ERR_CAPACITY and g["n_new"] == m
    assert np.all(g["geom_all"] == -7.0)


def test_compact_empty_and_bad_arguments():
    geom = torch.zeros((0, 4), device="cuda")
    vin = L.make_voxels(geom, torch.zeros((0, 8), device="cuda"), torch.zeros((0, 48), device="cuda"),
                        torch.zeros(0, dtype=torch.uint8, device="cuda"))
    vout = L.make_voxels(geom, torch.zeros((0, 8), device="cuda"), torch.zeros((0, 48), device="cuda"),
                         torch.zeros(0, dtype=torch.uint8, device="cuda"))
    nn = torch.full((1,), 5, dtype=torch.int64, device="cuda")
    ws = torch.empty(max(256, L.lv_compact_workspace_size(0)), dtype=torch.uint8, device="cuda")
    L.lv_compact(vin, None, [], vout, nn, ws)
    torch.cuda.synchronize()
    assert int(nn.item()) == 0
    assert L.lv_check_status(None) == L.LV_ERR_INVALID_ARG
