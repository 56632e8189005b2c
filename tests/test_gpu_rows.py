"""lv_rows_scatter against torch index copies: rows of 16-byte multiples (moved as
words), 1-byte and 12-byte rows and a misaligned array (moved byte by byte),
plain copies, several arrays in one launch; and the rollback of an in-place
topology change from the rows saved before it."""
import pytest
import torch

from paper_2511_02510_gb300 import litevoxel as L

pytestmark = pytest.mark.gpu


def test_scatter_matches_index_copy():
    g = torch.Generator(device="cuda").manual_seed(3)
    n, m = 5000, 777
    idx = torch.randperm(n, device="cuda", generator=g)[:m]
    arrays = [torch.rand(n, 4, device="cuda", generator=g), torch.randint(0, 255, (n,), device="cuda",
                                                                          dtype=torch.uint8, generator=g),
              torch.rand(n, 48, device="cuda", generator=g), torch.rand(n, 3, device="cuda", generator=g)]
    base = torch.rand(n * 4 + 1, device="cuda", generator=g)
    mis = base[1:].view(n, 4)  # 4-byte aligned, not 16
    arrays.append(mis)
    srcs = [torch.rand_like(a.float()).to(a.dtype) if a.dtype != torch.uint8 else
            torch.randint(0, 255, a.shape, device="cuda", dtype=torch.uint8, generator=g) for a in arrays]
    saved = [s[:m].contiguous() for s in srcs]
    want = [a.clone().index_copy_(0, idx, s) for a, s in zip(arrays, saved)]
    plain_dst = torch.zeros(n * 3, device="cuda")
    plain_src = torch.rand(n * 3, device="cuda", generator=g)
    L.lv_rows_scatter([(a, s, idx) for a, s in zip(arrays, saved)] + [(plain_dst, plain_src, None)])
    torch.cuda.synchronize()
    for a, w in zip(arrays, want):
        assert torch.equal(a, w)
    assert torch.equal(plain_dst, plain_src)


def test_rollback_of_an_inplace_topology_change():
    import bench
    from paper_2511_02510_gb300 import synth
    wl = bench.Workload(synth.scene_tiny(), bench.camera_for(0), synth.random_image(bench.W_IMG, bench.H_IMG, seed=3))
    pristine = [a.clone() for a in wl._state_arrays()]
    wl.step()
    torch.cuda.synchronize()
    assert int(wl.n_new.item()) != wl.n
    wl.prepare_restore(pristine)
    wl.step()  # ends with restore(): one lv_rows_scatter
    torch.cuda.synchronize()
    for a, p in zip(wl._state_arrays(), pristine):
        assert torch.equal(a[:wl.n], p[:wl.n])
    assert torch.equal(wl.ema, wl.ema0) and torch.equal(wl.state, wl.state0)
