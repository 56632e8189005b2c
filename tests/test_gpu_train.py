"""GPU parity of the rest of the training step: the transmittance
concentration term, the density TV term fused into the Adam update, and the
Adam update itself, against the FP64 oracle in oracle/train_aux.py.

Tolerances: the GPU works in FP32.  Moments take 2-3 roundings (a few ulps
of their largest term); the parameter update u = lr m^ / (sqrt(v^) + eps)
takes about 6 more, so the updated parameter is within 4e-6 |u| + ulp(p) of
the FP64 result; losses are FP32 per-thread partials summed in FP64 (rtol
1e-5).
FP16 / BF16 storage may round the other way when the FP32 and FP64 results
straddle a rounding boundary: at most one unit in the last place.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import np_
from oracle import train_aux as TA
from paper_2511_02510_gb300 import litevoxel as L

pytestmark = pytest.mark.gpu


def cu(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


def ws():
    return torch.empty(L.lv_train_workspace_size(), dtype=torch.uint8, device="cuda")


@pytest.mark.parametrize("n", [1, 777, 1_016_814])
def test_transmittance_loss(n):
    rng = np.random.default_rng(n)
    T = rng.uniform(0, 1, n).astype(np.float32)
    T[: n // 5] = 0.0
    loss = torch.zeros(1, device="cuda")
    g = torch.full((n,), 0.25, device="cuda")
    L.lv_transmittance_loss(cu(T), 0.3, loss, g, ws(), accumulate=True)
    torch.cuda.synchronize()
    ref, gref = TA.transmittance_concentration(T, 0.3)
    assert abs(float(loss.item()) - ref) <= 1e-5 * abs(ref) + 1e-12
    np.testing.assert_allclose(np_(g), 0.25 + gref, rtol=1e-6, atol=1e-9)
    g2 = torch.empty(n, device="cuda")
    L.lv_transmittance_loss(cu(T), 0.3, loss, g2, ws())
    torch.cuda.synchronize()
    np.testing.assert_allclose(np_(g2), gref, rtol=1e-6, atol=1e-12)


def adam_case(n, seed, step):
    rng = np.random.default_rng(seed)
    f = lambda *s: rng.normal(size=s).astype(np.float32)
    c = dict(density=f(n, 8), sh=f(n, 48) * 0.3, d_density=f(n, 8) * 1e-2, d_sh=f(n, 48) * 1e-3,
             m_d=f(n, 8) * 1e-3, v_d=np.abs(f(n, 8)) * 1e-5, m_s=f(n, 48) * 1e-4, v_s=np.abs(f(n, 48)) * 1e-7)
    if step == 1:
        for k in ("m_d", "v_d", "m_s", "v_s"):
            c[k][:] = 0.0
    return c


def params(step, tv):
    p = L.lv_adam_params()
    p.lr_density, p.lr_sh, p.beta1, p.beta2, p.eps, p.step, p.tv_weight = 0.05, 0.0025, 0.9, 0.999, 1e-15, step, tv
    return p


# the hyperparameters as the library receives them (FP32), for the oracle
F = lambda x: float(np.float32(x))
LR_D, LR_S, B1, B2, EPS = F(0.05), F(0.0025), F(0.9), F(0.999), F(1e-15)


@pytest.mark.parametrize("n,step,tv", [(1000, 1, 0.0), (65537, 7, 0.02), (300_000, 120, 1.5)])
def test_adam_voxels_fp32(n, step, tv):
    c = adam_case(n, n, step)
    t = {k: cu(v) for k, v in c.items()}
    tvl = torch.zeros(1, device="cuda")
    p = params(step, tv)
    L.lv_adam_voxels(t["density"], t["sh"], t["d_density"], t["d_sh"], t["m_d"], t["v_d"], t["m_s"], t["v_s"], p,
                     ws(), tv_loss=tvl)
    torch.cuda.synchronize()
    r = TA.adam_voxels(c["density"], c["sh"], c["d_density"], c["d_sh"], c["m_d"], c["v_d"], c["m_s"], c["v_s"],
                       LR_D, LR_S, B1, B2, EPS, step, tv_weight=F(tv))
    # moments: the FP32 gradient (photometric + TV, three rounded adds), two FP32 products and a sum:
    # a few ulps of the larger term (|b m| up to ~5e-3 / 5e-4, v terms ~1e-5 / 1e-7)
    def ulps(a, k=4):
        return k * np.spacing(np.float32(np.abs(a).max()))
    np.testing.assert_allclose(np_(t["m_d"]), r["m_density"], rtol=1e-6, atol=ulps(r["m_density"]))
    np.testing.assert_allclose(np_(t["v_d"]), r["v_density"], rtol=1e-6, atol=ulps(r["v_density"]))
    np.testing.assert_allclose(np_(t["m_s"]), r["m_sh"], rtol=1e-6, atol=ulps(r["m_sh"]))
    np.testing.assert_allclose(np_(t["v_s"]), r["v_sh"], rtol=1e-6, atol=ulps(r["v_sh"]))
    # parameters: p - u with u = lr m^ / (sqrt(v^) + eps): ~6 FP32 roundings (1e-6 relative) plus the
    # moments' own errors carried relatively (a few ulps of the larger of their two terms, large where
    # the terms cancel), plus the final subtraction's rounding (one ulp of p)
    for key, ref, p0, mp, vp, mr, vr in (("density", r["density"], c["density"], c["m_d"], c["v_d"],
                                          r["m_density"], r["v_density"]),
                                         ("sh", r["sh"], c["sh"], c["m_s"], c["v_s"], r["m_sh"], r["v_sh"])):
        got = np_(t[key]).astype(np.float64)
        u = np.abs(p0.astype(np.float64) - ref)
        sp = lambda a: np.spacing(np.abs(a).astype(np.float32)).astype(np.float64)
        em = 4 * sp(np.maximum(np.abs(B1 * mp), np.abs(mr - B1 * mp)))
        ev = 4 * sp(np.maximum(np.abs(B2 * vp), np.abs(vr - B2 * vp)))
        rel = 1e-6 + em / np.maximum(np.abs(mr), 1e-30) + 0.5 * ev / np.maximum(np.abs(vr), 1e-30)
        tol = rel * u + sp(ref)
        assert np.all(np.abs(got - ref) <= tol), (key, float((np.abs(got - ref) - tol).max()))
    assert abs(float(tvl.item()) - r["tv_loss"]) <= 1e-5 * abs(r["tv_loss"]) + 1e-12


def test_adam_voxels_mixed_storage_and_no_sh():
    n = 20000
    c = adam_case(n, 5, 3)
    t = {k: cu(v) for k, v in c.items()}
    dens16 = cu(c["density"], torch.float16)
    sh16 = cu(c["sh"], torch.bfloat16)
    sh_before = sh16.clone()
    L.lv_adam_voxels(dens16, sh16, t["d_density"], None, t["m_d"], t["v_d"], None, None, params(3, 0.1), ws())
    torch.cuda.synchronize()
    assert torch.equal(sh16, sh_before)                          # no SH gradient: SH and its moments untouched
    base = torch.as_tensor(c["density"]).half().float().numpy()
    r = TA.adam_voxels(base, None, c["d_density"], None, c["m_d"], c["v_d"], None, None, LR_D, LR_S, B1, B2, EPS, 3,
                       tv_weight=F(0.1))
    got = dens16.cpu().numpy().view(np.int16).astype(np.int32)
    want = r["density"].astype(np.float16).view(np.int16).astype(np.int32)
    assert np.abs(got - want).max() <= 1                          # at most one FP16 ulp apart
    assert (got != want).mean() < 1e-3
    # BF16 SH storage
    c2 = adam_case(4000, 6, 2)
    t2 = {k: cu(v) for k, v in c2.items()}
    sh16 = cu(c2["sh"], torch.bfloat16)
    L.lv_adam_voxels(t2["density"], sh16, t2["d_density"], t2["d_sh"], t2["m_d"], t2["v_d"], t2["m_s"], t2["v_s"],
                     params(2, 0.0), ws())
    torch.cuda.synchronize()
    base = torch.as_tensor(c2["sh"]).bfloat16().float().numpy()
    r = TA.adam(base, c2["d_sh"], c2["m_s"], c2["v_s"], LR_S, B1, B2, EPS, 2)[0]
    got = sh16.cpu().view(torch.int16).numpy().astype(np.int32)
    want = torch.as_tensor(r.astype(np.float32)).bfloat16().view(torch.int16).numpy().astype(np.int32)
    assert np.abs(got - want).max() <= 1


def test_adam_parameter_validation():
    n = 10
    t = {k: cu(v) for k, v in adam_case(n, 1, 2).items()}
    with pytest.raises(L.LvError):
        L.lv_adam_voxels(t["density"], t["sh"], t["d_density"], t["d_sh"], t["m_d"], t["v_d"], t["m_s"], t["v_s"],
                         params(0, 0.0), ws())
    p = params(1, 0.0)
    p.beta1 = 1.0
    with pytest.raises(L.LvError):
        L.lv_adam_voxels(t["density"], t["sh"], t["d_density"], t["d_sh"], t["m_d"], t["v_d"], t["m_s"], t["v_s"],
                         p, ws())


def test_training_iterations_reduce_the_loss():
    # forward -> LF loss + L_Tc -> backward (with dL/dT) -> Adam with TV, a few times on the tiny scene
    from paper_2511_02510_gb300 import synth
    from paper_2511_02510_gb300.raster import RasterContext, Scene
    sc = synth.scene_tiny()
    cam = synth.orbit_camera(64, 64, 60.0, 1.6, 30.0, 25.0, target=(0.5, 0.4, 0.5))
    scene = Scene.from_numpy(sc, "cuda")
    ctx = RasterContext([cam], scene.n)
    vox = scene.voxels()
    ctx.fit_capacity(vox)
    gt = cu(synth.smooth_image(64, 64, seed=3).reshape(-1, 3).astype(np.float32))
    lfp = L.lv_lf_params()
    lfp.eps, lfp.gamma_max, lfp.t0, lfp.t1, lfp.pctl_ppm = 1e-3, 0.6, 300.0, 600.0, 990000
    lf_ws = torch.empty(L.lv_lf_workspace_size([64], [64]), dtype=torch.uint8, device="cuda")
    tws = ws()
    n = scene.n
    md, vd = torch.zeros((n, 8), device="cuda"), torch.zeros((n, 8), device="cuda")
    ms, vs = torch.zeros((n, 48), device="cuda"), torch.zeros((n, 48), device="cuda")
    loss, tcl = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    dL = torch.empty((ctx.n_pix, 3), device="cuda")
    dT = torch.empty(ctx.n_pix, device="cuda")
    hist = []
    for it in range(30):
        ctx.reset_stats()
        ctx.forward(vox)
        L.lv_lf_weighted_loss(ctx.rgb, gt, [64], [64], 450.0, lfp, loss, dL, lf_ws)
        L.lv_transmittance_loss(ctx.T, 0.01, tcl, dT, tws)
        dd, ds = ctx.backward(vox, dL, None, dT)
        L.lv_adam_voxels(scene.density, scene.sh, dd, ds, md, vd, ms, vs, params(it + 1, 1e-4), tws)
        hist.append(float(loss.item()))
    ctx.check()
    assert hist[-1] < 0.95 * hist[0], hist
    assert sum(b < a for a, b in zip(hist, hist[1:])) >= 25        # decreasing almost every iteration


@pytest.mark.parametrize("count,dtype", [(1, torch.float32), (1003, torch.float32), (4096, torch.float16),
                                         (777, torch.bfloat16)])
def test_adam_array(count, dtype):
    rng = np.random.default_rng(count)
    p0 = rng.normal(size=count).astype(np.float32)
    g = (rng.normal(size=count) * 1e-2).astype(np.float32)
    m = (rng.normal(size=count) * 1e-3).astype(np.float32)
    v = (np.abs(rng.normal(size=count)) * 1e-5).astype(np.float32)
    pt, mt, vt = cu(p0, dtype), cu(m), cu(v)
    L.lv_adam_array(pt, cu(g), mt, vt, 0.01, params(4, 0.0))
    torch.cuda.synchronize()
    base = torch.as_tensor(p0).to(dtype).float().numpy()
    r, rm, rv = TA.adam(base, g, m, v, F(0.01), B1, B2, EPS, 4)
    np.testing.assert_allclose(np_(mt), rm, rtol=1e-6, atol=4 * np.spacing(np.float32(np.abs(rm).max())))
    np.testing.assert_allclose(np_(vt), rv, rtol=1e-6, atol=4 * np.spacing(np.float32(np.abs(rv).max())))
    if dtype == torch.float32:
        np.testing.assert_allclose(np_(pt), r, rtol=1e-6, atol=2e-6 * 0.01)
    else:
        bits = {torch.float16: torch.int16, torch.bfloat16: torch.int16}[dtype]
        got = pt.cpu().view(bits).numpy().astype(np.int32)
        want = torch.as_tensor(r.astype(np.float32)).to(dtype).view(bits).numpy().astype(np.int32)
        assert np.abs(got - want).max() <= 1
