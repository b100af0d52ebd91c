"""GPU parity and value of the learned interpolation correction.

- features: GPU stencil features / Lagrange values vs the oracle's (grid parity bar 1e-5);
- forward: GPU BF16 network vs the FP64 oracle evaluating the same (BF16-rounded) weights on
  the same inputs: <= 1e-3 of max |y|;
- gradients: GPU (BF16 operands, FP32 accumulation) vs FP64 oracle: <= 1e-2 per tensor;
- training: the trained correction beats plain Lagrange interpolation against the exact modal
  sum on held-out seas, without a worse finite-volume divergence.
"""
import numpy as np
import pytest

from oracle import divergence, interp as ointerp, mlp as omlp, modal
from tests._util import note_field, rel_linf, rel_linf_scaled, velocity_scale
from wavegen import configs, mesh as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12716_gb300 import build
    build.build()
    from paper_2005_12716_gb300 import api, learn
    return torch, api, learn


def bf16_round(a):
    """Round-to-nearest-even FP32 -> BF16 -> FP32 (what the packing kernel does)."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _rand_params(seed):
    p = omlp.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.1
    return p


def _rand_x(n, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, 68), np.float32)
    x[:, :64] = rng.uniform(-1, 1, (n, 64))
    x[:, 64:67] = rng.random((n, 3))
    return x


def test_features_match_oracle(env):
    torch, api, _ = env
    cfg = configs.jonswap3d_small()
    sea, z, tl, t = cfg["sea"], cfg["z_levels"], cfg["t_levels"], cfg["t_query"]
    pts = configs.mesh_points(cfg["mesh"])
    grid = api.fields_on_grid(api.upload_modes(sea), z, 2, tl)
    x, sc, lg, eta = api.mlp_features(grid, t, torch.from_numpy(pts).cuda())
    nodes, etas = [], []
    for tt in tl:
        n_, e_ = modal.fields_on_grid(modal.propagate(sea, tt), z, 2)
        nodes.append(n_)
        etas.append(e_)
    st, off, lag = ointerp.stencil_features(np.stack(nodes), sea["Lx"], sea["Ly"], z, tl, pts, t)
    n = len(pts)
    xg = x.cpu().numpy().reshape(n, 4, 68)
    sg = sc.cpu().numpy().reshape(n, 4)
    gs = xg[:, :, :64] * sg[:, :, None]
    vs = velocity_scale(st[:, 0], st[:, 1], st[:, 2])
    for f in range(4):
        scale = vs if f < 3 else np.max(np.abs(st[:, 3]))
        assert np.max(np.abs(gs[:, f] - st[:, f])) / scale <= 1e-5, f
        assert rel_linf_scaled(lg.cpu().numpy().reshape(n, 4)[:, f], lag[:, f], scale, field="uvwt"[f]) <= 1e-5
    np.testing.assert_allclose(xg[:, 0, 64:67], off, atol=2e-5)
    np.testing.assert_allclose(np.max(np.abs(xg[:, :, :64]), axis=2), 1.0, atol=1e-6)
    ref_eta = ointerp.interp_points(np.stack(nodes), np.stack(etas), sea["Lx"], sea["Ly"], z, tl,
                                    pts, t)["eta"]
    assert rel_linf(eta.cpu().numpy(), ref_eta) <= 1e-5


def test_forward_matches_oracle_bf16_weights(env):
    torch, api, _ = env
    p = _rand_params(11)
    mlp = api.Mlp(torch.from_numpy(api.mlp_flatten(p)))
    x = _rand_x(4 * 777, 12)
    y = mlp.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    pr = {k: (bf16_round(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
          for k, v in p.items()}
    yr, _ = omlp.forward(pr, x[:, :67].astype(np.float64))
    ref = yr[np.arange(len(x)), np.arange(len(x)) % 4]
    assert np.max(np.abs(y - ref)) / np.max(np.abs(ref)) <= 1e-3


def test_gradients_match_oracle(env):
    torch, api, _ = env
    p = _rand_params(21)
    mlp = api.Mlp(torch.from_numpy(api.mlp_flatten(p)))
    n = 3000
    x = _rand_x(n, 22)
    rng = np.random.default_rng(23)
    field = rng.integers(0, 4, n).astype(np.int32)
    target = (rng.standard_normal(n) * 0.3).astype(np.float32)
    batch = rng.choice(n, 1024, replace=False).astype(np.int32)
    g, loss = mlp.grad(torch.from_numpy(x).cuda(), torch.from_numpy(field).cuda(),
                       torch.from_numpy(target).cuda(), torch.from_numpy(batch).cuda())
    gd = api.mlp_unflatten(g.cpu().numpy())
    pr = {k: (bf16_round(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
          for k, v in p.items()}
    lr_, gr = omlp.loss_and_grad(pr, x[batch, :67].astype(np.float64), field[batch],
                                 target[batch].astype(np.float64))
    assert abs(float(loss.item()) - lr_) <= 1e-2 * lr_
    for k in gr:
        e = np.max(np.abs(gd[k] - gr[k])) / np.max(np.abs(gr[k]))
        assert e <= 1e-2, (k, e)


def test_checkpoint_roundtrip(env, tmp_path):
    torch, api, _ = env
    m = api.Mlp(api.mlp_init(5))
    m.step, m.seed = 17, 99
    m.m.fill_(0.25)
    path = tmp_path / "w.bin"
    m.save(str(path))
    m2 = api.Mlp.load(str(path))
    assert m2.step == 17 and m2.seed == 99
    assert torch.equal(m2.params, m.params) and torch.equal(m2.m, m.m)


def test_trained_correction_beats_plain_interpolation(env):
    """Train on random seas, evaluate on held-out seas against the FP64 modal sum."""
    torch, api, learn = env
    nx = ny = 64
    Lx = Ly = 4.0
    z = configs.jonswap3d_small()["z_levels"]
    x, f, tg = learn.make_dataset(48, 16384, nx, ny, Lx, Ly, z, seed=41)
    mlp = api.Mlp(api.mlp_init(42))
    losses = learn.train(mlp, x, f, tg, steps=4000, batch=8192, lr=2e-3, seed=43, log_every=100)
    assert losses[-1] < 0.5 * losses[0]
    rng = np.random.default_rng(44)
    err_plain, err_learned, div_plain, div_learned = [], [], [], []
    zlo, zhi = float(z[0]), float(z[-1])
    for s in range(3):
        sea = learn.random_sea(nx, ny, Lx, Ly, rng)
        modes = api.upload_modes(sea)
        grid = api.fields_on_grid(modes, z, 1, [0.0])
        pts = learn.sample_points(4000, Lx, Ly, zlo, zhi, rng)
        pd = torch.from_numpy(pts).cuda()
        plain, _ = api.interp(grid, 0.0, pd, p_mode="phit")
        lrn, _ = api.interp_learned(grid, 0.0, pd, mlp, p_mode="phit")
        ex = modal.fields_at_points(sea, pts.astype(np.float64), p_mode="phit")
        vs = velocity_scale(ex["u"], ex["v"], ex["w"])
        for store, o in ((err_plain, plain), (err_learned, lrn)):
            e = [np.sqrt(np.mean((o[k].cpu().numpy() - ex[k]) ** 2)) / vs for k in ("u", "v", "w")]
            store.append(np.mean(e))
        # divergence on a small hex mesh inside the domain
        ze = np.linspace(zlo + 0.05, -0.02, 7)
        m = M.cylinder_ogrid((2.0, 2.0), 0.3, 1.5, 10, 24, ze, 1.05)
        fc = torch.from_numpy(m["face_centres"].astype(np.float32)).cuda()
        area = torch.from_numpy(m["face_area"].astype(np.float32)).cuda()
        cf = torch.from_numpy(m["cell_faces"]).cuda()
        vol = torch.from_numpy(m["cell_volume"].astype(np.float32)).cuda()
        for store, fn in ((div_plain, api.interp), (div_learned, lambda g_, t_, p_: api.interp_learned(g_, t_, p_, mlp))):
            o, _ = fn(grid, 0.0, fc)
            d = api.fv_divergence(o["u"], o["v"], o["w"], area, cf, vol).cpu().numpy()
            store.append(np.sqrt(np.mean(d.astype(np.float64) ** 2)))
    note_field("rms_err_learned/plain", np.mean(err_learned) / np.mean(err_plain), 0.0)
    note_field("rms_div_learned/plain", np.mean(div_learned) / np.mean(div_plain), 0.0)
    assert np.mean(err_learned) < np.mean(err_plain), (err_learned, err_plain)
    # the interpolated divergence must be no worse than the plain interpolation's
    assert np.mean(div_learned) <= np.mean(div_plain), (div_learned, div_plain)


@pytest.mark.parametrize("order", ["mesh", "random"])
def test_fused_learned_gather_matches_oracle(env, order):
    """interp_learned (one fused kernel: stencil gather, features, three BF16 layers, correction)
    against the oracle chain on the FP64 grid: stencil features -> FP64 network on the same
    BF16-rounded weights -> lagrange + s_f * out_scale * y[f] -> Bernoulli. Mesh-ordered points
    take the staged-box path; random points (chunks whose box does not fit) the per-point path.
    Bar: 1e-5 of the field scale plus 1e-3 of the largest correction."""
    torch, api, _ = env
    cfg = configs.jonswap3d_small()
    sea, z, tl, t = cfg["sea"], cfg["z_levels"], cfg["t_levels"], cfg["t_query"]
    if order == "mesh":
        pts = configs.mesh_points(cfg["mesh"])[:5000]
    else:
        rng = np.random.default_rng(61)
        pts = np.stack([rng.uniform(0, sea["Lx"], 3001), rng.uniform(0, sea["Ly"], 3001),
                        rng.uniform(float(z[0]), float(z[-1]), 3001)], 1).astype(np.float32)
    p = _rand_params(31)
    out_scale = 0.05
    mlp = api.Mlp(torch.from_numpy(api.mlp_flatten(p)), out_scale=out_scale)
    grid = api.fields_on_grid(api.upload_modes(sea), z, 2, tl)
    got, _ = api.interp_learned(grid, t, torch.from_numpy(pts).cuda(), mlp, p_mode="phit")
    nodes, etas = [], []
    for tt in tl:
        n_, e_ = modal.fields_on_grid(modal.propagate(sea, tt), z, 2)
        nodes.append(n_)
        etas.append(e_)
    st, off, lag = ointerp.stencil_features(np.stack(nodes), sea["Lx"], sea["Ly"], z, tl, pts, t)
    pr = {k: (bf16_round(v) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64))
          for k, v in p.items()}
    n = len(pts)
    corr = np.zeros((n, 4))
    for f in range(4):
        x, s = omlp.features(st[:, f], off)
        y, _ = omlp.forward(pr, x)
        corr[:, f] = s * out_scale * y[:, f]
    ref = lag + corr
    vs = velocity_scale(ref[:, 0], ref[:, 1], ref[:, 2])
    cmax = np.max(np.abs(corr))
    for f, k in enumerate(("u", "v", "w", "p")):          # p_mode "phit": p is dphi/dt
        scale = vs if f < 3 else np.max(np.abs(ref[:, 3]))
        e = np.max(np.abs(got[k].cpu().numpy() - ref[:, f]))
        assert e <= 1e-5 * scale + 1e-3 * cmax, (k, e, scale, cmax)
    ref_eta = ointerp.interp_points(np.stack(nodes), np.stack(etas), sea["Lx"], sea["Ly"], z, tl,
                                    pts, t)["eta"]
    assert rel_linf(got["eta"].cpu().numpy(), ref_eta) <= 1e-5


def test_train_save_load_resume_bit_identical(env, tmp_path):
    """swense_mlp_train (the training loop in the library, mini-batches drawn from the seed and
    the step), swense_mlp_save and swense_mlp_load through the C ABI: 30 steps, a checkpoint, and
    20 more steps from the checkpoint give bit for bit the parameters and Adam moments of 50
    uninterrupted steps; the loss falls."""
    torch, api, learn = env
    z = configs.jonswap3d_small()["z_levels"]
    x, f, tg = learn.make_dataset(4, 2048, 64, 64, 4.0, 4.0, z, seed=61)
    losses = torch.zeros(50, dtype=torch.float32, device="cuda")

    def fresh():
        m = api.Mlp(api.mlp_init(62), out_scale=0.0)
        m.seed = 63
        return m
    a = fresh()
    a.train(x, f, tg, 30, batch=1024, lr=2e-3, schedule_steps=50, losses=losses[:30])
    assert a.step == 30 and a.out_scale > 0
    path = tmp_path / "mlp.bin"
    a.save(path)
    b = api.Mlp.load(path)
    assert (b.step, b.seed, b.out_scale) == (a.step, a.seed, a.out_scale)
    assert torch.equal(b.params, a.params) and torch.equal(b.m, a.m) and torch.equal(b.v, a.v)
    b.train(x, f, tg, 20, batch=1024, lr=2e-3, schedule_steps=50, losses=losses[30:])
    c = fresh()
    c.train(x, f, tg, 50, batch=1024, lr=2e-3, schedule_steps=50)
    assert c.step == b.step == 50 and c.out_scale == b.out_scale
    for t1, t2 in ((b.params, c.params), (b.m, c.m), (b.v, c.v), (b.packed, c.packed)):
        assert torch.equal(t1, t2)
    lo = losses.cpu().numpy()
    assert lo[-10:].mean() < lo[:10].mean()


def test_targets_are_the_scaled_residuals(env):
    """swense_mlp_targets: row 4 i + f = (exact_f - lagrange_f) / s_f with field id f."""
    torch, api, learn = env
    from paper_2005_12716_gb300 import _swense as S
    rng = np.random.default_rng(71)
    n = 5000
    ex = [torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda() for _ in range(4)]
    lg = torch.from_numpy(rng.standard_normal(4 * n).astype(np.float32)).cuda()
    sc = torch.from_numpy(rng.uniform(0.5, 2.0, 4 * n).astype(np.float32)).cuda()
    tg = torch.empty(4 * n, dtype=torch.float32, device="cuda")
    fd = torch.empty(4 * n, dtype=torch.int32, device="cuda")
    S.swense_mlp_targets(*ex, lg, sc, n, tg, fd)
    e = torch.stack(ex, 1).reshape(-1)
    assert torch.equal(tg, (e - lg) / sc)
    assert torch.equal(fd.cpu(), torch.arange(4, dtype=torch.int32).repeat(n))
