"""The training slice (Sec. 4.4, MSE term) through the C ABI: the GPU trainer's
loss and gradients against the oracle's FP64 autograd gradient, Adam steps
that lower the loss, and a short training on synthetic (guide, fine-step
reference) pairs whose held-out error falls far below the untrained network's;
the exported weight blob reproduces the trainer's outputs through
nsl_predict_lightmaps."""
import math

import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    nsl.load()
    return nsl


def _offsets():
    off, out = 0, []
    for name, shape, _ in I.param_spec(16):
        n = int(np.prod(shape))
        out.append((name, off, n))
        off += n
    return out


@pytest.mark.parametrize("weights", [None, (3.0, 1.0, 0.5, 2.0, 1.0, 4.0, 1.0, 0.25)])
def test_gradients_match_oracle(lib, weights):
    import torch
    from oracle import grad as OG
    B, H, W = 2, 16, 24
    rng = np.random.default_rng(50)
    guides = np.stack([np.stack([rng.uniform(0, 0.2, (H, W)), rng.uniform(0, 1, (H, W)), rng.uniform(0, 60, (H, W))])
                       for _ in range(B)]).astype(np.float32)
    targets = rng.uniform(0, 0.1, (B, 8, H, W)).astype(np.float32)
    blob = I.pack_blob(I.make_params(16, 0), 16)
    opts = lib.train_opts(batch=B, width=W, height=H) if weights is None else \
        lib.train_opts(batch=B, width=W, height=H, plane_weight=weights)
    tr = lib.Trainer(blob, opts)
    g_dev = torch.from_numpy(guides).cuda()
    t_dev = torch.from_numpy(targets).cuda()
    loss = tr.step(g_dev, t_dev, 1 / 40.0, update=False)
    grad = torch.empty(tr.n_params, device="cuda")
    tr.gradients(grad)
    torch.cuda.synchronize()
    flat = I.flat_params(I.make_params(16, 0)).astype(np.float64)
    ref_loss, ref_grad, _ = OG.mse_and_grad(flat, guides.astype(np.float64), targets.astype(np.float64), 16,
                                            1 / 40.0, plane_weight=weights)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    got = grad.cpu().numpy().astype(np.float64)
    worst = {}
    for name, o, n in _offsets():
        r = ref_grad[o:o + n]
        err = float(np.abs(got[o:o + n] - r).max() / max(np.abs(r).max(), 1e-30))
        worst[name] = err
    assert max(worst.values()) <= 2e-3, sorted(worst.items(), key=lambda kv: -kv[1])[:5]
    tr.close()


def test_adam_steps_lower_the_loss(lib):
    import torch
    B, H, W = 2, 32, 32
    rng = np.random.default_rng(51)
    guides = torch.from_numpy(np.stack([np.stack([rng.uniform(0, 0.2, (H, W)), rng.uniform(0, 1, (H, W)),
                                                  rng.uniform(0, 60, (H, W))]) for _ in range(B)]).astype(np.float32)).cuda()
    targets = torch.from_numpy(rng.uniform(0, 0.1, (B, 8, H, W)).astype(np.float32)).cuda()
    tr = lib.Trainer(I.pack_blob(I.make_params(16, 0), 16), lib.train_opts(batch=B, width=W, height=H, lr=1e-3))
    losses = [tr.step(guides, targets, 1 / 40.0) for _ in range(30)]
    assert losses[-1] < 0.05 * losses[0], losses[::5]
    tr.close()


def _dataset(lib, count, n, size, seed, step=2.0, hf=0.5):
    """(guides [count,3,S,S], targets [count,8,S,S]) of seeded blob x fBm
    volumes under seeded perspective cameras: the guide march and the
    fine-step reference (emissive plane 0)."""
    import torch
    blob = I.pack_blob(I.make_params(16, 0), 16)
    ctx = lib.Context((n, n, n), lib.NSL_F32, blob, size, size)
    g = torch.empty((count, 3, size, size), device="cuda")
    t = torch.zeros((count, 8, size, size), device="cuda")
    ref = torch.empty((7, size, size), device="cuda")
    for k in range(count):
        d = torch.from_numpy(I.blob_fbm_volume(n, seed + k)).cuda()
        cam = I.perspective_camera(n, seed + k, size, size)
        ctx.guiding_map(d, None, cam, step, g[k])
        lib.nsl_reference_lightmaps(ctx.ctx, None, None, cam, hf, ref)
        t[k, :7] = ref
    torch.cuda.synchronize()
    ctx.close()
    return g, t


def plane_weights(targets):
    """1 / (mean over frames of each lightmap plane's range)^2 for the six
    lightmap planes, 1 for T and E: the planes' squared errors on one scale."""
    t = targets.cpu().numpy()
    rng = [float(np.mean(np.abs(t[:, c]).max(axis=(1, 2)))) for c in range(6)]
    return [1.0 / max(r, 1e-3) ** 2 for r in rng] + [1.0, 1.0]


def test_training_fits_the_fine_reference(lib):
    """Adam with a cosine learning-rate decay on 48 synthetic pairs (32^3
    volumes, 32 x 32 perspective images, plane-weighted squared error) brings
    the held-out error far below the untrained network's, and the exported
    blob reproduces the trainer's forward through nsl_predict_lightmaps."""
    import torch
    n, S, B, steps, lr0 = 32, 32, 8, 1500, 2e-3
    ds = 1.0 / math.sqrt(3.0 * n * n)
    g_tr, t_tr = _dataset(lib, 48, n, S, seed=100)
    g_te, t_te = _dataset(lib, 8, n, S, seed=900)
    blob0 = I.pack_blob(I.make_params(16, 0), 16)
    tr = lib.Trainer(blob0, lib.train_opts(batch=B, width=S, height=S, lr=lr0, plane_weight=plane_weights(t_tr)))
    rng = np.random.default_rng(52)
    for it in range(steps):
        tr.set_lr(lr0 * 0.5 * (1.0 + math.cos(math.pi * it / steps)) + 1e-6)
        idx = torch.from_numpy(rng.choice(48, B, replace=False)).cuda()
        tr.step(g_tr[idx].contiguous(), t_tr[idx].contiguous(), ds)

    def held_out_err(blob):
        """Median over the held-out frames of the largest error over the seven
        physical planes, relative to the plane's range: max-abs and RMS."""
        ctx = lib.Context((n, n, n), lib.NSL_F32, blob, S, S)
        mx, rms = [], []
        out = torch.empty((8, S, S), device="cuda")
        for k in range(8):
            ctx.predict_lightmaps(g_te[k].contiguous(), S, S, lib.NSL_PREC_F32, out)
            torch.cuda.synchronize()
            o, t = out.cpu().numpy()[:7], t_te[k].cpu().numpy()[:7]
            r = [max(np.abs(t[c]).max(), 1e-30) for c in range(7)]
            mx.append(max(float(np.abs(o[c] - t[c]).max() / r[c]) for c in range(7)))
            rms.append(max(float(np.sqrt(((o[c] - t[c]) ** 2).mean()) / r[c]) for c in range(7)))
        ctx.close()
        return float(np.median(mx)), float(np.median(rms))
    before, after = held_out_err(blob0), held_out_err(tr.blob())
    print(f"\nheld-out error (median over 8 frames, max over planes, of range): untrained max {before[0]:.3g} "
          f"rms {before[1]:.3g}, trained max {after[0]:.3g} rms {after[1]:.3g}")
    assert after[0] < 0.05 * before[0] and after[1] < 0.02 * before[1] and after[1] < 0.4
    # the exported blob: nsl_predict_lightmaps (FP32) equals the trainer's own forward
    trained = tr.blob()
    ctx = lib.Context((n, n, n), lib.NSL_F32, trained, S, S)
    lm = torch.empty((8, S, S), device="cuda")
    ctx.predict_lightmaps(g_te[0].contiguous(), S, S, lib.NSL_PREC_F32, lm)
    torch.cuda.synchronize()
    ctx.close()
    tr2 = lib.Trainer(trained, lib.train_opts(batch=1, width=S, height=S))
    loss_same = tr2.step(g_te[0:1].contiguous(), lm[None].contiguous(), ds, update=False)
    assert loss_same <= 1e-10 * max(float((lm ** 2).mean()), 1e-30)
    tr.close()
    tr2.close()
