"""FP64 gradient of the training slice's loss (Sec. 4.4, the MSE term).

TEST INFRASTRUCTURE ONLY: the tests load it to check the GPU trainer's
gradients; the product path never imports it.

loss(params) = mean over images, planes and pixels of w_plane (net(guide) - target)^2,
with net the lightmap network of Sec. 4.3 (the oracle's nslo_net_forward) and
its gradient with respect to every parameter in weight-blob order.  The
network is assembled here from PyTorch float64 library operations (conv2d,
conv_transpose2d, max_pool2d, layer_norm, adaptive_avg_pool2d) in the order of
the oracle's forward, and differentiated by autograd; the tests pin both the
value (against the C oracle) and the gradient (against central differences of
the C oracle's loss).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as Fn

ADAPTER_PLANES = ((4, 5), (0, 1), (2, 3), (6, 7))   # F&B, L&R, U&D, A&E


def _split(flat, c0):
    """Parameter tensors of the flat blob vector, in blob order (views)."""
    c = [c0, 2 * c0, 4 * c0, 8 * c0]
    out, off = [], 0

    def take(*shape):
        nonlocal off
        n = int(np.prod(shape))
        t = flat[off:off + n].view(*shape)
        off += n
        return t
    convs = [(3, c[0]), (c[0], c[0]), (c[0], c[1]), (c[1], c[1]), (c[1], c[2]), (c[2], c[2]), (c[2], c[3]),
             (c[3], c[3])]
    for ci, co in convs:
        out.append(("conv", take(co, ci, 3, 3), take(co)))
    for up_in, up_out in ((c[3], c[2]), (c[2], c[1]), (c[1], c[0])):
        out.append(("up", take(up_in, up_out, 2, 2), take(up_out)))
        out.append(("conv", take(up_out, 2 * up_out, 3, 3), take(up_out)))
        out.append(("conv", take(up_out, up_out, 3, 3), take(up_out)))
    C = c0
    adapters = []
    for _ in range(4):
        a = {}
        a["ln1w"], a["ln1b"] = take(C), take(C)
        a["pw1w"], a["pw1b"] = take(2 * C, C), take(2 * C)
        a["dww"], a["dwb"] = take(2 * C, 1, 3, 3), take(2 * C)
        a["scaw"], a["scab"] = take(C, C), take(C)
        a["pw2w"], a["pw2b"] = take(C, C), take(C)
        a["beta"] = take(C)
        a["ln2w"], a["ln2b"] = take(C), take(C)
        a["f1w"], a["f1b"] = take(2 * C, C), take(2 * C)
        a["f2w"], a["f2b"] = take(C, C), take(C)
        a["gamma"] = take(C)
        a["hw"], a["hb"] = take(2, C), take(2)
        adapters.append(a)
    assert off == flat.numel(), (off, flat.numel())
    return out, adapters


def _forward(flat, guides, c0, depth_scale):
    layers, adapters = _split(flat, c0)
    x = guides.clone()
    x[:, 2] = x[:, 2] * depth_scale
    it = iter(layers)

    def conv(v):
        _, w, b = next(it)
        return torch.relu(Fn.conv2d(v, w, b, padding=1))

    def up(v):
        _, w, b = next(it)
        return Fn.conv_transpose2d(v, w, b, stride=2)
    s1 = conv(conv(x))
    s2 = conv(conv(Fn.max_pool2d(s1, 2)))
    s3 = conv(conv(Fn.max_pool2d(s2, 2)))
    bt = conv(conv(Fn.max_pool2d(s3, 2)))
    d = conv(conv(torch.cat([up(bt), s3], 1)))
    d = conv(conv(torch.cat([up(d), s2], 1)))
    F = conv(conv(torch.cat([up(d), s1], 1)))
    C = c0
    out = [None] * 8

    def pw(v, w, b):
        return Fn.conv2d(v, w[:, :, None, None], b)

    def ln(v, w, b):
        return Fn.layer_norm(v.permute(0, 2, 3, 1), (C,), w, b, eps=1e-6).permute(0, 3, 1, 2)
    for a, planes in zip(adapters, ADAPTER_PLANES):
        t = pw(ln(F, a["ln1w"], a["ln1b"]), a["pw1w"], a["pw1b"])
        t = Fn.conv2d(t, a["dww"], a["dwb"], padding=1, groups=2 * C)
        t = t[:, :C] * t[:, C:]
        t = t * pw(Fn.adaptive_avg_pool2d(t, 1), a["scaw"], a["scab"])
        y = F + pw(t, a["pw2w"], a["pw2b"]) * a["beta"][None, :, None, None]
        t = pw(ln(y, a["ln2w"], a["ln2b"]), a["f1w"], a["f1b"])
        z = y + pw(t[:, :C] * t[:, C:], a["f2w"], a["f2b"]) * a["gamma"][None, :, None, None]
        h = pw(z, a["hw"], a["hb"])
        out[planes[0]], out[planes[1]] = h[:, 0], h[:, 1]
    return torch.stack(out, 1)


def mse_and_grad(params_flat, guides, targets, c0, depth_scale, plane_weight=None):
    """(loss, gradient[n_params], outputs[B,8,H,W]) in float64 for guides
    [B,3,H,W] and targets [B,8,H,W]; plane_weight (8 values, default 1) weighs
    each output plane's squared error."""
    flat = torch.tensor(np.asarray(params_flat, np.float64), requires_grad=True)
    g = torch.from_numpy(np.asarray(guides, np.float64))
    t = torch.from_numpy(np.asarray(targets, np.float64))
    w = torch.ones(8, dtype=torch.float64) if plane_weight is None else torch.tensor(
        np.asarray(plane_weight, np.float64))
    out = _forward(flat, g, c0, depth_scale)
    loss = (w[None, :, None, None] * (out - t) ** 2).mean()
    loss.backward()
    return float(loss.detach()), flat.grad.numpy().copy(), out.detach().numpy()
