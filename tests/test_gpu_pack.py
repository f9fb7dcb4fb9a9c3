"""GPU parity of the packed two-texture export (Sec. 3, Fig. 2): the CUDA
kernel through the C ABI against the oracle, bit for bit in every format."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    nsl.load()
    import torch
    assert torch.cuda.is_available()
    return nsl


def _planes(H, W, seed):
    rng = np.random.default_rng(seed)
    lm = (rng.normal(size=(8, H, W)) * 0.6 + 0.4).astype(np.float32)
    # special values: NaN, infinities, signed zero, an exact tie (0.5 * 255 =
    # 127.5), a subnormal-range code
    flat = lm.reshape(8, -1)
    flat[0, :6] = [np.nan, np.inf, -np.inf, -0.0, 0.5, 1.0]
    flat[1, :3] = [0.25, 127.5 / 255.0, 2.0 ** -9]
    return lm


@pytest.mark.parametrize("H,W", [(8, 8), (24, 136), (512, 512)])
@pytest.mark.parametrize("fmt", [0, 1, 2], ids=["rgba8", "rgba16f", "rgba32f"])
def test_pack_bitwise(lib, orc, H, W, fmt):
    import torch
    lm = _planes(H, W, H * 7 + W + fmt)
    dt = {0: torch.uint8, 1: torch.float16, 2: torch.float32}[fmt]
    t1 = torch.empty((H, W, 4), dtype=dt, device="cuda")
    t2 = torch.empty((H, W, 4), dtype=dt, device="cuda")
    lib.nsl_pack_lightmaps(torch.from_numpy(lm).cuda(), W, H, fmt, t1, t2)
    torch.cuda.synchronize()
    r1, r2 = orc.pack_lightmaps(lm, fmt)
    g1, g2 = t1.cpu().numpy(), t2.cpu().numpy()
    if fmt == 0:
        np.testing.assert_array_equal(g1, r1)
        np.testing.assert_array_equal(g2, r2)
    else:   # bit patterns of every number; a NaN stays a NaN (its payload is not specified)
        bits = np.uint16 if fmt == 1 else np.uint32
        for g, r in ((g1, r1), (g2, r2)):
            nan = np.isnan(r)
            np.testing.assert_array_equal(np.isnan(g), nan)
            np.testing.assert_array_equal(g.view(bits)[~nan], r.view(bits)[~nan])


def test_pack_after_network(lib, orc):
    """The export of real network output: guide -> lightmaps -> textures."""
    import torch
    from paper_2604_03748_gb300 import inputs as I
    pf = I.small_case(24, 32, 24, seed=11, kind=I.PERSP, step=2.0)
    H, W = pf.camera.height, pf.camera.width
    ctx = lib.Context(pf.density.shape, lib.NSL_F32, I.pack_blob(I.make_params(16, 0), 16), W, H)
    g = torch.empty((3, H, W), device="cuda")
    lm = torch.empty((8, H, W), device="cuda")
    ctx.guiding_map(torch.from_numpy(pf.density).cuda(), torch.from_numpy(pf.mask).cuda(), pf.camera, pf.step, g)
    ctx.predict_lightmaps(g, W, H, lib.NSL_PREC_BF16, lm)
    t1 = torch.empty((H, W, 4), dtype=torch.uint8, device="cuda")
    t2 = torch.empty_like(t1)
    lib.nsl_pack_lightmaps(lm, W, H, lib.NSL_TEX_RGBA8, t1, t2)
    torch.cuda.synchronize()
    r1, r2 = orc.pack_lightmaps(lm.cpu().numpy(), 0)
    np.testing.assert_array_equal(t1.cpu().numpy(), r1)
    np.testing.assert_array_equal(t2.cpu().numpy(), r2)
    ctx.close()


def test_pack_rejects_bad_arguments(lib):
    import torch
    lm = torch.zeros((8, 16, 16), device="cuda")
    t = torch.empty((16, 16, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.NslError):
        lib.check(lib.load().nsl_pack_lightmaps(lm.data_ptr(), 16, 16, 5, t.data_ptr(), t.data_ptr(), None),
                  "pack")
    with pytest.raises(lib.NslError):
        lib.check(lib.load().nsl_pack_lightmaps(lm.data_ptr() + 4, 16, 16, 0, t.data_ptr(), t.data_ptr(), None),
                  "pack")
    with pytest.raises(lib.NslError):
        lib.check(lib.load().nsl_pack_lightmaps(lm.data_ptr(), 12, 16, 0, t.data_ptr(), t.data_ptr(), None),
                  "pack")
    with pytest.raises(ValueError):
        lib.nsl_pack_lightmaps(lm, 16, 16, 1, t, t)       # uint8 tensor for a half format
