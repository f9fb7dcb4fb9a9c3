"""Serving through the C ABI: resident plumes, HBM-budget admission with LRU
eviction, continuous batching over several streams.  The central check: every
request's lightmaps and shading are bitwise the same when it runs alone and
when it runs in a mix of concurrent requests of other plumes and sizes (and
equal to the batched render of the same frame)."""
import numpy as np
import pytest

from paper_2604_03748_gb300 import inputs as I

pytestmark = pytest.mark.gpu

C0 = 16


@pytest.fixture(scope="module")
def lib():
    from paper_2604_03748_gb300 import build, nsl
    build.build()
    nsl.load()
    import torch
    assert torch.cuda.is_available()
    return nsl


def _plumes(count=6, seed=31):
    """Small plumes of mixed sizes; each gets three request cameras."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.choice([24, 32, 40, 48]))
        w = int(rng.choice([32, 64, 96, 128]))
        h = int(rng.choice([32, 64, 96, 128]))
        vol = I.blob_fbm_volume(n, seed + k)
        if k % 2:
            vol = vol.astype(np.float16)
        mask = None
        if k % 3 == 0:
            mask, _ = I.sphere_mask(n, n / 6.0, seed + k)
        cams = [I.perspective_camera(n, 100 * k + j, w, h) if j != 1 else I.orbit_ortho_camera(n, 100 * k + j, w, h)
                for j in range(3)]
        out.append(dict(vol=vol, mask=mask, n=n, w=w, h=h, cams=cams, lights=[I.random_light(7 * k + j)
                                                                              for j in range(3)]))
    return out


def _bufs(p):
    """Output buffers for one request.  The server's streams do not wait on
    torch's stream, so the fill is finished before the buffers are handed over;
    the caller keeps both alive until the request completes."""
    import torch
    lm = torch.full((8, p["h"], p["w"]), float("nan"), dtype=torch.float32, device="cuda")
    rgba = torch.full((4, p["h"], p["w"]), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    return lm, rgba


def _memcpy_d2d(dst, src, nbytes):
    """cudaMemcpy through the CUDA runtime the library is linked against."""
    import ctypes
    import glob
    import os
    rt = None
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            pass
    if rt is None:
        cands = glob.glob(os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib*", "libcudart.so*"))
        rt = ctypes.CDLL(cands[0])
    rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    assert rt.cudaMemcpy(ctypes.c_void_p(dst), ctypes.c_void_p(src), nbytes, 3) == 0


def _server(lib, **kw):
    blob = I.pack_blob(I.make_params(C0, seed=0), C0)
    return lib.Server(blob, lib.server_opts(**kw))


@pytest.mark.parametrize("precision", [3, 1, 2, 4], ids=["f16", "bf16", "fp8", "bf16x3"])
def test_serving_alone_equals_mix(lib, precision):
    import torch
    plumes = _plumes()
    srv = _server(lib, hbm_budget_bytes=2 << 30, streams=2, max_batch=8, precision=precision)
    ids = [srv.add_plume(p["vol"], p["mask"], 2.0, p["w"], p["h"]) for p in plumes]
    # alone: one request at a time
    alone = {}
    for pid, p in zip(ids, plumes):
        for j in range(3):
            lm, rgba = _bufs(p)
            rid = srv.submit(pid, p["cams"][j], p["lights"][j], lm, rgba)
            lat = srv.wait(rid)
            assert lat > 0
            alone[(pid, j)] = (lm.cpu().numpy(), rgba.cpu().numpy())
    # the mix: every request in flight at once, interleaved across plumes
    # (three requests per plume also exercise the per-plume ordering)
    mix = {(pid, j): _bufs(p) for j in range(3) for pid, p in zip(ids, plumes)}
    rids = []
    for j in range(3):
        for pid, p in zip(ids, plumes):
            lm, rgba = mix[(pid, j)]
            rids.append(srv.submit(pid, p["cams"][j], p["lights"][j], lm, rgba))
    for rid in rids:
        srv.wait(rid)
    torch.cuda.synchronize()
    for key, (lm, rgba) in mix.items():
        assert np.array_equal(lm.cpu().numpy(), alone[key][0]), key
        assert np.array_equal(rgba.cpu().numpy(), alone[key][1]), key
    st = srv.stats()
    assert st["completed"] == st["submitted"] == 2 * 3 * len(plumes)
    assert st["failed"] == 0 and st["queued"] == 0 and st["running"] == 0
    assert st["batches"] < st["completed"]          # the mix was batched
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["used_bytes"] <= st["budget_bytes"]

    # the same frame through the batched render (resident state path too)
    p = plumes[0]
    b = lib.Batch(I.pack_blob(I.make_params(C0, seed=0), C0), max_plumes=1)
    item = dict(density=torch.from_numpy(np.ascontiguousarray(p["vol"])).cuda(),
                mask=None if p["mask"] is None else torch.from_numpy(p["mask"]).cuda(),
                camera=p["cams"][2], step=2.0, light=p["lights"][2],
                guide=torch.empty((3, p["h"], p["w"]), device="cuda"),
                lightmaps=torch.empty((8, p["h"], p["w"]), device="cuda"),
                rgba=torch.empty((4, p["h"], p["w"]), device="cuda"))
    b.render([item], precision)
    torch.cuda.synchronize()
    assert np.array_equal(item["lightmaps"].cpu().numpy(), alone[(ids[0], 2)][0])
    # a request without output buffers writes the plume's resident state
    rid = srv.submit(ids[0], p["cams"][2], p["lights"][2])
    srv.wait(rid)
    g_ptr, lm_ptr, _, resident = srv.plume_state(ids[0])
    assert resident and lm_ptr
    out = torch.empty((8, p["h"], p["w"]), device="cuda")
    _memcpy_d2d(out.data_ptr(), lm_ptr, out.numel() * 4)
    assert np.array_equal(out.cpu().numpy(), alone[(ids[0], 2)][0])
    b.close()
    srv.close()


def test_serving_eviction_under_small_budget(lib):
    import torch
    plumes = _plumes(count=8, seed=41)
    mb = 1 << 20

    def a256(v):
        return (v + 255) // 256 * 256

    # resident bytes of each plume (staged padded-quad grid + 15 state planes)
    # and the largest upload buffers; the budget holds the two slots' scratch,
    # their upload buffers and about half of the plumes
    foot = [a256((p["n"] + 1) ** 2 * (p["n"] + 2) * 16) + a256(15 * p["w"] * p["h"] * 4) for p in plumes]
    up = max(p["vol"].nbytes for p in plumes) + max(p["n"] ** 3 for p in plumes)
    budget = 2 * 32 * mb + 2 * up + sum(foot) // 2
    srv = _server(lib, hbm_budget_bytes=budget, scratch_bytes_per_stream=32 * mb, streams=2, max_batch=4)
    ids = [srv.add_plume(p["vol"], p["mask"], 2.0, p["w"], p["h"]) for p in plumes]
    alone = {}
    for pid, p in zip(ids, plumes):
        lm, rgba = _bufs(p)
        srv.wait(srv.submit(pid, p["cams"][0], p["lights"][0], lm, rgba))
        alone[pid] = lm.cpu().numpy()
    st = srv.stats()
    assert st["evictions"] > 0 and st["used_bytes"] <= st["budget_bytes"]
    assert st["resident_plumes"] < len(plumes)
    srv.reset_stats()
    # cycle over all plumes twice with everything in flight: admissions and
    # evictions interleave with running batches
    outs = [(pid, *_bufs(p)) for rep in range(2) for pid, p in zip(ids, plumes)]
    rids = []
    for pid, lm, rgba in outs:
        p = plumes[ids.index(pid)]
        rids.append(srv.submit(pid, p["cams"][0], p["lights"][0], lm, rgba))
        s = srv.stats()
        assert s["used_bytes"] <= s["budget_bytes"]
    srv.drain()
    torch.cuda.synchronize()
    for pid, lm, _ in outs:
        assert np.array_equal(lm.cpu().numpy(), alone[pid]), pid
    st = srv.stats()
    assert st["completed"] == len(outs) and st["failed"] == 0
    assert st["admissions"] > 0 and st["evictions"] > 0
    srv.close()


def test_serving_errors(lib):
    import torch
    mb = 1 << 20
    srv = _server(lib, hbm_budget_bytes=80 * mb, scratch_bytes_per_stream=32 * mb, streams=2)
    big = np.zeros((96, 96, 96), np.float32)           # staged 97*97*98*16 B = 14.8 MB: fits
    with pytest.raises(lib.NslError):                  # a 1024^2 frame's state alone is 63 MB
        srv.add_plume(big, None, 2.0, 1024, 1024)
    p = _plumes(count=1, seed=51)[0]
    pid = srv.add_plume(p["vol"], p["mask"], 2.0, p["w"], p["h"])
    with pytest.raises(lib.NslError):                  # larger than the plume's billboard
        srv.submit(pid, I.perspective_camera(p["n"], 1, p["w"] + 8, p["h"]), p["lights"][0])
    with pytest.raises(lib.NslError):
        srv.submit(pid + 5, p["cams"][0], p["lights"][0])
    rids = [srv.submit(pid, p["cams"][0], p["lights"][0]) for _ in range(4)]
    try:
        srv.remove_plume(pid)                          # refused while requests are pending ...
        removed_early = True
    except lib.NslError:
        removed_early = False
    srv.drain()
    assert not removed_early or srv.stats()["completed"] == 4
    srv.remove_plume(pid) if not removed_early else None   # ... accepted once idle
    with pytest.raises(lib.NslError):
        srv.submit(pid, p["cams"][0], p["lights"][0])
    with pytest.raises(lib.NslError):
        srv.wait(rids[0] + 1000)
    srv.close()
