"""GPU parity of the batched persistent description (many images of uneven
size and keypoint count in one launch, optionally replayed from a CUDA graph):
identical bits to the per-image calls, which are pinned to the oracle, plus
an oracle sample on the batch itself."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _small_batch(seed=5, bad_bits=256, hs_bits=256, levels=1):
    rng = np.random.default_rng(seed)
    sizes = [(640, 480), (1, 1), (33, 17), (300, 200), (129, 257), (800, 600)]
    counts = [700, 3, 0, 250, 77, 1300]
    scales = tuple(float(s) for s in synth.pyramid_scales(levels))
    imgs, kps = [], []
    for (w, h), c in zip(sizes, counts):
        imgs.append(synth.make_image(w, h, rng))
        k = synth.make_keypoints(c, w, h, rng, border=-10.0, scales=scales, angle_bins=None)
        kps.append(k)
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    bad = synth.make_bad_params(bad_bits, rng, level_scales=scales)
    hs = synth.make_hashsift_params(hs_bits, rng, bf16=True)
    return imgs, np.concatenate(kps), offs, bad, hs


def _per_image(ctx, bp, hp, imgs, kps, offs):
    bad, hs = [], []
    for i, im in enumerate(imgs):
        k = kps[offs[i]:offs[i + 1]]
        if len(k) == 0:
            continue
        bad.append(_u32(ctx.bad_describe(bp, _dev(im), _dev(k))))
        hs.append(_u32(ctx.hashsift_describe(hp, _dev(im), _dev(k))))
    return np.concatenate(bad), np.concatenate(hs)


@pytest.mark.parametrize("graph,cfg", [(False, None), (True, None), (True, (8, 4, 5, 4, 0, 0, 0)),
                                       (False, (4, 5, 4, 4, 1, 2, 0)), (True, (32, 6, 5, 1, 1, 1, 1))])
def test_batch_equals_per_image_calls(gpu_ctx, graph, cfg):
    """The batched launch gives the per-image calls' bits (which are pinned to
    the oracle) in the default shape and in shapes with every queue order of
    the HashSIFT items, both projection paths and every BAD sharing mode."""
    import torch
    imgs, kps, offs, bad, hs = _small_batch()
    bp, hp = gpu_ctx.bad_params(bad), gpu_ctx.hs_params(hs)
    ref_bad, ref_hs = _per_image(gpu_ctx, bp, hp, imgs, kps, offs)
    dimgs = [_dev(im) for im in imgs]
    b = gpu_ctx.batch(bp, hp, dimgs, offs)
    if cfg is not None:
        b.set_config(*cfg)
    n = len(kps)
    ob = torch.full((n, 8), -1, dtype=torch.int32, device="cuda")
    oh = torch.full((n, 8), -1, dtype=torch.int32, device="cuda")
    dk = _dev(kps)
    for _ in range(2):
        b.describe(dimgs, dk, ob, oh, graph=graph)
    assert gpu_ctx.sync_status() == 0
    assert np.array_equal(_u32(ob), ref_bad)
    assert np.array_equal(_u32(oh), ref_hs)
    # BAD against the oracle directly, all keypoints
    for i, im in enumerate(imgs):
        k = kps[offs[i]:offs[i + 1]]
        if len(k):
            assert np.array_equal(_u32(ob)[offs[i]:offs[i + 1]], oracle.bad_describe(im, k, bad)[0])


def test_graph_replay_sees_new_image_contents(gpu_ctx):
    import torch
    imgs, kps, offs, bad, hs = _small_batch(seed=6)
    bp, hp = gpu_ctx.bad_params(bad), gpu_ctx.hs_params(hs)
    dimgs = [_dev(im) for im in imgs]
    b = gpu_ctx.batch(bp, hp, dimgs, offs)
    n = len(kps)
    ob = torch.empty((n, 8), dtype=torch.int32, device="cuda")
    oh = torch.empty((n, 8), dtype=torch.int32, device="cuda")
    dk = _dev(kps)
    b.describe(dimgs, dk, ob, oh, graph=True)
    rng = np.random.default_rng(99)
    new = [synth.make_image(im.shape[1], im.shape[0], rng) for im in imgs]
    for d, im in zip(dimgs, new):
        d.copy_(torch.from_numpy(im))
    b.describe(dimgs, dk, ob, oh, graph=True)
    ref_bad, ref_hs = _per_image(gpu_ctx, bp, hp, new, kps, offs)
    assert np.array_equal(_u32(ob), ref_bad)
    assert np.array_equal(_u32(oh), ref_hs)


def test_autotune_keeps_results(gpu_ctx):
    import torch
    imgs, kps, offs, bad, hs = _small_batch(seed=7, bad_bits=512, hs_bits=512, levels=5)
    bp, hp = gpu_ctx.bad_params(bad), gpu_ctx.hs_params(hs)
    dimgs = [_dev(im) for im in imgs]
    b = gpu_ctx.batch(bp, hp, dimgs, offs)
    n = len(kps)
    ob = torch.empty((n, 16), dtype=torch.int32, device="cuda")
    oh = torch.empty((n, 16), dtype=torch.int32, device="cuda")
    dk = _dev(kps)
    best, ms = b.autotune(dimgs, dk, ob, oh, reps=2)
    assert ms > 0 and best == b.config()
    ob.fill_(-1)
    oh.fill_(-1)
    b.describe(dimgs, dk, ob, oh, graph=True)
    ref_bad, ref_hs = _per_image(gpu_ctx, bp, hp, imgs, kps, offs)
    assert np.array_equal(_u32(ob), ref_bad)
    assert np.array_equal(_u32(oh), ref_hs)


def test_batch_bad_only_hs_only_and_invalid(gpu_ctx):
    import torch
    import paper_2108_08380_gb300 as bd
    imgs, kps, offs, bad, hs = _small_batch(seed=8)
    kps[5, 0] = np.nan
    kps[900, 2] = -3.0
    bp, hp = gpu_ctx.bad_params(bad), gpu_ctx.hs_params(hs, precision=bd.BD_HS_FP32)
    dimgs = [_dev(im) for im in imgs]
    n = len(kps)
    dk = _dev(kps)
    b1 = gpu_ctx.batch(bp, None, dimgs, offs)
    ob = torch.full((n, 8), -1, dtype=torch.int32, device="cuda")
    b1.describe(dimgs, dk, ob, None)
    b2 = gpu_ctx.batch(None, hp, dimgs, offs)
    oh = torch.full((n, 8), -1, dtype=torch.int32, device="cuda")
    b2.describe(dimgs, dk, None, oh)
    assert gpu_ctx.sync_status() & bd.BD_FLAG_INVALID_KEYPOINT
    ref_bad, ref_hs = _per_image(gpu_ctx, bp, hp, imgs, kps, offs)
    gpu_ctx.sync_status()
    assert np.array_equal(_u32(ob), ref_bad)
    assert np.array_equal(_u32(oh), ref_hs)
    assert np.all(_u32(ob)[[5, 900]] == 0) and np.all(_u32(oh)[[5, 900]] == 0)


def test_batched_workload_full_size_sampled(gpu_ctx):
    """The batched workload (64 images 480x360..1920x1080, 200k keypoints on a
    5-level pyramid, BAD-512 + HashSIFT-512 with BF16 W) in the benchmark's
    launch configuration: every descriptor equals the per-image calls; a
    seeded sample of keypoints checked against the oracle."""
    import torch
    wl = synth.batch_workload(1002)
    bp, hp = gpu_ctx.bad_params(wl.bad), gpu_ctx.hs_params(wl.hs, band=1e-3)
    dimgs = [_dev(im) for im in wl.images]
    b = gpu_ctx.batch(bp, hp, dimgs, wl.kp_offsets)
    n = len(wl.kps)
    dk = _dev(wl.kps)
    ob = torch.empty((n, 16), dtype=torch.int32, device="cuda")
    oh = torch.empty((n, 16), dtype=torch.int32, device="cuda")
    b.describe(dimgs, dk, ob, oh, graph=True)
    assert gpu_ctx.sync_status() == 0
    ref_bad, ref_hs = _per_image(gpu_ctx, bp, hp, wl.images, wl.kps, wl.kp_offsets)
    assert np.array_equal(_u32(ob), ref_bad)
    assert np.array_equal(_u32(oh), ref_hs)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(wl.images), size=6, replace=False):
        lo, hi = wl.kp_offsets[i], wl.kp_offsets[i + 1]
        sel = np.sort(rng.choice(np.arange(lo, hi), size=min(40, hi - lo), replace=False))
        rb, _ = oracle.bad_describe(wl.images[i], wl.kps[sel], wl.bad)
        assert np.array_equal(_u32(ob)[sel], rb)
        ro = oracle.hs_describe(wl.images[i], wl.kps[sel], wl.hs)
        got = np.unpackbits(_u32(oh)[sel].view(np.uint8), axis=1, bitorder="little").astype(bool)
        sure = np.abs(ro["margins"]) > 2e-3
        assert np.array_equal(got[sure], (ro["margins"] > 0)[sure])


@pytest.mark.parametrize("hs_mode", [1, 4])
def test_fused_fp32_projection_equals_tensor_core_path(gpu_ctx, hs_mode):
    """The persistent kernel's own FP32 projection tiles give the bits of the
    tcgen05 BF16 + rescue kernel on the same histograms (both equal the FP32
    path), for FP32 W and for W exactly in BF16, with and without BAD."""
    import torch
    for bf16 in (False, True):
        imgs, kps, offs, bad, hs = _small_batch(seed=9 + bf16)
        if not bf16:
            rng = np.random.default_rng(3)
            hs = synth.make_hashsift_params(256, rng)
        bp, hp = gpu_ctx.bad_params(bad), gpu_ctx.hs_params(hs)
        dimgs = [_dev(im) for im in imgs]
        n = len(kps)
        dk = _dev(kps)
        for with_bad in (True, False):
            b = gpu_ctx.batch(bp if with_bad else None, hp, dimgs, offs)
            ob = torch.zeros((n, 8), dtype=torch.int32, device="cuda") if with_bad else None
            res = []
            for fused, half in ((0, 0), (1, 0), (1, 1)):
                oh = torch.full((n, 8), -1, dtype=torch.int32, device="cuda")
                b.set_config(8, 4, 2, hs_mode, fused, 0, half)
                b.describe(dimgs, dk, ob, oh, graph=bool(fused))
                res.append(_u32(oh))
            assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])
            assert gpu_ctx.sync_status() == 0
            b.close()


@pytest.mark.parametrize("cfg", [(8, 4, 0, 4, 0, 0, 0), (4, 2, 1, 1, 1, 0, 1), (32, 6, 2, 4, 1, 1, 0),
                                 (8, 4, 3, 4, 1, 1, 1), (4, 3, 3, 1, 0, 0, 0), (8, 5, 4, 4, 1, 2, 0),
                                 (4, 5, 5, 4, 1, 0, 0), (32, 5, 5, 1, 0, 2, 0)])
def test_timeline_respects_dependencies(gpu_ctx, cfg):
    """The item timeline lists every queued item once, and no item starts
    before what it depends on: an integral tile after the tiles to its left
    and above were claimed (they publish their aggregates before they
    wait), BAD items after all tiles of their image ended, projection tiles
    after the HashSIFT items of their 32 keypoints were claimed.  Recording
    it does not change the descriptors."""
    import math
    import torch
    from paper_2108_08380_gb300 import BD_ITEM_BAD, BD_ITEM_HASHSIFT, BD_ITEM_II_TILE, BD_ITEM_PROJ
    imgs, kps, offs, bad, hs = _small_batch(seed=21)
    bp, hp = gpu_ctx.bad_params(bad), gpu_ctx.hs_params(hs)
    dimgs = [_dev(im) for im in imgs]
    b = gpu_ctx.batch(bp, hp, dimgs, offs)
    n = len(kps)
    dk = _dev(kps)
    it, _, _, hm, fused, _, half = cfg
    b.set_config(*cfg)
    ob0 = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
    oh0 = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
    b.describe(dimgs, dk, ob0, oh0, graph=True)
    b.set_timeline(True)
    ob = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
    oh = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
    b.describe(dimgs, dk, ob, oh, graph=True)
    ev = b.timeline()
    assert gpu_ctx.sync_status() == 0
    assert np.array_equal(_u32(ob), _u32(ob0)) and np.array_equal(_u32(oh), _u32(oh0))

    ntx = [math.ceil(im.shape[1] / 128) for im in imgs]
    nty = [math.ceil(im.shape[0] / 32) for im in imgs]
    tiles = [a * b for a, b in zip(ntx, nty)]
    tile_img = np.repeat(np.arange(len(imgs)), tiles)
    counts = np.diff(offs)
    bad_items = [math.ceil(c / it) for c in counts]
    bad_img = np.repeat(np.arange(len(imgs)), bad_items)
    n_hs = math.ceil(n / hm)
    ptiles = 16 if half else 8  # projection tiles per 32 keypoints at 256 bits
    n_proj = math.ceil(n / 32) * ptiles if fused else 0
    expect = {BD_ITEM_II_TILE: sum(tiles), BD_ITEM_BAD: sum(bad_items),
              BD_ITEM_HASHSIFT: n_hs, BD_ITEM_PROJ: n_proj}
    assert len(ev) == sum(expect.values())
    by = {}
    for kind, cnt in expect.items():
        e = ev[ev["kind"] == kind]
        e = e[np.argsort(e["index"])]
        assert np.array_equal(e["index"], np.arange(cnt)), kind
        by[kind] = e
    assert np.all(ev["t_claim"] <= ev["t_ready"]) and np.all(ev["t_ready"] <= ev["t_end"])
    assert np.all(ev["cta"] >= 0) and np.all(ev["sm"] >= 0)
    tl, bd = by[BD_ITEM_II_TILE], by[BD_ITEM_BAD]
    first = np.concatenate([[0], np.cumsum(tiles)])
    for i in range(len(imgs)):
        mine = tl[first[i]:first[i + 1]]
        claim = mine["t_claim"].reshape(nty[i], ntx[i])
        ready = mine["t_ready"].reshape(nty[i], ntx[i])
        for ty in range(nty[i]):
            for tx in range(ntx[i]):
                need = [claim[ty, :tx].max(initial=0), claim[:ty].max(initial=0)]
                assert ready[ty, tx] >= max(need)
        if bad_items[i]:
            assert np.all(bd["t_ready"][bad_img == i] >= mine["t_end"].max())
    if fused:
        hsi, pr = by[BD_ITEM_HASHSIFT], by[BD_ITEM_PROJ]
        for g in range(math.ceil(n / 32)):
            first, last = (32 * g) // hm, (min(n, 32 * g + 32) - 1) // hm
            claimed = hsi["t_claim"][first:last + 1].max()
            assert np.all(pr["t_ready"][g * ptiles:(g + 1) * ptiles] >= claimed)
    b.set_timeline(False)
    b.close()


@pytest.mark.parametrize("fused,graph", [(1, True), (1, False), (0, True), (2, True)])
def test_batch_matchings_equal_bd_match(gpu_ctx, fused, graph):
    """Matchings set on the plan give the records bd_match gives on the same
    descriptors: inside the persistent launch (proj_fused = 1) or as the
    matching launch after the projection (proj_fused = 0).  Jobs cover both
    descriptors, both directions, an image pair of very different sizes, a
    query image and a train image without keypoints."""
    import torch
    from paper_2108_08380_gb300 import BD_DESC_BAD, BD_DESC_HASHSIFT
    imgs, kps, offs, bad, hs = _small_batch(seed=31)
    bp, hp = gpu_ctx.bad_params(bad), gpu_ctx.hs_params(hs)
    dimgs = [_dev(im) for im in imgs]
    b = gpu_ctx.batch(bp, hp, dimgs, offs)
    n = len(kps)
    dk = _dev(kps)
    cnt = np.diff(offs)
    spec = [(BD_DESC_BAD, 0, 5, 4, 5), (BD_DESC_HASHSIFT, 0, 5, 4, 5), (BD_DESC_BAD, 5, 0, 7, 10),
            (BD_DESC_HASHSIFT, 3, 4, 1, 1), (BD_DESC_BAD, 2, 0, 4, 5), (BD_DESC_HASHSIFT, 1, 2, 4, 5),
            (BD_DESC_BAD, 4, 4, 4, 5), (BD_DESC_HASHSIFT, 5, 3, 9, 10)]
    outs = [torch.full((max(int(cnt[q]), 1), 3), -7, dtype=torch.int32, device="cuda")
            if cnt[q] else None for (_, q, _, _, _) in spec]
    b.set_config(8, 4, 2, 4, 1 if fused else 0, 0, 1 if fused == 2 else 0)
    b.set_matches([(d, q, t, o, rn, rd) for (d, q, t, rn, rd), o in zip(spec, outs)])
    ob = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
    oh = torch.zeros((n, 8), dtype=torch.int32, device="cuda")
    for _ in range(2):  # the second call reuses the reset counters
        b.describe(dimgs, dk, ob, oh, graph=graph)
    assert gpu_ctx.sync_status() == 0
    for (d, q, t, rn, rd), o in zip(spec, outs):
        if o is None:
            continue
        desc = ob if d == BD_DESC_BAD else oh
        qd = desc[offs[q]:offs[q + 1]].contiguous()
        td = desc[offs[t]:offs[t + 1]].contiguous()
        ref = gpu_ctx.match(qd, td, 256, rn, rd)
        assert np.array_equal(o.cpu().numpy(), ref.cpu().numpy()), (d, q, t)
    # one job straight against the oracle
    d0 = _u32(ob)
    import paper_2108_08380_gb300 as bdm
    got = bdm.unpack_matches(outs[0])
    exp = oracle.match(d0[offs[0]:offs[1]], d0[offs[5]:offs[6]], 256)
    for g, r in zip(got, exp):
        assert np.array_equal(g, r)
    b.set_matches([])
    b.close()


def test_batch_matchings_rejected_without_descriptors(gpu_ctx):
    import torch
    from paper_2108_08380_gb300 import BD_DESC_BAD, BD_DESC_HASHSIFT, BindescError
    imgs, kps, offs, bad, hs = _small_batch(seed=32)
    bp = gpu_ctx.bad_params(bad)
    dimgs = [_dev(im) for im in imgs]
    b = gpu_ctx.batch(bp, None, dimgs, offs)
    o = torch.zeros((int(offs[1]), 3), dtype=torch.int32, device="cuda")
    with pytest.raises(BindescError):  # no HashSIFT parameters in the plan
        b.set_matches([(BD_DESC_HASHSIFT, 0, 5, o, 4, 5)])
    with pytest.raises(BindescError):  # image out of range
        b.set_matches([(BD_DESC_BAD, 0, 6, o, 4, 5)])
    with pytest.raises(BindescError):  # ratio above 1
        b.set_matches([(BD_DESC_BAD, 0, 5, o, 5, 4)])
    b.set_matches([(BD_DESC_BAD, 0, 5, o, 4, 5)])
    with pytest.raises(BindescError):  # the BAD output the job reads is missing
        b.describe(dimgs, _dev(kps), None, None)
    b.close()


@pytest.mark.parametrize("bits,levels", [(256, 1), (512, 5)])
def test_bad_shared_keypoints_equal_per_image_calls(gpu_ctx, bits, levels):
    """bad_shared = 0 (one keypoint per warp), 1 (the CTA's four warps split
    each keypoint's boxes and words) and 2 (warp pairs, two keypoints at a
    time) give the per-image BAD bits, invalid keypoints included (all-zero
    words)."""
    import torch
    imgs, kps, offs, bad, hs = _small_batch(seed=41, bad_bits=bits, hs_bits=256, levels=levels)
    kps[3, 1] = np.inf
    kps[1200, 3] = 1e30
    bp, hp = gpu_ctx.bad_params(bad), gpu_ctx.hs_params(hs)
    dimgs = [_dev(im) for im in imgs]
    b = gpu_ctx.batch(bp, None, dimgs, offs)
    n = len(kps)
    dk = _dev(kps)
    ref, _ = _per_image(gpu_ctx, bp, hp, imgs, kps, offs)
    gpu_ctx.sync_status()
    for it in (4, 8, 32):
        for shared in (0, 1, 2):
            ob = torch.full((n, bits // 32), -1, dtype=torch.int32, device="cuda")
            b.set_config(it, 4, 0, 4, 0, shared)
            b.describe(dimgs, dk, ob, None, graph=True)
            gpu_ctx.sync_status()
            assert np.array_equal(_u32(ob), ref), (it, shared)
    assert np.all(_u32(ob)[[3, 1200]] == 0)
    b.close()


@pytest.mark.parametrize("graph", [False, True])
def test_wait_limit_runs_out_then_next_call_is_exact(gpu_ctx, graph):
    """The persistent kernel's bounded dependency waits (error model: a wait
    that runs out raises BD_FLAG_TIMEOUT and bd_sync_status returns
    BD_ERR_TIMEOUT).  A 1 ns limit makes every wait that has to wait run out:
    the launch still returns, the flag is raised, and the next call with the
    default limit, on the same plan, gives the records of a clean call bit
    for bit, so the queue, readiness and matching arrival counters were
    reset by the launch that timed out."""
    import ctypes
    import torch
    import paper_2108_08380_gb300 as bdm
    from paper_2108_08380_gb300 import BD_DESC_BAD, BD_DESC_HASHSIFT
    imgs, kps, offs, bad, hs = _small_batch(seed=41)
    bp, hp = gpu_ctx.bad_params(bad), gpu_ctx.hs_params(hs)
    dimgs = [_dev(im) for im in imgs]
    b = gpu_ctx.batch(bp, hp, dimgs, offs)
    n = len(kps)
    dk = _dev(kps)
    cnt = np.diff(offs)
    # HashSIFT items last: each image's pass-2 tiles are queued right after
    # its pass-1 tiles, so they find them still running and have to wait
    b.set_config(8, 4, 0, 4, 1, 0, 0)
    spec = [(BD_DESC_BAD, 0, 5), (BD_DESC_HASHSIFT, 0, 5), (BD_DESC_BAD, 5, 0), (BD_DESC_HASHSIFT, 3, 4)]
    outs = [torch.empty((int(cnt[q]), 3), dtype=torch.int32, device="cuda") for (_, q, _) in spec]
    b.set_matches([(d, q, t, o, 4, 5) for (d, q, t), o in zip(spec, outs)])
    ob = torch.empty((n, 8), dtype=torch.int32, device="cuda")
    oh = torch.empty((n, 8), dtype=torch.int32, device="cuda")
    b.describe(dimgs, dk, ob, oh, graph=graph)
    assert gpu_ctx.sync_status() == 0
    ref = [t.clone() for t in [ob, oh] + outs]

    b.set_wait_limit(1)
    timed_out = False
    for _ in range(3):
        b.describe(dimgs, dk, ob, oh, graph=graph)
        f = ctypes.c_uint32(0)
        st = bdm.lib().bd_sync_status(gpu_ctx.handle, ctypes.byref(f))
        assert st in (bdm.BD_OK, bdm.BD_ERR_TIMEOUT)
        if st == bdm.BD_ERR_TIMEOUT:
            assert f.value & bdm.BD_FLAG_TIMEOUT
            timed_out = True
            break
    assert timed_out

    b.set_wait_limit(0)
    for t in [ob, oh] + outs:
        t.fill_(-3)
    for _ in range(2):
        b.describe(dimgs, dk, ob, oh, graph=graph)
        assert gpu_ctx.sync_status() == 0
        for got, exp in zip([ob, oh] + outs, ref):
            assert torch.equal(got, exp)
    b.set_matches([])
    b.close()


@pytest.mark.parametrize("band", [1e-3, 0.05, 1e9])
def test_projection_recheck_handoff_equals_in_place(gpu_ctx, band):
    """With the batch kernel's pre-split operand image and 16384 keypoints or
    more, the tcgen05 projection hands each block's band bits to otherwise
    idle warps for the FP32 re-check; the bits and the number of re-checked bits equal the
    per-image calls, whose epilogue re-checks its own bits.  At band 1e9
    every bit of a non-zero row is in the band, far past the hand-off's room,
    so most of them take the epilogue's own re-check.  Two launches in a row
    check that the hand-off's counters start from zero again."""
    import torch
    rng = np.random.default_rng(77)
    sizes, counts = [(1280, 720), (800, 600), (640, 480)], [9000, 5000, 3000]
    imgs = [synth.make_image(w, h, rng) for (w, h) in sizes]
    kps = np.concatenate([synth.make_keypoints(c, w, h, rng, border=-10.0, scales=(1.0,), angle_bins=None)
                          for (w, h), c in zip(sizes, counts)])
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    hs = synth.make_hashsift_params(256, rng, bf16=True)
    hp = gpu_ctx.hs_params(hs, band=band)
    dimgs = [_dev(im) for im in imgs]
    n = len(kps)
    dk = _dev(kps)
    ref, ref_cnt = [], 0
    gpu_ctx.rescued_count(reset=True)
    for i, im in enumerate(imgs):
        ref.append(_u32(gpu_ctx.hashsift_describe(hp, dimgs[i], _dev(kps[offs[i]:offs[i + 1]]))))
    ref = np.concatenate(ref)
    ref_cnt = gpu_ctx.rescued_count(reset=True)
    b = gpu_ctx.batch(None, hp, dimgs, offs)
    b.set_config(8, 4, 2, 4, 0, 0, 0)
    for graph in (False, True):
        oh = torch.full((n, 8), -1, dtype=torch.int32, device="cuda")
        b.describe(dimgs, dk, None, oh, graph=graph)
        assert gpu_ctx.sync_status() == 0
        assert np.array_equal(_u32(oh), ref)
        assert gpu_ctx.rescued_count(reset=True) == ref_cnt
    assert ref_cnt > 0
    b.close()
