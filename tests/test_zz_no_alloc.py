"""bd_bad_describe_noalloc, the entry point for callers that cannot call
cudaMalloc (device memory all reserved by another allocator, real-time loops
that cannot take cudaFree's synchronisation, plug-ins in hosts that forbid
allocation), against the regular bd_bad_describe through the C ABI: two
calls in a row must give the same descriptors bit for bit (the tolerance of
every BAD test), an image at the size limit must work, and an image beyond
the static area's limit must be refused with nothing launched.

Kept in a file of its own, collected last."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(hp, img, kps, out, stream):
    import paper_2108_08380_gb300 as bd
    h, w = img.shape
    return bd.lib().bd_bad_describe_noalloc(hp.handle, _p(img), w, h, img.stride(0), _p(kps),
                                            kps.shape[0], _p(out), ctypes.c_void_p(stream))


def test_noalloc_equals_bd_bad_describe_on_two_calls_in_a_row(gpu_ctx):
    import torch
    wl = synth.plain_workload(1000)
    hp = gpu_ctx.bad_params(wl.bad)
    imgs = [torch.from_numpy(wl.img_a).cuda(), torch.from_numpy(wl.img_b).cuda()]
    kps = torch.from_numpy(wl.kps_a).cuda()
    refs = [gpu_ctx.bad_describe(hp, im, kps) for im in imgs]
    outs = [torch.full_like(r, -1) for r in refs]
    stream = torch.cuda.current_stream().cuda_stream
    for im, o in zip(imgs, outs):
        assert _noalloc(hp, im, kps, o, stream) == 0
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)


def test_noalloc_at_the_size_limit_and_beyond(gpu_ctx):
    import torch
    import paper_2108_08380_gb300 as bd
    rng = np.random.default_rng(12)
    p = synth.make_bad_params(512, rng, level_scales=tuple(synth.pyramid_scales(5)))
    hp = gpu_ctx.bad_params(p)
    img = torch.from_numpy(synth.make_image(1920, 1080, rng)).cuda()
    kps = torch.from_numpy(synth.make_keypoints(3000, 1920, 1080, rng, border=0,
                                                scales=tuple(float(s) for s in p.level_scales),
                                                angle_bins=None)).cuda()
    ref = gpu_ctx.bad_describe(hp, img, kps)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.full_like(ref, -1)
        assert _noalloc(hp, img, kps, out, stream) == 0
        torch.cuda.synchronize()
        assert torch.equal(out, ref)

    big = torch.zeros((2160, 3840), dtype=torch.uint8, device="cuda")
    out = torch.full((kps.shape[0], 16), -7, dtype=torch.int32, device="cuda")
    st = _noalloc(hp, big, kps, out, stream)
    assert st == bd.BD_ERR_INVALID
    assert b"static area" in bd.lib().bd_last_error(gpu_ctx.handle)
    torch.cuda.synchronize()
    assert bool((out == -7).all())
