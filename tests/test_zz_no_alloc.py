"""tm_gen_secondary_noalloc: secondary rays without any device allocation.

It serves callers that cannot allocate device memory while they run (a
renderer with a fixed memory budget, code inside a stream capture).  Its scan
scratch is a static device array of the library, so two calls in a row share
it; each call must give exactly what the allocating tm_gen_secondary gives
for the same hits.  This file is collected last so that a failure here
leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TM_ERR_TOO_LARGE = 9
TM_NOALLOC_MAX_HITS = 1 << 24


def noalloc_fn(N):
    fn = N.lib.tm_gen_secondary_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int, ctypes.c_float, ctypes.c_uint64, P, P, P, P]
    fn.restype = ctypes.c_int
    return fn


def test_noalloc_matches_allocating_entry_point():
    from paper_2103_02309_gb300 import build
    build.build()
    from paper_2103_02309_gb300 import _native as N
    from paper_2103_02309_gb300 import tetmesh as tmx
    import scenegen as sg

    fn = noalloc_fn(N)
    s = sg.make_config("tiny")
    mesh = tmx.Mesh(s.points, s.tets, s.tris)
    start = mesh.locate(torch.tensor([s.camera.eye], dtype=torch.float32, device="cuda"))
    stream = torch.cuda.current_stream()
    # two different inputs, the second one smaller, on two calls in a row
    cases = [((0.5, 0.5, 0.05), 64, 64, 1, float("inf"), 11), ((0.5, 0.45, 0.06), 40, 25, 8, 0.05, 12)]
    for eye, w, h, per_hit, tmax, seed in cases:
        st = mesh.locate(torch.tensor([eye], dtype=torch.float32, device="cuda"))
        rays = tmx.gen_primary(tmx.make_camera(eye, 60.0, w, h), st)
        hits = mesh.trace(rays)
        n = hits.shape[0]
        ref_rays, ref_count, ref_src = mesh.gen_secondary(hits, per_hit, tmax, seed, src=True)
        out = torch.full((n * per_hit, 8), -3.0, dtype=torch.float32, device="cuda")
        count = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        src = torch.full((n * per_hit,), -1, dtype=torch.int32, device="cuda")
        status = fn(mesh.handle, ctypes.c_void_p(hits.data_ptr()), n, None, per_hit, tmax, seed,
                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(count.data_ptr()),
                    ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert status == 0, N.lib.tm_last_error().decode()
        torch.cuda.synchronize()
        k = int(ref_count.item())
        assert k > 0 and int(count.item()) == k
        a = out[:k].cpu().numpy().view(np.int32)
        b = ref_rays[:k].cpu().numpy().view(np.int32)
        assert np.array_equal(a, b)
        assert np.array_equal(src[:k].cpu().numpy(), ref_src[:k].cpu().numpy())
        assert (out[k:].cpu().numpy() == -3.0).all()
    del start

    # a request beyond the static capacity is refused before any work is launched
    big = TM_NOALLOC_MAX_HITS + 1
    dummy = torch.empty((1, 8), dtype=torch.int32, device="cuda")
    count = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    status = fn(mesh.handle, ctypes.c_void_p(dummy.data_ptr()), big, None, 1, float("inf"), 0,
                ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(count.data_ptr()), None,
                ctypes.c_void_p(stream.cuda_stream))
    assert status == TM_ERR_TOO_LARGE
    assert "capacity" in N.lib.tm_last_error().decode()
    torch.cuda.synchronize()
    assert int(count.item()) == -1          # untouched: nothing was launched or written
