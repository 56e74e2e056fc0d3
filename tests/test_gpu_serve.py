"""Serving (Sec. 3.2: only the global model renders novel views): dg_render
against the FP64 oracle on mixed resolutions; a request's image is the same
rendered alone, inside a mixed-resolution batch, and through the
continuous-batching loop with several batches in flight; the loop's buffers
stay resident."""
import numpy as np
import pytest
import torch

from paper_2405_13943_b300 import synth as S
from tests._util import curate_gaussians, pixel_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_13943_b300 import build as B
    B.build()
    from paper_2405_13943_b300 import dogs, serve
    return dogs, serve


def test_render_matches_oracle_on_mixed_resolutions(mods, oracle):
    D, srv = mods
    O = oracle
    cams = [S.cube_camera(96, 72, f=90.0), S.cube_camera(64, 80, f=60.0)]
    g = curate_gaussians(O, S.cube_scene(3000, 1201, sh_degree=3, log_scale_mu=-2.6), cams, 16, 16)
    assert g.n > 2800
    z = D.GaussianBuffer.from_synth(g)
    bg = (0.1, 0.0, 0.2)
    rb = srv.render_views(z, cams, bg=bg)
    f = O.render(O.params_from(g), 3, O.ViewPlan(cams, [(0, g.n), (0, g.n)], 16, 16), bg)
    masks = pixel_mask(f["views"])
    for v in range(2):
        err = np.abs(rb.view_image(v).cpu().numpy() - f["views"][v]["image"]).max(0)
        assert err[masks[v]].max() <= 1e-4, (v, err[masks[v]].max())
        assert masks[v].mean() > 0.99


def test_alone_equals_in_mix(mods):
    D, srv = mods
    z = D.GaussianBuffer.from_synth(S.city_scene(200_000, 5))
    res = [(320, 240), (640, 360), (160, 120), (480, 272)]
    cams = S.random_pose_cameras(11, 6, res, [1, 1, 1, 1], size=1000.0)
    mix = srv.render_views(z, cams)
    for i, c in enumerate(cams):
        alone = srv.render_views(z, [c])
        a = alone.view_image(0)
        b = mix.view_image(i)
        assert float((a - b).abs().max()) <= 1e-4
        assert float(a.abs().sum()) > 0


def test_server_results_equal_alone_with_batches_in_flight(mods):
    """A burst of nine requests at t = 0, then arrivals at 3,000/s; batches of
    at most 3 requests on 3 slots: several batches are on the GPU at once,
    and every request's image (taken from the loop itself) equals the same
    view rendered alone."""
    D, srv = mods
    z = D.GaussianBuffer.from_synth(S.city_scene(150_000, 6))
    res = [(320, 240), (640, 480), (200, 360)]
    arr = np.concatenate([np.zeros(9), S.poisson_arrivals(3, 3000.0, 0.04)])
    cams = S.random_pose_cameras(4, len(arr), res, [0.5, 0.3, 0.2])
    server = srv.RenderServer(z, budget_bytes=3e9, max_batch=3, n_streams=3, resolutions=res,
                              max_batch_pixels=3 * 640 * 480)
    ipp = server.calibrate(S.random_pose_cameras(5, 4, res, [0.5, 0.3, 0.2]))
    assert ipp >= 2.0 and len(server.slots) == 3
    seen = []
    out = server.run(cams, arr, keep_images=True, on_result=lambda i, im: seen.append((i, tuple(im.shape))))
    assert out["max_inflight_batches"] >= 2, out["max_inflight_batches"]
    assert out["requests"] == len(arr) and sorted(i for i, _ in seen) == list(range(len(arr)))
    lat = out["latency_s"]
    assert np.all(np.isfinite(lat)) and np.all(lat > 0)
    for i, c in enumerate(cams):
        alone = srv.render_views(z, [c]).view_image(0).cpu()
        got = out["images"][i]
        assert tuple(got.shape) == (3, c.height, c.width) == seen[[j for j, _ in seen].index(i)][1]
        assert float((got - alone).abs().max()) <= 1e-4, i
        assert float(alone.abs().sum()) > 0


def test_server_buffers_stay_resident(mods):
    """Slots are carved from free HBM once; serving allocates no device memory."""
    D, srv = mods
    z = D.GaussianBuffer.from_synth(S.city_scene(100_000, 7))
    res = [(320, 240), (640, 480)]
    server = srv.RenderServer(z, budget_bytes=2e9, max_batch=4, n_streams=2, resolutions=res,
                              max_batch_pixels=4 * 640 * 480)
    server.calibrate(S.random_pose_cameras(8, 4, res, [0.5, 0.5]))
    free, _ = torch.cuda.mem_get_info()
    assert server.free_hbm_at_provision is not None and server.resident_bytes() <= 2e9
    ptrs = [(s.image.data_ptr(), s.ws.data_ptr(), s.dev_cams.data_ptr()) for s in server.slots]
    before = torch.cuda.memory_allocated()
    arr = S.poisson_arrivals(9, 500.0, 0.1)
    out = server.run(S.random_pose_cameras(10, len(arr), res, [0.5, 0.5]), arr)
    torch.cuda.synchronize()
    assert out["capacity_retries"] == 0
    assert [(s.image.data_ptr(), s.ws.data_ptr(), s.dev_cams.data_ptr()) for s in server.slots] == ptrs
    assert torch.cuda.memory_allocated() == before
