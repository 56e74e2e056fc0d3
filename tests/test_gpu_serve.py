"""Serving: a request's image is the same rendered alone and inside a
mixed-resolution batch, and the continuous-batching loop completes every
request with finite latency."""
import numpy as np
import pytest
import torch

from paper_2405_13943_b300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_13943_b300 import build as B
    B.build()
    from paper_2405_13943_b300 import dogs, serve
    return dogs, serve


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


def test_server_completes_requests(mods):
    D, srv = mods
    z = D.GaussianBuffer.from_synth(S.city_scene(100_000, 6))
    arr = S.poisson_arrivals(3, 100.0, 1.0)
    cams = S.random_pose_cameras(4, len(arr), [(320, 240), (640, 480)], [0.5, 0.5])
    server = srv.RenderServer(z, budget_bytes=2e9, max_batch=4, n_streams=3)
    sample = S.random_pose_cameras(5, 4, [(320, 240), (640, 480)], [0.5, 0.5])
    ipp = server.calibrate(sample)
    assert ipp >= 2.0
    out = server.run(cams, arr)
    lat = out["latency_s"]
    assert np.all(np.isfinite(lat)) and np.all(lat > 0)
    assert out["requests"] == len(arr)
