"""Semi-dense front end on the GPU (cvo_frontend_select / cvo_frontend_cloud),
called through the C ABI, against oracle/frontend.py. Pixel selection is index
work: the kept pixels, their order and the back-projected points and features
must be identical bit for bit."""
import numpy as np
import pytest

import oracle
import synth
from oracle import frontend

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cvo():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1904_02266_gb300 as m
    return m


def _gpu_select(cvo, ctx, depth, hsv, params, cap):
    torch = pytest.importorskip("torch")
    xyz = torch.zeros((cap, 3), dtype=torch.float32, device="cuda")
    feat = torch.zeros((cap, 5), dtype=torch.float32, device="cuda")
    pix = torch.zeros(cap, dtype=torch.int32, device="cuda")
    n = ctx.frontend_select(depth, hsv, params, xyz, feat, pix)
    torch.cuda.synchronize()
    return xyz[:n].cpu().numpy(), feat[:n].cpu().numpy(), pix[:n].cpu().numpy()


@pytest.mark.parametrize("size,max_points,q", [((320, 240), 0, 80.0), ((640, 480), 20000, 80.0),
                                               ((160, 120), 0, 0.0), ((160, 120), 500, 99.0)])
def test_selection_is_bit_exact(cvo, size, max_points, q):
    W, H = size
    im = synth.room_frame_images(seed=synth.seed_for(7, W), width=W, height=H)
    with cvo.Context(device=0) as ctx:
        fp = cvo.cvo_frontend_params_default(fx=im["fx"], fy=im["fy"], cx=im["cx"], cy=im["cy"],
                                             percentile=q, max_points=max_points)
        xyz, feat, pix = _gpu_select(cvo, ctx, im["depth"], im["hsv"], fp, W * H)
    rx, rf, ridx = frontend.select(im["depth"], im["hsv"], im["fx"], im["fy"], im["cx"], im["cy"],
                                   percentile=q, max_points=max_points)
    assert pix.size == ridx.size and pix.size > 0
    assert np.array_equal(pix.astype(np.int64), ridx)
    assert np.array_equal(xyz, rx)
    assert np.array_equal(feat, rf)


def test_device_images_and_the_resident_cloud(cvo):
    torch = pytest.importorskip("torch")
    im = synth.room_frame_images(seed=synth.seed_for(7, 1), width=320, height=240)
    with cvo.Context(device=0) as ctx:
        fp = cvo.cvo_frontend_params_default(fx=im["fx"], fy=im["fy"], cx=im["cx"], cy=im["cy"],
                                             max_points=5000)
        d = torch.from_numpy(im["depth"]).cuda()
        h = torch.from_numpy(im["hsv"]).cuda()
        handle, n = ctx.frontend_cloud(d, h, fp)
        rx, rf, _ = frontend.select(im["depth"], im["hsv"], im["fx"], im["fy"], im["cx"],
                                    im["cy"], max_points=5000)
        assert n == rx.shape[0]
        # the same points uploaded from the host make the same cloud: every
        # sum over it agrees bit for bit
        ref = ctx.set_cloud(rx, rf)
        P = synth.random_motion(np.random.default_rng(1), 2.0, 0.02)
        a = ctx.eval(handle, handle, P, 0.05)
        b = ctx.eval(ref, ref, P, 0.05)
        assert a["F"] == b["F"] and np.array_equal(a["grad6"], b["grad6"])


def test_front_end_errors(cvo):
    with cvo.Context(device=0) as ctx:
        torch = pytest.importorskip("torch")
        out = torch.zeros((16, 3), dtype=torch.float32, device="cuda")
        fp = cvo.cvo_frontend_params_default()
        depth = np.zeros((4, 4), np.float32)            # nothing in range
        hsv = np.zeros((4, 4, 3), np.float32)
        with pytest.raises(cvo.CvoError) as e:
            ctx.frontend_select(depth, hsv, fp, out)
        assert e.value.code == cvo.CVO_ERR_INVALID_ARG
        with pytest.raises(cvo.CvoError) as e:
            ctx.frontend_select(np.ones((1, 4), np.float32), np.zeros((1, 4, 3), np.float32), fp,
                                out)
        assert e.value.code == cvo.CVO_ERR_INVALID_ARG
        bad = cvo.cvo_frontend_params_default(percentile=101.0)
        with pytest.raises(cvo.CvoError) as e:
            ctx.frontend_select(np.ones((4, 4), np.float32), hsv, bad, out)
        assert e.value.code == cvo.CVO_ERR_INVALID_ARG
        # more kept points than the output holds
        im = synth.room_frame_images(seed=synth.seed_for(7, 2), width=64, height=48)
        fp2 = cvo.cvo_frontend_params_default(fx=im["fx"], fy=im["fy"], cx=im["cx"], cy=im["cy"],
                                              percentile=0.0)
        with pytest.raises(cvo.CvoError) as e:
            ctx.frontend_select(im["depth"], im["hsv"], fp2, out)
        assert e.value.code == cvo.CVO_ERR_INVALID_ARG
