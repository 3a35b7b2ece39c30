"""The convolutional surrogate's kernels against the numpy reference
(tests/surrogate_ref.py), stage by stage: each device stage is recomputed
in FP64 from the device's own BF16 inputs of that stage, so a stage is
compared with its definition and rounding does not compound. A BF16 result
may differ by one unit in the last place where FP32 accumulation order puts
a value next to a rounding boundary; FP32 results (the output layer, the
parameter gradients summed with atomics) agree to 1e-5 of their scale.
Then: the prediction conserves every layer's mass, and training learns a
known linear map."""
import numpy as np
import pytest

from paper_2409_16659_gb300 import mlswlbm as B
from tests import surrogate_ref as R

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _case(batch=2, n=3, ny=12, nx=32, seed=1):
    rng = np.random.default_rng(seed)
    h = (rng.uniform(0.5, 1.0, (batch, n, 1, 1))
         + 0.03 * rng.standard_normal((batch, n, ny, nx))).astype(np.float32)
    return h, rng


def _bf16_close(got, want):
    """Equal up to one BF16 unit in the last place (relative 2^-7)."""
    tol = np.abs(want) * 2.0 ** -7 + 1e-30
    bad = np.abs(got - want) > tol
    assert bad.mean() < 1e-3, bad.mean()
    assert np.all(np.abs(got - want) <= 2 * tol + 1e-6 * np.abs(want).max())


def _surrogate(n, nx, ny, rng, batch=4):
    s = B.Surrogate(n, nx, ny, batch, seed=7)
    w = s.get_params()
    nb = sum(R.CH[1:])
    w[-nb:] = rng.normal(0.0, 0.1, nb).astype(np.float32)  # nonzero biases
    s.set_params(w)
    return s


def test_forward_stages_match_reference():
    h, rng = _case()
    bsz, n, ny, nx = h.shape
    with _surrogate(n, nx, ny, rng) as s:
        ht = torch.from_numpy(h).cuda()
        out = torch.empty_like(ht)
        s.predict(ht, out)
        torch.cuda.synchronize()
        npix = bsz * ny * nx
        ws, bs = R.split_params(s.get_params())
        wb = [R.bf16(w) for w in ws]
        x0 = R.from_bf16_bits(s.debug(2, (npix, 16), np.uint16)).reshape(bsz, ny, nx, 16)
        a1 = R.from_bf16_bits(s.debug(3, (npix, 32), np.uint16)).reshape(bsz, ny, nx, 32)
        a2 = R.from_bf16_bits(s.debug(4, (npix, 32), np.uint16)).reshape(bsz, ny, nx, 32)
        y = s.debug(0, (npix, 16), np.float32).reshape(bsz, ny, nx, 16)
        # input: (h - layer mean) * in_scale, zero channels above n
        mean = h.astype(np.float64).mean(axis=(2, 3))
        want = np.zeros((bsz, ny, nx, 16), np.float32)
        for b in range(bsz):
            for i in range(n):
                want[b, :, :, i] = (h[b, i] - np.float32(mean[b, i])) * np.float32(s.in_scale)
        _bf16_close(x0, R.bf16(want))
        # hidden layers from the device's own inputs
        _bf16_close(a1, R.bf16(np.maximum(R.conv(x0, wb[0]) + bs[0], 0).astype(np.float32)))
        _bf16_close(a2, R.bf16(np.maximum(R.conv(a1, wb[1]) + bs[1], 0).astype(np.float32)))
        yr = R.conv(a2, wb[2]) + bs[2]
        assert np.abs(y - yr).max() <= 1e-5 * np.abs(yr).max()
        # output: h + (y - layer mean of y) / out_scale, masses kept
        o = out.cpu().numpy()
        for b in range(bsz):
            for i in range(n):
                dy = y[b, :, :, i].astype(np.float64)
                want_o = h[b, i] + (dy - dy.mean()) / s.out_scale
                assert np.abs(o[b, i] - want_o).max() <= 1e-6
                assert abs(o[b, i].astype(np.float64).sum() - h[b, i].astype(np.float64).sum()) \
                    <= 1e-6 * np.abs(h[b, i]).sum()


def test_gradients_match_reference():
    h, rng = _case(seed=2)
    bsz, n, ny, nx = h.shape
    target = (h + 0.01 * rng.standard_normal(h.shape)).astype(np.float32)
    with _surrogate(n, nx, ny, rng) as s:
        ws, bs = R.split_params(s.get_params())
        wb = [R.bf16(w) for w in ws]
        ht, tt = torch.from_numpy(h).cuda(), torch.from_numpy(target).cuda()
        loss = s.train_step(ht, tt, 1e-12)
        npix = bsz * ny * nx
        rd = lambda k, c: R.from_bf16_bits(s.debug(k, (npix, c), np.uint16)).reshape(bsz, ny, nx, c)
        x0, a1, a2, dyv, da2, da1 = rd(2, 16), rd(3, 32), rd(4, 32), rd(5, 16), rd(6, 32), rd(7, 32)
        y = s.debug(0, (npix, 16), np.float32).reshape(bsz, ny, nx, 16)
        g = s.debug(1, (B.Surrogate.param_count(),), np.float32)
        gw, gb = R.split_params(g)
        # loss and its gradient
        t = np.moveaxis((target.astype(np.float64) - h) * s.out_scale, 1, 3)
        r = y[..., :n].astype(np.float64) - t
        cnt = npix * n
        assert loss == pytest.approx((r ** 2).sum() / cnt, rel=1e-5)
        want_dy = np.zeros_like(y)
        want_dy[..., :n] = (2 * r / cnt).astype(np.float32)
        _bf16_close(dyv, R.bf16(want_dy))
        # layer 2 parameters and the gradient of a2 (through its ReLU)
        for gw_l, want in ((gw[2], R.conv_weight_grad(a2, dyv)), (gb[2], dyv.sum(axis=(0, 1, 2)))):
            assert np.abs(gw_l - want).max() <= 1e-5 * np.abs(want).max()
        _bf16_close(da2, R.bf16((R.conv_input_grad(dyv, wb[2]) * (a2 > 0)).astype(np.float32)))
        # layer 1
        for gw_l, want in ((gw[1], R.conv_weight_grad(a1, da2)), (gb[1], da2.sum(axis=(0, 1, 2)))):
            assert np.abs(gw_l - want).max() <= 1e-5 * np.abs(want).max()
        _bf16_close(da1, R.bf16((R.conv_input_grad(da2, wb[1]) * (a1 > 0)).astype(np.float32)))
        # layer 0
        for gw_l, want in ((gw[0], R.conv_weight_grad(x0, da1)), (gb[0], da1.sum(axis=(0, 1, 2)))):
            assert np.abs(gw_l - want).max() <= 1e-5 * np.abs(want).max()


def test_training_learns_a_linear_smoothing():
    """Target: each layer relaxed by a few lattice-Laplacian steps, a change
    the network can represent; Adam brings the error well below its start."""
    rng = np.random.default_rng(4)
    bsz, n, ny, nx = 8, 2, 32, 32

    def batch():
        h = (0.8 + 0.05 * rng.standard_normal((bsz, n, ny, nx))).astype(np.float32)
        lap = (np.roll(h, 1, 2) + np.roll(h, -1, 2) + np.roll(h, 1, 3) + np.roll(h, -1, 3) - 4 * h)
        return h, (h + 0.02 * lap).astype(np.float32)

    with B.Surrogate(n, nx, ny, bsz, seed=5, in_scale=20.0, out_scale=50.0) as s:
        losses = []
        for it in range(300):
            h, t = batch()
            losses.append(s.train_step(torch.from_numpy(h).cuda(), torch.from_numpy(t).cuda(), 2e-3))
        assert np.mean(losses[-20:]) < 0.05 * np.mean(losses[:5])


def test_trained_on_dewetting_trajectories_it_beats_the_identity():
    """Trained for a short while on trajectories of the dewetting film, the
    surrogate predicts the held-out nonlinear windows (rupture and after)
    closer to the LBM than no change does, and its predictions keep every
    layer's mass."""
    import workloads
    from paper_2409_16659_gb300 import surrogate as S
    side, ninst, nwin = 64, 20, 130
    params = [workloads.dewet2_params(side) for _ in range(ninst)]
    heights = [workloads.dewet2_heights(side, seed=300 + j).astype(np.float32) for j in range(ninst)]
    traj = S.trajectories(params, heights, nwin)
    with B.Surrogate(2, side, side, 32, seed=3, in_scale=10.0, out_scale=40.0) as s:
        losses = S.train(s, traj, list(range(16)), 1500, 32, 2e-3, 2e-4, seed=4)
        assert losses[-50:].mean() < 0.2 * losses[:20].mean()
        err, ident, _ = S.window_errors(s, traj, list(range(16, 20)))
        late = slice(100, None)
        assert np.median(err[:, late]) < 0.6 * np.median(ident[:, late])
        h = traj[16:20, 110].contiguous()
        out = torch.empty_like(h)
        s.predict(h, out)
        m0 = h.double().sum(dim=(2, 3))
        m1 = out.double().sum(dim=(2, 3))
        assert float((m1 - m0).abs().max()) <= 1e-6 * float(m0.abs().max())
