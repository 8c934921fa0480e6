"""Pins of the FP64 reference network of the learned pressure stage.

* forward convolution equals scipy.ndimage.correlate summed over input
  channels (a library routine, zero boundary);
* the data gradient is the adjoint of the forward map: <conv(x), y> = <x, dgrad(y)>;
* weight and bias gradients of the full 4-layer network equal central finite
  differences of its MSE loss.
"""
import numpy as np
import pytest


def rnd(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_forward_equals_library_correlation():
    from scipy.ndimage import correlate
    from oracle import conv3d
    x = rnd((5, 6, 7, 3), 0); W = rnd((27, 3, 2), 1); b = rnd(2, 2)
    y = conv3d.conv_fwd(x, W, b)
    for o in range(2):
        ref = np.full(x.shape[:3], b[o])
        for c in range(3):
            k = W[:, c, o].reshape(3, 3, 3)        # k[dz+1, dy+1, dx+1]
            ref += correlate(x[..., c], k, mode="constant", cval=0.0)
        assert np.allclose(y[..., o], ref, rtol=1e-12, atol=1e-12)


def test_dgrad_is_the_adjoint():
    from oracle import conv3d
    x = rnd((4, 5, 6, 3), 3); W = rnd((27, 3, 4), 4); yv = rnd((4, 5, 6, 4), 5)
    lhs = np.sum(conv3d.conv_fwd(x, W, np.zeros(4)) * yv)
    rhs = np.sum(x * conv3d.conv_dgrad(yv, W))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_network_gradients_finite_difference():
    from oracle import conv3d
    rng = np.random.default_rng(6)
    chans = [4, 5, 5, 5, 1]
    params = [(0.3 * rng.standard_normal((27, chans[k], chans[k + 1])), 0.1 * rng.standard_normal(chans[k + 1]))
              for k in range(4)]
    x = rng.standard_normal((3, 4, 5, 4)); target = rng.standard_normal((3, 4, 5, 1))
    loss, grads = conv3d.net_loss_and_grads(x, target, params)
    h = 1e-6
    for k in range(4):
        W, b = params[k]
        for idx in [(0, 0, 0), (13, 1, 0), (26, chans[k] - 1, chans[k + 1] - 1)]:
            Wp = W.copy(); Wp[idx] += h
            Wm = W.copy(); Wm[idx] -= h
            pp = list(params); pp[k] = (Wp, b)
            pm = list(params); pm[k] = (Wm, b)
            fd = (conv3d.net_loss_and_grads(x, target, pp)[0] - conv3d.net_loss_and_grads(x, target, pm)[0]) / (2 * h)
            assert grads[k][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        bp = b.copy(); bp[0] += h
        bm = b.copy(); bm[0] -= h
        pp = list(params); pp[k] = (W, bp)
        pm = list(params); pm[k] = (W, bm)
        fd = (conv3d.net_loss_and_grads(x, target, pp)[0] - conv3d.net_loss_and_grads(x, target, pm)[0]) / (2 * h)
        assert grads[k][1][0] == pytest.approx(fd, rel=1e-5, abs=1e-9)
