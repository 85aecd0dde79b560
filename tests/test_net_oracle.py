"""Pins of the network oracle against definitions it does not share code with.

- bfloat16 rounding against torch's own float32 -> bfloat16 conversion;
- the 3x3x3 'same' correlation against scipy.ndimage.correlate and brute force;
- the backward pass against the adjoint identities and central differences;
- Adam against its closed form for a constant gradient.
"""
import numpy as np
import pytest

from oracle import net_oracle as NO


def _rng(s):
    return np.random.default_rng(s)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = _rng(1)
    a = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-8, 8, 20000)).astype(np.float32)
    # exact ties: float32 values whose lower 16 bits are 0x8000
    ties = (rng.integers(0, 2 ** 16, 1000, dtype=np.uint32) << 16 | np.uint32(0x8000)).view(np.float32)
    ties = ties[np.isfinite(ties)]
    for v in (a, ties, np.array([0.0, -0.0, 1.0, -1.0, 3.0e38], np.float32)):
        ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
        np.testing.assert_array_equal(NO.bf16_round(v), ref)


def test_conv3d_matches_scipy_correlate():
    from scipy import ndimage

    rng = _rng(2)
    x = rng.standard_normal((2, 6, 5, 7, 3))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    y = NO.conv3d(x, w, b)
    for o in range(3):
        for n in range(3):
            ref = b[o] + sum(ndimage.correlate(x[c, :, :, :, n], w[o, c], mode="constant", cval=0.0)
                             for c in range(2))
            np.testing.assert_allclose(y[o, :, :, :, n], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_brute_force():
    rng = _rng(3)
    x = rng.standard_normal((2, 3, 4, 3, 2))
    w = rng.standard_normal((2, 2, 3, 3, 3))
    y = NO.conv3d(x, w, None)
    _, d, h, wd, nb = x.shape
    for o in range(2):
        for z in range(d):
            for yy in range(h):
                for xx in range(wd):
                    for n in range(nb):
                        s = 0.0
                        for c in range(2):
                            for a in range(3):
                                for bb in range(3):
                                    for e in range(3):
                                        zi, yi, xi = z + a - 1, yy + bb - 1, xx + e - 1
                                        if 0 <= zi < d and 0 <= yi < h and 0 <= xi < wd:
                                            s += w[o, c, a, bb, e] * x[c, zi, yi, xi, n]
                        assert abs(y[o, z, yy, xx, n] - s) < 1e-12


def test_conv3d_backward_adjoint_identities():
    rng = _rng(4)
    x = rng.standard_normal((3, 5, 4, 6, 2))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    dy = rng.standard_normal((4, 5, 4, 6, 2))
    dx, dw, db = NO.conv3d_backward(x, w, dy)
    # <conv(x, w), dy> = <x, dx>: dx is the adjoint in x
    lhs = np.vdot(NO.conv3d(x, w, None), dy)
    assert abs(lhs - np.vdot(x, dx)) < 1e-9 * abs(lhs)
    # <conv(x, E), dy> = <E, dW> for any E: dW is the adjoint in w
    e = rng.standard_normal(w.shape)
    lhs = np.vdot(NO.conv3d(x, e, None), dy)
    assert abs(lhs - np.vdot(e, dw)) < 1e-9 * abs(lhs)
    np.testing.assert_allclose(db, dy.sum(axis=(1, 2, 3, 4)), rtol=1e-14)


def test_adjoint_pin_catches_a_flipped_kernel():
    """A plausible mistake (kernel not flipped in the input gradient) breaks the adjoint identity."""
    rng = _rng(5)
    x = rng.standard_normal((2, 4, 4, 4, 1))
    w = rng.standard_normal((2, 2, 3, 3, 3))
    dy = rng.standard_normal((2, 4, 4, 4, 1))
    wrong = NO.conv3d(dy, np.transpose(w, (1, 0, 2, 3, 4)), None)  # correlation instead of convolution
    lhs = np.vdot(NO.conv3d(x, w, None), dy)
    assert abs(lhs - np.vdot(x, wrong)) > 1e-3 * abs(lhs)
    right = NO.conv3d(dy, np.transpose(w, (1, 0, 2, 3, 4))[:, :, ::-1, ::-1, ::-1], None)
    assert abs(lhs - np.vdot(x, right)) < 1e-9 * abs(lhs)


def test_loss_gradients_match_central_differences():
    rng = _rng(6)
    params = NO.init_params(rng)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    u = rng.standard_normal((5, 4, 6, 2))
    t = rng.standard_normal((5, 4, 6, 2))
    loss, grads = NO.loss_and_grads(params, u, t, quantize=False)
    h = 1e-6
    for li in range(4):
        w, b = params[li]
        for _ in range(4):
            idx = tuple(int(rng.integers(0, s)) for s in w.shape)
            wp, wm = w.copy(), w.copy()
            wp[idx] += h
            wm[idx] -= h
            pp = list(params)
            pp[li] = (wp, b)
            lp = NO.loss_and_grads(pp, u, t, quantize=False)[0]
            pp[li] = (wm, b)
            lm = NO.loss_and_grads(pp, u, t, quantize=False)[0]
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[li][0][idx]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (li, idx)
        k = int(rng.integers(0, b.size))
        bp, bm = b.copy(), b.copy()
        bp[k] += h
        bm[k] -= h
        pp = list(params)
        pp[li] = (w, bp)
        lp = NO.loss_and_grads(pp, u, t, quantize=False)[0]
        pp[li] = (w, bm)
        lm = NO.loss_and_grads(pp, u, t, quantize=False)[0]
        assert abs((lp - lm) / (2 * h) - grads[li][1][k]) <= 1e-6 * max(1.0, abs(lp - lm) / (2 * h)) + 1e-9


def test_quantized_forward_close_to_exact():
    rng = _rng(7)
    params = NO.quantize_params(NO.init_params(rng))
    u = rng.standard_normal((6, 5, 4, 4))
    y_q, _ = NO.forward(params, u, quantize=True)
    y_e, _ = NO.forward(params, u, quantize=False)
    rel = np.linalg.norm(y_q - y_e) / np.linalg.norm(y_e)
    assert 0 < rel < 2e-2  # bfloat16 activations: ~2^-9 relative per rounding


def test_adam_closed_form_constant_gradient():
    rng = _rng(8)
    params = [(rng.standard_normal((2, 1, 3, 3, 3)), rng.standard_normal(2))]
    g = [(rng.standard_normal((2, 1, 3, 3, 3)), rng.standard_normal(2))]
    state = {}
    lr, eps = 1e-3, 1e-8
    p = params
    for k in range(1, 6):
        p = NO.adam_step(p, g, state, lr, eps=eps)
        # with a constant gradient, m_hat = g and v_hat = g^2 at every step
        for (p0, _), (pk, _), (gw, _) in [(params[0], p[0], g[0])]:
            np.testing.assert_allclose(pk, p0 - k * lr * gw / (np.abs(gw) + eps), rtol=1e-10, atol=1e-14)
        np.testing.assert_allclose(p[0][1], params[0][1] - k * lr * g[0][1] / (np.abs(g[0][1]) + eps),
                                   rtol=1e-10, atol=1e-14)


def test_pack_unpack_roundtrip():
    params = NO.init_params(_rng(9))
    flat = NO.pack_params(params)
    assert flat.size == NO.n_params() == (27 * 32 + 32) + 2 * (27 * 32 * 32 + 32) + (27 * 32 + 1)
    back = NO.unpack_params(flat)
    for (w, b), (w2, b2) in zip(params, back):
        np.testing.assert_array_equal(w, w2)
        np.testing.assert_array_equal(b, b2)
