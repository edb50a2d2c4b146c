"""Pins for the learned-correction oracle: a forward special case that reduces
to the pinned product, and every gradient against central finite differences."""
import numpy as np
import pytest

import oracle
from oracle import learned
from workloads import arrays


def _params(rng, bins, b, rank, ch, scale=0.3):
    shapes = learned.param_shapes(bins, b, rank, ch)
    p = {}
    for k, s in shapes.items():
        v = rng.standard_normal(s) * scale
        if k in ("A", "B"):
            v = v + 1j * rng.standard_normal(s) * scale
        p[k] = v
    return p


def test_forward_reduces_to_the_product():
    """B_k = spectrum block, A_k = I, convolutions off: f(r) = Z r (Eq. multL)."""
    nx, ny, b = 3, 2, 3
    mx, my = 5, 4
    gen = arrays.random_generator_blocks(nx, ny, b, seed=60)
    spec = oracle.spectrum(gen, mx, my)                       # (my, mx, b, b)
    bins = mx * my
    p = _params(np.random.default_rng(61), bins, b, b, 4)
    p["B"] = spec.reshape(bins, b, b)
    p["A"] = np.broadcast_to(np.eye(b), (bins, b, b)).astype(np.complex128).copy()
    for k in ("W1", "c1", "W2", "c2", "W3", "c3"):
        p[k] = np.zeros_like(p[k])
    rng = np.random.default_rng(62)
    r = rng.standard_normal((2, nx * ny * b)) + 1j * rng.standard_normal((2, nx * ny * b))
    np.testing.assert_allclose(learned.forward(gen, p, r, mx, my), oracle.matvec(gen, r.T).T, rtol=1e-12,
                               atol=1e-12)


@pytest.mark.parametrize("name", ["B", "A", "W1", "c1", "W2", "c2", "W3", "c3"])
def test_gradients_match_finite_differences(name):
    nx, ny, b = 3, 2, 3
    mx, my = 5, 3
    rank, ch = 2, 4
    gen = arrays.generator_blocks(nx, ny, b, seed=63)
    rng = np.random.default_rng(64)
    p = _params(rng, mx * my, b, rank, ch)
    n = 2
    r = rng.standard_normal((n, nx * ny * b)) + 1j * rng.standard_normal((n, nx * ny * b))
    e = rng.standard_normal((n, nx * ny * b)) + 1j * rng.standard_normal((n, nx * ny * b))
    _, grads = learned.loss_and_grads(gen, p, r, e, mx, my)
    flat = p[name].reshape(-1)
    gflat = grads[name].reshape(-1)
    idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
    h = 1e-6
    for i in idx:
        parts = [1.0, 1j] if np.iscomplexobj(flat) else [1.0]
        for unit in parts:
            q = {k: v.copy() for k, v in p.items()}
            q[name].reshape(-1)[i] += h * unit
            lp = learned.loss_only(gen, q, r, e, mx, my)
            q[name].reshape(-1)[i] -= 2 * h * unit
            lm = learned.loss_only(gen, q, r, e, mx, my)
            fd = (lp - lm) / (2 * h)
            an = gflat[i].real if unit == 1.0 else gflat[i].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, i, unit, fd, an)


def _conv_case(seed, n=2, H=3, W=5, ci=2, co=3):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, H, W, ci))
    w = rng.standard_normal((co, ci, 3, 3))                  # no symmetry: a flipped tap would show
    c = rng.standard_normal(co)
    return x, w, c


def test_conv3_delta_response_places_each_tap():
    """A unit impulse at (y0, x0) in channel i: the output at (y0 + 1 - dy, x0 + 1 - dx) (mod the grid) is
    c + w[:, i, dy, dx], the closed form of the circular correlation
    out[y, x] = c + sum w[dy, dx] in[(y + dy - 1) mod H, (x + dx - 1) mod W] on a non-square grid."""
    H, W = 4, 5
    _, w, c = _conv_case(70, H=H, W=W)
    for i in range(w.shape[1]):
        for y0, x0 in [(0, 0), (2, 3), (3, 4)]:
            x = np.zeros((1, H, W, w.shape[1]))
            x[0, y0, x0, i] = 1.0
            out = learned.conv3(x, w, c)
            seen = np.zeros((H, W), dtype=bool)
            for dy in range(3):
                for dx in range(3):
                    y, xx = (y0 + 1 - dy) % H, (x0 + 1 - dx) % W
                    np.testing.assert_allclose(out[0, y, xx], c + w[:, i, dy, dx], rtol=0, atol=1e-15)
                    seen[y, xx] = True
            np.testing.assert_allclose(out[0][~seen], np.broadcast_to(c, out[0][~seen].shape), rtol=0, atol=1e-15)


def test_conv3_matches_scipy_correlate_wrap():
    """Per (output, input) channel pair, conv3 is scipy.ndimage.correlate with mode='wrap' (an independent
    implementation of the same circular cross-correlation), plus the bias."""
    ndimage = pytest.importorskip("scipy.ndimage")
    x, w, c = _conv_case(71, H=6, W=4, ci=3, co=2)
    out = learned.conv3(x, w, c)
    for n in range(x.shape[0]):
        for o in range(w.shape[0]):
            ref = np.full(x.shape[1:3], c[o])
            for i in range(w.shape[1]):
                ref += ndimage.correlate(x[n, :, :, i], w[o, i], mode="wrap")
            np.testing.assert_allclose(out[n, :, :, o], ref, rtol=1e-13, atol=1e-13)


def test_conv3_matches_torch_circular_conv2d():
    """torch.nn.functional.conv2d (a cross-correlation) after circular padding by one cell: a third,
    independent implementation on the CPU."""
    torch = pytest.importorskip("torch")
    x, w, c = _conv_case(72, n=2, H=5, W=3, ci=2, co=4)
    xt = torch.from_numpy(np.ascontiguousarray(x.transpose(0, 3, 1, 2)))
    xt = torch.nn.functional.pad(xt, (1, 1, 1, 1), mode="circular")
    ref = torch.nn.functional.conv2d(xt, torch.from_numpy(w), torch.from_numpy(c)).numpy().transpose(0, 2, 3, 1)
    np.testing.assert_allclose(learned.conv3(x, w, c), ref, rtol=1e-12, atol=1e-12)


def test_channel_layout_is_re_im_interleaved():
    """Channel 2r carries Re h_r and channel 2r + 1 carries Im h_r."""
    rng = np.random.default_rng(73)
    h = rng.standard_normal((1, 2, 3, 4)) + 1j * rng.standard_normal((1, 2, 3, 4))
    ch = learned._to_channels(h)
    assert ch.shape == (1, 2, 3, 8)
    np.testing.assert_array_equal(ch[..., 4], h[..., 2].real)
    np.testing.assert_array_equal(ch[..., 5], h[..., 2].imag)
    np.testing.assert_array_equal(learned._from_channels(ch), h)
