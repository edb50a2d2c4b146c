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
