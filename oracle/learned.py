"""CPU oracle of the learned Fourier-domain correction (test infrastructure).

TEST INFRASTRUCTURE: used only by tests/ and the CPU legs of bench.py; the
solver library never imports it.

The network adds a learned correction to the block-Jacobi preconditioner of
Sec. III-B:  M(r) = P_K^{-1} r + f(r), with, for one column r in C^N,

  1. u = pad(r) on the (my, mx) cell grid (Eq. (xc2)); r^ = FFT2(u)/sqrt(mx my)
     for every basis index p (the 2-level blockwise DFT of Eq. (F2)).
  2. h_k = B_k r^_k                     per bin k, B_k in C^{R x b}   (encode)
  3. with h read as 2R real channels on the (ky, kx) grid (channel 2r = Re h_r,
     2r+1 = Im h_r), three 3x3 convolutions with circular padding:
       a1 = conv(h; W1, c1), x1 = relu(a1), a2 = conv(x1; W2, c2),
       x2 = relu(a2), a3 = conv(x2; W3, c3), g = h + a3
  4. z^_k = A_k g_k                     per bin k, A_k in C^{b x R}   (decode)
  5. f(r) = crop(IFFT2_unnormalised(z^)) / sqrt(mx my)

conv(x; W, c)[y, x, o] = c[o] + sum_{i, dy, dx} W[o, i, dy, dx] x[(y+dy-1) mod my, (x+dx-1) mod mx, i].
Training loss over a minibatch of pairs (r_c, e_c), e_c the exact correction:
  L = (1/n) sum_c || P_K^{-1} r_c + f(r_c) - e_c ||^2 / || e_c ||^2.
Gradients of complex parameters are dL/dRe + i dL/dIm.  Everything is
binary64 numpy; numpy's FFT is the library step for the DFTs.

Parity: gradients pinned by central finite differences (tests/test_oracle_learned.py).
"""
from __future__ import annotations

import numpy as np

import oracle


def param_shapes(bins: int, b: int, rank: int, ch: int) -> dict:
    return {"B": (bins, rank, b), "A": (bins, b, rank),
            "W1": (ch, 2 * rank, 3, 3), "c1": (ch,),
            "W2": (ch, ch, 3, 3), "c2": (ch,),
            "W3": (2 * rank, ch, 3, 3), "c3": (2 * rank,)}


def conv3(x: np.ndarray, w: np.ndarray, c: np.ndarray) -> np.ndarray:
    """x: (n, H, W, Ci); w: (Co, Ci, 3, 3); circular 3x3 convolution + bias."""
    out = np.broadcast_to(c, x.shape[:3] + (w.shape[0],)).copy()
    for dy in range(3):
        for dx in range(3):
            shifted = np.roll(x, shift=(1 - dy, 1 - dx), axis=(1, 2))   # x[(y+dy-1), (x+dx-1)]
            out += np.einsum("nhwi,oi->nhwo", shifted, w[:, :, dy, dx])
    return out


def conv3_backward(x: np.ndarray, w: np.ndarray, da: np.ndarray):
    """Gradients of conv3 w.r.t. x, w, c given da = dL/d(output)."""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for dy in range(3):
        for dxx in range(3):
            shifted = np.roll(x, shift=(1 - dy, 1 - dxx), axis=(1, 2))
            dw[:, :, dy, dxx] = np.einsum("nhwo,nhwi->oi", da, shifted)
            back = np.einsum("nhwo,oi->nhwi", da, w[:, :, dy, dxx])
            dx += np.roll(back, shift=(dy - 1, dxx - 1), axis=(1, 2))
    dc = da.sum(axis=(0, 1, 2))
    return dx, dw, dc


def _to_channels(h: np.ndarray) -> np.ndarray:
    """(n, H, W, R) complex -> (n, H, W, 2R) real, channel 2r = Re, 2r+1 = Im."""
    out = np.empty(h.shape[:3] + (2 * h.shape[3],))
    out[..., 0::2] = h.real
    out[..., 1::2] = h.imag
    return out


def _from_channels(x: np.ndarray) -> np.ndarray:
    return x[..., 0::2] + 1j * x[..., 1::2]


def forward(gen: np.ndarray, params: dict, r: np.ndarray, mx: int, my: int, keep: bool = False):
    """f(r) for columns r of shape (n, N); returns (n, N) complex (and the cache)."""
    nx, ny, b = (gen.shape[1] + 1) // 2, (gen.shape[0] + 1) // 2, gen.shape[2]
    n = r.shape[0]
    s = np.sqrt(mx * my)
    u = np.zeros((n, my, mx, b), dtype=np.complex128)
    u[:, :ny, :nx] = r.reshape(n, ny, nx, b)
    rh = np.fft.fft2(u, axes=(1, 2)) / s                              # (n, my, mx, b)
    B = params["B"].reshape(my, mx, -1, b)
    A = params["A"].reshape(my, mx, b, -1)
    h = np.einsum("yxrp,nyxp->nyxr", B, rh)
    hc = _to_channels(h)
    a1 = conv3(hc, params["W1"], params["c1"])
    x1 = np.maximum(a1, 0.0)
    a2 = conv3(x1, params["W2"], params["c2"])
    x2 = np.maximum(a2, 0.0)
    a3 = conv3(x2, params["W3"], params["c3"])
    g = _from_channels(hc + a3)
    zh = np.einsum("yxpr,nyxr->nyxp", A, g)
    z = np.fft.ifft2(zh, axes=(1, 2)) * (mx * my) / s
    out = z[:, :ny, :nx].reshape(n, -1)
    if keep:
        return out, dict(rh=rh, hc=hc, a1=a1, x1=x1, a2=a2, x2=x2, g=g)
    return out


def loss_and_grads(gen: np.ndarray, params: dict, r: np.ndarray, e: np.ndarray, mx: int, my: int):
    """Loss L and dL/dparam for a minibatch (r, e) of shape (n, N)."""
    nx, ny, b = (gen.shape[1] + 1) // 2, (gen.shape[0] + 1) // 2, gen.shape[2]
    n = r.shape[0]
    s = np.sqrt(mx * my)
    f, cache = forward(gen, params, r, mx, my, keep=True)
    base = oracle.block_jacobi_apply(gen, r.T).T
    q = base + f
    en2 = np.sum(np.abs(e) ** 2, axis=1)
    loss = float(np.mean(np.sum(np.abs(q - e) ** 2, axis=1) / en2))
    dz = 2.0 * (q - e) / en2[:, None] / n                              # dL/dRe + i dL/dIm
    pad = np.zeros((n, my, mx, b), dtype=np.complex128)
    pad[:, :ny, :nx] = dz.reshape(n, ny, nx, b)
    dzh = np.fft.fft2(pad, axes=(1, 2)) / s                            # adjoint of crop(ifft2_unnorm)/s
    A = params["A"].reshape(my, mx, b, -1)
    B = params["B"].reshape(my, mx, -1, b)
    g = cache["g"]
    dA = np.einsum("nyxp,nyxr->yxpr", dzh, np.conj(g))
    dg = np.einsum("yxpr,nyxp->nyxr", np.conj(A), dzh)
    dgc = _to_channels(dg)
    dhc = dgc.copy()
    dx2, dW3, dc3 = conv3_backward(cache["x2"], params["W3"], dgc)
    da2 = dx2 * (cache["a2"] > 0)
    dx1, dW2, dc2 = conv3_backward(cache["x1"], params["W2"], da2)
    da1 = dx1 * (cache["a1"] > 0)
    dh_c, dW1, dc1 = conv3_backward(cache["hc"], params["W1"], da1)
    dhc += dh_c
    dh = _from_channels(dhc)
    dB = np.einsum("nyxr,nyxp->yxrp", dh, np.conj(cache["rh"]))
    grads = {"B": dB.reshape(params["B"].shape), "A": dA.reshape(params["A"].shape),
             "W1": dW1, "c1": dc1, "W2": dW2, "c2": dc2, "W3": dW3, "c3": dc3}
    return loss, grads


def loss_only(gen, params, r, e, mx, my) -> float:
    f = forward(gen, params, r, mx, my)
    base = oracle.block_jacobi_apply(gen, r.T).T
    q = base + f
    return float(np.mean(np.sum(np.abs(q - e) ** 2, axis=1) / np.sum(np.abs(e) ** 2, axis=1)))
