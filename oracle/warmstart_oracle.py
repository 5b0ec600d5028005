"""Plain CPU reference of the learned warm-start network -- TEST INFRASTRUCTURE ONLY.

Only the test suite may import this module.  It shares no code with the CUDA library.

The network maps the input image x (H x W x 8: the state s_k = (phi_p, phi_nfa, mu_p, mu_nfa),
normalised per channel, and its change d_k = s_k - s_{k-1} divided by r_k, the RMS of d_k over the
image per channel) to the correction y of the linearly extrapolated next state in the same units,
s_{k+1} ~ s_k + d_k + y * out_scale * r_k:

    z1 = conv(x, W1) + b1,  a1 = relu(z1)       8 -> 32 channels
    z2 = conv(a1, W2) + b2, a2 = relu(z2)       32 -> 32
    y  = conv(a2, W3) + b3                      32 -> 4
    conv(x, W)[r, q, o] = sum_{ky, kx, c} x[r + ky - 1, q + kx - 1, c] W[3 ky + kx, c, o]
                          (zero outside the image)

with the loss L = (sum E^2 + lap * sum (G E)^2) / count, E = y - t, where G is the graph Laplacian
of the pixel grid: (G E)_p = sum over the 4-neighbours q of p inside the image of (E_q - E_p).  Everything is float64 numpy with loops
over the 9 taps only; `bf16=True` rounds to bfloat16 at the points where the GPU kernels store
bfloat16 values (input, weights, hidden activations, the output gradient and the hidden
gradients), so that the two can be compared closely.

Parameter vector layout (as the library's): w1[9][16][32] (input channels padded to 16), b1[32],
w2[9][32][32], b2[32], w3[9][32][8] (output channels padded to 8), b3[8].
"""
from __future__ import annotations

import numpy as np

C, CIN, COUT = 32, 16, 8
NIN, NOUT = 8, 4  # channels the network uses of the padded CIN, COUT
SHAPES = [("w1", (9, CIN, C)), ("b1", (C,)), ("w2", (9, C, C)), ("b2", (C,)), ("w3", (9, C, COUT)),
          ("b3", (COUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], np.float64).reshape(shape)
        k += n
    # padded channels do not exist in the network
    out["w1"] = out["w1"][:, :NIN, :]
    out["w3"] = out["w3"][:, :, :NOUT]
    out["b3"] = out["b3"][:NOUT]
    return out


def pack_grads(g: dict) -> np.ndarray:
    full = {"w1": np.zeros((9, CIN, C)), "b1": g["b1"], "w2": g["w2"], "b2": g["b2"],
            "w3": np.zeros((9, C, COUT)), "b3": np.zeros(COUT)}
    full["w1"][:, :NIN, :] = g["w1"]
    full["w3"][:, :, :NOUT] = g["w3"]
    full["b3"][:NOUT] = g["b3"]
    return np.concatenate([full[n].ravel() for n, _ in SHAPES])


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) via the float32 bit pattern."""
    f = np.asarray(a, np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def shift(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """s[r, q] = x[r + dy, q + dx], zero outside (x: H x W x C)."""
    H, W = x.shape[:2]
    s = np.zeros_like(x)
    r0, r1 = max(0, -dy), min(H, H - dy)
    q0, q1 = max(0, -dx), min(W, W - dx)
    s[r0:r1, q0:q1] = x[r0 + dy:r1 + dy, q0 + dx:q1 + dx]
    return s


def conv(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """3x3 'same' convolution (cross-correlation), x: H x W x Ci, w: 9 x Ci x Co."""
    out = np.zeros(x.shape[:2] + (w.shape[2],))
    for tap in range(9):
        out += shift(x, tap // 3 - 1, tap % 3 - 1) @ w[tap]
    return out


def conv_back_data(dz: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Gradient of sum(conv(x, w) * dz) with respect to x."""
    out = np.zeros(dz.shape[:2] + (w.shape[1],))
    for tap in range(9):
        out += shift(dz @ w[tap].T, -(tap // 3 - 1), -(tap % 3 - 1))
    return out


def conv_back_weight(x: np.ndarray, dz: np.ndarray) -> np.ndarray:
    """Gradient of sum(conv(x, w) * dz) with respect to w."""
    g = np.zeros((9, x.shape[2], dz.shape[2]))
    for tap in range(9):
        xs = shift(x, tap // 3 - 1, tap % 3 - 1)
        g[tap] = xs.reshape(-1, x.shape[2]).T @ dz.reshape(-1, dz.shape[2])
    return g


def change_scale(s: np.ndarray, q: np.ndarray) -> np.ndarray:
    """r[c] = sqrt(mean over the image of (s - q)[..., c]^2), at least 1e-30, rounded to float32."""
    d = np.asarray(s, np.float64) - np.asarray(q, np.float64)
    r = np.sqrt((d.reshape(-1, 4) ** 2).mean(0))
    return np.maximum(r, 1e-30).astype(np.float32).astype(np.float64)


def inputs(s: np.ndarray, q: np.ndarray, mean=None, inv_std=None) -> np.ndarray:
    """Network input from the state s and its predecessor q (H x W x 4 each): the normalised
    fields and their change in units of its RMS, in float32 as the library forms them."""
    f32 = np.float32
    mean = np.zeros(NIN) if mean is None else np.asarray(mean)
    inv_std = np.ones(NIN) if inv_std is None else np.asarray(inv_std)
    r = change_scale(s, q)
    raw = np.concatenate([np.asarray(s, f32), ((np.asarray(s, np.float64) - q) / r).astype(f32)], -1)
    return ((raw - mean.astype(f32)) * inv_std.astype(f32)).astype(np.float64)


def targets(s: np.ndarray, q: np.ndarray, n: np.ndarray, out_scale) -> np.ndarray:
    """Training target of y: ((n - s) - (s - q)) / (out_scale * r), float32 as the library."""
    e = (np.asarray(n, np.float64) - s) - (np.asarray(s, np.float64) - q)
    return (e / (change_scale(s, q) * np.asarray(out_scale, np.float64))).astype(np.float32).astype(np.float64)


def predict(p: dict, s: np.ndarray, q: np.ndarray, norm=None, bf: bool = False) -> np.ndarray:
    """Next-state prediction s + (s - q) + y * out_scale * r (norm = (mean[8], inv_std[8], out_scale[4]))."""
    mean, inv_std, out_scale = (None, None, np.ones(NOUT)) if norm is None else norm
    y, _ = forward(p, inputs(s, q, mean, inv_std), bf)
    return s + (s - q) + y * (np.asarray(out_scale, np.float64) * change_scale(s, q))


def forward(p: dict, x: np.ndarray, bf: bool = False):
    """Network output y (H x W x 4) for the input image x (H x W x 8)."""
    r = bf16 if bf else (lambda a: a)
    w1, w2, w3 = r(p["w1"]), r(p["w2"]), r(p["w3"])
    x = r(x)
    z1 = conv(x, w1) + p["b1"]
    a1 = r(np.maximum(z1, 0.0))
    z2 = conv(a1, w2) + p["b2"]
    a2 = r(np.maximum(z2, 0.0))
    y = conv(a2, w3) + p["b3"]
    return y, (x, a1, a2, w1, w2, w3)


def grid_laplacian(e: np.ndarray) -> np.ndarray:
    """(G e)_p = sum over the 4-neighbours q of p inside the image of (e_q - e_p) (e: H x W x C)."""
    H, W = e.shape[:2]
    g = np.zeros_like(e)
    for dy, dx in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        inside = np.zeros((H, W, 1))
        inside[max(0, -dy):min(H, H - dy), max(0, -dx):min(W, W - dx)] = 1.0
        g += (shift(e, dy, dx) - e) * inside
    return g


def backward(p: dict, cache, dy: np.ndarray, g: dict, bf: bool = False) -> None:
    """Accumulate into g the parameter gradients for the output gradient dy (H x W x 4) of the
    forward pass that returned `cache`."""
    r = bf16 if bf else (lambda a: a)
    x0, a1, a2, w1, w2, w3 = cache
    g["w3"] += conv_back_weight(a2, dy)
    g["b3"] += dy.sum((0, 1))
    dz2 = r(conv_back_data(dy, w3) * (a2 > 0))
    g["w2"] += conv_back_weight(a1, dz2)
    g["b2"] += dz2.sum((0, 1))
    dz1 = r(conv_back_data(dz2, w2) * (a1 > 0))
    g["w1"] += conv_back_weight(x0, dz1)
    g["b1"] += dz1.sum((0, 1))


def loss_and_grads(theta: np.ndarray, xs: np.ndarray, ts: np.ndarray, bf: bool = False, lap: float = 0.0):
    """Loss over a batch (xs: B x H x W x 8 inputs, ts: B x H x W x 4 targets) and its gradient
    vector; G is symmetric, so d/dE of sum (G E)^2 is 2 G (G E)."""
    p = unpack(theta)
    r = bf16 if bf else (lambda a: a)
    count = ts.size
    g = {k: np.zeros_like(v) for k, v in p.items()}
    L = 0.0
    for x, t in zip(xs, ts):
        y, cache = forward(p, x, bf)
        d = y - t
        ge = grid_laplacian(d)
        L += float((d * d).sum()) + lap * float((ge * ge).sum())
        backward(p, cache, r(2.0 * (d + lap * grid_laplacian(ge)) / count), g, bf)
    return L / count, pack_grads(g)


def residual_loss_and_grads(theta: np.ndarray, states, prevs, rhss, apply_A, norm=None, bf: bool = False,
                            apply_Pinv=None):
    """Loss against the residual of the time step and its gradient vector.

    states, prevs: B x H x W x 4 (s_k, s_{k-1}); rhss: B x H x W x 4, the right-hand side b of the
    step from s_k; apply_A: the symmetric block operator on an H x W x 4 image (node = pixel).
    Per sample and species (channels sp and sp + 2), r_ex = b - A (2 s - q) and r = r_ex - A c with
    c = y * out_scale * rms(s - q); |r|^2 is <r, z> with z = apply_Pinv(r) (a symmetric positive
    definite preconditioner) or z = r.  The loss is the mean of |r|^2 / |r_ex|^2 over samples and
    species, so 1 for the zero network.  dL/dc = -2 A z / (|r_ex|^2 * 2B)."""
    Pinv = apply_Pinv if apply_Pinv is not None else (lambda v: v)
    mean, inv_std, out_scale = (None, None, np.ones(NOUT)) if norm is None else norm
    p = unpack(theta)
    r16 = bf16 if bf else (lambda a: a)
    B = len(states)
    g = {k: np.zeros_like(v) for k, v in p.items()}
    L = 0.0
    for s, q, b in zip(states, prevs, rhss):
        y, cache = forward(p, inputs(s, q, mean, inv_std), bf)
        scale = np.asarray(out_scale, np.float64) * change_scale(s, q)
        c = y * scale
        rex = b - apply_A(2.0 * s - q)
        res = rex - apply_A(c)
        zex, z = Pinv(rex), Pinv(res)
        gA = apply_A(z)
        dc = np.zeros_like(c)
        for sp in (0, 1):
            ch = [sp, sp + 2]
            den = float((rex[..., ch] * zex[..., ch]).sum())
            if den > 0:
                L += float((res[..., ch] * z[..., ch]).sum()) / den
                dc[..., ch] = -2.0 * gA[..., ch] / (den * 2 * B)
        backward(p, cache, r16(dc * scale), g, bf)
    return L / (2 * B), pack_grads(g)
