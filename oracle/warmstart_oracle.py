"""Plain CPU reference of the learned warm-start network -- TEST INFRASTRUCTURE ONLY.

Only the test suite may import this module.  It shares no code with the CUDA library.

From the last three states s = s_k, q = s_{k-1}, q2 = s_{k-2} (each H x W x 4: phi_p, phi_nfa, mu_p,
mu_nfa) the network predicts the next state as a learned second-order extrapolation,

    s_{k+1} ~ s + d + theta * D,   d = s - q,   D = s - 2 q + q2,   theta = y * out_scale,

so the zero network is linear extrapolation and theta = 1 quadratic extrapolation; the correction
is confined to the (smooth) second difference, scaled pixel by pixel.  The input image x has 12
channels: the fields normalised per channel, d / r1 and D / r2, where r1, r2 are the RMS over the
image of d and D per channel (the first two groups also shifted and scaled by mean / inv_std):

    z1 = conv(x, W1) + b1,  a1 = relu(z1)       12 -> 32 channels
    z2 = conv(a1, W2) + b2, a2 = relu(z2)       32 -> 32
    y  = conv(a2, W3) + b3                      32 -> 4
    conv(x, W)[r, q, o] = sum_{ky, kx, c} x[r + ky - 1, q + kx - 1, c] W[3 ky + kx, c, o]
                          (zero outside the image)

Losses: in state space, L = (sum E^2 + lap * sum (G E)^2) / count with E = (theta D - e) / r1,
e = n - 2 s + q the linear extrapolation's error (n = s_{k+1}) and G the graph Laplacian of the
pixel grid, (G E)_p = sum over the 4-neighbours q of p inside the image of (E_q - E_p); or the
mean log ratio of the step's residual to linear extrapolation's (residual_loss_and_grads).  Everything is float64 numpy with loops over the 9
taps only; `bf16=True` rounds to bfloat16 at the points where the GPU kernels store bfloat16
values (input, weights, hidden activations, the output gradient and the hidden gradients), so
that the two can be compared closely.

Parameter vector layout (as the library's): w1[9][16][32] (input channels padded to 16), b1[32],
w2[9][32][32], b2[32], w3[9][32][8] (output channels padded to 8), b3[8].
"""
from __future__ import annotations

import numpy as np

C, CIN, COUT = 32, 16, 8
NIN, NOUT = 12, 4  # channels the network uses of the padded CIN, COUT
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
    return rms(np.asarray(s, np.float64) - np.asarray(q, np.float64))


def second_difference(s: np.ndarray, q: np.ndarray, q2: np.ndarray) -> np.ndarray:
    """D = s - 2 q + q2 (float64)."""
    return np.asarray(s, np.float64) - 2.0 * np.asarray(q, np.float64) + np.asarray(q2, np.float64)


def rms(d: np.ndarray) -> np.ndarray:
    """Per-channel RMS over the image, at least 1e-30, rounded to float32 (as the library keeps it)."""
    r = np.sqrt((np.asarray(d, np.float64).reshape(-1, 4) ** 2).mean(0))
    return np.maximum(r, 1e-30).astype(np.float32).astype(np.float64)


def inputs(s: np.ndarray, q: np.ndarray, q2: np.ndarray, mean=None, inv_std=None) -> np.ndarray:
    """Network input (H x W x 12) from the last three states, in float32 as the library forms it:
    (fields - mean[0:4]) * inv_std[0:4], (d / r1 - mean[4:8]) * inv_std[4:8], D / r2."""
    f32 = np.float32
    mean = np.zeros(8) if mean is None else np.asarray(mean)
    inv_std = np.ones(8) if inv_std is None else np.asarray(inv_std)
    d = np.asarray(s, np.float64) - q
    D = second_difference(s, q, q2)
    raw = np.concatenate([np.asarray(s, f32), (d / change_scale(s, q)).astype(f32)], -1)
    first = (raw - mean.astype(f32)) * inv_std.astype(f32)
    return np.concatenate([first, (D / rms(D)).astype(f32)], -1).astype(np.float64)


def predict(p: dict, s: np.ndarray, q: np.ndarray, q2: np.ndarray, norm=None, bf: bool = False) -> np.ndarray:
    """Next-state prediction s + d + (y * out_scale) * D (norm = (mean[8], inv_std[8], out_scale[4]))."""
    mean, inv_std, out_scale = (None, None, np.ones(NOUT)) if norm is None else norm
    y, _ = forward(p, inputs(s, q, q2, mean, inv_std), bf)
    return s + (np.asarray(s, np.float64) - q) + y * np.asarray(out_scale, np.float64) * second_difference(s, q, q2)


def forward(p: dict, x: np.ndarray, bf: bool = False):
    """Network output y (H x W x 4) for the input image x (H x W x 12)."""
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


def loss_and_grads(theta: np.ndarray, S, Q, Q2, Nn, norm=None, bf: bool = False, lap: float = 0.0):
    """State-space loss over a batch of consecutive states (each B x H x W x 4: s_k, s_{k-1},
    s_{k-2}, s_{k+1}) and its gradient vector: E = (theta D - e) / r1 with theta = y * out_scale,
    e = n - 2 s + q; G is symmetric, so d/dE of sum (G E)^2 is 2 G (G E);
    dL/dy = dL/dE * out_scale * D / r1."""
    mean, inv_std, out_scale = (None, None, np.ones(NOUT)) if norm is None else norm
    out_scale = np.asarray(out_scale, np.float64)
    p = unpack(theta)
    r = bf16 if bf else (lambda a: a)
    count = np.asarray(S).size
    g = {k: np.zeros_like(v) for k, v in p.items()}
    L = 0.0
    for s, q, q2, n in zip(S, Q, Q2, Nn):
        y, cache = forward(p, inputs(s, q, q2, mean, inv_std), bf)
        D = second_difference(s, q, q2)
        r1 = change_scale(s, q)
        e = np.asarray(n, np.float64) - 2.0 * np.asarray(s, np.float64) + q
        E = (y * out_scale * D - e) / r1
        ge = grid_laplacian(E)
        L += float((E * E).sum()) + lap * float((ge * ge).sum())
        dE = 2.0 * (E + lap * grid_laplacian(ge)) / count
        backward(p, cache, r(dE * out_scale * D / r1), g, bf)
    return L / count, pack_grads(g)


def residual_loss_and_grads(theta: np.ndarray, states, prevs, prevs2, rhss, apply_A, norm=None, bf: bool = False,
                            apply_Pinv=None):
    """Loss against the residual of the time step and its gradient vector.

    states, prevs, prevs2: B x H x W x 4 (s_k, s_{k-1}, s_{k-2}); rhss: B x H x W x 4, the right-hand
    side b of the step from s_k; apply_A: the symmetric block operator on an H x W x 4 image
    (node = pixel).  Per sample and species (channels sp and sp + 2), r_ex = b - A (2 s - q) (linear
    extrapolation) and r = r_ex - A c with c = theta D; |r|^2 is <r, z> with z = apply_Pinv(r) (a
    symmetric positive definite preconditioner) or z = r.  The loss is the mean of
    ln(|r|^2 / |r_ex|^2) over samples and species -- 0 for the zero network, negative where the
    prediction beats linear extrapolation; Krylov iteration counts grow with the logarithm of the
    initial residual, so every sample's relative gain counts alike.  dL/dc = -2 A z / (|r|^2 * 2B)
    and dL/dy = dL/dc * out_scale * D."""
    Pinv = apply_Pinv if apply_Pinv is not None else (lambda v: v)
    mean, inv_std, out_scale = (None, None, np.ones(NOUT)) if norm is None else norm
    out_scale = np.asarray(out_scale, np.float64)
    p = unpack(theta)
    r16 = bf16 if bf else (lambda a: a)
    B = len(states)
    g = {k: np.zeros_like(v) for k, v in p.items()}
    L = 0.0
    for s, q, q2, b in zip(states, prevs, prevs2, rhss):
        y, cache = forward(p, inputs(s, q, q2, mean, inv_std), bf)
        D = second_difference(s, q, q2)
        c = y * out_scale * D
        rex = b - apply_A(2.0 * s - q)
        res = rex - apply_A(c)
        zex, z = Pinv(rex), Pinv(res)
        gA = apply_A(z)
        dc = np.zeros_like(c)
        for sp in (0, 1):
            ch = [sp, sp + 2]
            den = float((rex[..., ch] * zex[..., ch]).sum())
            num = float((res[..., ch] * z[..., ch]).sum())
            if den > 0 and num > 0:
                L += np.log(num / den)
                dc[..., ch] = -2.0 * gA[..., ch] / (num * 2 * B)
        backward(p, cache, r16(dc * out_scale * D), g, bf)
    return L / (2 * B), pack_grads(g)
