"""Learned coarse propagator: plain FP64 forward / backward and one Adam step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

    G(u, t_n) = S(u) + Net([S(u), nu(t_n)/nu0])

S is the periodic integer shift by s = a * Delta t_slice / h cells (the exact
transport of the advection term over one slice when that is a whole number of
cells).  Net is four periodic 3x3x3 convolutions, 2 -> 16 -> 16 -> 16 -> 1
channels, with GELU after the first three.  Loss: mean squared error against
F(u) over all points of all samples.  Adam (Kingma & Ba, 2015) with bias
correction updates FP32 master weights.

Linear mode (``linear=True``): identity activations, biases ignored, and the
second input channel nu_hat * S(u) instead of the constant nu_hat, so that
G(u) is linear in u with a kernel that depends on nu(t_n).

BF16 emulation.  With ``bf16=True`` the values the CUDA path stores in
bfloat16 are rounded to bfloat16 (round to nearest even) at the same points:
weights, the network input, the three activations, and the gradients of the
three pre-activations and of the output.  Arithmetic stays FP64 otherwise.
"""
import numpy as np

from . import core

LAYERS = [(2, 16), (16, 16), (16, 16), (16, 1)]   # (cin, cout)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of an IEEE binary32; rounding adds half an
    ulp of the kept part (0x7FFF plus the kept lsb for ties-to-even) before
    truncating.  Inputs are first rounded to binary32."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed=0, scale=None):
    """He-style normal init, FP64 (weights W[cout][cin][3][3][3], biases zero)."""
    rng = np.random.default_rng(seed)
    params = []
    for li, (ci, co) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (27 * ci)) if scale is None else scale
        if li == len(LAYERS) - 1:
            std = 0.0 if scale is None else scale   # last layer starts at zero: G = S
        W = rng.standard_normal((co, ci, 3, 3, 3)) * std
        b = np.zeros(co)
        params.append([W, b])
    return params


def forward(u, nu_hat, params, shift, bf16_emul=False, linear=False):
    """Return (G(u), cache).  u: [n][n][n] FP64."""
    q = bf16 if bf16_emul else (lambda v: np.asarray(v, dtype=np.float64))
    su = core.shift(u, shift)
    if linear:
        x = np.stack([q(su), q(np.float64(nu_hat)) * q(su)])
    else:
        x = np.stack([q(su), q(np.full(su.shape, nu_hat))])
    cache = {"x": [x], "z": [], "su": su}
    h = x
    for li, (W, b) in enumerate(params):
        z = core.conv3d_fwd(h, q(W), np.zeros_like(b) if linear else b)
        cache["z"].append(z)
        if li < len(params) - 1:
            h = q(z if linear else core.gelu(z))
            cache["x"].append(h)
        else:
            h = z
    return su + h[0], cache


def loss_and_grads(u_list, nu_list, target_list, params, shift, bf16_emul=False, linear=False):
    """MSE over all points of all samples and its gradients (FP64).  In linear
    mode the bias gradients are zero (the biases are not used)."""
    q = bf16 if bf16_emul else (lambda v: np.asarray(v, dtype=np.float64))
    count = sum(u.size for u in u_list)
    grads = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
    loss = 0.0
    for u, nu_hat, tgt in zip(u_list, nu_list, target_list):
        out, c = forward(u, nu_hat, params, shift, bf16_emul, linear)
        r = out - tgt
        loss += float(np.sum(r * r))
        dz = q((2.0 / count) * r)[None]
        for li in range(len(params) - 1, -1, -1):
            W, _ = params[li]
            x = c["x"][li]
            dW, db = core.conv3d_wgrad(x, dz)
            grads[li][0] += dW
            if not linear:
                grads[li][1] += db
            if li == 0:
                break
            da = core.conv3d_dgrad(dz, q(W))
            dz = q(da if linear else da * core.gelu_grad(c["z"][li - 1]))
    return loss / count, grads


def adam_step(params, grads, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (in place) of params; m, v: first/second moments; step >= 1."""
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        for p, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm *= b1
            mm += (1 - b1) * g
            vv *= b2
            vv += (1 - b2) * g * g
            mhat = mm / (1 - b1 ** step)
            vhat = vv / (1 - b2 ** step)
            p -= lr * mhat / (np.sqrt(vhat) + eps)


def compose_linear(params, nu_hat):
    """The linear network (identity activations, biases unused) as one periodic
    cross-correlation of its input x = S(u):

        Net(x)[p] = sum_e K[e] x[p + e],   e in [-4, 4]^3,   K = K_0 + nu_hat K_1,

    K_c the kernel of input channel c of layer 1 carried through layers 2-4.
    Cross-correlations compose by adding offsets: (W2 (W1 x))[p] =
    sum_{d1, d2} W2[d2] W1[d1] x[p + d1 + d2], channels contracted in between.
    Returns K as [9][9][9], index (e_z + 4, e_y + 4, e_x + 4)."""
    K = []
    for ch in range(2):
        A = np.asarray(params[0][0], dtype=np.float64)[:, ch]     # [16][3][3][3]
        for W, _ in params[1:]:
            W = np.asarray(W, dtype=np.float64)
            r = A.shape[-1]
            B = np.zeros((W.shape[0],) + (r + 2,) * 3)
            for dz in range(3):
                for dy in range(3):
                    for dx in range(3):
                        B[:, dz:dz + r, dy:dy + r, dx:dx + r] += np.einsum(
                            "oi,izyx->ozyx", W[:, :, dz, dy, dx], A)
            A = B
        K.append(A[0])
    return K[0] + float(nu_hat) * K[1]


def apply_kernel(x, K):
    """sum_e K[e] x[p + e] on a periodic [n][n][n] field, K of odd edge."""
    x = np.asarray(x, dtype=np.float64)
    R = K.shape[0] // 2
    out = np.zeros_like(x)
    for ez in range(-R, R + 1):
        for ey in range(-R, R + 1):
            for ex in range(-R, R + 1):
                w = K[ez + R, ey + R, ex + R]
                if w != 0.0:
                    out += w * np.roll(x, (-ez, -ey, -ex), axis=(0, 1, 2))
    return out


def zeros_like_params(params):
    return [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
