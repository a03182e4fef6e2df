"""Oracle of the learned initial guess: a 4-level U-Net in plain numpy FP64.

Test infrastructure only (see oracle/__init__.py).  The paper has no
network: this is the initial-guess generator for the Newton-Krylov
fixed-point solve (Sec. 3.1.2, Eq. 43) whose cost grows with the distance of
the start from the fixed point.  The network maps per-point inputs (the
cylinder mask and a Reynolds-number plane) to a base-flow vorticity field.

Definition (everything the CUDA path computes, in the same order):

* conv3x3(h; W, b)[o, y, x] = b[o] + sum_{i, p, q} W[o, i, p, q]
  h[i, (y + p - 1) mod H, (x + q - 1) mod W]  (cross-correlation with
  periodic wrap, the domain's boundary condition), then ReLU;
* encoder level l = 0..3: two conv3x3 + ReLU at width c_l = width 2^l;
  between levels a 2x2 average pool;
* decoder level l = 2..0: nearest 2x upsampling of the level below,
  concatenated (upsampled channels first, then the encoder's skip), two
  conv3x3 + ReLU at width c_l;
* output: 1x1 convolution to one channel, no activation;
* loss: mean over all output points of (y - target)^2;
* Adam (Kingma & Ba): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
  theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Parameters are one flat vector, tensor by tensor in `layout()` order, each
weight [out][in][3][3] (or [1][c0] for the output layer) followed by its
bias [out].

bf16=True rounds, to bfloat16 with round-to-nearest-even, exactly the
values the CUDA path stores in bfloat16: the network input, the weights of
the 3x3 convolutions and the output layer, every ReLU output and every
pooled value.  Sums stay FP64 here (FP32 on the GPU).

Pins (tests/test_oracle_unet.py): conv3x3 against scipy.ndimage.correlate
with mode='wrap'; pooling and upsampling adjoint to their backward maps;
every parameter gradient against central differences of the loss; the first
Adam step against its closed form; bf16 rounding against exactly
representable and halfway cases.
"""
from __future__ import annotations

import numpy as np

LEVELS = 4


def layout(in_ch: int, width: int):
    """[(name, shape)] of the parameter tensors in flat order."""
    c = [width << l for l in range(LEVELS)]
    out = []

    def conv(name, ci, co):
        out.append((name + ".w", (co, ci, 3, 3)))
        out.append((name + ".b", (co,)))

    ci = in_ch
    for l in range(LEVELS):
        conv(f"enc{l}a", ci, c[l])
        conv(f"enc{l}b", c[l], c[l])
        ci = c[l]
    for l in range(LEVELS - 2, -1, -1):
        conv(f"dec{l}a", c[l + 1] + c[l], c[l])
        conv(f"dec{l}b", c[l], c[l])
    out.append(("out.w", (1, c[0])))
    out.append(("out.b", (1,)))
    return out


def param_count(in_ch: int, width: int) -> int:
    return int(sum(np.prod(s) for _, s in layout(in_ch, width)))


def unpack(theta: np.ndarray, in_ch: int, width: int) -> dict:
    p, k = {}, 0
    for name, shape in layout(in_ch, width):
        n = int(np.prod(shape))
        p[name] = theta[k:k + n].reshape(shape)
        k += n
    return p


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    Values are first rounded to float32 (the CUDA path's arithmetic)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _noop(a):
    return a


# ---------------------------------------------------------------- layers

def conv3x3(h, w, b):
    """h [B][ci][H][W], w [co][ci][3][3], b [co] -> [B][co][H][W]."""
    out = np.broadcast_to(b[None, :, None, None], (h.shape[0], w.shape[0]) + h.shape[2:]).copy()
    for p in range(3):
        for q in range(3):
            shifted = np.roll(h, shift=(1 - p, 1 - q), axis=(2, 3))   # h[.., y+p-1, x+q-1]
            out += np.einsum("oi,biyx->boyx", w[:, :, p, q], shifted)
    return out


def conv3x3_backward(h, w, gz):
    """Gradients of conv3x3 for the upstream gradient gz = dL/d(output)."""
    gh = np.zeros_like(h)
    gw = np.zeros_like(w)
    for p in range(3):
        for q in range(3):
            shifted = np.roll(h, shift=(1 - p, 1 - q), axis=(2, 3))
            gw[:, :, p, q] = np.einsum("boyx,biyx->oi", gz, shifted)
            gh += np.roll(np.einsum("oi,boyx->biyx", w[:, :, p, q], gz), shift=(p - 1, q - 1), axis=(2, 3))
    return gh, gw, gz.sum(axis=(0, 2, 3))


def pool2(h):
    B, C, H, W = h.shape
    return h.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def pool2_backward(g):
    return np.repeat(np.repeat(g, 2, axis=2), 2, axis=3) / 4.0


def up2(h):
    return np.repeat(np.repeat(h, 2, axis=2), 2, axis=3)


def up2_backward(g):
    B, C, H, W = g.shape
    return g.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


# ------------------------------------------------------------- network

def forward(theta, x, in_ch, width, bf16_storage=False):
    """Returns (y [B][H][W], cache for backward)."""
    r = bf16 if bf16_storage else _noop
    p = unpack(theta, in_ch, width)
    wq = {k: (r(v) if k.endswith(".w") else v) for k, v in p.items()}
    h = r(x)
    acts = []          # (name, input, relu output) per conv, in forward order
    skips = []
    for l in range(LEVELS):
        for s in "ab":
            z = conv3x3(h, wq[f"enc{l}{s}.w"], p[f"enc{l}{s}.b"])
            a = r(np.maximum(z, 0.0))
            acts.append((f"enc{l}{s}", h, a))
            h = a
        if l < LEVELS - 1:
            skips.append(h)
            h = r(pool2(h))
    for l in range(LEVELS - 2, -1, -1):
        h = np.concatenate([up2(h), skips[l]], axis=1)
        for s in "ab":
            z = conv3x3(h, wq[f"dec{l}{s}.w"], p[f"dec{l}{s}.b"])
            a = r(np.maximum(z, 0.0))
            acts.append((f"dec{l}{s}", h, a))
            h = a
    y = np.einsum("c,bcyx->byx", wq["out.w"][0], h) + p["out.b"][0]
    return y, dict(p=p, wq=wq, acts=acts, top=h, in_ch=in_ch, width=width)


def mse(y, target):
    """Loss and dL/dy."""
    d = y - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(cache, gy):
    """Flat gradient of the loss for dL/dy = gy (weights' gradients with
    respect to the stored, possibly rounded, weights)."""
    p, wq, acts = cache["p"], cache["wq"], {n: (i, a) for n, i, a in cache["acts"]}
    g = {}
    top = cache["top"]
    g["out.w"] = np.einsum("byx,bcyx->c", gy, top)[None, :]
    g["out.b"] = np.array([gy.sum()])
    gh = np.einsum("c,byx->bcyx", wq["out.w"][0], gy)
    skip_grad = {}
    c = [cache["width"] << l for l in range(LEVELS)]

    def through(name, gh_out):
        inp, a = acts[name]
        gz = gh_out * (a > 0)
        gin, gw, gb = conv3x3_backward(inp, wq[name + ".w"], gz)
        g[name + ".w"], g[name + ".b"] = gw, gb
        return gin

    for l in range(0, LEVELS - 1):
        gh = through(f"dec{l}b", gh)
        gh = through(f"dec{l}a", gh)
        # split the concatenation: upsampled channels first, then the skip
        skip_grad[l] = gh[:, c[l + 1]:]
        gh = up2_backward(gh[:, :c[l + 1]])
    # gh is now the gradient of the bottom level's output
    for l in range(LEVELS - 1, -1, -1):
        if l < LEVELS - 1:
            gh = pool2_backward(gh) + skip_grad[l]
        gh = through(f"enc{l}b", gh)
        gh = through(f"enc{l}a", gh)
    return np.concatenate([g[name].ravel() for name, _ in layout(cache["in_ch"], cache["width"])])


def gradient(theta, x, target, in_ch, width, bf16_storage=False):
    y, cache = forward(theta, x, in_ch, width, bf16_storage)
    loss, gy = mse(y, target)
    return loss, backward(cache, gy)


def adam_step(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t = 1 for the first step); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
