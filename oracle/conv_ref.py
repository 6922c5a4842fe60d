"""FP64 NumPy reference of the learned corrector's network, loss and gradients.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): used by the tests to check
the CUDA forward/backward kernels of include/lc.h.  Plain definitions:
3x3 convolutions with zero padding 1, ReLU between layers, a pixel-shuffled
last layer (channel f*r*r + sy*r + sx of coarse pixel (y, x) is fine cell
(r*y + sy, r*x + sx) of field f), and the weighted mean-squared loss; the
gradients by the chain rule, layer by layer.
"""
import numpy as np


def layers_of(cin, width, depth, cout):
    return [(cin if l == 0 else width, cout if l == depth - 1 else width) for l in range(depth)]


def unpack(params, layers):
    out, off = [], 0
    for ci, co in layers:
        w = np.asarray(params[off:off + co * ci * 9], dtype=np.float64).reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = np.asarray(params[off:off + co], dtype=np.float64)
        off += co
        out.append((w, b))
    return out


def pack(grads):
    return np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])


def conv3x3(x, w, b):
    """y[o] = b[o] + sum_c sum_(ky,kx) w[o,c,ky,kx] x[c, y+ky-1, x+kx-1] (zero padding)."""
    _, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    y = np.zeros((w.shape[0], H, W)) + b[:, None, None]
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("oc,chw->ohw", w[:, :, ky, kx], xp[:, ky:ky + H, kx:kx + W])
    return y


def _id(a):
    return a


def forward(params, layers, x, quant=None):
    """Activations of every layer.  quant (None: exact) rounds each
    convolution's input operand first, e.g. bf16_round for a network whose
    convolutions multiply BF16 operands."""
    q = quant or _id
    acts = [np.asarray(x, dtype=np.float64)]
    L = len(layers)
    for l, (w, b) in enumerate(unpack(params, layers)):
        z = conv3x3(q(acts[-1]), w, b)
        acts.append(np.maximum(z, 0.0) if l < L - 1 else z)
    return acts


def shuffle(y, r, nout):
    c, H, W = y.shape
    f = np.zeros((nout, H * r, W * r))
    for fi in range(nout):
        for sy in range(r):
            for sx in range(r):
                f[fi, sy::r, sx::r] = y[fi * r * r + sy * r + sx]
    return f


def unshuffle(fine, r, nout):
    _, Hf, Wf = fine.shape
    y = np.zeros((nout * r * r, Hf // r, Wf // r))
    for fi in range(nout):
        for sy in range(r):
            for sx in range(r):
                y[fi * r * r + sy * r + sx] = fine[fi, sy::r, sx::r]
    return y


def loss_and_grad(params, layers, x, target, r, nout, fw, quant=None):
    """Weighted MSE of the shuffled output against target and its gradient with
    respect to the packed parameters.  quant (None: exact) rounds the operands
    of every convolution -- forward inputs, and in the backward pass the
    incoming gradient and the layer input of each weight-gradient product and
    the incoming gradient of each input-gradient convolution -- the way a
    network on BF16 tensor-core products does.  The bias gradient of the last
    layer sums the unrounded dL/dy; those of the hidden layers sum their
    gradient as stored, i.e. rounded (a network that keeps hidden activations
    and their gradients in BF16)."""
    q = quant or _id
    acts = forward(params, layers, x, quant)
    wb = unpack(params, layers)
    y = acts[-1]
    fine = shuffle(y, r, nout)
    d = fine - np.asarray(target, dtype=np.float64)
    n = d[0].size
    loss = sum(fw[f] * np.sum(d[f] ** 2) / n for f in range(nout))
    gfine = np.stack([2.0 * fw[f] * d[f] / n for f in range(nout)])
    g = unshuffle(gfine, r, nout)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        w, b = wb[l]
        a = acts[l]
        _, H, W = a.shape
        ap = np.pad(q(a), ((0, 0), (1, 1), (1, 1)))
        gq = q(g)
        gw = np.zeros_like(w)
        for ky in range(3):
            for kx in range(3):
                gw[:, :, ky, kx] = np.einsum("ohw,chw->oc", gq, ap[:, ky:ky + H, kx:kx + W])
        grads[l] = (gw, (g if l == len(layers) - 1 else gq).sum(axis=(1, 2)))
        if l > 0:
            gp = np.pad(gq, ((0, 0), (1, 1), (1, 1)))
            ga = np.zeros_like(a)
            for ky in range(3):
                for kx in range(3):
                    ga += np.einsum("oc,ohw->chw", w[:, :, ky, kx], gp[:, 2 - ky:2 - ky + H, 2 - kx:2 - kx + W])
            g = ga * (a > 0)
    return loss, pack(grads)


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
