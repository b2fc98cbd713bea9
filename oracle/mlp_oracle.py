"""CPU oracle of the learned surrogate (periodic Fourier-feature MLP), numpy float64.

TEST INFRASTRUCTURE: only tests/ and the CPU legs of bench.py may import it;
the CUDA library never calls it.

The surrogate is not in arXiv:1611.02665; it stands in for a large B-spline
coefficient table. Definition (it matches include/mlp_surrogate.h):

  features  F_f(r) = sin(2 pi k x_d) for even f, cos(2 pi k x_d) for odd f,
            d = f // (2 nfreq), k = (f % (2 nfreq)) // 2 + 1, zero for
            f >= 6 nfreq (padding up to kin columns);
  hidden    a_l = silu(a_{l-1} W_l^T + b_l), silu(z) = z / (1 + e^-z);
  output    y = a_L W_out^T + b_out;
  loss      mean over batch and outputs of (y - target)^2;
  optimiser Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).

With ``bf16=True`` every tensor the GPU stores in bfloat16 (features,
weights, activations, backward deltas, forward-mode streams) is rounded to
bfloat16 (round to nearest even) at the same point, and everything else is
exact double precision, so the GPU result differs only by float32
accumulation order. With ``bf16=False`` it is the plain double-precision
network, which the CPU tests pin against finite differences and torch
autograd.
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _r(a, on):
    return bf16(a) if on else a


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_d1(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def silu_d2(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s))


def feature_count(nfreq):
    kin = (6 * nfreq + 63) // 64 * 64
    if kin % 128:
        kin += 64
    return kin


def features(x, y, z, nfreq, kin):
    """(F, dF, d2F): F [B, kin]; dF[d], d2F[d] [B, kin] are d/dx_d and d2/dx_d^2."""
    r = [np.asarray(c, dtype=np.float64) for c in (x, y, z)]
    B = r[0].shape[0]
    F = np.zeros((B, kin))
    dF = np.zeros((3, B, kin))
    d2F = np.zeros((3, B, kin))
    for d in range(3):
        cw = r[d] - np.floor(r[d])
        for k in range(1, nfreq + 1):
            w = 2.0 * np.pi * k
            s, c = np.sin(w * cw), np.cos(w * cw)
            fs = d * 2 * nfreq + 2 * (k - 1)
            F[:, fs], F[:, fs + 1] = s, c
            dF[d, :, fs], dF[d, :, fs + 1] = w * c, -w * s
            d2F[d, :, fs], d2F[d, :, fs + 1] = -w * w * s, -w * w * c
    return F, dF, d2F


def layer_shapes(nfreq, hidden, layers, nout):
    kin = feature_count(nfreq)
    shapes = []
    for l in range(layers + 1):
        shapes.append((hidden if l < layers else nout, kin if l == 0 else hidden))
    return shapes


def unpack(vec, nfreq, hidden, layers, nout):
    """[(W [out][in], b [out])] from the packed parameter vector (layer by layer, W then b)."""
    out, off = [], 0
    vec = np.asarray(vec, dtype=np.float64)
    for o, i in layer_shapes(nfreq, hidden, layers, nout):
        W = vec[off:off + o * i].reshape(o, i)
        off += o * i
        b = vec[off:off + o]
        off += o
        out.append((W, b))
    assert off == vec.size
    return out


def pack(layers_):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers_])


def forward(net, F, bf16_=True):
    """(y, zs, acts): output, hidden pre-activations, inputs of every linear layer."""
    a = _r(F, bf16_)
    zs, acts = [], [a]
    for W, b in net[:-1]:
        z = a @ _r(W, bf16_).T + b
        a = _r(silu(z), bf16_)
        zs.append(z)
        acts.append(a)
    W, b = net[-1]
    return a @ _r(W, bf16_).T + b, zs, acts


def loss_and_grads(net, F, target, bf16_=True):
    """(loss, [(dW, db)]) of the mean squared error, by the chain rule layer by layer."""
    y, zs, acts = forward(net, F, bf16_)
    B, nout = y.shape
    diff = y - target
    loss = float(np.mean(diff * diff))
    d = _r(2.0 * diff / (B * nout), bf16_)
    grads = [None] * len(net)
    for l in range(len(net) - 1, -1, -1):
        W, _ = net[l]
        grads[l] = (d.T @ acts[l], d.sum(axis=0))
        if l > 0:
            d = _r((d @ _r(W, bf16_)) * silu_d1(zs[l - 1]), bf16_)
    return loss, grads


def forward_mode(net, x, y, z, nfreq, kin, bf16_=True):
    """(v, g [B][3][nout], lap): values, gradients and Laplacians by forward-mode propagation."""
    F, dF, d2F = features(x, y, z, nfreq, kin)
    v = _r(F, bf16_)
    g = [_r(dF[d], bf16_) for d in range(3)]
    s = [_r(d2F[d], bf16_) for d in range(3)]
    for W, b in net[:-1]:
        Wr = _r(W, bf16_)
        zv = v @ Wr.T + b
        zg = [gd @ Wr.T for gd in g]
        zs = [sd @ Wr.T for sd in s]
        d1, d2 = silu_d1(zv), silu_d2(zv)
        v = _r(silu(zv), bf16_)
        s = [_r(d2 * zg[d] * zg[d] + d1 * zs[d], bf16_) for d in range(3)]
        g = [_r(d1 * zg[d], bf16_) for d in range(3)]
    W, b = net[-1]
    Wr = _r(W, bf16_)
    out_v = v @ Wr.T + b
    out_g = np.stack([gd @ Wr.T for gd in g], axis=1)
    out_l = sum(sd @ Wr.T for sd in s)
    return out_v, out_g, out_l


def adam_step(params, grads, m1, m2, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update (step counts from 1); returns (params, m1, m2)."""
    m1 = b1 * m1 + (1.0 - b1) * grads
    m2 = b2 * m2 + (1.0 - b2) * grads * grads
    mh = m1 / (1.0 - b1 ** step)
    vh = m2 / (1.0 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m1, m2


def forward_vg(net, F, dF, bf16_=True):
    """Forward mode over values and the three first derivatives only (the training form).

    Returns (v, g, zs, zgs, acts, actgs): outputs v [B][nout] and g [3][B][nout]; per hidden layer the
    pre-activation z and its tangents zg[d] (saved in float32 on the GPU, exact here); the inputs of every
    linear layer, a and its tangents ag[d] (bfloat16 on the GPU). Tangents carry no bias:
    z = a W^T + b, zg_d = ag_d W^T, a' = silu(z), ag'_d = silu'(z) zg_d.
    """
    a = _r(F, bf16_)
    ag = [_r(dF[d], bf16_) for d in range(3)]
    zs, zgs, acts, actgs = [], [], [a], [ag]
    for W, b in net[:-1]:
        Wr = _r(W, bf16_)
        z = a @ Wr.T + b
        zg = [g @ Wr.T for g in ag]
        d1 = silu_d1(z)
        a = _r(silu(z), bf16_)
        ag = [_r(d1 * g, bf16_) for g in zg]
        zs.append(z)
        zgs.append(zg)
        acts.append(a)
        actgs.append(ag)
    W, b = net[-1]
    Wr = _r(W, bf16_)
    return a @ Wr.T + b, np.stack([g @ Wr.T for g in ag]), zs, zgs, acts, actgs


def loss_and_grads_vg(net, F, dF, tv, tg, lam, bf16_=True):
    """(loss, [(dW, db)]) of the value-and-gradient loss

        L = mean((v - tv)^2) + lam * mean((g - tg)^2)

    (the first mean over positions and outputs, the second over positions, the 3 axes and outputs; tg is
    [3][B][nout]), by reverse mode through the forward-mode network, layer by layer.

    A hidden layer maps (z, zg_d) to (a, ag_d) = (silu(z), silu'(z) zg_d), so given the loss gradients
    (da, dag_d) of its outputs:  dzg_d = silu'(z) dag_d  and  dz = silu'(z) da + silu''(z) sum_d zg_d dag_d.
    A linear layer (z = a W^T + b, zg_d = ag_d W^T) gives dW = dz^T a + sum_d dzg_d^T ag_d, db = sum dz,
    da = dz W, dag_d = dzg_d W.
    """
    v, g, zs, zgs, acts, actgs = forward_vg(net, F, dF, bf16_)
    B, nout = v.shape
    dv_ = v - tv
    dg_ = g - tg
    loss = float(np.mean(dv_ * dv_) + lam * np.mean(dg_ * dg_))
    d = _r(2.0 * dv_ / (B * nout), bf16_)
    dgr = [_r(2.0 * lam * dg_[k] / (3 * B * nout), bf16_) for k in range(3)]
    grads = [None] * len(net)
    for l in range(len(net) - 1, -1, -1):
        W, _ = net[l]
        dW = d.T @ acts[l] + sum(dgr[k].T @ actgs[l][k] for k in range(3))
        grads[l] = (dW, d.sum(axis=0))
        if l > 0:
            Wr = _r(W, bf16_)
            da = d @ Wr
            dag = [x @ Wr for x in dgr]
            z, zg = zs[l - 1], zgs[l - 1]
            d1, d2 = silu_d1(z), silu_d2(z)
            d = _r(d1 * da + d2 * sum(zg[k] * dag[k] for k in range(3)), bf16_)
            dgr = [_r(d1 * dag[k], bf16_) for k in range(3)]
    return loss, grads
