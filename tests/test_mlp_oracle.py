"""Pins for the surrogate's CPU oracle (oracle/mlp_oracle.py), all on the CPU.

The double-precision network is checked against finite differences (loss
gradients, forward-mode derivatives, SiLU derivatives, feature derivatives)
and against torch autograd and torch.optim.Adam in float64 (library
routines); the bfloat16 rounding helper against torch's own conversion.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as mo

torch = pytest.importorskip("torch")

NF, H, LAYERS, NOUT = 3, 128, 2, 128


def _net(seed=0):
    rng = np.random.default_rng(seed)
    net = []
    for o, i in mo.layer_shapes(NF, H, LAYERS, NOUT):
        net.append((rng.uniform(-1, 1, (o, i)) * np.sqrt(3.0 / i), rng.uniform(-0.1, 0.1, o)))
    return net


def _pos(B, seed):
    rng = np.random.default_rng(seed)
    return rng.random(B), rng.random(B), rng.random(B)


def test_bf16_matches_torch():
    a = np.random.default_rng(1).normal(size=10000) * 10.0 ** np.random.default_rng(2).integers(-5, 5, 10000)
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(mo.bf16(a), ref)


def test_silu_derivatives():
    z = np.linspace(-8, 8, 401)
    h = 1e-5
    np.testing.assert_allclose(mo.silu_d1(z), (mo.silu(z + h) - mo.silu(z - h)) / (2 * h), atol=1e-9)
    np.testing.assert_allclose(mo.silu_d2(z), (mo.silu_d1(z + h) - mo.silu_d1(z - h)) / (2 * h), atol=1e-8)
    zt = torch.from_numpy(z).requires_grad_(True)
    (g,) = torch.autograd.grad(torch.nn.functional.silu(zt).sum(), zt)
    np.testing.assert_allclose(mo.silu_d1(z), g.numpy(), atol=1e-14)


def test_features_and_derivatives():
    kin = mo.feature_count(NF)
    x, y, z = _pos(7, 3)
    F, dF, d2F = mo.features(x, y, z, NF, kin)
    assert F.shape == (7, kin) and (F[:, 6 * NF:] == 0).all()
    np.testing.assert_allclose(F[:, 0], np.sin(2 * np.pi * x))
    np.testing.assert_allclose(F[:, 2 * NF + 3], np.cos(2 * np.pi * 2 * y))
    h = 1e-6
    e = np.eye(3) * h
    for d in range(3):
        Fp = mo.features(x + e[d, 0], y + e[d, 1], z + e[d, 2], NF, kin)[0]
        Fm = mo.features(x - e[d, 0], y - e[d, 1], z - e[d, 2], NF, kin)[0]
        np.testing.assert_allclose(dF[d], (Fp - Fm) / (2 * h), atol=1e-6)
        np.testing.assert_allclose(d2F[d], (Fp - 2 * F + Fm) / h ** 2, atol=2e-2 * np.abs(d2F[d]).max())
    # periodic in every coordinate
    np.testing.assert_allclose(mo.features(x + 1, y - 2, z + 3, NF, kin)[0], F, atol=1e-12)


def test_backward_matches_torch_autograd():
    net = _net(4)
    kin = mo.feature_count(NF)
    x, y, z = _pos(64, 5)
    F = mo.features(x, y, z, NF, kin)[0]
    tgt = np.random.default_rng(6).normal(size=(64, NOUT))
    loss, grads = mo.loss_and_grads(net, F, tgt, bf16_=False)
    tw = [(torch.from_numpy(W.copy()).requires_grad_(True), torch.from_numpy(b.copy()).requires_grad_(True))
          for W, b in net]
    a = torch.from_numpy(F)
    for W, b in tw[:-1]:
        a = torch.nn.functional.silu(a @ W.T + b)
    out = a @ tw[-1][0].T + tw[-1][1]
    tl = ((out - torch.from_numpy(tgt)) ** 2).mean()
    tl.backward()
    assert abs(tl.item() - loss) < 1e-12
    for (gW, gb), (W, b) in zip(grads, tw):
        np.testing.assert_allclose(gW, W.grad.numpy(), atol=1e-13)
        np.testing.assert_allclose(gb, b.grad.numpy(), atol=1e-13)


def test_backward_matches_finite_differences():
    net = _net(7)
    kin = mo.feature_count(NF)
    x, y, z = _pos(32, 8)
    F = mo.features(x, y, z, NF, kin)[0]
    tgt = np.random.default_rng(9).normal(size=(32, NOUT))
    _, grads = mo.loss_and_grads(net, F, tgt, bf16_=False)
    rng = np.random.default_rng(10)
    h = 1e-6
    for l in range(len(net)):
        W, b = net[l]
        for _ in range(4):
            o, i = rng.integers(0, W.shape[0]), rng.integers(0, min(W.shape[1], 6 * NF))
            Wp, Wm = W.copy(), W.copy()
            Wp[o, i] += h
            Wm[o, i] -= h
            lp = mo.loss_and_grads(net[:l] + [(Wp, b)] + net[l + 1:], F, tgt, False)[0]
            lm = mo.loss_and_grads(net[:l] + [(Wm, b)] + net[l + 1:], F, tgt, False)[0]
            assert abs((lp - lm) / (2 * h) - grads[l][0][o, i]) < 1e-7
        o = rng.integers(0, b.shape[0])
        bp, bm = b.copy(), b.copy()
        bp[o] += h
        bm[o] -= h
        lp = mo.loss_and_grads(net[:l] + [(W, bp)] + net[l + 1:], F, tgt, False)[0]
        lm = mo.loss_and_grads(net[:l] + [(W, bm)] + net[l + 1:], F, tgt, False)[0]
        assert abs((lp - lm) / (2 * h) - grads[l][1][o]) < 1e-7


def test_forward_mode_matches_finite_differences():
    net = _net(11)
    kin = mo.feature_count(NF)
    x, y, z = _pos(16, 12)
    v, g, lap = mo.forward_mode(net, x, y, z, NF, kin, bf16_=False)

    def V(dx, dy, dz):
        return mo.forward(net, mo.features(x + dx, y + dy, z + dz, NF, kin)[0], False)[0]

    np.testing.assert_allclose(v, V(0, 0, 0), atol=1e-13)
    h1, h2 = 1e-6, 1e-4
    e = np.eye(3)
    lap_fd = 0.0
    v0 = V(0, 0, 0)
    for d in range(3):
        gp, gm = V(*(h1 * e[d])), V(*(-h1 * e[d]))
        np.testing.assert_allclose(g[:, d], (gp - gm) / (2 * h1), atol=1e-6 * np.abs(g).max())
        lap_fd = lap_fd + (V(*(h2 * e[d])) - 2 * v0 + V(*(-h2 * e[d]))) / h2 ** 2
    np.testing.assert_allclose(lap, lap_fd, atol=1e-4 * np.abs(lap).max())


def test_adam_matches_torch():
    rng = np.random.default_rng(13)
    p = rng.normal(size=50)
    m1 = np.zeros(50)
    m2 = np.zeros(50)
    tp = torch.from_numpy(p.copy()).requires_grad_(True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 4):
        g = rng.normal(size=50)
        p, m1, m2 = mo.adam_step(p, g, m1, m2, step, 1e-2)
        tp.grad = torch.from_numpy(g.copy())
        opt.step()
        np.testing.assert_allclose(p, tp.detach().numpy(), atol=1e-12)


def test_pack_unpack_roundtrip():
    net = _net(14)
    vec = mo.pack(net)
    back = mo.unpack(vec, NF, H, LAYERS, NOUT)
    for (W, b), (W2, b2) in zip(net, back):
        np.testing.assert_array_equal(W, W2)
        np.testing.assert_array_equal(b, b2)


def _vg_case(B=12, seed=21):
    net = _net(seed)
    kin = mo.feature_count(NF)
    x, y, z = _pos(B, seed + 1)
    F, dF, _ = mo.features(x, y, z, NF, kin)
    rng = np.random.default_rng(seed + 2)
    tv = rng.normal(size=(B, NOUT))
    tg = rng.normal(size=(3, B, NOUT)) * 5.0
    return net, kin, (x, y, z), F, dF, tv, tg


def test_forward_vg_matches_forward_mode():
    """The training form's values and gradients are those of the inference forward mode (and of the plain
    forward pass for the values)."""
    net, kin, (x, y, z), F, dF, tv, tg = _vg_case()
    v, g, *_ = mo.forward_vg(net, F, dF, bf16_=False)
    fv, fg, _ = mo.forward_mode(net, x, y, z, NF, kin, bf16_=False)
    np.testing.assert_allclose(v, fv, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(np.transpose(g, (1, 0, 2)), fg, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(v, mo.forward(net, F, bf16_=False)[0], rtol=1e-12, atol=1e-12)


def test_vg_loss_gradients_finite_differences():
    """Every layer's dW and db against central differences of the value-and-gradient loss."""
    net, kin, _, F, dF, tv, tg = _vg_case()
    lam = 0.3
    loss, grads = mo.loss_and_grads_vg(net, F, dF, tv, tg, lam, bf16_=False)
    rng = np.random.default_rng(5)
    h = 1e-6
    for l, (W, b) in enumerate(net):
        for _ in range(4):
            i, j = rng.integers(W.shape[0]), rng.integers(W.shape[1])
            Wp = [(w.copy(), bb) for w, bb in net]
            Wm = [(w.copy(), bb) for w, bb in net]
            Wp[l][0][i, j] += h
            Wm[l][0][i, j] -= h
            fd = (mo.loss_and_grads_vg(Wp, F, dF, tv, tg, lam, False)[0]
                  - mo.loss_and_grads_vg(Wm, F, dF, tv, tg, lam, False)[0]) / (2 * h)
            assert abs(grads[l][0][i, j] - fd) <= 1e-6 * max(1.0, abs(fd)), (l, i, j, grads[l][0][i, j], fd)
        k = rng.integers(b.shape[0])
        bp = [(w, bb.copy()) for w, bb in net]
        bm = [(w, bb.copy()) for w, bb in net]
        bp[l][1][k] += h
        bm[l][1][k] -= h
        fd = (mo.loss_and_grads_vg(bp, F, dF, tv, tg, lam, False)[0]
              - mo.loss_and_grads_vg(bm, F, dF, tv, tg, lam, False)[0]) / (2 * h)
        assert abs(grads[l][1][k] - fd) <= 1e-6 * max(1.0, abs(fd)), (l, k, grads[l][1][k], fd)


def test_vg_loss_gradients_match_torch_double_backward():
    """The same loss built in torch float64 with the input gradients from autograd (create_graph), then
    differentiated with respect to every parameter: a library routine for the second-order chain rule."""
    net, kin, (x, y, z), F, dF, tv, tg = _vg_case(B=9, seed=31)
    lam = 0.7
    loss, grads = mo.loss_and_grads_vg(net, F, dF, tv, tg, lam, bf16_=False)
    P = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in net]
    r = torch.tensor(np.stack([x, y, z], axis=1), requires_grad=True)
    two_pi = 2 * np.pi
    cols = []
    for d in range(3):
        for k in range(1, NF + 1):
            cols += [torch.sin(two_pi * k * r[:, d]), torch.cos(two_pi * k * r[:, d])]
    Ft = torch.stack(cols, dim=1)
    Ft = torch.cat([Ft, torch.zeros(Ft.shape[0], kin - Ft.shape[1], dtype=Ft.dtype)], dim=1)
    a = Ft
    for W, b in P[:-1]:
        a = torch.nn.functional.silu(a @ W.T + b)
    out = a @ P[-1][0].T + P[-1][1]
    gout = torch.stack([torch.autograd.grad(out[:, n].sum(), r, create_graph=True)[0] for n in range(NOUT)],
                       dim=2)  # [B][3][nout]
    tgt_g = torch.tensor(np.transpose(tg, (1, 0, 2)))
    lt = ((out - torch.tensor(tv)) ** 2).mean() + lam * ((gout - tgt_g) ** 2).mean()
    assert abs(lt.item() - loss) <= 1e-9 * abs(loss)
    flat = torch.autograd.grad(lt, [t for pair in P for t in pair])
    for l in range(len(net)):
        np.testing.assert_allclose(grads[l][0], flat[2 * l].numpy(), rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(grads[l][1], flat[2 * l + 1].numpy(), rtol=1e-8, atol=1e-12)


def test_vg_loss_with_zero_lambda_is_the_value_loss():
    net, kin, _, F, dF, tv, tg = _vg_case()
    loss, grads = mo.loss_and_grads_vg(net, F, dF, tv, tg, 0.0, bf16_=True)
    l2, g2 = mo.loss_and_grads(net, F, tv, bf16_=True)
    assert abs(loss - l2) <= 1e-12 * abs(l2)
    for (a, b), (c, e) in zip(grads, g2):
        np.testing.assert_allclose(a, c, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(b, e, rtol=1e-12, atol=1e-15)
