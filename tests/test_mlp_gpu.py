"""GPU checks of the learned surrogate through its C ABI.

- the tcgen05 BF16 GEMM against a float64 matmul of the same bf16 inputs;
- one training step's loss and gradients against the CPU oracle
  (oracle/mlp_oracle.py, which mirrors the GPU's bfloat16 rounding points);
- a loss summed in a fixed order, and gradients after an Adam step (the
  bf16 weight copies follow the update);
- the Adam update, inference values and forward-mode gradients/Laplacians
  against the oracle; save/load;
- training on spline values produced by the spline kernels, and what the
  trained network gains over the spline it replaces at equal memory.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from paper_1611_02665_gb300 import capi, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


GEMM_CASES = [(128, 128, 64, 1), (128, 256, 64, 1), (300, 256, 512, 1), (1000, 384, 192, 1), (4096, 512, 512, 1),
              (512, 512, 4096, 7), (512, 128, 1024, 4), (77, 128, 128, 2)]
# CTA pairs (256 x 256 tiles on clusters of two): N a multiple of 256, no K split; ragged M down to a pair whose
# second CTA has no rows
PAIR_CASES = [(128, 256, 64, 1), (77, 256, 128, 1), (300, 256, 512, 1), (1000, 512, 192, 1), (4096, 512, 512, 1),
              (8192, 1024, 1024, 1)]


@pytest.mark.parametrize("M,N,K,splitk,kernel", [c + (capi.GEMM_AUTO,) for c in GEMM_CASES] +
                         [c + (capi.GEMM_ONE_CTA,) for c in GEMM_CASES[:5]] +
                         [c + (capi.GEMM_CTA_PAIR,) for c in PAIR_CASES] +
                         [c + (capi.GEMM_TWO_CTAS,) for c in GEMM_CASES])
def test_gemm_matches_float64_matmul(M, N, K, splitk, kernel):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A = (torch.rand((M, K), generator=g, device="cuda") * 2 - 1).to(torch.bfloat16)
    B = (torch.rand((N, K), generator=g, device="cuda") * 2 - 1).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), device="cuda")
    capi.mlp_gemm_bf16_ex(A, B, C, M, N, K, N, splitk, kernel)
    torch.cuda.synchronize()
    ref = A.double() @ B.double().T
    # products of bf16 values are exact in float32: only the float32 summation order differs
    assert _rel(C.cpu().numpy(), ref.cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("kernel", [capi.GEMM_ONE_CTA, capi.GEMM_CTA_PAIR, capi.GEMM_TWO_CTAS])
@pytest.mark.parametrize("M,N,ldc", [(300, 256, 268), (77, 128, 132), (4096, 512, 516), (33, 384, 384),
                                     (130, 512, 520)])
def test_gemm_writes_only_its_rows_and_columns(M, N, ldc, kernel):
    """The output leaves through TMA stores of 32-row boxes: rows past M (the ragged last box, and rows of
    the buffer below the matrix) and the row padding past N stay untouched."""
    K = 192
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N)
    A = (torch.rand((M, K), generator=g, device="cuda") * 2 - 1).to(torch.bfloat16)
    B = (torch.rand((N, K), generator=g, device="cuda") * 2 - 1).to(torch.bfloat16)
    buf = torch.full((M + 40, ldc), float("nan"), device="cuda")
    capi.mlp_gemm_bf16_ex(A, B, buf, M, N, K, ldc, 1, kernel)
    torch.cuda.synchronize()
    ref = (A.double() @ B.double().T).cpu().numpy()
    out = buf.cpu().numpy()
    assert _rel(out[:M, :N], ref) <= 1e-5
    assert np.isnan(out[:M, N:]).all() and np.isnan(out[M:]).all()


SMALL = dict(nfreq=4, hidden=128, layers=2, nout=128)
# layers 256 wide, run on CTA pairs (mlp_set_gemm_kernel 2) at these small sizes
WIDE = dict(nfreq=4, hidden=256, layers=2, nout=256)
# (shape, GEMM kernel) of the oracle checks: the library's choice on SMALL, CTA pairs and two CTAs per SM on WIDE
NETS = [pytest.param(SMALL, capi.GEMM_AUTO, id="small"), pytest.param(WIDE, capi.GEMM_CTA_PAIR, id="wide-pairs"),
        pytest.param(WIDE, capi.GEMM_TWO_CTAS, id="wide-two-ctas")]


def _surrogate(shape=SMALL, seed=3, kernel=0):
    s = capi.Surrogate(shape["nfreq"], shape["hidden"], shape["layers"], shape["nout"])
    capi.mlp_init(s.h, seed)
    capi.mlp_set_gemm_kernel(s.h, kernel)
    return s


def _params(s):
    p = np.zeros(capi.mlp_param_count(s.h), np.float32)
    capi.mlp_get_params(s.h, p)
    return p


def _net(p, shape=SMALL):
    return mo.unpack(p.astype(np.float64), shape["nfreq"], shape["hidden"], shape["layers"], shape["nout"])


@pytest.mark.parametrize("shape,kernel", NETS)
def test_train_step_loss_and_gradients_match_oracle(shape, kernel):
    B = 256
    with _surrogate(shape, kernel=kernel) as s:
        p = _params(s)
        x, y, z = inputs.uniform_positions(B, seed=31)
        tgt = np.random.default_rng(32).normal(size=(B, shape["nout"])).astype(np.float32)
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        loss = torch.zeros(1, device="cuda")
        capi.mlp_train_step(s.h, B, dx, dy, dz, torch.from_numpy(tgt).cuda(), shape["nout"], 0.0, loss)
        torch.cuda.synchronize()
        grads = np.zeros_like(p)
        capi.mlp_get_grads(s.h, grads)
        np.testing.assert_array_equal(_params(s), p)  # lr = 0 leaves the weights alone
    kin = mo.feature_count(shape["nfreq"])
    F = mo.features(x, y, z, shape["nfreq"], kin)[0]
    loss_ref, g_ref = mo.loss_and_grads(_net(p, shape), F, tgt.astype(np.float64), bf16_=True)
    assert abs(loss.item() - loss_ref) <= 1e-4 * loss_ref
    got = mo.unpack(grads.astype(np.float64), **shape)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(got, g_ref)):
        assert _rel(gW, rW) <= 1e-2, f"layer {l} dW"
        assert _rel(gb, rb) <= 1e-2, f"layer {l} db"


def test_loss_is_reproducible_and_copies_follow_adam():
    """The loss is summed in a fixed order (the same bits on every call), and after an Adam step the
    gradients of the next step match the oracle at the updated weights: the bf16 W and W^T copies that
    the forward and backward GEMMs read were rewritten from the new master weights."""
    B = 2048
    with _surrogate(seed=9) as s:
        x, y, z = inputs.uniform_positions(B, seed=91)
        tgt = np.random.default_rng(92).normal(size=(B, SMALL["nout"])).astype(np.float32)
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        dt = torch.from_numpy(tgt).cuda()
        losses = []
        for _ in range(3):
            loss = torch.zeros(1, device="cuda")
            capi.mlp_train_step(s.h, B, dx, dy, dz, dt, SMALL["nout"], 0.0, loss)
            torch.cuda.synchronize()
            losses.append(loss.item())
        assert losses[0] == losses[1] == losses[2]
        capi.mlp_train_step(s.h, B, dx, dy, dz, dt, SMALL["nout"], 3e-3)
        torch.cuda.synchronize()
        p = _params(s)
        loss = torch.zeros(1, device="cuda")
        capi.mlp_train_step(s.h, B, dx, dy, dz, dt, SMALL["nout"], 0.0, loss)
        torch.cuda.synchronize()
        grads = np.zeros_like(p)
        capi.mlp_get_grads(s.h, grads)
    kin = mo.feature_count(SMALL["nfreq"])
    F = mo.features(x, y, z, SMALL["nfreq"], kin)[0]
    loss_ref, g_ref = mo.loss_and_grads(_net(p), F, tgt.astype(np.float64), bf16_=True)
    assert abs(loss.item() - loss_ref) <= 1e-4 * loss_ref
    assert loss.item() < losses[0]
    got = mo.unpack(grads.astype(np.float64), **SMALL)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(got, g_ref)):
        assert _rel(gW, rW) <= 1e-2, f"layer {l} dW"
        assert _rel(gb, rb) <= 1e-2, f"layer {l} db"


def test_adam_update_matches_oracle():
    B = 128
    with _surrogate(seed=5) as s:
        p0 = _params(s)
        x, y, z = inputs.uniform_positions(B, seed=51)
        tgt = torch.from_numpy(np.random.default_rng(52).normal(size=(B, 128)).astype(np.float32)).cuda()
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        capi.mlp_train_step(s.h, B, dx, dy, dz, tgt, 128, 1e-3)
        torch.cuda.synchronize()
        g = np.zeros_like(p0)
        capi.mlp_get_grads(s.h, g)
        p1 = _params(s)
    ref, _, _ = mo.adam_step(p0.astype(np.float64), g.astype(np.float64), 0.0, 0.0, 1, 1e-3)
    np.testing.assert_allclose(p1, ref, atol=2e-6)


@pytest.mark.parametrize("shape,kernel", NETS + [pytest.param(SMALL, capi.GEMM_ONE_CTA, id="small-per-layer")])
def test_inference_and_forward_mode_match_oracle(shape, kernel):
    npos = 200
    with _surrogate(shape, seed=7, kernel=kernel) as s:
        p = _params(s)
        x, y, z = inputs.uniform_positions(npos, seed=71)
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        ld = shape["nout"] + 4
        v = torch.full((npos, ld), 7.0, device="cuda")
        capi.mlp_eval_v(s.h, npos, dx, dy, dz, v, ld)
        v2 = torch.zeros((npos, ld), device="cuda")
        g = torch.zeros((npos, 3, ld), device="cuda")
        lap = torch.zeros((npos, ld), device="cuda")
        capi.mlp_eval_vgl(s.h, npos, dx, dy, dz, v2, g, lap, ld)
        torch.cuda.synchronize()
    n = shape["nout"]
    kin = mo.feature_count(shape["nfreq"])
    rv, rg, rl = mo.forward_mode(_net(p, shape), x, y, z, shape["nfreq"], kin, bf16_=True)
    assert (v[:, n:] == 7.0).all()
    assert _rel(v[:, :n].cpu().numpy(), rv) <= 1e-2
    assert _rel(v2[:, :n].cpu().numpy(), rv) <= 1e-2
    assert _rel(g[:, :, :n].cpu().numpy(), rg) <= 2e-2
    assert _rel(lap[:, :n].cpu().numpy(), rl) <= 3e-2


def _infer_v(shape, kernel, npos, seed, pseed, ld=None):
    ld = ld or shape["nout"]
    with _surrogate(shape, seed=seed, kernel=kernel) as s:
        p = _params(s)
        x, y, z = inputs.uniform_positions(npos, seed=pseed)
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        v = torch.full((npos, ld), 7.0, device="cuda")
        capi.mlp_eval_v(s.h, npos, dx, dy, dz, v, ld)
        torch.cuda.synchronize()
        assert capi.mlp_device_status(s.h) == 0
    return p, (x, y, z), v.cpu().numpy()


@pytest.mark.parametrize("shape,kernel", [
    pytest.param(dict(nfreq=8, hidden=512, layers=3, nout=512), capi.GEMM_CTA_PAIR, id="wide-pairs"),
    pytest.param(dict(nfreq=8, hidden=512, layers=3, nout=512), capi.GEMM_TWO_CTAS, id="wide-two-ctas"),
    pytest.param(dict(nfreq=8, hidden=512, layers=3, nout=512), capi.GEMM_AUTO, id="wide-256-tiles")])
def test_inference_at_full_width(shape, kernel):
    """V inference of 12,001 positions through the 512-wide network: 128 x 256 tiles over the whole GPU
    (or 256 x 256 CTA-pair tiles), a ragged last row block; the values equal those of the one-CTA kernels
    (bit for bit with the same tiles, to FP32 summation order on pairs) and match the oracle on a sample."""
    npos = 12001
    n = shape["nout"]
    p, (x, y, z), v = _infer_v(shape, kernel, npos, seed=17, pseed=171)
    p2, _, v_ref = _infer_v(shape, capi.GEMM_ONE_CTA, npos, seed=17, pseed=171)
    np.testing.assert_array_equal(p, p2)
    if kernel == capi.GEMM_AUTO:
        np.testing.assert_array_equal(v, v_ref)
    else:
        assert _rel(v, v_ref) <= 1e-5
    rows = np.unique(np.concatenate([np.arange(3), np.random.default_rng(5).choice(npos, 40, replace=False),
                                     [npos - 1]]))
    kin = mo.feature_count(shape["nfreq"])
    rv = mo.forward_mode(_net(p, shape), x[rows], y[rows], z[rows], shape["nfreq"], kin, bf16_=True)[0]
    assert _rel(v[rows, :n], rv) <= 1e-2


@pytest.mark.parametrize("shape,kernel", NETS)
@pytest.mark.parametrize("npos", [1, 5, 6, 7, 13, 37])
def test_forward_mode_partial_row_groups(npos, shape, kernel):
    """Forward mode packs 6 positions per 32 rows: position counts that leave a group partly empty write
    exactly their own outputs (the columns past nout and the rows past npos keep their fill)."""
    with _surrogate(shape, seed=7, kernel=kernel) as s:
        p = _params(s)
        x, y, z = inputs.uniform_positions(npos, seed=72)
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        n = shape["nout"]
        ld = n + 4
        v = torch.full((npos + 2, ld), 7.0, device="cuda")
        g = torch.full((npos + 2, 3, ld), 7.0, device="cuda")
        lap = torch.full((npos + 2, ld), 7.0, device="cuda")
        capi.mlp_eval_vgl(s.h, npos, dx, dy, dz, v, g, lap, ld)
        torch.cuda.synchronize()
    kin = mo.feature_count(shape["nfreq"])
    rv, rg, rl = mo.forward_mode(_net(p, shape), x, y, z, shape["nfreq"], kin, bf16_=True)
    assert _rel(v[:npos, :n].cpu().numpy(), rv) <= 1e-2
    assert _rel(g[:npos, :, :n].cpu().numpy(), rg) <= 2e-2
    assert _rel(lap[:npos, :n].cpu().numpy(), rl) <= 3e-2
    for buf in (v, g, lap):
        assert (buf[..., n:] == 7.0).all()
        assert (buf[npos:] == 7.0).all()


def test_save_load_roundtrip(tmp_path):
    npos = 64
    x, y, z = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(npos, seed=81))
    path = tmp_path / "net.bin"
    with _surrogate(seed=9) as s:
        v1 = torch.zeros((npos, 128), device="cuda")
        capi.mlp_eval_v(s.h, npos, x, y, z, v1, 128)
        capi.mlp_save(s.h, path)
    with capi.Surrogate(**{"nfreq": 4, "hidden": 128, "layers": 2, "nout": 128}) as s2:
        capi.mlp_load(s2.h, path)
        v2 = torch.zeros((npos, 128), device="cuda")
        capi.mlp_eval_v(s2.h, npos, x, y, z, v2, 128)
        torch.cuda.synchronize()
    assert torch.equal(v1, v2)
    with capi.Surrogate(4, 256, 2, 128) as s3:
        with pytest.raises(capi.BsplineError):
            capi.mlp_load(s3.h, path)


def _spline_values(table, x, y, z, N):
    v = torch.empty((x.shape[0], N), device="cuda")
    capi.bspline_eval_v(table.h, x.shape[0], x, y, z, v, N)
    return v


def test_training_gain_over_equal_memory_spline():
    """Train on spline values from the spline kernel; compare with the spline that fits the same memory.

    Orbitals: 128 smooth plane-wave orbitals on a 24^3 grid (wavevectors up to 2).
    The network (8 frequencies, 3 x 256 SiLU, 128 outputs) holds ~0.2 M bf16 weights
    (0.4 MB); a 6^3-grid spline of the same orbitals (coefficients sampled at its
    knots) needs 9^3 x 128 x 4 B = 0.37 MB. The network must be the more accurate.
    """
    grid, N = (24, 24, 24), 128
    coef = inputs.plane_wave_coefs(grid, N, seed=61, device="cuda", nmodes=8, kmax=2, noise=0.0)
    fine = capi.Table(grid, N, capi.F32)
    capi.bspline_set_coefs(fine.h, coef)
    # the equal-memory spline: the same orbitals sampled at a 6^3 grid's knots
    cg = 6
    kk = (torch.arange(cg, device="cuda", dtype=torch.float64) / cg)
    X, Y, Z = torch.meshgrid(kk, kk, kk, indexing="ij")
    coarse_coef = _spline_values(fine, X.reshape(-1).contiguous(), Y.reshape(-1).contiguous(),
                                 Z.reshape(-1).contiguous(), N).reshape(cg, cg, cg, N)
    coarse = capi.Table((cg, cg, cg), N, capi.F32)
    capi.bspline_set_coefs(coarse.h, coarse_coef.contiguous())

    ntrain, B, steps = 1 << 16, 1024, 1500
    tx, ty, tz = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(ntrain, seed=62))
    ttarget = _spline_values(fine, tx, ty, tz, N)
    hx, hy, hz = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(4096, seed=63))
    href = _spline_values(fine, hx, hy, hz, N)

    shape = dict(nfreq=8, hidden=256, layers=3, nout=N)
    with _surrogate(shape, seed=11) as s:
        loss = torch.zeros(1, device="cuda")
        first = None
        for step in range(steps):
            lo = (step * B) % ntrain
            lr = 2e-3 * 0.5 * (1 + np.cos(np.pi * step / steps)) + 2e-5
            capi.mlp_train_step(s.h, B, tx[lo:lo + B], ty[lo:lo + B], tz[lo:lo + B], ttarget[lo:lo + B], N, lr,
                                loss)
            if step == 0:
                torch.cuda.synchronize()
                first = loss.item()
        torch.cuda.synchronize()
        last = loss.item()
        vn = torch.empty((4096, N), device="cuda")
        capi.mlp_eval_v(s.h, 4096, hx, hy, hz, vn, N)
        nbytes_net = 2 * (capi.mlp_param_count(s.h))
    vc = _spline_values(coarse, hx, hy, hz, N)
    torch.cuda.synchronize()
    rms = lambda e: float(torch.sqrt((e ** 2).mean()) / torch.sqrt((href ** 2).mean()))
    err_net, err_coarse = rms(vn - href), rms(vc - href)
    print(f"loss {first:.3e} -> {last:.3e}; held-out rel RMS: network {err_net:.3e}, "
          f"6^3 spline {err_coarse:.3e}; network {nbytes_net / 1e6:.2f} MB, coarse spline "
          f"{9 ** 3 * N * 4 / 1e6:.2f} MB, fine spline {27 ** 3 * N * 4 / 1e6:.2f} MB")
    assert last < 0.05 * first
    assert nbytes_net <= 1.1 * 9 ** 3 * N * 4
    assert err_net < err_coarse
    fine.close()
    coarse.close()


@pytest.mark.parametrize("shape,kernel", NETS)
@pytest.mark.parametrize("B,lam", [(96, 0.2), (128, 3.0)])
def test_train_step_vg_loss_and_gradients_match_oracle(B, lam, shape, kernel):
    """Training on values and gradients (4 rows per position): the loss and every layer's gradients
    against the oracle's reverse mode through the forward mode (same bfloat16 rounding points)."""
    n = shape["nout"]
    with _surrogate(shape, seed=13, kernel=kernel) as s:
        p = _params(s)
        x, y, z = inputs.uniform_positions(B, seed=131)
        rng = np.random.default_rng(132)
        tv = rng.normal(size=(B, n)).astype(np.float32)
        tg = (rng.normal(size=(B, 3, n)) * 5.0).astype(np.float32)
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        loss = torch.zeros(1, device="cuda")
        capi.mlp_train_step_vg(s.h, B, dx, dy, dz, torch.from_numpy(tv).cuda(), torch.from_numpy(tg).cuda(), n,
                               lam, 0.0, loss)
        torch.cuda.synchronize()
        grads = np.zeros_like(p)
        capi.mlp_get_grads(s.h, grads)
        np.testing.assert_array_equal(_params(s), p)
    kin = mo.feature_count(shape["nfreq"])
    F, dF, _ = mo.features(x, y, z, shape["nfreq"], kin)
    loss_ref, g_ref = mo.loss_and_grads_vg(_net(p, shape), F, dF, tv.astype(np.float64),
                                           np.transpose(tg, (1, 0, 2)).astype(np.float64), lam, bf16_=True)
    assert abs(loss.item() - loss_ref) <= 1e-4 * loss_ref
    got = mo.unpack(grads.astype(np.float64), **shape)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(got, g_ref)):
        assert _rel(gW, rW) <= 1e-2, f"layer {l} dW"
        assert _rel(gb, rb) <= 1e-2, f"layer {l} db"


def test_train_step_vg_without_gradient_term_is_the_value_step():
    """lambda = 0: the derivative rows carry zero loss gradient, so the step is the value-loss step on the
    same positions (up to the float32 order of the split-K sums over the longer batch)."""
    B, n = 256, SMALL["nout"]
    x, y, z = inputs.uniform_positions(B, seed=141)
    rng = np.random.default_rng(142)
    tv = torch.from_numpy(rng.normal(size=(B, n)).astype(np.float32)).cuda()
    tg = torch.from_numpy(rng.normal(size=(B, 3, n)).astype(np.float32)).cuda()
    dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
    out = []
    for vg in (False, True):
        with _surrogate(seed=14) as s:
            loss = torch.zeros(1, device="cuda")
            if vg:
                capi.mlp_train_step_vg(s.h, B, dx, dy, dz, tv, tg, n, 0.0, 0.0, loss)
            else:
                capi.mlp_train_step(s.h, B, dx, dy, dz, tv, n, 0.0, loss)
            torch.cuda.synchronize()
            gr = np.zeros(capi.mlp_param_count(s.h), np.float32)
            capi.mlp_get_grads(s.h, gr)
            out.append((loss.item(), gr))
    assert abs(out[0][0] - out[1][0]) <= 1e-5 * out[0][0]
    assert _rel(out[1][1], out[0][1]) <= 1e-5


def test_train_step_vg_argument_errors():
    with _surrogate() as s:
        d = torch.zeros(64, dtype=torch.float64, device="cuda")
        t = torch.zeros((64, 3, 128), device="cuda")
        for bad in (dict(batch=48), dict(lam=-1.0), dict(lam=float("nan")), dict(ld=64)):
            args = dict(batch=64, lam=0.1, ld=128)
            args.update(bad)
            with pytest.raises(capi.BsplineError) as e:
                capi.mlp_train_step_vg(s.h, args["batch"], d, d, d, t, t, args["ld"], args["lam"], 0.0)
            assert e.value.status == capi.ERR_ARG


def test_gradient_term_gain_on_spline_gradients():
    """Train the same network on spline targets from the spline kernels, once on values only and once with
    the gradient term (the spline's VGL gradients): on held-out positions the gradient-trained network's
    gradient and Laplacian errors against the spline are the smaller ones, at a comparable value error."""
    grid, N = (24, 24, 24), 128
    coef = inputs.plane_wave_coefs(grid, N, seed=61, device="cuda", nmodes=8, kmax=2, noise=0.0)
    spline = capi.Table(grid, N, capi.F32)
    capi.bspline_set_coefs(spline.h, coef)
    ntrain, B, steps = 1 << 15, 512, 1200
    tx, ty, tz = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(ntrain, seed=62))
    tv, tg, tl = spline.outputs(capi.VGL, ntrain)
    spline.eval(capi.VGL, tx, ty, tz, tv, tg, tl)
    P = 4096
    hx, hy, hz = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(P, seed=63))
    hv, hg, hl = spline.outputs(capi.VGL, P)
    spline.eval(capi.VGL, hx, hy, hz, hv, hg, hl)
    lam = float((tv ** 2).mean() / (tg ** 2).mean())  # both terms of the loss on the same scale
    shape = dict(nfreq=8, hidden=256, layers=3, nout=N)
    errs = {}
    for name, vg in (("values", False), ("values+gradients", True)):
        with _surrogate(shape, seed=11) as s:
            for step in range(steps):
                lo = (step * B) % ntrain
                sl = slice(lo, lo + B)
                lr = 2e-3 * 0.5 * (1 + np.cos(np.pi * step / steps)) + 2e-5
                if vg:
                    capi.mlp_train_step_vg(s.h, B, tx[sl], ty[sl], tz[sl], tv[sl], tg[sl], N, lam, lr)
                else:
                    capi.mlp_train_step(s.h, B, tx[sl], ty[sl], tz[sl], tv[sl], N, lr)
            mv, mg, ml = spline.outputs(capi.VGL, P)
            capi.mlp_eval_vgl(s.h, P, hx, hy, hz, mv, mg, ml, N)
            torch.cuda.synchronize()
        rms = lambda a, b: float(torch.sqrt(((a - b) ** 2).mean()) / torch.sqrt((b ** 2).mean()))
        errs[name] = (rms(mv, hv), rms(mg, hg), rms(ml, hl))
    spline.close()
    print(f"held-out rel RMS (v, g, l): {errs}")
    (v0, g0, l0), (v1, g1, l1) = errs["values"], errs["values+gradients"]
    assert g1 < 0.7 * g0 and l1 < l0
    assert v1 < 2.0 * v0


def test_training_workspace_across_batch_sizes():
    """One handle trained with a large batch, then smaller ones and the 4-row form (the workspace is
    sized by the largest and reused): each step's loss and gradients still match the oracle (the loss
    kernel's block counter must not depend on the batch)."""
    n = SMALL["nout"]
    kin = mo.feature_count(SMALL["nfreq"])
    rng = np.random.default_rng(151)
    with _surrogate(seed=15) as s:
        for B, vg in ((2048, False), (256, False), (128, True), (512, False), (96, True)):
            x, y, z = inputs.uniform_positions(B, seed=152 + B)
            tv = rng.normal(size=(B, n)).astype(np.float32)
            tg = rng.normal(size=(B, 3, n)).astype(np.float32)
            dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
            p = _params(s)
            loss = torch.full((1,), float("nan"), device="cuda")
            if vg:
                capi.mlp_train_step_vg(s.h, B, dx, dy, dz, torch.from_numpy(tv).cuda(), torch.from_numpy(tg).cuda(),
                                       n, 0.5, 0.0, loss)
            else:
                capi.mlp_train_step(s.h, B, dx, dy, dz, torch.from_numpy(tv).cuda(), n, 0.0, loss)
            torch.cuda.synchronize()
            grads = np.zeros_like(p)
            capi.mlp_get_grads(s.h, grads)
            F, dF, _ = mo.features(x, y, z, SMALL["nfreq"], kin)
            if vg:
                lref, gref = mo.loss_and_grads_vg(_net(p), F, dF, tv.astype(np.float64),
                                                  np.transpose(tg, (1, 0, 2)).astype(np.float64), 0.5, bf16_=True)
            else:
                lref, gref = mo.loss_and_grads(_net(p), F, tv.astype(np.float64), bf16_=True)
            assert abs(loss.item() - lref) <= 1e-4 * lref, (B, vg, loss.item(), lref)
            for l, ((gW, gb), (rW, rb)) in enumerate(zip(mo.unpack(grads.astype(np.float64), **SMALL), gref)):
                assert _rel(gW, rW) <= 1e-2 and _rel(gb, rb) <= 1e-2, (B, vg, l)
