"""U-Net layer kernels (BF16 tensor-core convolutions, FP32 weight gradients) against the
FP64 oracle.  Inputs and weights are rounded to BF16 first and the oracle runs on the
rounded values, so the remaining difference is the kernels' own: BF16 rounding of each
output (relative 2^-9, tolerance 4e-3 per layer) and FP32 accumulation."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import eptv_oracle as O
from oracle import unet_oracle as U
from paper_1009_2288_b300 import eptv as E
from paper_1009_2288_b300 import inputs as I
from paper_1009_2288_b300 import learned as L

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
BF = torch.bfloat16


def bf(a):
    """Round float64 numpy to bf16 (round to nearest even) and back."""
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(BF).double().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def nhwc(a_chw, stride=None, off=0):
    """[C][H][W] numpy -> torch bf16 [1][H][W][stride] with channels at [off, off+C)."""
    C, H, W = a_chw.shape
    t = torch.zeros(1, H, W, stride or C, dtype=BF, device=DEV)
    t[0, :, :, off:off + C] = torch.tensor(
        np.ascontiguousarray(np.asarray(a_chw, dtype=np.float32).transpose(1, 2, 0))).to(DEV).to(BF)
    return t


def chw(t, off=0, c=None):
    a = t[0].float().cpu().numpy()
    c = c or a.shape[2] - off
    return a[:, :, off:off + c].transpose(2, 0, 1).astype(np.float64)


def gpu_w(W):
    """[co][ci][3][3] -> [co][9][ci] float32 CUDA tensor."""
    co, ci = W.shape[:2]
    # (copy to a contiguous array first: a strided numpy view is not copied faithfully by
    # torch.tensor(..., device=cuda) in this environment)
    return torch.tensor(np.ascontiguousarray(np.asarray(W, np.float32).transpose(0, 2, 3, 1).reshape(co, 9, ci))).to(DEV)


PAIRS = [(16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (48, 16), (32, 16), (64, 32),
         (32, 96), (16, 48)]


@pytest.mark.parametrize("cin,cout", PAIRS)
def test_conv3x3_forward_matches_oracle(cin, cout):
    rng = np.random.Generator(np.random.PCG64(cin * 100 + cout))
    H, W = 12, 20                                   # ragged against the 8 x 16 tiles
    x = bf(rng.standard_normal((cin, H, W)))
    Wt = bf(rng.standard_normal((cout, cin, 3, 3)) / np.sqrt(9 * cin))
    b = rng.standard_normal(cout).astype(np.float32).astype(np.float64)
    want = np.maximum(U.conv3x3(x, Wt, b), 0.0)
    xs = cin + 8                                    # read a channel slice at offset 8
    xt = nhwc(x, stride=xs, off=8)
    wf = torch.empty(cout, 9, cin, dtype=BF, device=DEV)
    E.eptv_unet_weights_to_bf16(gpu_w(Wt), cout, cin, wf, None)
    y = torch.zeros(1, H, W, cout + 4, dtype=BF, device=DEV)
    E.eptv_unet_conv3x3(xt, 8, cin, wf, torch.tensor(b, dtype=torch.float32, device=DEV), cout, y, 2, True)
    torch.cuda.synchronize()
    got = chw(y, 2, cout)
    assert rel(got, want) < 4e-3
    assert float(y[..., :2].abs().max()) == 0.0 and float(y[..., cout + 2:].abs().max()) == 0.0


@pytest.mark.parametrize("cin,cout", [(16, 16), (48, 16), (96, 32), (32, 64), (16, 32)])
def test_conv3x3_data_and_weight_gradients_match_oracle(cin, cout):
    rng = np.random.Generator(np.random.PCG64(7 + cin + cout))
    H, W = 16, 24
    x = bf(rng.standard_normal((cin, H, W)))
    Wt = bf(rng.standard_normal((cout, cin, 3, 3)) / np.sqrt(9 * cin))
    dy = bf(rng.standard_normal((cout, H, W)))
    dx_want, dW_want, db_want = U.conv3x3_backward(x, Wt, dy)
    wb = torch.empty(cin, 9, cout, dtype=BF, device=DEV)
    E.eptv_unet_weights_to_bf16(gpu_w(Wt), cout, cin, None, wb)
    dyt = nhwc(dy)
    dx = torch.zeros(1, H, W, cin, dtype=BF, device=DEV)
    E.eptv_unet_conv3x3(dyt, 0, cout, wb, None, cin, dx, 0, False)
    dW = torch.zeros(cout, 9, cin, device=DEV)
    db = torch.zeros(cout, device=DEV)
    E.eptv_unet_conv3x3_wgrad(nhwc(x), 0, cin, dyt, 0, cout, dW, db)
    torch.cuda.synchronize()
    assert rel(chw(dx), dx_want) < 4e-3
    got_dW = dW.cpu().numpy().reshape(cout, 3, 3, cin).transpose(0, 3, 1, 2)
    assert rel(got_dW, dW_want) < 1e-5
    assert rel(db.cpu().numpy(), db_want) < 1e-5


def test_pool_upsample_relu_exact():
    rng = np.random.Generator(np.random.PCG64(3))
    x = bf(rng.standard_normal((16, 8, 12)))
    xt = nhwc(x, stride=32, off=16)
    y = torch.zeros(1, 4, 6, 16, dtype=BF, device=DEV)
    E.eptv_unet_maxpool2(xt, 16, 16, y, 0)
    assert np.array_equal(chw(y), U.maxpool2(x))
    dy = bf(rng.standard_normal((16, 4, 6)))
    dx = nhwc(np.ones((16, 8, 12)), stride=32, off=16)
    E.eptv_unet_maxpool2_bwd(xt, 16, 16, nhwc(dy), 0, dx, 16, True)
    assert np.allclose(chw(dx, 16, 16), bf(1.0 + U.maxpool2_backward(x, dy)), rtol=0, atol=1e-2)
    up = torch.zeros(1, 16, 24, 16, dtype=BF, device=DEV)
    E.eptv_unet_upsample2(xt, 16, 16, up, 0)
    assert np.array_equal(chw(up), U.upsample2(x))
    g = torch.zeros(1, 4, 6, 16, dtype=BF, device=DEV)
    dup = bf(rng.standard_normal((16, 8, 12)))
    E.eptv_unet_upsample2_bwd(nhwc(dup), 0, 16, g, 0)
    assert np.allclose(chw(g), U.upsample2_backward(dup), rtol=1e-2, atol=1e-2)
    a = nhwc(x)
    d = nhwc(dup)
    E.eptv_unet_relu_bwd(a, 0, d, 0, d, 0, 16)
    assert np.array_equal(chw(d), dup * (x > 0))


def test_adam_step_matches_formula():
    rng = np.random.Generator(np.random.PCG64(4))
    p0, g = rng.standard_normal(1000), rng.standard_normal(1000)
    m0, v0 = rng.standard_normal(1000) * 0.1, rng.uniform(0, 0.1, 1000)
    P, G, M, V = [torch.tensor(a, dtype=torch.float32, device=DEV) for a in (p0, g, m0, v0)]
    E.eptv_unet_adam(P, G, M, V, 1e-2, 0.9, 0.999, 1e-8, 3)
    m = 0.9 * m0 + 0.1 * g
    v = 0.999 * v0 + 0.001 * g * g
    want = p0 - 1e-2 * (m / (1 - 0.9 ** 3)) / (np.sqrt(v / (1 - 0.999 ** 3)) + 1e-8)
    assert np.allclose(P.cpu().numpy(), want, rtol=1e-5, atol=1e-6)


def test_network_forward_and_gradients_match_oracle():
    """The whole U-Net (10 convs, pools, upsampling, skips, head, loss) against the FP64
    oracle with the same (BF16-rounded) weights; BF16 activations through ten layers give
    errors of a few 1e-3 relative."""
    params = U.init_params(11)
    params = [[bf(a) for a in l] for l in params]
    net = L.UNet(seed=0, device=DEV)
    net.set_from_oracle_layout(params)
    net.bp_scale = 1.0
    rng = np.random.Generator(np.random.PCG64(12))
    x = bf(rng.uniform(0, 2, (2, 32, 40)))
    ft = rng.uniform(0, 1, (32, 40))
    wt = rng.uniform(0, 1, (32, 40))
    xt = torch.tensor(x, dtype=torch.float32, device=DEV)
    f0, w = net.forward(xt[0:1], xt[1:2] * L.F_SCALE)
    f0_o, w_o, _ = U.forward(params, x)
    assert rel(f0[0].double().cpu().numpy(), f0_o) < 2e-2
    assert rel(w[0].double().cpu().numpy(), w_o) < 2e-2
    loss = net.backward(torch.tensor(ft[None], dtype=torch.float32, device=DEV),
                        torch.tensor(wt[None], dtype=torch.float32, device=DEV))
    loss_o, grads_o = U.loss_and_grads(params, x, ft, wt)
    assert float(loss.item()) == pytest.approx(loss_o, rel=2e-2)
    nw = len(L.CONVS)
    for k in range(nw):
        co, ci = params[k][0].shape[:2]
        g = net.grads[k].cpu().numpy()[:, :, :ci].reshape(co, 3, 3, ci).transpose(0, 3, 1, 2)
        assert rel(g, grads_o[k][0]) < 6e-2, k
        assert rel(net.grads[nw + k].cpu().numpy(), grads_o[k][1]) < 6e-2, k
    assert rel(net.grads[2 * nw].cpu().numpy(), grads_o[10][0]) < 2e-2
    assert rel(net.grads[2 * nw + 1].cpu().numpy(), grads_o[10][1]) < 2e-2


def test_training_reduces_loss_on_fixed_batch():
    net = L.UNet(seed=1, device=DEV)
    rng = np.random.Generator(np.random.PCG64(5))
    x = torch.tensor(rng.uniform(0, 2, (4, 32, 32)), dtype=torch.float32, device=DEV)
    base = torch.tensor(rng.uniform(0, 0.04, (4, 32, 32)), dtype=torch.float32, device=DEV)
    ft = (x * 0.5).contiguous()
    wt = torch.sigmoid(x - 1.0).contiguous()
    losses = []
    for _ in range(150):
        net.forward(x, base)
        losses.append(float(net.backward(ft, wt).item()))
        net.adam_step(3e-3)
    assert losses[-1] < 0.3 * losses[0]


def test_pack_input_and_composed_head():
    """Input rows (two scaled planes, 14 zero channels) and the serving head
    f0 = max(base + s o0, 0), w = sigmoid(o1), against the oracle's head on the same BF16
    inputs."""
    rng = np.random.Generator(np.random.PCG64(21))
    npix = 1000
    a = rng.uniform(0, 3, npix).astype(np.float32)
    b = rng.uniform(-1, 1, npix).astype(np.float32)
    x = torch.full((npix, 16), 7.0, dtype=BF, device=DEV)          # stale content is overwritten
    E.eptv_unet_pack_input(torch.tensor(a).to(DEV), 0.5, torch.tensor(b).to(DEV), 3.0, x)
    got = x.float().cpu().numpy()
    assert np.array_equal(got[:, 0], bf(a.astype(np.float32) * np.float32(0.5)).astype(np.float32))
    assert np.array_equal(got[:, 1], bf(b.astype(np.float32) * np.float32(3.0)).astype(np.float32))
    assert not got[:, 2:].any()
    E.eptv_unet_pack_input(torch.tensor(a).to(DEV), 1.0, None, 0.0, x)
    assert not x.float()[:, 1:].any().item()
    feats = bf(rng.standard_normal((npix, 16)))
    hw = rng.standard_normal((2, 16)).astype(np.float32)
    hb = rng.standard_normal(2).astype(np.float32)
    base = rng.uniform(0, 0.04, npix).astype(np.float32)
    xt = torch.tensor(feats, dtype=torch.float32).to(BF).to(DEV).view(1, 1, npix, 16)
    f0 = torch.empty(npix, device=DEV)
    w = torch.empty(npix, device=DEV)
    E.eptv_unet_head(xt, torch.tensor(hw).to(DEV), torch.tensor(hb).to(DEV), f0=f0, w=w,
                     base=torch.tensor(base).to(DEV), f_scale=0.02)
    o = feats @ hw.T.astype(np.float64) + hb
    assert np.allclose(f0.cpu().numpy(), U.warm_start(o[:, 0], base, 0.02), rtol=0, atol=1e-6)
    assert np.allclose(w.cpu().numpy(), U.sigmoid(o[:, 1]), rtol=0, atol=1e-5)


def test_prior_weight_mode_matches_oracle():
    """EPTV_WEIGHTS_PRIOR: edge weights from a per-pixel map for the first prior_iters
    outer iterations (warm-start use), then Eq. (5)."""
    c = I.make_c1()
    g = c.geom
    geo = E.Geometry(g)
    rng = np.random.Generator(np.random.PCG64(6))
    wmap = rng.uniform(0.05, 1.0, (g.ny, g.nx)).astype(np.float32).astype(np.float64)
    f0 = (0.8 * c.f_true).astype(np.float32).astype(np.float64)
    p = I.EptvParams(n_outer=3, weights_mode=O.PRIOR, prior_iters=2)
    want = O.reconstruct(O.Operator(g), c.y, p, f0=f0, prior_w=wmap)
    f = torch.tensor(f0.astype(np.float32).ravel(), device=DEV)
    E.eptv_reconstruct(geo, p, torch.tensor(c.y.astype(np.float32).ravel(), device=DEV), f,
                       wprior=torch.tensor(wmap.astype(np.float32).ravel(), device=DEV))
    assert rel(f.double().cpu().numpy().reshape(g.ny, g.nx), want) < 1e-4
