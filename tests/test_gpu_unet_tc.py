"""The tensor-memory (tcgen05) 3x3 convolution of the learned warm-start network against
the FP64 U-Net oracle on BF16-rounded inputs (forward and data-gradient channel pairs),
on the image widths it tiles -- 128 and 256 (tiles of one row segment, two images) and 64
(tiles of two rows) -- with channel slices in and out, against the mma.sync kernel on the
same inputs, and the whole network forward on a size whose two upper levels use it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet_oracle as U
from paper_1009_2288_b300 import eptv as E
from paper_1009_2288_b300 import learned as L

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
BF = torch.bfloat16

PAIRS = [(16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (48, 16), (32, 16), (64, 32),
         (32, 96), (16, 48)]


def bf(a):
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(BF).double().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_w(Wt):
    co, ci = Wt.shape[:2]
    return torch.tensor(np.ascontiguousarray(np.asarray(Wt, np.float32).transpose(0, 2, 3, 1).reshape(co, 9, ci))).to(DEV)


def run_conv(x, Wt, b, xs_extra, yo, relu, path):
    """x: [n][C][H][W] float64 -> GPU conv (input channels at offset 8 of a wider tensor,
    output at offset yo of a tensor with cout + 8 channels) -> [n][cout][H][W]."""
    n, cin, H, W = x.shape
    cout = Wt.shape[0]
    xt = torch.zeros(n, H, W, cin + xs_extra, dtype=BF, device=DEV)
    xt[..., 8:8 + cin] = torch.tensor(np.ascontiguousarray(x.transpose(0, 2, 3, 1)), dtype=torch.float32).to(DEV).to(BF)
    wf = torch.empty(cout, 9, cin, dtype=BF, device=DEV)
    E.eptv_unet_weights_to_bf16(gpu_w(Wt), cout, cin, wf, None)
    y = torch.zeros(n, H, W, cout + 8, dtype=BF, device=DEV)
    E.eptv_unet_set_conv_kernel(path)
    try:
        E.eptv_unet_conv3x3(xt, 8, cin, wf, None if b is None else torch.tensor(b, dtype=torch.float32, device=DEV),
                            cout, y, yo, relu)
        torch.cuda.synchronize()
    finally:
        E.eptv_unet_set_conv_kernel(E.CONV_TENSOR_MEMORY)
    out = y.float().cpu().numpy()
    assert not out[..., :yo].any() and not out[..., yo + cout:].any()      # only the slice written
    return out[..., yo:yo + cout].transpose(0, 3, 1, 2).astype(np.float64)


@pytest.mark.parametrize("H,W,n", [(3, 128, 2), (2, 256, 1), (4, 64, 2)])
@pytest.mark.parametrize("cin,cout", PAIRS)
def test_tensor_memory_conv_matches_oracle(cin, cout, H, W, n):
    rng = np.random.Generator(np.random.PCG64(cin * 1000 + cout * 10 + W))
    x = bf(rng.standard_normal((n, cin, H, W)))
    Wt = bf(rng.standard_normal((cout, cin, 3, 3)) / np.sqrt(9 * cin))
    b = rng.standard_normal(cout).astype(np.float32).astype(np.float64)
    yo = 8 if (cin + cout) % 32 == 0 else 2           # 16-byte and 4-byte output stores
    got = run_conv(x, Wt, b, 8, yo, True, E.CONV_TENSOR_MEMORY_ALL)
    want = np.stack([np.maximum(U.conv3x3(x[i], Wt, b), 0.0) for i in range(n)])
    assert rel(got, want) < 4e-3
    ref = run_conv(x, Wt, b, 8, yo, True, E.CONV_MMA_SYNC)
    assert rel(got, ref) < 4e-3
    E.eptv_unet_tc_status()


def test_tensor_memory_conv_data_gradient_without_relu_or_bias():
    """The data gradient of a 96 -> 32 layer is the 32 -> 96 conv with the mirrored,
    channel-swapped weights: dx against the oracle's backward pass."""
    rng = np.random.Generator(np.random.PCG64(33))
    cin, cout, H, W = 96, 32, 4, 128
    x = bf(rng.standard_normal((cin, H, W)))
    Wt = bf(rng.standard_normal((cout, cin, 3, 3)) / np.sqrt(9 * cin))
    dy = bf(rng.standard_normal((cout, H, W)))
    dx_want, _, _ = U.conv3x3_backward(x, Wt, dy)
    wb = torch.empty(cin, 9, cout, dtype=BF, device=DEV)
    E.eptv_unet_weights_to_bf16(gpu_w(Wt), cout, cin, None, wb)
    dyt = torch.tensor(np.ascontiguousarray(dy.transpose(1, 2, 0))[None], dtype=torch.float32).to(DEV).to(BF)
    dx = torch.zeros(1, H, W, cin, dtype=BF, device=DEV)
    E.eptv_unet_set_conv_kernel(E.CONV_TENSOR_MEMORY_ALL)
    try:
        E.eptv_unet_conv3x3(dyt, 0, cout, wb, None, cin, dx, 0, False)
        torch.cuda.synchronize()
    finally:
        E.eptv_unet_set_conv_kernel(E.CONV_TENSOR_MEMORY)
    got = dx[0].float().cpu().numpy().transpose(2, 0, 1)
    assert rel(got, dx_want) < 4e-3
    E.eptv_unet_tc_status()


def test_network_forward_with_tensor_memory_convs_matches_oracle():
    """A 64 x 128 input with every tileable conv on the tensor-memory kernel: level 1
    (W = 128) and level 2 (W = 64) on it, level 3 (W = 32) on mma.sync; outputs and
    parameter gradients against the FP64 oracle as for the small network test."""
    params = U.init_params(13)
    params = [[bf(a) for a in l] for l in params]
    net = L.UNet(seed=0, device=DEV)
    net.set_from_oracle_layout(params)
    net.bp_scale = 1.0
    E.eptv_unet_set_conv_kernel(E.CONV_TENSOR_MEMORY_ALL)
    rng = np.random.Generator(np.random.PCG64(14))
    x = bf(rng.uniform(0, 2, (2, 64, 128)))
    ft = rng.uniform(0, 1, (64, 128))
    wt = rng.uniform(0, 1, (64, 128))
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
    E.eptv_unet_set_conv_kernel(E.CONV_TENSOR_MEMORY)
    E.eptv_unet_tc_status()
