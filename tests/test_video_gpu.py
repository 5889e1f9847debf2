"""3-D (video) blocks on the GPU: M x N x T areas, frame-major samples.

The method runs unchanged on the flattened area; the oracle builds its own
3-D DCT / WHT atoms and 3-D weighting function.  Same bars as the 2-D
parity tests: index sequence up to the first near tie, coefficients within
1e-9 (fp64 form) / 1e-3 (fp32 form), PSNR within 0.05 dB.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2204_14194_gb300 import binding as B
from paper_2204_14194_gb300 import workloads as W
from helpers import coef_rel_err, first_near_tie, psnr

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-9, 1e-9), "bf16x6": (1e-4, 1e-3)}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = B.Context(0)
    yield c
    c.close()


def _run(ctx, plan, samples, masks=None, iters=None):
    n = samples.shape[0]
    I = plan.iterations
    s = torch.from_numpy(np.ascontiguousarray(samples)).cuda()
    out = torch.empty_like(s)
    u = torch.full((n, I), -1, dtype=torch.int32, device="cuda")
    c = torch.full((n, I), float("nan"), dtype=torch.float64, device="cuda")
    if masks is None:
        plan.extrapolate_strided(s, out, u, c)
    else:
        m = torch.from_numpy(np.ascontiguousarray(masks)).cuda()
        plan.extrapolate_batch([{"samples": s[b], "support": m[b], "out": out[b], "sel_idx": u[b],
                                 "sel_coef": c[b], "iterations": int(iters[b])} for b in range(n)])
    ctx.sync()
    return out.cpu().numpy(), u.cpu().numpy(), c.cpu().numpy()


def _check(prec, out, u, c, samples, masks, phi, iters, gamma=0.5, rho=0.8):
    M, N, T = samples.shape[2], samples.shape[3], samples.shape[1]
    dup = O.find_duplicates(phi)
    w = np.stack([O.flat(O.weights3(M, N, T, rho, m)) for m in masks])
    ro, ru, rc, rm, st = O.se_original_batch(phi, w, O.flat(samples), gamma, int(max(iters)), dup,
                                             iters=np.asarray(iters), margins=True)
    assert st == 0
    tau, ctol = TOL[prec]
    for b in range(len(samples)):
        I = int(iters[b])
        t = first_near_tie(rm[b, :I], tau)
        np.testing.assert_array_equal(u[b][:t], ru[b, :t])
        if t:
            assert coef_rel_err(c[b][:t], rc[b, :t]).max() <= ctol
        np.testing.assert_array_equal(out[b][masks[b] > 0], samples[b][masks[b] > 0])
    loss = masks == 0
    assert abs(psnr(out, samples, loss) - psnr(ro.reshape(out.shape), samples, loss)) <= 0.05


@pytest.mark.parametrize("M,N,T,basis", [(16, 16, 4, "dct"), (8, 8, 8, "dct_wht")])
@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_video_blocks_on_the_default_pattern(ctx, M, N, T, basis, prec):
    n, I = 24, 60
    K = (2 if basis == "dct_wht" else 1) * M * N * T
    samples = np.stack([W.video_block(M, N, T, 300 + i) for i in range(n)])
    plan = ctx.plan(M, N, basis, K, 0.8, 0.5, I, prec=prec, T=T)
    out, u, c = _run(ctx, plan, samples)
    sup = W.centred_support3(M, N, T)
    _check(prec, out, u, c, samples, np.broadcast_to(sup, samples.shape).astype(np.uint8),
           O.flat(O.dictionary3(basis, M, N, T)), [I] * n)
    plan.close()


def test_video_blocks_with_their_own_masks(ctx):
    M, N, T, n = 8, 8, 4, 16
    rng = np.random.default_rng(9)
    samples = np.stack([W.video_block(M, N, T, 500 + i) for i in range(n)])
    masks = np.ones((n, T, M, N), dtype=np.uint8)
    for b in range(n):   # a moving lost box: M/2 x N/2 in two consecutive frames
        t0 = int(rng.integers(0, T - 1))
        r0, c0 = (int(v) for v in rng.integers(1, 4, size=2))
        masks[b, t0:t0 + 2, r0:r0 + M // 2, c0:c0 + N // 2] = 0
    iters = rng.integers(20, 61, size=n)
    plan = ctx.plan(M, N, "dct_wht", 2 * M * N * T, 0.8, 0.5, 60, prec="bf16x6", T=T)
    out, u, c = _run(ctx, plan, samples, masks, iters)
    _check("bf16x6", out, u, c, samples, masks, O.flat(O.dictionary3("dct_wht", M, N, T)), iters)
    plan.close()


def test_one_frame_is_the_2d_plan(ctx):
    wl = W.config2(64)
    a = ctx.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, 50, prec="bf16x6")
    b = ctx.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, 50, prec="bf16x6", T=1)
    ra = _run(ctx, a, wl.samples)
    rb = _run(ctx, b, wl.samples)
    for x, y in zip(ra, rb):
        np.testing.assert_array_equal(x, y)
    a.close()
    b.close()


def test_video_plan_validation(ctx):
    with pytest.raises(B.SeError):
        ctx.plan(8, 8, "wht", 192, 0.8, 0.5, 10, T=3)       # WHT needs T a power of two
    with pytest.raises(B.SeError):
        ctx.plan(8, 8, "dct", 64 * 65, 0.8, 0.5, 10, T=65)  # T <= 64
    with pytest.raises(B.SeError):
        ctx.plan(8, 8, "dct", 64 * 4, 0.8, 0.5, 10, T=3)    # K must be M N T
