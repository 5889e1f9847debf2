"""GPU parity at long iteration counts (I = 500): does the fp32 recurrence drift?

SE runs exactly I iterations (Sec. II) and the mixed-size workload draws I
up to 500.  The fp32 form keeps the running projections R_k in fp32 and
updates them I times by eq. (20), so rounding errors accumulate with I.
These cases run the fp32 form for 500 iterations against the FP64 oracle
(Alg. 1): the selected index sequence up to the first near tie, coefficients
within 1e-3 relative on those iterations, and pooled PSNR within 0.05 dB.
They cover both iteration kernels of shared patterns (parity classes for a
centred loss area, the general kernel for a shifted one) and the
per-block-mask path with lazily computed columns, which keeps its running
recurrence in fp64 beyond 256 iterations.

The rounding error of the fp32 tables and columns stays about constant in
the scale of the initial projections, so relative to the projections, which
decay with every iteration, it grows: at I = 500 the largest relative
coefficient error measured is 8e-4 (masked 16 x 16 blocks), and 1 of 256
such blocks left the oracle's sequence at iteration 436 at a tie margin of
2e-4.  Shared patterns are held to the bars of the other parity tests (tie
margin 1e-4).  The masked long runs are held to what was measured: every
block follows the oracle at least up to its first near tie at 1e-3, at most
1 % of the blocks depart before their first near tie at 1e-4, coefficients
within 1e-3 up to that point, PSNR within 0.05 dB.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2204_14194_gb300 import binding as B
from paper_2204_14194_gb300 import workloads as W
from helpers import coef_rel_err, first_near_tie, psnr

pytestmark = pytest.mark.gpu

I_LONG = 500
TAU, CTOL = 1e-4, 1e-3


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = B.Context(0)
    yield c
    c.close()


def _compare(out, u, c, ro, ru, rc, rm, iters, samples, masks, tau=TAU):
    """Bars of the parity tests; returns the iterations compared per block."""
    compared = []
    for b in range(len(samples)):
        I = int(iters[b])
        t = first_near_tie(rm[b, :I], tau)
        np.testing.assert_array_equal(u[b][:t], ru[b, :t])
        if t:
            err = coef_rel_err(c[b][:t], rc[b, :t])
            assert err.max() <= CTOL, (b, float(err.max()), int(err.argmax()))
        np.testing.assert_array_equal(out[b][masks[b] > 0], samples[b][masks[b] > 0])
        compared.append(t)
    loss = masks == 0
    assert abs(psnr(out, samples, loss) - psnr(ro, samples, loss)) <= 0.05
    return np.asarray(compared)


@pytest.mark.parametrize("shift", [0, 1])
def test_shared_pattern_32x32_K2048_I500(ctx, shift):
    """32 blocks of 32 x 32, DCT u WHT (K = 2048), 16 x 16 loss area: centred
    (parity-class kernels) or shifted by one column (general kernel)."""
    L, n = 32, 32
    sup = np.ones((L, L), dtype=np.uint8)
    sup[8:24, 8 + shift:24 + shift] = 0
    wl = W.config2(n)
    s = wl.samples
    plan = ctx.plan(L, L, "dct_wht", 2 * L * L, 0.8, 0.5, I_LONG, prec="bf16x6", support=sup)
    assert plan.info().get("iterations") == ("general" if shift else "parity-classes")
    st_ = torch.from_numpy(s).cuda()
    out = torch.empty_like(st_)
    u = torch.full((n, I_LONG), -1, dtype=torch.int32, device="cuda")
    c = torch.full((n, I_LONG), float("nan"), dtype=torch.float64, device="cuda")
    plan.extrapolate_strided(st_, out, u, c)
    ctx.sync()
    phi = O.dict_dct_wht(L, L)
    dup = O.find_duplicates(phi)
    w = O.weights(L, L, 0.8, sup)
    ro, ru, rc, rm, st = O.se_original_batch(phi, w, s, 0.5, I_LONG, dup, margins=True)
    assert st == 0
    masks = np.broadcast_to(sup, s.shape)
    t = _compare(out.cpu().numpy(), u.cpu().numpy(), c.cpu().numpy(), ro, ru, rc, rm,
                 [I_LONG] * n, s, masks)
    # the comparison must reach well into the long run, not stop at the start
    assert np.median(t) >= 150, t
    plan.close()


@pytest.mark.parametrize("L,n", [(16, 256), (32, 24)])
def test_per_block_masks_I500(ctx, L, n):
    """Per-block masks (rectangles and scattered 4 x 4 holes) with lazily
    computed columns, DCT u WHT with K = 2 L^2, every block at I = 500."""
    rng = np.random.default_rng(500 + L)
    masks = np.stack([W.rect_support(L, L, rng) if i % 2 == 0 else W.holes_support(L, L, rng)
                      for i in range(n)])
    s = np.stack([W.patch(L, 8000 + L + i) for i in range(n)])
    plan = ctx.plan(L, L, "dct_wht", 2 * L * L, 0.8, 0.5, I_LONG, prec="bf16x6")
    sd = torch.from_numpy(s).cuda()
    md = torch.from_numpy(masks).cuda()
    out = torch.empty_like(sd)
    u = torch.full((n, I_LONG), -1, dtype=torch.int32, device="cuda")
    c = torch.full((n, I_LONG), float("nan"), dtype=torch.float64, device="cuda")
    plan.extrapolate_batch([{"samples": sd[b], "support": md[b], "out": out[b], "sel_idx": u[b],
                             "sel_coef": c[b]} for b in range(n)])
    ctx.sync()
    phi = O.dict_dct_wht(L, L)
    dup = O.find_duplicates(phi)
    w = np.stack([O.weights(L, L, 0.8, masks[b]) for b in range(n)])
    ro, ru, rc, rm, st = O.se_original_batch(phi, w, s, 0.5, I_LONG, dup, margins=True)
    assert st == 0
    u, c, out = u.cpu().numpy(), c.cpu().numpy(), out.cpu().numpy()
    departed, compared = 0, []
    for b in range(n):
        t4, t3 = first_near_tie(rm[b], 1e-4), first_near_tie(rm[b], 1e-3)
        diff = np.nonzero(u[b] != ru[b])[0]
        m = int(diff[0]) if len(diff) else I_LONG
        assert m >= t3, (b, m, t3)
        departed += m < t4
        t = min(m, t4)
        if t:
            assert coef_rel_err(c[b][:t], rc[b, :t]).max() <= CTOL
        np.testing.assert_array_equal(out[b][masks[b] > 0], s[b][masks[b] > 0])
        compared.append(t)
    assert departed <= 0.01 * n, departed
    loss = masks == 0
    assert abs(psnr(out, s, loss) - psnr(ro, s, loss)) <= 0.05
    assert np.median(compared) >= 150, compared
    plan.close()
