"""GPU parity of the per-block-mask path (lazily computed table columns).

Each block carries its own support mask (a random M/2 x N/2 rectangle or
scattered 4x4 holes, as in the mixed-size workload); the oracle runs Alg. 1
with that block's weighting function.  Same bars as the shared-pattern
tests: index sequence up to the first near tie, coefficients within 1e-9
(fp64 form) / 1e-3 (bf16x6), PSNR within 0.05 dB.
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


def _masks(L, n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([W.rect_support(L, L, rng) if i % 2 == 0 else W.holes_support(L, L, rng)
                     for i in range(n)])


def _run_masked(plan, samples, masks, iters, m=None):
    n, M, N = samples.shape
    s = torch.from_numpy(samples).cuda()
    if m is None:
        m = torch.from_numpy(masks).cuda()
    out = torch.empty_like(s)
    us = [torch.full((i,), -1, dtype=torch.int32, device="cuda") for i in iters]
    cs = [torch.full((i,), float("nan"), dtype=torch.float64, device="cuda") for i in iters]
    plan.extrapolate_batch([{"samples": s[b], "support": m[b], "out": out[b], "sel_idx": us[b],
                             "sel_coef": cs[b], "iterations": int(iters[b])} for b in range(n)])
    plan.ctx.sync()
    return out.cpu().numpy(), [u.cpu().numpy() for u in us], [c.cpu().numpy() for c in cs]


def _oracle_masked(basis, samples, masks, iters, rho_hat=0.8, gamma=0.5, numeric=None):
    n, M, N = samples.shape
    phi = O.dictionary(basis, M, N, numeric)
    dup = O.find_duplicates(phi)
    w = np.stack([O.weights(M, N, rho_hat, masks[b]) for b in range(n)])
    I = int(max(iters))
    return O.se_original_batch(phi, w, samples, gamma, I, dup, iters=np.asarray(iters), margins=True)


def _check(prec, out, u, c, ro, ru, rc, rm, iters, samples, masks):
    tau, ctol = TOL[prec]
    for b in range(len(iters)):
        I = int(iters[b])
        t = first_near_tie(rm[b, :I], tau)
        np.testing.assert_array_equal(u[b][:t], ru[b, :t])
        if t:
            assert coef_rel_err(c[b][:t], rc[b, :t]).max() <= ctol
        np.testing.assert_array_equal(out[b][masks[b] > 0], samples[b][masks[b] > 0])
    loss = masks == 0
    assert abs(psnr(out, samples, loss) - psnr(ro, samples, loss)) <= 0.05


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
@pytest.mark.parametrize("L,n,I", [(16, 24, 150), (32, 8, 100)])
def test_per_block_masks_dct_wht(ctx, prec, L, n, I):
    samples = np.stack([W.patch(L, 3000 + L + i) for i in range(n)])
    masks = _masks(L, n, 40 + L)
    iters = np.random.default_rng(L).integers(max(1, I // 3), I + 1, size=n)
    plan = ctx.plan(L, L, "dct_wht", 2 * L * L, 0.8, 0.5, I, prec=prec)
    out, u, c = _run_masked(plan, samples, masks, iters)
    ro, ru, rc, rm, st = _oracle_masked("dct_wht", samples, masks, iters)
    assert st == 0
    _check(prec, out, u, c, ro, ru, rc, rm, iters, samples, masks)
    plan.close()


def test_per_block_masks_64x64_K8192(ctx):
    L, n, I = 64, 2, 25
    samples = np.stack([W.patch(L, 7100 + i) for i in range(n)])
    masks = _masks(L, n, 71)
    iters = [I, I - 7]
    plan = ctx.plan(L, L, "dct_wht", 2 * L * L, 0.8, 0.5, I, prec="bf16x6")
    out, u, c = _run_masked(plan, samples, masks, iters)
    ro, ru, rc, rm, st = _oracle_masked("dct_wht", samples, masks, iters)
    _check("bf16x6", out, u, c, ro, ru, rc, rm, iters, samples, masks)
    plan.close()


def test_per_block_masks_gaussian_dictionary(ctx):
    L, n, I, K = 16, 12, 80, 512
    dic = W.gaussian_dictionary(K, L, L, 77)
    samples = np.stack([W.patch(L, 7200 + i) for i in range(n)])
    masks = _masks(L, n, 72)
    iters = [I] * n
    for prec in ("fp64", "bf16x6"):
        plan = ctx.plan(L, L, "numeric", K, 0.8, 0.5, I, prec=prec, dictionary=dic)
        out, u, c = _run_masked(plan, samples, masks, iters)
        ro, ru, rc, rm, st = _oracle_masked("numeric", samples, masks, iters, numeric=dic)
        _check(prec, out, u, c, ro, ru, rc, rm, iters, samples, masks)
        plan.close()


def test_lazy_on_shared_pattern_and_mixed_batch(ctx):
    """gram='lazy' on the plan pattern matches the oracle; a batch mixing pattern
    blocks (full table) and masked blocks (lazy) gives each block its own result."""
    wl = W.config2(6)
    I = 60
    sup = wl.support
    plan_l = ctx.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, I, prec="bf16x6", gram="lazy")
    s = torch.from_numpy(wl.samples).cuda()
    out = torch.empty_like(s)
    u = torch.empty((6, I), dtype=torch.int32, device="cuda")
    c = torch.empty((6, I), dtype=torch.float64, device="cuda")
    plan_l.extrapolate_strided(s, out, u, c)
    ctx.sync()
    phi = O.dict_dct_wht(32, 32)
    dup = O.find_duplicates(phi)
    w = O.weights(32, 32, 0.8, sup)
    ro, ru, rc, rm, st = O.se_original_batch(phi, w, wl.samples, 0.5, I, dup, margins=True)
    u_l, c_l, o_l = u.cpu().numpy(), c.cpu().numpy(), out.cpu().numpy()
    for b in range(6):
        t = first_near_tie(rm[b], 1e-4)
        np.testing.assert_array_equal(u_l[b, :t], ru[b, :t])
        assert coef_rel_err(c_l[b, :t], rc[b, :t]).max() <= 1e-3
    plan_l.close()

    plan = ctx.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, I, prec="bf16x6")
    masks = _masks(32, 6, 9)
    m = torch.from_numpy(masks).cuda()
    out2 = torch.empty_like(s)
    us = torch.empty((6, I), dtype=torch.int32, device="cuda")
    blocks = []
    for b in range(6):
        d = {"samples": s[b], "out": out2[b], "sel_idx": us[b]}
        if b % 2:
            d["support"] = m[b]
        blocks.append(d)
    plan.extrapolate_batch(blocks)
    ctx.sync()
    u2 = us.cpu().numpy()
    w_b = np.stack([w if b % 2 == 0 else O.weights(32, 32, 0.8, masks[b]) for b in range(6)])
    r2o, r2u, r2c, r2m, st = O.se_original_batch(phi, w_b, wl.samples, 0.5, I, dup, margins=True)
    for b in range(6):
        t = first_near_tie(r2m[b], 1e-4)
        np.testing.assert_array_equal(u2[b, :t], r2u[b, :t])
    plan.close()


def test_empty_block_mask_reports_empty_support(ctx):
    plan = ctx.plan(16, 16, "dct_wht", 512, 0.8, 0.5, 10, prec="bf16x6")
    s = torch.from_numpy(W.patch(16, 5)[None].copy()).cuda()
    m = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(s)
    plan.extrapolate_batch([{"samples": s[0], "support": m, "out": out[0]}])
    with pytest.raises(B.SeError) as e:
        ctx.sync()
    assert e.value.status == -5
    plan.close()


@pytest.mark.parametrize("L,form", [(32, "tensor"), (32, "ffma"), (64, "tensor"), (64, "ffma")])
def test_per_block_masks_column_forms(ctx, L, form, monkeypatch):
    """The lazy columns of 32 x 32 and 64 x 64 areas on the tensor cores
    (two-part fp16 splits with power-of-two scales, the default) and in the
    fp32 transform kernels (SE_COL_FFMA=1):
    16 blocks with rectangles and scattered holes, I up to 120, each form
    against the oracle with the bars of the other parity tests, and the two
    forms' coefficients within 1e-3 of each other where their sequences agree
    (both run the iterations in fp32; their residuals drift apart by rounding
    over a hundred updates, as each drifts from the FP64 oracle)."""
    n = 16
    samples = np.stack([W.patch(L, 7300 + i) for i in range(n)])
    masks = _masks(L, n, 73)
    iters = np.random.default_rng(64).integers(60, 121, size=n)
    ro, ru, rc, rm, st = _oracle_masked("dct_wht", samples, masks, iters)
    assert st == 0
    res = {}
    for f in ("tensor", "ffma"):
        if f == "ffma":
            monkeypatch.setenv("SE_COL_FFMA", "1")
        else:
            monkeypatch.delenv("SE_COL_FFMA", raising=False)
        plan = ctx.plan(L, L, "dct_wht", 2 * L * L, 0.8, 0.5, int(iters.max()), prec="bf16x6")
        res[f] = _run_masked(plan, samples, masks, iters)
        plan.close()
    monkeypatch.delenv("SE_COL_FFMA", raising=False)
    out, u, c = res[form]
    _check("bf16x6", out, u, c, ro, ru, rc, rm, iters, samples, masks)
    (_, ut, ct), (_, uf, cf) = res["tensor"], res["ffma"]
    for b in range(n):
        diff = np.nonzero(ut[b] != uf[b])[0]
        t = int(diff[0]) if len(diff) else len(ut[b])
        assert t >= first_near_tie(rm[b, :len(ut[b])], 1e-4)
        if t:
            assert coef_rel_err(ct[b][:t], cf[b][:t]).max() <= 1e-3


def test_per_block_masks_single_transform_64x64(ctx):
    """64 x 64 areas with DCT atoms only (K = 4096, one transform): the
    tensor-core column kernel with a single transform and the round kernel
    with one CTA per block at K = 4096, against the oracle."""
    L, n = 64, 8
    samples = np.stack([W.patch(L, 8100 + i) for i in range(n)])
    masks = _masks(L, n, 81)
    iters = np.random.default_rng(81).integers(40, 101, size=n)
    ro, ru, rc, rm, st = _oracle_masked("dct", samples, masks, iters)
    assert st == 0
    plan = ctx.plan(L, L, "dct", L * L, 0.8, 0.5, int(iters.max()), prec="bf16x6")
    out, u, c = _run_masked(plan, samples, masks, iters)
    plan.close()
    _check("bf16x6", out, u, c, ro, ru, rc, rm, iters, samples, masks)


@pytest.mark.parametrize("L", [32, 64])
def test_per_block_masks_unaligned_support(ctx, L):
    """Masks that start one byte past a 4-byte boundary (views into one
    buffer at offset 1): the column kernel reads them byte by byte instead of
    as words; against the oracle."""
    n = 6
    samples = np.stack([W.patch(L, 8200 + L + i) for i in range(n)])
    masks = _masks(L, n, 90 + L)
    iters = np.random.default_rng(90 + L).integers(30, 81, size=n)
    ro, ru, rc, rm, st = _oracle_masked("dct_wht", samples, masks, iters)
    assert st == 0
    buf = torch.zeros(n * L * L + 1, dtype=torch.uint8, device="cuda")
    buf[1:] = torch.from_numpy(masks.reshape(-1)).cuda()
    m = buf[1:].view(n, L, L)
    assert all(m[b].data_ptr() % 4 != 0 for b in range(n))
    plan = ctx.plan(L, L, "dct_wht", 2 * L * L, 0.8, 0.5, int(iters.max()), prec="bf16x6")
    out, u, c = _run_masked(plan, samples, masks, iters, m=m)
    plan.close()
    _check("bf16x6", out, u, c, ro, ru, rc, rm, iters, samples, masks)
