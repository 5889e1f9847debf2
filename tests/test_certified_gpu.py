"""Certified mixed precision (SE_PREC_CERTIFIED) on the GPU.

The fp32 iteration kernel tracks the gap between the two best scores of
every selection (eq. 18); blocks where it closes below the certification
threshold are recomputed in fp64.  The selected-index sequence of every
block must therefore equal the fp64 form's, and the oracle's up to its
first near tie at the fp64 tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2204_14194_gb300 import binding as B
from paper_2204_14194_gb300 import workloads as W
from helpers import coef_rel_err, first_near_tie, psnr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = B.Context(0)
    yield c
    c.close()


def _run(ctx, plan, samples):
    n = samples.shape[0]
    I = plan.iterations
    s = torch.from_numpy(samples).cuda()
    out = torch.empty_like(s)
    u = torch.full((n, I), -1, dtype=torch.int32, device="cuda")
    c = torch.full((n, I), float("nan"), dtype=torch.float64, device="cuda")
    plan.extrapolate_strided(s, out, u, c)
    ctx.sync()
    return out.cpu().numpy(), u.cpu().numpy(), c.cpu().numpy()


@pytest.mark.parametrize("L,K,n", [(32, 2048, 2048), (16, 512, 2048)])
def test_certified_sequences_equal_the_fp64_form(ctx, L, K, n):
    if L == 32:
        wl = W.config2(n)
        samples, sup = wl.samples, wl.support
    else:
        samples = np.stack([W.patch(L, 6000 + i) for i in range(n)])
        sup = W.centred_support(L, L)
    I = 100
    pc = ctx.plan(L, L, "dct_wht", K, 0.8, 0.5, I, prec="certified")
    p64 = ctx.plan(L, L, "dct_wht", K, 0.8, 0.5, I, prec="fp64")
    s0 = ctx.cert_stats()
    oc, uc, cc = _run(ctx, pc, samples)
    s1 = ctx.cert_stats()
    o64, u64, c64 = _run(ctx, p64, samples)
    np.testing.assert_array_equal(uc, u64)
    recomputed = s1["recomputed"] - s0["recomputed"]
    assert s1["blocks"] - s0["blocks"] == n
    assert recomputed < 0.25 * n, recomputed
    # recomputed blocks are the fp64 form's bit for bit; the others within the fp32 tolerance
    exact = np.all(cc == c64, axis=1)
    assert exact.sum() >= recomputed
    for b in np.where(~exact)[0]:
        assert coef_rel_err(cc[b], c64[b]).max() <= 1e-3
    loss = np.broadcast_to(sup == 0, oc.shape)
    assert abs(psnr(oc, samples, loss) - psnr(o64, samples, loss)) <= 0.05
    # and the oracle's sequence up to its first near tie at the fp64 tolerance
    phi = O.dict_dct_wht(L, L)
    dup = O.find_duplicates(phi)
    w = O.weights(L, L, 0.8, sup)
    pick = np.random.default_rng(L).choice(n, 12, replace=False)
    ro, ru, rc, rm, st = O.se_original_batch(phi, w, samples[pick], 0.5, I, dup, margins=True)
    for i, b in enumerate(pick):
        t = first_near_tie(rm[i], 1e-9)
        np.testing.assert_array_equal(uc[b, :t], ru[i, :t])
    pc.close()
    p64.close()


def test_certified_plan_limits(ctx):
    with pytest.raises(B.SeError) as e:
        ctx.plan(64, 64, "dct_wht", 8192, 0.8, 0.5, 10, prec="certified")
    assert e.value.status == -1
    with pytest.raises(B.SeError) as e:
        ctx.plan(16, 16, "dct_wht", 512, 0.8, 0.5, 10, prec="certified", gram="lazy")
    assert e.value.status == -1
    p = ctx.plan(16, 16, "dct_wht", 512, 0.8, 0.5, 10, prec="certified")
    s = torch.from_numpy(W.patch(16, 1)[None].copy()).cuda()
    m = torch.from_numpy(W.centred_support(16, 16)).cuda()
    o = torch.empty_like(s)
    with pytest.raises(B.SeError) as e:
        p.extrapolate_batch([{"samples": s[0], "support": m, "out": o[0]}])
    assert e.value.status == -1
    with pytest.raises(B.SeError):
        p.extrapolate_noalloc(s, o)
    p.close()
