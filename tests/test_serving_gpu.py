"""Serving loop (se_submit / se_poll / se_cancel) on the GPU.

Results must be identical whether a request runs alone or mixed with other
requests of other plans and iteration counts, and identical to the batched
entry point; latency is reported per request.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2204_14194_gb300 import binding as B
from paper_2204_14194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = B.Context(0)
    yield c
    c.close()


def _submit_all(ctx, reqs):
    tickets = []
    for plan, s, I in reqs:
        out = np.empty_like(s)
        u = np.empty(I, dtype=np.int32)
        c = np.empty(I)
        t = ctx.submit(plan, s, out, u, c, iterations=I)
        tickets.append((t, out, u, c))
    res = []
    for t, out, u, c in tickets:
        st, lat = ctx.poll(t, timeout_us=60_000_000)
        assert st == B.SE_OK
        assert lat > 0
        res.append((out, u, c, lat))
    return res


def test_alone_equals_mixed_and_batch(ctx):
    p32 = ctx.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, 100, prec="bf16x6")
    p16 = ctx.plan(16, 16, "dct_wht", 512, 0.8, 0.5, 100, prec="bf16x6")
    wl = W.config2(64)
    s16 = np.stack([W.patch(16, 900 + i) for i in range(48)])
    rng = np.random.default_rng(5)

    alone = _submit_all(ctx, [(p32, wl.samples[10], 100)])[0]

    mix = [(p32, wl.samples[i], int(rng.integers(50, 151))) for i in range(64)]
    mix[10] = (p32, wl.samples[10], 100)
    mix += [(p16, s16[i], int(rng.integers(20, 301))) for i in range(48)]
    order = rng.permutation(len(mix))
    mixed_sorted = [mix[i] for i in order]
    res_sorted = _submit_all(ctx, mixed_sorted)
    res = [None] * len(mix)
    for k, i in enumerate(order):
        res[i] = res_sorted[k]

    np.testing.assert_array_equal(res[10][0], alone[0])
    np.testing.assert_array_equal(res[10][1], alone[1])
    np.testing.assert_array_equal(res[10][2], alone[2])

    # same as the batched entry point, block by block, for every iteration count
    for i in (0, 10, 63):
        plan, s, I = mix[i]
        sd = torch.from_numpy(s[None].copy()).cuda()
        od = torch.empty_like(sd)
        ud = torch.empty((1, I), dtype=torch.int32, device="cuda")
        cd = torch.empty((1, I), dtype=torch.float64, device="cuda")
        plan.extrapolate_strided(sd, od, ud, cd, iterations=I)
        ctx.sync()
        np.testing.assert_array_equal(res[i][0], od.cpu().numpy()[0])
        np.testing.assert_array_equal(res[i][1], ud.cpu().numpy()[0])
        np.testing.assert_array_equal(res[i][2], cd.cpu().numpy()[0])
    assert ctx.stats()["serving_slices"] >= 2
    p32.close()
    p16.close()


def test_poll_pending_cancel_and_unknown(ctx):
    p = ctx.plan(64, 64, "dct_wht", 8192, 0.8, 0.5, 300, prec="bf16x6")
    s = np.stack([W.patch(64, 40 + i) for i in range(200)])
    outs = [np.empty((64, 64)) for _ in range(200)]
    tickets = [ctx.submit(p, s[i], outs[i]) for i in range(200)]
    # the last request is queued behind 199 others: cancel it (or it already runs)
    st = ctx.cancel(tickets[-1])
    assert st in (B.SE_OK, B.SE_PENDING)
    done = 0
    for t in tickets[:-1]:
        st, _ = ctx.poll(t, timeout_us=120_000_000)
        done += st == B.SE_OK
    assert done == 199
    if st == B.SE_OK:
        with pytest.raises(B.SeError):
            ctx.poll(tickets[-1], timeout_us=0)
    with pytest.raises(B.SeError) as e:
        ctx.poll(10 ** 12, timeout_us=0)
    assert e.value.status == -7
    p.close()


def test_budget_too_small_rejects(ctx):
    small = B.Context(0, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(B.SeError) as e:
            small.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, 100)
        assert e.value.status == -2
    finally:
        small.close()


def test_masked_requests_alone_equal_mixed(ctx):
    """Requests with their own support masks (lazy columns inside the serving
    lanes) give bitwise the same result alone and mixed with pattern requests."""
    p16 = ctx.plan(16, 16, "dct_wht", 512, 0.8, 0.5, 120, prec="bf16x6")
    rng = np.random.default_rng(11)
    samples = [W.patch(16, 1200 + i) for i in range(40)]
    masks = [W.rect_support(16, 16, rng) if i % 2 else W.holes_support(16, 16, rng) for i in range(40)]
    iters = [int(v) for v in rng.integers(30, 121, size=40)]

    def run(indices, with_mask):
        tick = []
        for i in indices:
            out = np.empty((16, 16))
            u = np.empty(iters[i], dtype=np.int32)
            t = ctx.submit(p16, samples[i], out, u, None, iterations=iters[i],
                           support=masks[i] if with_mask[i] else None)
            tick.append((i, t, out, u))
        res = {}
        for i, t, out, u in tick:
            st, lat = ctx.poll(t, timeout_us=60_000_000)
            assert st == B.SE_OK
            res[i] = (out, u)
        return res

    with_mask = [i % 3 != 0 for i in range(40)]
    alone = run([5], with_mask)
    mixed = run(list(range(40)), with_mask)
    np.testing.assert_array_equal(alone[5][0], mixed[5][0])
    np.testing.assert_array_equal(alone[5][1], mixed[5][1])
    # and the same as the batched entry point with the same mask
    s = torch.from_numpy(samples[5][None].copy()).cuda()
    m = torch.from_numpy(masks[5]).cuda()
    o = torch.empty_like(s)
    ud = torch.empty(iters[5], dtype=torch.int32, device="cuda")
    p16.extrapolate_batch([{"samples": s[0], "support": m, "out": o[0], "sel_idx": ud,
                            "iterations": iters[5]}])
    ctx.sync()
    np.testing.assert_array_equal(o.cpu().numpy()[0], mixed[5][0])
    np.testing.assert_array_equal(ud.cpu().numpy(), mixed[5][1])
    p16.close()


def test_gaussian_masked_requests_alone_equal_mixed_and_match_the_oracle(ctx):
    """Requests on a numeric (Gaussian) dictionary with their own masks: the
    lazy columns of eq. (16) come from two-part fp16 products.  A request gives
    bitwise the same result alone and mixed with others, and every result
    meets the parity bars against the FP64 oracle (Alg. 1)."""
    import oracle as O
    from helpers import coef_rel_err, first_near_tie, psnr

    L, K, n = 32, 2048, 24
    dic = W.gaussian_dictionary(K, L, L, 932)
    p = ctx.plan(L, L, "numeric", K, 0.8, 0.5, 200, prec="bf16x6", dictionary=dic)
    rng = np.random.default_rng(13)
    samples = [W.patch(L, 1500 + i) for i in range(n)]
    masks = [W.rect_support(L, L, rng) if i % 2 else W.holes_support(L, L, rng) for i in range(n)]
    iters = [int(v) for v in rng.integers(100, 201, size=n)]

    def run(indices):
        tick = []
        for i in indices:
            out = np.empty((L, L))
            u = np.empty(iters[i], dtype=np.int32)
            c = np.empty(iters[i])
            t = ctx.submit(p, samples[i], out, u, c, iterations=iters[i], support=masks[i])
            tick.append((i, t, out, u, c))
        res = {}
        for i, t, out, u, c in tick:
            st, _ = ctx.poll(t, timeout_us=120_000_000)
            assert st == B.SE_OK
            res[i] = (out, u, c)
        return res

    alone = run([7])
    mixed = run(list(range(n)))
    for j in range(3):
        np.testing.assert_array_equal(alone[7][j], mixed[7][j])
    assert p.info().get("columns") == "f16x3"
    phi = np.ascontiguousarray(dic, dtype=np.float64)
    dup = O.find_duplicates(phi)
    s = np.stack(samples)
    w = np.stack([O.weights(L, L, 0.8, m) for m in masks])
    ro, ru, rc, rm, st = O.se_original_batch(phi, w, s, 0.5, max(iters), dup, iters=np.asarray(iters),
                                             margins=True)
    assert st == 0
    for i in range(n):
        t = first_near_tie(rm[i, :iters[i]], 1e-4)
        np.testing.assert_array_equal(mixed[i][1][:t], ru[i, :t])
        if t:
            assert coef_rel_err(mixed[i][2][:t], rc[i, :t]).max() <= 1e-3
    out = np.stack([mixed[i][0] for i in range(n)])
    loss = np.stack(masks) == 0
    assert abs(psnr(out, s, loss) - psnr(ro, s, loss)) <= 0.05
    p.close()
