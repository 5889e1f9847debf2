"""Autotuner, measured full-versus-lazy choice and CUDA graphs, on the GPU.

The autotuner may only choose between launches with identical results, so
every forced variant must reproduce the default bit for bit; the routing of
pattern blocks under SE_GRAM_AUTO must follow the ski-rental rule on the
measured costs; replayed graphs of the lazy rounds must give the same
results as direct launches.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2204_14194_gb300 import binding as B
from paper_2204_14194_gb300 import workloads as W
from helpers import coef_rel_err, first_near_tie

pytestmark = pytest.mark.gpu


def _ctx(force=None, tune_file=None):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    old = {k: os.environ.get(k) for k in ("SE_TUNE_FORCE", "SE_TUNE_FILE")}
    for k, v in (("SE_TUNE_FORCE", force), ("SE_TUNE_FILE", tune_file)):
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    try:
        return B.Context(0)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _run(ctx, plan, samples, masks=None, iters=None):
    n, M, N = samples.shape
    I = plan.iterations
    s = torch.from_numpy(samples).cuda()
    out = torch.empty_like(s)
    u = torch.full((n, I), -1, dtype=torch.int32, device="cuda")
    c = torch.full((n, I), float("nan"), dtype=torch.float64, device="cuda")
    if masks is None:
        plan.extrapolate_strided(s, out, u, c)
    else:
        m = torch.from_numpy(masks).cuda()
        plan.extrapolate_batch([{"samples": s[b], "support": m[b], "out": out[b], "sel_idx": u[b],
                                 "sel_coef": c[b], "iterations": int(iters[b]) if iters is not None else I}
                                for b in range(n)])
    ctx.sync()
    return out.cpu().numpy(), u.cpu().numpy(), c.cpu().numpy()


CASES = [
    # (name, M, basis, K, I, n, prec)
    ("dctwht32", 32, "dct_wht", 2048, 60, 200, "bf16x6"),   # transform schedule, iterate Kp 2048
    ("dctwht16", 16, "dct_wht", 512, 60, 300, "bf16x6"),    # transform schedule 16 x 16
    ("dct32", 32, "dct", 1024, 60, 200, "bf16x6"),         # parity classes at Kp 1024
    ("gauss32", 32, "numeric", 4096, 40, 300, "bf16x6"),    # GEMM tile, iterate Kp 4096
    ("dctwht64", 64, "dct_wht", 8192, 20, 40, "bf16x6"),    # iterate Kp 8192
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_forced_variants_are_bitwise_identical(case):
    name, L, basis, K, I, n, prec = case
    samples = np.stack([W.patch(L, 4000 + i) for i in range(n)])
    dic = W.gaussian_dictionary(K, L, L, 91) if basis == "numeric" else None
    res = []
    # variants 2 and 3 exist only for the projection GEMM (128 x 64 tiles, two
    # CTAs per SM); other keys take their last variant
    for v in (0, 1, 2, 3):
        ctx = _ctx(force=f"sep:={v},gemm_proj:={v},gemm_projg:={v},gemm_table:={v},iterate:={v},sym:={v},"
                         f"symr0:={v}")
        try:
            plan = ctx.plan(L, L, basis, K, 0.8, 0.5, I, prec=prec, dictionary=dic)
            res.append(_run(ctx, plan, samples))
            plan.close()
        finally:
            ctx.close()
    for r in res[1:]:
        for a, b in zip(res[0], r):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("n,I", [(300, 80), (4096, 80), (5, 33), (7, 1)])
def test_parity_class_iteration_variants_are_bitwise_identical(n, I):
    """Projections in registers, in shared memory, in tensor memory, and the
    last-updated class in registers with the rest in shared memory, each
    followed by the model kernel, and the last form evaluating the model of
    eq. 9 itself (variant 4): the same selections, coefficients and outputs,
    bit for bit."""
    samples = np.stack([W.patch(32, 7600 + i % 997) for i in range(n)])
    res = []
    for v in (0, 1, 2, 3, 4):
        ctx = _ctx(force=f"sym:={v}")
        try:
            plan = ctx.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, I, prec="bf16x6")
            assert plan.info().get("iterations") == "parity-classes"
            res.append(_run(ctx, plan, samples))
            plan.close()
        finally:
            ctx.close()
    for r in res[1:]:
        for x, y in zip(res[0], r):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("basis,K", [("dct_wht", 2048), ("dct", 1024), ("wht", 1024)])
def test_projection_variants_of_parity_plans_are_bitwise_identical(basis, K):
    """The two R0 kernels of a 32 x 32 parity-class plan (generic fold, 32 x 32
    tiles) give the same bits."""
    samples = np.stack([W.patch(32, 7000 + i) for i in range(300)])
    res = []
    os.environ["SE_R0_FFMA"] = "1"   # the fp32 kernels instead of the tensor-core one
    try:
        for v in (0, 1):
            ctx = _ctx(force=f"symr0:={v}")
            try:
                plan = ctx.plan(32, 32, basis, K, 0.8, 0.5, 50, prec="bf16x6")
                info = plan.info()
                assert info.get("iterations") == "parity-classes" and "projections" not in info
                res.append(_run(ctx, plan, samples))
                plan.close()
            finally:
                ctx.close()
    finally:
        os.environ.pop("SE_R0_FFMA", None)
    for r in res[1:]:
        for x, y in zip(res[0], r):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("basis,K", [("dct_wht", 2048), ("dct", 1024), ("wht", 1024)])
def test_tensor_core_projections_match_the_fp32_transforms(basis, K):
    """Split-TF32 tensor-core R0 (the 32 x 32 default) against the fp32 kernels:
    the same selections up to near ties, coefficients and outputs within the
    fp32 form's tolerance."""
    from helpers import coef_rel_err
    samples = np.stack([W.patch(32, 7300 + i) for i in range(300)])
    res = []
    for ffma in (False, True):
        if ffma:
            os.environ["SE_R0_FFMA"] = "1"
        try:
            ctx = _ctx()
            try:
                plan = ctx.plan(32, 32, basis, K, 0.8, 0.5, 60, prec="bf16x6")
                assert (plan.info().get("projections") == "split-tf32") != ffma
                res.append(_run(ctx, plan, samples))
                plan.close()
            finally:
                ctx.close()
        finally:
            os.environ.pop("SE_R0_FFMA", None)
    (o1, u1, c1), (o2, u2, c2) = res
    same = np.all(u1 == u2, axis=1)
    assert same.mean() >= 0.97, same.mean()
    for b in np.where(same)[0]:   # both within 1e-3 of the fp64 values
        assert coef_rel_err(c1[b], c2[b]).max() <= 2e-3
    d = np.abs(o1 - o2)[same]
    assert d.mean() <= 0.01 and d.max() <= 0.5, (d.mean(), d.max())


def test_autotuner_times_each_shape_once_and_persists(tmp_path):
    f = str(tmp_path / "tune.txt")
    # an asymmetric loss box: the general iteration kernel (whose launch shape
    # is tuned) runs instead of the parity-class one
    sup = np.ones((32, 32), dtype=np.uint8)
    sup[8:24, 9:25] = 0
    ctx = _ctx(tune_file=f)
    try:
        plan = ctx.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, 40, prec="bf16x6", support=sup)
        samples = np.stack([W.patch(32, 50 + i) for i in range(64)])
        r1 = _run(ctx, plan, samples)
        t1 = ctx.tuning_stats()["tunings"]
        assert t1 >= 2          # the transform schedule and the iteration kernel shape
        r2 = _run(ctx, plan, samples)
        assert ctx.tuning_stats()["tunings"] == t1
        for a, b in zip(r1, r2):
            np.testing.assert_array_equal(a, b)
        plan.close()
    finally:
        ctx.close()
    lines = open(f).read().split("\n")
    keys = [l.split()[0] for l in lines if l.strip()]
    assert any(k.startswith("sep:32x32") for k in keys)
    assert any(k.startswith("iterate:f32:2048") for k in keys)
    # a new context reads the choices back: nothing left to time
    ctx = _ctx(tune_file=f)
    try:
        plan = ctx.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, 40, prec="bf16x6", support=sup)
        _run(ctx, plan, samples)
        assert ctx.tuning_stats()["tunings"] == 0
        plan.close()
    finally:
        ctx.close()


def test_measured_costs_route_pattern_blocks():
    """After se_plan_autotune, a pattern batch without a built table goes to
    the lazy path exactly when the ski-rental rule says so, and both routes
    match the oracle."""
    ctx = _ctx()
    try:
        L, I = 16, 80
        plan = ctx.plan(L, L, "dct_wht", 512, 0.8, 0.5, I, prec="bf16x6")
        costs = plan.autotune(128)
        assert costs["table_ms"] > 0 and costs["full_ms_per_block"] > 0 and costs["lazy_ms_per_block"] > 0
        extra = costs["lazy_ms_per_block"] - costs["full_ms_per_block"]
        regret = 0.0   # extra cost of the pattern blocks served lazily since the last table build
        sup = W.centred_support(L, L)
        o = O
        phi = o.dict_dct_wht(L, L)
        dup = o.find_duplicates(phi)
        w = o.weights(L, L, 0.8, sup)
        for n in (1, 4096):
            plan.reset_tables()
            samples = np.stack([W.patch(L, 700 + i) for i in range(n)])
            builds0 = ctx.stats()["table_builds"]
            out, u, c = _run(ctx, plan, samples)
            built = ctx.stats()["table_builds"] > builds0
            expect_lazy = extra <= 0 or regret + n * extra < costs["table_ms"]
            assert built == (not expect_lazy), (n, costs, regret)
            regret = regret + n * extra if expect_lazy and extra > 0 else 0.0
            pick = np.arange(min(n, 6))
            ro, ru, rc, rm, st = o.se_original_batch(phi, w, samples[pick], 0.5, I, dup, margins=True)
            for i, b in enumerate(pick):
                t = first_near_tie(rm[i], 1e-4)
                np.testing.assert_array_equal(u[b, :t], ru[i, :t])
                assert coef_rel_err(c[b, :t], rc[i, :t]).max() <= 1e-3
            # costs were re-measured by the batch, so the next decision reads them again
            costs = plan.costs()
            extra = costs["lazy_ms_per_block"] - costs["full_ms_per_block"]
        plan.close()
    finally:
        ctx.close()


@pytest.mark.parametrize("basis,K", [("dct_wht", 512), ("numeric", 512)])
def test_graph_replay_matches_direct_launches(basis, K):
    L, n = 16, 48
    rng = np.random.default_rng(3)
    samples = np.stack([W.patch(L, 900 + i) for i in range(n)])
    masks = np.stack([W.rect_support(L, L, rng) if i % 2 else W.holes_support(L, L, rng) for i in range(n)])
    iters = rng.integers(20, 90, size=n)
    dic = W.gaussian_dictionary(K, L, L, 5) if basis == "numeric" else None
    ctx = _ctx()
    try:
        plan = ctx.plan(L, L, basis, K, 0.8, 0.5, 90, prec="bf16x6", dictionary=dic)
        ctx.set_graphs(False)
        direct = _run(ctx, plan, samples, masks, iters)
        ctx.set_graphs(True)
        g0 = ctx.tuning_stats()
        # a shape is run directly the first time, captured when it comes back, then replayed
        first = _run(ctx, plan, samples, masks, iters)
        g1 = ctx.tuning_stats()
        assert g1["graph_builds"] == g0["graph_builds"]
        second = _run(ctx, plan, samples, masks, iters)
        again = _run(ctx, plan, samples, masks, iters)
        g2 = ctx.tuning_stats()
        assert g2["graph_builds"] >= g0["graph_builds"] + 1
        assert g2["graph_replays"] >= g0["graph_replays"] + 1
        for ref in (first, second, again):
            for a, b in zip(direct, ref):
                np.testing.assert_array_equal(a, b)
        plan.close()
    finally:
        ctx.close()


def _mirrored_pattern(kind):
    """Symmetric 32 x 32 supports whose loss bounding boxes select each tile
    shape of the model kernel (16 x 8 tiles) and each form of the model in the
    iteration kernel: rows staged in the slots (square area, box from m0 = n0),
    rows read from global memory, or no fused form (more than two tiles)."""
    sup = np.ones((32, 32), dtype=np.uint8)
    if kind == "box8x8":        # one tile, staged rows
        sup[12:20, 12:20] = 0
    elif kind == "box16x16":    # two tiles, staged rows (the headline box)
        sup[8:24, 8:24] = 0
    elif kind == "box16x8":     # one tile, m0 != n0: rows from global memory
        sup[8:24, 12:20] = 0
    elif kind == "strip32x8":   # two tiles of 16 rows, rows from global memory
        sup[:, 12:20] = 0
    else:   # a centred box and four mirrored 2 x 2 holes: a 30 x 30 box, separate model kernel only
        sup[8:24, 8:24] = 0
        for r, c in ((1, 2), (2, 28)):
            for rr, cc in ((r, c), (30 - r, c), (r, 30 - c), (30 - r, 30 - c)):
                sup[rr:rr + 2, cc:cc + 2] = 0
    assert (sup == sup[::-1]).all() and (sup == sup[:, ::-1]).all()
    return sup


@pytest.mark.parametrize("kind", ["box8x8", "box16x16", "box16x8", "strip32x8", "holes"])
def test_iterations_with_the_model_in_one_kernel(kind):
    """The last-updated-class iterations that evaluate the model of eq. 9 in
    the same kernel (variant 4) give the bits of the same iterations followed
    by the tensor-core model kernel (variant 3) on every loss-box shape, and
    meet the oracle's bars (indices up to the first near tie at 1e-4,
    coefficients 1e-3, PSNR 0.05 dB).  Boxes of more than two output tiles
    keep the separate model kernel."""
    from helpers import OracleSetup, psnr
    sup = _mirrored_pattern(kind)
    n, I = 60, 70
    samples = np.stack([W.patch(32, 8100 + i) for i in range(n)])
    res, launches = [], []
    for v in (3, 4):
        ctx = _ctx(force=f"sym:={v}")
        try:
            plan = ctx.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, I, prec="bf16x6", support=sup)
            assert plan.info().get("iterations") == "parity-classes"
            _run(ctx, plan, samples)   # the table is built by the first call
            l0 = ctx.stats()["kernel_launches"]
            res.append(_run(ctx, plan, samples))
            launches.append(ctx.stats()["kernel_launches"] - l0)
            plan.close()
        finally:
            ctx.close()
    fused = kind != "holes"
    assert launches[1] == launches[0] - int(fused), launches   # no separate model kernel when fused
    for x, y in zip(res[0], res[1]):
        np.testing.assert_array_equal(x, y)
    out, u, c = res[1]
    o = OracleSetup("dct_wht", 32, 32, 0.8, sup, tables=False)
    ro, ru, rc, rm, st = O.se_original_batch(o.phi, o.w, samples, 0.5, I, o.dup, margins=True)
    assert st == 0
    for b in range(n):
        t = first_near_tie(rm[b], 1e-4)
        np.testing.assert_array_equal(u[b, :t], ru[b, :t])
        assert coef_rel_err(c[b, :t], rc[b, :t]).max() <= 1e-3
        np.testing.assert_array_equal(out[b][sup > 0], samples[b][sup > 0])
    loss = np.broadcast_to(sup == 0, out.shape)
    assert abs(psnr(out, samples, loss) - psnr(ro, samples, loss)) <= 0.05
