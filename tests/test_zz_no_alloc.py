"""se_extrapolate_noalloc, the entry point for callers that cannot allocate.

Such callers (a real-time loop that forbids allocation after start-up, or a
host that hands the library only its own input and output buffers) get the
strided batch computation with all per-call scratch in the library's static
device array.  This checks, through the C ABI, that two calls in a row give
the same results as se_extrapolate_strided within the parity tolerances, on
every form the call can take (parity-class, separable fp32 on a non-symmetric
pattern, separable fp64, dense split-bf16 tensor-core and dense fp64
products), that the second call leaves the device's free memory unchanged,
and that a batch larger than the static scratch is refused before any
launch.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2204_14194_gb300 import binding as B
from paper_2204_14194_gb300 import workloads as W

pytestmark = pytest.mark.gpu

COEF_TOL = {"bf16x6": 1e-3, "fp64": 1e-9}


def _shifted_support():
    """A 16 x 16 loss area off the centre: the weighting is not symmetric, so the
    plan takes the general separable fp32 kernels instead of the parity classes."""
    sup = np.ones((32, 32), dtype=np.uint8)
    sup[6:22, 10:26] = 0
    return sup


CASES = [
    ("bf16x6", 512, "auto", False),      # parity-class kernels (centred pattern)
    ("fp64", 300, "auto", False),        # separable transforms in fp64
    ("bf16x6", 256, "auto", True),       # separable fp32 transforms, general kernels
    ("bf16x6", 256, "dense", False),     # split-bf16 tcgen05 projections
    ("fp64", 128, "dense", False),       # fp64 matrix products
]


@pytest.mark.parametrize("prec,n,products,shifted", CASES)
def test_noalloc_matches_strided_on_two_calls(prec, n, products, shifted):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = B.Context(0)
    try:
        wl = W.config2(n)
        sup = _shifted_support() if shifted else None
        plan = ctx.plan(32, 32, "dct_wht", 2048, wl.rho_hat, wl.gamma, 100, prec=prec,
                        products=products, support=sup)
        if shifted:
            assert plan.info().get("iterations") != "parity-classes"
        s = torch.from_numpy(wl.samples).cuda()
        ref_o = torch.empty_like(s)
        ref_u = torch.empty((n, 100), dtype=torch.int32, device="cuda")
        ref_c = torch.empty((n, 100), dtype=torch.float64, device="cuda")
        plan.extrapolate_strided(s, ref_o, ref_u, ref_c)
        ctx.sync()
        ro, ru, rc = ref_o.cpu().numpy(), ref_u.cpu().numpy(), ref_c.cpu().numpy()
        loss = (wl.support if sup is None else sup) == 0
        for call in range(2):
            o = torch.full_like(s, float("nan"))
            u = torch.full((n, 100), -1, dtype=torch.int32, device="cuda")
            c = torch.full((n, 100), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            plan.extrapolate_noalloc(s, o, u, c)
            ctx.sync()
            free1 = torch.cuda.mem_get_info()[0]
            if call == 1:   # kernels are loaded by now: the call itself allocates nothing
                assert free1 == free0, (free0, free1)
            on, un, cn = o.cpu().numpy(), u.cpu().numpy(), c.cpu().numpy()
            np.testing.assert_array_equal(un, ru)
            rel = np.abs(cn - rc) / np.maximum(np.abs(rc), 1e-12 * np.abs(rc).max())
            assert rel.max() <= COEF_TOL[prec]
            np.testing.assert_array_equal(on[:, ~loss], wl.samples[:, ~loss])
            np.testing.assert_allclose(on[:, loss], ro[:, loss], rtol=1e-6, atol=1e-6)
        plan.close()
    finally:
        ctx.close()


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ctx = B.Context(0)
    try:
        plan = ctx.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, 100, prec="bf16x6")
        s = torch.zeros((4096, 32, 32), dtype=torch.float64, device="cuda")
        o = torch.empty_like(s)
        with pytest.raises(B.SeError) as e:
            plan.extrapolate_noalloc(s, o)
        assert e.value.status == -1
        assert "16 MiB" in str(e.value)
        plan.close()
        # argument errors are reported whatever the batch size, n = 0 included
        cert = ctx.plan(32, 32, "dct_wht", 2048, 0.8, 0.5, 100, prec="certified")
        with pytest.raises(B.SeError) as e:
            cert.extrapolate_noalloc(s[:0], o[:0])
        assert e.value.status == -1
        cert.close()
    finally:
        ctx.close()
