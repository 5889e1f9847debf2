"""The projection kernels' fp64 -> fp32 sample conversion (and the model
kernels' fp32 -> fp64 widening of the results), bit for bit.

In the fp32 form the samples enter eq. (12) rounded to fp32.  The kernels
round them on the integer pipe (cut the significand, round to nearest with
ties to even, carry into the exponent) and keep the hardware conversion for
the values whose result is not a normal float.  This compares the library's
conversion, through the C ABI, with numpy's IEEE 754 conversion on the CPU
and with torch's conversion on the GPU, on pixel values, random bit patterns
of every exponent, and the edge cases: exact ties, one ulp either side of a
tie, carries into the exponent, the overflow boundary, subnormal results,
zeros, infinities and NaNs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2204_14194_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _edge_cases():
    f = np.float32
    vals = [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 255.0, 0.5, 1e-300, -1e-300, 1e300, -1e300,
            float(np.finfo(f).max), float(np.finfo(f).tiny), float(np.finfo(f).smallest_subnormal)]
    out = list(vals)
    rng = np.random.default_rng(11)
    # floats of every binade, and the doubles half an ulp away (exact ties), one
    # double ulp either side of the tie, and the largest value below the next float
    for e in range(-149, 128):
        m = rng.integers(0, 1 << 23, size=4)
        for mm in m:
            x = np.ldexp(float((1 << 23) + int(mm)), e - 23) if e >= -126 else np.ldexp(float(mm), -149)
            if not np.isfinite(x):
                continue
            ulp = np.ldexp(1.0, max(e, -126) - 23)
            for v in (x, x + ulp / 2, x - ulp / 2, np.nextafter(x + ulp / 2, np.inf),
                      np.nextafter(x + ulp / 2, -np.inf), np.nextafter(x + ulp, -np.inf)):
                out += [v, -v]
    # significands of all ones: rounding up carries into the exponent
    for e in (-126, -1, 0, 7, 127):
        x = np.ldexp(float((1 << 24) - 1), e - 23)
        out += [x, x + np.ldexp(1.0, e - 24), np.nextafter(x + np.ldexp(1.0, e - 24), np.inf)]
    # the overflow boundary: max float plus half an ulp rounds to infinity
    mx = float(np.finfo(f).max)
    half = np.ldexp(1.0, 127 - 24)
    out += [mx + half, np.nextafter(mx + half, -np.inf), np.nextafter(mx + half, np.inf), -(mx + half)]
    return np.array(out, dtype=np.float64)


def _inputs():
    rng = np.random.default_rng(12)
    pixels = rng.uniform(0.0, 255.0, size=1 << 18)
    bits = rng.integers(0, np.iinfo(np.uint64).max, size=1 << 18, dtype=np.uint64, endpoint=True)
    random_bits = bits.view(np.float64)
    # the exponent range where the integer path applies, densely
    e = rng.integers(-126, 128, size=1 << 18)
    dense = np.ldexp(rng.uniform(1.0, 2.0, size=1 << 18), e) * rng.choice([-1.0, 1.0], size=1 << 18)
    return np.concatenate([_edge_cases(), pixels, random_bits, dense])


def test_sample_conversion_is_ieee_round_to_nearest_even():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    x = _inputs()
    ctx = B.Context(0)
    try:
        xd = torch.from_numpy(x).cuda()
        out = torch.full(x.shape, float("nan"), dtype=torch.float32, device="cuda")
        back = torch.full(x.shape, float("nan"), dtype=torch.float64, device="cuda")
        ctx.check_sample_conversion(xd, out, back)
        ctx.sync()
        got = out.cpu().numpy()
        # the widening of the results back to fp64 is exact
        wide = back.cpu().numpy()
        fin = ~np.isnan(got)
        np.testing.assert_array_equal(np.isnan(wide), ~fin)
        np.testing.assert_array_equal(wide[fin].view(np.uint64), got[fin].astype(np.float64).view(np.uint64))
        with np.errstate(over="ignore"):
            want = x.astype(np.float32)
        hw = xd.to(torch.float32).cpu().numpy()
        nan = np.isnan(want)
        np.testing.assert_array_equal(np.isnan(got), nan)
        np.testing.assert_array_equal(got[~nan].view(np.uint32), want[~nan].view(np.uint32))
        np.testing.assert_array_equal(got[~nan].view(np.uint32), hw[~nan].view(np.uint32))
    finally:
        ctx.close()
