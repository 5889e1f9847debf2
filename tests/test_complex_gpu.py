"""Complex-valued atoms on the GPU (DFT, binarised DFT, their union).

The library forms the Hermitian table and the projections from real GEMMs
of stacked real/imaginary rows and iterates on complex R_k; the oracle is
the complex Alg. 1 with its own atoms.  Same bars as the real parity tests:
index sequence up to the first near tie, complex coefficients within 1e-9
(fp64 form) / 1e-3 (split-bf16 form), PSNR of the real output within 0.05 dB.
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


@pytest.mark.parametrize("L,basis,n,I", [(16, "dft", 16, 60), (16, "bdft", 16, 60), (16, "dft_bdft", 16, 60),
                                         (32, "dft", 16, 60),
                                         (32, "dft_bdft", 6, 50),   # K = 2048: four warps per block
                                         (64, "dft", 2, 25)])       # K = 4096, DFT of w instead of a table
@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_complex_atoms_against_the_oracle(ctx, L, basis, n, I, prec):
    K = (2 if basis == "dft_bdft" else 1) * L * L
    samples = np.stack([W.patch(L, 8000 + 31 * L + i) for i in range(n)])
    sup = W.centred_support(L, L)
    plan = ctx.plan(L, L, basis, K, 0.8, 0.5, I, prec=prec)
    s = torch.from_numpy(samples).cuda()
    out = torch.empty_like(s)
    u = torch.full((n, I), -1, dtype=torch.int32, device="cuda")
    c = torch.full((n, I, 2), float("nan"), dtype=torch.float64, device="cuda")
    plan.extrapolate_strided(s, out, u, c)
    ctx.sync()
    out, u, c = out.cpu().numpy(), u.cpu().numpy(), c.cpu().numpy()
    cz = c[..., 0] + 1j * c[..., 1]

    phi = O.dict_complex(basis, L, L)
    # DFT atoms are orthonormal, so none is collinear with another (pinned on
    # the CPU); the pairwise search is only needed with binarised atoms
    dup = np.zeros(K, dtype=np.uint8) if basis == "dft" else O.find_duplicates_c(phi)
    w = O.weights(L, L, 0.8, sup)
    ro, ru, rc, rm, st = O.se_original_c_batch(phi, w, samples, 0.5, I, dup, margins=True)
    assert st == 0
    tau, ctol = TOL[prec]
    for b in range(n):
        t = first_near_tie(rm[b], tau)
        np.testing.assert_array_equal(u[b, :t], ru[b, :t])
        if t:
            assert coef_rel_err(cz[b, :t], rc[b, :t]).max() <= ctol
        assert not np.any(dup[u[b]])               # excluded (collinear) atoms are never selected
    np.testing.assert_array_equal(out[:, sup > 0], samples[:, sup > 0])
    loss = np.broadcast_to(sup == 0, out.shape)
    assert abs(psnr(out, samples, loss) - psnr(ro, samples, loss)) <= 0.05
    plan.close()


def test_complex_plan_limits(ctx):
    with pytest.raises(B.SeError):
        ctx.plan(16, 16, "dft", 300, 0.8, 0.5, 10)                      # K must be MN
    with pytest.raises(B.SeError):
        ctx.plan(16, 16, "dft", 256, 0.8, 0.5, 10, prec="certified")
    with pytest.raises(B.SeError):
        ctx.plan(16, 16, "dft", 256, 0.8, 0.5, 10, gram="lazy")
    p = ctx.plan(16, 16, "dft", 256, 0.8, 0.5, 10)
    s = torch.from_numpy(W.patch(16, 1)[None].copy()).cuda()
    m = torch.from_numpy(W.centred_support(16, 16)).cuda()
    o = torch.empty_like(s)
    with pytest.raises(B.SeError):
        p.extrapolate_batch([{"samples": s[0], "support": m, "out": o[0]}])
    p.close()
