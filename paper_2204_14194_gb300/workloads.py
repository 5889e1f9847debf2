"""Seeded synthetic inputs for Selective Extrapolation workloads.

This module produces the *inputs* of the method and nothing else: sample
patches and images, concealment-block positions, support/loss masks and
numerically defined (Gaussian) dictionaries.  It holds none of the method's
arithmetic (no weighting function, no scalar products, no selection); both
the CUDA library and the CPU oracle consume what it returns.

The paper evaluates on natural images (the Kodak set, Sec. V, Table II) that
are not available here.  The generator below stands in for them: every tile
is a linear gradient plus two 2-D sinusoids plus one step edge, clipped to
the 8-bit range [0, 255] and kept as float64.  All randomness comes from
``numpy.random.default_rng`` (PCG64); tiles draw from independent streams
spawned from one ``SeedSequence``.

Mask convention (Sec. II, Fig. 2 and eq. 4): ``support[m, n] = 1`` marks a
sample of the support area A, ``0`` a sample of the loss area B.  Arrays are
row-major with ``m`` the row (vertical) and ``n`` the column (horizontal)
coordinate.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = [
    "patch", "tiled_image", "centred_support", "rect_support",
    "holes_support", "gaussian_dictionary", "Workload", "config1",
    "config2", "config3", "config4", "extract_blocks",
]


def _draw_patch(rng: np.random.Generator, L: int, rows: np.ndarray,
                cols: np.ndarray) -> np.ndarray:
    """One generator draw evaluated on the pixel grid ``rows x cols``.

    ``rows``/``cols`` are pixel coordinates local to the tile whose side is
    ``L``; the random parameters are drawn in a fixed order so that a tile is
    reproducible from its stream alone.
    """
    base = rng.uniform(64.0, 192.0)
    gx, gy = rng.uniform(-1.0, 1.0, size=2) * 64.0 / L
    amps = rng.uniform(10.0, 40.0, size=2)
    freqs = rng.uniform(-0.25, 0.25, size=(2, 2))     # (fx, fy) cycles/px
    phases = rng.uniform(0.0, 2.0 * np.pi, size=2)
    theta = rng.uniform(0.0, np.pi)
    px, py = rng.uniform(0.0, L, size=2)
    height = rng.uniform(-60.0, 60.0)

    y = rows[:, None].astype(np.float64)
    x = cols[None, :].astype(np.float64)
    c = (L - 1) / 2.0
    v = base + gx * (x - c) + gy * (y - c)
    for i in range(2):
        v = v + amps[i] * np.sin(2.0 * np.pi * (freqs[i, 0] * x + freqs[i, 1] * y)
                                 + phases[i])
    side = (x - px) * np.cos(theta) + (y - py) * np.sin(theta)
    v = v + np.where(side >= 0.0, height, 0.0)
    return np.clip(v, 0.0, 255.0)


def patch(L: int, seed: int) -> np.ndarray:
    """A single ``L x L`` float64 patch from one generator draw."""
    rng = np.random.default_rng(seed)
    g = np.arange(L)
    return _draw_patch(rng, L, g, g)


def tiled_image(height: int, width: int, seed: int, tile: int = 64) -> np.ndarray:
    """A ``height x width`` float64 image built from independent ``tile``-sized draws.

    Tiles are laid out row-major; tile ``t`` draws from the ``t``-th child of
    ``SeedSequence(seed)``.  The seams between tiles add further edges.
    """
    ty = -(-height // tile)
    tx = -(-width // tile)
    children = np.random.SeedSequence(seed).spawn(ty * tx)
    img = np.empty((ty * tile, tx * tile), dtype=np.float64)
    g = np.arange(tile)
    for t in range(ty * tx):
        r, c = divmod(t, tx)
        rng = np.random.default_rng(children[t])
        img[r * tile:(r + 1) * tile, c * tile:(c + 1) * tile] = _draw_patch(rng, tile, g, g)
    return np.ascontiguousarray(img[:height, :width])


def centred_support(M: int, N: int) -> np.ndarray:
    """Support mask with the centred ``M/2 x N/2`` loss area (rows/cols M/4..3M/4-1)."""
    s = np.ones((M, N), dtype=np.uint8)
    s[M // 4: M // 4 + M // 2, N // 4: N // 4 + N // 2] = 0
    return s


def rect_support(M: int, N: int, rng: np.random.Generator) -> np.ndarray:
    """One ``M/2 x N/2`` loss rectangle at a uniform offset with >= M/8 support margin."""
    s = np.ones((M, N), dtype=np.uint8)
    hm, hn = M // 2, N // 2
    mm, mn = M // 8, N // 8
    r0 = int(rng.integers(mm, M - mm - hm + 1))
    c0 = int(rng.integers(mn, N - mn - hn + 1))
    s[r0:r0 + hm, c0:c0 + hn] = 0
    return s


def holes_support(M: int, N: int, rng: np.random.Generator) -> np.ndarray:
    """``M*N/64`` distinct 4x4 holes on the 4-aligned grid (a quarter of the area lost)."""
    s = np.ones((M, N), dtype=np.uint8)
    cells = (M // 4) * (N // 4)
    n_holes = (M * N) // 64
    picks = rng.choice(cells, size=n_holes, replace=False)
    for p in picks:
        r, c = divmod(int(p), N // 4)
        s[4 * r:4 * r + 4, 4 * c:4 * c + 4] = 0
    return s


def video_block(M: int, N: int, T: int, seed: int) -> np.ndarray:
    """A ``T x M x N`` (frame-major) float64 block of a moving scene: frame t is
    the ``M x N`` window at offset (t*vy, t*vx) of one larger generator draw,
    with a velocity (vy, vx) in {0, 1, 2}^2 pixels per frame drawn from the seed."""
    rng = np.random.default_rng(seed)
    vy, vx = (int(v) for v in rng.integers(0, 3, size=2))
    L = max(M, N) + 2 * T + 2
    big = patch(L, seed + 7919)
    return np.stack([big[t * vy:t * vy + M, t * vx:t * vx + N] for t in range(T)])


def centred_support3(M: int, N: int, T: int) -> np.ndarray:
    """Frame-major ``T x M x N`` support with the centred loss box of
    ``M/2 x N/2`` pixels in frames T/4 .. T/4 + max(T/2, 1) - 1 (for T = 1
    this is ``centred_support``)."""
    s = np.ones((T, M, N), dtype=np.uint8)
    t0, nt = T // 4, max(T // 2, 1)
    s[t0:t0 + nt, M // 4: M // 4 + M // 2, N // 4: N // 4 + N // 2] = 0
    return s


def gaussian_dictionary(K: int, M: int, N: int, seed: int) -> np.ndarray:
    """``K`` i.i.d. N(0,1) atoms of size ``M x N`` (atom-major), each of unit l2 norm over L."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((K, M * N))
    d /= np.sqrt(np.sum(d * d, axis=1, keepdims=True))
    return d.reshape(K, M, N)


def extract_blocks(img: np.ndarray, tops: np.ndarray, lefts: np.ndarray,
                   M: int, N: int) -> np.ndarray:
    """Copy the ``M x N`` areas with the given top-left corners into a ``[B, M, N]`` array."""
    B = len(tops)
    out = np.empty((B, M, N), dtype=np.float64)
    for b in range(B):
        out[b] = img[tops[b]:tops[b] + M, lefts[b]:lefts[b] + N]
    return out


@dataclass
class Workload:
    """A batch of concealment blocks that share one extrapolation-area size."""
    name: str
    M: int
    N: int
    basis: str                      # "dct", "wht", "dct_wht" or "numeric"
    K: int
    iterations: int
    gamma: float
    rho_hat: float
    samples: np.ndarray             # [B, M, N] float64 ground truth
    support: np.ndarray             # [M, N] uint8 shared pattern, or [B, M, N] per block
    dictionary: Optional[np.ndarray] = None   # [K, M, N] float64 for "numeric"
    iters_per_block: Optional[np.ndarray] = None
    psnr_mask: Optional[np.ndarray] = None    # [B, M, N] bool: loss pixels inside the image
    meta: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return int(self.samples.shape[0])


def config1() -> Workload:
    """One 32x32 patch (seed 1), centred 16x16 loss, K=2048 DCT u WHT, I=100, gamma=0.5, rho=0.8."""
    s = patch(32, 1)[None]
    return Workload("single_32x32_dctwht_K2048_I100", 32, 32, "dct_wht", 2048, 100,
                    0.5, 0.8, s, centred_support(32, 32))


def config2(n_blocks: int = 4096) -> Workload:
    """512x512 tiled image (seed 2); 32x32 areas at uniform corners in [0,480]^2 (seed 102)."""
    img = tiled_image(512, 512, 2)
    rng = np.random.default_rng(102)
    corners = rng.integers(0, 481, size=(4096, 2))
    corners = corners[:n_blocks]
    s = extract_blocks(img, corners[:, 0], corners[:, 1], 32, 32)
    return Workload("img512_4096blk_32x32_dctwht_K2048_I100", 32, 32, "dct_wht", 2048, 100,
                    0.5, 0.8, s, centred_support(32, 32), meta={"corners": corners})


def config3(n_blocks: Optional[int] = None) -> Workload:
    """1920x1080 image: its 16x16 grid of loss regions (120 x 68 = 8160 blocks), 32x32 areas.

    The canvas covers rows -8..1095 and columns -8..1927 so that every area
    extends 8 px around its loss region and all masks coincide.  Dictionary:
    K=4096 Gaussian atoms (seed 1003), I=200.
    """
    H, W, pad = 1080, 1920, 8
    canvas = tiled_image(H + 8 + pad * 2, W + pad * 2, 3)   # 1104 x 1936
    gy, gx = 68, 120
    tops = np.repeat(np.arange(gy) * 16, gx)
    lefts = np.tile(np.arange(gx) * 16, gy)
    if n_blocks is not None:
        tops, lefts = tops[:n_blocks], lefts[:n_blocks]
    s = extract_blocks(canvas, tops, lefts, 32, 32)
    # loss pixels of block (r, c) are canvas rows 16r+8..16r+23 == image rows 16r..16r+15
    psnr = np.zeros(s.shape, dtype=bool)
    for b in range(len(tops)):
        img_rows = tops[b] + np.arange(32) - pad
        inside = (img_rows >= 0) & (img_rows < H)
        psnr[b] = inside[:, None] & np.ones((1, 32), dtype=bool)
    psnr &= (centred_support(32, 32) == 0)[None]
    return Workload("img1920x1080_8160blk_32x32_gauss_K4096_I200", 32, 32, "numeric", 4096,
                    200, 0.5, 0.8, s, centred_support(32, 32),
                    dictionary=gaussian_dictionary(4096, 32, 32, 1003), psnr_mask=psnr)


def config4(n_blocks: int = 20000, seed: int = 4) -> List[Workload]:
    """Mixed areas 16/32/64 (K = 2MN, DCT u WHT), per-block masks, I uniform in [50, 500].

    Returns one ``Workload`` per area size (the thirds of the mix); masks are
    per block, half a random (M/2 x N/2) rectangle and half scattered 4x4 holes.
    """
    ss = np.random.SeedSequence(seed)
    child_masks, child_iters, child_patches = ss.spawn(3)
    thirds = [n_blocks // 3 + (1 if i < n_blocks % 3 else 0) for i in range(3)]
    rng_m = np.random.default_rng(child_masks)
    rng_i = np.random.default_rng(child_iters)
    pseeds = child_patches.spawn(n_blocks)
    out = []
    j = 0
    for L, nb in zip((16, 32, 64), thirds):
        samples = np.empty((nb, L, L))
        masks = np.empty((nb, L, L), dtype=np.uint8)
        for b in range(nb):
            rng = np.random.default_rng(pseeds[j])
            g = np.arange(L)
            samples[b] = _draw_patch(rng, L, g, g)
            masks[b] = rect_support(L, L, rng_m) if (b % 2 == 0) else holes_support(L, L, rng_m)
            j += 1
        iters = rng_i.integers(50, 501, size=nb)
        out.append(Workload(f"mixed_{L}x{L}_dctwht_K{2 * L * L}", L, L, "dct_wht", 2 * L * L,
                            int(iters.max()), 0.5, 0.8, samples, masks,
                            iters_per_block=iters))
    return out
