"""Seeded synthetic inputs for three-quarter sampling reconstruction.

This module only *draws* test inputs: high-resolution images, L-pixel
opaque-quadrant masks, and the sensor measurement that turns one into
low-resolution L-pixel values (Sec. II, Eq. 1: each L-pixel integrates the
three transparent high-resolution sub-pixels of its 2x2 footprint).  It holds
none of the reconstruction arithmetic and imports nothing else from this
package, so both the CPU oracle and the CUDA path can take their inputs from
here.

The paper evaluates on 100 natural 1200x1200 images (Sec. V-A), which are not
available; the images drawn here stand in for them:

* ``S`` 2-D sinusoids with per-axis frequency ~ U(-0.5, 0.5) cycles per HR
  pixel (up to HR Nyquist), phase ~ U(0, 2 pi), amplitude ~ U(0, 1);
* ``E`` straight step edges through a uniform point with direction
  ~ U(0, pi) and height ~ U(-1, 1) * mean sinusoid amplitude;
* min-max normalisation to [0, 1], optional Gaussian noise ``sigma``,
  clipping to [0, 1].

Masks hold one code per LR pixel, the index of its opaque quadrant:
0 = top-left, 1 = top-right, 2 = bottom-left, 3 = bottom-right.  A recurrent
mask tiles a ``T x T`` LR tile drawn uniformly from {0..3} (Sec. V-A uses a
random pattern repeating every 32 HR pixels, i.e. T = 16); a non-recurrent
mask draws every LR pixel independently.

Other sensor layouts (Sec. I: any periodically repeating layout) use
aperture codes instead: the set of transparent sub-pixels of each L-pixel,
bit ``2 * dy + dx`` for the sub-pixel at row offset dy, column offset dx.
Three-quarter sampling is the aperture ``15 ^ (1 << opaque)``, quarter
sampling a single bit, a regular LR sensor the full aperture 15.

All randomness comes from numpy's PCG64 generator, whose streams are the same
on every platform.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "image", "recurrent_mask", "random_mask", "measure", "workload",
    "batch_sizes", "OPAQUE_OFFSETS", "image_torch", "measure_torch",
    "APERTURE_SETS", "aperture_mask", "apertures_of", "workload_config",
]

# Named aperture sets for recurrent layouts other than three-quarter
# sampling (codes: bit 2 * dy + dx = transparent sub-pixel).
APERTURE_SETS = {
    "three_quarter": (14, 13, 11, 7),
    "quarter": (1, 2, 4, 8),
    "pairs": (3, 12, 5, 10),            # horizontal and vertical sub-pixel pairs
    "mixed": (1, 6, 13, 15),            # quarter, diagonal pair, three-quarter, full
    # every aperture symmetric under transposition: the atoms of (k1, k2) and
    # (k2, k1) coincide on every measurement when k1 - k2 = 16 (mod 32), so
    # those candidates tie exactly and only the tie rule separates them
    "symmetric": (1, 6, 14, 15),
    "all": tuple(range(1, 16)),         # every non-empty aperture
}

# (row, col) offset of the opaque sub-pixel inside the 2x2 footprint, by code.
OPAQUE_OFFSETS = ((0, 0), (0, 1), (1, 0), (1, 1))


def image(h: int, w: int, n_sin: int, n_edges: int, seed: int,
          sigma: float = 0.0) -> np.ndarray:
    """Return an ``h x w`` float64 image in [0, 1] drawn from ``seed``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fy = rng.uniform(-0.5, 0.5, n_sin)
    fx = rng.uniform(-0.5, 0.5, n_sin)
    ph = rng.uniform(0.0, 2.0 * np.pi, n_sin)
    amp = rng.uniform(0.0, 1.0, n_sin)
    yy = np.arange(h, dtype=np.float64)
    xx = np.arange(w, dtype=np.float64)
    # sin(2pi fy y + 2pi fx x + ph) = sin(a_y) cos(b_x) + cos(a_y) sin(b_x)
    ay = 2.0 * np.pi * np.outer(yy, fy) + ph[None, :]          # h x S
    bx = 2.0 * np.pi * np.outer(fx, xx)                         # S x w
    left = np.concatenate([np.sin(ay) * amp, np.cos(ay) * amp], axis=1)
    right = np.concatenate([np.cos(bx), np.sin(bx)], axis=0)
    img = left @ right
    mean_amp = float(amp.mean()) if n_sin else 1.0
    py = rng.uniform(0.0, h, n_edges)
    px = rng.uniform(0.0, w, n_edges)
    th = rng.uniform(0.0, np.pi, n_edges)
    hgt = rng.uniform(-1.0, 1.0, n_edges) * mean_amp
    for e in range(n_edges):
        ny, nx = np.sin(th[e]), np.cos(th[e])
        side = (yy[:, None] - py[e]) * ny + (xx[None, :] - px[e]) * nx > 0.0
        img += hgt[e] * side
    lo, hi = img.min(), img.max()
    img = (img - lo) / (hi - lo) if hi > lo else np.zeros_like(img)
    if sigma > 0.0:
        img = img + rng.normal(0.0, sigma, img.shape)
    return np.clip(img, 0.0, 1.0)


def image_torch(h: int, w: int, n_sin: int, n_edges: int, seed: int, sigma: float = 0.0,
                device: str = "cuda"):
    """The recipe of :func:`image` drawn with torch's generator on ``device``
    (for bulk training data; the values differ from :func:`image`'s)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))

    def u(n):
        return torch.rand(n, generator=g, device=device, dtype=torch.float64)

    fy, fx, ph, amp = u(n_sin) - 0.5, u(n_sin) - 0.5, 2.0 * np.pi * u(n_sin), u(n_sin)
    yy = torch.arange(h, device=device, dtype=torch.float64)
    xx = torch.arange(w, device=device, dtype=torch.float64)
    ay = 2.0 * np.pi * torch.outer(yy, fy) + ph[None, :]
    bx = 2.0 * np.pi * torch.outer(fx, xx)
    img = torch.cat([torch.sin(ay) * amp, torch.cos(ay) * amp], 1) @ torch.cat([torch.cos(bx), torch.sin(bx)], 0)
    mean_amp = float(amp.mean()) if n_sin else 1.0
    py, px, th = h * u(n_edges), w * u(n_edges), np.pi * u(n_edges)
    hgt = (2.0 * u(n_edges) - 1.0) * mean_amp
    for e in range(n_edges):
        side = (yy[:, None] - py[e]) * torch.sin(th[e]) + (xx[None, :] - px[e]) * torch.cos(th[e]) > 0.0
        img = img + hgt[e] * side
    lo, hi = img.min(), img.max()
    img = (img - lo) / (hi - lo) if float(hi) > float(lo) else torch.zeros_like(img)
    if sigma > 0.0:
        img = img + sigma * torch.randn(img.shape, generator=g, device=device, dtype=torch.float64)
    return img.clamp(0.0, 1.0)


def measure_torch(f, mask):
    """:func:`measure` for torch tensors (f: HR image, mask: LR codes)."""
    import torch
    lr_h, lr_w = mask.shape
    q = f[: 2 * lr_h, : 2 * lr_w].reshape(lr_h, 2, lr_w, 2).permute(0, 2, 1, 3).reshape(lr_h, lr_w, 4)
    opaque = torch.gather(q, 2, mask.long()[..., None])[..., 0]
    return q.sum(2) - opaque


def recurrent_mask(lr_h: int, lr_w: int, tile: int, seed: int) -> np.ndarray:
    """Opaque-quadrant codes of a ``tile x tile`` LR tile repeated periodically."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = rng.integers(0, 4, (tile, tile), dtype=np.uint8)
    reps = (-(-lr_h // tile), -(-lr_w // tile))
    return np.ascontiguousarray(np.tile(t, reps)[:lr_h, :lr_w])


def random_mask(lr_h: int, lr_w: int, seed: int) -> np.ndarray:
    """Independent opaque-quadrant code per LR pixel (a non-recurrent sensor)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 4, (lr_h, lr_w), dtype=np.uint8)


def aperture_mask(lr_h: int, lr_w: int, tile: int, seed: int, codes) -> np.ndarray:
    """Aperture codes of a ``tile x tile`` LR tile, each drawn uniformly from
    ``codes``, repeated periodically (``tile=0``: no repetition)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    codes = np.asarray(codes, dtype=np.uint8)
    if tile <= 0:
        return np.ascontiguousarray(codes[rng.integers(0, len(codes), (lr_h, lr_w))])
    t = codes[rng.integers(0, len(codes), (tile, tile))]
    reps = (-(-lr_h // tile), -(-lr_w // tile))
    return np.ascontiguousarray(np.tile(t, reps)[:lr_h, :lr_w])


def apertures_of(mask: np.ndarray) -> np.ndarray:
    """Aperture codes of an opaque-quadrant mask."""
    return (15 ^ (1 << mask.astype(np.uint8))).astype(np.uint8)


def measure(f: np.ndarray, mask: np.ndarray, layout: int = 0) -> np.ndarray:
    """Simulate the sensor of Eq. 1 (coefficients 1, a sum).

    ``y[p, q]`` is the sum of the transparent HR sub-pixels of the footprint
    ``f[2p:2p+2, 2q:2q+2]``: with ``layout=0`` ``mask[p, q]`` names the one
    opaque sub-pixel, with ``layout=1`` it is the aperture bit set.
    """
    lr_h, lr_w = mask.shape
    f = np.asarray(f, dtype=np.float64)[: 2 * lr_h, : 2 * lr_w]
    quad = f.reshape(lr_h, 2, lr_w, 2).transpose(0, 2, 1, 3).reshape(lr_h, lr_w, 4)
    if layout == 1:
        bits = (mask[..., None].astype(np.int64) >> np.arange(4)) & 1
        return (quad * bits).sum(axis=2)
    total = quad.sum(axis=2)
    opaque = np.take_along_axis(quad, mask[..., None].astype(np.int64), axis=2)[..., 0]
    return total - opaque


def batch_sizes(n: int, seed: int, lo=(256, 256), hi=(1536, 2048), mult: int = 8):
    """Uneven image sizes (h, w), multiples of ``mult``, drawn by ``seed``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hs = rng.integers(lo[0] // mult, hi[0] // mult + 1, n) * mult
    ws = rng.integers(lo[1] // mult, hi[1] // mult + 1, n) * mult
    return [(int(a), int(b)) for a, b in zip(hs, ws)]


# Workloads shaped like the paper's (Sec. V) at the sizes this library is
# measured on.  Each entry: HR size (h, w), sinusoids, edges, noise sigma,
# LR tile of the recurrent mask, image seed, mask seed.
_WORKLOADS = {
    "rljsde_64x64":      dict(h=64,   w=64,   n_sin=32,   n_edges=4,   sigma=0.0,   tile=4, seed=1000, mseed=8),
    "rljsde_1024x1024":  dict(h=1024, w=1024, n_sin=256,  n_edges=32,  sigma=0.005, tile=4, seed=2000, mseed=9),
    "rljsde_4096x3072":  dict(h=3072, w=4096, n_sin=2048, n_edges=256, sigma=0.0,   tile=8, seed=3000, mseed=10),
    "rljsde_4096x3072_t4": dict(h=3072, w=4096, n_sin=2048, n_edges=256, sigma=0.0,  tile=4, seed=5000, mseed=12),
    "rljsde_1200x1200":  dict(h=1200, w=1200, n_sin=256,  n_edges=32,  sigma=0.005, tile=16, seed=6000, mseed=13),
}


def workload_config(name: str) -> dict:
    """Recipe of a named workload: HR size, sinusoids, edges, noise, LR mask
    tile and seeds."""
    return dict(_WORKLOADS[name])


def workload(name: str, index: int = 0, random: bool = False):
    """Return ``(f, mask, y)`` for a named workload.

    ``f`` is the HR image (float64), ``mask`` the LR code array (uint8), and
    ``y`` the float32 L-pixel measurements.  ``random=True`` swaps the
    recurrent mask for a non-recurrent one of the same size.
    """
    cfg = _WORKLOADS[name]
    f = image(cfg["h"], cfg["w"], cfg["n_sin"], cfg["n_edges"],
              cfg["seed"] + index, cfg["sigma"])
    lr_h, lr_w = cfg["h"] // 2, cfg["w"] // 2
    if random:
        mask = random_mask(lr_h, lr_w, cfg["mseed"] + 100)
    else:
        mask = recurrent_mask(lr_h, lr_w, cfg["tile"], cfg["mseed"])
    y = measure(f, mask).astype(np.float32)
    return f, mask, y
