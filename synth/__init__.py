"""Seeded synthetic inputs for StyleBlit (Sýkora et al., EGSR 2018).

This module only manufactures inputs: guide images, style exemplars and
request streams with the shapes, value ranges and structure of the paper's
normal-guided (§4, Lit-Sphere-like setting) and texture-coordinate-guided (§4)
workloads.  It contains none of the method's arithmetic (no look-up table, no
seed hierarchy, no voting), so it can feed both the CPU oracle and the CUDA
library without coupling them.

All generators are deterministic functions of an integer seed (numpy PCG64).
Images are numpy arrays in interleaved HWC layout:
  * normal guide  : uint8  [H, W, 3], g = round((n + 1) / 2 * 255)
  * UV guide      : uint16 [H, W, 2], g = round(uv * 32) (5 fractional bits)
  * style exemplar: uint8  [H, W, 4] RGBA8

Generators that use transcendental functions (exp, sqrt, sin) may differ in
the last bit across platforms' libm; tests that store expected values use the
integer-only generators (`random_guide`, `random_style`, `identity_uv_guide`).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

UV_FRACTION_BITS = 5


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.uint64(seed))


# --------------------------------------------------------------------------
# integer-only generators (bit-identical on every platform)
# --------------------------------------------------------------------------

def random_guide(seed: int, height: int, width: int, channels: int,
                 bits: int = 8, low: int = 0, high: int | None = None) -> np.ndarray:
    """Uniform random guide values in [low, high] (inclusive)."""
    dtype = np.uint8 if bits == 8 else np.uint16
    if high is None:
        high = (1 << bits) - 1
    g = _rng(seed).integers(low, high + 1, size=(height, width, channels), dtype=np.int64)
    return g.astype(dtype)


def random_style(seed: int, height: int, width: int) -> np.ndarray:
    """Uniform random RGBA8 exemplar (alpha random too)."""
    return _rng(seed).integers(0, 256, size=(height, width, 4), dtype=np.int64).astype(np.uint8)


def identity_uv_guide(height: int, width: int, shift: int = UV_FRACTION_BITS) -> np.ndarray:
    """Source UV guide whose value at (x, y) is (x << shift, y << shift)."""
    ys, xs = np.mgrid[0:height, 0:width]
    g = np.stack([xs << shift, ys << shift], axis=-1)
    return g.astype(np.uint16)


def smooth_integer_guide(seed: int, height: int, width: int, channels: int = 2,
                         step: int = 8) -> np.ndarray:
    """A smooth-ish uint8 guide built from integer ramps plus seeded integer
    perturbations; useful for coherent chunks without transcendental math."""
    rng = _rng(seed)
    ys, xs = np.mgrid[0:height, 0:width].astype(np.int64)
    out = np.empty((height, width, channels), dtype=np.int64)
    for c in range(channels):
        ax, ay = rng.integers(-3, 4, size=2)
        off = rng.integers(0, 256)
        bumps = rng.integers(0, step, size=(height // step + 2, width // step + 2))
        noise = np.repeat(np.repeat(bumps, step, axis=0), step, axis=1)[:height, :width]
        out[..., c] = (off + ax * xs + ay * ys + noise) % 256
    return out.astype(np.uint8)


# --------------------------------------------------------------------------
# normal guides (§4, normal-based guidance)
# --------------------------------------------------------------------------

def _encode_normals(nx: np.ndarray, ny: np.ndarray, nz: np.ndarray) -> np.ndarray:
    n = np.stack([nx, ny, nz], axis=-1)
    g = np.rint((n + 1.0) * 0.5 * 255.0)
    return np.clip(g, 0, 255).astype(np.uint8)


def bump_normals(seed: int, height: int, width: int, n_bumps: int,
                 sigma_range: tuple[float, float]) -> np.ndarray:
    """Normals of a height field made of seeded Gaussian bumps.

    h(x, y) = sum_i A_i exp(-|(x, y) - mu_i|^2 / (2 sigma_i^2)) with mu_i
    uniform over the frame, sigma_i uniform in `sigma_range` and |A_i| uniform
    in [0.5 sigma_i, 2 sigma_i] with a random sign; n = normalize(-dh/dx,
    -dh/dy, 1), encoded as uint8.
    """
    rng = _rng(seed)
    mu_x = rng.uniform(0, width, n_bumps)
    mu_y = rng.uniform(0, height, n_bumps)
    sig = rng.uniform(sigma_range[0], sigma_range[1], n_bumps)
    amp = rng.uniform(0.5, 2.0, n_bumps) * sig * rng.choice([-1.0, 1.0], n_bumps)
    ys = np.arange(height, dtype=np.float64)[:, None]
    xs = np.arange(width, dtype=np.float64)[None, :]
    hx = np.zeros((height, width))
    hy = np.zeros((height, width))
    for i in range(n_bumps):
        dx = xs - mu_x[i]
        dy = ys - mu_y[i]
        # separable Gaussian: exp(-dx^2/2s^2) * exp(-dy^2/2s^2)
        s2 = 2.0 * sig[i] * sig[i]
        ex = np.exp(-dx * dx / s2)
        ey = np.exp(-dy * dy / s2)
        k = -amp[i] / (sig[i] * sig[i])
        hx += k * (dx * ex) * ey
        hy += k * ex * (dy * ey)
    nz = np.ones_like(hx)
    inv = 1.0 / np.sqrt(hx * hx + hy * hy + 1.0)
    return _encode_normals(-hx * inv, -hy * inv, nz * inv)


def sphere_normals(size: int) -> np.ndarray:
    """Normals of a sphere rendered into a size x size exemplar (disc radius
    size/2); outside the disc the silhouette normal (dx, dy, 0)/|.| is used."""
    c = size / 2.0
    r = size / 2.0
    ys, xs = np.mgrid[0:size, 0:size].astype(np.float64)
    dx = (xs + 0.5 - c) / r
    dy = (ys + 0.5 - c) / r
    rr = dx * dx + dy * dy
    inside = rr < 1.0
    nz = np.where(inside, np.sqrt(np.maximum(0.0, 1.0 - rr)), 0.0)
    rim = np.sqrt(np.maximum(rr, 1e-12))
    nx = np.where(inside, dx, dx / rim)
    ny = np.where(inside, dy, dy / rim)
    return _encode_normals(nx, ny, nz)


# --------------------------------------------------------------------------
# styles (hand-drawn exemplars stand-ins: stochastic textures)
# --------------------------------------------------------------------------

def value_noise_style(seed: int, height: int, width: int, octaves: int = 4,
                      base_cell: int = 64) -> np.ndarray:
    """Multi-octave value noise, RGB per channel, alpha 255."""
    rng = _rng(seed)
    out = np.zeros((height, width, 4), dtype=np.float64)
    ys = np.arange(height, dtype=np.float64)[:, None]
    xs = np.arange(width, dtype=np.float64)[None, :]
    total = 0.0
    for o in range(octaves):
        cell = max(2, base_cell >> o)
        gh = height // cell + 2
        gw = width // cell + 2
        lat = rng.random((gh, gw, 3))
        fy = ys / cell
        fx = xs / cell
        iy = np.floor(fy).astype(np.int64)
        ix = np.floor(fx).astype(np.int64)
        ty = fy - iy
        tx = fx - ix
        ty = ty * ty * (3 - 2 * ty)
        tx = tx * tx * (3 - 2 * tx)
        iy = np.broadcast_to(iy, (height, width))
        ix = np.broadcast_to(ix, (height, width))
        ty = np.broadcast_to(ty, (height, width))[..., None]
        tx = np.broadcast_to(tx, (height, width))[..., None]
        v00 = lat[iy, ix]
        v01 = lat[iy, ix + 1]
        v10 = lat[iy + 1, ix]
        v11 = lat[iy + 1, ix + 1]
        v = (v00 * (1 - tx) + v01 * tx) * (1 - ty) + (v10 * (1 - tx) + v11 * tx) * ty
        w = 0.5 ** o
        out[..., :3] += w * v
        total += w
    out[..., :3] /= total
    out[..., 3] = 1.0
    return np.clip(np.rint(out * 255.0), 0, 255).astype(np.uint8)


def add_strokes(seed: int, style: np.ndarray, n_strokes: int) -> np.ndarray:
    """Paint seeded random brush strokes (capsules) over an RGBA8 style."""
    rng = _rng(seed)
    img = style.copy()
    h, w = img.shape[:2]
    for _ in range(n_strokes):
        x0, y0 = rng.uniform(0, w), rng.uniform(0, h)
        ang = rng.uniform(0, 2 * math.pi)
        length = rng.uniform(20, 200)
        rad = rng.uniform(1.0, 4.0)
        col = rng.integers(0, 256, size=3)
        x1, y1 = x0 + length * math.cos(ang), y0 + length * math.sin(ang)
        bx0 = int(max(0, math.floor(min(x0, x1) - rad - 1)))
        bx1 = int(min(w, math.ceil(max(x0, x1) + rad + 2)))
        by0 = int(max(0, math.floor(min(y0, y1) - rad - 1)))
        by1 = int(min(h, math.ceil(max(y0, y1) + rad + 2)))
        if bx1 <= bx0 or by1 <= by0:
            continue
        ys, xs = np.mgrid[by0:by1, bx0:bx1].astype(np.float64)
        vx, vy = x1 - x0, y1 - y0
        t = np.clip(((xs - x0) * vx + (ys - y0) * vy) / (vx * vx + vy * vy), 0, 1)
        d2 = (xs - x0 - t * vx) ** 2 + (ys - y0 - t * vy) ** 2
        m = d2 <= rad * rad
        sub = img[by0:by1, bx0:bx1]
        sub[m, :3] = col
    return img


# --------------------------------------------------------------------------
# UV guides (§4, texture-coordinate guidance)
# --------------------------------------------------------------------------

def warped_uv_guide(seed: int, height: int, width: int, src_h: int, src_w: int,
                    n_triangles: int = 32) -> np.ndarray:
    """Target UV guide: the identity map of the target onto the source texture,
    pushed through a seeded piecewise-affine warp of random triangles.

    Each triangle gets an affine map about its centroid (rotation within
    +-10 degrees, scale in [0.8, 1.25]); later triangles overwrite earlier
    ones; pixels outside every triangle keep the identity map.  UVs are
    clamped to the source and stored with 5 fractional bits.
    """
    rng = _rng(seed)
    ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
    u = (xs + 0.5) * (src_w / width) - 0.5
    v = (ys + 0.5) * (src_h / height) - 0.5
    uu = u.copy()
    vv = v.copy()
    for _ in range(n_triangles):
        cx, cy = rng.uniform(0, width), rng.uniform(0, height)
        size = rng.uniform(0.05, 0.3) * min(width, height)
        angs = np.sort(rng.uniform(0, 2 * math.pi, 3))
        px = cx + size * np.cos(angs)
        py = cy + size * np.sin(angs)
        theta = math.radians(rng.uniform(-10, 10))
        sc = rng.uniform(0.8, 1.25)
        c, s = math.cos(theta) * sc, math.sin(theta) * sc
        # barycentric inside test over the triangle's bounding box
        x0 = int(max(0, math.floor(px.min())))
        x1 = int(min(width, math.ceil(px.max()) + 1))
        y0 = int(max(0, math.floor(py.min())))
        y1 = int(min(height, math.ceil(py.max()) + 1))
        if x1 <= x0 or y1 <= y0:
            continue
        X = xs[y0:y1, x0:x1]
        Y = ys[y0:y1, x0:x1]
        d = (py[1] - py[2]) * (px[0] - px[2]) + (px[2] - px[1]) * (py[0] - py[2])
        if abs(d) < 1e-9:
            continue
        l0 = ((py[1] - py[2]) * (X - px[2]) + (px[2] - px[1]) * (Y - py[2])) / d
        l1 = ((py[2] - py[0]) * (X - px[2]) + (px[0] - px[2]) * (Y - py[2])) / d
        l2 = 1.0 - l0 - l1
        m = (l0 >= 0) & (l1 >= 0) & (l2 >= 0)
        ucen = (cx + 0.5) * (src_w / width) - 0.5
        vcen = (cy + 0.5) * (src_h / height) - 0.5
        du = u[y0:y1, x0:x1] - ucen
        dv = v[y0:y1, x0:x1] - vcen
        wu = ucen + c * du - s * dv
        wv = vcen + s * du + c * dv
        uu[y0:y1, x0:x1] = np.where(m, wu, uu[y0:y1, x0:x1])
        vv[y0:y1, x0:x1] = np.where(m, wv, vv[y0:y1, x0:x1])
    uu = np.clip(uu, 0, src_w - 1)
    vv = np.clip(vv, 0, src_h - 1)
    scale = float(1 << UV_FRACTION_BITS)
    g = np.stack([np.rint(uu * scale), np.rint(vv * scale)], axis=-1)
    return g.astype(np.uint16)


# --------------------------------------------------------------------------
# workload presets
# --------------------------------------------------------------------------

@dataclass
class Exemplar:
    guide: np.ndarray      # source guide G_S, HWC
    style: np.ndarray      # source style C_S, RGBA8 HWC
    lut_bits: int          # LUT bits per guide channel


@dataclass
class Frame:
    guide: np.ndarray      # target guide G_T, HWC


@dataclass
class Workload:
    name: str
    exemplar: Exemplar
    frames: list[Frame]
    levels: int
    threshold: int
    blend_radius: int
    seed: int = 0
    extra: dict = field(default_factory=dict)


def normal_exemplar(seed: int, size: int, strokes: int = 0, octaves: int = 4,
                    lut_bits: int = 6) -> Exemplar:
    style = value_noise_style(seed, size, size, octaves=octaves,
                              base_cell=max(8, size // 16))
    if strokes:
        style = add_strokes(seed + 1, style, strokes)
    return Exemplar(guide=sphere_normals(size), style=style, lut_bits=lut_bits)


def workload_256(frame_seed: int = 1000) -> Workload:
    """256x256 normal-guided frame, 8 bumps (sigma 8-64 px), 256^2 sphere
    exemplar with value-noise style; 4 levels, threshold 300, no blend."""
    ex = normal_exemplar(1000 + 500, 256, octaves=3)
    fr = Frame(bump_normals(frame_seed, 256, 256, 8, (8.0, 64.0)))
    return Workload("normals-256x256-L4-T300-r0", ex, [fr], levels=4, threshold=300,
                    blend_radius=0, seed=frame_seed)


def workload_1080p(n_frames: int = 1, frame_seed: int = 2000) -> Workload:
    """1920x1080 normal-guided frames, 64 bumps (sigma 20-200 px), 1024^2
    sphere exemplar with multi-octave noise + strokes; 6 levels, threshold
    300, 5x5 blend."""
    ex = normal_exemplar(2000 + 500, 1024, strokes=400)
    frames = [Frame(bump_normals(frame_seed + i, 1080, 1920, 64, (20.0, 200.0)))
              for i in range(n_frames)]
    return Workload("normals-1920x1080-L6-T300-5x5", ex, frames, levels=6, threshold=300,
                    blend_radius=2, seed=frame_seed)


def workload_4k_uv(n_frames: int = 1, frame_seed: int = 3000) -> Workload:
    """3840x2160 UV-guided frames (piecewise-affine warp of 32 triangles),
    2048^2 identity-UV exemplar with noise texture; 7 levels, threshold 2^20,
    7x7 blend, 10 LUT bits per channel."""
    style = value_noise_style(3000 + 500, 2048, 2048, octaves=5, base_cell=128)
    ex = Exemplar(guide=identity_uv_guide(2048, 2048), style=style, lut_bits=10)
    frames = [Frame(warped_uv_guide(frame_seed + i, 2160, 3840, 2048, 2048, 32))
              for i in range(n_frames)]
    return Workload("uv-3840x2160-L7-T2^20-7x7", ex, frames, levels=7, threshold=1 << 20,
                    blend_radius=3, seed=frame_seed)


def batch_frame_sizes(seed: int, n_frames: int, min_w: int = 640, max_w: int = 3840):
    """Frame sizes of a mixed-resolution batch: width uniform (even) in
    [min_w, max_w], height = width * 9 / 16 rounded to even."""
    rng = _rng(seed)
    ws = rng.integers(min_w // 2, max_w // 2 + 1, size=n_frames) * 2
    return [(int(w), int(((w * 9) // 16) // 2 * 2)) for w in ws]


def poisson_arrivals(seed: int, rate_hz: float, n: int) -> np.ndarray:
    """Arrival times (s) of a seeded Poisson request stream."""
    rng = _rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))


def log_uniform_sizes(seed: int, n: int, min_px: int = 256 * 256,
                      max_px: int = 3840 * 2160):
    """Request frame sizes with pixel count log-uniform in [min_px, max_px],
    aspect 16:9 (square at the low end), dimensions even."""
    rng = _rng(seed)
    px = np.exp(rng.uniform(math.log(min_px), math.log(max_px), size=n))
    out = []
    for p in px:
        aspect = 1.0 + (16.0 / 9.0 - 1.0) * min(1.0, (p - min_px) / (1920 * 1080 - min_px))
        h = int(math.sqrt(p / aspect)) // 2 * 2
        w = int(h * aspect) // 2 * 2
        out.append((max(2, w), max(2, h)))
    return out
