"""Oracle of the semi-dense front end (Sec. 5: the points are the pixels with a
high intensity gradient, back-projected from the depth image).

TEST INFRASTRUCTURE ONLY (see the package docstring): the reference the GPU
front end (``cvo_frontend_cloud``) is checked against. Selecting pixels is
index work, so the definition is written out in the precision the GPU takes
every decision in, and the two must agree bit for bit on which pixels are
kept and in what order:

  valid      depth_min <= depth <= depth_max (depth finite)
  gradient   of the intensity I = V channel, in FP32: central differences
             0.5 (I[x+1] - I[x-1]) inside, one-sided differences at the image
             border (numpy.gradient with edge_order 1)
  magnitude  sqrt(gx^2 + gy^2) in FP32, each operation rounded once
  threshold  the linear-interpolation percentile of the valid pixels'
             magnitudes (numpy's 'linear' method, evaluated in FP64)
  kept       valid and magnitude > threshold, in raster order; when more
             than max_points are kept, the ranks floor(k m / max_points),
             k = 0 .. max_points - 1, of the m kept pixels
  point      z = depth, x = ((u - cx) / fx) z, y = ((v - cy) / fy) z in FP32
  features   H, S, V, and clip(gx / grad_scale, -1, 1), clip(gy / grad_scale,
             -1, 1) in FP32
"""
from __future__ import annotations

import numpy as np

f32 = np.float32


def gradient_fp32(img):
    """Central differences inside, one-sided at the border, FP32 (x along
    columns, y along rows)."""
    I = np.asarray(img, dtype=f32)
    gx = np.empty_like(I)
    gy = np.empty_like(I)
    gx[:, 1:-1] = f32(0.5) * (I[:, 2:] - I[:, :-2])
    gx[:, 0] = I[:, 1] - I[:, 0]
    gx[:, -1] = I[:, -1] - I[:, -2]
    gy[1:-1, :] = f32(0.5) * (I[2:, :] - I[:-2, :])
    gy[0, :] = I[1, :] - I[0, :]
    gy[-1, :] = I[-1, :] - I[-2, :]
    return gx, gy


def percentile_linear(values, q):
    """numpy's 'linear' percentile, written out: position h = (n - 1) q / 100
    between the order statistics a = v[floor h] and b = v[ceil h], value
    a + (b - a) t for t = h - floor h < 0.5, else b - (b - a)(1 - t), in FP64."""
    v = np.sort(np.asarray(values, dtype=np.float64))
    n = v.size
    h = (n - 1) * (q / 100.0)
    lo = int(np.floor(h))
    hi = min(lo + 1, n - 1)
    t = h - lo
    a, b = v[lo], v[hi]
    d = b - a
    return a + d * t if t < 0.5 else b - d * (1.0 - t)


def select(depth, hsv, fx, fy, cx, cy, depth_min=0.5, depth_max=5.0, percentile=80.0,
           grad_scale=0.05, max_points=0):
    """The front end's output: (xyz (n, 3) float32, features (n, 5) float32,
    kept pixel indices (n,) in raster order)."""
    depth = np.asarray(depth, dtype=f32)
    hsv = np.asarray(hsv, dtype=f32)
    H, W = depth.shape
    valid = np.isfinite(depth) & (depth >= f32(depth_min)) & (depth <= f32(depth_max))
    gx, gy = gradient_fp32(hsv[..., 2])
    mag = np.sqrt(gx * gx + gy * gy)            # FP32, one rounding per operation
    if not valid.any():
        return (np.zeros((0, 3), f32), np.zeros((0, 5), f32), np.zeros(0, np.int64))
    thr = percentile_linear(mag[valid], percentile)
    keep = valid & (mag.astype(np.float64) > thr)
    idx = np.flatnonzero(keep.reshape(-1))
    m = idx.size
    if max_points and m > max_points:
        k = np.arange(max_points, dtype=np.int64)
        idx = idx[(k * m) // max_points]
    v_pix, u_pix = np.divmod(idx, W)
    z = depth.reshape(-1)[idx]
    x = ((u_pix.astype(f32) - f32(cx)) / f32(fx)) * z
    y = ((v_pix.astype(f32) - f32(cy)) / f32(fy)) * z
    xyz = np.stack([x, y, z], axis=1).astype(f32)
    gs = f32(grad_scale)
    feats = np.concatenate([hsv.reshape(-1, 3)[idx],
                            np.clip(gx.reshape(-1)[idx] / gs, f32(-1), f32(1))[:, None],
                            np.clip(gy.reshape(-1)[idx] / gs, f32(-1), f32(1))[:, None]],
                           axis=1).astype(f32)
    return xyz, feats, idx
