"""Seeded synthetic colored point clouds for CVO tests and benchmarks.

Shared by the oracle tests, the CUDA parity tests and the benchmark. It holds
no arithmetic of the registration method itself (no kernel sums, no gradient,
no exponential map): only scene sampling, ray casting and rigid motions built
from unit quaternions.

Workloads (stand-ins for the paper's TUM RGB-D sequences, which are not
available here; the paper's experiments use Kinect frames of indoor scenes,
Sec. 5):

* ``planes_pair``: points sampled on three mutually orthogonal 2 m x 2 m
  planes (a room corner), 5 mm Gaussian noise, 5-D features (3 colour
  channels from smooth sinusoidal textures + 2 texture-gradient components);
  the source is an independent resample moved by a seeded rotation and
  translation.
* ``room_pair``: a procedural room (6 x 5 x 3 m box + 20 seeded cuboids with
  per-face sinusoidal textures) ray-cast to 640x480 depth + colour by a
  pinhole camera (fx = fy = 525, cx = 319.5, cy = 239.5), depth kept in
  0.5-5 m with 1 % multiplicative noise, semi-dense selection of pixels whose
  intensity-gradient magnitude exceeds the 80th percentile, then a seeded
  subsample to an exact point count. The second frame is rendered after a
  seeded camera motion.
* ``batch_pairs``: many planes pairs of uneven sizes.

Every generator returns float32 arrays, the ground-truth pose ``P_gt`` (4x4
float64, maps source coordinates into the target frame) and its seed.
"""
from __future__ import annotations

import numpy as np

FEAT_DIM = 5


def seed_for(config: int, pair: int = 0) -> int:
    """Seed convention: 1234 + 1000 * config + pair."""
    return 1234 + 1000 * int(config) + int(pair)


# --------------------------------------------------------------------------
# rigid motions (unit quaternions; independent of the solver's exp map)
# --------------------------------------------------------------------------

def quat_to_matrix(q) -> np.ndarray:
    w, x, y, z = [float(c) for c in q]
    n = np.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / n, x / n, y / n, z / n
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def axis_angle_matrix(axis, angle_rad: float) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    h = 0.5 * angle_rad
    return quat_to_matrix([np.cos(h), *(np.sin(h) * axis)])


def unit_vector(rng) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def rigid(R, T) -> np.ndarray:
    P = np.eye(4)
    P[:3, :3] = R
    P[:3, 3] = T
    return P


def inverse(P) -> np.ndarray:
    R, T = P[:3, :3], P[:3, 3]
    return rigid(R.T, -R.T @ T)


def random_motion(rng, deg: float, meters: float) -> np.ndarray:
    """Rotation by exactly ``deg`` about a uniform random axis and a
    translation of exactly ``meters`` along a uniform random direction."""
    R = axis_angle_matrix(unit_vector(rng), np.deg2rad(deg))
    return rigid(R, meters * unit_vector(rng))


def transform(P, pts) -> np.ndarray:
    return pts @ P[:3, :3].T + P[:3, 3]


# --------------------------------------------------------------------------
# config 1: three orthogonal planes
# --------------------------------------------------------------------------

class _PlaneTextures:
    """Per plane and per channel: 0.5 + 0.5 sin(2 pi k.(u, v) + phi), with
    |k| uniform in [1, 4] cycles/m and a random direction."""

    def __init__(self, rng, n_planes=3, n_ch=3):
        ang = rng.uniform(0, 2 * np.pi, size=(n_planes, n_ch))
        mag = rng.uniform(1.0, 4.0, size=(n_planes, n_ch))
        self.k = np.stack([mag * np.cos(ang), mag * np.sin(ang)], axis=-1)  # (P, C, 2)
        self.phi = rng.uniform(0, 2 * np.pi, size=(n_planes, n_ch))

    def features(self, plane, uv):
        k = self.k[plane]                   # (n, C, 2)
        phase = 2 * np.pi * np.einsum("ncd,nd->nc", k, uv) + self.phi[plane]
        col = 0.5 + 0.5 * np.sin(phase)     # (n, 3): H, S, V
        # analytic derivative of the V channel along the plane axes, scaled
        # by its largest possible magnitude (pi |k|) into [-1, 1]
        kv = k[:, 2, :]
        dv = (np.pi * np.cos(phase[:, 2]))[:, None] * kv
        dv = dv / (np.pi * np.linalg.norm(kv, axis=1, keepdims=True))
        return np.concatenate([col, dv], axis=1)


def _sample_planes(rng, tex, n, noise, extent=2.0):
    plane = np.arange(n) % 3
    uv = rng.uniform(0.0, extent, size=(n, 2))
    pts = np.zeros((n, 3))
    # plane 0: x = 0 (y, z) = uv; plane 1: y = 0 (x, z) = uv; plane 2: z = 0 (x, y) = uv
    for p, (a, b) in enumerate([(1, 2), (0, 2), (0, 1)]):
        m = plane == p
        pts[m, a] = uv[m, 0]
        pts[m, b] = uv[m, 1]
    pts += rng.normal(scale=noise, size=pts.shape)
    return pts, tex.features(plane, uv)


def planes_pair(n_x=2000, n_z=2000, seed=None, deg=5.0, meters=0.05, noise=0.005):
    """Target X and source Z on three orthogonal planes; Z is an independent
    resample moved by a rotation of ``deg`` degrees about a random axis and a
    translation of ``meters``. P_gt maps Z's coordinates back into X's frame."""
    seed = seed_for(1) if seed is None else seed
    rng = np.random.default_rng(seed)
    tex = _PlaneTextures(rng)
    X, FX = _sample_planes(rng, tex, n_x, noise)
    Zw, FZ = _sample_planes(rng, tex, n_z, noise)
    M = random_motion(rng, deg, meters)     # moves the resample
    Z = transform(M, Zw)
    return {"X": X.astype(np.float32), "FX": FX.astype(np.float32),
            "Z": Z.astype(np.float32), "FZ": FZ.astype(np.float32),
            "P_gt": inverse(M), "seed": seed}


def batch_pairs(n_pairs=256, seed=None, n_range=(2000, 40000), deg_max=5.0, meters_max=0.05,
                ell0_range=(0.12, 0.18)):
    """Uneven batch: each pair a planes_pair with sizes uniform in n_range,
    motions up to deg_max / meters_max and its own initial lengthscale."""
    seed = seed_for(3) if seed is None else seed
    rng = np.random.default_rng(seed)
    out = []
    for p in range(n_pairs):
        n_x, n_z = rng.integers(n_range[0], n_range[1] + 1, size=2)
        d = planes_pair(int(n_x), int(n_z), seed=seed * 7919 + p,
                        deg=float(rng.uniform(0.0, deg_max)),
                        meters=float(rng.uniform(0.0, meters_max)))
        d["ell0"] = float(rng.uniform(*ell0_range))
        out.append(d)
    return out


# --------------------------------------------------------------------------
# configs 2 and 4: ray-cast procedural room
# --------------------------------------------------------------------------

class Room:
    """Axis-aligned room box with axis-aligned cuboids, each face textured by
    three sinusoids (H, S, V) over its two in-plane world coordinates."""

    def __init__(self, rng, size=(6.0, 5.0, 3.0), n_cuboids=20, keep_clear=None):
        self.size = np.asarray(size, dtype=np.float64)
        lo, hi = [np.zeros(3)], [self.size.copy()]
        while len(lo) < n_cuboids + 1:
            dims = np.array([rng.uniform(0.2, 1.0), rng.uniform(0.2, 1.0), rng.uniform(0.2, 1.5)])
            pos = np.array([rng.uniform(0.0, self.size[0] - dims[0]),
                            rng.uniform(0.0, self.size[1] - dims[1]), 0.0])
            if keep_clear is not None:
                c = np.clip(keep_clear, pos, pos + dims)
                if np.linalg.norm(c - keep_clear) < 1.0:
                    continue
            lo.append(pos)
            hi.append(pos + dims)
        self.lo, self.hi = np.array(lo), np.array(hi)
        nf = len(lo) * 6
        ang = rng.uniform(0, 2 * np.pi, size=(nf, 3))
        mag = rng.uniform(1.0, 4.0, size=(nf, 3))
        self.k = np.stack([mag * np.cos(ang), mag * np.sin(ang)], axis=-1)
        self.phi = rng.uniform(0, 2 * np.pi, size=(nf, 3))

    def cast(self, origin, dirs):
        """Nearest hit of rays origin + t dirs (t > 0). Returns t (inf on a
        miss) and the face id (box * 6 + axis * 2 + side)."""
        n = dirs.shape[0]
        best_t = np.full(n, np.inf)
        face = np.full(n, -1, dtype=np.int64)
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / dirs
            for b in range(self.lo.shape[0]):
                t1 = (self.lo[b] - origin) * inv
                t2 = (self.hi[b] - origin) * inv
                tmin, tmax = np.minimum(t1, t2), np.maximum(t1, t2)
                tmin = np.where(np.isnan(tmin), -np.inf, tmin)
                tmax = np.where(np.isnan(tmax), np.inf, tmax)
                tn, tf = tmin.max(axis=1), tmax.min(axis=1)
                if b == 0:   # inside the room: the exit point is the wall hit
                    t = tf
                    ax = tmax.argmin(axis=1)
                    side = (dirs[np.arange(n), ax] > 0).astype(np.int64)
                    ok = tf > 0
                else:
                    t = tn
                    ax = tmin.argmax(axis=1)
                    side = (dirs[np.arange(n), ax] < 0).astype(np.int64)
                    ok = (tn <= tf) & (tn > 0)
                upd = ok & (t < best_t)
                best_t[upd] = t[upd]
                face[upd] = b * 6 + ax[upd] * 2 + side[upd]
        return best_t, face

    def colour(self, pts, face):
        ax = (face // 2) % 3
        other = np.stack([np.where(ax == 0, 1, 0), np.where(ax == 2, 1, 2)], axis=1)
        uv = np.take_along_axis(pts, other, axis=1)
        k = self.k[face]
        phase = 2 * np.pi * np.einsum("ncd,nd->nc", k, uv) + self.phi[face]
        return 0.5 + 0.5 * np.sin(phase)


def _camera_rotation(yaw, pitch):
    """Camera-to-world rotation; camera axes x right, y down, z forward.
    Zero yaw/pitch looks along world +x with world +z up."""
    base = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])
    cy, sy, cp, sp = np.cos(yaw), np.sin(yaw), np.cos(pitch), np.sin(pitch)
    Rz = np.array([[cy, -sy, 0.0], [sy, cy, 0.0], [0.0, 0.0, 1.0]])
    Ry = np.array([[cp, 0.0, sp], [0.0, 1.0, 0.0], [-sp, 0.0, cp]])
    return Rz @ Ry @ base


def render(room, T_wc, rng, width=640, height=480, fx=525.0, fy=525.0, cx=319.5, cy=239.5,
           depth_range=(0.5, 5.0), depth_noise=0.01):
    """Ray-cast one RGB-D frame. Returns per-pixel camera-frame points (H, W, 3),
    HSV colour (H, W, 3) and a validity mask."""
    u, v = np.meshgrid(np.arange(width, dtype=np.float64), np.arange(height, dtype=np.float64))
    d_c = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], axis=-1).reshape(-1, 3)
    d_w = d_c @ T_wc[:3, :3].T
    t, face = room.cast(T_wc[:3, 3], d_w)
    hit = np.isfinite(t)
    pts_w = T_wc[:3, 3] + t[:, None] * d_w
    col = np.zeros((d_c.shape[0], 3))
    col[hit] = room.colour(pts_w[hit], face[hit])
    depth = t * (1.0 + depth_noise * rng.normal(size=t.shape))   # d_c has unit z
    valid = hit & (depth >= depth_range[0]) & (depth <= depth_range[1])
    pts_c = np.where(valid[:, None], depth[:, None] * d_c, 0.0)
    return pts_c.reshape(height, width, 3), col.reshape(height, width, 3), valid.reshape(height, width)


def select_points(pts, col, valid, rng, n_points, mode="gradient", percentile=80.0,
                  grad_scale=0.05):
    """Semi-dense selection (Sec. 5: high intensity-gradient pixels) and a
    seeded subsample to exactly n_points. Features: H, S, V and the two
    intensity-gradient components divided by grad_scale and clipped to [-1, 1]."""
    inten = col[..., 2]
    gy, gx = np.gradient(inten)
    mag = np.hypot(gx, gy)
    if mode == "gradient":
        thr = np.percentile(mag[valid], percentile)
        keep = valid & (mag > thr)
    else:
        keep = valid
    idx = np.flatnonzero(keep.reshape(-1))
    if idx.size > n_points:
        idx = np.sort(rng.choice(idx, size=n_points, replace=False))
    feats = np.concatenate([col.reshape(-1, 3),
                            np.clip(gx.reshape(-1, 1) / grad_scale, -1, 1),
                            np.clip(gy.reshape(-1, 1) / grad_scale, -1, 1)], axis=1)
    return pts.reshape(-1, 3)[idx], feats[idx]


def room_pair(n_points=20000, seed=None, deg=3.0, meters=0.03, mode="gradient", width=640,
              height=480):
    """Two ray-cast frames of one procedural room; X from frame 1, Z from frame
    2 (each in its own camera frame). P_gt = T_wc1^{-1} T_wc2 maps frame-2
    camera coordinates into frame 1."""
    seed = seed_for(2) if seed is None else seed
    rng = np.random.default_rng(seed)
    cam = np.array([rng.uniform(0.6, 1.0), rng.uniform(2.0, 3.0), rng.uniform(1.2, 1.6)])
    room = Room(rng, keep_clear=cam)
    R1 = _camera_rotation(rng.uniform(-0.35, 0.35), rng.uniform(-0.25, -0.05))
    T_wc1 = rigid(R1, cam)
    M = random_motion(rng, deg, meters)
    T_wc2 = T_wc1 @ M
    p1, c1, v1 = render(room, T_wc1, rng, width, height)
    p2, c2, v2 = render(room, T_wc2, rng, width, height)
    X, FX = select_points(p1, c1, v1, rng, n_points, mode)
    Z, FZ = select_points(p2, c2, v2, rng, n_points, mode)
    return {"X": X.astype(np.float32), "FX": FX.astype(np.float32),
            "Z": Z.astype(np.float32), "FZ": FZ.astype(np.float32),
            "P_gt": M, "seed": seed}


# --------------------------------------------------------------------------
# config 5: camera streams served against resident keyframes
# --------------------------------------------------------------------------

def stream_keyframe(kf_seed: int, n_kf: int, noise=0.005):
    """Keyframe of one stream: points on the textured planes of kf_seed."""
    rng = np.random.default_rng(kf_seed)
    tex = _PlaneTextures(rng)
    X, FX = _sample_planes(rng, tex, n_kf, noise)
    return X.astype(np.float32), FX.astype(np.float32)


def stream_frame(kf_seed: int, frame: int, n: int, deg=3.0, meters=0.03, noise=0.005):
    """Frame `frame` of a keyframe's epoch: a fresh sample of the same textured
    planes moved by its own seeded motion. Returns (Z, FZ, P_gt)."""
    rng = np.random.default_rng(kf_seed)
    tex = _PlaneTextures(rng)
    rng2 = np.random.default_rng([kf_seed, frame])
    Zw, FZ = _sample_planes(rng2, tex, n, noise)
    M = random_motion(rng2, deg, meters)
    return transform(M, Zw).astype(np.float32), FZ.astype(np.float32), inverse(M)


def serving_trace(n_streams=64, rate_hz=30.0, duration_s=20.0, n_range=(5000, 60000),
                  keyframe_every=10, seed=None):
    """Open-loop arrivals of camera frames: per stream, exponential
    inter-arrival times of mean 1/rate_hz (Poisson), frame sizes uniform in
    n_range, a new keyframe (of its own size in n_range) every keyframe_every
    frames. Returns the requests sorted by arrival time, each a dict with
    t (s), stream, kf_seed, n_kf, frame (index in the keyframe's epoch), n."""
    seed = seed_for(5) if seed is None else seed
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_streams):
        t = float(rng.exponential(1.0 / rate_hz))
        k = 0
        kf_seed = n_kf = None
        while t < duration_s:
            if k % keyframe_every == 0:
                kf_seed = seed * 100003 + s * 1009 + k
                n_kf = int(rng.integers(n_range[0], n_range[1] + 1))
            out.append({"t": t, "stream": s, "kf_seed": kf_seed, "n_kf": n_kf,
                        "frame": k % keyframe_every, "n": int(rng.integers(n_range[0],
                                                                        n_range[1] + 1))})
            k += 1
            t += float(rng.exponential(1.0 / rate_hz))
    out.sort(key=lambda r: r["t"])
    return out


# --------------------------------------------------------------------------
# odometry over a stream: a camera trajectory through one room
# --------------------------------------------------------------------------

def room_trajectory(n_frames=30, n_points=20000, seed=None, step_deg=3.0, step_m=0.03,
                    width=640, height=480, mode="gradient"):
    """Frames of one camera moving through a procedural room: each step is a
    seeded motion of step_deg / step_m (as between the two frames of
    room_pair). Returns frames (X_k, F_k) in their own camera frames, the
    camera-to-world poses T_wc_k, and the relative poses P_gt_k that map frame
    k+1's coordinates into frame k (the pose the solver estimates with frame k
    as target and frame k+1 as source)."""
    seed = seed_for(6) if seed is None else seed
    rng = np.random.default_rng(seed)
    cam = np.array([rng.uniform(0.8, 1.2), rng.uniform(2.0, 3.0), rng.uniform(1.2, 1.6)])
    room = Room(rng, keep_clear=cam)
    T = rigid(_camera_rotation(rng.uniform(-0.35, 0.35), rng.uniform(-0.25, -0.05)), cam)
    poses, frames, rel = [T], [], []
    for k in range(n_frames - 1):
        M = random_motion(rng, step_deg, step_m)
        rel.append(M)
        T = T @ M
        poses.append(T)
    for T_wc in poses:
        p, c, v = render(room, T_wc, rng, width, height)
        X, F = select_points(p, c, v, rng, n_points, mode)
        frames.append((X.astype(np.float32), F.astype(np.float32)))
    return {"frames": frames, "T_wc": poses, "P_gt": rel, "seed": seed}


def room_frame_images(seed=None, width=640, height=480):
    """One rendered RGB-D frame as images: depth (H, W) float32 (0 where
    invalid: no hit, or outside 0.5-5 m), HSV colour (H, W, 3) float32, and
    the pinhole intrinsics (fx, fy, cx, cy) of render."""
    seed = seed_for(7) if seed is None else seed
    rng = np.random.default_rng(seed)
    cam = np.array([rng.uniform(0.6, 1.0), rng.uniform(2.0, 3.0), rng.uniform(1.2, 1.6)])
    room = Room(rng, keep_clear=cam)
    T_wc = rigid(_camera_rotation(rng.uniform(-0.35, 0.35), rng.uniform(-0.25, -0.05)), cam)
    fx = fy = 525.0 * width / 640.0
    cx, cy = (width - 1) / 2.0, (height - 1) / 2.0
    p, c, v = render(room, T_wc, rng, width, height, fx, fy, cx, cy)
    depth = np.where(v, p[..., 2], 0.0).astype(np.float32)
    return {"depth": depth, "hsv": c.astype(np.float32), "fx": fx, "fy": fy, "cx": cx, "cy": cy}
