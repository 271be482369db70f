"""Seeded synthetic inputs for the tracker: scenes, depth frames, trajectories.

This module produces INPUTS only and holds none of the tracking method's
arithmetic (no fitness, no PST update, no fusion).  Tests, the benchmark and
the oracle comparisons all draw their inputs from here, so both sides of every
parity check see identical data.

The paper measures on ICL-NUIM, TUM, ETH3D and FastCaMo (Sec. 5.1); none of
those datasets is available, so a closed analytic scene stands in for them:
an axis-aligned room (six walls) with three spheres, rendered by exact
closed-form ray casting (ray/plane and ray/sphere intersections, no graphics
API), with depth noise N(0, (1 mm * z^2)^2) and camera trajectories at the
fast-motion speeds of the paper's FastCaMo-Synth statistics (Sec. 5.1,
Table speed-info: up to ~4 m/s and ~2-3 rad/s).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# --------------------------------------------------------------------------- configs
# Workload presets.  "tiny" and "paper" follow the two plain-PFO workloads the
# tracker is specified on; the others widen them (batch, precision, learned).
CONFIGS = {
    "tiny": dict(dims=64, voxel=0.04, trunc=0.12, dtype="f32", width=80, height=60, stride=1,
                 n_particles=1024, k_max=10, frames=1, speed=3.0, ang_speed=3.0, noise=False,
                 wall_inset=0.30, seed=0),
    "paper": dict(dims=512, voxel=0.01, trunc=0.06, dtype="i16", width=640, height=480, stride=4,
                  n_particles=20000, k_max=20, frames=300, speed=3.0, ang_speed=3.0, noise=True,
                  wall_inset=0.20, seed=0),
    "precision": dict(dims=512, voxel=0.01, trunc=0.06, dtype="f16", width=640, height=480, stride=4,
                      n_particles=20000, k_max=20, frames=1000, speed=4.0, ang_speed=3.0, noise=True,
                      wall_inset=0.20, seed=0),
    # Sec. 4 multi-resolution PST: (1024, 1/8), (3072, 1/16), (10240, 1/32) of the pixels in turn,
    # read as strides 3, 4 and 6 (1/9, 1/16, 1/36 of the pixels)
    "multires": dict(dims=512, voxel=0.01, trunc=0.06, dtype="i16", width=640, height=480, stride=4,
                     n_particles=10240, levels=([1024, 3072, 10240], [3, 4, 6]), k_max=20, frames=300,
                     speed=3.0, ang_speed=3.0, noise=True, wall_inset=0.20, seed=0),
    # learned proposal: plain PFO at 10k particles labels the frames; the proposal
    # then runs k_learned iterations (seeds 100.. train, 1000.. held out)
    "learned": dict(dims=512, voxel=0.01, trunc=0.06, dtype="i16", width=640, height=480, stride=4,
                    n_particles=10000, k_max=20, k_learned=5, frames=1000, speed=4.0, ang_speed=3.0, noise=True,
                    wall_inset=0.20, seed=0, train_seeds=list(range(100, 164)), test_seeds=list(range(1000, 1008)),
                    r_first=[0.05, 0.05, 0.05, 0.15, 0.15, 0.15], label_substeps=2),
}


def batched_specs(n_seq: int = 16, seed: int = 0):
    """Uneven sequences stepped together: depth 80x60 .. 320x240, TSDF 256^3 .. 512^3
    over the same 5.12 m room extent, 10k .. 40k particles, int16 storage."""
    rng = np.random.default_rng(30_000 + seed)
    sizes = [(80, 60), (160, 120), (240, 180), (320, 240)]
    specs = []
    for i in range(n_seq):
        w, h = sizes[int(rng.integers(0, len(sizes)))]
        dims = int(rng.choice([256, 384, 512]))
        voxel = 5.12 / dims
        specs.append(dict(dims=dims, voxel=voxel, trunc=6 * voxel, dtype="i16", width=w, height=h, stride=1,
                          n_particles=int(rng.integers(10_000, 40_001)), k_max=20, speed=3.0, ang_speed=3.0,
                          noise=True, wall_inset=0.20, seed=seed + i))
    return specs


def intrinsics(width: int, height: int, z_min: float = 0.1, z_max: float = 8.0) -> dict:
    """Pinhole intrinsics scaled from the 640x480 f = 525 px camera."""
    f = 525.0 * width / 640.0
    return dict(fx=f, fy=f, cx=(width - 1) / 2.0, cy=(height - 1) / 2.0, width=int(width), height=int(height),
                z_min=float(z_min), z_max=float(z_max))


# --------------------------------------------------------------------------- rotations (input side)
def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _qrot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _qcanon(q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    return -q if q[0] < 0 else q


def axis_angle_quat(axis, angle):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    return _qcanon(np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * axis]))


def look_at_quat(eye, target, up=(0.0, 0.0, 1.0)):
    """Camera->world rotation with the camera z axis towards target (x right, y down)."""
    z = np.asarray(target, np.float64) - np.asarray(eye, np.float64)
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    if np.linalg.norm(x) < 1e-6:
        x = np.cross(z, np.array([1.0, 0.0, 0.0]))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=1)
    # matrix -> quaternion (Shepperd)
    tr = np.trace(R)
    if tr > 0:
        s = math.sqrt(tr + 1.0) * 2
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    elif R[0, 0] > R[1, 1] and R[0, 0] > R[2, 2]:
        s = math.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2]) * 2
        q = [(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
    elif R[1, 1] > R[2, 2]:
        s = math.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2]) * 2
        q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s]
    else:
        s = math.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1]) * 2
        q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s]
    return _qcanon(q)


# --------------------------------------------------------------------------- scene
@dataclasses.dataclass
class Scene:
    lo: np.ndarray          # room interior lower corner (m)
    hi: np.ndarray          # room interior upper corner (m)
    centres: np.ndarray     # (S, 3) sphere centres
    radii: np.ndarray       # (S,) sphere radii

    def sdf(self, p):
        """Signed distance to the nearest surface, positive in free space (p: (..., 3))."""
        p = np.asarray(p, np.float64)
        d = np.minimum(p - self.lo, self.hi - p).min(axis=-1)
        for c, r in zip(self.centres, self.radii):
            d = np.minimum(d, np.linalg.norm(p - c, axis=-1) - r)
        return d

    def raycast(self, origin, dirs):
        """Hit parameter t >= 0 of rays origin + t * dirs (dirs: (..., 3), unnormalised)."""
        dirs = np.asarray(dirs, np.float64)
        o = np.asarray(origin, np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            tw = np.where(dirs > 0, (self.hi - o) / dirs, np.where(dirs < 0, (self.lo - o) / dirs, np.inf))
        t = tw.min(axis=-1)
        for c, r in zip(self.centres, self.radii):
            oc = o - c
            a = (dirs * dirs).sum(-1)
            b = 2.0 * (dirs * oc).sum(-1)
            cc = oc @ oc - r * r
            disc = b * b - 4 * a * cc
            ok = disc >= 0
            sq = np.sqrt(np.where(ok, disc, 0.0))
            t1 = (-b - sq) / (2 * a)
            t2 = (-b + sq) / (2 * a)
            ts = np.where(t1 > 1e-9, t1, np.where(t2 > 1e-9, t2, np.inf))
            t = np.where(ok, np.minimum(t, ts), t)
        return t


def camera_margin(scene: "Scene") -> float:
    """Distance the camera keeps from the walls: 0.8 m, or 35 % of the room
    size in rooms under 2.3 m."""
    return min(0.8, 0.35 * float((scene.hi - scene.lo).min()))


def make_scene(volume_extent: float, wall_inset: float, seed: int, n_spheres: int = 3) -> Scene:
    """Room = the volume minus wall_inset on every side; spheres of radius
    U[0.2, 0.6] m (scaled down for rooms under 4 m), centres at least 0.3 m
    inside the walls and surfaces at least 0.3 m outside the camera's box."""
    rng = np.random.default_rng(10_000 + seed)
    lo = np.full(3, wall_inset)
    hi = np.full(3, volume_extent - wall_inset)
    scale = min(1.0, (hi[0] - lo[0]) / 4.0)
    probe = Scene(lo=lo, hi=hi, centres=np.zeros((0, 3)), radii=np.zeros(0))
    m = camera_margin(probe)
    box_lo, box_hi = lo + m, hi - m
    centres, radii = [], []
    for _ in range(10_000):
        if len(radii) == n_spheres:
            break
        r = rng.uniform(0.2, 0.6) * scale
        c = rng.uniform(lo + 0.3, hi - 0.3)
        gap = np.linalg.norm(np.maximum(0.0, np.maximum(box_lo - c, c - box_hi)))
        if gap >= r + 0.3:
            centres.append(c)
            radii.append(r)
    return Scene(lo=lo, hi=hi, centres=np.array(centres).reshape(-1, 3), radii=np.array(radii))


def render_depth(scene: Scene, pose, K: dict, noise_rng=None, noise_scale: float = 0.001) -> np.ndarray:
    """Depth image (H, W) float32 at camera->world pose (q w,x,y,z, t) by
    closed-form ray casting; depth = distance along the optical axis; pixels
    whose depth falls outside (z_min, z_max] are 0 (invalid).  With noise_rng,
    N(0, (noise_scale * z^2)^2) is added."""
    W, H = K["width"], K["height"]
    pose = np.asarray(pose, np.float64)
    R = _qrot(pose[:4])
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    dc = np.stack([(u - K["cx"]) / K["fx"], (v - K["cy"]) / K["fy"], np.ones_like(u)], axis=-1)
    dw = dc @ R.T  # z component of the camera-frame direction is 1, so t = depth
    z = scene.raycast(pose[4:], dw)
    if noise_rng is not None:
        z = z + noise_rng.normal(0.0, 1.0, size=z.shape) * noise_scale * z * z
    z = np.where((z > K["z_min"]) & (z <= K["z_max"]) & np.isfinite(z), z, 0.0)
    return z.astype(np.float32)


def _quat_to_rot_torch(q):
    w, x, y, z = q.unbind(-1)
    return torch_stack3x3(
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y))


def torch_stack3x3(*e):
    import torch

    return torch.stack([torch.stack(e[0:3], -1), torch.stack(e[3:6], -1), torch.stack(e[6:9], -1)], -2)


def render_depth_batch(scene: Scene, poses, K: dict, seed: int, noise: bool = True, noise_scale: float = 0.001,
                       device="cuda", chunk: int = 32):
    """Depth images (F, H, W) float32 on the device for camera->world poses (F, 7):
    the closed-form ray casting of render_depth evaluated with torch in float64
    on the device, for large synthetic sets.  The noise N(0, (noise_scale z^2)^2)
    comes from a torch generator seeded with `seed`: the same distribution as
    render_depth, not the same draws."""
    import torch

    P = torch.as_tensor(np.asarray(poses, np.float64), device=device)
    n_f = P.shape[0]
    W, H = int(K["width"]), int(K["height"])
    vv, uu = torch.meshgrid(torch.arange(H, dtype=torch.float64, device=device),
                            torch.arange(W, dtype=torch.float64, device=device), indexing="ij")
    dc = torch.stack([(uu - K["cx"]) / K["fx"], (vv - K["cy"]) / K["fy"], torch.ones_like(uu)], -1)
    lo = torch.as_tensor(scene.lo, dtype=torch.float64, device=device)
    hi = torch.as_tensor(scene.hi, dtype=torch.float64, device=device)
    inf = torch.tensor(float("inf"), dtype=torch.float64, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    out = torch.empty((n_f, H, W), dtype=torch.float32, device=device)
    for s in range(0, n_f, chunk):
        p = P[s:s + chunk]
        n = p.shape[0]
        R = _quat_to_rot_torch(p[:, :4])
        d = torch.einsum("hwk,njk->nhwj", dc, R)  # world ray directions, unit depth along the optical axis
        o = p[:, 4:].view(n, 1, 1, 3)
        tw = torch.where(d > 0, (hi - o) / d, torch.where(d < 0, (lo - o) / d, inf))
        t = tw.amin(-1)
        for c, r in zip(scene.centres, scene.radii):
            oc = o - torch.as_tensor(c, dtype=torch.float64, device=device)
            a = (d * d).sum(-1)
            b = 2.0 * (d * oc).sum(-1)
            cc = (oc * oc).sum(-1) - float(r) * float(r)
            disc = b * b - 4 * a * cc
            sq = torch.sqrt(torch.clamp(disc, min=0.0))
            t1 = (-b - sq) / (2 * a)
            t2 = (-b + sq) / (2 * a)
            ts = torch.where(t1 > 1e-9, t1, torch.where(t2 > 1e-9, t2, inf))
            t = torch.where(disc >= 0, torch.minimum(t, ts), t)
        if noise:
            t = t + torch.randn(t.shape, generator=gen, dtype=torch.float64, device=device) * noise_scale * t * t
        valid = (t > K["z_min"]) & (t <= K["z_max"]) & torch.isfinite(t)
        out[s:s + n] = torch.where(valid, t, torch.zeros_like(t)).to(torch.float32)
    return out


# --------------------------------------------------------------------------- trajectories
def make_trajectory(scene: Scene, n_frames: int, speed: float, ang_speed: float, seed: int,
                    fps: float = 30.0, walk_sigma: float = 0.05, scan_gain: float = 3.0) -> np.ndarray:
    """(n_frames, 7) camera->world poses at constant linear speed (m/s) and
    angular speed (rad/s); the direction and the rotation axis follow smooth
    seeded random walks (walk_sigma per frame); the path reflects off planes
    `margin` inside the walls (camera_margin) and off spheres.  Rendering the
    same motion statistics at k x fps takes walk_sigma / sqrt(k).

    Scanning: each frame's rotation axis is the random-walk axis plus
    scan_gain * (z_cam x (room centre - position)) (metres), which turns the
    optical axis back towards the room's interior the further the camera is
    from the centre, as a hand-held scan of a room does; a camera staring at
    one flat wall from close by is the failure case the paper names for any
    purely geometric tracker (Sec. 5.6).  scan_gain = 0 gives the plain random
    walk starting at the room centre."""
    rng = np.random.default_rng(20_000 + seed)
    margin = camera_margin(scene)
    lo, hi = scene.lo + margin, scene.hi - margin
    centre = 0.5 * (scene.lo + scene.hi)

    def free(p):
        return all(np.linalg.norm(p - c) > r + 0.5 for c, r in zip(scene.centres, scene.radii))

    # start in the camera's box, clear of the spheres and (when scanning) at least
    # 1 m from the room centre, so that the first frames already look across the room
    p = centre.copy()
    for _ in range(1000):
        if free(p) and (scan_gain == 0.0 or np.linalg.norm(p - centre) >= min(1.0, 0.5 * float((hi - lo).min()))):
            break
        p = rng.uniform(lo, hi)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    q = look_at_quat(p, p + rng.normal(size=3))
    dt = 1.0 / fps
    out = np.zeros((n_frames, 7))
    for f in range(n_frames):
        out[f, :4] = q
        out[f, 4:] = p
        d = d + rng.normal(size=3) * walk_sigma
        d /= np.linalg.norm(d)
        nxt = p + speed * dt * d
        for a in range(3):
            if (nxt[a] < lo[a] and d[a] < 0) or (nxt[a] > hi[a] and d[a] > 0):
                d[a] = -d[a]
        for c, r in zip(scene.centres, scene.radii):
            n = nxt - c
            dist = np.linalg.norm(n)
            if dist < r + 0.5 and d @ n < 0:
                n /= dist
                d = d - 2 * (d @ n) * n
        p = np.clip(p + speed * dt * d, lo, hi)
        axis = axis + rng.normal(size=3) * walk_sigma
        axis /= np.linalg.norm(axis)
        turn = axis + scan_gain * np.cross(_qrot(q)[:, 2], centre - out[f, 4:])
        q = _qcanon(_qmul(axis_angle_quat(turn, ang_speed * dt), q))
    return out


# --------------------------------------------------------------------------- volumes written directly
def analytic_tsdf(sdf_fn, dims, voxel: float, origin, trunc: float, observed_band: float | None = None):
    """Normalised truncated SDF sampled at voxel centres: F = clip(sdf / trunc, -1, 1),
    NaN where sdf < -observed_band (never observed behind the surface).
    Returns a float64 array shaped (dz, dy, dx)."""
    dx, dy, dz = dims
    o = np.asarray(origin, np.float64)
    F = np.empty((dz, dy, dx), np.float64)
    y, x = np.meshgrid((np.arange(dy) + 0.5) * voxel + o[1], (np.arange(dx) + 0.5) * voxel + o[0], indexing="ij")
    for k in range(dz):  # one z slab at a time keeps 512^3 fills within a few hundred MB
        z = np.full_like(x, (k + 0.5) * voxel + o[2])
        s = sdf_fn(np.stack([x, y, z], axis=-1))
        f = np.clip(s / trunc, -1.0, 1.0)
        if observed_band is not None:
            f = np.where(s < -observed_band, np.nan, f)
        F[k] = f
    return F


def analytic_tsdf_torch(scene: Scene, dims, voxel: float, origin, trunc: float, observed_band: float | None = None,
                        device="cuda"):
    """analytic_tsdf evaluated with torch on the device (float32 values, NaN where
    unobserved), for 512^3 volumes; shaped (dz, dy, dx)."""
    import torch

    dx, dy, dz = dims
    o = [float(v) for v in origin]
    lo = torch.as_tensor(scene.lo, dtype=torch.float64, device=device)
    hi = torch.as_tensor(scene.hi, dtype=torch.float64, device=device)
    yy, xx = torch.meshgrid((torch.arange(dy, dtype=torch.float64, device=device) + 0.5) * voxel + o[1],
                            (torch.arange(dx, dtype=torch.float64, device=device) + 0.5) * voxel + o[0], indexing="ij")
    F = torch.empty((dz, dy, dx), dtype=torch.float32, device=device)
    for k in range(dz):
        p = torch.stack([xx, yy, torch.full_like(xx, (k + 0.5) * voxel + o[2])], -1)
        d = torch.minimum(p - lo, hi - p).amin(-1)
        for c, r in zip(scene.centres, scene.radii):
            d = torch.minimum(d, torch.linalg.norm(p - torch.as_tensor(c, dtype=torch.float64, device=device), dim=-1)
                              - float(r))
        f = torch.clamp(d / trunc, -1.0, 1.0)
        if observed_band is not None:
            f = torch.where(d < -observed_band, torch.full_like(f, float("nan")), f)
        F[k] = f.to(torch.float32)
    return F


def encode_values(F: np.ndarray, dtype: str) -> np.ndarray:
    """Storage codes of normalised TSDF values: float32 / float16 with NaN for
    unobserved, or int16 round(F * 32767) with -32768 for unobserved."""
    if dtype == "f32":
        return F.astype(np.float32)
    if dtype == "f16":
        return F.astype(np.float16)
    if dtype == "i16":
        c = np.where(np.isnan(F), -32768, np.clip(np.rint(np.nan_to_num(F) * 32767.0), -32767, 32767))
        return c.astype(np.int16)
    raise ValueError(dtype)


def decode_values(codes: np.ndarray) -> np.ndarray:
    """Exact float64 values of storage codes (inverse of encode_values)."""
    if codes.dtype == np.int16:
        F = codes.astype(np.float64) / 32767.0
        return np.where(codes == -32768, np.nan, F)
    return codes.astype(np.float64)


def random_pst_offsets(n, seed):
    """Generic random 6-vectors in the unit ball for host-side tests (not a PST)."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 6))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v *= rng.uniform(size=(n, 1)) ** (1.0 / 6.0)
    return v
