"""Analytic G-buffers: what a rasteriser would hand the fragment stage.

Each pixel gets the surface UV of the nearest hit (FP32), the unit vector from
the surface point to the eye expressed in the surface's tangent frame
(x along dP/du, y along dP/dv, z along the outward normal; FP64 then FP32),
and the id of the object hit (-1 for a miss, whose UV and direction are 0).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np


@dataclass
class GBuffer:
    uv: np.ndarray    # F x 2 float32
    dir: np.ndarray   # F x 3 float32
    obj: np.ndarray   # F int32
    width: int
    height: int
    views: int

    @property
    def F(self) -> int:
        return int(self.obj.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _normalize(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _camera_rays(eye, target, width: int, height: int, fov_deg: float, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Unit ray directions (height*width x 3, row-major, row 0 at the top) of a pinhole camera."""
    eye = np.asarray(eye, dtype=np.float64)
    f = _normalize(np.asarray(target, dtype=np.float64) - eye)
    up = np.asarray(up, dtype=np.float64)
    if abs(float(np.dot(f, up))) > 0.999:
        up = np.array([0.0, 1.0, 0.0]) if abs(up[1]) < 0.5 else np.array([1.0, 0.0, 0.0])
    r = _normalize(np.cross(f, up))
    u = np.cross(r, f)
    th = np.tan(np.radians(fov_deg) / 2.0)
    aspect = width / height
    x = (2.0 * (np.arange(width) + 0.5) / width - 1.0) * th * aspect
    y = (1.0 - 2.0 * (np.arange(height) + 0.5) / height) * th
    rays = f[None, None, :] + x[None, :, None] * r[None, None, :] + y[:, None, None] * u[None, None, :]
    return _normalize(rays.reshape(-1, 3))


def quad_scene(seed: int, width: int = 256, height: int = 256, fov_deg: float = 50.0) -> GBuffer:
    """The quad [-1, 1]^2 at z = 0 (normal +z, UV = ((x+1)/2, (y+1)/2), tangent
    frame = world axes) seen by a pinhole camera whose eye lies on the upper
    hemisphere (cosine of the polar angle U[0.2, 1]) at distance U[2, 3] from a
    seeded point of the quad it looks at.  One object, id 0."""
    rng = _rng(seed)
    target = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), 0.0])
    z = rng.uniform(0.2, 1.0)
    phi = rng.uniform(0.0, 2.0 * np.pi)
    dist = rng.uniform(2.0, 3.0)
    s = np.sqrt(1.0 - z * z)
    eye = target + dist * np.array([s * np.cos(phi), s * np.sin(phi), z])
    rays = _camera_rays(eye, target, width, height, fov_deg, up=(0.0, 0.0, 1.0))
    F = rays.shape[0]
    uv = np.zeros((F, 2))
    d = np.zeros((F, 3))
    obj = np.full(F, -1, dtype=np.int32)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = -eye[2] / rays[:, 2]
    P = eye[None, :] + t[:, None] * rays
    hit = (rays[:, 2] < 0) & (np.abs(P[:, 0]) <= 1.0) & (np.abs(P[:, 1]) <= 1.0)
    uv[hit, 0] = (P[hit, 0] + 1.0) / 2.0
    uv[hit, 1] = (P[hit, 1] + 1.0) / 2.0
    d[hit] = _normalize(eye[None, :] - P[hit])
    obj[hit] = 0
    return GBuffer(uv.astype(np.float32), d.astype(np.float32), obj, width, height, 1)


def _sphere_plane_view(eye: np.ndarray, width: int, height: int, fov_deg: float, plane_half: float,
                       uv_out: np.ndarray, dir_out: np.ndarray, obj_out: np.ndarray) -> None:
    """Ray-cast the unit sphere (id 0) and the ground plane y = -1, |x|, |z| <= plane_half (id 1)."""
    rays = _camera_rays(eye, (0.0, 0.0, 0.0), width, height, fov_deg, up=(0.0, 1.0, 0.0))
    F = rays.shape[0]
    b = rays @ eye
    c = float(eye @ eye) - 1.0
    disc = b * b - c
    t_s = np.full(F, np.inf)
    ok = disc >= 0.0
    ts = -b[ok] - np.sqrt(disc[ok])
    t_s[ok] = np.where(ts > 0.0, ts, np.inf)
    t_p = np.full(F, np.inf)
    down = rays[:, 1] < 0.0
    tp = (-1.0 - eye[1]) / rays[down, 1]
    Pp = eye[None, :] + tp[:, None] * rays[down]
    inside = (np.abs(Pp[:, 0]) <= plane_half) & (np.abs(Pp[:, 2]) <= plane_half) & (tp > 0.0)
    tmp = np.full(tp.shape, np.inf)
    tmp[inside] = tp[inside]
    t_p[down] = tmp
    sph = np.isfinite(t_s) & (t_s <= t_p)
    pln = np.isfinite(t_p) & ~sph

    uv_out[:] = 0.0
    dir_out[:] = 0.0
    obj_out[:] = -1

    # Sphere: lat-long UV, u = (phi + pi) / 2 pi with phi = atan2(z, x), v = theta / pi with
    # theta the polar angle from +y; tangent x along dP/dphi, y along dP/dtheta, z = P.
    P = eye[None, :] + t_s[sph, None] * rays[sph]
    P = _normalize(P)
    theta = np.arccos(np.clip(P[:, 1], -1.0, 1.0))
    phi = np.arctan2(P[:, 2], P[:, 0])
    polar = (P[:, 0] ** 2 + P[:, 2] ** 2) < 1e-24
    phi = np.where(polar, 0.0, phi)
    T = np.stack([-np.sin(phi), np.zeros_like(phi), np.cos(phi)], axis=1)
    Bv = np.stack([np.cos(theta) * np.cos(phi), -np.sin(theta), np.cos(theta) * np.sin(phi)], axis=1)
    I = _normalize(eye[None, :] - P)
    uv_out[sph, 0] = (phi + np.pi) / (2.0 * np.pi)
    uv_out[sph, 1] = theta / np.pi
    dir_out[sph, 0] = np.einsum("ij,ij->i", I, T)
    dir_out[sph, 1] = np.einsum("ij,ij->i", I, Bv)
    dir_out[sph, 2] = np.einsum("ij,ij->i", I, P)
    obj_out[sph] = 0

    # Plane: UV = ((x + h) / 2h, (z + h) / 2h); tangent frame (+x, +z, +y).
    P = eye[None, :] + t_p[pln, None] * rays[pln]
    I = _normalize(eye[None, :] - P)
    uv_out[pln, 0] = (P[:, 0] + plane_half) / (2.0 * plane_half)
    uv_out[pln, 1] = (P[:, 2] + plane_half) / (2.0 * plane_half)
    dir_out[pln, 0] = I[:, 0]
    dir_out[pln, 1] = I[:, 2]
    dir_out[pln, 2] = I[:, 1]
    obj_out[pln] = 1


def sphere_plane_poses(seed: int, views: int = 60, radius: float = 3.5, step_deg: float = 6.0) -> np.ndarray:
    """Eye positions of an orbit around the origin: azimuth step_deg apart from a
    seeded start, elevation U[10, 40] degrees per pose.  views x 3."""
    rng = _rng(seed)
    az0 = rng.uniform(0.0, 2.0 * np.pi)
    el = np.radians(rng.uniform(10.0, 40.0, views))
    az = az0 + np.radians(step_deg) * np.arange(views)
    return radius * np.stack([np.cos(el) * np.cos(az), np.sin(el), np.cos(el) * np.sin(az)], axis=1)


def sphere_plane_scene(seed: int, views: int = 60, width: int = 1920, height: int = 1080, fov_deg: float = 60.0,
                       plane_half: float = 4.0, view_range: tuple[int, int] | None = None,
                       out: tuple[np.ndarray, np.ndarray, np.ndarray] | None = None,
                       threads: int | None = None) -> GBuffer:
    """Unit sphere (id 0) plus ground plane (id 1) from `views` orbit poses,
    stacked view-major (view, row, column).  view_range selects a contiguous
    subset of the poses (for sharding across ranks); `out` supplies the
    destination arrays (e.g. pinned host memory) of shape (F, 2), (F, 3), (F,)."""
    eyes = sphere_plane_poses(seed, views)
    lo, hi = view_range if view_range is not None else (0, views)
    per = width * height
    F = (hi - lo) * per
    if out is None:
        uv = np.empty((F, 2), dtype=np.float32)
        d = np.empty((F, 3), dtype=np.float32)
        obj = np.empty(F, dtype=np.int32)
    else:
        uv, d, obj = out
    def one(k):
        sl = slice(k * per, (k + 1) * per)
        _sphere_plane_view(eyes[lo + k], width, height, fov_deg, plane_half, uv[sl], d[sl], obj[sl])

    # numpy releases the GIL inside large array operations, so views render in parallel threads
    workers = max(1, min(hi - lo, threads or (os.cpu_count() or 1)))
    if workers == 1:
        for k in range(hi - lo):
            one(k)
    else:
        with ThreadPoolExecutor(workers) as ex:
            list(ex.map(one, range(hi - lo)))
    return GBuffer(uv, d, obj, width, height, hi - lo)


def voronoi_planes_scene(seed: int, n_objects: int = 64, views: int = 4, width: int = 3840, height: int = 2160,
                         fov_deg: float = 60.0, view_range: tuple[int, int] | None = None) -> GBuffer:
    """Many objects on one screen: the screen is split into Voronoi regions of
    n_objects seeded sites; region k shows object k as a plane at a seeded pose
    (normal tilted up to 60 degrees from the view axis, distance U[2, 6]) seen by
    the view's pinhole camera, with UV clamped to [0, 1] (plane extent 2 x 2)."""
    rng = _rng(seed)
    lo, hi = view_range if view_range is not None else (0, views)
    per = width * height
    F = (hi - lo) * per
    uv = np.empty((F, 2), dtype=np.float32)
    d = np.empty((F, 3), dtype=np.float32)
    obj = np.empty(F, dtype=np.int32)
    sites_all = rng.uniform(0.0, 1.0, (views, n_objects, 2))
    tilt = np.radians(rng.uniform(0.0, 60.0, (views, n_objects)))
    spin = rng.uniform(0.0, 2.0 * np.pi, (views, n_objects))
    roll = rng.uniform(0.0, 2.0 * np.pi, (views, n_objects))
    dist = rng.uniform(2.0, 6.0, (views, n_objects))
    th = np.tan(np.radians(fov_deg) / 2.0)
    aspect = width / height
    xs = (2.0 * (np.arange(width) + 0.5) / width - 1.0) * th * aspect
    ys = (1.0 - 2.0 * (np.arange(height) + 0.5) / height) * th
    def one(k):
        v = lo + k
        sl = slice(k * per, (k + 1) * per)
        # Voronoi region of every pixel (screen coordinates in [0, 1]^2), chunked by rows.
        region = np.empty((height, width), dtype=np.int32)
        px = (np.arange(width) + 0.5) / width
        sites = sites_all[v]
        for r0 in range(0, height, 256):
            r1 = min(height, r0 + 256)
            py = (np.arange(r0, r1) + 0.5) / height
            dx = px[None, :, None] - sites[None, None, :, 0]
            dy = py[:, None, None] - sites[None, None, :, 1]
            region[r0:r1] = np.argmin(dx * dx + dy * dy, axis=2)
        region = region.reshape(-1)
        # Camera at the origin looking down -z; ray of each pixel.
        rays = np.empty((height, width, 3))
        rays[..., 0] = xs[None, :]
        rays[..., 1] = ys[:, None]
        rays[..., 2] = -1.0
        rays = _normalize(rays.reshape(-1, 3))
        uvv = np.zeros((per, 2))
        dd = np.zeros((per, 3))
        oo = np.full(per, -1, dtype=np.int32)
        for o in range(n_objects):
            m = region == o
            if not m.any():
                continue
            # Plane through C = dist * (ray of the site) with normal N tilted from the view axis.
            sx = (2.0 * sites[o, 0] - 1.0) * th * aspect
            sy = (1.0 - 2.0 * sites[o, 1]) * th
            cdir = _normalize(np.array([sx, sy, -1.0]))
            C = dist[v, o] * cdir
            back = -cdir
            helper = np.array([0.0, 1.0, 0.0]) if abs(back[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
            e1 = _normalize(np.cross(helper, back))
            e2 = np.cross(back, e1)
            N = np.cos(tilt[v, o]) * back + np.sin(tilt[v, o]) * (np.cos(spin[v, o]) * e1 + np.sin(spin[v, o]) * e2)
            t1 = _normalize(np.cross(N, helper if abs(N @ helper) < 0.9 else np.array([1.0, 0.0, 0.0])))
            t2 = np.cross(N, t1)
            Tx = np.cos(roll[v, o]) * t1 + np.sin(roll[v, o]) * t2
            Ty = np.cross(N, Tx)
            R = rays[m]
            denom = R @ N
            t = (C @ N) / denom
            P = t[:, None] * R
            rel = P - C[None, :]
            u = np.clip(0.5 + 0.5 * (rel @ Tx), 0.0, 1.0)
            w = np.clip(0.5 + 0.5 * (rel @ Ty), 0.0, 1.0)
            I = _normalize(-P)
            front = (t > 0) & (denom < 0)
            idx = np.nonzero(m)[0]
            uvv[idx, 0] = np.where(front, u, 0.0)
            uvv[idx, 1] = np.where(front, w, 0.0)
            dd[idx, 0] = np.where(front, I @ Tx, 0.0)
            dd[idx, 1] = np.where(front, I @ Ty, 0.0)
            dd[idx, 2] = np.where(front, I @ N, 0.0)
            oo[idx] = np.where(front, o, -1)
        uv[sl] = uvv
        d[sl] = dd
        obj[sl] = oo

    # numpy releases the GIL inside large array operations: views render in parallel threads
    with ThreadPoolExecutor(max(1, min(hi - lo, os.cpu_count() or 1))) as ex:
        list(ex.map(one, range(hi - lo)))
    return GBuffer(uv, d, obj, width, height, hi - lo)


def quad_views(seed: int, views: int, width: int, height: int, fov_deg: float = 50.0) -> GBuffer:
    """`views` pinhole views of the quad (each drawn like quad_scene with seed
    seed + k), stacked view-major."""
    gs = [quad_scene(seed + k, width, height, fov_deg) for k in range(views)]
    return GBuffer(np.concatenate([g.uv for g in gs]), np.concatenate([g.dir for g in gs]),
                   np.concatenate([g.obj for g in gs]), width, height, views)
