"""Seeded synthetic scenes and scans for the S-BKI map update.

This module only produces *inputs*: labelled points in a sensor frame plus the
sensor pose, in the shapes of the paper's workloads (a single ray-cast scan, a
64-beam LiDAR street sequence, a pinhole depth-camera sequence, and mixed-size
scans for independent maps).  It contains none of the mapping arithmetic
(no free-space sampling, voxelisation, kernel or Dirichlet update); the oracle
and the CUDA path both consume what it returns.

Geometry is analytic ray casting against axis-aligned boxes, vertical
cylinders, ellipsoids and a ground plane, in float64, followed by the stated
noise models.  Every random draw comes from ``numpy.random.Generator(PCG64)``
with the seed given, so a config and seed always give the same bytes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# scene description
# --------------------------------------------------------------------------


@dataclass
class Scene:
    """Primitives of a static scene; every surface carries one class id >= 1."""

    # ground plane z = 0 limited to [x0, x1] x [y0, y1]; class chosen per hit by
    # ``ground_bands``: list of (|y| upper bound, class) applied in order.
    ground_rect: tuple = (-10.0, 10.0, -10.0, 10.0)
    ground_bands: list = field(default_factory=lambda: [(math.inf, 1)])
    boxes_lo: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    boxes_hi: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    boxes_cls: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    cyl: np.ndarray = field(default_factory=lambda: np.zeros((0, 5)))  # cx, cy, r, z0, z1
    cyl_cls: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    ell_c: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    ell_r: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    ell_cls: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    num_classes: int = 10

    def add_box(self, lo, hi, cls):
        self.boxes_lo = np.vstack([self.boxes_lo, np.asarray(lo, float)[None]])
        self.boxes_hi = np.vstack([self.boxes_hi, np.asarray(hi, float)[None]])
        self.boxes_cls = np.append(self.boxes_cls, np.int32(cls))

    def add_cyl(self, cx, cy, r, z0, z1, cls):
        self.cyl = np.vstack([self.cyl, np.array([[cx, cy, r, z0, z1]], float)])
        self.cyl_cls = np.append(self.cyl_cls, np.int32(cls))

    def add_ell(self, c, radii, cls):
        self.ell_c = np.vstack([self.ell_c, np.asarray(c, float)[None]])
        self.ell_r = np.vstack([self.ell_r, np.asarray(radii, float)[None]])
        self.ell_cls = np.append(self.ell_cls, np.int32(cls))

    def contains(self, p, margin=0.0):
        """True if point p lies inside (or within margin of) any solid."""
        p = np.asarray(p, float)
        if len(self.boxes_lo) and np.any(np.all((p >= self.boxes_lo - margin) & (p <= self.boxes_hi + margin), axis=1)):
            return True
        if len(self.cyl):
            d = np.hypot(p[0] - self.cyl[:, 0], p[1] - self.cyl[:, 1])
            if np.any((d <= self.cyl[:, 2] + margin) & (p[2] >= self.cyl[:, 3] - margin) & (p[2] <= self.cyl[:, 4] + margin)):
                return True
        if len(self.ell_c):
            q = (p - self.ell_c) / (self.ell_r + margin)
            if np.any(np.sum(q * q, axis=1) <= 1.0):
                return True
        return False


# --------------------------------------------------------------------------
# analytic ray casting (float64)
# --------------------------------------------------------------------------

_CHUNK = 2048


def _cull(scene: Scene, origin, max_range):
    """Indices of primitives whose bounding box comes within max_range of origin."""
    o = np.asarray(origin, float)

    def near(lo, hi):
        q = np.clip(o, lo, hi)
        return np.nonzero(np.linalg.norm(q - o, axis=1) <= max_range)[0]

    ib = near(scene.boxes_lo, scene.boxes_hi) if len(scene.boxes_lo) else np.zeros(0, int)
    if len(scene.cyl):
        clo = np.stack([scene.cyl[:, 0] - scene.cyl[:, 2], scene.cyl[:, 1] - scene.cyl[:, 2], scene.cyl[:, 3]], 1)
        chi = np.stack([scene.cyl[:, 0] + scene.cyl[:, 2], scene.cyl[:, 1] + scene.cyl[:, 2], scene.cyl[:, 4]], 1)
        ic = near(clo, chi)
    else:
        ic = np.zeros(0, int)
    ie = near(scene.ell_c - scene.ell_r, scene.ell_c + scene.ell_r) if len(scene.ell_c) else np.zeros(0, int)
    return ib, ic, ie


def _az_interval(o, lo, hi):
    """Conservative azimuth interval (centre, half width) of xy boxes seen from o."""
    cx = np.stack([lo[:, 0], hi[:, 0], lo[:, 0], hi[:, 0]], 1) - o[0]
    cy = np.stack([lo[:, 1], lo[:, 1], hi[:, 1], hi[:, 1]], 1) - o[1]
    mid = np.arctan2(0.5 * (lo[:, 1] + hi[:, 1]) - o[1], 0.5 * (lo[:, 0] + hi[:, 0]) - o[0])
    ang = np.arctan2(cy, cx)
    dev = np.abs((ang - mid[:, None] + np.pi) % (2 * np.pi) - np.pi)
    half = dev.max(axis=1) + 1e-6
    inside = (o[0] >= lo[:, 0] - 1e-9) & (o[0] <= hi[:, 0] + 1e-9) & (o[1] >= lo[:, 1] - 1e-9) & (o[1] <= hi[:, 1] + 1e-9)
    half = np.where(inside | (half > np.pi / 2), np.pi, half)
    return mid, half


def _sel(mid, half, a_mid, a_half):
    if len(mid) == 0:
        return np.zeros(0, int)
    dev = np.abs((mid - a_mid + np.pi) % (2 * np.pi) - np.pi)
    return np.nonzero(dev <= half + a_half)[0]


def raycast(scene: Scene, origin, dirs, max_range):
    """First-hit distance and class for unit rays from one origin.

    Rays are processed in chunks of similar azimuth; only primitives whose
    azimuth interval overlaps the chunk's are tested (a conservative cull).
    Returns (t, cls): t = inf and cls = 0 where nothing is hit within max_range.
    """
    o = np.asarray(origin, float)
    dirs = np.asarray(dirs, float)
    n = len(dirs)
    t_out = np.full(n, np.inf)
    c_out = np.zeros(n, np.int32)
    ib, ic, ie = _cull(scene, o, max_range)
    blo, bhi, bcl = scene.boxes_lo[ib], scene.boxes_hi[ib], scene.boxes_cls[ib]
    cy, ccl = scene.cyl[ic], scene.cyl_cls[ic]
    ec, er, ecl = scene.ell_c[ie], scene.ell_r[ie], scene.ell_cls[ie]
    b_mid, b_half = _az_interval(o, blo, bhi)
    c_mid, c_half = _az_interval(o, np.stack([cy[:, 0] - cy[:, 2], cy[:, 1] - cy[:, 2]], 1) if len(cy) else np.zeros((0, 2)),
                                 np.stack([cy[:, 0] + cy[:, 2], cy[:, 1] + cy[:, 2]], 1) if len(cy) else np.zeros((0, 2)))
    e_mid, e_half = _az_interval(o, ec - er, ec + er)
    x0, x1, y0, y1 = scene.ground_rect
    az = np.arctan2(dirs[:, 1], dirs[:, 0])
    order = np.argsort(az, kind="stable")
    for s in range(0, n, _CHUNK):
        idx = order[s:s + _CHUNK]
        d = dirs[idx]
        m = len(d)
        a = az[idx]
        a_mid = 0.5 * (a[0] + a[-1])
        a_half = 0.5 * (a[-1] - a[0]) + 1e-6
        if np.any(np.abs(d[:, 0]) + np.abs(d[:, 1]) < 1e-9):
            a_half = np.pi  # vertical rays: no azimuth cull
        best = np.full(m, np.inf)
        bcls = np.zeros(m, np.int32)
        # ground plane z = 0
        with np.errstate(divide="ignore", invalid="ignore"):
            tg = np.where(d[:, 2] < -1e-12, -o[2] / d[:, 2], np.inf)
        fin = np.isfinite(tg)
        tf = np.where(fin, tg, 0.0)  # rays that miss the plane: no inf * 0
        gx = o[0] + tf * d[:, 0]
        gy = o[1] + tf * d[:, 1]
        okg = fin & (gx >= x0) & (gx <= x1) & (gy >= y0) & (gy <= y1)
        tg = np.where(okg, tg, np.inf)
        gcls = np.zeros(m, np.int32)
        ay = np.abs(gy)
        assigned = np.zeros(m, bool)
        for bound, cls in scene.ground_bands:
            sel = (~assigned) & (ay < bound)
            gcls[sel] = cls
            assigned |= sel
        upd = tg < best
        best = np.where(upd, tg, best)
        bcls = np.where(upd, gcls, bcls)
        # axis-aligned boxes (slab test), rays x boxes
        jb = _sel(b_mid, b_half, a_mid, a_half)
        if len(jb):
            lo, hi, cl = blo[jb], bhi[jb], bcl[jb]
            dd = np.where(np.abs(d) < 1e-12, 1e-12, d)
            inv = 1.0 / dd
            t1 = (lo[None, :, :] - o[None, None, :]) * inv[:, None, :]
            t2 = (hi[None, :, :] - o[None, None, :]) * inv[:, None, :]
            tn = np.max(np.minimum(t1, t2), axis=2)
            tf = np.min(np.maximum(t1, t2), axis=2)
            hit = (tf >= tn) & (tn > 1e-9)
            tb = np.where(hit, tn, np.inf)
            j = np.argmin(tb, axis=1)
            tbm = tb[np.arange(m), j]
            upd = tbm < best
            best = np.where(upd, tbm, best)
            bcls = np.where(upd, cl[j], bcls)
        # vertical cylinders: side wall and top cap
        jc = _sel(c_mid, c_half, a_mid, a_half)
        if len(jc):
            cyl, cl = cy[jc], ccl[jc]
            ox = o[0] - cyl[None, :, 0]
            oy = o[1] - cyl[None, :, 1]
            qa = (d[:, 0:1] ** 2 + d[:, 1:2] ** 2)
            qb = 2.0 * (d[:, 0:1] * ox + d[:, 1:2] * oy)
            qc = ox * ox + oy * oy - cyl[None, :, 2] ** 2
            disc = qb * qb - 4.0 * qa * qc
            with np.errstate(invalid="ignore", divide="ignore"):
                ts = (-qb - np.sqrt(np.maximum(disc, 0.0))) / (2.0 * qa)
            zs = o[2] + ts * d[:, 2:3]
            side = (disc >= 0) & (qa > 1e-18) & (ts > 1e-9) & (zs >= cyl[None, :, 3]) & (zs <= cyl[None, :, 4])
            tside = np.where(side, ts, np.inf)
            with np.errstate(invalid="ignore", divide="ignore"):
                tc = np.where(np.abs(d[:, 2:3]) > 1e-12, (cyl[None, :, 4] - o[2]) / d[:, 2:3], np.inf)
            cxh = o[0] + tc * d[:, 0:1] - cyl[None, :, 0]
            cyh = o[1] + tc * d[:, 1:2] - cyl[None, :, 1]
            cap = np.isfinite(tc) & (tc > 1e-9) & (cxh * cxh + cyh * cyh <= cyl[None, :, 2] ** 2)
            tcap = np.where(cap, tc, np.inf)
            tt = np.minimum(tside, tcap)
            j = np.argmin(tt, axis=1)
            ttm = tt[np.arange(m), j]
            upd = ttm < best
            best = np.where(upd, ttm, best)
            bcls = np.where(upd, cl[j], bcls)
        # ellipsoids
        je = _sel(e_mid, e_half, a_mid, a_half)
        if len(je):
            c0, r0, cl = ec[je], er[je], ecl[je]
            op = (o[None, None, :] - c0[None, :, :]) / r0[None, :, :]
            dp = d[:, None, :] / r0[None, :, :]
            qa = np.sum(dp * dp, axis=2)
            qb = 2.0 * np.sum(op * dp, axis=2)
            qc = np.sum(op * op, axis=2) - 1.0
            disc = qb * qb - 4.0 * qa * qc
            with np.errstate(invalid="ignore"):
                te = (-qb - np.sqrt(np.maximum(disc, 0.0))) / (2.0 * qa)
            te = np.where((disc >= 0) & (te > 1e-9), te, np.inf)
            j = np.argmin(te, axis=1)
            tem = te[np.arange(m), j]
            upd = tem < best
            best = np.where(upd, tem, best)
            bcls = np.where(upd, cl[j], bcls)
        far = best > max_range
        best[far] = np.inf
        bcls[far] = 0
        t_out[idx] = best
        c_out[idx] = bcls
    return t_out, c_out


# --------------------------------------------------------------------------
# poses and sensors
# --------------------------------------------------------------------------


def pose_matrix(position, yaw=0.0, pitch=0.0, roll=0.0, base=None):
    """4x4 row-major world_from_sensor: R = Rz(yaw) Ry(pitch) Rx(roll) [@ base]."""
    cz, sz = math.cos(yaw), math.sin(yaw)
    cyy, syy = math.cos(pitch), math.sin(pitch)
    cx, sx = math.cos(roll), math.sin(roll)
    rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1.0]])
    ry = np.array([[cyy, 0, syy], [0, 1.0, 0], [-syy, 0, cyy]])
    rx = np.array([[1.0, 0, 0], [0, cx, -sx], [0, sx, cx]])
    r = rz @ ry @ rx
    if base is not None:
        r = r @ base
    t = np.eye(4)
    t[:3, :3] = r
    t[:3, 3] = position
    return t


def lidar_dirs(n_beams, n_az, el_top_deg, el_bot_deg):
    """Unit ray directions in the sensor frame, beam-major order."""
    el = np.deg2rad(np.linspace(el_top_deg, el_bot_deg, n_beams))
    az = 2.0 * np.pi * np.arange(n_az) / n_az
    e, a = np.meshgrid(el, az, indexing="ij")
    d = np.stack([np.cos(e) * np.cos(a), np.cos(e) * np.sin(a), np.sin(e)], -1)
    return d.reshape(-1, 3)


# camera frame: x right, y down, z forward; expressed in a world-aligned frame
# whose forward is +x and up is +z by this fixed rotation.
_CAM_TO_FLU = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])


def _label_noise(rng, labels, frac, num_classes, candidates=None):
    """Replace a fraction of labels by a different class drawn uniformly."""
    n = len(labels)
    k = int(round(frac * n))
    if k == 0:
        return labels
    if candidates is None:
        idx = rng.choice(n, size=k, replace=False)
    else:
        cand = np.asarray(candidates)
        if len(cand) >= k:
            idx = rng.choice(cand, size=k, replace=False)
        else:
            rest = np.setdiff1d(np.arange(n), cand)
            idx = np.concatenate([cand, rng.choice(rest, size=k - len(cand), replace=False)])
    off = rng.integers(1, num_classes, size=len(idx))  # 1..K-1: never the same class
    lab = labels.copy()
    lab[idx] = (labels[idx] - 1 + off) % num_classes + 1
    return lab


def _scan(scene, pose, dirs_sensor, max_range, range_sigma, rng, min_range=0.0):
    """Cast sensor rays, keep hits, add Gaussian range noise; sensor-frame output."""
    r = pose[:3, :3]
    o = pose[:3, 3]
    dw = dirs_sensor @ r.T
    t, cls = raycast(scene, o, dw, max_range)
    ok = np.isfinite(t) & (t >= min_range)
    t = t[ok]
    ds = dirs_sensor[ok]
    cls = cls[ok]
    if range_sigma > 0:
        t = t + rng.normal(0.0, range_sigma, size=len(t))
    pts = (ds * t[:, None]).astype(np.float32)
    return pts, cls.astype(np.int32)


# --------------------------------------------------------------------------
# workload 0: one ray-cast scan of a small walled region
# --------------------------------------------------------------------------

SMALL_SCENE_PARAMS = dict(res=0.1, length_scale=0.3, sigma0=1.0, alpha0=0.001, free_step=0.3,
                          num_classes=10, min_range=0.0, max_range=100.0)


def small_region_scene(seed=0, keep_clear_band=1.3):
    """20x20x4 m region: ground (class 1), 4 walls (class 2), 6 boxes (3..8),
    4 vertical cylinders (9, 10).  Solids keep out of the band |y| < keep_clear_band
    for |x| < 6 and of a disc around the origin, so sensors placed there are in free space."""
    rng = np.random.default_rng(seed)
    sc = Scene(num_classes=10)
    sc.ground_rect = (-10.0, 10.0, -10.0, 10.0)
    sc.ground_bands = [(math.inf, 1)]
    th = 0.2
    sc.add_box([-10 - th, -10 - th, 0], [-10, 10 + th, 4], 2)
    sc.add_box([10, -10 - th, 0], [10 + th, 10 + th, 4], 2)
    sc.add_box([-10, -10 - th, 0], [10, -10, 4], 2)
    sc.add_box([-10, 10, 0], [10, 10 + th, 4], 2)

    def clear(cx, cy, half):
        if abs(cx) < 6.0 + half and abs(cy) < keep_clear_band + half:
            return False
        return math.hypot(cx, cy) > 2.0 + half

    placed = 0
    while placed < 6:
        sz = rng.uniform(0.5, 3.0, size=3)
        c = rng.uniform(-9.0 + sz[:2] / 2, 9.0 - sz[:2] / 2)
        if not clear(c[0], c[1], max(sz[0], sz[1]) / 2):
            continue
        sc.add_box([c[0] - sz[0] / 2, c[1] - sz[1] / 2, 0.0], [c[0] + sz[0] / 2, c[1] + sz[1] / 2, sz[2]], 3 + placed)
        placed += 1
    placed = 0
    while placed < 4:
        r = rng.uniform(0.15, 0.5)
        h = rng.uniform(1.0, 4.0)
        c = rng.uniform(-9.0, 9.0, size=2)
        if not clear(c[0], c[1], r):
            continue
        sc.add_cyl(c[0], c[1], r, 0.0, h, 9 + (placed % 2))
        placed += 1
    return sc


def small_region_scan(seed=0, n_az=100, n_el=100, el_half_deg=15.0, range_sigma=0.02, label_noise=0.05):
    """A single scan: sensor at (0, 0, 1.5), n_az x n_el rays over 360 x 30 degrees."""
    sc = small_region_scene(seed)
    rng = np.random.default_rng(seed + 1000)
    el = np.deg2rad(rng.uniform(-el_half_deg, el_half_deg, size=n_el))
    az = rng.uniform(0.0, 2.0 * np.pi, size=n_az)
    e, a = np.meshgrid(el, az, indexing="ij")
    dirs = np.stack([np.cos(e) * np.cos(a), np.cos(e) * np.sin(a), np.sin(e)], -1).reshape(-1, 3)
    pose = pose_matrix([0.0, 0.0, 1.5])
    pts, lab = _scan(sc, pose, dirs, 100.0, range_sigma, rng)
    lab = _label_noise(rng, lab, label_noise, sc.num_classes)
    return dict(points=pts, labels=lab, pose=pose, num_classes=sc.num_classes)


# --------------------------------------------------------------------------
# workload 1: LiDAR street sequence
# --------------------------------------------------------------------------

STREET_PARAMS = dict(res=0.1, length_scale=0.3, sigma0=0.1, alpha0=0.001, free_step=0.3,
                     num_classes=19, min_range=0.0, max_range=50.0)

# primitive type -> class id (19 occupied classes)
STREET_CLASSES = dict(road=1, parking=2, sidewalk=3, terrain=4, facade=5, fence=6, canopy=7, trunk=8,
                      pole=9, sign=10, car=11, truck=12, cycle=13, moto=14, van=15, person=16,
                      rider=17, ground_patch=18, low_wall=19)


def street_scene(seed=1, length=250.0, x_start=-70.0):
    """Straight street along +x: road, parking strips, sidewalks, facades at |y| ~ 8-12 m
    with seeded setbacks and gaps, poles with signs, trees, bushes, parked and moving
    vehicles, pedestrians, fences, low walls and ground patches."""
    rng = np.random.default_rng(seed)
    C = STREET_CLASSES
    sc = Scene(num_classes=19)
    x_end = x_start + length
    sc.ground_rect = (x_start, x_end, -40.0, 40.0)
    sc.ground_bands = [(3.5, C["road"]), (5.0, C["parking"]), (8.0, C["sidewalk"]), (math.inf, C["terrain"])]
    for side in (-1.0, 1.0):
        # facades with setbacks and gaps; gaps get a fence or a low wall
        x = x_start
        while x < x_end:
            seg = rng.uniform(8.0, 30.0)
            y0 = 8.0 + rng.uniform(0.0, 4.0)
            h = rng.uniform(5.0, 20.0)
            lo = [x, y0 if side > 0 else -y0 - 10.0, 0.0]
            hi = [min(x + seg, x_end), y0 + 10.0 if side > 0 else -y0, h]
            sc.add_box(lo, hi, C["facade"])
            x += seg
            gap = rng.uniform(0.0, 6.0)
            if gap > 1.0:
                yy = 8.2 + rng.uniform(0.0, 1.0)
                if rng.random() < 0.5:
                    lo = [x, yy if side > 0 else -yy - 0.1, 0.0]
                    hi = [x + gap, yy + 0.1 if side > 0 else -yy, rng.uniform(1.0, 2.0)]
                    sc.add_box(lo, hi, C["fence"])
                else:
                    lo = [x, yy if side > 0 else -yy - 0.4, 0.0]
                    hi = [x + gap, yy + 0.4 if side > 0 else -yy, rng.uniform(0.4, 1.0)]
                    sc.add_box(lo, hi, C["low_wall"])
            x += gap
        # poles, some carrying a sign plate
        x = x_start + rng.uniform(0.0, 10.0)
        while x < x_end:
            y = side * rng.uniform(7.0, 7.8)
            h = rng.uniform(4.0, 8.0)
            sc.add_cyl(x, y, rng.uniform(0.08, 0.15), 0.0, h, C["pole"])
            if rng.random() < 0.4:
                sc.add_box([x - 0.04, y - 0.4, h - 1.0], [x + 0.04, y + 0.4, h - 0.2], C["sign"])
            x += rng.uniform(10.0, 20.0)
        # trees on the sidewalk edge
        x = x_start + rng.uniform(0.0, 8.0)
        while x < x_end:
            y = side * rng.uniform(6.0, 7.0)
            th = rng.uniform(2.0, 3.0)
            sc.add_cyl(x, y, rng.uniform(0.15, 0.3), 0.0, th, C["trunk"])
            rr = rng.uniform(1.2, 2.5)
            sc.add_ell([x, y, th + rr * 0.8], [rr, rr, rr * 0.8], C["canopy"])
            x += rng.uniform(8.0, 18.0)
        # bushes and ground patches on the terrain beyond the facades line
        for _ in range(int(length / 12)):
            x = rng.uniform(x_start, x_end)
            y = side * rng.uniform(12.5, 25.0)
            r = rng.uniform(0.5, 1.5, size=3)
            sc.add_ell([x, y, r[2] * 0.6], r, C["canopy"])
        for _ in range(int(length / 20)):
            x = rng.uniform(x_start, x_end)
            y = side * rng.uniform(5.2, 7.8)
            w = rng.uniform(0.5, 2.0, size=2)
            sc.add_box([x, y - w[1] / 2, 0.0], [x + w[0], y + w[1] / 2, 0.05], C["ground_patch"])
        # parked vehicles on the parking strip
        x = x_start + rng.uniform(0.0, 5.0)
        while x < x_end:
            kind = rng.random()
            if kind < 0.7:
                ln, wd, ht, cls = rng.uniform(3.8, 4.8), rng.uniform(1.6, 1.9), rng.uniform(1.3, 1.6), C["car"]
            elif kind < 0.85:
                ln, wd, ht, cls = rng.uniform(6.0, 9.0), rng.uniform(2.2, 2.5), rng.uniform(2.5, 3.5), C["truck"]
            else:
                ln, wd, ht, cls = rng.uniform(4.5, 5.5), rng.uniform(1.8, 2.0), rng.uniform(1.8, 2.3), C["van"]
            yc = side * (3.6 + wd / 2 + rng.uniform(0.0, 0.3))
            sc.add_box([x, yc - wd / 2, 0.15], [x + ln, yc + wd / 2, ht], cls)
            x += ln + rng.uniform(0.5, 8.0)
        # two-wheelers and people on the sidewalk
        for _ in range(int(length / 15)):
            x = rng.uniform(x_start, x_end)
            y = side * rng.uniform(5.2, 6.0)
            kind = rng.random()
            if kind < 0.35:
                sc.add_box([x, y - 0.3, 0.0], [x + 1.7, y + 0.3, 1.1], C["cycle"] if rng.random() < 0.5 else C["moto"])
            elif kind < 0.85:
                sc.add_cyl(x, y, 0.25, 0.0, rng.uniform(1.5, 1.9), C["person"])
            else:
                sc.add_box([x, y - 0.3, 0.0], [x + 1.7, y + 0.3, 1.0], C["cycle"])
                sc.add_cyl(x + 0.85, y, 0.25, 1.0, 1.8, C["rider"])
    # occasional moving vehicle in the opposite lane (never in the sensor lane y < 0)
    x = x_start + rng.uniform(0.0, 30.0)
    while x < x_end:
        sc.add_box([x, 0.8, 0.15], [x + 4.5, 2.6, 1.5], C["car"])
        x += rng.uniform(25.0, 60.0)
    return sc


def street_sequence(n_scans=100, seed=1, n_beams=64, n_az=2048, range_sigma=0.03, label_noise=0.10,
                    first=0, scene=None):
    """LiDAR-shaped scans along the street: poses 1 m apart along x at y = -1.75,
    sensor height 1.73 m, yaw ~ N(0, 1 deg); beams evenly over +2 to -24.8 degrees.

    Yields dicts (points [n,3] float32 sensor frame, labels [n] int32 in 1..19 with label
    noise, clean_labels [n] the same points' labels before the noise, pose 4x4).
    Scan i depends only on (seed, i), so any sub-range can be generated alone."""
    sc = street_scene(seed) if scene is None else scene
    dirs = lidar_dirs(n_beams, n_az, 2.0, -24.8)
    for i in range(first, first + n_scans):
        rng = np.random.default_rng([seed, 7919, i])
        yaw = math.radians(rng.normal(0.0, 1.0))
        pose = pose_matrix([float(i), -1.75, 1.73], yaw=yaw)
        pts, clean = _scan(sc, pose, dirs, STREET_PARAMS["max_range"], range_sigma, rng)
        lab = _label_noise(rng, clean, label_noise, sc.num_classes)
        yield dict(points=pts, labels=lab, clean_labels=clean, pose=pose, num_classes=sc.num_classes)


# --------------------------------------------------------------------------
# workload 2: depth-camera (stereo-shaped) sequence in a furnished room
# --------------------------------------------------------------------------

ROOM_PARAMS = dict(res=0.05, length_scale=0.15, sigma0=0.1, alpha0=0.001, free_step=0.15,
                   num_classes=11, min_range=0.3, max_range=8.0)
ROOM_SIZE = (10.0, 8.0, 3.0)


def room_scene(seed=2):
    """10 x 8 x 3 m room: floor 1, ceiling 2, walls 3/4, tables 5, cabinets 6, chairs 7,
    sofas 8, small objects 9, lamps 10 (cylinders), plants 11 (ellipsoids)."""
    rng = np.random.default_rng(seed)
    X, Y, Z = ROOM_SIZE
    sc = Scene(num_classes=11)
    sc.ground_rect = (-X / 2, X / 2, -Y / 2, Y / 2)
    sc.ground_bands = [(math.inf, 1)]
    th = 0.2
    sc.add_box([-X / 2, -Y / 2, Z], [X / 2, Y / 2, Z + th], 2)
    sc.add_box([-X / 2 - th, -Y / 2, 0], [-X / 2, Y / 2, Z], 3)
    sc.add_box([X / 2, -Y / 2, 0], [X / 2 + th, Y / 2, Z], 3)
    sc.add_box([-X / 2, -Y / 2 - th, 0], [X / 2, -Y / 2, Z], 4)
    sc.add_box([-X / 2, Y / 2, 0], [X / 2, Y / 2 + th, Z], 4)
    for _ in range(6):  # cabinets against the walls
        w, d, h = rng.uniform(0.6, 1.5), rng.uniform(0.4, 0.6), rng.uniform(1.2, 2.2)
        if rng.random() < 0.5:
            x = rng.uniform(-X / 2 + w, X / 2 - w)
            y = Y / 2 - d if rng.random() < 0.5 else -Y / 2
            sc.add_box([x, y, 0], [x + w, y + d, h], 6)
        else:
            y = rng.uniform(-Y / 2 + w, Y / 2 - w)
            x = X / 2 - d if rng.random() < 0.5 else -X / 2
            sc.add_box([x, y, 0], [x + d, y + w, h], 6)
    for _ in range(5):  # tables with objects, chairs
        cx, cy = rng.uniform(-X / 2 + 1.5, X / 2 - 1.5), rng.uniform(-Y / 2 + 1.5, Y / 2 - 1.5)
        w, d = rng.uniform(0.8, 1.6), rng.uniform(0.6, 1.0)
        sc.add_box([cx - w / 2, cy - d / 2, 0.7], [cx + w / 2, cy + d / 2, 0.75], 5)
        for sx in (-1, 1):
            for sy in (-1, 1):
                sc.add_box([cx + sx * (w / 2 - 0.05) - 0.03, cy + sy * (d / 2 - 0.05) - 0.03, 0.0],
                           [cx + sx * (w / 2 - 0.05) + 0.03, cy + sy * (d / 2 - 0.05) + 0.03, 0.7], 5)
        for _ in range(rng.integers(1, 4)):
            ox, oy = cx + rng.uniform(-w / 3, w / 3), cy + rng.uniform(-d / 3, d / 3)
            s = rng.uniform(0.08, 0.25, size=3)
            sc.add_box([ox, oy, 0.75], [ox + s[0], oy + s[1], 0.75 + s[2]], 9)
        for sy in (-1, 1):
            ch = [cx - 0.22, cy + sy * (d / 2 + 0.35) - 0.22, 0.0]
            sc.add_box(ch, [ch[0] + 0.44, ch[1] + 0.44, 0.45], 7)
            sc.add_box([ch[0], ch[1] + (0.4 if sy > 0 else 0.0), 0.45], [ch[0] + 0.44, ch[1] + (0.44 if sy > 0 else 0.04), 0.95], 7)
    for _ in range(2):  # sofas
        cx, cy = rng.uniform(-X / 2 + 1.5, X / 2 - 1.5), rng.uniform(-Y / 2 + 1.5, Y / 2 - 1.5)
        sc.add_box([cx - 1.0, cy - 0.45, 0.0], [cx + 1.0, cy + 0.45, 0.45], 8)
        sc.add_box([cx - 1.0, cy + 0.3, 0.45], [cx + 1.0, cy + 0.45, 0.9], 8)
    for _ in range(4):  # floor lamps
        sc.add_cyl(rng.uniform(-X / 2 + 0.5, X / 2 - 0.5), rng.uniform(-Y / 2 + 0.5, Y / 2 - 0.5),
                   rng.uniform(0.02, 0.05), 0.0, rng.uniform(1.4, 1.8), 10)
    for _ in range(4):  # plants
        r = rng.uniform(0.2, 0.5, size=3)
        sc.add_ell([rng.uniform(-X / 2 + 0.6, X / 2 - 0.6), rng.uniform(-Y / 2 + 0.6, Y / 2 - 0.6), r[2] + 0.1], r, 11)
    return sc


def _camera_rays(w=640, h=480, fx=525.0, fy=525.0, cx=319.5, cy=239.5):
    u, v = np.meshgrid(np.arange(w, dtype=float), np.arange(h, dtype=float))
    x = (u - cx) / fx
    y = (v - cy) / fy
    return np.stack([x, y, np.ones_like(x)], -1).reshape(-1, 3)  # z = 1 (depth scale)


def _boundary_pixels(lab_img, valid, radius=2):
    """Flat indices of valid pixels within `radius` px of a different label."""
    h, w = lab_img.shape
    b = np.zeros_like(valid)
    for dy in range(-radius, radius + 1):
        for dx in range(-radius, radius + 1):
            if dx == 0 and dy == 0:
                continue
            sh = np.full_like(lab_img, -1)
            ys = slice(max(dy, 0), h + min(dy, 0))
            yd = slice(max(-dy, 0), h + min(-dy, 0))
            xs = slice(max(dx, 0), w + min(dx, 0))
            xd = slice(max(-dx, 0), w + min(-dx, 0))
            sh[yd, xd] = lab_img[ys, xs]
            b |= (sh != lab_img) & (sh >= 0)
    return np.nonzero((b & valid).reshape(-1))[0]


def room_sequence(n_frames=200, seed=2, label_noise=0.15, first=0, scene=None, width=640, height=480):
    """Depth frames from a camera on a smooth seeded random walk (0.05 m/frame,
    <= 2 deg/frame) inside the room; depth noise sigma = 0.0025 d^2; 15 % label
    noise placed on pixels within 2 px of a label boundary (remainder uniform).

    Yields dicts (points [n,3] float32 camera frame x right / y down / z forward,
    labels, pose 4x4 world_from_camera).  The walk is replayed from frame 0, so
    frame i is identical whatever `first` is."""
    sc = room_scene(seed) if scene is None else scene
    rays = _camera_rays(width, height)
    rng_walk = np.random.default_rng([seed, 31337])
    X, Y, _ = ROOM_SIZE
    pos = np.array([0.0, 0.0, 1.5])
    yaw, pitch = 0.0, math.radians(-10.0)
    vel = np.array([1.0, 0.0, 0.0])
    pmin, pmax = ROOM_PARAMS["min_range"], ROOM_PARAMS["max_range"]
    for i in range(first + n_frames):
        if i > 0:
            vel = vel + rng_walk.normal(0.0, 0.3, size=3) * np.array([1, 1, 0.2])
            to_c = -pos[:2] / np.array([X / 2 - 1.0, Y / 2 - 1.0])
            vel[:2] += 0.5 * to_c * (np.abs(to_c) > 0.6)
            vel[2] += 0.5 * (1.5 - pos[2])
            vel /= max(np.linalg.norm(vel), 1e-9)
            step = pos + 0.05 * vel
            if sc.contains(step, margin=0.35):
                vel = -vel
                step = pos + 0.05 * vel
            if not sc.contains(step, margin=0.35):
                pos = step
            yaw += math.radians(float(np.clip(rng_walk.normal(0.0, 1.0), -2.0, 2.0)))
            pitch = float(np.clip(pitch + math.radians(float(np.clip(rng_walk.normal(0.0, 0.5), -1.0, 1.0))),
                                  math.radians(-30), math.radians(10)))
        if i < first:
            continue
        pose = pose_matrix(pos, yaw=yaw, pitch=-pitch, base=_CAM_TO_FLU)
        rng = np.random.default_rng([seed, 104729, i])
        r = pose[:3, :3]
        dn = rays / np.linalg.norm(rays, axis=1, keepdims=True)
        t, cls = raycast(sc, pos, dn @ r.T, pmax * 2.0)
        depth = t * dn[:, 2]  # z component in the camera frame
        valid = np.isfinite(depth) & (depth >= pmin) & (depth <= pmax)
        lab_img = np.where(valid, cls, -1).reshape(height, width)
        cand = _boundary_pixels(lab_img, valid.reshape(height, width))
        z = depth + rng.normal(0.0, 1.0, size=len(depth)) * 0.0025 * depth * depth
        idx = np.nonzero(valid)[0]
        pts = (rays[idx] * z[idx, None]).astype(np.float32)
        lab = cls[idx].astype(np.int32)
        pos_in_valid = np.full(len(depth), -1)
        pos_in_valid[idx] = np.arange(len(idx))
        lab = _label_noise(rng, lab, label_noise, sc.num_classes, candidates=pos_in_valid[cand])
        yield dict(points=pts, labels=lab, pose=pose, num_classes=sc.num_classes)


# --------------------------------------------------------------------------
# workload 3: differentiable fit on the small region
# --------------------------------------------------------------------------

DIFF_PARAMS = dict(res=0.1, length_scale=0.3, sigma0=1.0, alpha0=0.001, free_step=0.3,
                   num_classes=10, min_range=0.0, max_range=50.0)


def small_region_lidar_sequence(n_scans=20, seed=3, holdout=0.2, n_beams=64, n_az=2048):
    """The small-region scene scanned by a 64-beam LiDAR from poses at
    x in {-4.75, -4.25, ..., 4.75}, z = 1.5, yaw jitter 1 degree.  20 % of each
    scan's hits are withheld (seeded) and returned separately."""
    sc = small_region_scene(0)
    dirs = lidar_dirs(n_beams, n_az, 2.0, -24.8)
    xs = -4.75 + 0.5 * np.arange(20)
    for i in range(n_scans):
        rng = np.random.default_rng([seed, 4099, i])
        pose = pose_matrix([float(xs[i % 20]), 0.0, 1.5], yaw=math.radians(rng.normal(0.0, 1.0)))
        pts, lab = _scan(sc, pose, dirs, DIFF_PARAMS["max_range"], 0.02, rng)
        lab = _label_noise(rng, lab, 0.05, sc.num_classes)
        hold = rng.random(len(pts)) < holdout
        yield dict(points=pts[~hold], labels=lab[~hold], held_points=pts[hold], held_labels=lab[hold],
                   pose=pose, num_classes=sc.num_classes)


# --------------------------------------------------------------------------
# workload 4: independent maps, one scan each, log-uniform sizes
# --------------------------------------------------------------------------

BATCH_PARAMS = dict(res=0.1, length_scale=0.3, sigma0=0.1, alpha0=0.001, free_step=0.3,
                    min_range=0.0, max_range=50.0)


def batch_scans(n_maps=32, seed=4, n_min=5000, n_max=250000):
    """One scan per independent map; N log-uniform in [n_min, n_max]; each scan is
    LiDAR-shaped (street scene, first pose, 128 x 4096 rays subsampled to N) or
    depth-shaped (room scene, first frame, pixels subsampled to N) by a seeded coin."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_maps)).astype(np.int64)
    kinds = rng.random(n_maps) < 0.5
    street = street_scene(1)
    lid_pose = pose_matrix([0.0, -1.75, 1.73])
    dirs = lidar_dirs(128, 4096, 2.0, -24.8)
    lid_pts, lid_lab = _scan(street, lid_pose, dirs, 50.0, 0.03, np.random.default_rng([seed, 1]))
    lid_lab = _label_noise(np.random.default_rng([seed, 2]), lid_lab, 0.10, 19)
    room = next(room_sequence(1, seed=2))
    out = []
    for m in range(n_maps):
        r = np.random.default_rng([seed, 3, m])
        if kinds[m]:
            n = min(int(sizes[m]), len(lid_pts))
            idx = np.sort(r.choice(len(lid_pts), size=n, replace=False))
            out.append(dict(points=lid_pts[idx], labels=lid_lab[idx], pose=lid_pose, num_classes=19, kind="lidar"))
        else:
            n = min(int(sizes[m]), len(room["points"]))
            idx = np.sort(r.choice(len(room["points"]), size=n, replace=False))
            out.append(dict(points=room["points"][idx], labels=room["labels"][idx], pose=room["pose"],
                            num_classes=11, kind="depth"))
    return out


# --------------------------------------------------------------------------
# tiny hand-built inputs for unit tests
# --------------------------------------------------------------------------


def random_cloud(n, seed, extent=1.0, num_classes=3, center=(0.0, 0.0, 0.0)):
    """n uniformly random points (float32) with labels in 1..num_classes."""
    rng = np.random.default_rng(seed)
    pts = (rng.uniform(-extent, extent, size=(n, 3)) + np.asarray(center)).astype(np.float32)
    lab = rng.integers(1, num_classes + 1, size=n).astype(np.int32)
    return pts, lab
