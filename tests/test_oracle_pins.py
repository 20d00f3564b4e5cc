"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own arithmetic: closed-form
values of the sparse kernel (Eq. kernel), exact quadratures, brute-force
all-pairs sums (Eq. alpha_kernel) written with numpy, Dirichlet moments from
scipy (Eq. mode, Eq. variance), the binary counting/BKI special case
(Sec. III), counts fixed by construction for the counting model (Eq. alpha),
and finite differences of the oracle's own forward for its
analytic gradient.  None of them needs a GPU.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize, stats

from synth import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- kernel (Eq. kernel)

def test_kernel_closed_form_values(orc):
    # f(0) = 1 (k = sigma0 at d = 0), f(1/2) = 1/6, f(r >= 1) = 0
    assert orc.kernel_f(0.0) == pytest.approx(1.0, abs=1e-15)
    assert orc.kernel_f(0.5) == pytest.approx(1.0 / 6.0, abs=1e-15)
    for r in (1.0, 1.0 + 1e-12, 1.5, 10.0):
        assert orc.kernel_f(r) == 0.0
    # FP64 cancellation near r = 1 leaves at most a few 1e-16 below zero
    assert orc.kernel_f(1.0 - 1e-9) >= -1e-15


def test_kernel_zero_slope_and_fifth_order_contact(orc):
    h = 1e-6
    assert (orc.kernel_f(h) - orc.kernel_f(0.0)) / h == pytest.approx(0.0, abs=1e-5)
    # near r = 1 the kernel touches zero to fifth order: f ~ (4 pi^4 / 45) (1 - r)^5
    for eps in (1e-2, 3e-3):
        assert orc.kernel_f(1.0 - eps) / eps ** 5 == pytest.approx(4 * math.pi ** 4 / 45, rel=2e-2)
    assert orc.kernel_df(0.0) == pytest.approx(0.0, abs=1e-14)
    assert orc.kernel_df(1.0 - 1e-9) == pytest.approx(0.0, abs=1e-12)


def test_kernel_monotone_nonnegative_and_derivative(orc):
    r = np.linspace(0.0, 1.0, 2001)
    f = np.array([orc.kernel_f(x) for x in r])
    assert np.all(f >= -1e-15)
    assert np.all(np.diff(f) <= 1e-15)
    # derivative agrees with a central difference of f
    rng = np.random.default_rng(0)
    for x in rng.uniform(0.01, 0.99, size=50):
        h = 1e-6
        fd = (orc.kernel_f(x + h) - orc.kernel_f(x - h)) / (2 * h)
        assert orc.kernel_df(x) == pytest.approx(fd, abs=1e-8)


def test_kernel_integrals(orc):
    # exact: int_0^1 f dr = 1/3 ; ball integral int_{|u|<1} f(|u|) du = 2 (pi^2 - 6) / (9 pi)
    i1, _ = integrate.quad(orc.kernel_f, 0.0, 1.0, epsabs=1e-13)
    assert i1 == pytest.approx(1.0 / 3.0, abs=1e-12)
    i3, _ = integrate.quad(lambda r: 4 * math.pi * r * r * orc.kernel_f(r), 0.0, 1.0, epsabs=1e-13)
    assert i3 == pytest.approx(2 * (math.pi ** 2 - 6) / (9 * math.pi), abs=1e-12)
    i2, _ = integrate.quad(lambda r: 2 * math.pi * r * orc.kernel_f(r), 0.0, 1.0, epsabs=1e-13)
    assert i2 == pytest.approx((4 * math.pi ** 2 - 15) / (18 * math.pi), abs=1e-12)


def test_paper_parameter_defaults(orc):
    gold = json.load(open(os.path.join(GOLD, "paper_parameters.json")))
    p = orc.params()
    for k in ("length_scale", "sigma0", "alpha0", "res", "free_thresh", "occ_thresh"):
        assert getattr(p, k) == pytest.approx(gold[k])


# ---------------------------------------------------------------- a1: transform and validate

def test_transform_exact_yaw90_and_drops(orc):
    p = orc.params(min_range=0.5, max_range=10.0)
    T = np.eye(4)
    T[:3, :3] = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]
    T[:3, 3] = [1.0, 2.0, 3.0]
    pts = np.array([[1, 0, 0], [0, 2, 0], [np.nan, 0, 1], [0.1, 0, 0], [20, 0, 0], [0, 0, np.inf], [0, 0, -4]],
                   np.float32)
    w, idx = orc.transform(p, pts, T)
    assert idx.tolist() == [0, 1, 6]
    np.testing.assert_array_equal(w, np.array([[1, 3, 3], [-1, 2, 3], [1, 2, -1]], np.float32))


# ---------------------------------------------------------------- a2: free samples (Sec. III)

def test_free_samples_exact_binary_step(orc):
    p = orc.params(free_step=0.25, num_classes=3)
    T = np.eye(4)
    xyz, lab = orc.samples(p, np.array([[1.0, 0, 0], [0, 0, 0.5]], np.float32), np.array([2, 3]), T)
    # hits first (input order), then samples of ray 0 (j = 1, 2, 3) and ray 1 (j = 1)
    np.testing.assert_array_equal(lab, [2, 3, 0, 0, 0, 0])
    np.testing.assert_array_equal(xyz, np.array([[1, 0, 0], [0, 0, 0.5], [0.75, 0, 0], [0.5, 0, 0], [0.25, 0, 0],
                                                 [0, 0, 0.25]], np.float32))


def test_free_samples_geometry(orc):
    """Samples lie on the segment from the origin to the hit, spaced by s,
    the last within (0, s] of the sensor; count = ceil(r/s) - 1 away from ties."""
    rng = np.random.default_rng(1)
    s = 0.3
    p = orc.params(free_step=s, num_classes=2)
    T = np.eye(4)
    T[:3, 3] = [0.5, -0.25, 1.5]
    d = rng.normal(size=(40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rr = rng.uniform(0.05, 12.0, size=40)
    pts = (d * rr[:, None]).astype(np.float32)
    xyz, lab = orc.samples(p, pts, np.ones(40, np.int32), T)
    free = xyz[40:].astype(np.float64)
    o = T[:3, 3]
    pos = 0
    for i in range(40):
        n = int(math.ceil(rr[i] / s)) - 1
        seg = free[pos:pos + n]
        pos += n
        t = np.linalg.norm(seg - o, axis=1)
        np.testing.assert_allclose(t, rr[i] - s * np.arange(1, n + 1), atol=2e-5)
        cr = np.cross(seg - o, np.tile(d[i], (n, 1)))
        assert np.abs(cr).max(initial=0.0) < 2e-5
        if n:
            assert 0.0 < t[-1] <= s + 2e-5
    assert pos == len(free)
    assert np.all(lab[40:] == 0)


# ---------------------------------------------------------------- a3: downsampling

def test_downsample_centroids_by_cell_and_label(orc):
    p = orc.params(res=1.0, free_step=100.0, num_classes=3)  # no free samples: every r < s
    T = np.eye(4)
    pts = np.array([[0.25, 0.25, 0.25], [0.75, 0.25, 0.25], [0.5, 0.75, 0.75],  # cell (0,0,0) label 1
                    [0.5, 0.5, 0.5],                                         # cell (0,0,0) label 2
                    [1.5, 0.5, 0.5], [-0.5, 0.5, 0.5]], np.float32)          # cells (1,0,0), (-1,0,0)
    lab = np.array([1, 1, 1, 2, 1, 1], np.int32)
    xyz, ol, st = orc.training_set(p, pts, lab, T)
    got = {(tuple(np.floor(x).astype(int)), int(l)): tuple(x) for x, l in zip(xyz, ol)}
    assert st == dict(hits=6, free=0, train=4)
    assert got[((0, 0, 0), 1)] == (0.5, np.float32(1.25 / 3), np.float32(1.25 / 3))
    assert got[((0, 0, 0), 2)] == (0.5, 0.5, 0.5)
    assert got[((1, 0, 0), 1)] == (1.5, 0.5, 0.5)
    assert got[((-1, 0, 0), 1)] == (-0.5, 0.5, 0.5)


def test_voxel_index_floor_boundaries(orc):
    # floorf(x * fp32(1/res)): negative side floors down; 0.1f * 10f rounds to 1
    p = orc.params(res=0.1, length_scale=0.05, sigma0=1.0, num_classes=1)
    m = orc.OracleMap(p)
    m.insert_training(np.array([[-0.05, 0.05, 0.05], [0.1, 0.05, 0.05]], np.float32), np.array([1, 1]))
    keys, alpha, pairs = m.export()
    touched = keys[pairs > 0]
    assert sorted(map(tuple, touched)) == [(-1, 0, 0), (1, 0, 0)]


# ---------------------------------------------------------------- a5: accumulation (Eq. alpha_kernel)

def _bruteforce(orc, p, xyz, lab):
    """numpy all-pairs: every voxel centre in the padded bounding box x every point."""
    res, l = p.res, p.length_scale
    lo = np.floor(xyz.min(0) / res).astype(int) - int(math.ceil(l / res)) - 2
    hi = np.floor(xyz.max(0) / res).astype(int) + int(math.ceil(l / res)) + 2
    g = np.stack(np.meshgrid(*[np.arange(a, b + 1) for a, b in zip(lo, hi)], indexing="ij"), -1).reshape(-1, 3)
    c = (g + 0.5) * res
    K1 = p.num_classes + 1
    acc = {}
    x64 = xyz.astype(np.float64)
    for i in range(len(x64)):
        e = c - x64[i]
        d2 = (e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1]) + e[:, 2] * e[:, 2]
        for j in np.nonzero(d2 < l * l)[0]:
            key = tuple(g[j])
            if key not in acc:
                acc[key] = [np.zeros(K1), 0]
            acc[key][0][lab[i]] += p.sigma0 * orc.kernel_f(math.sqrt(d2[j]) / l)
            acc[key][1] += 1
    return acc


@pytest.mark.parametrize("seed,res,l", [(0, 0.1, 0.3), (1, 0.1, 0.25), (2, 0.05, 0.15), (3, 0.2, 0.3)])
def test_stencil_equals_bruteforce(orc, seed, res, l):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-0.6, 0.6, size=(150, 3)).astype(np.float32)
    xyz[:5] = np.round(xyz[:5] / res) * res  # points on voxel faces
    lab = rng.integers(0, 4, size=150).astype(np.int32)
    p = orc.params(res=res, length_scale=l, sigma0=0.7, num_classes=3, block_edge=4)
    m = orc.OracleMap(p)
    m.insert_training(xyz, lab)
    keys, alpha, pairs = m.export()
    ref = _bruteforce(orc, p, xyz, lab)
    touched = {tuple(k): i for i, k in enumerate(keys) if pairs[i] > 0}
    assert set(touched) == set(ref)
    for k, i in touched.items():
        assert pairs[i] == ref[k][1]
        np.testing.assert_allclose(alpha[i] - p.alpha0, ref[k][0], rtol=1e-12, atol=1e-15)
    # voxels of allocated blocks that no point reached hold exactly the prior
    assert np.all(alpha[pairs == 0] == p.alpha0)
    # blocks: exactly those holding a touched voxel (block edge 4)
    bk = {tuple(np.floor_divide(np.array(k), 4)) for k in ref}
    assert set(map(tuple, m.block_keys())) == bk


def test_alpha_bruteforce_entry_matches_numpy(orc):
    rng = np.random.default_rng(5)
    xyz = rng.uniform(-0.5, 0.5, size=(80, 3)).astype(np.float32)
    lab = rng.integers(0, 3, size=80).astype(np.int32)
    p = orc.params(res=0.1, length_scale=0.3, sigma0=0.5, num_classes=2)
    ref = _bruteforce(orc, p, xyz, lab)
    keys = np.array(list(ref.keys()))
    a, pc = orc.alpha_bruteforce(p, xyz, lab, keys)
    for i, k in enumerate(ref):
        assert pc[i] == ref[k][1]
        np.testing.assert_allclose(a[i] - p.alpha0, ref[k][0], rtol=1e-12, atol=1e-15)


def test_lattice_mass_matches_ball_integral(orc):
    """Sum over voxel centres of k(c_v, x), averaged over uniform offsets of x,
    equals sigma0 (l/res)^3 * 2(pi^2-6)/(9 pi) (the lattice sum of a smooth
    compactly supported function equals its integral up to a tiny aliasing term)."""
    rng = np.random.default_rng(7)
    res, l, s0 = 0.1, 0.3, 1.0
    n = 3000
    grid = np.stack(np.meshgrid(np.arange(15), np.arange(15), np.arange(14), indexing="ij"), -1).reshape(-1, 3)[:n]
    xyz = (grid * 1.0 + rng.uniform(0.0, res, size=(n, 3))).astype(np.float32)  # 1 m apart: no overlap
    p = orc.params(res=res, length_scale=l, sigma0=s0, num_classes=1)
    m = orc.OracleMap(p)
    m.insert_training(xyz, np.ones(n, np.int32))
    keys, alpha, pairs = m.export()
    per_point = (alpha[:, 1] - p.alpha0).sum() / n
    expect = s0 * (l / res) ** 3 * 2 * (math.pi ** 2 - 6) / (9 * math.pi)
    assert per_point == pytest.approx(expect, rel=2e-3)
    # in-support pairs per point ~ ball volume in voxels = 4/3 pi 3^3
    assert pairs.sum() / n == pytest.approx(4 / 3 * math.pi * 27, rel=2e-2)


def test_binary_reversion_to_bki_occupancy(orc):
    """With one occupied class (K = 1), alpha^0 and alpha^1 are the two counts of
    binary BKI occupancy (Sec. III reverts to the counting sensor model); with
    K > 1 and only class c observed, alpha^c equals the occupied count and every
    other occupied class keeps the prior."""
    rng = np.random.default_rng(11)
    xyz = rng.uniform(-0.5, 0.5, size=(120, 3)).astype(np.float32)
    occ = rng.random(120) < 0.4
    p1 = orc.params(res=0.1, length_scale=0.3, sigma0=1.0, num_classes=1)
    m1 = orc.OracleMap(p1)
    m1.insert_training(xyz, occ.astype(np.int32))
    keys, a1, pairs = m1.export()
    # binary BKI: beta = sum_free k, alpha = sum_occ k  (numpy brute force)
    c = (keys + 0.5) * 0.1
    d = np.linalg.norm(c[:, None, :] - xyz[None].astype(np.float64), axis=2)
    kf = np.vectorize(orc.kernel_f)(np.minimum(d / 0.3, 1.0))
    np.testing.assert_allclose(a1[:, 1] - 0.001, kf[:, occ].sum(1), rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(a1[:, 0] - 0.001, kf[:, ~occ].sum(1), rtol=1e-10, atol=1e-13)
    p5 = orc.params(res=0.1, length_scale=0.3, sigma0=1.0, num_classes=5)
    m5 = orc.OracleMap(p5)
    m5.insert_training(xyz, np.where(occ, 4, 0).astype(np.int32))
    k5, a5, _ = m5.export()
    np.testing.assert_array_equal(k5, keys)
    np.testing.assert_allclose(a5[:, [0, 4]], a1, rtol=1e-12)
    assert np.all(a5[:, [1, 2, 3, 5]] == 0.001)


def test_scan_additivity_and_sigma0_linearity(orc):
    sc = scenes.small_region_scan(0, n_az=30, n_el=20)
    pts, lab, T = sc["points"], sc["labels"], sc["pose"]
    half = len(pts) // 2
    p = orc.params(**{**scenes.SMALL_SCENE_PARAMS, "sigma0": 1.0})
    both = orc.OracleMap(p)
    both.insert_scan(pts[:half], lab[:half], T)
    both.insert_scan(pts[half:], lab[half:], T)
    kb, ab, pb = both.export()
    A = orc.OracleMap(p)
    A.insert_scan(pts[:half], lab[:half], T)
    B = orc.OracleMap(p)
    B.insert_scan(pts[half:], lab[half:], T)
    aa, pa = A.alpha_at(kb)
    bb, pbb = B.alpha_at(kb)
    np.testing.assert_allclose(ab, aa + bb - p.alpha0, rtol=1e-12)
    np.testing.assert_array_equal(pb, pa + pbb)
    p2 = orc.params(**{**scenes.SMALL_SCENE_PARAMS, "sigma0": 0.25})
    C = orc.OracleMap(p2)
    C.insert_scan(pts[:half], lab[:half], T)
    C.insert_scan(pts[half:], lab[half:], T)
    kc, ac, _ = C.export()
    np.testing.assert_array_equal(kc, kb)
    np.testing.assert_allclose(ac - p.alpha0, 0.25 * (ab - p.alpha0), rtol=1e-12, atol=1e-16)


def test_conservation_per_voxel(orc):
    """sum_k (alpha_v^k - alpha0) = sum_i k(c_v, x_i) over all labels."""
    rng = np.random.default_rng(13)
    xyz = rng.uniform(-0.4, 0.4, size=(60, 3)).astype(np.float32)
    lab = rng.integers(0, 6, size=60).astype(np.int32)
    p = orc.params(res=0.1, length_scale=0.3, sigma0=0.3, num_classes=5)
    m = orc.OracleMap(p)
    m.insert_training(xyz, lab)
    keys, alpha, _ = m.export()
    a_one, _ = orc.alpha_bruteforce(orc.params(res=0.1, length_scale=0.3, sigma0=0.3, num_classes=1), xyz,
                                    np.zeros(60, np.int32), keys)
    np.testing.assert_allclose((alpha - p.alpha0).sum(1), a_one[:, 0] - p.alpha0, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- a5 of the counting model (Eq. alpha)

def test_counting_model_counts_by_construction(orc):
    """Eq. (alpha): alpha_j^k = alpha0 + the number of training points of class k
    inside cell j.  Points are placed well inside chosen voxels (the voxel is
    known by construction, not computed), so every count is fixed in advance."""
    rng = np.random.default_rng(23)
    res = 0.1
    cells = rng.integers(-12, 12, size=(25, 3))
    cells[1] = cells[0]                                 # one voxel holds two groups
    cells[2] = cells[0] + np.array([0, 0, 1])
    which = rng.integers(0, len(cells), size=300)
    u = rng.uniform(0.2, 0.8, size=(300, 3))
    xyz = ((cells[which] + u) * res).astype(np.float32)
    lab = rng.integers(0, 4, size=300).astype(np.int32)
    expect = {}
    for c, l in zip(map(tuple, cells[which]), lab):
        expect.setdefault(c, np.zeros(4))[l] += 1.0
    p = orc.params(res=res, length_scale=0.3, sigma0=0.1, num_classes=3, sensor_model=1)
    m = orc.OracleMap(p)
    m.insert_training(xyz, lab)
    keys, alpha, pairs = m.export()
    got = {tuple(k): (a, n) for k, a, n in zip(keys, alpha, pairs)}
    for c, cnt in expect.items():
        np.testing.assert_array_equal(got[c][0], p.alpha0 + cnt)   # integer counts: exact in FP64
        assert got[c][1] == cnt.sum()
    rest = [k for k in got if k not in expect]
    assert all(np.all(got[k][0] == p.alpha0) and got[k][1] == 0 for k in rest)
    # allocated blocks: exactly the 8^3 blocks that hold a point (Python floor division)
    blocks = {tuple(np.asarray(c) // 8) for c in expect}
    assert set(map(tuple, m.block_keys())) == blocks
    # the kernel parameters do not enter the counting model
    m2 = orc.OracleMap(orc.params(res=res, length_scale=0.17, sigma0=5.0, num_classes=3, sensor_model=1))
    m2.insert_training(xyz, lab)
    np.testing.assert_array_equal(m2.export()[1], alpha)


def test_counting_model_reverts_to_binary_counting_sensor(orc):
    """With K = 1 the counting model is the binary counting sensor model (Sec. IV):
    along one beam every free sample adds a miss to its voxel and the hit adds a
    hit, so E[theta^occ] = (alpha0 + hits) / (2 alpha0 + hits + misses)."""
    a0 = 0.001
    p = orc.params(res=0.1, free_step=0.3, alpha0=a0, num_classes=1, sensor_model=1)
    T = np.eye(4)
    T[:3, 3] = [0.02, 0.05, 0.05]
    m = orc.OracleMap(p)
    st = m.insert_scan(np.array([[1.0, 0.0, 0.0]], np.float32), np.array([1], np.int32), T)
    assert st == dict(hits=1, free=3, train=4)          # samples at t = 0.7, 0.4, 0.1 (reading K3)
    q = np.array([[1.02, 0.05, 0.05], [0.72, 0.05, 0.05], [0.42, 0.05, 0.05], [0.12, 0.05, 0.05],
                  [0.55, 0.05, 0.05], [1.02, 0.15, 0.05]], np.float32)
    r = m.query(q)
    occ = (a0 + 1.0) / (2 * a0 + 1.0)
    free = a0 / (2 * a0 + 1.0)
    np.testing.assert_allclose(r["p_occ"], [occ, free, free, free, 0.5, 0.5], rtol=1e-14)
    np.testing.assert_array_equal(r["state"], [2, 0, 0, 0, 1, 1])
    # a second scan from the same pose doubles every count
    m.insert_scan(np.array([[1.0, 0.0, 0.0]], np.float32), np.array([1], np.int32), T)
    a, n = m.alpha_at(np.array([[10, 0, 0], [7, 0, 0]]))
    np.testing.assert_array_equal(a, a0 + np.array([[0.0, 2.0], [2.0, 0.0]]))
    np.testing.assert_array_equal(n, [2, 2])


def test_counting_model_mass_equals_training_points(orc):
    """Each training point is counted exactly once: the increments of a whole
    scan sum to the number of training points, per class and in total."""
    sc = scenes.small_region_scan(0, n_az=40, n_el=30)
    prm = dict(scenes.SMALL_SCENE_PARAMS, sensor_model=1)
    p = orc.params(**prm)
    xyz, lab, st = orc.training_set(p, sc["points"], sc["labels"], sc["pose"])
    m = orc.OracleMap(p)
    assert m.insert_scan(sc["points"], sc["labels"], sc["pose"]) == st
    keys, alpha, pairs = m.export()
    K1 = p.num_classes + 1
    counts = np.rint(alpha - p.alpha0)
    np.testing.assert_allclose(alpha - p.alpha0, counts, rtol=0, atol=1e-9)   # whole counts
    np.testing.assert_array_equal(counts.sum(0), np.bincount(lab, minlength=K1))
    assert pairs.sum() == len(xyz)
    np.testing.assert_array_equal(counts.sum(1), pairs)


# ---------------------------------------------------------------- read-off (Eq. mode, Eq. variance)

def test_readoff_matches_dirichlet_moments(orc):
    rng = np.random.default_rng(17)
    xyz = rng.uniform(-0.3, 0.3, size=(400, 3)).astype(np.float32)
    lab = rng.integers(0, 4, size=400).astype(np.int32)
    p = orc.params(res=0.1, length_scale=0.3, sigma0=2.0, num_classes=3)
    m = orc.OracleMap(p)
    m.insert_training(xyz, lab)
    keys, alpha, pairs = m.export()
    sel = np.nonzero(pairs > 0)[0][:200]
    q = ((keys[sel] + 0.5) * 0.1).astype(np.float32)
    out = m.query(q)
    for j, i in enumerate(sel):
        a = alpha[i]
        np.testing.assert_allclose(out["probs"][j], stats.dirichlet.mean(a), rtol=1e-12)
        np.testing.assert_allclose(out["var"][j], stats.dirichlet.var(a), rtol=1e-10)
        assert out["label"][j] == int(np.argmax(a))
        assert out["p_occ"][j] == pytest.approx(1.0 - stats.dirichlet.mean(a)[0], abs=1e-12)
        if np.all(a > 1):
            # MAP of Dir(a): maximise the log density on the simplex
            def neg(z):
                t = np.exp(z - z.max())
                t /= t.sum()
                return -stats.dirichlet.logpdf(np.clip(t, 1e-300, 1), a)
            z0 = np.log(a)
            zz = optimize.minimize(neg, z0, method="Nelder-Mead", options=dict(xatol=1e-12, fatol=1e-14,
                                                                               maxiter=20000)).x
            t = np.exp(zz - zz.max())
            t /= t.sum()
            np.testing.assert_allclose(out["mode"][j], t, atol=2e-5)
        else:
            assert np.all(np.isnan(out["mode"][j]))


def test_readoff_prior_ties_and_states(orc):
    p = orc.params(res=0.1, length_scale=0.3, sigma0=1.0, num_classes=3)
    m = orc.OracleMap(p)
    out = m.query(np.array([[5.0, 5.0, 5.0]], np.float32))  # nothing mapped: prior
    np.testing.assert_allclose(out["probs"][0], 0.25)
    assert out["label"][0] == 0  # tie -> lowest index
    assert out["state"][0] == 1  # unknown
    # a voxel reached only by free points is free; only by class-2 points is occupied
    m.insert_training(np.array([[0.05, 0.05, 0.05]], np.float32), np.array([0]))
    m.insert_training(np.array([[2.05, 0.05, 0.05]], np.float32), np.array([2]))
    out = m.query(np.array([[0.05, 0.05, 0.05], [2.05, 0.05, 0.05]], np.float32))
    assert out["state"].tolist() == [0, 2]
    assert out["label"].tolist() == [0, 2]


# ---------------------------------------------------------------- differentiable form

def _grad_case(orc, seed=19, n=40, nh=60):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-0.35, 0.35, size=(n, 3))
    lab = rng.integers(0, 4, size=n).astype(np.int32)
    held = rng.uniform(-0.3, 0.3, size=(nh, 3)).astype(np.float32)
    hl = rng.integers(0, 4, size=nh).astype(np.int32)
    return xyz, lab, held, hl


def test_gradient_matches_central_differences(orc):
    xyz, lab, held, hl = _grad_case(orc)
    base = dict(res=0.1, length_scale=0.3, sigma0=0.8, num_classes=3)
    p = orc.params(**base)
    ll, gl, gs, gx = orc.heldout_grad(p, xyz, lab, held, hl)
    h = 1e-4
    fd_l = (orc.heldout_ll(orc.params(**{**base, "length_scale": 0.3 + h}), xyz, lab, held, hl) -
            orc.heldout_ll(orc.params(**{**base, "length_scale": 0.3 - h}), xyz, lab, held, hl)) / (2 * h)
    fd_s = (orc.heldout_ll(orc.params(**{**base, "sigma0": 0.8 + h}), xyz, lab, held, hl) -
            orc.heldout_ll(orc.params(**{**base, "sigma0": 0.8 - h}), xyz, lab, held, hl)) / (2 * h)
    assert gl == pytest.approx(fd_l, rel=1e-3)
    assert gs == pytest.approx(fd_s, rel=1e-3)
    for i in range(0, len(xyz), 4):
        for d in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = (orc.heldout_ll(p, xp, lab, held, hl) - orc.heldout_ll(p, xm, lab, held, hl)) / (2 * h)
            assert gx[i, d] == pytest.approx(fd, rel=1e-3, abs=1e-6)


def test_class_scales_against_bruteforce(orc):
    """Reading K13: class k's kernel is sigma0 * sigma0_scale[k] * f; a numpy
    all-pairs sum with distinct per-class scales fixes which scale each
    training point takes."""
    rng = np.random.default_rng(29)
    xyz = rng.uniform(-0.4, 0.4, size=(80, 3)).astype(np.float32)
    lab = rng.integers(0, 5, size=80).astype(np.int32)
    scale = np.array([0.5, 1.0, 2.0, 3.5, 0.25])
    p = orc.params(res=0.1, length_scale=0.3, sigma0=0.6, num_classes=4, sigma0_scale=scale)
    m = orc.OracleMap(p)
    m.insert_training(xyz, lab)
    keys, alpha, pairs = m.export()
    bf = _bruteforce(orc, orc.params(res=0.1, length_scale=0.3, sigma0=0.6, num_classes=4), xyz, lab)
    for k, a, n in zip(map(tuple, keys), alpha, pairs):
        want = bf.get(k, [np.zeros(5), 0])
        np.testing.assert_allclose(a - p.alpha0, want[0] * scale, rtol=1e-12, atol=1e-15)
        assert n == want[1]
    got, _ = orc.alpha_bruteforce(p, xyz, lab, keys[:50])
    np.testing.assert_allclose(got, alpha[:50], rtol=1e-12)


def test_gradient_in_class_scales(orc):
    """dLL/d sigma0_scale[k] against central differences, and the scaling
    identity sum_k s_k dLL/ds_k = sigma0 dLL/dsigma0 (alpha increments are
    linear in sigma0 s_k)."""
    xyz, lab, held, hl = _grad_case(orc)
    scale = [0.7, 1.3, 1.0, 2.2]
    base = dict(res=0.1, length_scale=0.3, sigma0=0.8, num_classes=3, sigma0_scale=scale)
    ll, gsc = orc.heldout_grad_scale(orc.params(**base), xyz, lab, held, hl)
    h = 1e-5
    for k in range(4):
        up, dn = list(scale), list(scale)
        up[k] += h
        dn[k] -= h
        fd = (orc.heldout_ll(orc.params(**{**base, "sigma0_scale": up}), xyz, lab, held, hl) -
              orc.heldout_ll(orc.params(**{**base, "sigma0_scale": dn}), xyz, lab, held, hl)) / (2 * h)
        assert gsc[k] == pytest.approx(fd, rel=1e-4, abs=1e-8)
    _, _, gs, _ = orc.heldout_grad(orc.params(**base), xyz, lab, held, hl)
    assert float(np.dot(scale, gsc)) == pytest.approx(0.8 * gs, rel=1e-10)


def test_extended_block_association_against_bruteforce(orc):
    """Reading K14: with association 1 a voxel takes only the points whose
    voxel lies in its block or a face neighbour; a numpy all-pairs sum with
    that rule, and the exact map minus the left-out (edge and corner
    neighbour) pairs."""
    rng = np.random.default_rng(31)
    B, res, l = 4, 0.1, 0.3
    xyz = (np.round(rng.uniform(-0.6, 0.6, size=(120, 3)) / (B * res)) * (B * res)
           + rng.uniform(-0.12, 0.12, size=(120, 3))).astype(np.float32)  # around block corners and edges
    lab = rng.integers(0, 3, size=120).astype(np.int32)
    base = dict(res=res, length_scale=l, sigma0=0.5, num_classes=2, block_edge=B)
    ext = orc.OracleMap(orc.params(**base, association=1))
    ext.insert_training(xyz, lab)
    keys, alpha, pairs = ext.export()
    vox = np.floor(xyz * np.float32(1 / res)).astype(np.int64)
    pblk = np.floor_divide(vox, B)
    c = (keys + 0.5) * res
    kb = np.floor_divide(keys, B)
    x64 = xyz.astype(np.float64)
    want = np.zeros((len(keys), 3))
    npairs = np.zeros(len(keys), np.int64)
    for i in range(len(xyz)):
        e = c - x64[i]
        d2 = (e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1]) + e[:, 2] * e[:, 2]
        face = np.abs(kb - pblk[i]).sum(1) <= 1
        sel = (d2 < l * l) & face
        want[sel, lab[i]] += 0.5 * np.array([orc.kernel_f(math.sqrt(v) / l) for v in d2[sel]])
        npairs[sel] += 1
    np.testing.assert_allclose(alpha - 0.001, want, rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(pairs, npairs)
    # the exact map has every pair; the extended one drops some here (points near edges and corners)
    exact = orc.OracleMap(orc.params(**base))
    exact.insert_training(xyz, lab)
    ea, ep = exact.alpha_at(keys)
    assert np.all(ep >= pairs) and ep.sum() > pairs.sum()


def test_point_queries_against_bruteforce_and_voxel_centres(orc):
    """Eq. (alpha_kernel) at arbitrary points: a numpy all-pairs sum; at voxel
    centres it equals the map's alpha; it is continuous (f has zero slope at
    r = 1, so alpha is Lipschitz in the query point)."""
    rng = np.random.default_rng(33)
    xyz = rng.uniform(-0.5, 0.5, size=(90, 3)).astype(np.float32)
    lab = rng.integers(0, 4, size=90).astype(np.int32)
    scale = [1.0, 0.5, 2.0, 1.5]
    p = orc.params(res=0.1, length_scale=0.3, sigma0=0.9, num_classes=3, sigma0_scale=scale)
    pts = rng.uniform(-0.7, 0.7, size=(40, 3))
    got = orc.alpha_at_points(p, xyz, lab, pts)
    x64 = xyz.astype(np.float64)
    for q in range(len(pts)):
        e = pts[q] - x64
        d = np.sqrt((e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1]) + e[:, 2] * e[:, 2])
        want = np.full(4, p.alpha0)
        for i in np.nonzero(d < 0.3)[0]:
            want[lab[i]] += 0.9 * scale[lab[i]] * orc.kernel_f(d[i] / 0.3)
        np.testing.assert_allclose(got[q], want, rtol=1e-12)
    m = orc.OracleMap(p)
    m.insert_training(xyz, lab)
    keys, alpha, _ = m.export()
    sel = rng.choice(len(keys), size=60, replace=False)
    np.testing.assert_allclose(orc.alpha_at_points(p, xyz, lab, (keys[sel] + 0.5) * 0.1), alpha[sel], rtol=1e-12)
    step = 1e-6 * rng.normal(size=pts.shape)
    diff = np.abs(orc.alpha_at_points(p, xyz, lab, pts + step) - got).sum(1)
    assert np.all(diff <= 90 * 0.9 * 2.0 * 4.0 / 0.3 * np.linalg.norm(step, axis=1))


def test_soft_labels_grouping_and_weights(orc):
    """Reading K15: hits grouped by (cell, most probable class); per class the
    exact mean of the members' weights.  Three hits of one cell, K = 2."""
    p = orc.params(res=1.0, free_step=100.0, num_classes=2)  # no free samples: every r < s
    pts = np.array([[0.25, 0.5, 0.5], [0.75, 0.5, 0.5], [0.5, 0.25, 0.5]], np.float32)
    probs = np.array([[0.75, 0.25], [0.625, 0.375], [0.25, 0.75]], np.float32)
    xyz, w, st = orc.soft_training_set(p, pts, probs, np.eye(4))
    assert st == dict(hits=3, free=0, train=2)
    got = {int(np.argmax(wi)): (tuple(x), tuple(wi)) for x, wi in zip(xyz, w)}
    assert got[1] == ((0.5, 0.5, 0.5), (0.0, 0.6875, 0.3125))
    assert got[2] == ((0.5, 0.25, 0.5), (0.0, 0.25, 0.75))


def test_soft_labels_reduce_to_hard_labels_and_are_linear(orc):
    """One-hot probability vectors give the hard-label map exactly (same groups,
    centroids and kernel sums); weights a e_j + b e_k give a times the class-j
    map plus b times the class-k map."""
    sc = scenes.small_region_scan(1, n_az=30, n_el=20)
    prm = dict(scenes.SMALL_SCENE_PARAMS)
    K = prm["num_classes"]
    hard = orc.OracleMap(orc.params(**prm))
    st_hard = hard.insert_scan(sc["points"], sc["labels"], sc["pose"])
    soft = orc.OracleMap(orc.params(**prm))
    onehot = np.eye(K, dtype=np.float32)[sc["labels"] - 1]
    assert soft.insert_scan_soft(sc["points"], onehot, sc["pose"]) == st_hard
    for a, b in zip(soft.export(), hard.export()):
        np.testing.assert_array_equal(a, b)
    rng = np.random.default_rng(35)
    xyz = rng.uniform(-0.4, 0.4, size=(50, 3)).astype(np.float32)
    w = np.zeros((50, K + 1), np.float32)
    w[:, 2], w[:, 5] = 0.25, 0.75
    mix = orc.OracleMap(orc.params(**prm))
    mix.insert_training_soft(xyz, w)
    parts = []
    for c in (2, 5):
        m = orc.OracleMap(orc.params(**prm))
        m.insert_training(xyz, np.full(50, c, np.int32))
        parts.append(m.export())
    keys, alpha, pairs = mix.export()
    np.testing.assert_array_equal(keys, parts[0][0])
    np.testing.assert_array_equal(pairs, parts[0][2])
    a0 = prm["alpha0"]
    want = 0.25 * (parts[0][1] - a0) + 0.75 * (parts[1][1] - a0)
    np.testing.assert_allclose(alpha - a0, want, rtol=1e-12, atol=1e-15)


def test_per_class_support_against_bruteforce(orc):
    """Reading K16: class k's kernel has support l_k = l * l_scale[k]; a numpy
    all-pairs sum with per-class supports for hard labels, and the soft path
    with one-hot weights giving the same map."""
    rng = np.random.default_rng(39)
    xyz = rng.uniform(-0.35, 0.35, size=(70, 3)).astype(np.float32)
    lab = rng.integers(0, 4, size=70).astype(np.int32)
    ls = np.array([1.0, 0.5, 1.6, 0.8])
    base = dict(res=0.1, length_scale=0.25, sigma0=0.6, num_classes=3, l_scale=ls)
    m = orc.OracleMap(orc.params(**base))
    m.insert_training(xyz, lab)
    keys, alpha, pairs = m.export()
    c = (keys + 0.5) * 0.1
    want = np.zeros((len(keys), 4))
    npairs = np.zeros(len(keys), np.int64)
    x64 = xyz.astype(np.float64)
    for i in range(len(xyz)):
        lk = 0.25 * ls[lab[i]]
        e = c - x64[i]
        d2 = (e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1]) + e[:, 2] * e[:, 2]
        sel = d2 < lk * lk
        want[sel, lab[i]] += 0.6 * np.array([orc.kernel_f(math.sqrt(v) / lk) for v in d2[sel]])
        npairs[sel] += 1
    np.testing.assert_allclose(alpha - 0.001, want, rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(pairs, npairs)
    got, gp = orc.alpha_bruteforce(orc.params(**base), xyz, lab, keys)
    np.testing.assert_allclose(got, alpha, rtol=1e-12)
    np.testing.assert_array_equal(gp, pairs)
    soft = orc.OracleMap(orc.params(**base))
    soft.insert_training_soft(xyz, np.eye(4, dtype=np.float32)[lab])
    for a, b in zip(soft.export(), m.export()):
        np.testing.assert_array_equal(a, b)


def test_gradient_sigma0_and_euler_identities(orc):
    """alpha - alpha0 is linear in sigma0; alpha_v depends on (x_i - c_v)/l only,
    so l dLL/dl + sum_i (x_i - c_v) . dLL/dx_i = 0 when every held-out point is
    in one voxel v."""
    xyz, lab, held, hl = _grad_case(orc, seed=23)
    held = np.tile(np.array([[0.05, 0.05, 0.05]], np.float32), (20, 1))
    hl = np.arange(20, dtype=np.int32) % 4
    p = orc.params(res=0.1, length_scale=0.3, sigma0=0.8, num_classes=3)
    ll, gl, gs, gx = orc.heldout_grad(p, xyz, lab, held, hl)
    c = np.array([0.05, 0.05, 0.05])
    euler = 0.3 * gl + np.sum((xyz - c) * gx)
    assert abs(euler) < 1e-9 * max(1.0, abs(0.3 * gl))
    # d alpha / d sigma0 = (alpha - alpha0) / sigma0  =>  dLL/dsigma0 = sum_v g_v . (alpha_v - alpha0) / sigma0
    m = orc.OracleMap(p)
    m.insert_training(xyz.astype(np.float32), lab)
    a, _ = m.alpha_at(np.array([[0, 0, 0]]))
    S = a[0].sum()
    g = np.array([np.sum(hl == k) / a[0][k] for k in range(4)]) - len(hl) / S
    assert gs == pytest.approx(float(g @ (a[0] - 0.001) / 0.8), rel=1e-5)


# ---------------------------------------------------------------- a whole scan

def test_small_scan_training_set_invariants(orc):
    sc = scenes.small_region_scan(0, n_az=40, n_el=30)
    p = orc.params(**scenes.SMALL_SCENE_PARAMS)
    xyz, lab, st = orc.training_set(p, sc["points"], sc["labels"], sc["pose"])
    samp, slab = orc.samples(p, sc["points"], sc["labels"], sc["pose"])
    assert st["hits"] + st["free"] == len(samp)
    assert st["train"] == len(xyz)
    # one training point per distinct (cell, label) of the samples
    cells = np.floor(samp * np.float32(1 / 0.1)).astype(np.int64)
    distinct = {(tuple(c), int(l)) for c, l in zip(cells, slab)}
    assert len(distinct) == len(xyz)
    # every centroid lies in (or on the FP32 edge of) its cell's box
    tc = np.floor(xyz * np.float32(10.0)).astype(np.int64)
    inside = {(tuple(c), int(l)) for c, l in zip(tc, lab)}
    assert len(inside & distinct) >= len(xyz) - 2
    with pytest.raises(ValueError):
        orc.training_set(p, sc["points"][:3], np.array([1, 11, 2]), sc["pose"])


def _f32_round_fraction(fr):
    """Nearest FP32 to a Fraction, ties to even (exact rational comparisons)."""
    from fractions import Fraction
    if fr == 0:
        return 0.0
    x = np.float32(float(fr))  # within an ulp or two of the answer
    cands = {x, np.nextafter(x, np.float32(np.inf)), np.nextafter(x, np.float32(-np.inf))}
    cands |= {np.nextafter(c, np.float32(np.inf)) for c in list(cands)} | \
        {np.nextafter(c, np.float32(-np.inf)) for c in list(cands)}
    best = min(cands, key=lambda c: (abs(Fraction(float(c)) - fr),
                                     int(np.frombuffer(np.float32(c).tobytes(), np.uint32)[0]) & 1))
    return float(best)


def test_exact_mean_against_rational_arithmetic(orc):
    """Reading K4 (centroid = exact mean rounded once to FP32) against Python
    Fractions: same-sign cells, mixed magnitudes over many binades, near-ties,
    subnormals and long segments."""
    from fractions import Fraction
    rng = np.random.default_rng(31)
    cases = []
    for _ in range(300):
        n = int(rng.integers(1, 40))
        base = rng.uniform(-50, 50)
        cases.append((base + rng.uniform(0, 0.1, size=n)).astype(np.float32))
    for _ in range(100):  # a cell next to a coordinate plane: values spanning many binades
        n = int(rng.integers(2, 300))
        cases.append((rng.uniform(0, 0.1, size=n) * 10.0 ** rng.integers(-30, 0, size=n)).astype(np.float32))
    for _ in range(50):  # exact halfway cases: two neighbouring floats
        a = np.float32(rng.uniform(1, 2))
        cases.append(np.array([a, np.nextafter(a, np.float32(3))], np.float32))
    cases.append(np.array([1e-45, 3e-45, 1e-44], np.float32))  # subnormals
    cases.append(np.full(5000, np.float32(0.1)) + rng.uniform(0, 1e-3, 5000).astype(np.float32))
    cases.append(-np.abs(rng.normal(size=17)).astype(np.float32))
    for v in cases:
        exact = sum(Fraction(float(x)) for x in v) / len(v)
        assert orc.exact_mean_f32(v) == _f32_round_fraction(exact), v[:4]


def test_slab_split_of_the_oracle_gradient_is_exact(orc):
    """The full-size GPU test runs the oracle's held-out gradient per slab of
    held-out points in parallel and adds the slabs' terms; on a small case
    that sum equals one call over everything (FP64 summation order only)."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_gpu_fullsize import _oracle_grad_parallel, _world
    prm = dict(scenes.DIFF_PARAMS)
    sc = next(iter(scenes.small_region_lidar_sequence(1, n_beams=16, n_az=256)))
    x, lab, _ = orc.training_set(orc.params(**prm), sc["points"], sc["labels"], sc["pose"])
    held = _world(sc["held_points"], sc["pose"])
    hl = sc["held_labels"].astype(np.int32)
    ll, gl, gs, gx = orc.heldout_grad(orc.params(**prm), x.astype(np.float64), lab, held, hl)
    pll, pgl, pgs, pgx = _oracle_grad_parallel(prm, x, lab.astype(np.int32), held, hl, slabs=5)
    assert pll == pytest.approx(ll, rel=1e-12)
    assert pgl == pytest.approx(gl, rel=1e-10) and pgs == pytest.approx(gs, rel=1e-10)
    assert np.abs(pgx - gx).max() <= 1e-10 * np.abs(gx).max()
