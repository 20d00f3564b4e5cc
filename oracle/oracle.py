"""ctypes front end of the FP64 S-BKI oracle (``sbki_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module; the product package never does.  It
shares no code with the CUDA library.  Functions take and return numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbki_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class OrcParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("res", "length_scale", "sigma0", "alpha0", "free_step", "ds_res",
                                          "min_range", "max_range", "free_thresh", "occ_thresh")] + \
               [("num_classes", C.c_int32), ("block_edge", C.c_int32), ("sensor_model", C.c_int32),
                ("sigma0_scale", C.c_double * 32), ("association", C.c_int32), ("l_scale", C.c_double * 32)]


def params(res=0.1, length_scale=0.3, sigma0=0.1, alpha0=0.001, free_step=0.3, ds_res=None, min_range=0.0,
           max_range=1e30, free_thresh=0.47, occ_thresh=0.6, num_classes=10, block_edge=8, sensor_model=0,
           sigma0_scale=None, association=0, l_scale=None, **_ignored):
    """Parameter block; defaults follow Table (parameters) and Sec. V-A of the paper.
    sensor_model 0: kernel inference, Eq. (alpha_kernel); 1: counting model, Eq. (alpha).
    sigma0_scale: per-class multipliers of sigma0 (classes 0..K; default all 1).
    association 0: every voxel within l (exact); 1: the extended block (reading K14).
    l_scale: per-class multipliers of the length scale (reading K16; default all 1)."""
    sc = [1.0] * 32
    if sigma0_scale is not None:
        for k, v in enumerate(sigma0_scale):
            sc[k] = float(v)
    ls = [1.0] * 32
    if l_scale is not None:
        for k, v in enumerate(l_scale):
            ls[k] = float(v)
    return OrcParams(res, length_scale, sigma0, alpha0, free_step, res if ds_res is None else ds_res, min_range,
                     max_range, free_thresh, occ_thresh, num_classes, block_edge, sensor_model,
                     (C.c_double * 32)(*sc), association, (C.c_double * 32)(*ls))


_P = C.POINTER


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i64, f64, i32 = C.c_int64, C.c_double, C.c_int32
            vp = C.c_void_p
            L.orc_map_create.restype = vp
            L.orc_map_create.argtypes = [_P(OrcParams)]
            L.orc_map_destroy.argtypes = [vp]
            L.orc_kernel_f.restype = f64
            L.orc_kernel_f.argtypes = [f64]
            L.orc_kernel_df.restype = f64
            L.orc_kernel_df.argtypes = [f64]
            L.orc_exact_mean_f32.restype = C.c_float
            L.orc_exact_mean_f32.argtypes = [vp, i64]
            L.orc_transform.restype = i64
            L.orc_transform.argtypes = [_P(OrcParams), vp, i64, vp, vp, vp]
            L.orc_samples.restype = i64
            L.orc_samples.argtypes = [_P(OrcParams), vp, vp, i64, vp, vp, vp, i64]
            L.orc_training_set.restype = i64
            L.orc_training_set.argtypes = [_P(OrcParams), vp, vp, i64, vp, vp, vp, i64, vp]
            L.orc_map_insert_training.restype = C.c_int
            L.orc_map_insert_training.argtypes = [vp, vp, vp, i64]
            L.orc_map_insert_scan.restype = C.c_int
            L.orc_map_insert_scan.argtypes = [vp, vp, vp, i64, vp, vp]
            L.orc_map_num_blocks.restype = i64
            L.orc_map_num_blocks.argtypes = [vp]
            L.orc_map_block_keys.argtypes = [vp, vp]
            L.orc_map_export.restype = i64
            L.orc_map_export.argtypes = [vp, vp, vp, vp]
            L.orc_map_alpha_at.argtypes = [vp, vp, i64, vp, vp]
            L.orc_alpha_bruteforce.argtypes = [_P(OrcParams), vp, vp, i64, vp, i64, vp, vp]
            L.orc_map_query.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp]
            L.orc_alpha_at_points.argtypes = [_P(OrcParams), vp, vp, i64, vp, i64, vp]
            L.orc_soft_training_set.restype = i64
            L.orc_soft_training_set.argtypes = [_P(OrcParams), vp, vp, i64, vp, vp, vp, i64, vp]
            L.orc_map_insert_training_soft.restype = C.c_int
            L.orc_map_insert_training_soft.argtypes = [vp, vp, vp, i64]
            L.orc_map_insert_scan_soft.restype = C.c_int
            L.orc_map_insert_scan_soft.argtypes = [vp, vp, vp, i64, vp, vp]
            L.orc_heldout_grad.restype = f64
            L.orc_heldout_grad.argtypes = [_P(OrcParams), vp, vp, i64, vp, vp, i64, vp, vp, vp]
            L.orc_heldout_grad_scale.restype = f64
            L.orc_heldout_grad_scale.argtypes = [_P(OrcParams), vp, vp, i64, vp, vp, i64, vp]
            L.orc_heldout_ll.restype = f64
            L.orc_heldout_ll.argtypes = [_P(OrcParams), vp, vp, i64, vp, vp, i64]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def kernel_f(r: float) -> float:
    return lib().orc_kernel_f(float(r))


def kernel_df(r: float) -> float:
    return lib().orc_kernel_df(float(r))


def exact_mean_f32(values):
    """Reading K4: exact mean of FP32 values rounded once to FP32."""
    v = _f32(values).reshape(-1)
    return float(lib().orc_exact_mean_f32(_ptr(v), len(v)))


def transform(p, points, pose):
    """Step a1: world coordinates (float32) of the kept points and their indices."""
    pts = _f32(points).reshape(-1, 3)
    T = _f64(pose).reshape(16)
    out = np.empty_like(pts)
    idx = np.empty(len(pts), np.int64)
    n = lib().orc_transform(C.byref(p), _ptr(pts), len(pts), _ptr(T), _ptr(out), _ptr(idx))
    return out[:n], idx[:n]


def samples(p, points, labels, pose):
    """Steps a1+a2: hits then free samples in source order (xyz float32, labels)."""
    pts, lab, T = _f32(points).reshape(-1, 3), _i32(labels), _f64(pose).reshape(16)
    n = lib().orc_samples(C.byref(p), _ptr(pts), _ptr(lab), len(pts), _ptr(T), None, None, 0)
    if n < 0:
        raise ValueError("label out of range")
    xyz = np.empty((n, 3), np.float32)
    ol = np.empty(n, np.int32)
    lib().orc_samples(C.byref(p), _ptr(pts), _ptr(lab), len(pts), _ptr(T), _ptr(xyz), _ptr(ol), n)
    return xyz, ol


def training_set(p, points, labels, pose):
    """Steps a1..a3: (xyz float32 [P,3], labels int32 [P], stats dict)."""
    pts, lab, T = _f32(points).reshape(-1, 3), _i32(labels), _f64(pose).reshape(16)
    st = np.zeros(3, np.int64)
    # the training set is never larger than hits + free samples; size from a2's count
    cap = lib().orc_samples(C.byref(p), _ptr(pts), _ptr(lab), len(pts), _ptr(T), None, None, 0)
    if cap < 0:
        raise ValueError("label out of range")
    xyz = np.empty((max(cap, 1), 3), np.float32)
    ol = np.empty(max(cap, 1), np.int32)
    n = lib().orc_training_set(C.byref(p), _ptr(pts), _ptr(lab), len(pts), _ptr(T), _ptr(xyz), _ptr(ol), cap,
                               _ptr(st))
    return xyz[:n].copy(), ol[:n].copy(), dict(hits=int(st[0]), free=int(st[1]), train=int(st[2]))


def alpha_bruteforce(p, xyz, labels, keys):
    """alpha at voxel keys [q,3] from a training set by summing over all points."""
    xyz, lab = _f32(xyz).reshape(-1, 3), _i32(labels)
    keys = np.ascontiguousarray(keys, dtype=np.int64).reshape(-1, 3)
    K1 = p.num_classes + 1
    alpha = np.empty((len(keys), K1), np.float64)
    pairs = np.empty(len(keys), np.int64)
    lib().orc_alpha_bruteforce(C.byref(p), _ptr(xyz), _ptr(lab), len(xyz), _ptr(keys), len(keys), _ptr(alpha),
                               _ptr(pairs))
    return alpha, pairs


def soft_training_set(p, points, probs, pose):
    """Steps a1..a3 with soft labels (reading K15): probs [n,K] over classes 1..K.
    Returns (xyz float32 [P,3], weights float32 [P,K+1], stats dict)."""
    pts, pr, T = _f32(points).reshape(-1, 3), _f32(probs).reshape(len(points), -1), _f64(pose).reshape(16)
    K1 = p.num_classes + 1
    st = np.zeros(3, np.int64)
    n = lib().orc_soft_training_set(C.byref(p), _ptr(pts), _ptr(pr), len(pts), _ptr(T), None, None, 0, _ptr(st))
    xyz = np.empty((max(n, 1), 3), np.float32)
    w = np.empty((max(n, 1), K1), np.float32)
    lib().orc_soft_training_set(C.byref(p), _ptr(pts), _ptr(pr), len(pts), _ptr(T), _ptr(xyz), _ptr(w), n, _ptr(st))
    return xyz[:n], w[:n], dict(hits=int(st[0]), free=int(st[1]), train=int(st[2]))


def alpha_at_points(p, xyz, labels, pts):
    """Eq. (alpha_kernel) at arbitrary world points pts [q,3] (FP64) from a training set: alpha [q,K+1]."""
    xyz, lab = _f32(xyz).reshape(-1, 3), _i32(labels)
    pts = _f64(pts).reshape(-1, 3)
    alpha = np.empty((len(pts), p.num_classes + 1), np.float64)
    lib().orc_alpha_at_points(C.byref(p), _ptr(xyz), _ptr(lab), len(xyz), _ptr(pts), len(pts), _ptr(alpha))
    return alpha


def heldout_ll(p, xyz64, labels, held_xyz, held_labels):
    xyz64, lab = _f64(xyz64).reshape(-1, 3), _i32(labels)
    hx, hl = _f32(held_xyz).reshape(-1, 3), _i32(held_labels)
    return lib().orc_heldout_ll(C.byref(p), _ptr(xyz64), _ptr(lab), len(xyz64), _ptr(hx), _ptr(hl), len(hx))


def heldout_grad(p, xyz64, labels, held_xyz, held_labels):
    """(LL, dLL/dl, dLL/dsigma0, dLL/dxyz [n,3]) in FP64."""
    xyz64, lab = _f64(xyz64).reshape(-1, 3), _i32(labels)
    hx, hl = _f32(held_xyz).reshape(-1, 3), _i32(held_labels)
    gl = C.c_double()
    gs = C.c_double()
    gx = np.zeros_like(xyz64)
    ll = lib().orc_heldout_grad(C.byref(p), _ptr(xyz64), _ptr(lab), len(xyz64), _ptr(hx), _ptr(hl), len(hx),
                                C.byref(gl), C.byref(gs), _ptr(gx))
    return ll, gl.value, gs.value, gx


def heldout_grad_scale(p, xyz64, labels, held_xyz, held_labels):
    """(LL, dLL/d sigma0_scale[k] for k = 0..K) in FP64."""
    xyz64, lab = _f64(xyz64).reshape(-1, 3), _i32(labels)
    hx, hl = _f32(held_xyz).reshape(-1, 3), _i32(held_labels)
    gsc = np.zeros(p.num_classes + 1)
    ll = lib().orc_heldout_grad_scale(C.byref(p), _ptr(xyz64), _ptr(lab), len(xyz64), _ptr(hx), _ptr(hl), len(hx),
                                      _ptr(gsc))
    return ll, gsc


class OracleMap:
    """A persistent FP64 map: per-scan updates accumulate (Sec. IV)."""

    def __init__(self, p):
        self.p = p
        self.K1 = p.num_classes + 1
        self._h = lib().orc_map_create(C.byref(p))

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.orc_map_destroy(h)

    def insert_scan(self, points, labels, pose):
        pts, lab, T = _f32(points).reshape(-1, 3), _i32(labels), _f64(pose).reshape(16)
        st = np.zeros(3, np.int64)
        if lib().orc_map_insert_scan(self._h, _ptr(pts), _ptr(lab), len(pts), _ptr(T), _ptr(st)) != 0:
            raise ValueError("label out of range")
        return dict(hits=int(st[0]), free=int(st[1]), train=int(st[2]))

    def insert_training(self, xyz, labels):
        xyz, lab = _f32(xyz).reshape(-1, 3), _i32(labels)
        if lib().orc_map_insert_training(self._h, _ptr(xyz), _ptr(lab), len(xyz)) != 0:
            raise ValueError("label out of range")

    def insert_training_soft(self, xyz, weights):
        """Eq. (alpha_kernel) with weight vectors (reading K15): xyz [n,3], weights [n,K+1]."""
        xyz, w = _f32(xyz).reshape(-1, 3), _f32(weights).reshape(-1, self.K1)
        lib().orc_map_insert_training_soft(self._h, _ptr(xyz), _ptr(w), len(xyz))

    def insert_scan_soft(self, points, probs, pose):
        """A scan with soft labels (reading K15): probs [n,K] over classes 1..K."""
        pts, T = _f32(points).reshape(-1, 3), _f64(pose).reshape(16)
        pr = _f32(probs).reshape(len(pts), self.K1 - 1)
        st = np.zeros(3, np.int64)
        lib().orc_map_insert_scan_soft(self._h, _ptr(pts), _ptr(pr), len(pts), _ptr(T), _ptr(st))
        return dict(hits=int(st[0]), free=int(st[1]), train=int(st[2]))

    def block_keys(self):
        n = lib().orc_map_num_blocks(self._h)
        k = np.empty((n, 3), np.int64)
        if n:
            lib().orc_map_block_keys(self._h, _ptr(k))
        return k

    def export(self):
        """(voxel keys [cnt,3] sorted lexicographically, alpha [cnt,K+1], pairs [cnt])."""
        n = lib().orc_map_export(self._h, None, None, None)
        keys = np.empty((n, 3), np.int64)
        alpha = np.empty((n, self.K1), np.float64)
        pairs = np.empty(n, np.int64)
        if n:
            lib().orc_map_export(self._h, _ptr(keys), _ptr(alpha), _ptr(pairs))
        return keys, alpha, pairs

    def alpha_at(self, keys):
        keys = np.ascontiguousarray(keys, dtype=np.int64).reshape(-1, 3)
        a = np.empty((len(keys), self.K1), np.float64)
        pc = np.empty(len(keys), np.int64)
        lib().orc_map_alpha_at(self._h, _ptr(keys), len(keys), _ptr(a), _ptr(pc))
        return a, pc

    def query(self, xyz):
        """Read-off at world points: dict(probs, var, mode, label, p_occ, state)."""
        xyz = _f32(xyz).reshape(-1, 3)
        q = len(xyz)
        out = dict(probs=np.empty((q, self.K1)), var=np.empty((q, self.K1)), mode=np.empty((q, self.K1)),
                   label=np.empty(q, np.int32), p_occ=np.empty(q), state=np.empty(q, np.int32))
        lib().orc_map_query(self._h, _ptr(xyz), q, _ptr(out["probs"]), _ptr(out["var"]), _ptr(out["mode"]),
                            _ptr(out["label"]), _ptr(out["p_occ"]), _ptr(out["state"]))
        return out
