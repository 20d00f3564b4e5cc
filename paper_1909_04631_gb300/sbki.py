"""Thin ctypes binding of libsbki (include/sbki.h).

Argument marshalling only: every step of the map update runs in the CUDA
kernels of libsbki.so.  Arrays may be numpy arrays (host memory) or torch
tensors (host or CUDA); CUDA tensors are passed by device pointer and used in
stream order on the map's stream.  There is no CPU fallback: if the library
is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

OK, ERR_INVALID_ARG, ERR_LABEL_RANGE, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_NOT_FOUND = range(7)
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "label out of range", 3: "capacity exceeded", 4: "CUDA error",
                5: "device wait timed out", 6: "not found"}

EXPORTED = ["sbki_default_params", "sbki_create_map", "sbki_destroy_map", "sbki_insert_scan",
            "sbki_insert_scan_async", "sbki_sync", "sbki_training_set", "sbki_insert_training", "sbki_query_probs",
            "sbki_voxel_count", "sbki_export", "sbki_profile", "sbki_profile_read", "sbki_kernel_values", "sbki_last_error", "sbki_status_string",
            "sbki_training_set_noalloc", "sbki_grad_clear", "sbki_heldout_loglik", "sbki_grad_add_alpha",
            "sbki_backward", "sbki_forward_alpha", "sbki_grad", "sbki_insert_batch", "sbki_select_map",
            "sbki_get_tuning", "sbki_set_tuning", "sbki_import", "sbki_selftest_bounded_wait", "sbki_backward_scales",
            "sbki_query_points", "sbki_insert_scan_soft", "sbki_training_set_soft", "sbki_export_blocks"]


class SbkiError(RuntimeError):
    def __init__(self, status: int, message: str, count=None):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status
        self.count = count  # a count the failing call still reported (output-capacity errors), else None


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("res", "length_scale", "sigma0", "alpha0", "free_step", "ds_res",
                                          "min_range", "max_range", "free_thresh", "occ_thresh")] + \
               [("num_classes", C.c_int32), ("block_edge", C.c_int32), ("pool_blocks", C.c_int64),
                ("sample_capacity", C.c_int64), ("track_pairs", C.c_int32), ("device", C.c_int32),
                ("accumulate_mode", C.c_int32), ("num_maps", C.c_int32),
                ("cuda_stream", C.c_void_p), ("sensor_model", C.c_int32), ("sigma0_scale", C.c_double * 32),
                ("association", C.c_int32), ("l_scale", C.c_double * 32)]


class Scan(C.Structure):
    _fields_ = [("points", C.c_void_p), ("labels", C.c_void_p), ("n", C.c_int64), ("pose", C.c_double * 16),
                ("map_id", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("accumulate_ctas_per_sm", C.c_int32), ("accumulate_chunk", C.c_int32),
                ("touch_ctas_per_sm", C.c_int32), ("ingest_ctas_per_sm", C.c_int32)]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class ProfileData(C.Structure):
    _fields_ = [("inserts", C.c_int64), ("launches", C.c_int64), ("ingest_ms", C.c_double),
                ("blocks_ms", C.c_double), ("accumulate_ms", C.c_double), ("readback_bytes", C.c_int64)]

    def as_dict(self):
        return {n: (float(getattr(self, n)) if n.endswith("_ms") else int(getattr(self, n))) for n, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("hits", "dropped", "free_samples", "train_points", "touched_blocks",
                                         "new_blocks", "pairs", "touched_voxels", "total_blocks")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsbki.so (building it first if it is missing and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError("libsbki.so is not built; run paper_1909_04631_gb300.build.build()")
            _build.build()
        L = C.CDLL(_build.LIB)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        P = C.POINTER
        L.sbki_default_params.argtypes = [P(Params)]
        L.sbki_create_map.argtypes = [P(Params), P(vp)]
        L.sbki_destroy_map.argtypes = [vp]
        L.sbki_destroy_map.restype = None
        L.sbki_insert_scan.argtypes = [vp, vp, vp, i64, vp, P(Stats)]
        L.sbki_insert_scan_async.argtypes = [vp, vp, vp, i64, vp]
        L.sbki_sync.argtypes = [vp, P(Stats)]
        L.sbki_training_set.argtypes = [vp, vp, vp, i64, vp, vp, i64, P(i64)]
        L.sbki_insert_training.argtypes = [vp, vp, i64, P(Stats)]
        L.sbki_training_set_noalloc.argtypes = [P(Params), vp, vp, i64, vp, vp, i64, P(i64)]
        L.sbki_query_probs.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp]
        L.sbki_insert_batch.argtypes = [vp, vp, i32, P(Stats)]
        L.sbki_select_map.argtypes = [vp, i32]
        L.sbki_get_tuning.argtypes = [vp, P(Tuning)]
        L.sbki_import.argtypes = [vp, vp, vp, i64]
        L.sbki_selftest_bounded_wait.argtypes = [i32, P(i32)]
        L.sbki_set_tuning.argtypes = [vp, P(Tuning)]
        L.sbki_grad_clear.argtypes = [vp]
        L.sbki_heldout_loglik.argtypes = [vp, vp, vp, i64, i32, P(C.c_double)]
        L.sbki_grad_add_alpha.argtypes = [vp, vp, vp, i64, P(i64)]
        L.sbki_backward.argtypes = [vp, vp, i64, P(C.c_double), P(C.c_double), vp]
        L.sbki_backward_scales.argtypes = [vp, vp, i64, vp]
        L.sbki_forward_alpha.argtypes = [P(Params), vp, i64, vp, vp, i64, P(i64)]
        L.sbki_grad.argtypes = [P(Params), vp, i64, vp, vp, i64, P(C.c_double), P(C.c_double), vp]
        L.sbki_query_points.argtypes = [P(Params), vp, i64, vp, i64, vp]
        L.sbki_insert_scan_soft.argtypes = [vp, vp, vp, i64, vp, P(Stats)]
        L.sbki_export_blocks.argtypes = [vp, vp, vp, i64, P(i64)]
        L.sbki_training_set_soft.argtypes = [vp, vp, vp, i64, vp, vp, vp, i64, P(i64)]
        L.sbki_voxel_count.argtypes = [vp, P(i64)]
        L.sbki_export.argtypes = [vp, vp, vp, vp, i64, P(i64)]
        L.sbki_last_error.argtypes = [vp]
        L.sbki_last_error.restype = C.c_char_p
        L.sbki_profile.argtypes = [vp, i32, i32]
        L.sbki_profile.restype = C.c_int
        L.sbki_profile_read.argtypes = [vp, P(ProfileData)]
        L.sbki_profile_read.restype = C.c_int
        L.sbki_kernel_values.argtypes = [vp, i64, vp, i32, vp]
        L.sbki_kernel_values.restype = C.c_int
        L.sbki_status_string.argtypes = [C.c_int]
        L.sbki_status_string.restype = C.c_char_p
        for f in ("sbki_default_params", "sbki_create_map", "sbki_insert_scan", "sbki_insert_scan_async", "sbki_sync",
                  "sbki_training_set", "sbki_insert_training", "sbki_query_probs", "sbki_voxel_count",
                  "sbki_export", "sbki_training_set_noalloc", "sbki_grad_clear", "sbki_heldout_loglik",
                  "sbki_grad_add_alpha", "sbki_backward", "sbki_forward_alpha", "sbki_grad", "sbki_insert_batch",
                  "sbki_select_map", "sbki_get_tuning", "sbki_set_tuning", "sbki_import",
                  "sbki_selftest_bounded_wait", "sbki_backward_scales", "sbki_query_points", "sbki_insert_scan_soft",
                  "sbki_training_set_soft", "sbki_export_blocks"):
            getattr(L, f).restype = C.c_int
        _lib = L
        return L


def set_param(p: Params, k: str, v) -> None:
    """p.k = v; sigma0_scale takes a sequence of per-class scales (classes
    0..len-1; the remaining entries keep their values)."""
    if not hasattr(p, k):
        raise TypeError("unknown parameter %r" % k)
    if k in ("sigma0_scale", "l_scale"):
        vals = [float(x) for x in v]
        if len(vals) > 32:
            raise ValueError("at most 32 classes")
        arr = getattr(p, k)
        for i, x in enumerate(vals):
            arr[i] = x
        return
    setattr(p, k, v)


def default_params(**kw) -> Params:
    p = Params()
    load().sbki_default_params(C.byref(p))
    for k, v in kw.items():
        set_param(p, k, v)
    return p


def check_noalloc_args(params: Params, points, labels, out) -> None:
    """Refuses arguments that would make sbki_training_set_noalloc read or
    write past a buffer: points must be float32 [n,3], labels int32 [n], out
    float32 [cap,4], all contiguous CUDA tensors on device params.device.
    TypeError for a wrong kind, dtype or device; ValueError for a wrong shape."""
    import torch
    want = (("points", points, torch.float32), ("labels", labels, torch.int32), ("out", out, torch.float32))
    for name, t, dt in want:
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise TypeError("%s must be a CUDA tensor" % name)
        if t.dtype != dt:
            raise TypeError("%s must be %s, got %s" % (name, dt, t.dtype))
        if t.device.index != params.device:
            raise TypeError("%s is on cuda:%s, the parameters name cuda:%d" % (name, t.device.index, params.device))
        if not t.is_contiguous():
            raise TypeError("%s must be contiguous" % name)
    if points.dim() != 2 or points.shape[1] != 3:
        raise ValueError("points must have shape [n,3], got %s" % (tuple(points.shape),))
    if labels.dim() != 1 or labels.shape[0] != points.shape[0]:
        raise ValueError("labels must have shape [%d], got %s" % (points.shape[0], tuple(labels.shape)))
    if out.dim() != 2 or out.shape[1] != 4:
        raise ValueError("out must have shape [cap,4], got %s" % (tuple(out.shape),))


def training_set_noalloc(params: Params, points, labels, pose, out):
    """Training set of a scan (steps a1-a3) through the entry point that
    allocates nothing: points [n,3] float32, labels [n] int32 and out [cap,4]
    float32 are CUDA tensors on params.device (the caller's memory); work runs
    on params.cuda_stream.  Returns the number of points written to out.  When
    out is too small, the SbkiError raised carries the full count in .count
    (the first cap points are written)."""
    check_noalloc_args(params, points, labels, out)
    L = load()
    T = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
    cnt = C.c_int64()
    st = L.sbki_training_set_noalloc(C.byref(params), C.c_void_p(points.data_ptr()), C.c_void_p(labels.data_ptr()),
                                     points.shape[0], T.ctypes.data_as(C.c_void_p), C.c_void_p(out.data_ptr()),
                                     out.shape[0], C.byref(cnt))
    if st != OK:
        raise SbkiError(st, L.sbki_last_error(None).decode(), count=cnt.value)
    return cnt.value


def _as_i64(x, tail):
    if hasattr(x, "data_ptr"):
        import torch
        return x.to(torch.int64).contiguous()
    return np.ascontiguousarray(x, dtype=np.int64).reshape(-1, tail)


def forward_alpha(params: Params, xyzl):
    """(keys int64 [n,3], alpha float32 [n,K+1]) of a training set xyzl [p,4] at every
    voxel of the blocks it reaches (a map is created and destroyed inside)."""
    L = load()
    x = _as(xyzl, np.float32, 4)
    xp, keep = _ptr(x)
    cnt = C.c_int64()
    st = L.sbki_forward_alpha(C.byref(params), xp, x.shape[0], None, None, 0, C.byref(cnt))
    if st != OK:
        raise SbkiError(st, L.sbki_last_error(None).decode())
    n = cnt.value
    K1 = params.num_classes + 1
    keys = np.empty((max(n, 1), 3), np.int64)
    alpha = np.empty((max(n, 1), K1), np.float32)
    st = L.sbki_forward_alpha(C.byref(params), xp, x.shape[0], keys.ctypes.data_as(C.c_void_p),
                              alpha.ctypes.data_as(C.c_void_p), n, C.byref(cnt))
    if st != OK:
        raise SbkiError(st, L.sbki_last_error(None).decode())
    return keys[:cnt.value], alpha[:cnt.value]


def query_points(params: Params, xyzl, pts, out=None):
    """Eq. (alpha_kernel) at arbitrary points pts [q,3] from a training set xyzl
    [p,4] (stateless): alpha [q,K+1] float32.  numpy arrays or CUDA tensors;
    out (optional) receives the result in place."""
    L = load()
    x = _as(xyzl, np.float32, 4)
    q = _as(pts, np.float32, 3)
    K1 = params.num_classes + 1
    nq = q.shape[0]
    if out is None:
        if hasattr(q, "data_ptr"):
            import torch
            out = torch.empty((nq, K1), dtype=torch.float32, device=q.device)
        else:
            out = np.empty((nq, K1), np.float32)
    xp, k1 = _ptr(x)
    qp, k2 = _ptr(q)
    op, k3 = _ptr(out)
    st = L.sbki_query_points(C.byref(params), xp, x.shape[0], qp, nq, op)
    if st != OK:
        raise SbkiError(st, L.sbki_last_error(None).decode())
    return out


def grad(params: Params, xyzl, keys, grad_alpha):
    """(dL/dl, dL/dsigma0, dL/dxyz [p,3]) for dL/dalpha given at voxel keys."""
    L = load()
    x = _as(xyzl, np.float32, 4)
    k = _as_i64(keys, 3)
    gvals = _as(grad_alpha, np.float32, params.num_classes + 1)
    xp, k1 = _ptr(x)
    kp, k2 = _ptr(k)
    gp, k3 = _ptr(gvals)
    gx = np.empty((max(x.shape[0], 1), 3), np.float32)
    gl, gs = C.c_double(), C.c_double()
    st = L.sbki_grad(C.byref(params), xp, x.shape[0], kp, gp, k.shape[0], C.byref(gl), C.byref(gs),
                     gx.ctypes.data_as(C.c_void_p))
    if st != OK:
        raise SbkiError(st, L.sbki_last_error(None).decode())
    return gl.value, gs.value, gx[:x.shape[0]]


def selftest_bounded_wait(device=0):
    """Status the device reported when a bounded wait ran out (expected: ERR_TIMEOUT)."""
    L = load()
    out = C.c_int32()
    st = L.sbki_selftest_bounded_wait(int(device), C.byref(out))
    if st != OK:
        raise SbkiError(st, L.sbki_last_error(None).decode())
    return out.value


def kernel_values(r, method=0):
    """f(r) of Eq. (kernel) on the GPU (method 0: update form, 1: trigonometric form)."""
    import torch
    rt = torch.as_tensor(r, dtype=torch.float32).cuda().contiguous()
    out = torch.empty_like(rt)
    st = load().sbki_kernel_values(C.c_void_p(rt.data_ptr()), rt.numel(), C.c_void_p(out.data_ptr()), int(method),
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != OK:
        raise SbkiError(st, "sbki_kernel_values failed")
    return out.cpu().numpy()


def _ptr(x):
    """(pointer, keepalive) for a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None, None
    if hasattr(x, "data_ptr"):  # torch tensor
        if not x.is_contiguous():
            x = x.contiguous()
        return C.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x)
    return a.ctypes.data_as(C.c_void_p), a


def _as(x, dtype, shape_tail=None):
    if hasattr(x, "data_ptr"):
        import torch
        tdt = {np.float32: torch.float32, np.int32: torch.int32, np.float64: torch.float64}[dtype]
        if x.dtype != tdt:
            x = x.to(tdt)
        return x.contiguous()
    a = np.ascontiguousarray(x, dtype=dtype)
    if shape_tail is not None:
        a = a.reshape(-1, shape_tail)
    return a


class Map:
    """A semantic S-BKI map on one GPU (owner of its device pool and hash)."""

    def __init__(self, params: Params | None = None, stream=None, **kw):
        L = load()
        # a private copy: keyword overrides and the stream never alter the caller's params
        self.params = Params.from_buffer_copy(params) if params is not None else default_params(**kw)
        if params is not None and kw:
            for k, v in kw.items():
                set_param(self.params, k, v)
        if stream is not None:
            self.params.cuda_stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.K1 = self.params.num_classes + 1
        h = C.c_void_p()
        st = L.sbki_create_map(C.byref(self.params), C.byref(h))
        if st != OK:
            raise SbkiError(st, L.sbki_last_error(None).decode())
        self._h = h
        self._L = L

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._L.sbki_destroy_map(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        if st != OK:
            raise SbkiError(st, self._L.sbki_last_error(self._h).decode())

    # ----------------------------------------------------------- updates
    def insert_scan(self, points, labels, pose, sync=True):
        pts = _as(points, np.float32, 3)
        lab = _as(labels, np.int32)
        T = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
        pp, k1 = _ptr(pts)
        lp, k2 = _ptr(lab)
        n = pts.shape[0] if hasattr(pts, "shape") else len(pts)
        if sync:
            s = Stats()
            self._check(self._L.sbki_insert_scan(self._h, pp, lp, n, T.ctypes.data_as(C.c_void_p), C.byref(s)))
            return s.as_dict()
        self._check(self._L.sbki_insert_scan_async(self._h, pp, lp, n, T.ctypes.data_as(C.c_void_p)))
        self._keep = (k1, k2, T)
        return None

    def sync(self):
        s = Stats()
        self._check(self._L.sbki_sync(self._h, C.byref(s)))
        return s.as_dict()

    def training_set(self, points, labels, pose, cap=None):
        """(xyz float32 [P,3], labels int32 [P]) of a scan (steps a1-a3), host arrays."""
        pts = _as(points, np.float32, 3)
        lab = _as(labels, np.int32)
        T = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
        pp, k1 = _ptr(pts)
        lp, k2 = _ptr(lab)
        n = pts.shape[0]
        cnt = C.c_int64()
        if cap is None:
            cap = int(self.params.sample_capacity)
        out = np.empty((max(cap, 1), 4), np.float32)
        self._check(self._L.sbki_training_set(self._h, pp, lp, n, T.ctypes.data_as(C.c_void_p),
                                              out.ctypes.data_as(C.c_void_p), cap, C.byref(cnt)))
        P = cnt.value
        return out[:P, :3].copy(), out[:P, 3].astype(np.int32)

    def insert_scan_soft(self, points, probs, pose):
        """One scan update with soft labels: probs [n,K] float32 over classes 1..K."""
        pts = _as(points, np.float32, 3)
        n = pts.shape[0]
        pr = _as(probs, np.float32, int(self.params.num_classes))
        T = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
        pp, k1 = _ptr(pts)
        qp, k2 = _ptr(pr)
        s = Stats()
        self._check(self._L.sbki_insert_scan_soft(self._h, pp, qp, n, T.ctypes.data_as(C.c_void_p), C.byref(s)))
        return s.as_dict()

    def training_set_soft(self, points, probs, pose, cap=None):
        """(xyz float32 [P,3], weights float32 [P,K+1]) of a scan with soft labels, host arrays."""
        pts = _as(points, np.float32, 3)
        n = pts.shape[0]
        pr = _as(probs, np.float32, int(self.params.num_classes))
        T = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
        pp, k1 = _ptr(pts)
        qp, k2 = _ptr(pr)
        if cap is None:
            cap = int(self.params.sample_capacity)
        K1 = int(self.params.num_classes) + 1
        xyz = np.empty((max(cap, 1), 3), np.float32)
        w = np.empty((max(cap, 1), K1), np.float32)
        cnt = C.c_int64()
        self._check(self._L.sbki_training_set_soft(self._h, pp, qp, n, T.ctypes.data_as(C.c_void_p),
                                                   xyz.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p),
                                                   cap, C.byref(cnt)))
        P = cnt.value
        return xyz[:P].copy(), w[:P].copy()

    def insert_training(self, xyz, labels):
        """Eq. (alpha_kernel) for a given training set (world xyz, labels 0..K)."""
        if hasattr(xyz, "data_ptr"):
            import torch
            xyzl = torch.cat([xyz.float().reshape(-1, 3), labels.reshape(-1, 1).float()], 1).contiguous()
        else:
            xyzl = np.concatenate([np.asarray(xyz, np.float32).reshape(-1, 3),
                                   np.asarray(labels, np.float32).reshape(-1, 1)], 1)
            xyzl = np.ascontiguousarray(xyzl, np.float32)
        p, keep = _ptr(xyzl)
        s = Stats()
        self._check(self._L.sbki_insert_training(self._h, p, xyzl.shape[0], C.byref(s)))
        return s.as_dict()

    # ----------------------------------------------------------- read-off
    def query(self, xyz, var=True, mode=True, label=True, p_occ=True, state=True):
        """Read-off at world points (host arrays out): dict(probs, var, mode, label, p_occ, state)."""
        x = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
        q = len(x)
        out = dict(probs=np.empty((q, self.K1), np.float32))
        if var:
            out["var"] = np.empty((q, self.K1), np.float32)
        if mode:
            out["mode"] = np.empty((q, self.K1), np.float32)
        if label:
            out["label"] = np.empty(q, np.int32)
        if p_occ:
            out["p_occ"] = np.empty(q, np.float32)
        if state:
            out["state"] = np.empty(q, np.int32)
        g = lambda k: out[k].ctypes.data_as(C.c_void_p) if k in out else None  # noqa: E731
        self._check(self._L.sbki_query_probs(self._h, x.ctypes.data_as(C.c_void_p), q, g("probs"), g("var"),
                                             g("mode"), g("label"), g("p_occ"), g("state")))
        return out

    def query_device(self, xyz, probs, var=None, mode=None, label=None, p_occ=None, state=None):
        """Read-off with caller-owned (e.g. torch CUDA) buffers."""
        ptrs = [_ptr(a) for a in (xyz, probs, var, mode, label, p_occ, state)]
        q = xyz.shape[0]
        self._check(self._L.sbki_query_probs(self._h, *[p for p, _ in ptrs[:1]], q, *[p for p, _ in ptrs[1:]]))

    def profile(self, enable=True, reset=True):
        """Turn per-stage CUDA-event timing on/off (and reset the totals)."""
        self._check(self._L.sbki_profile(self._h, int(enable), int(reset)))

    def profile_read(self):
        d = ProfileData()
        self._check(self._L.sbki_profile_read(self._h, C.byref(d)))
        return d.as_dict()

    def voxel_count(self):
        c = C.c_int64()
        self._check(self._L.sbki_voxel_count(self._h, C.byref(c)))
        return c.value

    # ------------------------------------------------- launch shapes
    def get_tuning(self):
        t = Tuning()
        self._check(self._L.sbki_get_tuning(self._h, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        t = Tuning()
        self._check(self._L.sbki_get_tuning(self._h, C.byref(t)))
        for k, v in kw.items():
            if not hasattr(t, k):
                raise TypeError("unknown tuning field %r" % k)
            setattr(t, k, int(v))
        self._check(self._L.sbki_set_tuning(self._h, C.byref(t)))

    # ------------------------------------------------- several maps, batched updates
    def select(self, map_id):
        """Make map `map_id` of the handle the one single-map calls act on."""
        self._check(self._L.sbki_select_map(self._h, int(map_id)))
        self.active = int(map_id)

    def insert_batch(self, scans):
        """One batched update: scans is a list of dict(points, labels, pose, map_id)
        (numpy arrays or torch tensors); returns the batch's total stats."""
        arr = (Scan * len(scans))()
        keep = []
        for i, sc in enumerate(scans):
            pts = _as(sc["points"], np.float32, 3)
            lab = _as(sc["labels"], np.int32)
            pp, k1 = _ptr(pts)
            lp, k2 = _ptr(lab)
            keep += [pts, lab, k1, k2]
            arr[i].points = pp
            arr[i].labels = lp
            arr[i].n = pts.shape[0]
            T = np.ascontiguousarray(sc["pose"], dtype=np.float64).reshape(16)
            for k in range(16):
                arr[i].pose[k] = float(T[k])
            arr[i].map_id = int(sc.get("map_id", 0))
        s = Stats()
        self._check(self._L.sbki_insert_batch(self._h, arr, len(scans), C.byref(s)))
        return s.as_dict()

    # ------------------------------------------------- differentiable form
    def grad_clear(self):
        """Zero the map's gradient buffer dL/dalpha."""
        self._check(self._L.sbki_grad_clear(self._h))

    def heldout_loglik(self, xyz, labels, grad=False):
        """Held-out log-likelihood of world points with labels 0..K; with grad=True
        dLL/dalpha is added into the map's gradient buffer."""
        x = _as(xyz, np.float32, 3)
        lab = _as(labels, np.int32)
        xp, k1 = _ptr(x)
        lp, k2 = _ptr(lab)
        ll = C.c_double()
        self._check(self._L.sbki_heldout_loglik(self._h, xp, lp, x.shape[0], int(bool(grad)), C.byref(ll)))
        return ll.value

    def grad_add_alpha(self, keys, grad_alpha):
        """Add dL/dalpha given at voxel keys [n,3]; returns the rows no block holds."""
        k = _as_i64(keys, 3)
        gvals = _as(grad_alpha, np.float32, self.K1)
        kp, k1 = _ptr(k)
        gp, k2 = _ptr(gvals)
        missed = C.c_int64()
        self._check(self._L.sbki_grad_add_alpha(self._h, kp, gp, k.shape[0], C.byref(missed)))
        return missed.value

    def backward(self, xyzl, grad_xyz=True):
        """(dL/dl, dL/dsigma0, dL/dxyz [p,3] or None) for the inserted training set
        xyzl [p,4] (x, y, z, label); dL/dxyz is a CUDA tensor when xyzl is one."""
        x = _as(xyzl, np.float32, 4)
        p = x.shape[0]
        xp, keep = _ptr(x)
        gx = None
        if grad_xyz:
            if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
                import torch
                gx = torch.empty((p, 3), dtype=torch.float32, device=x.device)
            else:
                gx = np.empty((max(p, 1), 3), np.float32)
        gxp, keep2 = _ptr(gx)
        gl, gs = C.c_double(), C.c_double()
        self._check(self._L.sbki_backward(self._h, xp, p, C.byref(gl), C.byref(gs), gxp))
        if gx is not None and not hasattr(gx, "data_ptr"):
            gx = gx[:p]
        return gl.value, gs.value, gx

    def backward_scales(self, xyzl):
        """dL/d sigma0_scale[k] for k = 0..K (numpy float64) for the inserted
        training set xyzl [p,4]."""
        x = _as(xyzl, np.float32, 4)
        xp, keep = _ptr(x)
        out = np.zeros(32, np.float64)
        self._check(self._L.sbki_backward_scales(self._h, xp, x.shape[0], out.ctypes.data_as(C.c_void_p)))
        return out[: self.K1].copy()

    def import_(self, keys, alpha):
        """Restore exported contents (keys [n,3], alpha [n,K+1] with prior) into the selected map."""
        k = _as_i64(keys, 3)
        a = _as(alpha, np.float32, self.K1)
        kp, k1 = _ptr(k)
        ap, k2 = _ptr(a)
        self._check(self._L.sbki_import(self._h, kp, ap, k.shape[0]))

    def export_blocks(self, device=None):
        """(keys int64 [n,3], alpha float32 [n,K+1]) of the selected map in pool
        order, computed on the device; CUDA tensors on `device` (a torch device)
        when given, else numpy arrays."""
        cnt = C.c_int64()
        self._check(self._L.sbki_export_blocks(self._h, None, None, 0, C.byref(cnt)))
        n = cnt.value
        if device is not None:
            import torch
            keys = torch.empty((n, 3), dtype=torch.int64, device=device)
            alpha = torch.empty((n, self.K1), dtype=torch.float32, device=device)
        else:
            keys = np.empty((n, 3), np.int64)
            alpha = np.empty((n, self.K1), np.float32)
        if n > 0:
            kp, k1 = _ptr(keys)
            ap, k2 = _ptr(alpha)
            self._check(self._L.sbki_export_blocks(self._h, kp, ap, n, C.byref(cnt)))
        return keys, alpha

    def export(self, pairs=False):
        """(keys int64 [n,3], alpha float32 [n,K+1], pairs int32 [n] or None), sorted by key."""
        n = self.voxel_count()
        keys = np.empty((max(n, 1), 3), np.int64)
        alpha = np.empty((max(n, 1), self.K1), np.float32)
        pc = np.empty(max(n, 1), np.int32) if pairs else None
        cnt = C.c_int64()
        self._check(self._L.sbki_export(self._h, keys.ctypes.data_as(C.c_void_p), alpha.ctypes.data_as(C.c_void_p),
                                        pc.ctypes.data_as(C.c_void_p) if pairs else None, n, C.byref(cnt)))
        n = cnt.value
        return keys[:n], alpha[:n], (pc[:n] if pairs else None)
