"""The C-ABI library loads and exports every symbol include/sbki.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sbki.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sbki_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("sbki_create_map", "sbki_insert_scan", "sbki_query_probs", "sbki_export", "sbki_destroy_map"):
        assert f in names


def test_library_exports_every_declared_symbol():
    from paper_1909_04631_gb300 import build, sbki
    if not os.path.exists(build.LIB):
        try:
            build.build()
        except RuntimeError as e:  # no nvcc on this machine
            pytest.skip(str(e))
    lib = ctypes.CDLL(build.LIB)
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(sbki.EXPORTED) == _declared()


def test_status_strings_without_gpu():
    from paper_1909_04631_gb300 import sbki
    L = sbki.load()
    for code, text in sbki.STATUS_NAMES.items():
        assert L.sbki_status_string(code).decode() == text


def test_params_struct_matches_header_defaults():
    from paper_1909_04631_gb300 import sbki
    p = sbki.default_params()
    assert (p.length_scale, p.sigma0, p.alpha0, p.res, p.free_thresh, p.occ_thresh) == (0.3, 0.1, 0.001, 0.1, 0.47,
                                                                                      0.6)
    assert p.accumulate_mode == 0 and p.track_pairs == 0


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Offsets and sizes of the ctypes structures equal those gcc gives the header's structs."""
    from paper_1909_04631_gb300 import sbki
    structs = {"sbki_params": sbki.Params, "sbki_stats": sbki.Stats, "sbki_profile_data": sbki.ProfileData,
               "sbki_scan": sbki.Scan, "sbki_tuning": sbki.Tuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sbki.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().split("\n") if l)
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(py, f).offset, (cname, f)


def test_create_map_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1909_04631_gb300 import sbki
    with pytest.raises(sbki.SbkiError):
        sbki.Map(sbki.default_params())


def test_create_map_rejects_bad_params():
    from paper_1909_04631_gb300 import sbki
    for bad in (dict(res=0.0), dict(block_edge=6), dict(num_classes=40), dict(max_range=float("inf")),
                dict(length_scale=5.0), dict(alpha0=0.0), dict(sensor_model=2),
                dict(sensor_model=1, accumulate_mode=1), dict(sigma0_scale=[1.0, 0.0]),
                dict(sigma0_scale=[1.0, float("nan")])):
        with pytest.raises(sbki.SbkiError) as e:
            sbki.Map(sbki.default_params(**bad))
        assert e.value.status == sbki.ERR_INVALID_ARG


def test_set_param_fills_class_arrays_and_rejects_unknown_names():
    from paper_1909_04631_gb300 import sbki
    p = sbki.Params()
    for k in range(32):
        p.sigma0_scale[k] = 1.0
    sbki.set_param(p, "sigma0_scale", [0.5, 2.0])
    assert list(p.sigma0_scale[:3]) == [0.5, 2.0, 1.0]
    sbki.set_param(p, "num_classes", 7)
    assert p.num_classes == 7
    with pytest.raises(TypeError):
        sbki.set_param(p, "no_such_field", 1)
    with pytest.raises(ValueError):
        sbki.set_param(p, "sigma0_scale", [1.0] * 33)


class _FakeTensor:
    """Stands in for a CUDA tensor (dtype, shape, device, layout only) so the
    binding's argument checks run without a GPU."""

    def __init__(self, shape, dtype, device=0, cuda=True, contiguous=True):
        import types
        self.shape, self.dtype, self.is_cuda, self._contig = tuple(shape), dtype, cuda, contiguous
        self.device = types.SimpleNamespace(index=device)

    def dim(self):
        return len(self.shape)

    def is_contiguous(self):
        return self._contig


def test_noalloc_binding_refuses_malformed_arguments():
    """Each argument the allocation-free entry point would misread (wrong
    dtype, shape, device or layout) is refused before the library is called."""
    import torch
    from paper_1909_04631_gb300 import sbki
    p = sbki.Params()
    p.device = 0
    F = _FakeTensor
    good = dict(points=F((10, 3), torch.float32), labels=F((10,), torch.int32), out=F((64, 4), torch.float32))
    sbki.check_noalloc_args(p, **good)
    bad = [
        (TypeError, dict(points=F((10, 3), torch.float64))),
        (TypeError, dict(labels=F((10,), torch.int64))),
        (TypeError, dict(out=F((64, 4), torch.float16))),
        (TypeError, dict(out=F((64, 4), torch.float32, cuda=False))),
        (TypeError, dict(labels=F((10,), torch.int32, device=1))),
        (TypeError, dict(points=F((10, 3), torch.float32, contiguous=False))),
        (ValueError, dict(points=F((10, 4), torch.float32))),
        (ValueError, dict(points=F((30,), torch.float32), labels=F((30,), torch.int32))),
        (ValueError, dict(labels=F((9,), torch.int32))),
        (ValueError, dict(out=F((256,), torch.float32))),
        (ValueError, dict(out=F((64, 3), torch.float32))),
    ]
    for err, change in bad:
        args = dict(good, **change)
        with pytest.raises(err):
            sbki.check_noalloc_args(p, **args)
        with pytest.raises(err):  # the public call checks before it reaches the library
            sbki.training_set_noalloc(p, args["points"], args["labels"], np.eye(4), args["out"])
