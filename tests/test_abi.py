"""The C-ABI library builds, loads without a GPU and exports every symbol the
header declares; argument checks that need no device work on CPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "inim.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2604_13880_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2604_13880_gb300 import build
        build.build()
    return _lib.load()


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(inim_\w+)\s*\(", txt, re.M)))


def test_header_symbols_exported(lib):
    from paper_2604_13880_gb300 import _lib
    names = declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(_lib.declared_symbols())


def test_struct_layout_matches_header(tmp_path):
    # compile a C program against the header and compare sizes/offsets with ctypes
    from paper_2604_13880_gb300 import _lib
    src = tmp_path / "t.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "inim.h"\n'
                   'int main(){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(inim_params), sizeof(inim_step_stats),'
                   ' sizeof(inim_job), offsetof(inim_job, params), offsetof(inim_params, form),'
                   ' offsetof(inim_params, bdv_value));'
                   'printf("%zu %zu %zu %zu\\n", sizeof(inim_quality_out), offsetof(inim_quality_out, n_present),'
                   ' sizeof(inim_series), offsetof(inim_series, stats));return 0;}\n')
    exe = tmp_path / "t"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = list(map(int, subprocess.check_output([str(exe)]).split()))
    want = [ctypes.sizeof(_lib.inim_params), ctypes.sizeof(_lib.inim_step_stats), ctypes.sizeof(_lib.inim_job),
            _lib.inim_job.params.offset, _lib.inim_params.form.offset, _lib.inim_params.bdv_value.offset,
            ctypes.sizeof(_lib.inim_quality_out), _lib.inim_quality_out.n_present.offset,
            ctypes.sizeof(_lib.inim_series), _lib.inim_series.stats.offset]
    assert got == want


def test_defaults_and_status(lib):
    import paper_2604_13880_gb300 as P
    p = P.params()
    assert (p.log2_res, p.max_iters, p.stall_window) == (10, 512, 32)
    assert abs(p.xi_stop - 0.01) < 1e-9 and p.bdv_scale == 1.0
    assert P.inim_status_string(0) == "ok"
    assert "capacity" in P.inim_status_string(-5)


def test_map_argument_checks(lib):
    # these fail before any device work
    xy = np.zeros((3, 2), np.float32)
    off = np.array([0, 3], np.int32)
    reg = np.zeros(1, np.int32)
    h = ctypes.c_void_p()
    bad_idx = np.array([0, 1, 7], np.int32)
    assert lib.inim_map_create(xy.ctypes.data, 3, off.ctypes.data, 1, bad_idx.ctypes.data, reg.ctypes.data,
                               1, 0, ctypes.byref(h)) == -1
    idx = np.array([0, 1, 2], np.int32)
    assert lib.inim_map_create(xy.ctypes.data, 3, off.ctypes.data, 1, idx.ctypes.data, reg.ctypes.data,
                               0, 0, ctypes.byref(h)) == -1
    bad_reg = np.array([4], np.int32)
    assert lib.inim_map_create(xy.ctypes.data, 3, off.ctypes.data, 1, idx.ctypes.data, bad_reg.ctypes.data,
                               2, 0, ctypes.byref(h)) == -1
    nan = np.full((3, 2), np.nan, np.float32)
    assert lib.inim_map_create(nan.ctypes.data, 3, off.ctypes.data, 1, idx.ctypes.data, reg.ctypes.data,
                               1, 0, ctypes.byref(h)) == -1
    assert b"range" in lib.inim_last_error() or b"coordinates" in lib.inim_last_error()


def test_background_values_match_the_oracle(lib):
    # Eq. (Mb) is host arithmetic in the library: checked against the oracle
    import paper_2604_13880_gb300 as P
    from oracle import inim_oracle as O
    vals = np.random.default_rng(21).lognormal(0.0, 1.0, (11, 17)).astype(np.float32)
    for a_min, a_max, t0, t1 in [(0.2, 0.9, 0, None), (0.35, 0.6, 3, 7), (0.1, 0.15, 5, 5)]:
        got, frac = P.inim_background_values(vals, 10, a_min, a_max, t0, -1 if t1 is None else t1)
        want, _, a_i = O.background_values(vals.astype(np.float64), 10, a_min, a_max, t0, t1)
        np.testing.assert_allclose(got, want, rtol=1e-12)
        np.testing.assert_allclose(frac, a_i, rtol=1e-14)
    # a constant global integral puts every step at a_max (library and oracle)
    const = np.ones((4, 5), np.float32)
    got, frac = P.inim_background_values(const, 9, 0.3, 0.8)
    want, _, a_i = O.background_values(const.astype(np.float64), 9, 0.3, 0.8)
    np.testing.assert_allclose(frac, [0.8] * 4, rtol=1e-15)
    np.testing.assert_allclose(got, want, rtol=1e-12)
    with pytest.raises(P.InimError):
        P.inim_background_values(vals, 10, 0.6, 0.4)
    with pytest.raises(P.InimError):
        P.inim_background_values(vals, 10, 0.2, 0.9, 6, 2)
    bad = vals.copy()
    bad[2, 3] = -1.0
    with pytest.raises(P.InimError):
        P.inim_background_values(bad, 10, 0.2, 0.9)


def test_interpolated_frames_match_the_oracle(lib):
    # the frame values of Sec. 5.5 are host arithmetic in the library
    import paper_2604_13880_gb300 as P
    from oracle import inim_oracle as O
    vals = np.random.default_rng(22).lognormal(0.0, 1.0, (5, 13)).astype(np.float32)
    for f in (1, 4, 10):
        got = P.inim_interpolate_values(vals, f)
        want = O.interpolate_series(vals.astype(np.float64), f).astype(np.float32)
        assert got.shape == ((5 - 1) * f + 1, 13)
        np.testing.assert_array_equal(got, want)
        np.testing.assert_array_equal(got[::f], vals)        # every f-th frame is a time step
    assert P.inim_interpolate_values(vals[:1], 10).shape == (1, 13)
    with pytest.raises(P.InimError):
        P.inim_interpolate_values(vals, 0)


def test_quality_argument_checks(lib):
    # rejected before any device work
    from paper_2604_13880_gb300 import _lib
    out = _lib.inim_quality_out()
    xy = np.zeros((3, 2), np.float32)
    assert lib.inim_quality(None, None, xy.ctypes.data, 8, ctypes.byref(out), None, None) == -1
    assert b"NULL" in lib.inim_last_error()


def test_run_dynamic_argument_checks(lib):
    import paper_2604_13880_gb300 as P
    p = P.params(log2_res=8)
    vals = np.ones((2, 3), np.float32)
    out = np.empty((2, 4, 2), np.float32)
    assert lib.inim_run_dynamic(None, vals.ctypes.data, 2, ctypes.byref(p), 0.2, 0.8, 0, -1, None,
                                out.ctypes.data, None, None) == -1
    assert b"inim_run_dynamic" in lib.inim_last_error()
