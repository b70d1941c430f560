"""C-ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every symbol include/synax.h declares, its struct layout matches the
Python binding, and host-side validation rejects malformed problems before
anything is enqueued (no CUDA call is made on these paths)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2410_01136_gb300 import _native, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def L():
    from paper_2410_01136_gb300 import build
    build()
    return _native.lib()


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(synax_\w+)\s*\(", text)
    return sorted(set(names))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "synax_forward" in names and "synax_adjoint" in names
    for n in names:
        assert hasattr(L, n), f"libsynax does not export {n}"
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n
    # and the binding declares a signature for every one of them
    for n in names:
        assert n in _native.SIGNATURES, n


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    fields = [f for f, _ in _native.SynaxProblem._fields_]
    body = "\n".join(f'printf("{f} %zu\\n", offsetof(synax_problem, {f}));' for f in fields)
    src.write_text(f"""#include <stdio.h>
#include <stddef.h>
#include "synax.h"
int main(void) {{ printf("size %zu\\n", sizeof(synax_problem)); {body} return 0; }}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    assert int(got["size"]) == ctypes.sizeof(_native.SynaxProblem)
    for f in fields:
        assert int(got[f]) == getattr(_native.SynaxProblem, f).offset, f


def call_forward(L, prob_struct):
    # maps pointer is a dummy non-NULL value: validation fails before any use.
    return L.synax_forward(ctypes.byref(prob_struct), ctypes.c_void_p(16), None)


def good():
    return inputs.config2().replace(nside=4, n_steps=64)


@pytest.mark.parametrize("mutate,code", [
    (lambda s: setattr(s, "nside", 3), _native.SYNAX_EINVAL),
    (lambda s: setattr(s, "nside", 0), _native.SYNAX_EINVAL),
    (lambda s: setattr(s, "nside", 16384), _native.SYNAX_EINVAL),
    (lambda s: setattr(s, "n_steps", 0), _native.SYNAX_EINVAL),
    (lambda s: setattr(s, "n_steps", 65537), _native.SYNAX_EINVAL),
    (lambda s: setattr(s, "n_freq", 0), _native.SYNAX_EINVAL),
    (lambda s: setattr(s, "n_freq", 17), _native.SYNAX_EINVAL),
    (lambda s: setattr(s, "model_id", 7), _native.SYNAX_EINVAL),
    (lambda s: setattr(s, "n_theta", 15), _native.SYNAX_EINVAL),
    (lambda s: s.theta.__setitem__(3, float("nan")), _native.SYNAX_ENONFINITE),
    (lambda s: s.freq_hz.__setitem__(0, float("inf")), _native.SYNAX_ENONFINITE),
    (lambda s: s.freq_hz.__setitem__(1, -1.0), _native.SYNAX_EINVAL),
    (lambda s: s.obs_kpc.__setitem__(2, float("nan")), _native.SYNAX_ENONFINITE),
    (lambda s: setattr(s, "r_max_kpc", 0.0), _native.SYNAX_EINVAL),
    (lambda s: setattr(s, "flags", 1 << 7), _native.SYNAX_EINVAL),
    (lambda s: setattr(s, "rm_rule", 3), _native.SYNAX_EINVAL),
    (lambda s: s.theta.__setitem__(13, 0.2), _native.SYNAX_EINVAL),     # p too small for Eq. 2
    (lambda s: s.theta.__setitem__(9, 0.0), _native.SYNAX_EINVAL),      # z_h
    (lambda s: s.theta.__setitem__(11, 1.6), _native.SYNAX_EINVAL),     # theta_X >= pi/2
    (lambda s: setattr(s, "pix_begin", -1), _native.SYNAX_EINVAL),
    (lambda s: setattr(s, "pix_begin", 193), _native.SYNAX_EINVAL),
    (lambda s: (setattr(s, "pix_begin", 100), setattr(s, "pix_count", 93)), _native.SYNAX_EINVAL),
    (lambda s: (setattr(s, "flags", _native.SYNAX_BOX_CLIP), s.box_kpc.__setitem__(2, 0.01)),
     _native.SYNAX_EINVAL),   # observer outside the box
])
def test_validation_rejects(L, mutate, code):
    s = _native.problem_struct(good())
    mutate(s)
    assert call_forward(L, s) == code
    assert L.synax_strerror(code)


def test_empty_range_and_null(L):
    s = _native.problem_struct(good())
    s.pix_begin = 192          # empty pixel range: nothing to do, no launch
    assert L.synax_forward(ctypes.byref(s), None, None) == _native.SYNAX_OK
    assert L.synax_forward(None, ctypes.c_void_p(16), None) == _native.SYNAX_EINVAL
    s = _native.problem_struct(good())
    assert L.synax_forward(ctypes.byref(s), None, None) == _native.SYNAX_EINVAL


def test_adjoint_validation(L):
    s = _native.problem_struct(good())
    n = ctypes.c_size_t(0)
    assert L.synax_adjoint_workspace_bytes(ctypes.byref(s), ctypes.byref(n)) == _native.SYNAX_OK
    dummy = ctypes.c_void_p(16)
    # chi^2 mode without target / with bad sigma
    assert L.synax_adjoint(ctypes.byref(s), None, None, 1.0, dummy, None, None, dummy,
                           n.value, None) == _native.SYNAX_EINVAL
    assert L.synax_adjoint(ctypes.byref(s), None, dummy, float("nan"), dummy, None, None, dummy,
                           n.value, None) == _native.SYNAX_ENONFINITE
    assert L.synax_adjoint(ctypes.byref(s), None, dummy, -1.0, dummy, None, None, dummy,
                           n.value, None) == _native.SYNAX_EINVAL
    # no gradient buffer
    assert L.synax_adjoint(ctypes.byref(s), dummy, None, 1.0, None, None, None, dummy,
                           n.value, None) == _native.SYNAX_EINVAL
    if n.value > 0:
        assert L.synax_adjoint(ctypes.byref(s), dummy, None, 1.0, dummy, None, None, dummy,
                               n.value - 1, None) == _native.SYNAX_ESPACE
    toy = _native.problem_struct(inputs.toy_problem(nside=2, n_steps=8))
    assert L.synax_adjoint(ctypes.byref(toy), dummy, None, 1.0, dummy, None, None, dummy,
                           1 << 30, None) == _native.SYNAX_ENOTSUP


def _grid_struct():
    """A grid-model problem struct with a dummy (never dereferenced) grid pointer."""
    s = _native.problem_struct(inputs.config2().replace(nside=4, n_steps=64, box_clip=True))
    s.model_id = inputs.MODEL_GRID
    s.n_theta = 3
    for k, v in enumerate(inputs.grid_theta()):
        s.theta[k] = v
    s.grid_dev = 16
    s.grid_n[0], s.grid_n[1], s.grid_n[2] = 4, 4, 2
    return s


@pytest.mark.parametrize("mutate", [
    lambda s: setattr(s, "flags", 0),                          # the grid needs rays that end at the box
    lambda s: setattr(s, "grid_dev", None),
    lambda s: s.grid_n.__setitem__(0, 1),
    lambda s: s.grid_n.__setitem__(2, 0),
    lambda s: (s.grid_n.__setitem__(0, 2048), s.grid_n.__setitem__(1, 2048), s.grid_n.__setitem__(2, 256)),
    lambda s: setattr(s, "reserved", 1),
    lambda s: setattr(s, "n_theta", 8),
    lambda s: s.theta.__setitem__(1, 0.2),                     # p
])
def test_grid_validation_rejects(L, mutate):
    s = _grid_struct()
    s.pix_begin = 192                                          # valid problems do nothing
    assert L.synax_forward(ctypes.byref(s), None, None) == _native.SYNAX_OK
    mutate(s)
    assert L.synax_forward(ctypes.byref(s), ctypes.c_void_p(16), None) == _native.SYNAX_EINVAL


def test_wmap_stack_validation(L):
    s = _native.problem_struct(inputs.wmap_stack_problem(nside=4, n_steps=16))
    s.pix_begin = 192
    assert L.synax_forward(ctypes.byref(s), None, None) == _native.SYNAX_OK
    bad = _native.problem_struct(inputs.wmap_stack_problem(nside=4, n_steps=16))
    bad.n_theta = 18
    assert L.synax_forward(ctypes.byref(bad), ctypes.c_void_p(16), None) == _native.SYNAX_EINVAL
    bad = _native.problem_struct(inputs.wmap_stack_problem(nside=4, n_steps=16))
    bad.theta[17] = 0.2                                  # p below Eq. 2's range
    assert L.synax_forward(ctypes.byref(bad), ctypes.c_void_p(16), None) == _native.SYNAX_EINVAL


def test_adjoint_grid_workspace_query(L):
    g = _grid_struct()
    n = ctypes.c_size_t(0)
    assert L.synax_adjoint_grid_workspace_bytes(ctypes.byref(g), ctypes.byref(n)) == _native.SYNAX_OK
    theta_only = ctypes.c_size_t(0)
    assert L.synax_adjoint_workspace_bytes(ctypes.byref(g), ctypes.byref(theta_only)) == _native.SYNAX_OK
    assert n.value >= theta_only.value + 16 * 4 * 4 * 2          # FP32: a float4 per node
    s = _native.problem_struct(good())
    assert L.synax_adjoint_grid_workspace_bytes(ctypes.byref(s), ctypes.byref(n)) == _native.SYNAX_ENOTSUP
    dummy = ctypes.c_void_p(16)
    g.pix_begin = 0
    need = ctypes.c_size_t(0)
    L.synax_adjoint_grid_workspace_bytes(ctypes.byref(g), ctypes.byref(need))
    assert L.synax_adjoint_grid(ctypes.byref(g), dummy, None, 1.0, dummy, None, None, dummy, dummy,
                                need.value - 1, None) == _native.SYNAX_ESPACE


def test_adjoint_grid_validation(L):
    dummy = ctypes.c_void_p(16)
    s = _native.problem_struct(good())
    assert L.synax_adjoint_grid(ctypes.byref(s), dummy, None, 1.0, dummy, None, None, dummy, dummy,
                                1 << 30, None) == _native.SYNAX_ENOTSUP
    g = _grid_struct()
    assert L.synax_adjoint_grid(ctypes.byref(g), dummy, None, 1.0, dummy, None, None, None, dummy,
                                1 << 30, None) == _native.SYNAX_EINVAL
    g.reserved = 2
    assert L.synax_adjoint_grid(ctypes.byref(g), dummy, None, 1.0, dummy, None, None, dummy, dummy,
                                1 << 30, None) == _native.SYNAX_EINVAL
    assert L.synax_adjoint_grid(None, dummy, None, 1.0, dummy, None, None, dummy, dummy,
                                1 << 30, None) == _native.SYNAX_EINVAL


def test_version_and_strerror(L):
    assert L.synax_version() >= 100
    for code in range(-7, 1):
        assert isinstance(L.synax_strerror(code), bytes)


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "LIB_PATH", "/nonexistent/libsynax.so")
    with pytest.raises(RuntimeError, match="not built"):
        _native.lib()


def test_problem_struct_roundtrip():
    p = inputs.config2().replace(pix_begin=5, pix_count=7, rm_rule=2, f64=True)
    s = _native.problem_struct(p)
    assert s.nside == 64 and s.n_steps == 512 and s.n_freq == 4 and s.n_theta == 16
    assert s.flags == _native.SYNAX_F64 and s.rm_rule == 2 and s.pix_begin == 5 and s.pix_count == 7
    assert np.allclose(list(s.theta)[:16], p.theta)


def test_build_function_not_shadowed_by_submodule():
    import paper_2410_01136_gb300 as pkg
    pkg.build()
    from paper_2410_01136_gb300 import build
    assert callable(build)


def test_batch_plan_validation_on_host(L):
    """Plan validation happens before any CUDA call."""
    a = _native.problem_struct(good())
    arr = (_native.SynaxProblem * 2)(a, a)
    h = ctypes.c_void_p()
    assert L.synax_batch_plan_create(arr, 0, ctypes.byref(h)) == _native.SYNAX_EINVAL
    assert L.synax_batch_plan_create(None, 2, ctypes.byref(h)) == _native.SYNAX_EINVAL
    b = _native.problem_struct(good().replace(freq_hz=(1e9,)))
    arr2 = (_native.SynaxProblem * 2)(a, b)
    assert L.synax_batch_plan_create(arr2, 2, ctypes.byref(h)) == _native.SYNAX_EINVAL
    c = _native.problem_struct(good().replace(f64=True))
    arr3 = (_native.SynaxProblem * 1)(c)
    assert L.synax_batch_plan_create(arr3, 1, ctypes.byref(h)) == _native.SYNAX_ENOTSUP
    bad = _native.problem_struct(good())
    bad.nside = 3
    arr4 = (_native.SynaxProblem * 1)(bad)
    assert L.synax_batch_plan_create(arr4, 1, ctypes.byref(h)) == _native.SYNAX_EINVAL
    assert L.synax_batch_run(None, None, None, 0, 1.0, None, None, None, None) == _native.SYNAX_EINVAL


def test_set_lanes_per_ray_validation(L):
    assert L.synax_set_lanes_per_ray(-1, 12) == _native.SYNAX_EINVAL
    assert L.synax_set_lanes_per_ray(512, 7) == _native.SYNAX_EINVAL
    for lanes in (8, 16, 32, 0):
        assert L.synax_set_lanes_per_ray(512, lanes) == _native.SYNAX_OK
    assert L.synax_set_lanes_per_ray(-1, 0) == _native.SYNAX_OK


def test_wait_selftest_rejects_null(L):
    assert L.synax_wait_selftest(None, ctypes.c_void_p(16), None) == _native.SYNAX_EINVAL
    assert L.synax_wait_selftest(ctypes.c_void_p(16), None, None) == _native.SYNAX_EINVAL


def test_every_entry_point_is_documented():
    """Each function the header declares sits under a comment block (its
    passage, arguments, layout, ownership and errors)."""
    import re
    lines = open(os.path.join(ROOT, "include", "synax.h")).read().split("\n")
    decl = re.compile(r"^(?:int|void|size_t|int64_t|double|const char\*)\s+\**(synax_\w+)\s*\(")
    undocumented = []
    for i, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        j = i - 1
        # step over the other declarations of the same block and continuation lines
        while j >= 0 and (decl.match(lines[j]) or lines[j].startswith("typedef")
                          or (lines[j].startswith(" ") and not lines[j].lstrip().startswith(("*", "/*")))):
            j -= 1
        if j < 0 or not lines[j].rstrip().endswith("*/"):
            undocumented.append(m.group(1))
    assert not undocumented, undocumented


def test_checked_mode_host_side(L):
    """SYNAX_CHECKED: the bounds predicate the kernels use classifies indexes
    on both sides of an extent correctly (run on the host), and the flag
    passes host validation while an unknown flag bit does not."""
    assert L.synax_checked_selftest() == _native.SYNAX_OK
    prob = inputs.config2().replace(nside=4, n_steps=16, checked=True)
    s = _native.problem_struct(prob)
    assert s.flags & _native.SYNAX_CHECKED
    n = ctypes.c_size_t(0)
    assert L.synax_adjoint_workspace_bytes(ctypes.byref(s), ctypes.byref(n)) == _native.SYNAX_OK
    s.flags |= 1 << 3
    assert L.synax_adjoint_workspace_bytes(ctypes.byref(s), ctypes.byref(n)) == _native.SYNAX_EINVAL
    assert L.synax_strerror(_native.SYNAX_EBOUNDS).decode().startswith("device-side index check")


def test_last_status_detail_without_a_read(L):
    """Before any synax_last_status call on this thread the detail is zero."""
    site, index = ctypes.c_int(-1), ctypes.c_longlong(-1)
    assert L.synax_last_status_detail(ctypes.byref(site), ctypes.byref(index)) == _native.SYNAX_OK
    assert (site.value, index.value) == (0, 0)
    assert L.synax_last_status_detail(None, None) == _native.SYNAX_OK
