"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/ddgi.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in ("ddgi.h",):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(ddgi_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_10796_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2009_10796_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(declared_functions())


def test_binding_array_lengths_match_header():
    """Fixed-length array parameters (`float ms[8]`) have ctypes arrays of
    the same length, in the same position."""
    import ctypes as C
    from paper_2009_10796_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "ddgi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    checked = 0
    for name, params in re.findall(r"\b(ddgi_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
        if name not in _lib.SIGNATURES:
            continue
        argtypes = _lib.SIGNATURES[name][1]
        for k, prm in enumerate(p.strip() for p in params.split(",")):
            m = re.search(r"\[(\d+)\]\s*$", prm)
            if not m:
                continue
            t = argtypes[k]
            assert issubclass(t, C.Array) and t._length_ == int(m.group(1)), (name, k, prm, t)
            checked += 1
    assert checked >= 4


def test_version_and_error_without_gpu(lib):
    import paper_2009_10796_gb300 as g
    L = g.load()
    assert L.ddgi_version() >= 1
    # a host-side argument error needs no device
    import ctypes as C
    out = C.c_void_p()
    assert L.ddgi_volume_create(None, C.byref(out)) == 1
    assert b"NULL" in L.ddgi_last_error()


def test_texel_bytes_without_gpu(lib):
    import paper_2009_10796_gb300 as g
    L = g.load()
    assert [L.ddgi_texel_bytes(0, f) for f in (g.IRR_FP32, g.IRR_FP16, g.IRR_RGB9E5)] == [16, 8, 4]
    assert [L.ddgi_texel_bytes(1, f) for f in (g.DIST_FP32, g.DIST_FP16)] == [8, 4]
    assert L.ddgi_texel_bytes(0, 7) == 0 and L.ddgi_texel_bytes(2, 0) == 0


def test_struct_layouts_match_header(tmp_path):
    """ctypes structs mirror the C structs: compare with what gcc lays out."""
    import ctypes as C
    import subprocess
    from paper_2009_10796_gb300 import _lib
    structs = {"ddgi_lights": _lib.Lights, "ddgi_volume_desc": _lib.VolumeDesc,
               "ddgi_volume_info": _lib.VolumeInfo, "ddgi_update_params": _lib.UpdateParams}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ddgi.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_descriptor_limits_without_gpu(lib):
    """Descriptor checks run before any device call: the ray lists index
    rays with 32-bit ints (probes x rays below 2^31), converge batches and
    optimizer iterations have ranges."""
    import ctypes as C
    import paper_2009_10796_gb300 as g
    import synth
    from paper_2009_10796_gb300 import api
    L = g.load()
    out = C.c_void_p()
    for kw, msg in [(dict(counts=(2048, 1024, 32), rays_per_probe=64), b"2^31"),
                    (dict(converge_batches=65), b"converge_batches"),
                    (dict(optimizer_iters=17), b"optimizer_iters")]:
        d = api.desc_struct(synth.room_volume(**kw))
        assert L.ddgi_volume_create(C.byref(d), C.byref(out)) == 1
        assert msg in L.ddgi_last_error(), (kw, L.ddgi_last_error())
