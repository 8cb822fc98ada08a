"""The C ABI library builds, loads and exports every entry point that
include/haru.h declares (no GPU work: nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2211_07340_gb300 as haru


@pytest.fixture(scope="module")
def libpath():
    return haru.build_library()


def test_header_declares_the_boundary():
    syms = haru.declared_symbols()
    for name in ("haru_create", "haru_destroy", "haru_ref_load", "haru_ref_build", "haru_sdtw_batch",
                 "haru_strerror", "haru_config_default", "haru_last_status"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in haru.declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_exports_are_plain_c(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for s in haru.declared_symbols():
        assert s in exported  # unmangled C names


def test_host_only_calls_without_gpu(libpath):
    lib = haru.lib()
    assert lib.haru_strerror(haru.HARU_EINVAL) == b"invalid argument"
    assert lib.haru_strerror(12345) == b"unknown error"
    cfg = haru.default_config()
    assert cfg.tile_cols == 4096 and cfg.serve_prefix == 250
    assert lib.haru_config_default(None) == haru.HARU_EINVAL
    assert lib.haru_create(None, 0, None) == haru.HARU_EINVAL
    # null context is rejected, never dereferenced
    assert lib.haru_sdtw_batch(None, 0, None, None, 0, None, None, 0, 0) == haru.HARU_EINVAL
    assert lib.haru_ref_length(None) == 0
    lib.haru_destroy(None)


def test_header_constants_match_binding():
    txt = open(haru.HEADER).read()
    for name in ("HARU_INT16_QMAX", "HARU_INT16_CAP", "HARU_MAX_QUERY", "HARU_RAW", "HARU_ON_DEVICE"):
        assert f"#define {name} " in txt
    assert haru.HARU_INT16_CAP == 32767 - 2 * haru.HARU_INT16_QMAX
    # every numeric #define the binding re-exports has the header's value
    seen = 0
    for name, val in re.findall(r"^#define (HARU_[A-Z0-9_]+) \(?(-?\d+)u?\)?", txt, re.M):
        if hasattr(haru, name):
            assert getattr(haru, name) == int(val), name
            seen += 1
    assert seen >= 12
    assert (haru.HARU_FP32, haru.HARU_INT16, haru.HARU_INT16_ACC32) == (0, 1, 2)


def _struct_fields(txt, name):
    body = re.search(r"typedef struct \{([^{}]*)\} " + name + ";", txt).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in (d.strip() for d in body.split(";") if d.strip()):
        # "type a" or "type a, b, c": every declarator's name, in order
        names += [re.findall(r"(\w+)\s*(?:\[\d+\])?$", part.strip())[0] for part in decl.split(",")]
    return names


@pytest.mark.parametrize("cname,pyname", [("haru_config", "haru_config"), ("haru_result", "haru_result"),
                                          ("haru_batch_stats", "haru_batch_stats"),
                                          ("haru_stream_stats", "haru_stream_stats")])
def test_struct_layouts_match_header(cname, pyname):
    """The ctypes mirrors list the header's fields in the header's order."""
    txt = open(haru.HEADER).read()
    fields = [f[0] for f in getattr(haru, pyname)._fields_]
    assert fields == _struct_fields(txt, cname)
