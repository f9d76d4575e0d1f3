"""CPU-only checks of the C ABI: the library builds, loads without a GPU and
exports exactly the entry points include/sdmd.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(inc, f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for mm in re.finditer(r"SDMD_API\s+[\w\s\*]*?\b(sdmd_\w+)\s*\(", txt):
            names.add(mm.group(1))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_1612_07875_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    d = _declared()
    for name in ("sdmd_create", "sdmd_destroy", "sdmd_push", "sdmd_modes", "sdmd_gram",
                 "sdmd_last_error"):
        assert name in d


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = _declared() - exported
    assert not missing, missing
    extra = {s for s in exported if s.startswith("sdmd_")} - _declared()
    assert not extra, extra


def test_binding_matches_header(built):
    from paper_1612_07875_gb300 import sdmd
    assert set(sdmd.exported_symbols()) == _declared()
    L = sdmd.lib()
    for name in _declared():
        assert hasattr(L, name)


def test_last_error_is_empty_string_before_any_failure(built):
    from paper_1612_07875_gb300 import sdmd
    assert isinstance(sdmd.sdmd_last_error(), str)


def test_argument_errors_need_no_gpu(built):
    from paper_1612_07875_gb300 import sdmd
    with pytest.raises(sdmd.SdmdError) as ei:
        sdmd.sdmd_create(0, 8, sdmd.SDMD_F32)
    assert ei.value.code == sdmd.SDMD_ERR_ARG
    with pytest.raises(sdmd.SdmdError) as ei:
        sdmd.sdmd_create(100, 1, sdmd.SDMD_F32)
    assert ei.value.code == sdmd.SDMD_ERR_ARG
    with pytest.raises(sdmd.SdmdError) as ei:
        sdmd.sdmd_create(100, sdmd.SDMD_MAX_M + 1, sdmd.SDMD_U8)
    assert ei.value.code == sdmd.SDMD_ERR_ARG
    with pytest.raises(sdmd.SdmdError) as ei:
        sdmd.sdmd_create(100, 8, 7)
    assert ei.value.code == sdmd.SDMD_ERR_ARG
    assert "dtype" in sdmd.sdmd_last_error()
    # NULL handles are rejected before any CUDA call
    for fn, args in ((sdmd.sdmd_push, (None, None)), (sdmd.sdmd_count, (None,)),
                     (sdmd.sdmd_modes, (None, 3, None, None))):
        with pytest.raises(sdmd.SdmdError):
            fn(*args)
    sdmd.sdmd_destroy(None)


def test_graft_entry_build_runs(built):
    import __graft_entry__ as g
    g.build()


def test_binding_constants_match_header():
    # every enum value and size limit the header defines (dtypes, statuses,
    # options, reconstruction kinds, trace classes, stream states, maxima)
    # has the same value in the Python binding
    from paper_1612_07875_gb300 import sdmd
    txt = ""
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt += open(os.path.join(inc, f)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(SDMD_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt)}
    consts.update({m.group(1): int(m.group(2))
                   for m in re.finditer(r"#define\s+(SDMD_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", txt)})
    assert len(consts) > 20
    for name, value in consts.items():
        assert getattr(sdmd, name, None) == value, name
