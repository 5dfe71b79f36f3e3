"""The C-ABI library builds, loads and exports every entry point of include/dugks.h.

No compute calls are made here (no GPU needed)."""
import os
import re

from paper_2007_07760_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(dugks_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return names


def test_library_exports_every_declared_symbol():
    lib = native.lib()
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    bound = {s[0] for s in native.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_params_struct_layout_matches_header():
    # int32 nx, ny; double W, M, cfl; int32 x5; (pad) double phiA, phiB
    assert native.dugks_params.phiB.offset + 8 == __import__("ctypes").sizeof(native.dugks_params)
    assert native.dugks_params.W.offset == 8 and native.dugks_params.order.offset == 32


def test_allocation_hook_arguments():
    # host-only entry point: argument checks, arming and disarming
    assert native.dugks_selftest_fail_allocs(-1, 1) == native.DUGKS_EINVAL
    assert native.dugks_selftest_fail_allocs(0, -1) == native.DUGKS_EINVAL
    assert native.dugks_selftest_fail_allocs(3, 1) == native.DUGKS_OK
    assert native.dugks_selftest_fail_allocs(0, 0) == native.DUGKS_OK
