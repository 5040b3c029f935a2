"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/sdd.h declares, and rejects invalid arguments before
touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names += re.findall(r"^[A-Za-z_][\w \t\*]*?\b(sdd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1310_3435_gb300 import native
    return native.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("sdd_mesh_plan", "sdd_interface_mc", "sdd_subdomain_solve",
                     "sdd_mesh_generate", "sdd_plan_destroy", "sdd_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    from paper_1310_3435_gb300 import native as N
    d = N.make_density(N.SDD_FAMILY_BUMPS, [1, 5.0, 0.5, 0.5, 50.0, 50.0])
    for (n, sx, sy) in ((2, 1, 1), (33, 0, 2), (33, 2, 33)):
        with pytest.raises(N.SddError) as e:
            N.sdd_mesh_plan(n, sx, sy, d)
        assert e.value.code == N.SDD_ERR_INVALID_ARG
    bad = N.make_density(N.SDD_FAMILY_BUMPS, [7])
    with pytest.raises(N.SddError) as e:
        N.sdd_mesh_plan(33, 2, 2, bad)
    assert e.value.code == N.SDD_ERR_INVALID_ARG
    with pytest.raises(N.SddError) as e:
        N.sdd_mesh_plan(33, 2, 2, N.make_density(9, [1.0] * 5))
    assert e.value.code == N.SDD_ERR_INVALID_ARG
    with pytest.raises(N.SddError) as e:
        N.sdd_mesh_plan(33, 2, 2, d, bmap_mode=7)
    assert e.value.code == N.SDD_ERR_INVALID_ARG
    assert "mode" in N.sdd_last_error()
    assert N.sdd_kernel_launches() >= 0


def test_null_plan_is_rejected(lib):
    from paper_1310_3435_gb300 import native as N
    mc = N.mc_params(100, 1e-4)
    rc = lib.sdd_interface_mc(None, ctypes.byref(mc), None, None, None, None)
    assert rc == N.SDD_ERR_INVALID_ARG
    lib.sdd_plan_destroy(None)          # a no-op
