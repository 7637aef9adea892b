"""The C ABI library loads and exports every entry point include/kad.h declares
(no GPU needed: nothing here calls into the device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "kad.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(kad_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1903_09422_gb300 import build
    build.build()
    from paper_1903_09422_gb300 import kad
    return kad.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("kad_graph_create", "kad_run", "kad_graph_free", "kad_status_string"):
        assert must in names
    assert len(names) >= 10


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in kad.h but not exported"


def test_binding_covers_the_header():
    from paper_1903_09422_gb300 import kad
    assert set(kad.EXPORTS) <= set(declared_functions())


def test_host_only_entry_points(lib):
    from paper_1903_09422_gb300 import kad
    assert kad.status_string(0) == "ok"
    assert "symmetric" in kad.status_string(2)
    assert kad.version() >= (0, 1)
    o = kad.options()
    assert o.epoch_size == 1000 and o.calib_div == 100 and o.mcap == -1


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    from paper_1903_09422_gb300 import kad
    h = ctypes.c_void_p()
    # n < 2 and NULL arrays are refused on the host
    assert lib.kad_graph_create(1, None, None, 0, None, ctypes.byref(h)) == 1
    assert lib.kad_run(None, 0.1, 0.1, 1, None, None, None) == 1
    assert lib.kad_run_order(None, None, 0) == 1
    lib.kad_graph_free(None)
