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


def header_struct_fields(name):
    """(field, bytes) of `typedef struct { ... } name;` in include/kad.h, in order."""
    src = open(os.path.join(ROOT, "include", "kad.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src).group(1)
    scalar = {"int32_t": 4, "uint32_t": 4, "int64_t": 8, "uint64_t": 8, "double": 8}
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, rest = decl.split(None, 1)
        for item in rest.split(","):
            item = item.strip()
            m = re.fullmatch(r"(\*?)\s*(\w+)(?:\[(\d+)\])?", item)
            assert m, item
            size = 8 if m.group(1) else scalar[ctype]
            out.append((m.group(2), size * int(m.group(3) or 1)))
    return out


@pytest.mark.parametrize("cname,pyname", [("kad_options", "Options"), ("kad_result", "Result"),
                                          ("kad_server_options", "ServerOptions")])
def test_binding_structs_match_the_header(cname, pyname):
    from paper_1903_09422_gb300 import kad
    cls = getattr(kad, pyname)
    py = [(f[0], ctypes.sizeof(f[1])) for f in cls._fields_]
    assert py == header_struct_fields(cname)


def test_pair_cost_defaults_to_the_library_choice(lib):
    from paper_1903_09422_gb300 import kad
    assert kad.options().pair_cost == 0
    assert kad.options(pair_cost=64).pair_cost == 64
