"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/gld.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_1808_00270_gb300 import binding
from paper_1808_00270_gb300 import build as B

HEADER = os.path.join(B.ROOT, "include", "gld.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(gld_[a-z0-9_]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gld_create", "gld_set_kernels", "gld_step", "gld_vacf", "gld_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_matches_header():
    assert set(binding.exported_symbols()) == set(declared_functions())


def test_params_struct_layout_matches_header():
    # the ctypes mirror must list the fields of gld_params in header order
    text = open(HEADER).read()
    body = text[text.index("typedef struct gld_params {"): text.index("} gld_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b([a-zA-Z_0-9]+)\s*[,;]", body)
    assert [f for f, _ in binding.Params._fields_] == fields


def _fields(name):
    text = open(HEADER).read()
    end = text.index("} %s;" % name)
    body = text[text.rindex("typedef struct", 0, end): end]
    body = body[body.index("{") + 1:]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return re.findall(r"\b([a-zA-Z_0-9]+)\s*[,;]", body)


def test_server_struct_layouts_match_header():
    assert [f for f, _ in binding.Request._fields_] == _fields("gld_request")
    assert [f for f, _ in binding.ServerParams._fields_] == _fields("gld_server_params")
    assert len(binding.SRV_STATS) == 11  # GLD_SRV_N


def test_profile_families_match_header():
    text = open(HEADER).read()
    n = int(re.search(r"GLD_PROF_N\s*=\s*(\d+)", text).group(1))
    assert len(binding.GLD.PROF_NAMES) == n
