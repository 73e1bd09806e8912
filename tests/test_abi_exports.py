"""The C-ABI library builds, loads without a GPU and exports every entry
point include/*.h declares (no compute calls here)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(pm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import paper_2603_01122_gb300 as pm
    pm.build()
    return pm.library()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("pm_update_posterior", "pm_predict_occupancy", "pm_create", "pm_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_uses_the_c_names(lib):
    import paper_2603_01122_gb300 as pm
    for n in declared_functions():
        assert hasattr(pm, n), f"binding has no {n}"


def test_version_string(lib):
    import paper_2603_01122_gb300 as pm
    assert "sm_103a" in pm.pm_version()


def test_no_oracle_in_product_path():
    """The product package never imports, links or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_2603_01122_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            for pat in (r"import\s+oracle", r"from\s+oracle", r"liboracle", r"pm_oracle", r"orc_\w+\("):
                assert not re.search(pat, text), (path, pat)
