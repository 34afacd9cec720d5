"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no compute calls: these run without a GPU)."""
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
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(cdi_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2110_13055_gb300 import _build, cdi
    _build.build()
    return cdi.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cdi_create_domain", "cdi_solve_flow", "cdi_set_potential",
                     "cdi_init_transport", "cdi_step_transport", "cdi_query_adsorbed",
                     "cdi_query_outlet", "cdi_destroy_domain"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2110_13055_gb300 import cdi
    bound = {name for name, _, _ in cdi.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_version_and_null_handling(lib):
    from paper_2110_13055_gb300 import cdi
    assert cdi.version() >= 100
    # argument checks run before any device work
    out = cdi.c_void_p()
    st = lib.cdi_create_domain(None, None, None, None, cdi.ctypes.byref(out))
    assert st == 1 and not out.value
    assert "NULL" in cdi.last_error(None)
    desc = cdi.cdi_domain_desc(2, 4, 4, 2, 1e-7, 0, 1, 0)   # nz must be 1 in 2D
    import numpy as np
    m = np.zeros((4, 4), np.uint8)
    st = lib.cdi_create_domain(cdi.ctypes.byref(desc), m.ctypes.data_as(cdi.c_void_p), None,
                               None, cdi.ctypes.byref(out))
    assert st == 1
    desc = cdi.cdi_domain_desc(2, 4, 4, 1, 1e-7, 0, 1, 0)
    m[:, 0] = 1                                              # inlet column all solid
    st = lib.cdi_create_domain(cdi.ctypes.byref(desc), m.ctypes.data_as(cdi.c_void_p), None,
                               None, cdi.ctypes.byref(out))
    assert st == 1 and "inlet" in cdi.last_error(None)
    lib.cdi_destroy_domain(None)


def test_product_path_does_not_import_the_oracle():
    """The package and its CUDA sources never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2110_13055_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(f).read()
            assert "import oracle" not in text and "from oracle" not in text, f
            assert "cdi_oracle" not in text, f


def test_every_entry_point_cites_its_passage():
    """Each declaration's comment cites the passage of the paper that defines
    the operation, or says that the paper has no counterpart."""
    text = open(os.path.join(ROOT, "include", "cdi.h")).read()
    missing = []
    for m in re.finditer(r"(/\*(?:(?!\*/).)*\*/)\s*\n(?:[^;/]*?)\b(cdi_\w+)\s*\(", text, flags=re.S):
        comment = re.sub(r"\s*\n\s*\*\s*", " ", m.group(1))
        if not re.search(r"Sec\. ?\d|Eq\. ?\d|Fig\. ?\d|no counterpart", comment, flags=re.I):
            missing.append(m.group(2))
    assert not missing, missing
