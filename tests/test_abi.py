"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/esmm.h (no compute calls: this runs without a GPU)."""
import os
import re

from paper_2107_12027_gb300 import build, esmm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "esmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(esmm_[a-z_]+)\s*\(", src))


def test_library_exports_every_declared_symbol():
    build.build()
    declared = _declared()
    assert "esmm_rhs" in declared and "esmm_rk_step" in declared
    assert declared == set(esmm.SYMBOLS)
    L = esmm.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert "sm_103a" in esmm.version()


def test_binding_rejects_wrong_array_types():
    import numpy as np
    import pytest
    with pytest.raises(AssertionError):
        esmm._ptr(np.zeros(4, dtype=np.float32))
    with pytest.raises(AssertionError):
        esmm._ptr(np.zeros((4, 4))[:, ::2])


def test_named_schemes_host_logic():
    # Sec. 6: MM-O6 is the sixth-order (p = 3) EC scheme, MM-O5 the ES scheme
    # with WENO5 dissipation on the 2p = 6 EC flux; UM-* are the same on the
    # static mesh
    from paper_2107_12027_gb300 import esmm
    assert esmm.SCHEMES["MM-O6"] == dict(p=3, w=0, move_mesh=1)
    assert esmm.SCHEMES["MM-O5"] == dict(p=3, w=5, move_mesh=1)
    assert esmm.SCHEMES["UM-O5"] == dict(p=3, w=5, move_mesh=0)
    prm = {}
    assert esmm._apply_scheme("UM-O5", 2, 3, prm) == (3, 5) and prm == {"move_mesh": 0}
    prm = {"move_mesh": 1}
    assert esmm._apply_scheme("UM-O5", 2, 3, prm) == (3, 5) and prm == {"move_mesh": 1}
    prm = {}
    assert esmm._apply_scheme(None, 2, 3, prm) == (2, 3) and prm == {}


# the calls that define a step of the method, each of which must cite the
# passage that defines it (a section, equation, proposition or theorem)
CITED_CALLS = ("esmm_grid_create", "esmm_set_eos", "esmm_set_order", "esmm_set_params", "esmm_state_set",
               "esmm_rhs", "esmm_cfl_dt", "esmm_mesh_redistribute", "esmm_rk_step", "esmm_rk_step_given",
               "esmm_set_inflow", "esmm_totals", "esmm_mhd_eigen")


def _comment_before(src, name):
    """The comment block documenting a declaration: the last /* ... */ that
    ends before it, across any declarations that share it."""
    at = src.index("int %s(" % name)
    end = src.rindex("*/", 0, at)
    start = src.rindex("/*", 0, end)
    return src[start:end]


def test_method_calls_cite_their_defining_passage():
    src = open(os.path.join(ROOT, "include", "esmm.h")).read()
    cite = re.compile(r"\b(Sec\.|eq\.|eqs\.|Prop\.|Thm\.)\s*[A-Za-z0-9_]")
    for name in CITED_CALLS:
        assert cite.search(_comment_before(src, name)), name
