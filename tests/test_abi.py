"""CPU checks of the C-ABI library: it builds, loads, exports every entry
point include/srj.h declares, and its host-side scheme table (written
independently of the oracle) agrees with the oracle's.  No GPU calls."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT, read_golden


def _declared():
    src = open(os.path.join(ROOT, "include", "srj.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(srj_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2011_06636_gb300 import _build, srj
    _build.build()
    return srj.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2011_06636_gb300 import srj
    names = _declared()
    assert len(names) >= 11
    assert sorted(srj.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_version_and_level_table(lib):
    from paper_2011_06636_gb300 import srj
    assert "sm_103a" in srj.srj_version()
    for lv, M in read_golden("appB_levels.txt"):
        assert srj.srj_level_m(int(lv)) == int(M)
    assert srj.srj_level_m(25) == -1 and srj.srj_level_m(-1) == -1


@pytest.mark.parametrize("level", range(25))
def test_library_factors_equal_oracle_bitwise(lib, orc, level):
    from paper_2011_06636_gb300 import srj
    got = srj.srj_scheme_omegas(level)
    ref = orc.level_omegas(level)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref)


def test_bad_level_rejected(lib):
    from paper_2011_06636_gb300 import srj
    with pytest.raises(srj.SrjError):
        srj.srj_scheme_omegas(25)


def test_binding_structs_and_enums_match_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C layout (sizes and
    field offsets from a host C compile of include/srj.h) and the binding's
    enum constants the header's values."""
    import subprocess
    from paper_2011_06636_gb300 import srj
    structs = {"srj_grid": srj.srj_grid, "srj_stencil": srj.srj_stencil,
               "srj_opts": srj.srj_opts, "srj_stats": srj.srj_stats,
               "srj_mg_opts": srj.srj_mg_opts, "srj_move_record": srj.srj_move_record}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "srj.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    enums = ["SRJ_TOL_REL", "SRJ_TOL_ABS", "SRJ_TOL_DINF", "SRJ_BC_DIRICHLET", "SRJ_BC_NEUMANN",
             "SRJ_PREC_F64", "SRJ_PREC_F32", "SRJ_PREC_MIXED", "SRJ_SEL_HEURISTIC",
             "SRJ_SEL_INCREASING", "SRJ_SEL_FIXED", "SRJ_SEL_MLP", "SRJ_SEL_JACOBI",
             "SRJ_EUNSUPPORTED"]
    for e in enums:
        lines.append('printf("%s %%d\\n", (int)%s);' % (e, e))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o",
                           str(exe), str(src)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[name + "." + field]) == getattr(cls, field).offset, (name, field)
    for e in enums:
        assert int(got[e]) == getattr(srj, e), e
