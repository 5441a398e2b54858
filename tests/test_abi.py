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
