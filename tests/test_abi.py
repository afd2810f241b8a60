"""The C-ABI library loads and exports every entry point include/*.h declares
(no compute call: these run without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(stc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1608_01102_gb300 import build, stc
    build.build()
    return stc.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    from paper_1608_01102_gb300 import stc
    assert set(_declared()) == set(stc.SIGNATURES)


def test_default_params_follow_the_paper(lib):
    from paper_1608_01102_gb300 import stc
    p = stc.default_params(128, 128, 40)
    assert p.dt == 1.0 / 40 and p.ao_iters == 2 and p.pre == 2 and p.post == 2
    assert p.coarse_sweeps == 10 and p.taylor_tol == 1e-5 and p.beta == 1.0


def test_params_struct_layout_matches_header(lib):
    """Field order of the ctypes mirror equals the C declaration order."""
    from paper_1608_01102_gb300 import stc
    src = open(os.path.join(ROOT, "include", "stc.h")).read()
    body = src[src.index("typedef struct {"):src.index("} stc_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b([a-zA-Z_0-9]+)\s*[,;]", body)
    assert names == [f for f, _ in stc.StcParams._fields_]


def test_missing_library_fails_loudly(tmp_path):
    from paper_1608_01102_gb300 import stc
    with pytest.raises(RuntimeError):
        stc.load(str(tmp_path / "libstc.so"))
