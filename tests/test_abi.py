"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry
point declared in include/mpcg.h with the binding's signatures (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpcg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_14268_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2504_14268_gb300 import mpcg

    assert sorted(mpcg.SIGNATURES) == _declared()


def test_struct_layouts():
    from paper_2504_14268_gb300 import mpcg

    assert ctypes.sizeof(mpcg.CResult) == 296
    assert mpcg.REC_DTYPE.itemsize == 80
    assert ctypes.sizeof(mpcg.COptions) == 264
    assert ctypes.sizeof(mpcg.Csr) == 40


def test_options_default_matches_paper(lib):
    """mpcg_options_default runs on the host only; it must give the Section 4.1 / 5 values."""
    from paper_2504_14268_gb300 import mpcg

    L = mpcg.lib()
    o = mpcg.COptions()
    L.mpcg_options_default(ctypes.byref(o))
    assert (o.b_bins, o.r_bins, o.t_bin, o.min_k, o.nprec) == (10, 10, 1000, 10, 5)
    assert o.eps_min == 1e-16 and (o.w1, o.w2, o.w3) == (1.0, 0.1, 10.0)
    assert (o.lr, o.gamma, o.eps0, o.eps_floor) == (0.1, 0.9, 1.0, 0.1)
    assert list(o.precs)[:5] == [0, 1, 2, 3, 4]
    assert list(o.cost)[:5] == [0.8, 0.6, 0.8, 1.0, 2.0]
    assert o.edge_tol == 5e-3 and o.stepped == 0 and o.variant == 0 and o.joint == 0
    assert L.mpcg_mlp_nparams(64, 5) == 64 * 16 + 64 + 64 * 64 + 64 + 20 * 64 + 20


def test_product_path_has_no_cpu_fallback():
    """The binding refuses to run when the library is missing instead of computing on the CPU."""
    import importlib

    from paper_2504_14268_gb300 import build, mpcg

    src = open(mpcg.__file__).read()
    assert "import oracle" not in src and "from oracle" not in src
    for f in os.listdir(os.path.join(ROOT, "paper_2504_14268_gb300")):
        if f.endswith(".py"):
            t = open(os.path.join(ROOT, "paper_2504_14268_gb300", f)).read()
            assert not re.search(r"^\s*(import|from)\s+oracle", t, flags=re.M), f
