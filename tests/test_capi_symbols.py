"""The C-ABI library and the oracle build here (no GPU), and the library exports every entry
point that include/mhd.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:mhd_status_t|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_four_paper_calls():
    names = _declared()
    for n in ("mhd_grid_create", "mhd_step", "pcg_solve", "mhd_adjoint_step"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1811_02605_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    import paper_1811_02605_gb300 as P
    assert sorted(P.SYMBOLS) == _declared()


def test_oracle_builds_and_is_separate():
    import oracle
    path = oracle.build()
    assert os.path.exists(path)
    # the product library never links the oracle: none of its sources lives under oracle/, and
    # none of the oracle's entry points is exported
    from paper_1811_02605_gb300 import build as B
    assert all(os.sep + "oracle" + os.sep not in src for src in B.sources())
    lib = ctypes.CDLL(B.build())
    for name in ("og_pcg", "og_step", "og_force", "og_ilu0"):
        assert not hasattr(lib, name), name


def test_binding_kernel_names_match_the_header():
    # the diagnostics' kernel ids (MHD_KERNEL_*) and the binding's name list agree in number
    src = open(os.path.join(ROOT, "include", "mhd.h")).read()
    count = int(re.search(r"MHD_KERNEL_COUNT\s*=\s*(\d+)", src).group(1))
    import paper_1811_02605_gb300 as P
    assert len(P.KERNELS) == count
    ids = dict((m.group(1).lower(), int(m.group(2)))
               for m in re.finditer(r"MHD_KERNEL_(\w+)\s*=\s*(\d+)", src) if m.group(1) != "COUNT")
    for k, name in enumerate(P.KERNELS):
        assert ids.get(name) == k, (name, k)


def test_binding_rejects_missing_library(tmp_path, monkeypatch):
    import paper_1811_02605_gb300 as P
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(P, "_lib", None)
    with pytest.raises(RuntimeError):
        P.lib()
