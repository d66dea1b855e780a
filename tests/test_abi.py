"""The C ABI library builds for sm_103a, loads, and exports every function
that include/finrl_gb300.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        with open(os.path.join(ROOT, "include", fn)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"#.*", "", src)
        src = re.sub(r"typedef struct \{.*?\}\s*\w+;", "", src, flags=re.S)
        for m in re.finditer(r"\b([A-Za-z_]\w*)\s*\(", src):
            prev = src[:m.start()].rstrip()
            if prev.endswith(("typedef", "(")):
                continue
            names.add(m.group(1))
    return names - {"if", "sizeof"}


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    declared = _declared_functions()
    assert len(declared) >= 20
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(built_lib):
    from paper_2501_10709_gb300 import _lib
    assert _declared_functions() == set(_lib.SIGNATURES)


def test_binding_loads_without_a_gpu(built_lib):
    import paper_2501_10709_gb300 as fr
    lib = fr.lib()
    assert lib.fr_version().decode().startswith("finrl_gb300")
    assert lib.fr_last_error().decode() == ""


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2501_10709_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        _lib.load()


def test_fault_injection_knob_checks_its_arguments(built_lib):
    import paper_2501_10709_gb300 as fr
    for bad in ((0, 0, 1), (4, 0, 1), (fr.FAULT_ALLOC, -1, 1), (fr.FAULT_POLL, 0, -2)):
        with pytest.raises(fr.FrError) as ei:
            fr.fr_fault_inject(*bad)
        assert ei.value.code == fr._lib.FR_EINVAL
    for k in (fr.FAULT_ALLOC, fr.FAULT_SUBMIT, fr.FAULT_POLL):
        fr.fr_fault_inject(k, 2, 1)
        fr.fr_fault_inject(k, 0, 0)                     # disarmed again
