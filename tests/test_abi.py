"""The C-ABI library builds for sm_103a, loads, and exports every symbol the
public header declares (no GPU needed: no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b((?:als|alsncg)_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1508_03110_gb300 import build
    build.build()
    from paper_1508_03110_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("als_create", "als_sweep", "alsncg_step", "als_loss", "als_grad",
                 "als_linesearch_coeffs", "als_foldin", "als_destroy"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, f"declared in include/ but not exported: {missing}"


def test_binding_covers_the_header():
    from paper_1508_03110_gb300 import _lib
    assert _declared() <= set(_lib.SIGNATURES), _declared() - set(_lib.SIGNATURES)


def test_version_string(lib):
    assert b"sm_103a" in lib.als_version()


def test_config_defaults_are_the_papers(lib):
    import ctypes
    from paper_1508_03110_gb300 import _lib
    cfg = _lib.Config()
    lib.als_config_default(ctypes.byref(cfg))
    assert (cfg.ls_alpha0, cfg.ls_tau, cfg.ls_c) == (10.0, 0.9, 0.5)
    assert cfg.ls_max_shrinks == 200 and cfg.precision == _lib.ALS_FP64


def test_missing_library_fails_loudly(tmp_path):
    from paper_1508_03110_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved
