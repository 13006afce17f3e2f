"""The C-ABI library loads and exports every entry point include/*.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

import paper_1311_0378_gb300 as rc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\(", text):
            name = m.group(1)
            pre = text[:m.start()].rstrip()
            if name.startswith("recon_") and not pre.endswith(("define", "return")):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_1311_0378_gb300.build as b
    b.build()
    return rc.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("recon_init", "recon_run", "recon_batch", "recon_free"):
        assert f in names
    assert names == set(rc.SYMBOLS), names ^ set(rc.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_strerror_and_null_handling(lib):
    assert rc.recon_strerror(rc.RECON_EMARKER).startswith("marker")
    assert rc.recon_strerror(99) == "unknown status"
    assert lib.recon_free(None) == rc.RECON_OK
    assert lib.recon_sync(None) == rc.RECON_EINVAL
    assert lib.recon_run(None, None, None, 4, 4, 8) == rc.RECON_EINVAL
    assert lib.recon_init(None, 0, None, 0) == rc.RECON_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(rc, "_lib", None)
    monkeypatch.setattr(rc, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        rc.recon_strerror(0)
