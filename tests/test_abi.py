"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/stokesmg.h
and include/warmstart.h declare (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in ("stokesmg.h", "warmstart.h"):
        src = open(os.path.join(ROOT, "include", hdr)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?(?:[a-z_0-9]+\s+)+\**\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2312_10615_gb300 import build as nb
    path = nb.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    import paper_2312_10615_gb300 as smg
    assert sorted(smg.EXPORTS) == _declared()


def test_strerror_and_opts_without_gpu():
    import paper_2312_10615_gb300 as smg
    assert smg.stokes_strerror(0) == "ok"
    assert "breakdown" in smg.stokes_strerror(smg.ERR_BREAKDOWN).lower()
    o = smg.stokes_opts_default()
    assert o.gamma == 1e-3 and o.kb_vanka == 1 and o.precision == smg.PREC_FP64


def test_sm103a_target_in_build_flags():
    from paper_2312_10615_gb300 import build as nb
    assert "arch=compute_103a,code=sm_103a" in " ".join(nb.ARCH)
