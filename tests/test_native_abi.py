"""The C-ABI library builds, loads without a GPU and exports every function
that include/*.h declares (no compute calls here)."""
import glob
import os
import re

from paper_2401_09283_gb300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        # every "name(" in the header is a function declaration
        names.update(re.findall(r"\b(bp_[a-z0-9_]+|motion_step)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    build.build_library()
    import ctypes
    L = ctypes.CDLL(build.LIB)
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding knows all of them too
    assert set(native.EXPORTS) <= names
