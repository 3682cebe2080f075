"""The bounds-checking debug build (-DBP_BOUNDS_CHECK): every staged,
gathered and scattered index of the kernels is checked, on cases that reach
every staging and edge path; no check may fire, and the results still match
the oracle.  The reporting path is tested by a synthetic failure that touches
no memory.  The debug library is built here (it is not part of the release
build) and loaded by a child process through BP_GB300_LIB."""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():  # pragma: no cover - GPU machine only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_flags_nothing_and_matches_the_oracle():
    from paper_2401_09283_gb300 import build
    lib = build.build_library(variant="bounds")
    env = dict(os.environ, BP_GB300_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_probe.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    print(out)
    assert out["library"] == lib
    assert out["flags"] == 0 and out["first"] == -1, out
    for name, (e_vol, e_grad) in out["cases"]:
        assert e_vol <= 1e-5 and e_grad <= 1e-3, (name, e_vol, e_grad)
    flags, first = out["selftest"]
    assert flags == 1 << 7 and first == (7 << 56) | (7 << 28) | 9
    assert out["cleared"] == [0, -1]


def test_release_build_reports_bounds_checking_unsupported():
    import ctypes
    from paper_2401_09283_gb300 import native as N
    ctx = N.context(0)
    flags, first = ctypes.c_uint(), ctypes.c_longlong()
    rc = N.lib().bp_bounds_check(ctx, 0, ctypes.byref(flags), ctypes.byref(first))
    assert rc == -4  # BP_ERR_UNSUPPORTED
