"""The checked build (-DLOGDET_CHECKED): device-side bounds checks of every
index the Krylov passes take from memory and canary words around every
workspace buffer, in place of the sanitizers (closed on this pool).

The same workload (tests/checked_workload.py: every kind of solve on small
inputs) runs in two subprocesses, against the checked and the normal build.
The checked run must report no index violation and no changed canary byte,
and its estimates must equal the normal build's bit for bit (the checks
redirect nothing on valid inputs and change no arithmetic)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_07004_gb300 import build as BB  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(lib):
    env = dict(os.environ, LOGDET_LIB=lib)
    p = subprocess.run([sys.executable, os.path.join(HERE, "checked_workload.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_checked_build_finds_nothing_and_matches_bitwise():
    checked_lib = BB.build(checked=True)
    normal_lib = BB.build()
    got = _run(checked_lib)
    ref = _run(normal_lib)
    rep = got.pop("report")
    assert rep == {"checked": True, "device_violations": 0, "canary_bytes": 0}
    assert ref.pop("report")["checked"] is False
    assert got == ref
