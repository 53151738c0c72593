"""The t-pass launch-shape tuning (and the lateral solve's kernel choice)
persists across processes: the first plan of a geometry writes its choices to
the tuning file (NLOS_TUNE_CACHE), a
later process reads them instead of timing again (so it writes nothing), and
a file made under another key (device, SM count, compile time) is ignored and
replaced."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MAGIC = "nlos-gb300 t-pass tuning v1"
SXY_KIND = 9  # the lateral-solve entry of the tuning file (after the nine t-pass kinds)

SCRIPT = r"""
import sys, time
sys.path.insert(0, {root!r})
from paper_2301_00406_gb300 import nlos
mask = __import__("numpy").zeros((32, 32), "uint8")
mask[1::4, 3::4] = 1
t = time.time()
for m in (None, mask):
    nlos.Plan(32, 32, 256, 32e-12, mask=m).close()
print("plans_s", time.time() - t)
"""


def _run(path):
    env = dict(os.environ, NLOS_TUNE_CACHE=str(path))
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=300)
    print(r.stdout, r.stderr[-2000:])
    assert r.returncode == 0
    return r.stdout


def test_tuning_file_written_then_reused(tmp_path):
    path = tmp_path / "sub" / "tune"
    _run(path)
    lines = path.read_text().splitlines()
    assert lines[0] == MAGIC
    assert " SMs | " in lines[1]
    entries = [tuple(map(int, l.split())) for l in lines[2:]]
    assert entries and all(len(e) == 4 and e[1] == 256 for e in entries)
    tpass = [e for e in entries if e[0] != SXY_KIND]
    sxy = [e for e in entries if e[0] == SXY_KIND]
    assert {e[2] for e in tpass} == {32 * 32, 8 * 8}   # full grid and the 8 x 8 sampled columns
    # the lateral solve's kernel for 32 x 32 planes: the shared-memory passes
    # (1) or the half-warp transforms (2), chosen once for both plans
    assert len(sxy) == 1 and sxy[0][2] == 32 and sxy[0][3] in (1, 2)
    before = (path.stat().st_mtime_ns, path.read_text())
    _run(path)                                          # read, nothing new to time: not rewritten
    assert (path.stat().st_mtime_ns, path.read_text()) == before


def test_tuning_file_of_another_key_is_replaced(tmp_path):
    path = tmp_path / "tune"
    path.write_text(f"{MAGIC}\nsome other GPU | 7 SMs | another build\n0 256 1024 2\n")
    _run(path)
    lines = path.read_text().splitlines()
    assert lines[0] == MAGIC and "some other GPU" not in lines[1] and " SMs | " in lines[1]
