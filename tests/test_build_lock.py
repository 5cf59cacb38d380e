"""The library build takes turns across processes (the ranks of a multi-GPU launch may all call
it at once): two processes whose builds would overlap run them one after the other.  The compile
step is replaced by a stand-in that records its interval, so no nvcc is needed."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import sys, time
sys.path.insert(0, {root!r})
from paper_0905_3331_gb300 import build as b
b.up_to_date = lambda: False
def fake(verbose, extra_flags):
    t0 = time.time()
    time.sleep(1.0)
    with open({log!r}, "a") as fh:
        fh.write(f"{{t0}} {{time.time()}}\n")
    return b.LIB
b._build_locked = fake
b.build()
"""


def test_concurrent_builds_take_turns(tmp_path):
    log = str(tmp_path / "intervals.txt")
    code = _CHILD.format(root=ROOT, log=log)
    procs = [subprocess.Popen([sys.executable, "-c", code]) for _ in range(2)]
    for p in procs:
        assert p.wait(timeout=60) == 0
    iv = sorted(tuple(map(float, line.split())) for line in open(log))
    assert len(iv) == 2
    assert iv[0][1] <= iv[1][0] + 1e-3  # the second build starts after the first has finished
