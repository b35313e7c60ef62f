"""The planted-slip check (oracle/plant_slips.py) works end to end: two of
its slips, compiled into temporary copies of the oracle, are each failed by
the pin tests, and the oracle's own source is left as it was.  (The full
check, all slips, takes about 1.6 minutes on 8 jobs and is run by hand.)"""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_two_planted_slips_are_caught():
    src = os.path.join(ROOT, "oracle", "oracle.cpp")
    before = open(src).read()
    p = subprocess.run([sys.executable, os.path.join(ROOT, "oracle", "plant_slips.py"), "-j", "2",
                        "bary swap", "snell inverted"], cwd=ROOT, capture_output=True, text=True)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "2 of 2 slips caught" in p.stdout
    assert open(src).read() == before
