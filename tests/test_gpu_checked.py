"""The checked build (-DSD_CHECKED): its kernels test the indices they
compute before using them.  A mixed workload that reaches the kernels' edge
cases (checked_workload.py) must record no failed check there, and give
bitwise the outputs of the normal build (the checks only skip accesses that
would be out of range)."""
import json
import os
import subprocess
import sys

import pytest

import checked_workload

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_records_no_failed_check_and_matches(sdlib):
    sd = sdlib
    subprocess.run([sys.executable, "-c",
                    "from paper_2503_11213_gb300 import build as b; b.build(checked=True)"],
                   cwd=ROOT, check=True)
    env = dict(os.environ, SDIRT_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_workload.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["count"] == 0, res
    assert res["site"] == 0
    plain = checked_workload.run(sd)
    assert res["hashes"] == plain
    # the normal build compiles the checks away
    with pytest.raises(sd.SdError):
        sd.api.check_status()
