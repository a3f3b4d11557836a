"""Bounds-checked build on the GPU: every stencil kernel, run on small and
ragged boxes with libllb_checked.so (each index compared with its buffer's
extent, an access out of range skipped and recorded), records no
out-of-range access and still matches the FP64 oracle.

The cases run in a child process (tests/checked_cases.py) so that the checked
library is the only one that process loads."""
import json
import os
import subprocess
import sys

import pytest

from paper_2301_01622_gb300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# least number of cases each group must actually run (not skipped as unsupported)
MIN_RUN = {"one": 140, "two": 50, "pop": 30, "batch": 10, "adjoint": 12}


def _run_group(group):
    if not os.path.exists(B.LIB_CHECKED):
        pytest.fail("libllb_checked.so not built (build() builds it beside libllb.so)")
    env = dict(os.environ, LLB_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py"), group], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, f"checked cases '{group}' failed:\n{r.stdout[-3000:]}\n{r.stderr[-3000:]}"
    return [json.loads(line) for line in r.stdout.splitlines() if line.startswith("{")]


@pytest.mark.parametrize("group", list(MIN_RUN))
def test_checked_kernels_in_bounds_and_exact(group):
    res = _run_group(group)
    out_of_range = [c for c in res if c["site"] != 0]
    assert not out_of_range, f"out-of-range accesses recorded: {out_of_range[:5]}"
    ran = [c for c in res if c["skip"] is None]
    bad = [c for c in ran if not c["err"] <= c["tol"]]
    assert not bad, f"checked build differs from the oracle: {bad[:5]}"
    assert len(ran) >= MIN_RUN[group], f"only {len(ran)} of {len(res)} cases ran"
