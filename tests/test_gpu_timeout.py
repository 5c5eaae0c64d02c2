"""The bounded waits of the tensor-core product end a stalled pipeline with an error status
instead of a hang (failure detection without a GPU fault).  A child process sets
GLASSO_TEST_TC_NO_LOADS=1, under which the product's producer thread issues no operand load, so
the MMA thread's bounded wait on the first stage runs out (about two seconds); the kernel then
leaves without writing, the solve returns GLASSO_ERR_TIMEOUT, and the same process can still
solve (in the FP64 form, which uses no tensor-core product) on the same context."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np
from paper_2205_10027_gb300 import binding, inputs
S = inputs.sample_covariance(inputs.theta_chain(300), 300, np.random.default_rng(1))
h = binding.Handle(precision="bf16x3", autotune=False)
try:
    h.solve(S, 0.2, 1e-6)
    print("STATUS", 0)
except binding.GlassoError as e:
    print("STATUS", e.status)
h.close()
with binding.Handle(precision="fp64") as f:
    _, res = f.solve(S, 0.2, 1e-8)
print("AFTER", res["status"])
"""


def test_tensor_core_wait_times_out_with_a_status():
    env = dict(os.environ, GLASSO_TEST_TC_NO_LOADS="1", GLASSO_TUNE_CACHE="off")
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = dict(l.split() for l in out.stdout.splitlines() if l.startswith(("STATUS", "AFTER")))
    assert lines["STATUS"] == "8", out.stdout    # GLASSO_ERR_TIMEOUT
    assert lines["AFTER"] == "0", out.stdout     # the context is still usable
