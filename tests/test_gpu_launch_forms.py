"""The launch structure changes no arithmetic: a BF16x3 solve gives bit-identical iterates with
the factorisation and products launched as programmatic dependent launches or the ordinary
way (GLASSO_NO_PDL=1), and with the tier-2 log-det terms formed on a second stream beside the
trial's factorisation or in line after it (GLASSO_NO_SPEC_TIER2=1).  The switches are read
once per process, so each form runs in a child process; the child checks that the rounding
band was met (tier 2 decided some steps), so the concurrent form was exercised."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, json, hashlib
sys.path.insert(0, {root!r})
import numpy as np
from paper_2205_10027_gb300 import binding, inputs
n = 576
S = inputs.sample_covariance(inputs.theta_grid(24, n=n), n // 2, np.random.default_rng(31))
with binding.Handle(precision="bf16x3", autotune=False) as h:
    h.begin(S, 0.1)
    tiers, trials = [], []
    for _ in range(40):
        st, res = h.step(1e-9)
        tiers.append(res["step_tier"])
        trials.append(res["trials"])
        if st != 11:
            break
    theta = np.empty((n, n), np.float64)
    h.end(theta)
print("RESULT", json.dumps(dict(tiers=tiers, trials=trials,
                                digest=hashlib.sha256(theta.tobytes()).hexdigest())))
"""


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    env.setdefault("GLASSO_TUNE_CACHE", "off")
    p = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    line = [ln for ln in p.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_launch_forms_give_identical_iterates():
    base = _run({})
    assert 2 in base["tiers"], "the rounding band was never met: the concurrent tier-2 form did not run"
    for extra in ({"GLASSO_NO_PDL": "1"}, {"GLASSO_NO_SPEC_TIER2": "1"},
                  {"GLASSO_NO_PDL": "1", "GLASSO_NO_SPEC_TIER2": "1"}):
        other = _run(extra)
        assert other == base, (extra, other, base)
