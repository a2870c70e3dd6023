"""Failure detection without a GPU fault.

- Host-side injection: BDM_FAULT_ALLOC=n makes the n-th device allocation of
  the process fail.  Every failing call must return BDM_E_NOMEM, and the
  context (or a new one) must work afterwards.  Each case runs in a fresh
  process, because the allocation counter is per process.
- A bounded device wait that runs out: with the test hook of bdm_tuning the
  ordered grid scan waits for a tile word that nothing writes and gives up
  after a few polls; bdm_sync then reports BDM_E_TIMEOUT, no kernel hangs,
  and the context steps correctly afterwards.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2503_10796_gb300 import binding, workloads
pop = workloads.plain_fp64(n=3000, precision=1)
pop.params.sort_interval = 2
out = {"events": []}
ctx = None
for attempt in range(3):
    try:
        if ctx is None:
            ctx = binding.Context(binding.make_params(pop.params), pop.n + 8)
            out["events"].append("created")
        if "set" not in out["events"]:
            ctx.set_agents(0, pop.xyz, pop.diameter)
            out["events"].append("set")
        ctx.step(3)
        ctx.sync()
        out["events"].append("stepped")
        break
    except binding.BdmError as e:
        out["events"].append(f"error {e.code}")
x, _ = ctx.get_agents(0)
out["finite"] = bool(np.isfinite(x).all())
out["iterations"] = ctx.stats(0)["iterations"]
print(json.dumps(out))
"""


@pytest.mark.parametrize("n", [1, 5, 12, 20, 28, 40])
def test_injected_allocation_failure(n):
    env = dict(os.environ, BDM_FAULT_ALLOC=str(n))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    errors = [e for e in out["events"] if e.startswith("error")]
    # at most one injected failure, always reported as BDM_E_NOMEM
    assert errors in ([], ["error -2"]), out
    assert out["events"][-1] == "stepped" and out["finite"], out
    print(f"FAULT_ALLOC n={n}: {out['events']}")


def test_bounded_wait_reports_timeout(orc):
    from paper_2503_10796_gb300 import binding
    import oracle
    pop = workloads.uniform_fraction(20000, precision=0)
    ctx = binding.Context(binding.make_params(pop.params), pop.n + 8)
    ctx.set_agents(0, pop.xyz, pop.diameter)
    t = ctx.get_tuning()
    ctx.set_tuning(**dict(t, test_flags=1))
    ctx.step(1)
    with pytest.raises(binding.BdmError) as e:
        ctx.sync()
    assert e.value.code == -5
    # the context stays usable: the hook off, the agents set again, the
    # step matches the oracle
    ctx.set_tuning(**dict(t, test_flags=0))
    ctx.set_agents(0, pop.xyz, pop.diameter)
    ctx.step(2)
    ctx.sync()
    x, _ = ctx.get_agents(0)
    o = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    o.step(2)
    x_o, _, _ = o.get()
    assert np.abs(x - x_o).max() <= 1e-9 * pop.diameter.max()


def test_unknown_test_hooks_are_rejected(orc):
    """Test hooks are bits 0 and 1 of test_flags; any other bit is refused
    and leaves the tuning as it was."""
    from paper_2503_10796_gb300 import binding
    pop = workloads.plain_fp64(n=200, precision=0)
    ctx = binding.Context(binding.make_params(pop.params), pop.n + 8)
    ctx.set_agents(0, pop.xyz, pop.diameter)
    t = ctx.get_tuning()
    for bad in (4, 8, 1 << 30, -1):
        with pytest.raises(binding.BdmError) as e:
            ctx.set_tuning(**dict(t, test_flags=bad))
        assert e.value.code == -1, bad
    assert ctx.get_tuning() == t
    ctx.step(2)
    ctx.sync()
