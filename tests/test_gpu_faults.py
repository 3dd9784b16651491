"""Failure detection without a GPU fault.

* A bounded device wait that runs out: a test knob makes every TMA barrier
  expect more bytes than its copy delivers, so the barrier never completes
  (the copy itself lands); the kernel's bounded waits expire, it raises the
  timeout flag and exits with nothing in flight.  The host reads
  HJLO_ETIMEOUT and the context stays usable.
* An allocation failure injected on the host (HJLO_TEST_FAIL_ALLOC) gives
  HJLO_ENOMEM from plan creation, without exhausting device memory.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounded_wait_runs_out_and_context_survives(monkeypatch):
    from paper_1210_4090_gb300 import hjlo
    shape, dx, h, P, W = (64, 96), (1 / 64, 1 / 96), 0.05, (0.3, 0.1), (8, 12)
    rng = np.random.default_rng(0)
    u0, V = rng.normal(size=shape) * 0.3, rng.normal(size=shape) * 0.2
    monkeypatch.setenv("HJLO_TEST_EXTRA_TX", "16")
    monkeypatch.setenv("HJLO_TEST_WAIT_NS", "1000000")
    plan = hjlo.Plan(shape, dx, h, P, W)
    u = torch.tensor(u0, device="cuda")
    plan.step(u, u, torch.tensor(V, device="cuda"))
    with pytest.raises(hjlo.HjloError) as ei:
        plan.sync()
    assert ei.value.name == "HJLO_ETIMEOUT"
    plan.close()
    monkeypatch.delenv("HJLO_TEST_EXTRA_TX")
    monkeypatch.delenv("HJLO_TEST_WAIT_NS")
    plan = hjlo.Plan(shape, dx, h, P, W)
    u = torch.tensor(u0, device="cuda")
    plan.step(u, u, torch.tensor(V, device="cuda"))
    assert plan.sync()["error_flags"] == 0
    assert np.array_equal(u.cpu().numpy(), O.run(u0, dx, h, P, W, V, 1))


def test_injected_allocation_failure_reports_enomem():
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1210_4090_gb300 import hjlo\n"
        "try:\n"
        "    hjlo.Plan((32, 32), 1/32, 0.1, (0.2, 0.1), (3, 3))\n"
        "    print('created')\n"
        "except hjlo.HjloError as e:\n"
        "    print(e.name)\n"
        "p = hjlo.Plan((32, 32), 1/32, 0.1, (0.2, 0.1), (3, 3))\n"
        "print('second ok')\n" % ROOT)
    env = dict(os.environ, HJLO_TEST_FAIL_ALLOC="2")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "HJLO_ENOMEM" in r.stdout and "second ok" in r.stdout
