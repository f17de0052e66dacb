"""Device-detected errors: a step whose states become non-finite latches NUMA_ERR_NONFINITE
in the context's device status word; numa_status reports it once and clears it.  Detection
happens where the step evaluates the equation of state -- the P' pre-pass of each step's
input and the fused P' output of each implicit stage -- and in the ARK4/ARK5 final
combination, with integer tests of the exponent bits.  (The data are ordinary IEEE
infinities and NaNs: nothing here faults the device.)"""
import numpy as np
import pytest

from helpers import Case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def pkg():
    import paper_1702_04316_gb300 as p
    p.lib()
    return p


CASE = (4, 6, 3, 4, 80e3, 120e3, 10e3)


def make(pkg, **kw):
    case = Case(*CASE[:3], CASE[3], *CASE[4:])
    g = pkg.Numa(*case.args[:6], case.args[6], case.dt_for(15.0), 300.0, case.n_bv, **kw)
    return case, g


@pytest.mark.parametrize("field,value", [(4, float("nan")), (0, float("inf")), (1, float("nan"))])
@pytest.mark.parametrize("scheme", ["ark2", "ark3", "ark5"])
def test_step_latches_nonfinite(pkg, torch, field, value, scheme):
    """A NaN or infinity anywhere in the state (theta', rho' or u) is reported after one
    step; the status reads clear afterwards."""
    case, g = make(pkg, scheme=scheme)
    q0 = case.state(81, kind="balanced")
    q = torch.from_numpy(q0).cuda()
    g.step_imex1d(q.clone(), g.empty_state(), 1)
    assert g.status() == pkg.NUMA_OK
    bad = q.clone()
    bad[field, case.mesh.nnode // 2] = value
    g.step_imex1d(bad, g.empty_state(), 1)
    assert g.status() == pkg.NUMA_ERR_NONFINITE
    assert g.status() == pkg.NUMA_OK                       # read once, then cleared
    g.close()


def test_explicit_and_host_runs_latch_nonfinite(pkg, torch):
    case, g = make(pkg)
    q0 = case.state(82, kind="balanced")
    bad = torch.from_numpy(q0.copy())
    bad[4, 7] = float("nan")
    g.step_explicit_rk(bad.cuda(), case.dt_for(1.0), g.empty_state(), 1)
    assert g.status() == pkg.NUMA_ERR_NONFINITE
    qh = bad.pin_memory()
    g.run_host(0, qh, 1)                                   # the pipelined host run
    assert g.status() == pkg.NUMA_ERR_NONFINITE
    good = torch.from_numpy(q0.copy()).pin_memory()
    g.run_host(0, good, 2)
    g.step_explicit_rk(torch.from_numpy(q0).cuda(), case.dt_for(1.0), g.empty_state(), 2)
    assert g.status() == pkg.NUMA_OK
    g.close()


def test_clean_runs_report_ok(pkg, torch):
    for kw in ({}, {"precision": "mixed"}, {"precision": "rhs32"}, {"scheme": "ark4"}):
        case, g = make(pkg, **kw)
        q = torch.from_numpy(case.state(83, kind="balanced")).cuda()
        g.step_imex1d(q, None, 3)
        assert g.status() == pkg.NUMA_OK, kw
        g.close()


_TIMEOUT_SCRIPT = r"""
import os, time, torch
import paper_1702_04316_gb300 as pkg
g = pkg.Numa(4, 4, 4, 10e3, 10e3, 10e3, 4, 9.0)
b = torch.randn(g.ncol * g.M, dtype=torch.float64, device="cuda",
                generator=torch.Generator(device="cuda").manual_seed(9))
x0 = g.solve_columns(b)
assert g.status() == pkg.NUMA_OK
os.environ["NUMA_TEST_SOLVE_TIMEOUT"] = "1"
t0 = time.time()
g.solve_columns(b, torch.empty_like(b))
torch.cuda.synchronize()
elapsed = time.time() - t0
st = g.status()
del os.environ["NUMA_TEST_SOLVE_TIMEOUT"]
x2 = g.solve_columns(b)
print(st, g.status(), "%.3f" % elapsed, int(torch.equal(x2, x0)))
"""


def test_bulk_copy_wait_gives_up_with_a_status():
    """The stand-alone solve waits on mbarriers for its bulk copies, every wait bounded (1 s).
    NUMA_TEST_SOLVE_TIMEOUT=1 arms the first factor row's barrier of every warp for 16 bytes
    more than its copy delivers, so that wait runs out (no fault: the barrier simply never
    completes).  The kernel latches NUMA_ERR_TIMEOUT, drains its copies with the same bound
    and returns; numa_status reports it, and the next solve in the same context is exact
    again.  Run in a child process so that the switch touches no other test."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root)
    env.pop("NUMA_TEST_SOLVE_TIMEOUT", None)
    r = subprocess.run([sys.executable, "-c", _TIMEOUT_SCRIPT], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    st, st2, elapsed, same = r.stdout.split()
    import paper_1702_04316_gb300 as p
    assert int(st) == p.NUMA_ERR_TIMEOUT
    assert int(st2) == p.NUMA_OK
    assert 0.9 < float(elapsed) < 60.0                 # the 1 s bound, then the drain
    assert same == "1"
