"""Failure detection without a GPU fault.

The wave kernel's dependency waits are bounded.  rot_selftest_wait_timeout
starts a small launch whose items wait on counters that nothing advances;
with a 200 ms limit they give up, the launch reports ROT_ETIMEOUT, and the
device keeps working: a normal rot_apply right after is still bit-exact.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2412_01852_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_device_stays_usable():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_01852_gb300 as rs
    from paper_2412_01852_gb300 import _native, build
    build.build()
    lib = _native.load()
    t0 = time.perf_counter()
    code = lib.rot_selftest_wait_timeout(200, None)
    el = time.perf_counter() - t0
    assert code == 4, _native.status_string(code)        # ROT_ETIMEOUT
    assert 0.15 < el < 30.0
    A, C, S = wl.problem(70, 90, 12, seed=3)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    Cd = torch.from_numpy(np.ascontiguousarray(C.T)).cuda().t()
    Sd = torch.from_numpy(np.ascontiguousarray(S.T)).cuda().t()
    rs.rot_apply(Ad, Cd, Sd)
    rs.rot_device_status()
    ref = oracle.rot_sequence(A, C, S)
    assert np.array_equal(Ad.cpu().numpy().view(np.uint64), ref.view(np.uint64))
