"""Serving: continuous batching of requests on resident matrices.

Each matrix's final value must equal the oracle applying that matrix's
requests one after another in submission order, bit for bit: a result is the
same alone and in the mix, whatever batches and streams the scheduler used.
"""
import numpy as np
import pytest

import oracle
from paper_2412_01852_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_01852_gb300 import api, build
    build.build()
    return api


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def bits(x):
    return np.ascontiguousarray(x).view(np.uint64)


def test_mixed_requests_equal_sequential_oracle(api):
    r = np.random.default_rng(9)
    sizes = [128, 256, 512, 128, 256, 96, 300, 128]
    mats = [wl.matrix(n, n, seed=500 + i) for i, n in enumerate(sizes)]
    devm = [dev(A) for A in mats]
    expected = [A.copy() for A in mats]
    reqs = []
    for q in range(80):
        i = int(r.integers(0, len(sizes)))
        k = int(r.integers(2, 65))
        reqs.append((i,) + wl.rotations(sizes[i], k, seed=9000 + q))
    with api.Server(hbm_budget_bytes=256 << 20, max_inflight=12, streams=3, max_batch=5) as srv:
        handles = [srv.register(A) for A in devm]
        # A burst: requests arrive faster than launches finish, so the
        # scheduler has several admissible requests per step.
        tickets = [srv.submit(handles[i], C, S) for (i, C, S) in reqs]
        for t in tickets:
            srv.wait(t, 60000)
        st = srv.stats()
        assert st["completed"] == 80 and st["pending"] == 0 and st["inflight"] == 0
        assert st["launches"] < 80          # requests were batched together
        assert st["mean_batch"] > 1.0
        assert st["p99_ms"] >= st["p50_ms"] > 0
    for (i, C, S) in reqs:
        expected[i] = oracle.rot_sequence(expected[i], C, S)
    for A, E in zip(devm, expected):
        assert np.array_equal(bits(A.cpu().numpy()), bits(E))


def test_budget_refusal_and_serialisation(api):
    # 2 MiB arena: a 1024 x 1024, k = 64 request needs more and is refused;
    # small ones that fit only one at a time still all complete.
    with api.Server(hbm_budget_bytes=2 << 20, max_inflight=8, streams=2, max_batch=8) as srv:
        big = dev(wl.matrix(1024, 1024, seed=1))
        hb = srv.register(big)
        C, S = wl.rotations(1024, 64, seed=2)
        with pytest.raises(Exception) as ei:
            srv.submit(hb, C, S)
        assert getattr(ei.value, "code", None) == 3  # ROT_ENOMEM
        assert srv.stats()["rejected"] == 1
        A = wl.matrix(200, 200, seed=3)
        Ad = dev(A)
        h = srv.register(Ad)
        exp = A
        ts = []
        for q in range(6):
            C, S = wl.rotations(200, 40, seed=30 + q)
            ts.append(srv.submit(h, C, S))
            exp = oracle.rot_sequence(exp, C, S)
        for t in ts:
            srv.wait(t, 60000)
    assert np.array_equal(bits(Ad.cpu().numpy()), bits(exp))


@pytest.mark.parametrize("max_fused_k", [0, 16])
def test_fused_requests_on_one_matrix(api, max_fused_k):
    """Requests queued on one matrix go out fused (their sequences concatenated,
    up to max_fused_k of them, or all when it is 0); the result is the same
    bits as applying them one after another."""
    A = wl.matrix(300, 260, seed=9)
    Ad = dev(A)
    exp = A
    with api.Server(hbm_budget_bytes=256 << 20, max_inflight=64, streams=4, max_batch=64,
                    max_fused_k=max_fused_k) as srv:
        h = srv.register(Ad)
        reqs = [wl.rotations(260, 3 + (q * 7) % 29, seed=90 + q) for q in range(24)]
        ts = [srv.submit(h, C, S) for (C, S) in reqs]     # a burst: later ones queue
        for t in ts:
            srv.wait(t, 60000)
        st = srv.stats()
        for (C, S) in reqs:
            exp = oracle.rot_sequence(exp, C, S)
        assert st["completed"] == 24
        if max_fused_k == 0:
            assert st["launches"] < 24       # queued requests were fused
    assert np.array_equal(bits(Ad.cpu().numpy()), bits(exp))


def test_host_wait_runs_out_then_completes(api):
    with api.Server(hbm_budget_bytes=512 << 20, max_inflight=4, streams=2, max_batch=4) as srv:
        A = dev(wl.matrix(2048, 2048, seed=4))
        h = srv.register(A)
        ts = []
        for q in range(12):               # serialised on one matrix: tens of ms in total
            C, S = wl.rotations(2048, 64, seed=40 + q)
            ts.append(srv.submit(h, C, S))
        assert srv.try_wait(ts[-1], 0) == 4   # ROT_ETIMEOUT: still queued behind the others
        for t in ts:
            srv.wait(t, 120000)


def test_destroy_drains_submitted_work(api):
    A = wl.matrix(256, 256, seed=6)
    Ad = dev(A)
    exp = A
    srv = api.Server(hbm_budget_bytes=64 << 20, max_inflight=4, streams=2, max_batch=2)
    h = srv.register(Ad)
    for q in range(5):
        C, S = wl.rotations(256, 17, seed=60 + q)
        srv.submit(h, C, S)
        exp = oracle.rot_sequence(exp, C, S)
    srv.close()                           # no wait: destroy must finish them
    assert np.array_equal(bits(Ad.cpu().numpy()), bits(exp))


def test_wide_and_narrow_matrices_mixed_equal_sequential_oracle(api):
    """Matrices of wide_rows rows or more go out in launches of their own (one
    at a time, one CTA per SM); small ones in other launches beside them.  Every
    matrix still ends equal to the oracle's sequential application, and each
    request reports a latency."""
    r = np.random.default_rng(17)
    shapes = [(1024, 300), (1100, 257), (128, 128), (64, 200), (256, 256), (1024, 64)]
    mats = [wl.matrix(m, n, seed=700 + i) for i, (m, n) in enumerate(shapes)]
    devm = [dev(A) for A in mats]
    expected = [A.copy() for A in mats]
    reqs = []
    for q in range(60):
        i = int(r.integers(0, len(shapes)))
        k = int(r.integers(2, 40))
        reqs.append((i,) + wl.rotations(shapes[i][1], k, seed=9500 + q))
    with api.Server(hbm_budget_bytes=512 << 20, max_inflight=16, streams=4, max_batch=6, wide_rows=1024) as srv:
        handles = [srv.register(A) for A in devm]
        tickets = [srv.submit(handles[i], C, S) for (i, C, S) in reqs]
        lat = [srv.wait_latency(t, 60000) for t in tickets]
        assert all(x > 0 for x in lat)
        st = srv.stats()
        assert st["completed"] == 60 and st["pending"] == 0 and st["inflight"] == 0
    for (i, C, S) in reqs:
        expected[i] = oracle.rot_sequence(expected[i], C, S)
    for A, E in zip(devm, expected):
        assert np.array_equal(bits(A.cpu().numpy()), bits(E))
