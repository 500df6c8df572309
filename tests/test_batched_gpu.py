"""Batched persistent launch (many independent problems) against the oracle.

Each problem of a batch must come out bit-identical to the oracle and to a
rot_apply call on that problem alone (rows of different problems never meet,
and within a problem every element sees the same operations in the same
order).
"""
import numpy as np
import pytest

import oracle
from paper_2412_01852_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_01852_gb300 as rs
    from paper_2412_01852_gb300 import build
    build.build()
    return rs


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def bits(x):
    return np.ascontiguousarray(x).view(np.uint64)


def uneven_shapes(seed, count):
    r = np.random.default_rng(seed)
    shapes = []
    for _ in range(count):
        m = int(r.integers(1, 300))
        n = int(r.integers(2, 200))
        k = int(r.integers(1, 40))
        shapes.append((m, n, k))
    shapes += [(0, 5, 3), (7, 1, 4), (9, 6, 0), (33, 2, 50), (64, 17, 16)]
    return shapes


def test_batched_bit_exact_against_oracle_and_alone(rs):
    from paper_2412_01852_gb300 import api
    shapes = uneven_shapes(3, 24)
    host, devs = [], []
    for i, (m, n, k) in enumerate(shapes):
        A, C, S = wl.problem(m, n, k, seed=1000 + i)
        host.append((A, C, S))
        devs.append((dev(A), dev(C), dev(S)))
    alone = []
    for (A, C, S) in host:
        Ad = dev(A)
        if A.size and A.shape[1] > 1 and C.shape[1] > 0:
            rs.rot_apply(Ad, dev(C), dev(S))
        alone.append(Ad)
    with api.BatchPlan(devs) as plan:
        info = plan.info()
        assert info["problems"] == sum(1 for (m, n, k) in shapes if m > 0 and n > 1 and k > 0)
        plan.execute()
    rs.rot_device_status()
    for (A, C, S), (Ad, _, _), Aal in zip(host, devs, alone):
        ref = oracle.rot_sequence(A, C, S)
        out = Ad.cpu().numpy()
        assert np.array_equal(bits(out), bits(ref))
        assert np.array_equal(bits(out), bits(Aal.cpu().numpy()))


def test_batched_cuda_graph_replay(rs):
    from paper_2412_01852_gb300 import api
    shapes = [(100, 80, 20), (33, 130, 5), (257, 40, 33)]
    host = [wl.problem(m, n, k, seed=77 + i) for i, (m, n, k) in enumerate(shapes)]
    devs = [(dev(A), dev(C), dev(S)) for (A, C, S) in host]
    plan = api.BatchPlan(devs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.execute()                       # first execution outside the capture
    torch.cuda.synchronize()
    for (Ad, _, _), (A, _, _) in zip(devs, host):
        Ad.copy_(dev(A))                     # reset A
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.execute()
    g.replay()
    torch.cuda.synchronize()
    rs.rot_device_status()
    for (Ad, _, _), (A, C, S) in zip(devs, host):
        assert np.array_equal(bits(Ad.cpu().numpy()), bits(oracle.rot_sequence(A, C, S)))
    g.replay()                               # a second replay applies the rotations again
    torch.cuda.synchronize()
    for (Ad, _, _), (A, C, S) in zip(devs, host):
        twice = oracle.rot_sequence(oracle.rot_sequence(A, C, S), C, S)
        assert np.array_equal(bits(Ad.cpu().numpy()), bits(twice))
    plan.close()


def test_batched_512_instance_recipe_sampled(rs):
    """512 instances, m log-uniform [64,4096], n log-uniform [32,2048], k uniform [1,96].

    Every instance runs in the batch; 16 of them are checked on 8 sampled rows
    each against the oracle (rows are independent), and against rot_apply alone.
    """
    from paper_2412_01852_gb300 import api
    shapes = wl.batch_shapes(512, seed=4)
    g = np.random.default_rng(4)
    check = set(g.choice(512, 16, replace=False).tolist()) | {int(np.argmax([m * n * k for m, n, k in shapes]))}
    devs, keep = [], {}
    for i, (m, n, k) in enumerate(shapes):
        A, C, S = wl.problem(m, n, k, seed=40000 + i)
        devs.append((dev(A), dev(C), dev(S)))
        if i in check:
            keep[i] = (A, C, S)
    plan = api.BatchPlan(devs)
    plan.execute()
    torch.cuda.synchronize()
    rs.rot_device_status()
    for i, (A, C, S) in keep.items():
        m = A.shape[0]
        rows = np.unique(np.concatenate([[0, m - 1], g.choice(m, min(m, 6), replace=False)]))
        ref = oracle.rot_sequence(A[rows], C, S)
        out = devs[i][0][torch.from_numpy(rows).cuda()].cpu().numpy()
        assert np.array_equal(bits(out), bits(ref)), i
        Aal = dev(A)
        rs.rot_apply(Aal, devs[i][1], devs[i][2])
        assert torch.equal(Aal, devs[i][0])
    plan.close()


def test_autotune_leaves_data_alone(rs):
    from paper_2412_01852_gb300 import api
    shapes = [(300, 200, 40), (64, 500, 16), (1000, 64, 8)]
    host = [wl.problem(m, n, k, seed=5 + i) for i, (m, n, k) in enumerate(shapes)]
    devs = [(dev(A), dev(C), dev(S)) for (A, C, S) in host]
    best, ms = api.batch_autotune(devs)
    assert best["K"] in (4, 8, 16) and best["NB"] in (32, 64, 128) and best["ctas_per_sm"] in (1, 2)
    assert ms > 0
    for (Ad, _, _), (A, _, _) in zip(devs, host):
        assert np.array_equal(bits(Ad.cpu().numpy()), bits(A))
    # A plan created without explicit tuning now picks the cached choice.
    with api.BatchPlan(devs) as plan:
        assert plan.info()["tuning"] == best
        plan.execute()
    rs.rot_device_status()
    for (Ad, _, _), (A, C, S) in zip(devs, host):
        assert np.array_equal(bits(Ad.cpu().numpy()), bits(oracle.rot_sequence(A, C, S)))


def test_autotuned_single_problem_drives_rot_apply(rs):
    """A batch of one problem tunes its shape; rot_apply then runs the wavefront
    kernel with the cached tiling and still equals the oracle bit for bit."""
    from paper_2412_01852_gb300 import api
    m, n, k = 300, 400, 48
    A, C, S = wl.problem(m, n, k, seed=71)
    Ad, Cd, Sd = dev(A), dev(C), dev(S)
    best, ms = api.batch_autotune([(Ad, Cd, Sd)])
    assert ms > 0 and best["K"] in (4, 8, 16)
    rs.rot_apply(Ad, Cd, Sd)
    rs.rot_device_status()
    assert np.array_equal(bits(Ad.cpu().numpy()), bits(oracle.rot_sequence(A, C, S)))


def test_batched_with_caller_workspace(rs):
    """rot_apply_batched_ws: caller-owned scratch, same bits as the oracle."""
    from paper_2412_01852_gb300 import api
    shapes = uneven_shapes(5, 16)
    host, devs = [], []
    for i, (m, n, k) in enumerate(shapes):
        A, C, S = wl.problem(m, n, k, seed=3000 + i)
        host.append((A, C, S))
        devs.append((dev(A), dev(C), dev(S)))
    nbytes = api.batched_workspace_size(devs)
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
    api.rot_apply_batched_ws(devs, ws)
    torch.cuda.synchronize()
    rs.rot_device_status()
    for (A, C, S), (Ad, _, _) in zip(host, devs):
        assert np.array_equal(bits(Ad.cpu().numpy()), bits(oracle.rot_sequence(A, C, S)))
