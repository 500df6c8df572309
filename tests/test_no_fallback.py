"""The product path has no CPU fallback: without the CUDA library, or given
host tensors, the binding raises instead of computing anything."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2412_01852_gb300 as rs
from paper_2412_01852_gb300 import _native
from paper_2412_01852_gb300 import workloads as wl


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "lib_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _native.load()


@pytest.mark.parametrize("fn,dtype", [(rs.rot_apply, torch.float64), (rs.rot_apply_f32, torch.float32)])
def test_host_tensors_are_refused(fn, dtype):
    A, C, S = wl.problem(40, 30, 5, seed=3)
    At = torch.from_numpy(np.asfortranarray(A)).to(dtype)
    Ct = torch.from_numpy(np.asfortranarray(C)).to(dtype)
    St = torch.from_numpy(np.asfortranarray(S)).to(dtype)
    before = At.clone()
    with pytest.raises(ValueError, match="CUDA tensor"):
        fn(At, Ct, St)
    assert torch.equal(At, before)
