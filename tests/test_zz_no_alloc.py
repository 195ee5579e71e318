"""occri_orbitals_noalloc: the orbital stage for callers that cannot allocate device
memory during the call. It must
give what the allocating entry point occri_orbitals gives, call after call, although
every call reuses the library's one static scratch array.

This file is named to be collected last, so that a run stopping at its first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from workloads import small_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2207_09028_gb300 as occri
    occri.load_library()
    return torch


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-6)])
def test_noalloc_orbitals_match_allocating_entry_point(torch_cuda, precision, tol):
    import paper_2207_09028_gb300 as occri
    torch = torch_cuda
    lib = occri.load_library()
    w = small_workload(mesh=(2, 1, 2), counts=(2, 2, 1, 1), grid=(12, 12, 12), nocc=3, seed=21)
    plan = occri.Plan.from_workload(w, precision=precision)
    C = torch.from_numpy(w.C).cuda()
    ref = plan.orbitals(C).cpu().numpy()
    scale = np.abs(ref).max()
    for call in range(2):
        out = torch.full((w.nk, w.nocc) + tuple(w.grid), float("nan"), dtype=torch.complex128,
                         device=C.device)
        plan.set_stream()
        st = lib.occri_orbitals_noalloc(plan._h, ctypes.c_void_p(C.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()))
        assert st == occri.OCCRI_OK, (call, st)
        plan.sync()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert np.abs(got - ref).max() <= tol * scale, (call, np.abs(got - ref).max())


def test_noalloc_rejects_problems_beyond_the_static_array(torch_cuda):
    import paper_2207_09028_gb300 as occri
    torch = torch_cuda
    lib = occri.load_library()
    # 8 k x 8 orbitals x 48^3 points x 8 B = 56.6 MB of FP32 orbitals > 32 MiB
    w = small_workload(mesh=(2, 2, 2), counts=(2, 1, 1), grid=(48, 48, 48), nocc=8, seed=2)
    plan = occri.Plan.from_workload(w, precision="mixed")
    C = torch.from_numpy(w.C).cuda()
    out = torch.zeros((w.nk, w.nocc) + tuple(w.grid), dtype=torch.complex128, device=C.device)
    st = lib.occri_orbitals_noalloc(plan._h, ctypes.c_void_p(C.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()))
    assert st == occri.OCCRI_EINVAL
    plan.sync()
    assert float(out.abs().max().cpu()) == 0.0
