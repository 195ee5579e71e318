"""The C ABI: the library loads, exports every symbol include/occri.h declares, and
rejects invalid problems on the host before touching the GPU (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2207_09028_gb300 as occri
from workloads import small_workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "occri.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(occri_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(occri.LIB_PATH):
        from paper_2207_09028_gb300 import _build
        _build.build()
    return occri.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_symbols()
    assert "occri_k_build" in names and "occri_plan_create" in names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(names) == sorted(occri.EXPORTED)


def test_status_strings(lib):
    for st in range(7):
        assert lib.occri_status_string(st).decode()
    assert lib.occri_status_string(99).decode() == "unknown status"


def _create(w, **over):
    args = dict(lattice=w.lattice, xyz=w.xyz, shell_atom=w.shell_atom, shell_l=w.shell_l,
                shell_alpha=w.shell_alpha, kfrac=w.kfrac, nocc=w.nocc, grid=w.grid,
                kernel=w.kernel, omega=w.omega, g0_mode=w.g0_mode, precision="fp64",
                stream=ctypes.c_void_p(0))
    args.update(over)
    return occri.Plan(**args)


@pytest.mark.parametrize("over,status", [
    (dict(nocc=0), occri.OCCRI_EINVAL),
    (dict(nocc=99), occri.OCCRI_EINVAL),
    (dict(grid=(7, 7, 7)), occri.OCCRI_EINVAL),
    (dict(grid=(3, 3, 3)), occri.OCCRI_EINVAL),
    (dict(grid=(70, 70, 70)), occri.OCCRI_EINVAL),
    (dict(shell_l=np.array([0, 4, 1, 0, 0, 1])), occri.OCCRI_EINVAL),
    (dict(shell_alpha=np.array([1.0, -1.0, 1.0, 1.0, 1.0, 1.0])), occri.OCCRI_EINVAL),
    (dict(kernel="erfc", omega=0.0), occri.OCCRI_EINVAL),
    (dict(kernel="erf", omega=0.3, g0_mode=1), occri.OCCRI_EINVAL),
    (dict(kernel="coulomb", g0_mode=1), occri.OCCRI_EINVAL),
    (dict(kernel="erf_trunc", omega=0.0), occri.OCCRI_EINVAL),
    (dict(kernel="erf_trunc", omega=0.3, g0_mode=2), occri.OCCRI_EINVAL),
    (dict(kernel=5, omega=0.3), occri.OCCRI_EINVAL),
    (dict(precision=7), occri.OCCRI_EINVAL),
    (dict(lattice=np.zeros((3, 3))), occri.OCCRI_EINVAL),
    (dict(shell_atom=np.array([1, 0, 0, 1, 1, 1])), occri.OCCRI_EINVAL),
    (dict(shell_atom=np.array([0, 0, 0, 1, 1, 2])), occri.OCCRI_EINVAL),
    (dict(grid=(8, 8, 12)), occri.OCCRI_EUNSUPPORTED),
    (dict(grid=(6, 6, 6)), occri.OCCRI_EUNSUPPORTED),
    (dict(kfrac=np.array([[1 / 97, 0, 0]])), occri.OCCRI_EUNSUPPORTED),
])
def test_invalid_problems_rejected_on_host(lib, over, status):
    w = small_workload(counts=(2, 1), nocc=2, grid=(8, 8, 8))
    assert list(w.shell_l) == [0, 0, 1, 0, 0, 1]
    with pytest.raises(occri.OccriError) as e:
        _create(w, **over)
    assert e.value.status == status


def test_null_arguments(lib):
    assert lib.occri_plan_destroy(None) == occri.OCCRI_EINVAL
    assert lib.occri_k_build(None, None, None, None, None) == occri.OCCRI_EINVAL
    assert lib.occri_vjp(None, None, 1.0, None, None) == occri.OCCRI_EINVAL
    assert lib.occri_plan_sync(None, None) == occri.OCCRI_EINVAL
    assert lib.occri_k_assemble_paper(None, 1, None, None, None, None) == occri.OCCRI_EINVAL
    assert lib.occri_k_build_conduction(None, None, None, None) == occri.OCCRI_EINVAL
    assert lib.occri_plan_autotune(None, 0, None) == occri.OCCRI_EINVAL
    assert lib.occri_plan_tuning(None, None) == occri.OCCRI_EINVAL
    assert lib.occri_plan_set_tuning(None, None) == occri.OCCRI_EINVAL


def test_batch_rejects_invalid_arguments_on_the_host(lib):
    """occri_batch_* check their arguments before any CUDA call."""
    vp = ctypes.c_void_p
    out = vp(123)
    assert lib.occri_batch_create(ctypes.byref(out), None, 1, None) == occri.OCCRI_EINVAL
    assert out.value is None
    none_plans = (vp * 2)(None, None)
    assert lib.occri_batch_create(ctypes.byref(out), none_plans, 2, None) == occri.OCCRI_EINVAL
    assert lib.occri_batch_create(ctypes.byref(out), none_plans, 0, None) == occri.OCCRI_EINVAL
    assert lib.occri_batch_create(None, none_plans, 2, None) == occri.OCCRI_EINVAL
    assert lib.occri_batch_build(None, none_plans, None, None, None) == occri.OCCRI_EINVAL
    cell, k = ctypes.c_int(0), ctypes.c_int(0)
    assert lib.occri_batch_sync(None, ctypes.byref(cell), ctypes.byref(k)) == occri.OCCRI_EINVAL
    assert cell.value == -1 and k.value == -1
    assert lib.occri_batch_destroy(None) == occri.OCCRI_EINVAL
