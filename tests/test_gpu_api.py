"""Entry points beyond the plain build, through the C ABI on the GPU:

* occri_k_build_once (the one-shot signature) gives what a plan's build gives;
* exchange_build, the differentiable (K, E_x) of one build, whose backward runs
  occri_vjp_full: a loss on K and E_x differentiated by autograd matches central
  differences of the FP64 oracle in C and in omega;
* the error paths, with the failures made on purpose but without any fault of the GPU:
  a bounded device wait that runs out (OCCRI_ETIMEOUT from occri_plan_sync; the copy
  producer issues nothing, so no copy is ever in flight) and a device allocation that
  fails (OCCRI_ENOMEM), each followed by normal builds on the same plan or process.
"""
import numpy as np
import pytest

import oracle as O
from workloads import small_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2207_09028_gb300 as occri
    occri.load_library()
    return torch


def test_build_once_matches_plan_build(torch_cuda):
    import paper_2207_09028_gb300 as occri
    torch = torch_cuda
    w = small_workload(mesh=(1, 1, 2), grid=(12, 12, 12), counts=(2, 1), nocc=2, seed=61)
    C = torch.from_numpy(w.C).cuda()
    for prec in ("fp64", "mixed"):
        plan = occri.Plan.from_workload(w, precision=prec)
        _, K, Ex = plan.build(C)
        plan.close()
        K1, Ex1 = occri.build_once(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha,
                                   w.kfrac, C, w.nocc, w.grid, w.kernel, w.omega, w.g0_mode,
                                   precision=prec)
        torch.cuda.synchronize()
        # the same kernels; only the order of the FP64 atomic sums may differ
        assert torch.allclose(K, K1, rtol=1e-12, atol=1e-15) and torch.allclose(Ex, Ex1, rtol=1e-12), prec


def test_build_once_reports_errors(torch_cuda):
    import paper_2207_09028_gb300 as occri
    torch = torch_cuda
    w = small_workload(mesh=(1, 1, 2), grid=(8, 8, 8), counts=(2, 1), nocc=2, seed=3)
    C = w.C.copy()
    C[1, :, 1] = C[1, :, 0]   # rank-deficient at k = 1
    with pytest.raises(occri.OccriError) as e:
        occri.build_once(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha, w.kfrac,
                         torch.from_numpy(C).cuda(), w.nocc, w.grid, precision="fp64")
    assert e.value.status == occri.OCCRI_ENOTPD
    with pytest.raises(occri.OccriError) as e:
        occri.build_once(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha, w.kfrac,
                         torch.from_numpy(w.C).cuda(), w.nocc, (8, 8, 7), precision="fp64")
    assert e.value.status == occri.OCCRI_EINVAL


# ------------------------------------------------------------------ autograd through K and E_x

def _oracle_loss(w, C, G, a):
    """L = Re sum conj(G) K + a E_x, from the FP64 oracle."""
    chi = O.bloch_aos(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha, w.kfrac,
                      grid=w.grid)
    psi = O.orbitals_on_grid(chi, C)
    g0 = O.g0_value(w.kernel, w.omega, w.g0_mode)
    kc = O.occri_kc(w.lattice, w.grid, w.kfrac, psi, chi, w.kernel, w.omega, g0)
    k, _, ex = O.ace_assemble(C, kc)
    return float(np.real(np.sum(np.conj(G) * k))) + a * ex


@pytest.mark.parametrize("kind,g0_mode", [("erfc", 1), ("coulomb", 0)])
def test_exchange_build_autograd_matches_oracle_differences(torch_cuda, kind, g0_mode):
    import paper_2207_09028_gb300 as occri
    torch = torch_cuda
    omega = 0.4 if kind != "coulomb" else 0.0
    w = small_workload(mesh=(1, 2, 1), grid=(9, 9, 9), counts=(2, 1), nocc=2, kernel=kind,
                       omega=omega, g0_mode=g0_mode, seed=71)
    rng = np.random.default_rng(11)
    G = rng.standard_normal((w.nk, w.nao, w.nao)) + 1j * rng.standard_normal((w.nk, w.nao, w.nao))
    a = 0.7
    plan = occri.Plan.from_workload(w, precision="fp64")
    C = torch.from_numpy(w.C).cuda().requires_grad_(True)
    om = torch.tensor(omega, dtype=torch.float64, requires_grad=True) if kind != "coulomb" else None
    K, Ex = occri.exchange_build(plan, C, om)
    loss = (torch.conj(torch.from_numpy(G).cuda()) * K).real.sum() + a * Ex
    loss.backward()
    gC = C.grad.cpu().numpy()
    assert abs(float(loss) - _oracle_loss(w, w.C, G, a)) <= 1e-10 * abs(float(loss))
    h = 1e-5
    for trial in range(2):
        d = rng.standard_normal(w.C.shape) + 1j * rng.standard_normal(w.C.shape)
        fd = (_oracle_loss(w, w.C + h * d, G, a) - _oracle_loss(w, w.C - h * d, G, a)) / (2 * h)
        an = float(np.real(np.sum(np.conj(gC) * d)))
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-3), (trial, fd, an)
    if om is not None:
        fdw = (_oracle_loss(w.with_kernel(kind, omega + h, g0_mode), w.C, G, a) -
               _oracle_loss(w.with_kernel(kind, omega - h, g0_mode), w.C, G, a)) / (2 * h)
        assert abs(float(om.grad) - fdw) <= 1e-6 * abs(fdw), (float(om.grad), fdw)


def test_exchange_build_backward_after_another_build(torch_cuda):
    """backward rebuilds when the plan ran another build since the forward."""
    import paper_2207_09028_gb300 as occri
    torch = torch_cuda
    w = small_workload(mesh=(1, 1, 2), grid=(9, 9, 9), counts=(2, 1), nocc=2, seed=72)
    plan = occri.Plan.from_workload(w, precision="fp64")
    C = torch.from_numpy(w.C).cuda().requires_grad_(True)
    _, Ex = occri.exchange_build(plan, C)
    Ex.backward()
    g_ref = C.grad.clone()
    C.grad = None
    _, Ex = occri.exchange_build(plan, C)
    other = small_workload(mesh=(1, 1, 2), grid=(9, 9, 9), counts=(2, 1), nocc=2, seed=73)
    plan.build(torch.from_numpy(other.C).cuda(), want_k=False)
    Ex.backward()
    assert torch.allclose(C.grad, g_ref, rtol=1e-12, atol=0)
    # and the E_x seed alone reproduces (4/N_k) K_{mu i}
    KC, _, _ = plan.build(C.detach())
    assert torch.allclose(g_ref, 4.0 / w.nk * KC, rtol=1e-11, atol=1e-14)


# ------------------------------------------------------------------ error paths

def test_device_wait_timeout_is_reported_and_plan_recovers(torch_cuda):
    """OCCRI_FAULT_WAIT: the bulk-copy producers issue nothing, every consumer's bounded
    wait gives up after 50 ms, and occri_plan_sync returns OCCRI_ETIMEOUT. The next builds
    on the same plan are exact again."""
    import paper_2207_09028_gb300 as occri
    torch = torch_cuda
    # FP64 waves of nocc <= 8 accumulate through the bulk-copy pass
    w = small_workload(mesh=(1, 1, 2), grid=(12, 12, 12), counts=(2, 1), nocc=2, seed=81)
    plan = occri.Plan.from_workload(w, precision="fp64")
    C = torch.from_numpy(w.C).cuda()
    KC0, K0, Ex0 = plan.build(C)
    plan.inject_fault(occri.OCCRI_FAULT_WAIT, 50.0)
    with pytest.raises(occri.OccriError) as e:
        plan.build(C)
    assert e.value.status == occri.OCCRI_ETIMEOUT
    plan.inject_fault(occri.OCCRI_FAULT_NONE, 2000.0)
    for _ in range(2):
        KC1, K1, Ex1 = plan.build(C)
        assert torch.allclose(KC1, KC0, rtol=1e-12, atol=1e-15)
        assert torch.allclose(K1, K0, rtol=1e-12, atol=1e-15)
        assert torch.allclose(Ex1, Ex0, rtol=1e-12)


def test_inject_fault_rejects_bad_arguments(torch_cuda):
    import paper_2207_09028_gb300 as occri
    w = small_workload(mesh=(1, 1, 1), grid=(8, 8, 8), counts=(2, 1), nocc=2, seed=82)
    plan = occri.Plan.from_workload(w, precision="fp64")
    for fault, ms in ((7, 10.0), (occri.OCCRI_FAULT_WAIT, 0.0), (occri.OCCRI_FAULT_WAIT, 1e9)):
        with pytest.raises(occri.OccriError) as e:
            plan.inject_fault(fault, ms)
        assert e.value.status == occri.OCCRI_EINVAL


@pytest.mark.parametrize("nth", [1, 4, 12])
def test_allocation_failure_in_plan_create(torch_cuda, nth):
    import paper_2207_09028_gb300 as occri
    torch = torch_cuda
    w = small_workload(mesh=(1, 1, 2), grid=(8, 8, 8), counts=(2, 1), nocc=2, seed=83)
    free0 = torch.cuda.mem_get_info()[0]
    occri.fail_allocation(nth)
    try:
        with pytest.raises(occri.OccriError) as e:
            occri.Plan.from_workload(w, precision="mixed")
        assert e.value.status == occri.OCCRI_ENOMEM
    finally:
        occri.fail_allocation(0)
    torch.cuda.synchronize()
    # what the failed creation took is given back (allow for allocator granularity)
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)
    plan = occri.Plan.from_workload(w, precision="mixed")
    plan.build(torch.from_numpy(w.C).cuda())


def test_allocation_failure_in_adjoint_and_host_staging(torch_cuda):
    import paper_2207_09028_gb300 as occri
    torch = torch_cuda
    w = small_workload(mesh=(1, 1, 2), grid=(8, 8, 8), counts=(2, 1), nocc=2, seed=84)
    plan = occri.Plan.from_workload(w, precision="fp64")
    C = torch.from_numpy(w.C).cuda()
    KC, _, _ = plan.build(C)
    for nth in (1, 3):
        occri.fail_allocation(nth)
        try:
            with pytest.raises(occri.OccriError) as e:
                plan.vjp_full(C, 1.0)
            assert e.value.status == occri.OCCRI_ENOMEM
        finally:
            occri.fail_allocation(0)
    g = plan.vjp_full(C, 1.0)
    assert torch.allclose(g, 4.0 / w.nk * KC, rtol=1e-11, atol=1e-14)
    occri.fail_allocation(2)
    try:
        with pytest.raises(occri.OccriError) as e:
            plan.k_build_host(w.C)
        assert e.value.status == occri.OCCRI_ENOMEM
    finally:
        occri.fail_allocation(0)
    kc, _, _ = plan.k_build_host(w.C)
    assert np.allclose(kc, KC.cpu().numpy(), rtol=1e-12, atol=1e-15)
