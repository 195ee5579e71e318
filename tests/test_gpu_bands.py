"""The paper's form of the assembly (Sec. II.C, Eq. occrikop) and the conduction-band
columns (Sec. II.D) through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from workloads import small_workload
from workloads.synthetic import analytic_overlap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

occri = pytest.importorskip("paper_2207_09028_gb300")

# K-level bars: FP64 relative to max|K|; mixed |dK| <= 1e-5 Ha
TOL_K = {"fp64": 1e-10, "mixed": 1e-5}


def _chi(w):
    return O.bloch_aos(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha, w.kfrac,
                       grid=w.grid)


def _g0(w):
    return O.g0_value(w.kernel, w.omega, w.g0_mode)


def _overlap(w):
    return analytic_overlap(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha, w.kfrac)


def _sub(w, C, nocc):
    """The same workload with other orbitals (C [nk, nao, nocc])."""
    from dataclasses import replace
    return replace(w, C=np.ascontiguousarray(C), nocc=nocc)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mesh,kind,omega,g0_mode", [((1, 1, 1), "coulomb", 0.0, 0),
                                                     ((1, 2, 1), "erfc", 0.5, 1)])
def test_paper_assembly_matches_oracle(prec, mesh, kind, omega, g0_mode):
    w = small_workload(mesh=mesh, grid=(9, 9, 9), nocc=3, kernel=kind, omega=omega,
                       g0_mode=g0_mode)
    plan = occri.Plan.from_workload(w, precision=prec)
    C = torch.from_numpy(w.C).cuda()
    KC, _, _ = plan.build(C, want_k=False)
    S = torch.from_numpy(_overlap(w)).cuda()
    K = plan.assemble_paper(S, C, KC)
    torch.cuda.synchronize()
    k_gpu = K.cpu().numpy()
    # the assembly alone: the oracle's formula on the GPU's own KC, to FP64 rounding
    ref_same = O.assemble_paper(_overlap(w), w.C, KC.cpu().numpy())
    assert np.abs(k_gpu - ref_same).max() < 1e-12 * np.abs(ref_same).max()
    # the whole chain against the oracle's Algorithm 3
    psi = O.orbitals_on_grid(_chi(w), w.C)
    kc_ref = O.occri_kc(w.lattice, w.grid, w.kfrac, psi, _chi(w), w.kernel, w.omega, _g0(w))
    ref = O.assemble_paper(_overlap(w), w.C, kc_ref)
    bar = TOL_K[prec] * (np.abs(ref).max() if prec == "fp64" else 1.0)
    assert np.abs(k_gpu - ref).max() < bar
    # K C = KC + S C (M_raw^H - M): exact on the occupied space up to the anti-Hermitian part
    # of M_raw = C^H KC (rounding of KC; zero in exact arithmetic)
    kcg = KC.cpu().numpy()
    ovl = _overlap(w)
    for k in range(w.nk):
        m_raw = np.conj(w.C[k].T) @ kcg[k]
        m = 0.5 * (m_raw + np.conj(m_raw.T))
        want = kcg[k] + ovl[k] @ w.C[k] @ (np.conj(m_raw.T) - m)
        assert np.abs(k_gpu[k] @ w.C[k] - want).max() < 1e-12 * np.abs(kcg).max()
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_conduction_columns_match_oracle(prec):
    nocc, nr = 3, 2
    w = small_workload(mesh=(1, 2, 1), grid=(9, 9, 9), nocc=nocc + nr)
    plan_all = occri.Plan.from_workload(w, precision=prec)
    w_r = _sub(w, w.C[:, :, nocc:], nr)
    plan_r = occri.Plan.from_workload(w_r, precision=prec)
    C = torch.from_numpy(w.C).cuda()
    kcr = plan_all.k_build_conduction(plan_r, C).cpu().numpy()
    chi = _chi(w)
    psi = O.orbitals_on_grid(chi, w.C)
    ref = O.occri_kc(w.lattice, w.grid, w.kfrac, psi, chi, w.kernel, w.omega, _g0(w),
                     nsum=nocc)[:, :, nocc:]
    bar = TOL_K[prec] * (np.abs(ref).max() if prec == "fp64" else 1.0)
    assert np.abs(kcr - ref).max() < bar
    plan_all.close()
    plan_r.close()


def test_conduction_rejects_plans_of_different_cells():
    w = small_workload(mesh=(1, 2, 1), grid=(9, 9, 9), nocc=4)
    plan_all = occri.Plan.from_workload(w, precision="fp64")
    w_r = small_workload(mesh=(1, 2, 1), grid=(10, 10, 10), nocc=2)
    plan_r = occri.Plan.from_workload(w_r, precision="fp64")
    C = torch.from_numpy(w.C).cuda()
    with pytest.raises(occri.OccriError) as e:
        plan_all.k_build_conduction(plan_r, C)
    assert e.value.status == occri.OCCRI_EINVAL
    plan_all.close()
    plan_r.close()
