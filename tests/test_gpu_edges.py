"""Every compiled grid edge through the C ABI against the FP64 oracle with explicit DFTs.

The pair passes are compiled once per cubic edge (a radix plan, plane pitches and launch
shapes per edge), so each edge is its own code. Each case is a small 2-atom cell on a
1x1x2 k-mesh (a diagonal wave with q = 0 and an off-diagonal one with q = (0, 0, 1/2)),
built on the GPU in FP64 and in mixed precision, and compared with the oracle whose
transforms are explicit separable DFT-matrix products (no FFT library on either side).

The 60^3 edge, which the paper-scale bench runs, gets more: nocc 8 (an off-diagonal wave
of 64 fields, the same launch shape as every off-diagonal wave of the 6x6x6-k, 350-AO
bench cell), nocc 12 (the mixed path's separate inverse and bulk-copy accumulation), a
Gamma-only cell with s, p, d and f shells, and the FFT-mode oracle beside the DFT one.

Tolerances: FP64 max|dK| <= 1e-10 max|K| and |dE_x| <= 1e-10 |E_x|; mixed max|dK| <= 1e-5
Ha and |dE_x| <= 1e-6 Ha.
"""
import functools

import numpy as np
import pytest

import oracle as O
from workloads import small_workload

pytestmark = pytest.mark.gpu

EDGES = [8, 9, 10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 36, 40, 45, 48, 50, 54, 60, 64]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2207_09028_gb300 as occri
    occri.load_library()
    return torch


def _edge_workload(n, nocc=2, mesh=(1, 1, 2), counts=(1, 1), a_ang=3.0):
    return small_workload(mesh=mesh, grid=(n, n, n), counts=counts, nocc=nocc, a_ang=a_ang,
                          seed=500 + n)


@functools.lru_cache(maxsize=None)
def _oracle(n, nocc=2, mesh=(1, 1, 2), counts=(1, 1), a_ang=3.0, dft=True):
    w = _edge_workload(n, nocc, mesh, counts, a_ang)
    chi = O.bloch_aos(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha, w.kfrac,
                      grid=w.grid)
    psi = O.orbitals_on_grid(chi, w.C)
    kc = O.occri_kc(w.lattice, w.grid, w.kfrac, psi, chi, w.kernel, w.omega, 0.0, dft=dft)
    k, _, ex = O.ace_assemble(w.C, kc)
    return dict(kc=kc, k=k, ex=ex)


def _gpu(torch, w, precision):
    import paper_2207_09028_gb300 as occri
    plan = occri.Plan.from_workload(w, precision=precision)
    C = torch.from_numpy(w.C).cuda()
    KC, K, Ex = plan.build(C)
    out = dict(kc=KC.cpu().numpy(), k=K.cpu().numpy(), ex=float(Ex.cpu()[0]),
               tc=plan.contraction_tc)
    plan.close()
    return out


def _check(got, ref, precision, what):
    dk = np.abs(got["k"] - ref["k"]).max()
    de = abs(got["ex"] - ref["ex"])
    if precision == "fp64":
        assert dk <= 1e-10 * np.abs(ref["k"]).max(), (what, dk)
        assert np.abs(got["kc"] - ref["kc"]).max() <= 1e-10 * np.abs(ref["kc"]).max(), what
        assert de <= 1e-10 * abs(ref["ex"]), (what, de)
    else:
        assert dk <= 1e-5, (what, dk)
        assert de <= 1e-6, (what, got["ex"], ref["ex"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n", EDGES)
def test_every_edge_matches_explicit_dft_oracle(torch_cuda, n, precision):
    w = _edge_workload(n)
    _check(_gpu(torch_cuda, w, precision), _oracle(n), precision, f"edge {n}")


# the tensor-core contraction reads the grid through tiles of 32 points: a few edges with
# ragged last tiles (9^3, 25^3, 45^3) and exact ones, on the bench cell's lattice constant
# (a supercell large enough for the tensor-core path, which the plan must report)
@pytest.mark.parametrize("n", [9, 24, 25, 45, 48])
def test_tensor_core_contraction_edges(torch_cuda, n):
    w = _edge_workload(n, a_ang=5.43)
    got = _gpu(torch_cuda, w, "mixed_tc")
    assert got["tc"]
    _check(got, _oracle(n, a_ang=5.43), "mixed_tc", f"edge {n}")


# ------------------------------------------------------------------ the bench's edge, 60^3

# the bench cell's lattice constant (5.43 A), so that E_x is of the bench cell's size
BENCH_EDGE_CASES = [
    dict(nocc=8, mesh=(1, 1, 2), counts=(2, 1, 1)),       # 64-field off-diagonal wave
    dict(nocc=12, mesh=(1, 1, 2), counts=(2, 1, 1)),      # nocc > 8: pass C + bulk pass D
    dict(nocc=8, mesh=(1, 1, 1), counts=(2, 1, 1, 1)),    # s, p, d, f shells at Gamma
]


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_tc"])
@pytest.mark.parametrize("case", range(len(BENCH_EDGE_CASES)))
def test_bench_edge_60_matches_oracle(torch_cuda, case, precision):
    c = BENCH_EDGE_CASES[case]
    w = _edge_workload(60, c["nocc"], c["mesh"], c["counts"], 5.43)
    key = (60, c["nocc"], c["mesh"], c["counts"], 5.43)
    ref = _oracle(*key, dft=True)
    if case == 0:   # the two oracle transforms agree with each other first
        ref_fft = _oracle(*key, dft=False)
        assert np.abs(ref_fft["kc"] - ref["kc"]).max() <= 1e-12 * np.abs(ref["kc"]).max()
    got = _gpu(torch_cuda, w, precision)
    if precision == "mixed_tc" and c["mesh"] != (1, 1, 1):
        assert got["tc"]
    _check(got, ref, precision, f"60^3 case {c}")
