"""Batches of uneven cells built by one CUDA-graph launch (occri_batch_*).

The five cells of the lattice-constant scan (3.57 to 6.48 A, 3x3x3 to 2x2x2 k, 52 to 150
AOs, 30^3 to 45^3 grids, erfc kernel) are built as one batch. Every cell must give what
its own plan gives alone and what the oracle gives (golden values written by
tests/golden/make_golden.py); replaying the captured graph must give the same again,
and new output buffers must trigger a new capture that is still right.
"""
import os

import numpy as np
import pytest

import oracle as O
from workloads import config

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# the same bars as the per-cell golden tests (test_gpu_parity.py)
E_TOL = {"fp64": lambda e: 1e-10 * abs(e), "mixed": lambda e: 1e-6}
K_TOL = {"fp64": lambda k: 1e-10 * np.abs(k).max(), "mixed": lambda k: 1e-5}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _golden(name):
    path = os.path.join(GOLDEN, name + ".npz")
    if not os.path.exists(path):
        pytest.skip(f"golden {name} not generated")
    return dict(np.load(path))


def _outputs(torch, pl):
    dev = torch.device("cuda")
    return (torch.empty((pl.nk, pl.nao, pl.nocc), dtype=torch.complex128, device=dev),
            torch.empty((pl.nk, pl.nao, pl.nao), dtype=torch.complex128, device=dev),
            torch.zeros(1, dtype=torch.float64, device=dev))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_of_uneven_cells_matches_cells_alone_and_oracle(torch_cuda, precision):
    import paper_2207_09028_gb300 as occri
    torch = torch_cuda
    cells = config("cfg4")
    plans = [occri.Plan.from_workload(w, precision=precision) for w in cells]
    Cs = [torch.from_numpy(w.C).cuda() for w in cells]

    alone = [pl.build(C) for pl, C in zip(plans, Cs)]
    batch = occri.Batch(plans)
    outs = [_outputs(torch, pl) for pl in plans]
    KCs, Ks, Exs = ([o[i] for o in outs] for i in range(3))
    batch.build(Cs, KCs, Ks, Exs)
    first = [(kc.cpu().numpy(), k.cpu().numpy(), float(e.cpu()[0])) for kc, k, e in zip(KCs, Ks, Exs)]

    for w, (kc_a, k_a, ex_a), (kc, k, ex) in zip(cells, alone, first):
        g = _golden(w.name)
        k_ref, _, _ = O.ace_assemble(w.C, g["kc"])
        # the batch is the same computation as the cell alone (FP64 sums may add in
        # another order)
        assert np.abs(kc - kc_a.cpu().numpy()).max() <= 1e-12 * np.abs(kc).max(), w.name
        assert abs(ex - float(ex_a.cpu()[0])) <= 1e-12 * abs(ex), w.name
        # and it meets the oracle's golden values
        assert np.abs(k - k_ref).max() <= K_TOL[precision](k_ref), w.name
        assert abs(ex - float(g["ex"])) <= E_TOL[precision](float(g["ex"])), w.name

    # replay of the captured graph
    for t in Exs:
        t.zero_()
    batch.build(Cs, KCs, Ks, Exs)
    for (kc0, k0, ex0), kc, e in zip(first, KCs, Exs):
        assert np.abs(kc.cpu().numpy() - kc0).max() <= 1e-12 * np.abs(kc0).max()
        assert abs(float(e.cpu()[0]) - ex0) <= 1e-12 * abs(ex0)

    # new buffers (and no K output): a new capture
    Exs2 = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in plans]
    batch.build(Cs, None, None, Exs2)
    for (kc0, k0, ex0), e in zip(first, Exs2):
        assert abs(float(e.cpu()[0]) - ex0) <= 1e-12 * abs(ex0)
    batch.close()
    for pl in plans:
        pl.close()


def test_batch_mixes_precisions_and_reports_the_failing_cell(torch_cuda):
    """A batch may hold plans of different precision; a cell whose -C^H K C is not
    positive definite is reported with its index."""
    import paper_2207_09028_gb300 as occri
    torch = torch_cuda
    cells = config("cfg4")[2:4]
    plans = [occri.Plan.from_workload(cells[0], precision="fp64"),
             occri.Plan.from_workload(cells[1], precision="mixed")]
    Cs = [torch.from_numpy(w.C).cuda() for w in cells]
    Exs = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in plans]
    batch = occri.Batch(plans)
    batch.build(Cs, None, None, Exs)
    for w, e in zip(cells, Exs):
        g = _golden(w.name)
        assert abs(float(e.cpu()[0]) - float(g["ex"])) <= 1e-6
    # a zero orbital in cell 1, k = 1 makes C^H K C singular there
    bad = cells[1].C.copy()
    bad[1, :, 0] = 0.0
    Cs[1] = torch.from_numpy(bad).cuda()
    with pytest.raises(occri.OccriError) as err:
        batch.build(Cs, None, None, Exs)
    assert err.value.status == occri.OCCRI_ENOTPD and err.value.bad_k == 1
    assert "cell 1" in str(err.value)
    batch.close()
    for pl in plans:
        pl.close()
