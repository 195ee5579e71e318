"""Write the oracle's expected values for the parity tests.

Calls only ``oracle`` and the seeded input generators in ``workloads``; no
value here comes from the GPU path. Usage:

    python tests/golden/make_golden.py cfg1 cfg2 cfg3_erfc cfg3_erf cfg4

Each config writes ``tests/golden/<name>.npz`` with E_x, the AO-occupied
block KC[k, mu, i] and (for erfc/erf kernels) dE_x/d omega.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from workloads import config  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def solve(w):
    t0 = time.time()
    chi = O.bloch_aos(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha, w.kfrac,
                      grid=w.grid)
    psi = O.orbitals_on_grid(chi, w.C)
    g0 = O.g0_value(w.kernel, w.omega, w.g0_mode)
    y = O.occri_kc(w.lattice, w.grid, w.kfrac, psi, None, w.kernel, w.omega, g0)
    kc = O.contract_kc(w.lattice, chi, y)
    del chi
    _, m, ex = O.ace_assemble(w.C, kc)
    out = dict(ex=np.array(ex), kc=kc, m=m, nao=np.array(w.nao), nk=np.array(w.nk))
    if w.kernel in ("erfc", "erf"):
        out["domega"] = np.array(O.grad_omega(w.lattice, w.grid, w.kfrac, psi, w.kernel,
                                              w.omega, w.g0_mode))
    print(f"{w.name}: E_x = {ex:.12f}  ({time.time() - t0:.1f} s)", flush=True)
    return out


def main(names):
    for name in names:
        ws = config(name)
        if isinstance(ws, list):
            for w in ws:
                np.savez(os.path.join(HERE, w.name + ".npz"), **solve(w))
        else:
            np.savez(os.path.join(HERE, name + ".npz"), **solve(ws))


if __name__ == "__main__":
    main(sys.argv[1:] or ["cfg1", "cfg2"])
