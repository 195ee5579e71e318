"""Seeded synthetic cells, bases, k-meshes and orbital coefficients.

The paper's workloads (Sec. III, computational details) are 2-atom fcc
semiconductors with large uncontracted Gaussian bases on a 6x6x6 k-mesh.
Their basis-set, pseudopotential and geometry data are not available here, so
every workload is synthetic: an fcc primitive cell with two identical atoms
at (0,0,0) and (1/4,1/4,1/4) (conventional-cubic reading), shells of real
solid-harmonic primitives with geometric exponent ladders, a Gamma-centred
mesh, and random orbital coefficients made orthonormal with Lowdin's method.

What lives here is input preparation only. The orthonormalisation uses the
analytic (Obara-Saika) overlap of the lattice-summed primitives, which the
exchange build never computes; the build itself accepts any full-rank C.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903

# Real solid-harmonic polynomials as monomial dictionaries {(a,b,c): coeff}
# for x^a y^b z^c, in AO order m = -l..l (p: x, y, z).
_POLY = {
    0: [{(0, 0, 0): 1.0}],
    1: [{(1, 0, 0): 1.0}, {(0, 1, 0): 1.0}, {(0, 0, 1): 1.0}],
    2: [
        {(1, 1, 0): 1.0},
        {(0, 1, 1): 1.0},
        {(0, 0, 2): 2.0, (2, 0, 0): -1.0, (0, 2, 0): -1.0},
        {(1, 0, 1): 1.0},
        {(2, 0, 0): 1.0, (0, 2, 0): -1.0},
    ],
    3: [
        {(2, 1, 0): 3.0, (0, 3, 0): -1.0},
        {(1, 1, 1): 1.0},
        {(0, 1, 2): 4.0, (2, 1, 0): -1.0, (0, 3, 0): -1.0},
        {(0, 0, 3): 2.0, (2, 0, 1): -3.0, (0, 2, 1): -3.0},
        {(1, 0, 2): 4.0, (3, 0, 0): -1.0, (1, 2, 0): -1.0},
        {(2, 0, 1): 1.0, (0, 2, 1): -1.0},
        {(3, 0, 0): 1.0, (1, 2, 0): -3.0},
    ],
}


@dataclasses.dataclass
class Workload:
    """One synthetic exchange-build problem (all lengths in bohr)."""

    name: str
    lattice: np.ndarray          # (3,3) rows a_1, a_2, a_3
    xyz: np.ndarray              # (natm,3)
    shell_atom: np.ndarray       # (nshell,) int32
    shell_l: np.ndarray          # (nshell,) int32
    shell_alpha: np.ndarray      # (nshell,) float64
    kfrac: np.ndarray            # (nk,3) fractional k-points
    nocc: int
    grid: Tuple[int, int, int]
    kernel: str                  # 'coulomb' | 'erfc' | 'erf'
    omega: float
    g0_mode: int                 # 0: drop G+q=0; 1: f(x->0) (erfc only)
    C: np.ndarray                # (nk,nao,nocc) complex128
    seed: int

    @property
    def nao(self) -> int:
        return int(np.sum(2 * self.shell_l + 1))

    @property
    def nk(self) -> int:
        return int(self.kfrac.shape[0])

    @property
    def ng(self) -> int:
        return int(np.prod(self.grid))

    def with_kernel(self, kernel: str, omega: float = 0.0, g0_mode: int = 0) -> "Workload":
        return dataclasses.replace(self, kernel=kernel, omega=omega, g0_mode=g0_mode)


def fcc_cell(a_angstrom: float) -> Tuple[np.ndarray, np.ndarray]:
    """fcc primitive vectors and a 2-atom (zincblende/diamond) basis, in bohr."""
    a = a_angstrom * BOHR_PER_ANGSTROM
    lattice = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    xyz = np.array([[0.0, 0.0, 0.0], [0.25 * a, 0.25 * a, 0.25 * a]])
    return lattice, xyz


def geometric_exponents(n: int, lo: float, hi: float) -> np.ndarray:
    """n exponents spaced geometrically over [lo, hi]; n == 1 gives sqrt(lo*hi)."""
    if n <= 0:
        return np.zeros(0)
    if n == 1:
        return np.array([math.sqrt(lo * hi)])
    j = np.arange(n, dtype=float)
    return lo * (hi / lo) ** (j / (n - 1))


def make_shells(natm: int, counts_per_l: Sequence[int], lo: float, hi: float):
    """Shell arrays in AO order: atom -> l ascending -> exponent ascending."""
    atom, ls, alpha = [], [], []
    for ia in range(natm):
        for l, n in enumerate(counts_per_l):
            for a in geometric_exponents(n, lo, hi):
                atom.append(ia)
                ls.append(l)
                alpha.append(a)
    return (np.array(atom, dtype=np.int32), np.array(ls, dtype=np.int32),
            np.array(alpha, dtype=np.float64))


def gamma_mesh(n1: int, n2: int, n3: int) -> np.ndarray:
    """Gamma-centred mesh kappa = j/n, index k = (j1*n2 + j2)*n3 + j3."""
    j = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    return (j.reshape(-1, 3) / np.array([n1, n2, n3], dtype=float)).astype(np.float64)


def random_coefficients(rng: np.random.Generator, nk: int, nao: int, nocc: int,
                        complex_: bool) -> np.ndarray:
    if complex_:
        x = (rng.standard_normal((nk, nao, nocc)) + 1j * rng.standard_normal((nk, nao, nocc)))
        return x / math.sqrt(2.0)
    return rng.standard_normal((nk, nao, nocc)).astype(np.complex128)


# ----------------------------------------------------------------------------
# analytic overlap of lattice-summed primitives (input preparation only)
# ----------------------------------------------------------------------------

def _os1d(la: int, lb: int, a: float, b: float, xab: np.ndarray) -> np.ndarray:
    """1-D Obara-Saika overlaps S[i,j] of x^i e^{-a(x-A)^2} and x^j e^{-b(x-B)^2}."""
    p = a + b
    xpa = -b / p * xab
    xpb = a / p * xab
    s = np.zeros((la + 1, lb + 1) + xab.shape)
    s[0, 0] = math.sqrt(math.pi / p) * np.exp(-a * b / p * xab * xab)
    for i in range(la + 1):
        for j in range(lb + 1):
            if i == 0 and j == 0:
                continue
            if i > 0:
                v = xpa * s[i - 1, j]
                if i > 1:
                    v = v + (i - 1) / (2 * p) * s[i - 2, j]
                if j > 0:
                    v = v + j / (2 * p) * s[i - 1, j - 1]
            else:
                v = xpb * s[i, j - 1]
                if j > 1:
                    v = v + (j - 1) / (2 * p) * s[i, j - 2]
            s[i, j] = v
    return s


def _shell_pair_overlap(l1: int, a: float, l2: int, b: float, dab: np.ndarray) -> np.ndarray:
    """Unnormalised overlaps [2l1+1, 2l2+1, n] for centre differences dab = A - B."""
    sx = _os1d(l1, l2, a, b, dab[:, 0])
    sy = _os1d(l1, l2, a, b, dab[:, 1])
    sz = _os1d(l1, l2, a, b, dab[:, 2])
    out = np.zeros((2 * l1 + 1, 2 * l2 + 1, dab.shape[0]))
    for m1, p1 in enumerate(_POLY[l1]):
        for e1, c1 in p1.items():
            for m2, p2 in enumerate(_POLY[l2]):
                for e2, c2 in p2.items():
                    out[m1, m2] += c1 * c2 * sx[e1[0], e2[0]] * sy[e1[1], e2[1]] * sz[e1[2], e2[2]]
    return out


def _norms(l: int, a: float) -> np.ndarray:
    s = _shell_pair_overlap(l, a, l, a, np.zeros((1, 3)))
    return 1.0 / np.sqrt(np.diagonal(s[:, :, 0]))


def _mesh_of(kfrac: np.ndarray, dmax: int = 64) -> np.ndarray:
    """Smallest per-axis n with n*kappa integral for every k-point."""
    out = []
    for ax in range(3):
        for n in range(1, dmax + 1):
            v = kfrac[:, ax] * n
            if np.all(np.abs(v - np.round(v)) < 1e-9):
                out.append(n)
                break
        else:
            raise ValueError("k-points are not on a rational mesh")
    return np.array(out)


def analytic_overlap(lattice, xyz, shell_atom, shell_l, shell_alpha, kfrac,
                     eps: float = 1e-17) -> np.ndarray:
    """S^k_{mu nu} = sum_T e^{i k.T} <phi_mu(r-A)|phi_nu(r-B-T)>, shape (nk,nao,nao)."""
    lattice = np.asarray(lattice, float)
    recip_t = np.linalg.inv(lattice)            # columns b_i/(2 pi)
    mesh = _mesh_of(kfrac)
    nbin = int(np.prod(mesh))
    nao = int(np.sum(2 * shell_l + 1))
    off = np.concatenate([[0], np.cumsum(2 * shell_l + 1)])
    s_bins = np.zeros((nbin, nao, nao))
    norms = [_norms(int(l), float(a)) for l, a in zip(shell_l, shell_alpha)]
    amin = float(np.min(shell_alpha))
    rmax_all = math.sqrt(-math.log(eps) / (amin / 2.0)) + 2.0
    bnorm = np.linalg.norm(recip_t, axis=0)
    nat = xyz.shape[0]
    for ia in range(nat):
        for ib in range(nat):
            dcen = xyz[ia] - xyz[ib]
            f0 = dcen @ recip_t
            nb = np.ceil(rmax_all * bnorm).astype(int) + 1
            grids = [np.arange(int(np.floor(f0[d])) - nb[d], int(np.ceil(f0[d])) + nb[d] + 1)
                     for d in range(3)]
            nn = np.stack(np.meshgrid(*grids, indexing="ij"), -1).reshape(-1, 3)
            dab = dcen[None, :] - nn @ lattice          # A - B - T
            dist = np.linalg.norm(dab, axis=1)
            keep = dist <= rmax_all
            nn, dab, dist = nn[keep], dab[keep], dist[keep]
            bins = np.mod(nn, mesh)
            bidx = (bins[:, 0] * mesh[1] + bins[:, 1]) * mesh[2] + bins[:, 2]
            sa = np.nonzero(shell_atom == ia)[0]
            sb = np.nonzero(shell_atom == ib)[0]
            for s1 in sa:
                l1, a1 = int(shell_l[s1]), float(shell_alpha[s1])
                for s2 in sb:
                    l2, a2 = int(shell_l[s2]), float(shell_alpha[s2])
                    mu = a1 * a2 / (a1 + a2)
                    r = math.sqrt(-math.log(eps) / mu) + 2.0
                    sel = dist <= r
                    if not np.any(sel):
                        continue
                    blk = _shell_pair_overlap(l1, a1, l2, a2, dab[sel])
                    blk *= norms[s1][:, None, None] * norms[s2][None, :, None]
                    acc = np.zeros((nbin, blk.shape[0], blk.shape[1]))
                    np.add.at(acc, bidx[sel], np.moveaxis(blk, 2, 0))
                    s_bins[:, off[s1]:off[s1 + 1], off[s2]:off[s2 + 1]] += acc
    lbins = np.stack(np.meshgrid(*[np.arange(m) for m in mesh], indexing="ij"), -1).reshape(-1, 3)
    phase = np.exp(2j * np.pi * (kfrac @ lbins.T))    # (nk, nbin)
    sk = (phase @ s_bins.reshape(nbin, -1)).reshape(kfrac.shape[0], nao, nao)
    return 0.5 * (sk + np.conj(np.swapaxes(sk, 1, 2)))


def lowdin_orthonormalize(x: np.ndarray, s: np.ndarray) -> np.ndarray:
    """C_k = X_k (X_k^H S^k X_k)^{-1/2}."""
    out = np.empty_like(x)
    for k in range(x.shape[0]):
        m = np.conj(x[k].T) @ s[k] @ x[k]
        m = 0.5 * (m + np.conj(m.T))
        w, u = np.linalg.eigh(m)
        out[k] = x[k] @ (u * (1.0 / np.sqrt(w))[None, :]) @ np.conj(u.T)
    return out


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def _build(name, a_ang, mesh, counts, lo, hi, nocc, grid, kernel, omega, g0_mode, seed,
           complex_c=True) -> Workload:
    lattice, xyz = fcc_cell(a_ang)
    sa, sl, sx = make_shells(2, counts, lo, hi)
    kfrac = gamma_mesh(*mesh)
    nao = int(np.sum(2 * sl + 1))
    rng = np.random.default_rng(seed)
    x = random_coefficients(rng, kfrac.shape[0], nao, nocc, complex_c)
    s = analytic_overlap(lattice, xyz, sa, sl, sx, kfrac)
    c = lowdin_orthonormalize(x, s)
    return Workload(name, lattice, xyz, sa, sl, sx, kfrac, nocc, tuple(grid), kernel, omega,
                    g0_mode, c, seed)


_CFG4 = [  # (a [A], mesh, shells/atom (s,p,d), nocc, grid)
    (3.57, (3, 3, 3), (6, 5, 1), 4, 30),
    (4.05, (3, 3, 2), (9, 5, 3), 4, 32),
    (5.43, (2, 2, 2), (9, 6, 5), 4, 36),
    (5.65, (2, 2, 2), (11, 8, 6), 8, 40),
    (6.48, (2, 2, 2), (11, 8, 8), 8, 45),
]


def config_names() -> List[str]:
    return ["cfg1", "cfg2", "cfg3_erfc", "cfg3_erf", "cfg4", "cfg5"]


def config(name: str):
    """Return the named workload (a list of five for 'cfg4')."""
    if name == "cfg1":
        return _build("cfg1", 5.43, (1, 1, 1), (7, 2), 0.1, 20.0, 4, (24, 24, 24),
                      "coulomb", 0.0, 0, 1010, complex_c=False)
    if name == "cfg2":
        return _build("cfg2", 5.43, (2, 2, 2), (9, 6, 5), 0.08, 30.0, 4, (36, 36, 36),
                      "coulomb", 0.0, 0, 1020)
    if name in ("cfg3_erfc", "cfg3_erf"):
        w = _build(name, 5.43, (4, 4, 4), (15, 10, 11), 0.08, 30.0, 4, (48, 48, 48),
                   "erfc", 0.11, 1, 1030)
        return w if name == "cfg3_erfc" else w.with_kernel("erf", 0.3, 0)
    if name == "cfg4":
        out = []
        for ic, (a, mesh, counts, nocc, g) in enumerate(_CFG4):
            out.append(_build(f"cfg4_cell{ic}", a, mesh, counts, 0.08, 30.0, nocc, (g, g, g),
                              "erfc", 0.11, 1, 1040 + ic))
        return out
    if name == "cfg5":
        return _build("cfg5", 5.43, (6, 6, 6), (20, 14, 10, 9), 0.06, 40.0, 8, (60, 60, 60),
                      "coulomb", 0.0, 0, 1050)
    raise KeyError(name)


def small_workload(name="small", a_ang=3.0, mesh=(1, 1, 1), counts=(2, 1), lo=0.3, hi=3.0,
                   nocc=2, grid=(8, 8, 8), kernel="coulomb", omega=0.0, g0_mode=0, seed=7,
                   complex_c=None) -> Workload:
    """A tiny workload for oracle pins and parity tests (same recipe, small sizes)."""
    if complex_c is None:
        complex_c = int(np.prod(mesh)) > 1
    return _build(name, a_ang, mesh, counts, lo, hi, nocc, grid, kernel, omega, g0_mode, seed,
                  complex_c=complex_c)
