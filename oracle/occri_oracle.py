"""Plain FP64 oracle of the occ-RI-K exact-exchange build (test infrastructure).

Conventions (the paper leaves them open; each is a reading of the cited passage):
* Bloch AOs chi_{mu k}(r) = sum_T e^{i k.T} phi_mu(r - A_mu - T), without the
  N_k^{-1/2} of Sec. II.A; the cell integral then carries an explicit 1/N_k.
* Grid r_n = sum_i (n_i/N_i) a_i with n_3 fastest; forward transform
  e^{-iG.r} with 1/N_g (numpy ``fftn``/N_g); bin m <-> G = sum_i m_i b_i.
* Pair density of (k,i) with (k',j), q = k - k':
  rho(r) = conj(psi_{jk'}(r)) psi_{ik}(r) e^{-iq.r}  (Eq. aodf),
  W(r) = e^{+iq.r} N_g IFFT[v_q . FFT(rho)/N_g]       (Eqs. Vrao, VGao),
  Y_{ik}(r) += psi_{jk'}(r) W(r)                        (Eq. occrikinterm),
  K_{mu i}(k) = -(Omega/(N_k N_g)) sum_n conj(chi_{mu k}) Y_{ik}  (Eq. occrik).
* Kernel per bin: x_i = m_i + q_i reduced to [-N_i/2, N_i/2); at an exact tie
  x_i = -N_i/2 both aliases are averaged; G+q = 0 takes the value g0.
* Closed shell: E_x = (1/N_k) sum_k Tr(C_k^H K_{mu i}(k)).

TEST INFRASTRUCTURE: imported only by tests, smoke() and bench.py's CPU legs.
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import Dict, List, Optional, Tuple

import numpy as np

__all__ = [
    "cell_volume", "reciprocal_vectors", "grid_points", "SOLID_HARMONICS",
    "eval_solid_harmonic", "gaussian_moment", "primitive_norms", "image_cutoff",
    "bloch_aos", "orbitals_on_grid", "grid_phase", "kernel_bins", "kernel_bins_domega",
    "g0_value", "apply_coulomb_operator", "occri_kc", "contract_kc", "mori_k", "aori_k",
    "ace_assemble", "exchange_energy", "exchange_energy_parseval", "grad_c",
    "grad_omega", "grid_overlap", "dft_matrices", "mesh_denominators", "supercell_lattice",
    "truncation_radius", "madelung_potential", "kernel_value", "assemble_paper",
]

EPS_AO = 1e-16   # AO screening threshold: terms below it are dropped (C10 reading)


# ----------------------------------------------------------------------------
# lattice and grid (Sec. II.A; GPW real-space grid, Sec. II.A eqs. aodf/Vrao)
# ----------------------------------------------------------------------------

def cell_volume(lattice: np.ndarray) -> float:
    return float(abs(np.linalg.det(np.asarray(lattice, float))))


def reciprocal_vectors(lattice: np.ndarray) -> np.ndarray:
    """Rows b_j with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, float)).T


def grid_points(lattice: np.ndarray, grid) -> np.ndarray:
    """r_n = sum_i (n_i/N_i) a_i, flattened with n_3 fastest -> (N_g, 3)."""
    n1, n2, n3 = grid
    f = np.stack(np.meshgrid(np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3,
                             indexing="ij"), -1).reshape(-1, 3)
    return f @ np.asarray(lattice, float)


# ----------------------------------------------------------------------------
# primitives: real solid harmonics x exact normalisation x Gaussian
# ----------------------------------------------------------------------------

# Unnormalised real solid harmonics P_lm, m = -l..l (p ordered x, y, z), as
# {(a,b,c): coeff} for x^a y^b z^c.
SOLID_HARMONICS: Dict[int, List[Dict[Tuple[int, int, int], float]]] = {
    0: [{(0, 0, 0): 1.0}],
    1: [{(1, 0, 0): 1.0}, {(0, 1, 0): 1.0}, {(0, 0, 1): 1.0}],
    2: [{(1, 1, 0): 1.0},                                    # xy
        {(0, 1, 1): 1.0},                                    # yz
        {(0, 0, 2): 2.0, (2, 0, 0): -1.0, (0, 2, 0): -1.0},  # 3z^2 - r^2
        {(1, 0, 1): 1.0},                                    # xz
        {(2, 0, 0): 1.0, (0, 2, 0): -1.0}],                  # x^2 - y^2
    3: [{(2, 1, 0): 3.0, (0, 3, 0): -1.0},                   # y(3x^2 - y^2)
        {(1, 1, 1): 1.0},                                    # xyz
        {(0, 1, 2): 4.0, (2, 1, 0): -1.0, (0, 3, 0): -1.0},  # y(4z^2 - x^2 - y^2)
        {(0, 0, 3): 2.0, (2, 0, 1): -3.0, (0, 2, 1): -3.0},  # z(2z^2 - 3x^2 - 3y^2)
        {(1, 0, 2): 4.0, (3, 0, 0): -1.0, (1, 2, 0): -1.0},  # x(4z^2 - x^2 - y^2)
        {(2, 0, 1): 1.0, (0, 2, 1): -1.0},                   # z(x^2 - y^2)
        {(3, 0, 0): 1.0, (1, 2, 0): -3.0}],                  # x(x^2 - 3y^2)
}


def eval_solid_harmonic(l: int, m_index: int, x, y, z):
    out = 0.0
    for (a, b, c), coeff in SOLID_HARMONICS[l][m_index].items():
        out = out + coeff * x ** a * y ** b * z ** c
    return out


def _double_factorial(n: int) -> int:
    out = 1
    while n > 1:
        out *= n
        n -= 2
    return out


def gaussian_moment(a: int, b: int, c: int, p: float) -> float:
    """Integral over R^3 of x^a y^b z^c exp(-p r^2)."""
    out = 1.0
    for e in (a, b, c):
        if e % 2:
            return 0.0
        out *= _double_factorial(e - 1) / (2.0 * p) ** (e // 2) * math.sqrt(math.pi / p)
    return out


def primitive_norms(l: int, alpha: float) -> np.ndarray:
    """N_lm with integral of (N_lm P_lm e^{-alpha r^2})^2 equal to 1, for m = -l..l."""
    out = []
    for poly in SOLID_HARMONICS[l]:
        sq = 0.0
        for e1, c1 in poly.items():
            for e2, c2 in poly.items():
                sq += c1 * c2 * gaussian_moment(e1[0] + e2[0], e1[1] + e2[1], e1[2] + e2[2],
                                                2.0 * alpha)
        out.append(1.0 / math.sqrt(sq))
    return np.array(out)


def image_cutoff(l: int, alpha: float, eps: float = EPS_AO) -> float:
    """Radius beyond which every primitive of the shell is below eps.

    Bound: |N_lm P_lm(d)| <= N_lm sum|coeff| |d|^l, so the radius solves
    c R^l e^{-alpha R^2} = eps on the decreasing side (R >= sqrt(l/(2 alpha))).
    """
    norms = primitive_norms(l, alpha)
    c = max(n * sum(abs(v) for v in poly.values())
            for n, poly in zip(norms, SOLID_HARMONICS[l]))
    lo = math.sqrt(l / (2.0 * alpha)) if l > 0 else 0.0
    f = lambda r: math.log(c) + l * math.log(max(r, 1e-300)) - alpha * r * r - math.log(eps)
    hi = max(lo, 1.0)
    while f(hi) > 0:
        hi *= 2.0
    if f(lo) <= 0:
        return lo
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
    return hi


# ----------------------------------------------------------------------------
# (a) Bloch AOs on the grid (Sec. II.A, first equation; C1 normalisation)
# ----------------------------------------------------------------------------

def _lattice_images(lattice, centre, radius):
    """Integer n with |centre + n.lattice| <= radius."""
    lattice = np.asarray(lattice, float)
    frac = np.asarray(centre, float) @ np.linalg.inv(lattice)
    bn = np.linalg.norm(np.linalg.inv(lattice), axis=0)
    nb = np.ceil(radius * bn).astype(int) + 1
    axes = [np.arange(int(np.floor(-frac[d])) - nb[d], int(np.ceil(-frac[d])) + nb[d] + 1)
            for d in range(3)]
    nn = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    d = centre[None, :] + nn @ lattice
    return nn[np.linalg.norm(d, axis=1) <= radius]


def bloch_aos(lattice, xyz, shell_atom, shell_l, shell_alpha, kfrac, grid=None,
              points=None, eps: float = EPS_AO) -> np.ndarray:
    """chi[k, mu, n] = sum_T e^{2 pi i kappa_k . n_T} phi_mu(r_n - A_mu - T).

    The image sum runs over every lattice translation T that brings the shell
    within its cutoff radius of a point; each (point, image) term below the
    threshold eps is dropped, per point.
    """
    lattice = np.asarray(lattice, float)
    pts = grid_points(lattice, grid) if points is None else np.asarray(points, float)
    kfrac = np.asarray(kfrac, float)
    nk, npts = kfrac.shape[0], pts.shape[0]
    nao = int(np.sum(2 * np.asarray(shell_l) + 1))
    chi = np.zeros((nk, nao, npts), dtype=np.complex128)
    centre = pts.mean(axis=0)
    rpts = float(np.max(np.linalg.norm(pts - centre, axis=1)))
    mu0 = 0
    for s in range(len(shell_l)):
        l, alpha = int(shell_l[s]), float(shell_alpha[s])
        a = np.asarray(xyz[shell_atom[s]], float)
        norms = primitive_norms(l, alpha)
        rcut = image_cutoff(l, alpha, eps)
        images = _lattice_images(lattice, a - centre, rcut + rpts)
        for n_t in images:
            t = n_t @ lattice
            d = pts - a[None, :] - t[None, :]
            r2 = np.einsum("ij,ij->i", d, d)
            idx = np.nonzero(r2 <= rcut * rcut)[0]
            if idx.size == 0:
                continue
            dx, dy, dz = d[idx, 0], d[idx, 1], d[idx, 2]
            g = np.exp(-alpha * r2[idx])
            phase = np.exp(2j * np.pi * (kfrac @ n_t))
            for m in range(2 * l + 1):
                val = norms[m] * eval_solid_harmonic(l, m, dx, dy, dz) * g
                chi[:, mu0 + m, idx] += phase[:, None] * val[None, :]
        mu0 += 2 * l + 1
    return chi


def orbitals_on_grid(chi: np.ndarray, C: np.ndarray) -> np.ndarray:
    """psi[k, i, n] = sum_mu C^k_{mu i} chi[k, mu, n]  (Eq. occmo)."""
    return np.einsum("kmi,kmn->kin", C, chi)


def grid_overlap(lattice, chi: np.ndarray, grid) -> np.ndarray:
    """S^k = (Omega/N_g) sum_n conj(chi_mu) chi_nu (GPW quadrature of the cell overlap)."""
    ng = int(np.prod(grid))
    return cell_volume(lattice) / ng * np.einsum("kmn,kvn->kmv", np.conj(chi), chi)


# ----------------------------------------------------------------------------
# (d) Fourier-space kernel per bin (Eqs. VGao, recipcoul; C3, C8)
# ----------------------------------------------------------------------------

def _frac(x: float, dmax: int = 1 << 20) -> Fraction:
    return Fraction(float(x)).limit_denominator(dmax)


def _axis_reduction(n: int, q: Fraction):
    """Per bin m: reduced x (first alias), second alias (== first unless tied), zero flag."""
    xa, xb, zero = [], [], []
    half = Fraction(n, 2)
    for m in range(n):
        x = Fraction(m) + q
        x = x - n * math.floor(x / n + Fraction(1, 2))
        tie = (x == -half)
        xa.append(float(x))
        xb.append(float(x + n) if tie else float(x))
        zero.append(x == 0)
    return np.array(xa), np.array(xb), np.array(zero)


def mesh_denominators(kfrac) -> Tuple[int, int, int]:
    """Per axis, the least D with every k-point coordinate a multiple of 1/D: the k-mesh's
    supercell is D_1 a_1, D_2 a_2, D_3 a_3 (the Born-von Karman cell of Sec. II.A)."""
    kfrac = np.atleast_2d(np.asarray(kfrac, float))
    out = []
    for d in range(3):
        den = 1
        for x in kfrac[:, d]:
            den = den * _frac(x).denominator // math.gcd(den, _frac(x).denominator)
        out.append(den)
    return tuple(out)


def supercell_lattice(lattice, kfrac) -> np.ndarray:
    D = mesh_denominators(kfrac)
    return np.asarray(lattice, float) * np.array(D, float)[:, None]


def truncation_radius(lattice, kfrac) -> float:
    """R_c of the truncated kernels: (4 pi / 3) R_c^3 = the supercell volume (Sec. II.A,
    the Spencer-Alavi truncation)."""
    return (3.0 * cell_volume(supercell_lattice(lattice, kfrac)) / (4.0 * math.pi)) ** (1.0 / 3.0)


def _lattice_sums(lat, eta, fn_real, fn_recip, tol=1e-17):
    """sum over R != 0 of fn_real(|R|) and over G != 0 of fn_recip(|G|^2), R on the lattice
    `lat` and G on its reciprocal lattice, in shells grown until a whole shell adds < tol."""
    b = reciprocal_vectors(lat)
    out = []
    for vecs, fn in ((lat, fn_real), (b, fn_recip)):
        if fn is None:
            out.append(0.0)
            continue
        total, n = 0.0, 1
        while True:
            shell = 0.0
            rng = range(-n, n + 1)
            for i in rng:
                for j in rng:
                    for k in rng:
                        if max(abs(i), abs(j), abs(k)) != n:
                            continue
                        v = i * vecs[0] + j * vecs[1] + k * vecs[2]
                        shell += fn(v)
            total += shell
            if abs(shell) < tol and n > 2:
                break
            n += 1
        out.append(total)
    return out


def madelung_potential(lat, eta: Optional[float] = None) -> float:
    """Potential at the origin of the periodic images of a unit point charge in a uniform
    neutralising background (the charge itself excluded), lattice rows `lat`, by Ewald's
    split: sum_{R != 0} erfc(eta R)/R + (4 pi/V) sum_{G != 0} e^{-G^2/(4 eta^2)}/G^2
    - pi/(eta^2 V) - 2 eta/sqrt(pi)."""
    from scipy.special import erfc
    vol = cell_volume(lat)
    if eta is None:
        eta = math.sqrt(math.pi) / vol ** (1.0 / 3.0)
    real, recip = _lattice_sums(
        lat, eta, lambda v: erfc(eta * np.linalg.norm(v)) / np.linalg.norm(v),
        lambda g: 4.0 * math.pi / vol * math.exp(-(g @ g) / (4 * eta * eta)) / (g @ g))
    return real + recip - math.pi / (eta * eta * vol) - 2.0 * eta / math.sqrt(math.pi)


def g0_value(kind: str, omega: float, g0_mode: int, lattice=None, kfrac=None) -> float:
    """Value used for the bin G+q = 0 (Eq. VGao's chi; C3 reading).

    g0_mode 0: the term is dropped. g0_mode 1: f(x -> 0), for the kernels with a finite
    limit (erfc: pi/omega^2; the truncated kernels, Sec. II.A). g0_mode 2: the Madelung
    correction of the k-mesh's supercell (volume V, lattice and kfrac needed): Coulomb
    chi = -V v_M with v_M the supercell's Madelung potential; erf chi = V 2 omega/sqrt(pi)
    - sum_{G != 0} 4 pi e^{-G^2/(4 omega^2)}/G^2 over the supercell's reciprocal lattice
    (the integral of the kernel minus its lattice sum)."""
    if g0_mode == 0:
        return 0.0
    if g0_mode == 1:
        if kind == "erfc":
            return math.pi / (omega * omega)
        rc = truncation_radius(lattice, kfrac)
        if kind == "coulomb_trunc":
            return 2.0 * math.pi * rc * rc
        if kind == "erf_trunc":
            return 4.0 * math.pi * ((rc * rc / 2.0 - 1.0 / (4.0 * omega * omega)) *
                                    math.erf(omega * rc) +
                                    rc * math.exp(-(omega * rc) ** 2) / (2.0 * omega * math.sqrt(math.pi)))
        raise ValueError(f"g0_mode 1 is not defined for the {kind} kernel")
    if g0_mode == 2:
        sc = supercell_lattice(lattice, kfrac)
        vol = cell_volume(sc)
        if kind == "coulomb":
            return -vol * madelung_potential(sc)
        if kind == "erf":
            _, recip = _lattice_sums(sc, omega, None, lambda g: 4.0 * math.pi * math.exp(
                -(g @ g) / (4 * omega * omega)) / (g @ g))
            return vol * 2.0 * omega / math.sqrt(math.pi) - recip
        raise ValueError(f"g0_mode 2 is not defined for the {kind} kernel")
    raise ValueError(g0_mode)


def _kernel_value(kind: str, omega: float, g2: np.ndarray, rc: float = 0.0) -> np.ndarray:
    """f(|G+q|) of Eq. recipcoul (and of the truncated kernels of Sec. II.A, radius rc)
    for |G+q|^2 = g2 > 0."""
    base = 4.0 * np.pi / g2
    if kind == "coulomb":
        return base
    if kind == "coulomb_trunc":
        # 1 - cos(x R_c) = 2 sin^2(x R_c / 2)
        return base * 2.0 * np.sin(0.5 * np.sqrt(g2) * rc) ** 2
    y = g2 / (4.0 * omega * omega)
    if kind == "erfc":
        return base * (-np.expm1(-y))
    if kind == "erf":
        return base * np.exp(-y)
    if kind == "erf_trunc":
        # Eq. lrtrunc: f = (4 pi/x^2) [-erf(w R) cos(x R) + e^{-y} Re erf(w R + i x/(2w))],
        # with e^{-y} erf(z) = e^{-y} - e^{-w^2 R^2} e^{-i x R} w_F(i z) (w_F the Faddeeva
        # function, bounded there), which removes the cancellation Appendix A describes
        from scipy.special import wofz
        x = np.sqrt(g2)
        wr = omega * rc
        faddeeva = wofz(-x / (2.0 * omega) + 1j * wr)
        t = np.exp(-y) - math.exp(-wr * wr) * np.real(np.exp(-1j * x * rc) * faddeeva)
        return base * (-math.erf(wr) * np.cos(x * rc) + t)
    raise ValueError(kind)


def _kernel_domega(kind: str, omega: float, g2: np.ndarray) -> np.ndarray:
    """d f/d omega for |G+q|^2 = g2 > 0."""
    if kind == "coulomb":
        return np.zeros_like(g2)
    e = np.exp(-g2 / (4.0 * omega * omega)) * 2.0 * np.pi / omega ** 3
    return -e if kind == "erfc" else e


def _bins(lattice, grid, qfrac, fn, zero_value):
    b = reciprocal_vectors(lattice)
    axes = [_axis_reduction(int(grid[d]), _frac(qfrac[d])) for d in range(3)]
    zero = axes[0][2][:, None, None] & axes[1][2][None, :, None] & axes[2][2][None, None, :]
    v = np.zeros(tuple(int(g) for g in grid))
    for c1 in (0, 1):
        for c2 in (0, 1):
            for c3 in (0, 1):
                x1 = axes[0][c1][:, None, None, None]
                x2 = axes[1][c2][None, :, None, None]
                x3 = axes[2][c3][None, None, :, None]
                gv = x1 * b[0] + x2 * b[1] + x3 * b[2]
                g2 = np.einsum("abcd,abcd->abc", gv, gv)
                g2 = np.where(zero, 1.0, g2)
                v += fn(g2) / 8.0
    v[zero] = zero_value
    return v


def _rc(kind: str, lattice, kfrac) -> float:
    return truncation_radius(lattice, kfrac) if kind.endswith("_trunc") else 0.0


def kernel_value(kind: str, omega: float, g2, rc: float = 0.0) -> np.ndarray:
    """f(|G+q|) for |G+q|^2 = g2 > 0 (public name of the per-bin kernel)."""
    return _kernel_value(kind, omega, np.asarray(g2, float), rc)


def kernel_bins(lattice, grid, qfrac, kind: str, omega: float, g0: float,
                rc: float = 0.0) -> np.ndarray:
    """v_q(m) on the FFT bins (tie-averaged); G+q = 0 takes g0; rc: truncation radius."""
    return _bins(lattice, grid, qfrac, lambda g2: _kernel_value(kind, omega, g2, rc), g0)


def kernel_bins_domega(lattice, grid, qfrac, kind: str, omega: float, g0_mode: int):
    """d v_q(m)/d omega on the bins; G+q = 0 gives d g0/d omega."""
    dg0 = -2.0 * math.pi / omega ** 3 if (g0_mode == 1 and kind == "erfc") else 0.0
    return _bins(lattice, grid, qfrac, lambda g2: _kernel_domega(kind, omega, g2), dg0)


def grid_phase(grid, qfrac) -> np.ndarray:
    """e^{i q.r_n} = exp(2 pi i sum_i q_i n_i / N_i) on the grid."""
    n1, n2, n3 = grid
    f = (qfrac[0] * np.arange(n1)[:, None, None] / n1 + qfrac[1] * np.arange(n2)[None, :, None] / n2
         + qfrac[2] * np.arange(n3)[None, None, :] / n3)
    return np.exp(2j * np.pi * f)


def dft_matrices(grid):
    """Dense 1-D forward DFT matrices F_N[m, n] = e^{-2 pi i m n / N}, one per axis."""
    out = []
    for n in grid:
        j = np.arange(n)
        out.append(np.exp(-2j * np.pi * np.outer(j, j) / n))
    return out


def apply_coulomb_operator(f: np.ndarray, v: np.ndarray, qfrac, dft: bool = False) -> np.ndarray:
    """V_q[f](r) = e^{iq.r} N_g IFFT[v_q . FFT(f e^{-iq.r})/N_g]  (Eqs. aodf, Vrao, VGao).

    ``f`` has shape ``grid``. With ``dft=True`` the transforms are explicit
    separable DFT-matrix products instead of numpy's FFT.
    """
    grid = f.shape
    ng = int(np.prod(grid))
    ph = grid_phase(grid, qfrac)
    rho = f * np.conj(ph)
    if dft:
        # three 1-D DFT-matrix products, one axis at a time (the separable definition)
        f1, f2, f3 = dft_matrices(grid)
        rhohat = np.einsum("ai,bj,ck,ijk->abc", f1, f2, f3, rho, optimize=True) / ng
        u = np.einsum("ai,bj,ck,ijk->abc", np.conj(f1), np.conj(f2), np.conj(f3), v * rhohat,
                      optimize=True)
    else:
        rhohat = np.fft.fftn(rho) / ng
        u = ng * np.fft.ifftn(v * rhohat)
    return ph * u


# ----------------------------------------------------------------------------
# (c)-(e) occ-RI-K (Algorithm 3) and the conventional builds (Algorithms 1, 2)
# ----------------------------------------------------------------------------

def occri_kc(lattice, grid, kfrac, psi: np.ndarray, chi: Optional[np.ndarray], kind: str,
             omega: float, g0: float, dft: bool = False, return_y: bool = False,
             nsum: Optional[int] = None):
    """AO-occupied block K_{mu i}(k) of Eq. occrik by Algorithm 3.

    psi: (nk, nocc, N_g). For every (k, i) and every (k', j): form the pair
    density, apply the kernel-fused transform round trip, accumulate
    Y_{ik} += psi_{jk'} W (Eq. occrikinterm); then contract with conj(chi).
    If chi is None, only Y is returned.

    nsum (conduction-band extension, Sec. II.D): the orbitals j summed over are the
    first nsum of psi (the occupied ones), while outputs are formed for every orbital
    of psi, so K_{mu p} for p beyond nsum is the exchange operator built from the
    occupied orbitals applied to the extra (conduction) orbital p.
    """
    grid = tuple(int(g) for g in grid)
    nk, nocc, ng = psi.shape
    nj = nocc if nsum is None else int(nsum)
    y = np.zeros_like(psi)
    for k in range(nk):
        for kp in range(nk):
            q = np.asarray(kfrac[k], float) - np.asarray(kfrac[kp], float)
            v = kernel_bins(lattice, grid, q, kind, omega, g0, _rc(kind, lattice, kfrac))
            for i in range(nocc):
                for j in range(nj):
                    f = (np.conj(psi[kp, j]) * psi[k, i]).reshape(grid)
                    w = apply_coulomb_operator(f, v, q, dft=dft).reshape(-1)
                    y[k, i] += psi[kp, j] * w
    if chi is None:
        return y
    kc = contract_kc(lattice, chi, y)
    return (kc, y) if return_y else kc


def contract_kc(lattice, chi: np.ndarray, y: np.ndarray) -> np.ndarray:
    """K_{mu i}(k) = -(Omega/(N_k N_g)) sum_n conj(chi_{mu k}(r_n)) Y_{ik}(r_n)."""
    nk, _, ng = chi.shape
    return -cell_volume(lattice) / (nk * ng) * np.einsum("kmn,kin->kmi", np.conj(chi), y)


def mori_k(lattice, grid, kfrac, chi: np.ndarray, psi: np.ndarray, kind: str, omega: float,
           g0: float) -> np.ndarray:
    """Conventional GPW exchange K^k_{mu nu} by MO-RI-K (Algorithm 2, Eq. exxmo).

    For every (k, nu) and (k', j): potential of conj(psi_{jk'}) chi_{nu k},
    accumulate W_nu += psi_{jk'} V, then K_{mu nu} = -c sum_n conj(chi_mu) W_nu.
    """
    grid = tuple(int(g) for g in grid)
    nk, nao, ng = chi.shape
    nocc = psi.shape[1]
    c = cell_volume(lattice) / (nk * ng)
    kmat = np.zeros((nk, nao, nao), dtype=np.complex128)
    for k in range(nk):
        wacc = np.zeros((nao, ng), dtype=np.complex128)
        for kp in range(nk):
            q = np.asarray(kfrac[k], float) - np.asarray(kfrac[kp], float)
            v = kernel_bins(lattice, grid, q, kind, omega, g0, _rc(kind, lattice, kfrac))
            for nu in range(nao):
                for j in range(nocc):
                    f = (np.conj(psi[kp, j]) * chi[k, nu]).reshape(grid)
                    wacc[nu] += psi[kp, j] * apply_coulomb_operator(f, v, q).reshape(-1)
        kmat[k] = -c * np.conj(chi[k]) @ wacc.T
    return kmat


def aori_k(lattice, grid, kfrac, chi: np.ndarray, C: np.ndarray, kind: str, omega: float,
           g0: float) -> np.ndarray:
    """Conventional GPW exchange by AO-RI-K (Algorithm 1, Eqs. aointerm, aointerm2, aok).

    psi~_{sigma k'} = sum_lambda P^{k'}_{lambda sigma} chi_{lambda k'} with
    P^{k'} = C C^H; potentials of conj(chi_{sigma k'}) chi_{nu k} for every AO pair.
    """
    grid = tuple(int(g) for g in grid)
    nk, nao, ng = chi.shape
    c = cell_volume(lattice) / (nk * ng)
    pmat = np.einsum("kli,ksi->kls", C, np.conj(C))
    psit = np.einsum("kls,kln->ksn", pmat, chi)
    kmat = np.zeros((nk, nao, nao), dtype=np.complex128)
    for k in range(nk):
        wacc = np.zeros((nao, ng), dtype=np.complex128)
        for kp in range(nk):
            q = np.asarray(kfrac[k], float) - np.asarray(kfrac[kp], float)
            v = kernel_bins(lattice, grid, q, kind, omega, g0, _rc(kind, lattice, kfrac))
            for nu in range(nao):
                for s in range(nao):
                    f = (np.conj(chi[kp, s]) * chi[k, nu]).reshape(grid)
                    wacc[nu] += psit[kp, s] * apply_coulomb_operator(f, v, q).reshape(-1)
        kmat[k] = -c * np.conj(chi[k]) @ wacc.T
    return kmat


# ----------------------------------------------------------------------------
# (f) occ-RI assembly in ACE form and the exchange energy
# ----------------------------------------------------------------------------

def ace_assemble(C: np.ndarray, kc: np.ndarray):
    """K_k = KC (C^H KC)^{-1} KC^H via the Cholesky factor of -M (C5, C6 readings).

    Returns (K[nk,nao,nao], M[nk,nocc,nocc], E_x). M is Hermitised before the
    factorisation; E_x = (1/N_k) sum_k Re Tr M_k.
    """
    nk, nao, nocc = C.shape
    kmat = np.zeros((nk, nao, nao), dtype=np.complex128)
    mmat = np.zeros((nk, nocc, nocc), dtype=np.complex128)
    ex = 0.0
    for k in range(nk):
        m = np.conj(C[k].T) @ kc[k]
        m = 0.5 * (m + np.conj(m.T))
        mmat[k] = m
        low = np.linalg.cholesky(-m)                       # -M = L L^H
        xi = np.linalg.solve(np.conj(low), kc[k].T).T      # xi L^H = KC
        kmat[k] = -xi @ np.conj(xi.T)
        ex += float(np.real(np.trace(m)))
    return kmat, mmat, ex / nk


def assemble_paper(ovl: np.ndarray, C: np.ndarray, kc: np.ndarray) -> np.ndarray:
    """K ~ PKP + PKQ + QKP (Eq. occrikop) in the AO basis, from the AO-occupied block.

    With the occupied projector P = C C^H S (S = ovl, the AO overlap of each k, C
    S-orthonormal), <mu|K|j> = KC, and M = C^H KC (Hermitised):
      <mu|PKP|nu> = (S C M C^H S),   <mu|PKQ|nu> = (S C KC^H) - (S C M C^H S),
      <mu|QKP|nu> = (KC C^H S) - (S C M C^H S),
    which sum to K = KC C^H S + S C KC^H - S C M C^H S per k. C may also hold chosen
    conduction bands after the occupied ones (with kc their K_{mu p}, Sec. II.D); P is
    then the projector on all of them.
    """
    nk, nao, ncol = C.shape
    kmat = np.zeros((nk, nao, nao), dtype=np.complex128)
    for k in range(nk):
        m = np.conj(C[k].T) @ kc[k]
        m = 0.5 * (m + np.conj(m.T))
        sc = ovl[k] @ C[k]
        kmat[k] = (kc[k] @ np.conj(sc.T) + sc @ np.conj(kc[k].T)
                   - sc @ m @ np.conj(sc.T))
    return kmat


def exchange_energy(C: np.ndarray, kc: np.ndarray) -> float:
    """E_x = (1/N_k) sum_k Re Tr(C_k^H K_{mu i}(k)) (closed shell, C2 reading)."""
    return float(np.real(np.einsum("kmi,kmi->", np.conj(C), kc))) / C.shape[0]


def exchange_energy_parseval(lattice, grid, kfrac, psi: np.ndarray, kind: str, omega: float,
                             g0: float) -> float:
    """E_x = -(Omega/N_k^2) sum_{k k' i j} sum_m v_q(m) |rho^hat(m)|^2 (discrete Parseval)."""
    grid = tuple(int(g) for g in grid)
    nk, nocc, ng = psi.shape
    tot = 0.0
    for k in range(nk):
        for kp in range(nk):
            q = np.asarray(kfrac[k], float) - np.asarray(kfrac[kp], float)
            v = kernel_bins(lattice, grid, q, kind, omega, g0, _rc(kind, lattice, kfrac))
            ph = grid_phase(grid, q)
            for i in range(nocc):
                for j in range(nocc):
                    rho = (np.conj(psi[kp, j]) * psi[k, i]).reshape(grid) * np.conj(ph)
                    rh = np.fft.fftn(rho) / ng
                    tot += float(np.sum(v * np.abs(rh) ** 2))
    return -cell_volume(lattice) / nk ** 2 * tot


# ----------------------------------------------------------------------------
# adjoint of E_x
# ----------------------------------------------------------------------------

def grad_c(kc: np.ndarray) -> np.ndarray:
    """Gradient of E_x w.r.t. C_k in the conjugate-Wirtinger convention (2 dE/dC*).

    E_x is quadratic in C and in C*, and every orbital enters once as i and
    once as j, so dE/dC*_{mu i}(k) = (2/N_k) K_{mu i}(k); the returned value is
    twice that.
    """
    return 4.0 / kc.shape[0] * kc


def grad_omega(lattice, grid, kfrac, psi: np.ndarray, kind: str, omega: float,
               g0_mode: int) -> float:
    """dE_x/d omega = -(Omega/N_k^2) sum_{k k' i j} sum_m (d v_q(m)/d omega) |rho^hat(m)|^2."""
    grid = tuple(int(g) for g in grid)
    nk, nocc, ng = psi.shape
    tot = 0.0
    for k in range(nk):
        for kp in range(nk):
            q = np.asarray(kfrac[k], float) - np.asarray(kfrac[kp], float)
            dv = kernel_bins_domega(lattice, grid, q, kind, omega, g0_mode)
            ph = grid_phase(grid, q)
            for i in range(nocc):
                for j in range(nocc):
                    rho = (np.conj(psi[kp, j]) * psi[k, i]).reshape(grid) * np.conj(ph)
                    rh = np.fft.fftn(rho) / ng
                    tot += float(np.sum(dv * np.abs(rh) ** 2))
    return -cell_volume(lattice) / nk ** 2 * tot
