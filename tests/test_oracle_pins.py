"""Pins of the FP64 oracle against things other than itself.

Each test names the passage of arXiv:2207.09028 (or the mathematical fact)
that fixes the expected value, and is chosen so that a plausible mistake in
the oracle (a dropped term, a wrong sign, index or normalisation) fails it.
"""
import math

import numpy as np
import pytest

import oracle as O
from workloads import config, small_workload
from workloads.synthetic import analytic_overlap


def _chi(w, grid=None, points=None, kfrac=None):
    return O.bloch_aos(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha,
                       w.kfrac if kfrac is None else kfrac, grid=w.grid if grid is None else grid,
                       points=points)


def _g0(w):
    return O.g0_value(w.kernel, w.omega, w.g0_mode)


def _kc(w, chi=None, C=None, dft=False, kind=None, omega=None, g0=None):
    chi = _chi(w) if chi is None else chi
    C = w.C if C is None else C
    psi = O.orbitals_on_grid(chi, C)
    return O.occri_kc(w.lattice, w.grid, w.kfrac, psi, chi, kind or w.kernel,
                      w.omega if omega is None else omega, _g0(w) if g0 is None else g0, dft=dft)


# ---------------------------------------------------------------- primitives

def _laplacian(poly):
    out = {}
    for (a, b, c), v in poly.items():
        for d, e in enumerate((a, b, c)):
            if e >= 2:
                key = [a, b, c]
                key[d] -= 2
                out[tuple(key)] = out.get(tuple(key), 0.0) + v * e * (e - 1)
    return out


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_solid_harmonics_are_harmonic_and_independent(l):
    """Real solid harmonics are homogeneous of degree l, harmonic, and 2l+1 independent."""
    polys = O.SOLID_HARMONICS[l]
    assert len(polys) == 2 * l + 1
    for p in polys:
        assert all(sum(e) == l for e in p)
        assert all(abs(v) < 1e-14 for v in _laplacian(p).values())
    # Gram matrix of the polynomials under exp(-r^2) must be diagonal (orthogonal
    # on the sphere) and positive.
    gram = np.zeros((2 * l + 1, 2 * l + 1))
    for i, p in enumerate(polys):
        for j, q in enumerate(polys):
            gram[i, j] = sum(c1 * c2 * O.gaussian_moment(e1[0] + e2[0], e1[1] + e2[1],
                                                         e1[2] + e2[2], 1.0)
                             for e1, c1 in p.items() for e2, c2 in q.items())
    assert np.all(np.diag(gram) > 0)
    assert np.abs(gram - np.diag(np.diag(gram))).max() < 1e-13


@pytest.mark.parametrize("l,alpha", [(0, 0.7), (1, 1.3), (2, 0.9), (3, 1.6)])
def test_primitive_normalisation_by_quadrature(l, alpha):
    """Integral of phi^2 is 1 by brute-force quadrature (independent of the moment formula)."""
    h, n = 0.11, 121
    x = (np.arange(n) - n // 2) * h
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    g = np.exp(-alpha * (X * X + Y * Y + Z * Z))
    norms = O.primitive_norms(l, alpha)
    for m in range(2 * l + 1):
        phi = norms[m] * O.eval_solid_harmonic(l, m, X, Y, Z) * g
        assert abs(np.sum(phi * phi) * h ** 3 - 1.0) < 1e-10


def test_image_cutoff_bounds_every_primitive():
    for l, alpha in [(0, 0.06), (1, 0.5), (2, 3.0), (3, 40.0)]:
        r = O.image_cutoff(l, alpha)
        norms = O.primitive_norms(l, alpha)
        rng = np.random.default_rng(0)
        d = rng.standard_normal((2000, 3))
        d *= r / np.linalg.norm(d, axis=1)[:, None]
        for m in range(2 * l + 1):
            v = norms[m] * O.eval_solid_harmonic(l, m, d[:, 0], d[:, 1], d[:, 2]) * math.exp(-alpha * r * r)
            assert np.abs(v).max() <= 1.0000001e-16


# ---------------------------------------------------------------- Bloch AOs

def test_grid_overlap_matches_analytic_obara_saika():
    """GPW quadrature of <chi_mu k|chi_nu k> equals the analytic lattice-summed overlap.

    On a grid that resolves the products, the trapezoid rule is spectrally
    exact, so this pins the oracle's AO values (polynomials, normalisation,
    image sums, Bloch phases) against an independent integral code.
    """
    w = small_workload(a_ang=2.6, mesh=(2, 1, 1), counts=(2, 1, 1), lo=0.35, hi=0.9,
                       grid=(24, 24, 24), nocc=2)
    chi = _chi(w)
    s_grid = O.grid_overlap(w.lattice, chi, w.grid)
    s_ref = analytic_overlap(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha, w.kfrac)
    assert np.abs(s_grid - s_ref).max() < 1e-9 * np.abs(s_ref).max()


def test_bloch_periodicity():
    """chi_{mu k}(r + a_i) = e^{i k.a_i} chi_{mu k}(r) (Sec. II.A Bloch sum)."""
    w = small_workload(mesh=(2, 2, 1), counts=(1, 1, 1, 1), grid=(6, 6, 6))
    rng = np.random.default_rng(3)
    pts = rng.random((40, 3)) @ w.lattice
    base = _chi(w, points=pts)
    for ax in range(3):
        shifted = _chi(w, points=pts + w.lattice[ax])
        ph = np.exp(2j * np.pi * w.kfrac[:, ax])
        assert np.abs(shifted - ph[:, None, None] * base).max() < 1e-13 * np.abs(base).max()


# ---------------------------------------------------------------- kernel + transforms

@pytest.mark.parametrize("grid", [(6, 6, 6), (5, 6, 7), (4, 9, 5)])
@pytest.mark.parametrize("q", [(0.0, 0.0, 0.0), (0.5, -0.5, 0.25), (1 / 3, 0.5, -2 / 3)])
@pytest.mark.parametrize("kind", ["coulomb", "erfc", "erf"])
def test_plane_waves_are_eigenfunctions(grid, q, kind):
    """P8: V_q[e^{i(G_m+q).r}] = v_q(m) e^{i(G_m+q).r} for every bin, ties and G+q=0 included."""
    w = small_workload()
    lat = w.lattice
    v = O.kernel_bins(lat, grid, np.array(q), kind, 0.7, 0.37)
    n1, n2, n3 = grid
    n = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1)
    rng = np.random.default_rng(1)
    for _ in range(6):
        m = [rng.integers(0, g) for g in grid]
        arg = sum((m[d] + q[d]) * n[..., d] / grid[d] for d in range(3))
        f = np.exp(2j * np.pi * arg)
        out = O.apply_coulomb_operator(f, v, np.array(q))
        assert np.abs(out - v[tuple(m)] * f).max() < 1e-12 * max(1.0, abs(v[tuple(m)]))


def test_kernel_bins_inversion_symmetric():
    """With tie averaging, v_{-q}(-m) = v_q(m), so a real density gives a real potential."""
    w = config("cfg1")
    for grid in [(6, 6, 6), (5, 6, 8)]:
        for q in [(0.0, 0.0, 0.0), (0.5, 0.0, -0.5), (0.25, 0.5, 0.75)]:
            q = np.array(q)
            v = O.kernel_bins(w.lattice, grid, q, "coulomb", 0.0, 0.0)
            vm = O.kernel_bins(w.lattice, grid, -q, "coulomb", 0.0, 0.0)
            idx = tuple((-np.arange(g)) % g for g in grid)
            assert np.allclose(vm[np.ix_(*idx)], v, rtol=1e-15, atol=0)


def test_kernel_closed_forms_and_g0():
    """Eq. recipcoul at generic bins; G+q=0 takes g0 = pi/omega^2 for erfc (its x->0 limit)."""
    w = small_workload()
    b = O.reciprocal_vectors(w.lattice)
    grid = (7, 7, 7)
    omega = 0.45
    v_c = O.kernel_bins(w.lattice, grid, np.zeros(3), "coulomb", 0.0, 0.0)
    v_s = O.kernel_bins(w.lattice, grid, np.zeros(3), "erfc", omega, math.pi / omega ** 2)
    v_l = O.kernel_bins(w.lattice, grid, np.zeros(3), "erf", omega, 0.0)
    g = b[0] + 2 * b[1] - b[2]
    g2 = g @ g
    assert abs(v_c[1, 2, 6] - 4 * math.pi / g2) < 1e-14 * v_c[1, 2, 6]
    assert abs(v_l[1, 2, 6] - 4 * math.pi / g2 * math.exp(-g2 / (4 * omega ** 2))) < 1e-14
    assert abs(v_s[1, 2, 6] + v_l[1, 2, 6] - v_c[1, 2, 6]) < 1e-13 * v_c[1, 2, 6]
    assert v_c[0, 0, 0] == 0.0 and v_l[0, 0, 0] == 0.0
    assert v_s[0, 0, 0] == math.pi / omega ** 2
    # the erfc kernel is continuous at the origin: tiny |G+q| approaches g0
    tiny = O.kernel_bins(w.lattice, grid, np.array([1e-4, 0, 0]), "erfc", omega, 0.0)[0, 0, 0]
    assert abs(tiny - math.pi / omega ** 2) < 1e-6 * math.pi / omega ** 2


def test_explicit_dft_equals_fft():
    """P12: explicit separable DFT mode agrees with numpy's FFT mode."""
    w = small_workload(mesh=(1, 1, 2), grid=(6, 5, 4), counts=(2, 1))
    a = _kc(w)
    b = _kc(w, dft=True)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


# ---------------------------------------------------------------- exactness of occ-RI-K

def _conventional(w, chi, which="mo"):
    psi = O.orbitals_on_grid(chi, w.C)
    if which == "mo":
        return O.mori_k(w.lattice, w.grid, w.kfrac, chi, psi, w.kernel, w.omega, _g0(w))
    return O.aori_k(w.lattice, w.grid, w.kfrac, chi, w.C, w.kernel, w.omega, _g0(w))


@pytest.mark.parametrize("mesh,kind", [((1, 1, 1), "coulomb"), ((1, 2, 1), "erfc"),
                                       ((2, 1, 1), "erf")])
def test_ace_reproduces_conventional_on_occupied_space(mesh, kind):
    """P1: K_ACE C = K_conv C; C^H K_ACE C = M; K_ACE Hermitian; K_ACE - K_conv PSD, C in its kernel.

    K_conv is the brute-force MO-RI-K build (Algorithm 2), a separate code path.
    """
    omega = {"coulomb": 0.0, "erfc": 0.5, "erf": 0.6}[kind]
    w = small_workload(mesh=mesh, grid=(8, 8, 8), kernel=kind, omega=omega,
                       g0_mode=1 if kind == "erfc" else 0)
    chi = _chi(w)
    kc = _kc(w, chi=chi)
    k_conv = _conventional(w, chi)
    k_ace, m, ex = O.ace_assemble(w.C, kc)
    scale = np.abs(k_conv).max()
    for k in range(w.nk):
        assert np.abs(k_conv[k] @ w.C[k] - kc[k]).max() < 1e-12 * scale
        assert np.abs(k_ace[k] @ w.C[k] - kc[k]).max() < 1e-12 * scale
        assert np.abs(np.conj(w.C[k].T) @ k_ace[k] @ w.C[k] - m[k]).max() < 1e-12 * scale
        assert np.abs(k_ace[k] - np.conj(k_ace[k].T)).max() < 1e-13 * scale
        d = k_ace[k] - k_conv[k]
        assert np.linalg.eigvalsh(0.5 * (d + np.conj(d.T))).min() > -1e-12 * scale
        assert np.abs(d @ w.C[k]).max() < 1e-12 * scale


def _virtual_complement(ovl_k, c_k):
    """An S-orthonormal basis V of the AO-space complement of span(c_k): V^H S V = 1,
    c_k^H S V = 0 (complete QR in the Cholesky frame of S)."""
    low = np.linalg.cholesky(ovl_k)
    ut = np.conj(low.T) @ c_k
    q, _ = np.linalg.qr(ut, mode="complete")
    return np.linalg.solve(np.conj(low.T), q[:, c_k.shape[1]:])


def _overlap(w):
    return analytic_overlap(w.lattice, w.xyz, w.shell_atom, w.shell_l, w.shell_alpha, w.kfrac)


@pytest.mark.parametrize("mesh,kind", [((1, 1, 1), "coulomb"), ((1, 2, 1), "erfc")])
def test_conduction_band_columns_apply_the_occupied_exchange(mesh, kind):
    """Sec. II.D (conduction bands): with the inner sum restricted to the occupied orbitals,
    every column p of K_{mu p} (occupied or conduction) equals the full exchange operator of
    the occupied density (brute-force AO-RI-K, Algorithm 1) applied to orbital p, and the
    occupied columns equal the plain occ-RI-K build."""
    nocc, nr = 3, 2
    omega = 0.5 if kind == "erfc" else 0.0
    w = small_workload(mesh=mesh, grid=(8, 8, 8), nocc=nocc + nr, kernel=kind, omega=omega,
                       g0_mode=1 if kind == "erfc" else 0)
    chi = _chi(w)
    psi = O.orbitals_on_grid(chi, w.C)
    kc_ext = O.occri_kc(w.lattice, w.grid, w.kfrac, psi, chi, w.kernel, w.omega, _g0(w),
                        nsum=nocc)
    c_occ = np.ascontiguousarray(w.C[:, :, :nocc])
    k_full = O.aori_k(w.lattice, w.grid, w.kfrac, chi, c_occ, w.kernel, w.omega, _g0(w))
    kc_occ = _kc(w, chi=chi, C=c_occ)
    scale = np.abs(k_full).max()
    for k in range(w.nk):
        assert np.abs(k_full[k] @ w.C[k] - kc_ext[k]).max() < 1e-12 * scale
    assert np.abs(kc_ext[:, :, :nocc] - kc_occ).max() < 1e-12 * scale
    # the restriction matters: summing over the conduction orbitals too changes them
    kc_all = _kc(w, chi=chi)
    assert np.abs(kc_all[:, :, nocc:] - kc_ext[:, :, nocc:]).max() > 1e-3 * scale


@pytest.mark.parametrize("mesh,kind", [((1, 1, 1), "coulomb"), ((1, 2, 1), "erfc")])
def test_paper_form_assembly_drops_only_the_virtual_block(mesh, kind):
    """Eq. occrikop: K ~ PKP + PKQ + QKP. With V an S-orthonormal basis of the virtual space,
    K_full - K = S V (V^H K_full V) V^H S exactly (the QKQ block and nothing else), K C = KC,
    C^H K C = C^H KC, and K is Hermitian. K_full is the brute-force AO-RI-K build."""
    omega = 0.5 if kind == "erfc" else 0.0
    w = small_workload(mesh=mesh, grid=(8, 8, 8), nocc=3, kernel=kind, omega=omega,
                       g0_mode=1 if kind == "erfc" else 0)
    chi = _chi(w)
    ovl = _overlap(w)
    kc = _kc(w, chi=chi)
    k_full = O.aori_k(w.lattice, w.grid, w.kfrac, chi, w.C, w.kernel, w.omega, _g0(w))
    k_pap = O.assemble_paper(ovl, w.C, kc)
    scale = np.abs(k_full).max()
    for k in range(w.nk):
        v = _virtual_complement(ovl[k], w.C[k])
        sv = ovl[k] @ v
        qkq = sv @ (np.conj(v.T) @ k_full[k] @ v) @ np.conj(sv.T)
        assert np.abs(k_full[k] - k_pap[k] - qkq).max() < 1e-11 * scale
        assert np.abs(qkq).max() > 1e-3 * scale
        assert np.abs(k_pap[k] @ w.C[k] - kc[k]).max() < 1e-12 * scale
        assert np.abs(k_pap[k] - np.conj(k_pap[k].T)).max() < 1e-13 * scale
        assert np.abs(np.conj(v.T) @ k_pap[k] @ v).max() < 1e-12 * scale


def test_paper_form_with_conduction_bands_keeps_their_blocks():
    """Sec. II.D: with the chosen conduction bands R appended to C (and their K_{mu p} from
    the occupied density), the assembly keeps every block touching P or R and drops only
    the rest-rest block: K_full - K = S V (V^H K_full V) V^H S with V spanning the
    complement of occupied + R. (The printed six-term sum counts RKR three times; the
    reading taken is K ~ K - S~KS~, S~ the projector on the remaining bands.)"""
    nocc, nr = 3, 2
    w = small_workload(mesh=(1, 2, 1), grid=(8, 8, 8), nocc=nocc + nr)
    chi = _chi(w)
    ovl = _overlap(w)
    psi = O.orbitals_on_grid(chi, w.C)
    kc_ext = O.occri_kc(w.lattice, w.grid, w.kfrac, psi, chi, w.kernel, w.omega, _g0(w),
                        nsum=nocc)
    c_occ = np.ascontiguousarray(w.C[:, :, :nocc])
    k_full = O.aori_k(w.lattice, w.grid, w.kfrac, chi, c_occ, w.kernel, w.omega, _g0(w))
    k_pap = O.assemble_paper(ovl, w.C, kc_ext)
    scale = np.abs(k_full).max()
    for k in range(w.nk):
        v = _virtual_complement(ovl[k], w.C[k])
        sv = ovl[k] @ v
        rest = sv @ (np.conj(v.T) @ k_full[k] @ v) @ np.conj(sv.T)
        assert np.abs(k_full[k] - k_pap[k] - rest).max() < 1e-11 * scale
        r = w.C[k][:, nocc:]
        assert np.abs(np.conj(r.T) @ (k_pap[k] - k_full[k]) @ r).max() < 1e-12 * scale


def test_energy_identities_occri_mori_aori():
    """P2/P3/P4: E_x by trace = by Parseval = by MO-RI-K = by AO-RI-K, and E_x < 0."""
    w = small_workload(mesh=(1, 1, 2), grid=(8, 8, 8), counts=(2, 1), nocc=2)
    chi = _chi(w)
    kc = _kc(w, chi=chi)
    e_tr = O.exchange_energy(w.C, kc)
    psi = O.orbitals_on_grid(chi, w.C)
    e_p = O.exchange_energy_parseval(w.lattice, w.grid, w.kfrac, psi, w.kernel, w.omega, _g0(w))
    e_mo = float(np.real(np.einsum("kmi,kmv,kvi->", np.conj(w.C), _conventional(w, chi, "mo"),
                                   w.C))) / w.nk
    e_ao = float(np.real(np.einsum("kmi,kmv,kvi->", np.conj(w.C), _conventional(w, chi, "ao"),
                                   w.C))) / w.nk
    assert e_tr < 0
    for e in (e_p, e_mo, e_ao):
        assert abs(e - e_tr) < 1e-12 * abs(e_tr)


def test_square_c_makes_ace_exact():
    """P10: with nocc = nao (square invertible C) the ACE form equals the full K."""
    w = small_workload(counts=(2, 1), nocc=10, grid=(8, 8, 8))
    chi = _chi(w)
    kc = _kc(w, chi=chi)
    k_ace, _, _ = O.ace_assemble(w.C, kc)
    k_conv = _conventional(w, chi)
    assert np.abs(k_ace - k_conv).max() < 1e-11 * np.abs(k_conv).max()


def test_gamma_real_orbitals_give_real_symmetric_k():
    """P6: at Gamma with real C on an fcc cell and even grid, K is real symmetric."""
    w = config("cfg1")
    kc = _kc(w)
    k_ace, _, _ = O.ace_assemble(w.C, kc)
    assert np.abs(k_ace.imag).max() < 1e-14 * np.abs(k_ace).max()
    assert np.abs(k_ace[0] - k_ace[0].T).max() < 1e-14 * np.abs(k_ace).max()


def test_kmesh_equals_gamma_supercell():
    """P5: E_x(cell, n-mesh) = E_x(Gamma supercell)/N_k (Tables II/III: k-points vs supercells).

    Supercell orbitals C^sc_{(mu,L),(i,k)} = e^{i k.L} C^k_{mu i}/sqrt(N_k).
    """
    w = small_workload(mesh=(1, 1, 2), grid=(6, 6, 6), counts=(2, 1), nocc=2)
    e_cell = O.exchange_energy(w.C, _kc(w))
    nk, nao, nocc = w.C.shape
    sc_lat = w.lattice.copy()
    sc_lat[2] *= 2
    offs = [np.array([0, 0, 0]), np.array([0, 0, 1])]
    xyz = np.concatenate([w.xyz + o @ w.lattice for o in offs])
    natm = w.xyz.shape[0]
    sa = np.concatenate([w.shell_atom + natm * j for j in range(2)])
    sl = np.concatenate([w.shell_l] * 2)
    sx = np.concatenate([w.shell_alpha] * 2)
    csc = np.zeros((2 * nao, nk * nocc), dtype=complex)
    for ik in range(nk):
        for j, o in enumerate(offs):
            csc[j * nao:(j + 1) * nao, ik * nocc:(ik + 1) * nocc] = (
                np.exp(2j * np.pi * w.kfrac[ik] @ o) * w.C[ik] / math.sqrt(nk))
    gsc = (6, 6, 12)
    chi_sc = O.bloch_aos(sc_lat, xyz, sa, sl, sx, np.zeros((1, 3)), grid=gsc)
    psi = O.orbitals_on_grid(chi_sc, csc[None])
    kc = O.occri_kc(sc_lat, gsc, np.zeros((1, 3)), psi, chi_sc, "coulomb", 0.0, 0.0)
    e_sc = O.exchange_energy(csc[None], kc)
    assert abs(e_sc / nk - e_cell) < 1e-12 * abs(e_cell)


def test_isolated_gaussian_erfc_closed_form():
    """P7: one normalised s Gaussian in a large cubic box, erfc kernel with g0 = pi/omega^2.

    The short-range self-exchange of a Gaussian charge of exponent beta = 2 alpha is
    sqrt(2 beta/pi) - (2/sqrt(pi)) (2/beta + 1/omega^2)^{-1/2} (textbook Gaussian
    Coulomb integrals), so E_x = minus that.
    """
    alpha, omega, box = 0.5, 1.0, 12.0
    lat = box * np.eye(3)
    xyz = np.array([[box / 2] * 3])
    grid = (48, 48, 48)
    chi = O.bloch_aos(lat, xyz, np.array([0]), np.array([0]), np.array([alpha]),
                      np.zeros((1, 3)), grid=grid)
    C = np.ones((1, 1, 1), dtype=complex)
    psi = O.orbitals_on_grid(chi, C)
    kc = O.occri_kc(lat, grid, np.zeros((1, 3)), psi, chi, "erfc", omega, math.pi / omega ** 2)
    beta = 2 * alpha
    exact = -(math.sqrt(2 * beta / math.pi)
              - 2 / math.sqrt(math.pi) * (2 / beta + 1 / omega ** 2) ** -0.5)
    assert abs(O.exchange_energy(C, kc) - exact) < 1e-10


def test_kernel_linearity_erfc_plus_erf_is_coulomb():
    """P11: v_erfc + v_erf = v_Coulomb (Eq. recipcoul), so K is additive (g0 = 0)."""
    w = small_workload(mesh=(2, 1, 1), grid=(6, 6, 6))
    chi = _chi(w)
    a = _kc(w, chi=chi, kind="erfc", omega=0.4, g0=0.0)
    b = _kc(w, chi=chi, kind="erf", omega=0.4, g0=0.0)
    c = _kc(w, chi=chi, kind="coulomb", omega=0.0, g0=0.0)
    assert np.abs(a + b - c).max() < 1e-13 * np.abs(c).max()


# ---------------------------------------------------------------- singularity treatments
# (Sec. II.A: the Madelung correction chi of Eq. VGao, the Spencer-Alavi truncated Coulomb
# kernel and the truncated long-range kernel of Eq. lrtrunc with Appendix A's stable form)

def _golden_scalar(name, key):
    path = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden", name)
    for line in open(path):
        parts = line.split()
        if parts and parts[0] == key:
            return float(parts[1])
    raise KeyError(key)


def test_madelung_potential_of_the_simple_cubic_lattice():
    alpha = _golden_scalar("madelung_simple_cubic.txt", "alpha")
    for L in (1.0, 7.5):
        for eta in (None, 0.9 / L, 2.5 / L):   # the Ewald split must not matter
            v = O.madelung_potential(L * np.eye(3), eta)
            assert abs(v * L + alpha) < 1e-11, (L, eta, v)


def test_madelung_chi_of_the_coulomb_and_erf_kernels():
    """chi = -V v_M for Coulomb; for erf, the integral of the kernel minus its lattice sum,
    which differs from Coulomb's by the short-range images -V sum_{R != 0} erfc(w R)/R and
    from erfc's chi = pi/w^2 (v_erf + v_erfc = v_Coulomb) accordingly."""
    from scipy.special import erfc
    lat = small_workload(a_ang=3.0).lattice
    kf = O.grid_points(np.eye(3), (2, 1, 2))        # a 2 x 1 x 2 Gamma-centred mesh
    sc = O.supercell_lattice(lat, kf)
    assert np.allclose(sc, lat * np.array([2, 1, 2])[:, None])
    vol = O.cell_volume(sc)
    chi_c = O.g0_value("coulomb", 0.0, 2, lat, kf)
    assert abs(chi_c + vol * O.madelung_potential(sc)) < 1e-12 * abs(chi_c)
    assert chi_c > 0                                   # v_M < 0: more exchange, not less
    for w in (0.3, 0.8, 1.5):
        chi_e = O.g0_value("erf", w, 2, lat, kf)
        n = np.arange(-12, 13)
        R = (n[:, None, None, None] * sc[0] + n[None, :, None, None] * sc[1] +
             n[None, None, :, None] * sc[2]).reshape(-1, 3)
        r = np.linalg.norm(R, axis=1)
        r = r[r > 0]
        images = float(np.sum(erfc(w * r) / r))       # brute force, converged for these w
        assert abs(chi_c - (chi_e + math.pi / w ** 2) + vol * images) < 1e-9 * abs(chi_c), w
    # a kernel too smooth to see the lattice: only the integral V 2 w / sqrt(pi) is left
    assert abs(O.g0_value("erf", 0.05, 2, lat, kf) - vol * 0.1 / math.sqrt(math.pi)) < 1e-10


def _fourier_radial(rv, x, rc):
    """Fourier transform of a radial potential cut at rc, given rv(r) = r v(r):
    4 pi / x int_0^rc rv(r) sin(x r) dr (x > 0), or 4 pi int_0^rc r rv(r) dr (x = 0)."""
    from scipy.integrate import quad
    if x == 0.0:
        return 4 * math.pi * quad(lambda r: r * rv(r), 0, rc, epsabs=1e-13, epsrel=1e-13)[0]
    val = quad(rv, 0, rc, weight="sin", wvar=x, epsabs=1e-13, epsrel=1e-13, limit=400)[0]
    return 4 * math.pi / x * val


@pytest.mark.parametrize("x", [0.05, 0.7, 3.0, 11.0, 40.0])
def test_truncated_kernels_are_the_fourier_transforms_of_the_cut_potentials(x):
    from scipy.special import erf
    rc, w = 6.2, 0.45
    f_c = O.kernel_value("coulomb_trunc", 0.0, np.array([x * x]), rc)[0]
    assert abs(f_c - _fourier_radial(lambda r: 1.0, x, rc)) < 1e-9 * abs(f_c) + 1e-12
    f_e = O.kernel_value("erf_trunc", w, np.array([x * x]), rc)[0]
    ref = _fourier_radial(lambda r: erf(w * r), x, rc)
    assert abs(f_e - ref) < 1e-9 * max(abs(ref), 1e-3), (f_e, ref)


def test_truncated_kernels_x_to_zero_limits():
    from scipy.special import erf
    w = small_workload(mesh=(1, 2, 1))
    rc = O.truncation_radius(w.lattice, w.kfrac)
    assert abs(4 * math.pi / 3 * rc ** 3 - 2 * O.cell_volume(w.lattice)) < 1e-10 * rc ** 3
    g0c = O.g0_value("coulomb_trunc", 0.0, 1, w.lattice, w.kfrac)
    assert abs(g0c - _fourier_radial(lambda r: 1.0, 0.0, rc)) < 1e-10 * g0c
    g0e = O.g0_value("erf_trunc", 0.4, 1, w.lattice, w.kfrac)
    ref = _fourier_radial(lambda r: erf(0.4 * r), 0.0, rc)
    assert abs(g0e - ref) < 1e-10 * ref
    # and the kernels approach them continuously
    for kind, g0 in (("coulomb_trunc", g0c), ("erf_trunc", g0e)):
        f = O.kernel_value(kind, 0.4, np.array([1e-8]), rc)[0]
        assert abs(f - g0) < 1e-5 * g0, kind


def test_isolated_gaussian_coulomb_with_madelung_correction():
    """One normalised s Gaussian (exponent alpha, density exponent beta = 2 alpha) in a
    large cubic box, Coulomb kernel with the Madelung chi: the images in the neutralising
    background cancel against chi up to the Ewald terms, leaving E_x = -(sqrt(2 beta/pi) +
    2 pi / (beta L^3)) (Ewald's identity with splitting eta^2 = beta/2; erfc(eta L) terms
    are below 1e-20 here)."""
    alpha, box = 0.9, 11.0
    lat = box * np.eye(3)
    xyz = np.array([[box / 2] * 3])
    grid = (54, 54, 54)
    kf = np.zeros((1, 3))
    chi = O.bloch_aos(lat, xyz, np.array([0]), np.array([0]), np.array([alpha]), kf, grid=grid)
    C = np.ones((1, 1, 1), dtype=complex)
    psi = O.orbitals_on_grid(chi, C)
    g0 = O.g0_value("coulomb", 0.0, 2, lat, kf)
    kc = O.occri_kc(lat, grid, kf, psi, chi, "coulomb", 0.0, g0)
    beta = 2 * alpha
    exact = -(math.sqrt(2 * beta / math.pi) + 2 * math.pi / (beta * box ** 3))
    assert abs(O.exchange_energy(C, kc) - exact) < 1e-8


@pytest.mark.parametrize("kind,g0_mode,omega", [("coulomb_trunc", 1, 0.0), ("erf_trunc", 1, 0.5),
                                                 ("coulomb", 2, 0.0), ("erf", 2, 0.5)])
def test_kmesh_equals_gamma_supercell_with_singularity_treatments(kind, g0_mode, omega):
    """P5 again: the truncation radius and the Madelung chi belong to the k-mesh's supercell,
    which is the same for the cell with its mesh and for the Gamma supercell."""
    w = small_workload(mesh=(1, 1, 2), grid=(6, 6, 6), counts=(2, 1), nocc=2)
    chi = _chi(w)
    psi = O.orbitals_on_grid(chi, w.C)
    g0 = O.g0_value(kind, omega, g0_mode, w.lattice, w.kfrac)
    e_cell = O.exchange_energy(w.C, O.occri_kc(w.lattice, w.grid, w.kfrac, psi, chi, kind,
                                               omega, g0))
    nk, nao, nocc = w.C.shape
    sc_lat = w.lattice.copy()
    sc_lat[2] *= 2
    offs = [np.array([0, 0, 0]), np.array([0, 0, 1])]
    xyz = np.concatenate([w.xyz + o @ w.lattice for o in offs])
    natm = w.xyz.shape[0]
    sa = np.concatenate([w.shell_atom + natm * j for j in range(2)])
    csc = np.zeros((2 * nao, nk * nocc), dtype=complex)
    for ik in range(nk):
        for j, o in enumerate(offs):
            csc[j * nao:(j + 1) * nao, ik * nocc:(ik + 1) * nocc] = (
                np.exp(2j * np.pi * w.kfrac[ik] @ o) * w.C[ik] / math.sqrt(nk))
    gsc = (6, 6, 12)
    kg = np.zeros((1, 3))
    chi_sc = O.bloch_aos(sc_lat, xyz, sa, np.concatenate([w.shell_l] * 2),
                         np.concatenate([w.shell_alpha] * 2), kg, grid=gsc)
    psi_sc = O.orbitals_on_grid(chi_sc, csc[None])
    g0_sc = O.g0_value(kind, omega, g0_mode, sc_lat, kg)
    assert abs(g0_sc - g0) < 1e-10 * abs(g0)
    e_sc = O.exchange_energy(csc[None], O.occri_kc(sc_lat, gsc, kg, psi_sc, chi_sc, kind, omega,
                                                   g0_sc))
    assert abs(e_sc / nk - e_cell) < 1e-11 * abs(e_cell)


# ---------------------------------------------------------------- adjoint

def _energy(w, C, chi, omega=None):
    return O.exchange_energy(C, _kc(w, chi=chi, C=C, omega=omega))


def test_grad_c_matches_central_differences():
    """P9: 2 dE/dC* = (4/N_k) K_{mu i}(k), checked against central differences (h = 1e-5)."""
    w = small_workload(mesh=(1, 2, 1), grid=(6, 6, 6), nocc=2, kernel="erfc", omega=0.5,
                       g0_mode=1)
    chi = _chi(w)
    g = O.grad_c(_kc(w, chi=chi))
    rng = np.random.default_rng(11)
    for _ in range(2):
        d = rng.standard_normal(w.C.shape) + 1j * rng.standard_normal(w.C.shape)
        h = 1e-5
        fd = (_energy(w, w.C + h * d, chi) - _energy(w, w.C - h * d, chi)) / (2 * h)
        an = float(np.real(np.sum(np.conj(g) * d)))
        assert abs(fd - an) < 1e-7 * abs(an)


@pytest.mark.parametrize("kind,g0_mode", [("erfc", 1), ("erfc", 0), ("erf", 0)])
def test_grad_omega_matches_central_differences(kind, g0_mode):
    w = small_workload(mesh=(2, 1, 1), grid=(6, 6, 6), nocc=2, kernel=kind, omega=0.45,
                       g0_mode=g0_mode)
    chi = _chi(w)
    psi = O.orbitals_on_grid(chi, w.C)
    an = O.grad_omega(w.lattice, w.grid, w.kfrac, psi, kind, 0.45, g0_mode)
    h = 1e-5
    ep = O.exchange_energy(w.C, _kc(w, chi=chi, omega=0.45 + h,
                                    g0=O.g0_value(kind, 0.45 + h, g0_mode)))
    em = O.exchange_energy(w.C, _kc(w, chi=chi, omega=0.45 - h,
                                    g0=O.g0_value(kind, 0.45 - h, g0_mode)))
    assert abs((ep - em) / (2 * h) - an) < 1e-7 * abs(an)
