"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics (not against itself).  CPU only."""
import numpy as np
import pytest

from oracle import agf2_oracle as O
from paper_2106_03508_gb300.synth import make_system, random_poles


def small(nmo=7, nocc=2, naux=9, seed=11):
    s = make_system(nmo, nocc, naux, seed)
    return s


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ---- Eq. (fock_matrix) against explicit four-index sums ------------------
def test_fock_matrix_explicit_loops():
    s = small(5, 2, 6, 3)
    rng = np.random.default_rng(5)
    h = rng.standard_normal((5, 5)); h = h + h.T
    D = rng.standard_normal((5, 5)); D = D + D.T
    eri = np.zeros((5, 5, 5, 5))
    for p in range(5):
        for q in range(5):
            for r in range(5):
                for t in range(5):
                    eri[p, q, r, t] = sum(s.L[Q, p, q] * s.L[Q, r, t] for Q in range(s.naux))
    F = np.zeros((5, 5))
    for p in range(5):
        for q in range(5):
            F[p, q] = h[p, q]
            for r in range(5):
                for t in range(5):
                    F[p, q] += (eri[p, q, r, t] - 0.5 * eri[p, t, r, q]) * D[r, t]
    assert rel(O.fock_matrix(h, s.L, D), F) < 1e-13


def test_hcore_gives_diagonal_fock():
    s = small(8, 3, 10, 4)
    h = O.hcore_from_mo_energies(s.eps, s.L, s.nocc)
    F = O.fock_matrix(h, s.L, O.hf_density(8, 3))
    assert np.max(np.abs(F - np.diag(s.eps))) < 1e-13


# ---- Eqs. (mp2_zeroth_moment), (mp2_first_moment) -------------------------
@pytest.mark.parametrize("nmo,nq,no,naux,seed", [(6, 6, 2, 7, 1), (5, 13, 6, 8, 2), (7, 15, 4, 5, 3)])
def test_moments_vs_explicit_sums(nmo, nq, no, naux, seed):
    """GEMM-structured moments == explicit sums over four-index pole ERIs,
    with a generic (non-unitary, more poles than orbitals) coupling matrix."""
    s = make_system(nmo, 2, naux, seed)
    e, C, mu = random_poles(nmo, nq, no, seed + 100)
    Uh, Up = O.build_moments(s.L, e, C, mu)
    Bh, Bp = O.build_moments_loops(s.L, e, C, mu)
    Bh = 0.5 * (Bh + Bh.transpose(0, 2, 1))
    Bp = 0.5 * (Bp + Bp.transpose(0, 2, 1))
    for n in range(2):
        assert rel(Uh[n], Bh[n]) < 1e-12
        assert rel(Up[n], Bp[n]) < 1e-12


def test_moments_loops_symmetric_and_psd():
    """The exact double sum is symmetric and U^(0) is positive semidefinite
    (it is the Gram matrix of the S/D-factorised couplings)."""
    s = make_system(6, 2, 7, 9)
    e, C, mu = random_poles(6, 12, 5, 9)
    Bh, Bp = O.build_moments_loops(s.L, e, C, mu)
    for B in (Bh, Bp):
        assert rel(B[0], B[0].T) < 1e-12 and rel(B[1], B[1].T) < 1e-12
        assert np.min(np.linalg.eigvalsh(B[0])) > -1e-10 * np.max(np.abs(B[0]))


def test_moments_homogeneity():
    """(pq|rs) is quadratic in L, each moment quadratic in (pq|rs): U(lam L) = lam^4 U(L)."""
    s = make_system(9, 3, 12, 21)
    e, C, mu = random_poles(9, 20, 8, 21)
    U1 = O.build_moments(s.L, e, C, mu)
    U2 = O.build_moments(1.7 * s.L, e, C, mu)
    for a, b in zip(U1, U2):
        assert rel(b, 1.7 ** 4 * a) < 1e-13


def test_moments_energy_shift():
    """Shifting all pole energies by t: occupied/virtual sets fixed, the hole
    weight e_i+e_j-e_a shifts by t, the particle weight e_a+e_b-e_i by t:
    U^(1) -> U^(1) + t U^(0), U^(0) unchanged."""
    s = make_system(8, 3, 10, 5)
    e, C, mu = random_poles(8, 18, 7, 5)
    Uh, Up = O.build_moments(s.L, e, C, mu)
    Vh, Vp = O.build_moments(s.L, e + 0.37, C, mu + 0.37)
    for U, V in ((Uh, Vh), (Up, Vp)):
        assert rel(V[0], U[0]) < 1e-13
        assert rel(V[1], U[1] + 0.37 * U[0]) < 1e-12


def _sd_auxiliaries(L, eps, nocc):
    """Uncompressed greater self-energy of Eq. (mp2_self_energy) at the HF
    reference as explicit auxiliaries: for a <= b, i the pair couplings
    S = (pa|bi) + (pb|ai), D = (pa|bi) - (pb|ai) with weights 1/2, 3/2
    (a = b: (pa|ai), weight 1), energy e_a + e_b - e_i."""
    eri = np.einsum("Qpq,Qrs->pqrs", L, L)
    N = len(eps)
    vs, Es = [], []
    for a in range(nocc, N):
        for b in range(a, N):
            for i in range(nocc):
                x1 = eri[:, a, b, i]
                x2 = eri[:, b, a, i]
                w = eps[a] + eps[b] - eps[i]
                if a == b:
                    vs.append(x1); Es.append(w)
                else:
                    vs.append(np.sqrt(0.5) * (x1 + x2)); Es.append(w)
                    vs.append(np.sqrt(1.5) * (x1 - x2)); Es.append(w)
    return np.array(Es), np.array(vs).T


def test_uncompressed_greater_self_energy_moments_and_mp2():
    """(1) The explicit 1h2p auxiliaries reproduce U_>^(0,1) of the oracle.
    (2) Galitskii-Migdal with them at the HF reference equals the closed-shell
    MP2 energy sum_{ijab} (ia|jb)[2(ia|jb) - (ib|ja)]/(e_i+e_j-e_a-e_b),
    written here as explicit loops."""
    s = make_system(9, 3, 11, 17)
    N, no = s.nmo, s.nocc
    E, v = _sd_auxiliaries(s.L, s.eps, no)
    Uh, Up = O.build_moments(s.L, s.eps, np.eye(N), 0.5 * (s.eps[no - 1] + s.eps[no]))
    assert rel(v @ v.T, Up[0]) < 1e-12
    assert rel(v @ np.diag(E) @ v.T, Up[1]) < 1e-12
    e2 = O.energy_2body(s.eps[:no], np.eye(N)[:, :no], E, v)
    eri = np.einsum("Qpq,Qrs->pqrs", s.L, s.L)
    emp2 = 0.0
    for i in range(no):
        for j in range(no):
            for a in range(no, N):
                for b in range(no, N):
                    emp2 += eri[i, a, j, b] * (2 * eri[i, a, j, b] - eri[i, b, j, a]) / (
                        s.eps[i] + s.eps[j] - s.eps[a] - s.eps[b])
    assert abs(e2 - emp2) < 1e-12 * abs(emp2)
    assert abs(O.mp2_energy(s.L, s.eps, no) - emp2) < 1e-12 * abs(emp2)


# ---- compression, Eq. (block_lanczos_chol_3) -------------------------------
def test_compression_conserves_moments():
    s = make_system(10, 3, 14, 8)
    e, C, mu = random_poles(10, 25, 9, 8)
    for U in O.build_moments(s.L, e, C, mu):
        E, v = O.compress(U[0], U[1])
        assert rel(v @ v.T, U[0]) < 1e-12
        assert rel(v @ np.diag(E) @ v.T, U[1]) < 1e-11
        assert np.all(np.diff(E) >= 0)


def test_compression_rejects_non_pd():
    U0 = np.diag([1.0, -1e-3, 2.0])
    with pytest.raises(O.NotPositiveDefinite):
        O.compress(U0, np.eye(3))


def test_compression_exact_for_few_auxiliaries():
    """A self-energy with exactly N auxiliaries is reproduced exactly
    (energies identical), as the block-Lanczos step spans it."""
    rng = np.random.default_rng(3)
    N = 6
    E0 = np.sort(rng.uniform(-3, 3, N))
    v0 = rng.standard_normal((N, N))
    E, v = O.compress(v0 @ v0.T, v0 @ np.diag(E0) @ v0.T)
    assert np.max(np.abs(E - E0)) < 1e-9 * np.linalg.cond(v0)


# ---- extended Hamiltonian and Fock loop -----------------------------------
def test_extended_eigenvectors_complete():
    rng = np.random.default_rng(2)
    N = 6
    F = rng.standard_normal((N, N)); F = F + F.T
    E = rng.uniform(-3, 3, 2 * N)
    v = rng.standard_normal((N, 2 * N))
    e, C = O.diagonalise(F, E, v)
    assert rel(C @ C.T, np.eye(N)) < 1e-13
    H = O.extended_hamiltonian(F, E, v)
    w, V = np.linalg.eigh(H)
    assert np.max(np.abs(H @ V - V * w)) < 1e-12


def test_aufbau_and_shift_electron_count():
    s = make_system(8, 3, 10, 12)
    h = O.hcore_from_mo_energies(s.eps, s.L, s.nocc)
    e, C, mu = s.eps, np.eye(8), 0.5 * (s.eps[2] + s.eps[3])
    Uh, Up = O.build_moments(s.L, e, C, mu)
    Eh, vh = O.compress(Uh[0], Uh[1])
    Ep, vp = O.compress(Up[0], Up[1])
    E = np.concatenate([Eh, Ep]); v = np.concatenate([vh, vp], 1)
    F = O.fock_matrix(h, s.L, O.hf_density(8, 3))
    info = O.solve_shift(F, E, v, s.nelec)
    assert info.converged
    ee, CC = O.diagonalise(F, E + info.delta, v)
    k, mu, n = O.aufbau(ee, CC, s.nelec)
    assert abs(n - s.nelec) < 1e-10
    assert ee[k - 1] < mu < ee[k]


def test_fock_loop_fixed_point_and_count():
    s = make_system(8, 3, 10, 12)
    h = O.hcore_from_mo_energies(s.eps, s.L, s.nocc)
    Uh, Up = O.build_moments(s.L, s.eps, np.eye(8), 0.5 * (s.eps[2] + s.eps[3]))
    Eh, vh = O.compress(Uh[0], Uh[1])
    Ep, vp = O.compress(Up[0], Up[1])
    E = np.concatenate([Eh, Ep]); v = np.concatenate([vh, vp], 1)
    fr = O.fock_loop(h, s.L, s.nelec, E, v, O.hf_density(8, 3))
    assert fr.converged
    k = fr.nocc_qmo
    assert abs(2 * np.sum(fr.C[:, :k] ** 2) - s.nelec) < 1e-9
    # D is a fixed point: rediagonalising with F[D] returns D
    e2, C2 = O.diagonalise(O.fock_matrix(h, s.L, fr.D), fr.E_shift, v)
    D2 = 2 * C2[:, :k] @ C2[:, :k].T
    assert np.max(np.abs(D2 - fr.D)) < 1e-8


def test_weak_coupling_limit():
    """L -> lam L with lam small: the correlation vanishes as lam^4, so
    E_tot -> E_HF and IP -> -eps_HOMO."""
    s = make_system(8, 3, 10, 30)
    L = 1e-2 * s.L
    h = O.hcore_from_mo_energies(s.eps, L, s.nocc)
    r = O.run(h, L, s.nelec, s.eps, max_iter=5)
    assert abs(r.E_tot - r.E_hf) < 1e-6
    assert abs(r.ip + s.eps[2]) < 1e-5
    assert abs(r.ea + s.eps[3]) < 1e-5


def test_first_iteration_two_body_vs_mp2_gap_reported():
    """Compressed first-iteration E_2b approximates E_MP2 (not equal): the
    Galitskii-Migdal sum with only N compressed auxiliaries; the gap is
    finite and both are negative."""
    s = make_system(8, 3, 10, 40)
    L = 0.3 * s.L
    N, no = s.nmo, s.nocc
    Uh, Up = O.build_moments(L, s.eps, np.eye(N), 0.5 * (s.eps[no - 1] + s.eps[no]))
    Ep, vp = O.compress(Up[0], Up[1])
    e2 = O.energy_2body(s.eps[:no], np.eye(N)[:, :no], Ep, vp)
    emp2 = O.mp2_energy(L, s.eps, no)
    assert e2 < 0 and emp2 < 0
    assert abs(e2 - emp2) < abs(emp2)


def _pair_loops(L, e, C, mu, hole_pairs, part_pairs, nmom=1):
    """Brute force: the moment sums of Eqs. (mp2_zeroth_moment),
    (mp2_first_moment) over four-index pole ERIs, restricted to ordered outer
    pairs whose unordered version is listed (positions in the occupied /
    virtual pole lists)."""
    N = L.shape[1]
    occ = [x for x in range(len(e)) if e[x] < mu]
    vir = [x for x in range(len(e)) if not e[x] < mu]
    g = O.pole_eris(L, C)
    out = []
    for pairs, outer, inner in ((hole_pairs, occ, vir), (part_pairs, vir, occ)):
        keep = {(min(x, y), max(x, y)) for x, y in pairs}
        U = np.zeros((nmom + 1, N, N))
        for p in range(N):
            for q in range(N):
                for xi, i in enumerate(outer):
                    for xj, j in enumerate(outer):
                        if (min(xi, xj), max(xi, xj)) not in keep:
                            continue
                        for c in inner:
                            t = g[p, i, j, c] * (2.0 * g[q, i, j, c] - g[q, j, i, c])
                            for n in range(nmom + 1):
                                U[n, p, q] += t * (e[i] + e[j] - e[c]) ** n
        out.append(0.5 * (U + U.transpose(0, 2, 1)))
    return out


def test_slice_additivity():
    """The moments are sums over the outer pole pairs (the summed indices the
    paper distributes over ranks): pair sets that partition all unordered
    outer pairs give partial moments adding to the whole build, in both
    sectors; and one pair set's partial moments equal the explicit
    four-index sums restricted to those ordered pairs (so the partial build
    restricts the right indices)."""
    s = make_system(6, 2, 7, 44)
    e, C, mu = random_poles(6, 11, 4, 44)
    o, v = 4, 7
    rng = np.random.default_rng(3)
    hp = [(x, y) for x in range(o) for y in range(x, o)]
    pp = [(x, y) for x in range(v) for y in range(x, v)]
    lab_h = rng.integers(0, 3, len(hp))
    lab_p = rng.integers(0, 3, len(pp))
    Uh, Up = O.build_moments(s.L, e, C, mu)
    Sh, Sp = np.zeros_like(Uh), np.zeros_like(Up)
    for k in range(3):
        ph, pq = O.build_moments_pairs(s.L, e, C, mu, 1,
                                       [hp[t] for t in range(len(hp)) if lab_h[t] == k],
                                       [pp[t] for t in range(len(pp)) if lab_p[t] == k])
        Sh += ph
        Sp += pq
    assert rel(Sh, Uh) < 1e-13 and rel(Sp, Up) < 1e-13
    sel_h = [hp[t] for t in range(len(hp)) if lab_h[t] == 1]
    sel_p = [pp[t] for t in range(len(pp)) if lab_p[t] == 1]
    ph, pq = O.build_moments_pairs(s.L, e, C, mu, 1, sel_h, sel_p)
    bh, bp = _pair_loops(s.L, e, C, mu, sel_h, sel_p)
    assert rel(ph, bh) < 1e-12 and rel(pq, bp) < 1e-12
    # a genuine slice: it is neither zero nor the whole
    assert 0.05 < np.max(np.abs(ph)) / np.max(np.abs(Uh)) < 0.95
    # slices of the first summed index (i for the hole sector, a for the
    # particle sector) of the per-index form partition the sums as well, and
    # one slice is the explicit sum over the ordered pairs starting there
    Th, Tp = np.zeros_like(Uh), np.zeros_like(Up)
    for part in (([0, 3], [1, 4, 6]), ([1], [0, 5]), ([2], [2, 3])):
        ph, pq = O.build_moments(s.L, e, C, mu, 1, outer_occ=part[0], outer_vir=part[1])
        Th += ph
        Tp += pq
    assert rel(Th, Uh) < 1e-13 and rel(Tp, Up) < 1e-13
    ph, pq = O.build_moments(s.L, e, C, mu, 1, outer_occ=[1], outer_vir=[4])
    bh, _ = _ordered_first_loops(s.L, e, C, mu, [1], [])
    _, bp = _ordered_first_loops(s.L, e, C, mu, [], [4])
    assert rel(ph, bh) < 1e-12 and rel(pq, bp) < 1e-12


def _ordered_first_loops(L, e, C, mu, first_occ, first_vir, nmom=1):
    """Brute force: the moment sums restricted to outer pairs whose first
    index is listed (positions in the occupied / virtual pole lists)."""
    N = L.shape[1]
    occ = [x for x in range(len(e)) if e[x] < mu]
    vir = [x for x in range(len(e)) if not e[x] < mu]
    g = O.pole_eris(L, C)
    out = []
    for first, outer, inner in ((first_occ, occ, vir), (first_vir, vir, occ)):
        U = np.zeros((nmom + 1, N, N))
        for p in range(N):
            for q in range(N):
                for xi in first:
                    i = outer[xi]
                    for j in outer:
                        for c in inner:
                            t = g[p, i, j, c] * (2.0 * g[q, i, j, c] - g[q, j, i, c])
                            for n in range(nmom + 1):
                                U[n, p, q] += t * (e[i] + e[j] - e[c]) ** n
        out.append(0.5 * (U + U.transpose(0, 2, 1)))
    return out


def _eri(L):
    naux, N, _ = L.shape
    g = np.zeros((N, N, N, N))
    for p in range(N):
        for q in range(N):
            for r in range(N):
                for t in range(N):
                    g[p, q, r, t] = sum(L[Q, p, q] * L[Q, r, t] for Q in range(naux))
    return g


def test_energy_1body_hf_closed_form():
    """At the aufbau density D0 (nocc doubly occupied orbitals) the one-body
    energy 1/2 Tr[D0 (h + F[D0])] is the closed-shell Hartree-Fock energy
    sum_i 2 h_ii + sum_ij [2 (ii|jj) - (ij|ji)], written here from explicit
    four-index ERIs and a generic symmetric h."""
    s = make_system(6, 2, 5, 61)
    rng = np.random.default_rng(61)
    h = rng.standard_normal((6, 6)); h = h + h.T
    g = _eri(s.L)
    nocc = 2
    ehf = sum(2.0 * h[i, i] for i in range(nocc))
    for i in range(nocc):
        for j in range(nocc):
            ehf += 2.0 * g[i, i, j, j] - g[i, j, j, i]
    D0 = O.hf_density(6, nocc)
    got = O.energy_1body(h, O.fock_matrix(h, s.L, D0), D0)
    assert abs(got - ehf) < 1e-13 * max(1.0, abs(ehf))


def test_energy_1body_general_density():
    """At a non-idempotent density the one-body energy is
    sum_pq D_pq h_pq + 1/2 sum_pqrs D_pq D_rs [(pq|rs) - 1/2 (ps|rq)]
    (Eq. fock_matrix inserted in 1/2 Tr[D (h + F)]), as explicit loops."""
    s = make_system(5, 2, 6, 62)
    rng = np.random.default_rng(62)
    h = rng.standard_normal((5, 5)); h = h + h.T
    D = rng.standard_normal((5, 5)); D = D + D.T
    g = _eri(s.L)
    ref = float(np.sum(D * h))
    for p in range(5):
        for q in range(5):
            for r in range(5):
                for t in range(5):
                    ref += 0.5 * D[p, q] * D[r, t] * (g[p, q, r, t] - 0.5 * g[p, t, r, q])
    got = O.energy_1body(h, O.fock_matrix(h, s.L, D), D)
    assert abs(got - ref) < 1e-12 * max(1.0, abs(ref))


def test_moment_elements_match_full_build():
    s = make_system(9, 2, 11, 71)
    e, C, mu = random_poles(9, 22, 8, 71)
    Uh, Up = O.build_moments(s.L, e, C, mu)
    pq = [(0, 0), (3, 7), (8, 2), (5, 5)]
    eh, ep = O.moment_elements(s.L, e, C, mu, pq)
    for t, (p, q) in enumerate(pq):
        for n in range(2):
            assert abs(eh[t, n] - Uh[n, p, q]) <= 1e-12 * np.max(np.abs(Uh[n]))
            assert abs(ep[t, n] - Up[n, p, q]) <= 1e-12 * np.max(np.abs(Up[n]))


def test_spectral_function_single_pole_and_hf():
    """One pole of unit weight gives the Lorentzian eta/pi/((w-e)^2+eta^2);
    at the HF reference (C = I) A_p is one Lorentzian at eps_p."""
    w = np.linspace(-3, 3, 101)
    A, Ao = O.spectral_function(np.array([0.4]), np.ones((1, 1)), w, 0.05)
    assert np.allclose(A, 0.05 / np.pi / ((w - 0.4) ** 2 + 0.05 ** 2), rtol=1e-14)
    eps = np.array([-1.0, 0.3, 2.0])
    A, Ao = O.spectral_function(eps, np.eye(3), w, 0.1)
    for p in range(3):
        assert np.allclose(Ao[p], 0.1 / np.pi / ((w - eps[p]) ** 2 + 0.01), rtol=1e-14)


def test_spectral_function_sum_rule():
    """Completeness sum_x C_px^2 = 1 of the extended eigenvectors: each A_p
    integrates to the closed-form Lorentzian mass inside the grid, and the
    trace to N times ... summed the same way."""
    rng = np.random.default_rng(4)
    N = 5
    F = rng.standard_normal((N, N)); F = F + F.T
    e, C = O.diagonalise(F, rng.uniform(-3, 3, 2 * N), 0.5 * rng.standard_normal((N, 2 * N)))
    eta, a, b = 0.05, -40.0, 40.0
    w = np.linspace(a, b, 400001)
    A, Ao = O.spectral_function(e, C, w, eta)
    mass = (np.arctan((b - e) / eta) - np.arctan((a - e) / eta)) / np.pi   # per pole
    expect = (C * C) @ mass
    integ = np.trapezoid(Ao, w, axis=1)
    assert np.allclose(integ, expect, atol=1e-6)
    assert abs(np.trapezoid(A, w) - expect.sum()) < 1e-5
    assert abs(expect.sum() - N) < 0.01


@pytest.mark.parametrize("m", [0, 1, 2])
def test_block_lanczos_conserves_moments(m):
    """m+1 block-Lanczos steps from the moments reproduce U^(0..2m+1) of a
    self-energy with many auxiliaries; m = 0 equals the Cholesky compression."""
    rng = np.random.default_rng(10 + m)
    N, K = 4, 40
    E0 = rng.uniform(-2, 2, K)
    v0 = rng.standard_normal((N, K)) / np.sqrt(K)
    nmom = 2 * m + 1
    U = np.array([v0 @ np.diag(E0 ** n) @ v0.T for n in range(nmom + 1)])
    E, v = O.compress_block_lanczos(U)
    assert E.shape == ((m + 1) * N,) and v.shape == (N, (m + 1) * N)
    for n in range(nmom + 1):
        assert rel(v @ np.diag(E ** n) @ v.T, U[n]) < 1e-9
    if m == 0:
        E1, v1 = O.compress(U[0], U[1])
        assert np.allclose(E, E1, atol=1e-12)
        assert rel(v1 @ v1.T, v @ v.T) < 1e-12


def test_block_lanczos_exact_for_small_self_energy():
    """A self-energy with exactly (m+1) N auxiliaries is recovered exactly."""
    rng = np.random.default_rng(5)
    N, m = 3, 1
    K = (m + 1) * N
    E0 = np.sort(rng.uniform(-2, 2, K))
    v0 = rng.standard_normal((N, K))
    U = np.array([v0 @ np.diag(E0 ** n) @ v0.T for n in range(2 * m + 2)])
    E, v = O.compress_block_lanczos(U)
    assert np.max(np.abs(np.sort(E) - E0)) < 1e-8


def test_run_nmom3_weak_coupling_and_moments():
    """AGF2 with moments 0..3 conserved: weak-coupling limit still gives
    E_tot -> E_HF, and its first iteration's compressed auxiliaries reproduce
    all four moments of each sector."""
    s = make_system(8, 3, 10, 30)
    L = 1e-2 * s.L
    h = O.hcore_from_mo_energies(s.eps, L, s.nocc)
    r = O.run(h, L, s.nelec, s.eps, max_iter=3, nmom=3)
    assert abs(r.E_tot - r.E_hf) < 1e-6
    s = make_system(8, 3, 10, 31)
    Uh, Up = O.build_moments(s.L, s.eps, np.eye(8), 0.5 * (s.eps[2] + s.eps[3]), nmom=3)
    for U in (Uh, Up):
        E, v = O.compress_block_lanczos(U)
        for n in range(4):
            assert rel(v @ np.diag(E ** n) @ v.T, U[n]) < 1e-8


def test_block_lanczos_resolvent_energy_converges_to_mp2():
    """With the Hartree-Fock propagator, the Galitskii-Migdal sum over the
    compressed particle self-energy tends to the closed-form MP2 energy as
    more moments are conserved (the uncompressed sum is MP2 exactly): the
    error shrinks at every step and is below 1e-4 relative at nmom = 7."""
    s = make_system(16, 4, 48, 11, scale=0.08)
    N = s.nmo
    mu = 0.5 * (s.eps[3] + s.eps[4])
    mp2 = O.mp2_energy(s.L, s.eps, s.nocc)
    errs = []
    for nmom in (1, 3, 5, 7):
        _, Up = O.build_moments(s.L, s.eps, np.eye(N), mu, nmom=nmom)
        E, v = O.compress_block_lanczos(Up)
        e2 = O.energy_2body(s.eps[:4], np.eye(N)[:, :4], E, v)
        errs.append(abs(e2 - mp2))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4 * abs(mp2), errs


def test_compression_independent_of_the_factor_of_u0():
    """The physical self-energy of the compressed auxiliaries does not depend
    on which factor T of U^(0) = T T^T is used: with the symmetric square root
    in place of the lower Cholesky factor, M' = T'^-1 U1 T'^-T is an orthogonal
    similarity of M, so the auxiliary energies agree and so does
    Sigma(w) = v (w - E)^-1 v^T at any w."""
    s = make_system(10, 3, 30, 41)
    e, C, mu = random_poles(10, 30, 11, 42)
    Uh, Up = O.build_moments(s.L, e, C, mu)
    for U in (Uh, Up):
        E, v = O.compress(U[0], U[1])
        lam, Z = np.linalg.eigh(U[0])
        Ts = Z @ np.diag(np.sqrt(lam)) @ Z.T              # symmetric square root
        Tinv = np.linalg.inv(Ts)
        Es, W = np.linalg.eigh(Tinv @ U[1] @ Tinv.T)
        vs = Ts @ W
        assert np.max(np.abs(E - Es)) < 1e-10 * np.max(np.abs(E))
        for w in (-7.3, 0.41, 5.9):
            sig = (v / (w - E)) @ v.T
            sig_s = (vs / (w - Es)) @ vs.T
            assert rel(sig, sig_s) < 1e-9


def test_run_general_basis_start_matches_canonical():
    """Started from eig(F[D0]) in a rotated orbital basis (hcore, every L^Q and
    D0 rotated by one orthogonal matrix), the iteration is the same physics as
    the canonical-basis start: energies, IP and EA agree."""
    s = make_system(8, 3, 10, 30)
    L = 0.3 * s.L
    h = O.hcore_from_mo_energies(s.eps, L, s.nocc)
    rng = np.random.default_rng(2)
    Qm, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    hr = Qm.T @ h @ Qm
    Lr = np.einsum("pi,Qpq,qj->Qij", Qm, L, Qm)
    D0r = Qm.T @ O.hf_density(8, 3) @ Qm
    a = O.run(h, L, s.nelec, s.eps, max_iter=3, conv_tol=0.0, fock_tol=1e-12)
    b = O.run(hr, Lr, s.nelec, None, max_iter=3, conv_tol=0.0, fock_tol=1e-12, D0=D0r)
    for key in ("E_hf", "E_1b", "E_2b", "E_tot", "ip", "ea", "mu"):
        assert abs(getattr(a, key) - getattr(b, key)) <= 1e-9 * max(1.0, abs(getattr(a, key))), key
