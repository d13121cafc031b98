"""FP64 CPU oracle for moment-truncated AGF2 (Backhouse, Santana-Bonilla, Booth,
arXiv 2106.03508).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The library under
``paper_2106_03508_gb300`` never calls it and shares no code with it; the
only shared module is the seeded input generator (random draws only).

Everything is plain NumPy/SciPy in float64 and follows the paper's equations
in order:

* Eq. (fock_matrix)           ``fock_matrix``
* Eq. (mp2_self_energy)       the moments below are its spectral moments
* Eqs. (mp2_zeroth_moment), (mp2_first_moment) and the "analogous" greater
  (particle) sector          ``build_moments`` (per-i / per-a GEMM form) and
                             ``build_moments_loops`` (explicit sums, tiny N);
                             the contribution of chosen outer pole pairs
                             (the summed indices the paper distributes)
                             ``build_moments_pairs``
* Eq. (block_lanczos_chol_3) and the M-block that follows it
                              ``compress``; the higher truncations of the
                              compression paragraph (moments 0..2m+1, m+1
                              block-Lanczos steps from the moments)
                              ``compress_block_lanczos``
* Eq. (post_compression_h) / (dyson_eq_eig)
                              ``diagonalise``
* the density relaxation with a chemical potential keeping the electron count
  in the non-idempotent density (text after Eq. dyson_eq_eig)
                              ``aufbau``, ``solve_shift``, ``fock_loop``
* energies / IP / EA          ``energy_1body``, ``energy_2body`` (IP/EA in ``run``)
* the outer self-consistency  ``run`` (any odd nmom)
* the broadened spectral function of the artemisinin figures
                              ``spectral_function``

Readings taken where the paper is silent (identical on the CUDA side):
  - occupied poles are those with e < mu (a pole exactly at mu is virtual);
  - U is symmetrised as (U + U^T)/2 (the exact sum is symmetric under i<->j);
  - compression uses the lower Cholesky factor T of U^(0) and
    M = T^-1 U^(1) T^-T, so that T M T^T = U^(1) (the paper's (T^-1)^dagger
    U^(1) T^-1 would need T^dagger T = U^(0));
  - mu: aufbau count k minimising |2 sum_{x<k} |C_x|^2 - nelec| and mu at the
    HOQMO/LUQMO midpoint; auxiliary energies shifted by a common delta found
    by bisection on n(delta; k fixed) - nelec;
  - the Fock loop stops when max|dD| < tol_D or after max_cycle cycles
    (50 by default);
  - two-body energy: Galitskii-Migdal pole form with the occupied QMOs and the
    particle-sector auxiliaries;
  - IP = -e_HOQMO, EA = -e_LUQMO.

Parity is pinned (tests/test_oracle.py) by brute-force four-index sums, the
MP2 closed form at the HF reference, the closed-shell Hartree-Fock energy
and the general one-body energy from explicit four-index ERIs, additivity of
the moments over outer-pair slices (and a slice against restricted explicit
sums), the S/D factorisation of the exact
uncompressed self-energy, homogeneity, the compression identities (and
their independence from the factor of U^(0)), the block-Lanczos moment
conservation and its MP2 limit, completeness of the extended eigenvectors,
electron-count conservation, the spectral sum rule and the weak-coupling
limit.  The converged IP/EA/E_tot of the full iteration are
parity unpinned beyond these invariants (the paper's numbers need molecular
data).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


# --------------------------------------------------------------------------
# Mean field: Eq. (fock_matrix) with (pq|rs) = sum_Q L^Q_pq L^Q_rs
# --------------------------------------------------------------------------
def coulomb_exchange(L: np.ndarray, D: np.ndarray):
    """J_pq = sum_rs (pq|rs) D_rs,  K_pq = sum_rs (ps|rq) D_rs."""
    gamma = np.einsum("Qrs,rs->Q", L, D)
    J = np.einsum("Q,Qpq->pq", gamma, L)
    K = np.zeros_like(D)
    for Q in range(L.shape[0]):
        K += L[Q] @ D.T @ L[Q]
    return J, K


def fock_matrix(h: np.ndarray, L: np.ndarray, D: np.ndarray) -> np.ndarray:
    J, K = coulomb_exchange(L, D)
    return h + J - 0.5 * K


def hf_density(nmo: int, nocc: int) -> np.ndarray:
    D = np.zeros((nmo, nmo))
    D[np.arange(nocc), np.arange(nocc)] = 2.0
    return D


def hcore_from_mo_energies(eps: np.ndarray, L: np.ndarray, nocc: int) -> np.ndarray:
    """h such that F[D0] = diag(eps) at the aufbau density D0 (synthetic recipe)."""
    D0 = hf_density(len(eps), nocc)
    J, K = coulomb_exchange(L, D0)
    return np.diag(eps) - (J - 0.5 * K)


# --------------------------------------------------------------------------
# Self-energy moments, Eqs. (mp2_zeroth_moment), (mp2_first_moment)
# --------------------------------------------------------------------------
def split_poles(e: np.ndarray, C: np.ndarray, mu: float):
    occ = e < mu
    return e[occ], C[:, occ], e[~occ], C[:, ~occ]


def rotate(L: np.ndarray, Co: np.ndarray, Cv: np.ndarray):
    """DF integrals in the pole basis: (xi|Q), (xa|Q), (ia|Q)."""
    Lxo = L @ Co                       # [Q, N, o]
    Lxv = L @ Cv                       # [Q, N, v]
    Lov = Co.T[None, :, :] @ Lxv       # [Q, o, v]
    return Lxo, Lxv, Lov


def build_moments(L, e, C, mu, nmom: int = 1, outer_occ=None, outer_vir=None):
    """U_<^(n), U_>^(n) for n = 0..nmom, each [nmom+1, N, N].

    Hole:     U_pq = sum_{ija} (pi|ja)[2(qi|ja) - (qj|ia)] (e_i+e_j-e_a)^n
    Particle: U_pq = sum_{abi} (pa|bi)[2(qa|bi) - (qb|ai)] (e_a+e_b-e_i)^n
    evaluated one summed index (i, resp. a) at a time, as in the paper's
    block-distributed algorithm.  ``outer_occ`` / ``outer_vir`` (positions
    in the occupied / virtual pole lists) restrict that first summed index
    to a slice -- the share one of the paper's ranks computes; the slices of
    a partition add up to the whole.
    """
    N = L.shape[1]
    eo, Co, ev, Cv = split_poles(e, C, mu)
    Lxo, Lxv, Lov = rotate(L, Co, Cv)
    Lvo = Lov.transpose(0, 2, 1)       # (ai|Q) = (ia|Q)
    Uh = np.zeros((nmom + 1, N, N))
    Up = np.zeros((nmom + 1, N, N))
    for i in (range(len(eo)) if outer_occ is None else outer_occ):
        X = np.tensordot(Lxo[:, :, i], Lov, axes=(0, 0))        # (pi|ja) [p,j,a]
        Xk = np.tensordot(Lxo, Lov[:, i, :], axes=(0, 0))       # (pj|ia) [p,j,a]
        Xt = (2.0 * X - Xk).reshape(N, -1)
        w = (eo[i] + eo[:, None] - ev[None, :]).reshape(-1)
        X = X.reshape(N, -1)
        for n in range(nmom + 1):
            Uh[n] += (X * w ** n) @ Xt.T
    for a in (range(len(ev)) if outer_vir is None else outer_vir):
        X = np.tensordot(Lxv[:, :, a], Lvo, axes=(0, 0))        # (pa|bi) [p,b,i]
        Xk = np.tensordot(Lxv, Lvo[:, a, :], axes=(0, 0))       # (pb|ai) [p,b,i]
        Xt = (2.0 * X - Xk).reshape(N, -1)
        w = (ev[a] + ev[:, None] - eo[None, :]).reshape(-1)
        X = X.reshape(N, -1)
        for n in range(nmom + 1):
            Up[n] += (X * w ** n) @ Xt.T
    Uh = 0.5 * (Uh + Uh.transpose(0, 2, 1))
    Up = 0.5 * (Up + Up.transpose(0, 2, 1))
    return Uh, Up


def build_moments_pairs(L, e, C, mu, nmom: int = 1, hole_pairs=(), part_pairs=()):
    """Contribution of chosen outer pole pairs to the moments (the summed
    outer indices that the paper's parallel algorithm hands out in blocks).

    ``hole_pairs`` lists unordered pairs (x, y), x <= y, of positions in the
    occupied pole list (poles with e < mu in ascending pole order); the pair
    contributes the ordered terms (i, j) = (x, y) and, for x != y, (y, x) of
    U_<^(n)_pq = sum_{ija} (pi|ja)[2(qi|ja) - (qj|ia)] (e_i+e_j-e_a)^n.
    ``part_pairs`` does the same for the virtual outer pair (a, b) of the
    particle sector.  Summed over every unordered pair, this is
    ``build_moments``.  Returns the symmetrised (hole, particle) partial
    moments, each [nmom+1, N, N]."""
    N = L.shape[1]
    eo, Co, ev, Cv = split_poles(e, C, mu)
    Lxo, Lxv, Lov = rotate(L, Co, Cv)
    Lvo = Lov.transpose(0, 2, 1)
    out = []
    for pairs, Lx, Lp, e_out, e_in in ((hole_pairs, Lxo, Lov, eo, ev),
                                      (part_pairs, Lxv, Lvo, ev, eo)):
        U = np.zeros((nmom + 1, N, N))
        for x, y in pairs:
            ordered = [(x, y)] if x == y else [(x, y), (y, x)]
            for i, j in ordered:
                Xij = np.tensordot(Lx[:, :, i], Lp[:, j, :], axes=(0, 0))   # (pi|jc) [p, c]
                Xji = np.tensordot(Lx[:, :, j], Lp[:, i, :], axes=(0, 0))   # (pj|ic) [p, c]
                w = e_out[i] + e_out[j] - e_in
                for n in range(nmom + 1):
                    U[n] += (Xij * w ** n) @ (2.0 * Xij - Xji).T
        out.append(0.5 * (U + U.transpose(0, 2, 1)))
    return out[0], out[1]


def moment_elements(L, e, C, mu, pq, nmom: int = 1):
    """Selected elements U^(n)_pq of both sectors straight from the definition
    (Eqs. mp2_zeroth_moment, mp2_first_moment), one (p, q) at a time:
    X_p[i,j,a] = (pi|ja), U_pq = sum_ija X_p[i,j,a] (2 X_q[i,j,a] - X_q[j,i,a]) w^n.
    For sampled parity at sizes where the full build is out of reach.
    Returns (hole [len(pq), nmom+1], particle [len(pq), nmom+1]), symmetrised."""
    eo, Co, ev, Cv = split_poles(e, C, mu)
    Lxo, Lxv, Lov = rotate(L, Co, Cv)
    Lvo = Lov.transpose(0, 2, 1)
    wh = eo[:, None, None] + eo[None, :, None] - ev[None, None, :]
    wp = ev[:, None, None] + ev[None, :, None] - eo[None, None, :]

    def xh(p):  # (pi|ja) [i, j, a]
        return np.tensordot(Lxo[:, p, :], Lov, axes=(0, 0))

    def xp(p):  # (pa|bi) [a, b, i]
        return np.tensordot(Lxv[:, p, :], Lvo, axes=(0, 0))

    out_h = np.zeros((len(pq), nmom + 1))
    out_p = np.zeros((len(pq), nmom + 1))
    for t, (p, q) in enumerate(pq):
        for X, w, out in ((xh, wh, out_h), (xp, wp, out_p)):
            Xp, Xq = X(p), X(q)
            tp = Xp * (2.0 * Xq - Xq.transpose(1, 0, 2))
            tq = Xq * (2.0 * Xp - Xp.transpose(1, 0, 2))
            for n in range(nmom + 1):
                out[t, n] = 0.5 * (np.sum(tp * w ** n) + np.sum(tq * w ** n))
    return out_h, out_p


def pole_eris(L, C):
    """Four-index ERIs in the pole basis by brute force: (px|yz), p physical."""
    eri = np.einsum("Qpq,Qrs->pqrs", L, L)
    return np.einsum("pqrs,qx,ry,sz->pxyz", eri, C, C, C)


def build_moments_loops(L, e, C, mu, nmom: int = 1):
    """Explicit-sum moments from four-index ERIs; pure Python, tiny sizes only."""
    N = L.shape[1]
    occ = [x for x in range(len(e)) if e[x] < mu]
    vir = [x for x in range(len(e)) if not e[x] < mu]
    g = pole_eris(L, C)                # g[p, x, y, z] = (px|yz)
    Uh = np.zeros((nmom + 1, N, N))
    Up = np.zeros((nmom + 1, N, N))
    for p in range(N):
        for q in range(N):
            for i in occ:
                for j in occ:
                    for a in vir:
                        t = g[p, i, j, a] * (2.0 * g[q, i, j, a] - g[q, j, i, a])
                        w = e[i] + e[j] - e[a]
                        for n in range(nmom + 1):
                            Uh[n, p, q] += t * w ** n
            for a in vir:
                for b in vir:
                    for i in occ:
                        t = g[p, a, b, i] * (2.0 * g[q, a, b, i] - g[q, b, a, i])
                        w = e[a] + e[b] - e[i]
                        for n in range(nmom + 1):
                            Up[n, p, q] += t * w ** n
    return Uh, Up


# --------------------------------------------------------------------------
# Moment-conserving compression, Eq. (block_lanczos_chol_3) and M-block
# --------------------------------------------------------------------------
class NotPositiveDefinite(ValueError):
    pass


def compress(U0: np.ndarray, U1: np.ndarray):
    """One block-Lanczos step as a Cholesky: T T^T = U0, M = T^-1 U1 T^-T,
    M = W diag(E) W^T, couplings v = T W.  Conserves v v^T = U0 and
    v diag(E) v^T = U1.  Returns (E[N] ascending, v[N, N])."""
    try:
        T = np.linalg.cholesky(U0)
    except np.linalg.LinAlgError as exc:
        raise NotPositiveDefinite(str(exc)) from exc
    Y = sla.solve_triangular(T, U1, lower=True)          # T^-1 U1
    M = sla.solve_triangular(T, Y.T, lower=True)         # T^-1 (T^-1 U1)^T
    M = 0.5 * (M + M.T)
    E, W = np.linalg.eigh(M)
    return E, T @ W


def compress_block_lanczos(U):
    """Moment-conserving compression for nmom = 2m+1 (U has 2m+2 moments,
    U[n] = v E^n v^T): m+1 steps of block Lanczos on the auxiliary space,
    driven by the moments alone.  With Q_i = sum_k E^k V C[i][k] (V = v^T),
    Q_i^T E^n Q_j = sum_kl C[i][k]^T U^(k+l+n) C[j][l]:
      U0 = B0 B0^T (lower Cholesky), C[1][0] = B0^-T,
      A_i = Q_i^T E Q_i,  R_i = E Q_i - Q_i A_i - Q_{i-1} B_{i-1}^T,
      R_i^T R_i = B_i^T B_i (B_i upper),  Q_{i+1} = R_i B_i^-1.
    The block-tridiagonal H = [[A_1, B_1^T], [B_1, A_2, ...]] of size (m+1) N
    with couplings [B0, 0, ...] conserves U^(0..2m+1); diagonalised,
    H = W diag(E') W^T, the auxiliaries are (E', B0 W[:N]).  m = 0 is
    Eq. (block_lanczos_chol_3) with its M-block.  Returns (E' [(m+1)N],
    v' [N, (m+1)N])."""
    nmom = U.shape[0] - 1
    if nmom % 2 != 1:
        raise ValueError("nmom must be odd (2m+1)")
    m = (nmom - 1) // 2
    N = U.shape[1]
    try:
        B0 = np.linalg.cholesky(U[0])
    except np.linalg.LinAlgError as exc:
        raise NotPositiveDefinite(str(exc)) from exc

    def mom(Ci, Cj, n):  # Q_i^T E^n Q_j
        out = np.zeros((N, N))
        for k, a in enumerate(Ci):
            for l, b in enumerate(Cj):
                out += a.T @ U[k + l + n] @ b
        return out

    C_prev = None
    C_cur = [sla.solve_triangular(B0, np.eye(N), lower=True).T]   # B0^-T
    A_blocks, B_blocks = [], []
    B_prev = None
    for i in range(m + 1):
        A = mom(C_cur, C_cur, 1)
        A = 0.5 * (A + A.T)
        A_blocks.append(A)
        if i == m:
            break
        # coefficients of R_i
        CR = [np.zeros((N, N)) for _ in range(len(C_cur) + 1)]
        for k, c in enumerate(C_cur):
            CR[k + 1] += c
            CR[k] -= c @ A
        if C_prev is not None:
            for k, c in enumerate(C_prev):
                CR[k] -= c @ B_prev.T
        S = mom(CR, CR, 0)
        S = 0.5 * (S + S.T)
        try:
            Lc = np.linalg.cholesky(S)
        except np.linalg.LinAlgError as exc:
            raise NotPositiveDefinite(str(exc)) from exc
        B = Lc.T                                      # B^T B = S
        Binv = sla.solve_triangular(B, np.eye(N), lower=False)
        C_prev, C_cur = C_cur, [c @ Binv for c in CR]
        B_prev = B
        B_blocks.append(B)
    nb = m + 1
    H = np.zeros((nb * N, nb * N))
    for i in range(nb):
        H[i * N:(i + 1) * N, i * N:(i + 1) * N] = A_blocks[i]
    for i in range(m):
        H[(i + 1) * N:(i + 2) * N, i * N:(i + 1) * N] = B_blocks[i]
        H[i * N:(i + 1) * N, (i + 1) * N:(i + 2) * N] = B_blocks[i].T
    E, W = np.linalg.eigh(H)
    return E, B0 @ W[:N, :]


# --------------------------------------------------------------------------
# Extended Hamiltonian, Eq. (post_compression_h) / (dyson_eq_eig)
# --------------------------------------------------------------------------
def extended_hamiltonian(F, E, v):
    N, M = v.shape
    H = np.zeros((N + M, N + M))
    H[:N, :N] = F
    H[:N, N:] = v
    H[N:, :N] = v.T
    H[N:, N:] = np.diag(E)
    return H


def diagonalise(F, E, v):
    """Poles e[N+M] (ascending) and physical couplings C[N, N+M]."""
    w, V = np.linalg.eigh(extended_hamiltonian(F, E, v))
    return w, V[: F.shape[0], :]


def aufbau(e, C, nelec):
    """Number k of occupied QMOs minimising |2 sum_{x<k} |C_x|^2 - nelec|,
    mu at the HOQMO/LUQMO midpoint, and that count's electron number."""
    wts = np.sum(C * C, axis=0)
    cum = np.concatenate([[0.0], 2.0 * np.cumsum(wts)])
    k = int(np.argmin(np.abs(cum - nelec)))
    k = min(max(k, 1), len(e) - 1)
    mu = 0.5 * (e[k - 1] + e[k])
    return k, mu, cum[k]


def electron_number(F, E, v, k, delta):
    e, C = diagonalise(F, E + delta, v)
    return 2.0 * np.sum(C[:, :k] ** 2)


@dataclass
class ShiftInfo:
    delta: float
    nerr: float
    evals: int
    converged: bool


def solve_shift(F, E, v, nelec, tol=1e-11, max_iter=200, step0=1.0, max_expand=60):
    """Common shift delta of the auxiliary energies with
    n(delta; k) = nelec, k = the aufbau count at delta = 0.  n increases with
    delta; bracket by doubling steps, then bisection until |n - nelec| < tol
    or the bracket is below 1e-14 wide."""
    e0, C0 = diagonalise(F, E, v)
    k, _, _ = aufbau(e0, C0, nelec)
    evals = 1
    f0 = 2.0 * np.sum(C0[:, :k] ** 2) - nelec
    if abs(f0) < tol:
        return ShiftInfo(0.0, f0, evals, True)
    lo, flo, hi, fhi = (0.0, f0, None, None) if f0 < 0 else (None, None, 0.0, f0)
    step = step0
    for _ in range(max_expand):
        d = (step if lo is not None else -step)
        f = electron_number(F, E, v, k, d) - nelec
        evals += 1
        if f < 0:
            lo, flo = d, f
        else:
            hi, fhi = d, f
        if lo is not None and hi is not None:
            break
        step *= 2.0
    if lo is None or hi is None:
        best = 0.0 if lo is None and hi is None else (lo if lo is not None else hi)
        return ShiftInfo(best, flo if lo is not None else fhi, evals, False)
    best, fbest = (lo, flo) if abs(flo) < abs(fhi) else (hi, fhi)
    for _ in range(max_iter):
        if abs(fbest) < tol or hi - lo < 1e-14:
            break
        mid = 0.5 * (lo + hi)
        f = electron_number(F, E, v, k, mid) - nelec
        evals += 1
        if abs(f) < abs(fbest):
            best, fbest = mid, f
        if f < 0:
            lo = mid
        else:
            hi = mid
    return ShiftInfo(best, fbest, evals, abs(fbest) < tol)


@dataclass
class FockResult:
    D: np.ndarray
    F: np.ndarray
    e: np.ndarray
    C: np.ndarray
    mu: float
    nocc_qmo: int
    E_shift: np.ndarray
    cycles: int
    converged: bool
    nerr: float


def diis_extrapolate(hist):
    """Pulay extrapolation: c minimising |sum_i c_i r_i| with sum_i c_i = 1,
    next input = sum_i c_i (x_i + r_i) for history entries (x_i, r_i)."""
    m = len(hist)
    B = np.zeros((m + 1, m + 1))
    for a in range(m):
        for b in range(m):
            B[a, b] = np.sum(hist[a][1] * hist[b][1])
    B[m, :m] = 1.0
    B[:m, m] = 1.0
    rhs = np.zeros(m + 1)
    rhs[m] = 1.0
    c = np.linalg.solve(B, rhs)[:m]
    return sum(c[a] * (hist[a][0] + hist[a][1]) for a in range(m))


def fock_loop(h, L, nelec, E_se, v_se, D, tol_D=1e-10, max_cycle=50, shift_tol=1e-11,
              damping=0.3, diis_start=10, diis_space=6):
    """Relax D = 2 C_occ C_occ^T self-consistently with F[D], keeping the
    electron count through a common shift of the auxiliary energies.

    Cycle c (1-based): solve the shift, diagonalise, aufbau, D_new, F_out =
    F[D_new].  The next input Fock matrix is F + damping (F_out - F) for
    c < diis_start, then the Pulay extrapolation over the last
    ``diis_space`` (input, output - input) pairs."""
    E = np.array(E_se, dtype=np.float64, copy=True)
    F = fock_matrix(h, L, D)
    hist = []
    converged = False
    cyc = 0
    info = None
    for cyc in range(1, max_cycle + 1):
        info = solve_shift(F, E, v_se, nelec, tol=shift_tol)
        E = E + info.delta
        e, C = diagonalise(F, E, v_se)
        k, mu, _ = aufbau(e, C, nelec)
        D_new = 2.0 * C[:, :k] @ C[:, :k].T
        F_out = fock_matrix(h, L, D_new)
        dD = np.max(np.abs(D_new - D))
        D = D_new
        if dD < tol_D:
            converged = True
            break
        if cyc >= diis_start and diis_space > 1:
            hist.append((F, F_out - F))
            if len(hist) > diis_space:
                hist.pop(0)
        if len(hist) > 1:
            F = diis_extrapolate(hist)
        else:
            F = F + damping * (F_out - F)
    F = fock_matrix(h, L, D)
    return FockResult(D, F, e, C, mu, k, E, cyc, converged, info.nerr)


# --------------------------------------------------------------------------
# Energies
# --------------------------------------------------------------------------
def energy_1body(h, F, D):
    return 0.5 * np.sum(D * (h + F))


def energy_2body(e_occ, C_occ, E_vir, v_vir):
    """Galitskii-Migdal pole form: sum_{x occ} sum_k (C_x . v_k)^2 / (e_x - E_k)."""
    if C_occ.shape[1] == 0 or v_vir.shape[1] == 0:
        return 0.0
    V = C_occ.T @ v_vir                                  # [x, k]
    return float(np.sum(V * V / (e_occ[:, None] - E_vir[None, :])))


def mp2_energy(L, eps, nocc):
    """Closed-shell MP2 from the HF reference (textbook closed form)."""
    Lov = L[:, :nocc, nocc:]
    g = np.einsum("Qia,Qjb->iajb", Lov, Lov)
    eo, ev = eps[:nocc], eps[nocc:]
    den = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]
    return float(np.sum(g * (2.0 * g - g.transpose(0, 3, 2, 1)) / den))


# --------------------------------------------------------------------------
# Outer AGF2 self-consistency
# --------------------------------------------------------------------------
@dataclass
class IterRecord:
    it: int
    E_1b: float
    E_2b: float
    E_tot: float
    ip: float
    ea: float
    mu: float
    fock_cycles: int


@dataclass
class RunResult:
    E_hf: float
    E_1b: float
    E_2b: float
    E_tot: float
    ip: float
    ea: float
    mu: float
    iterations: int
    converged: bool
    e: np.ndarray
    C: np.ndarray
    D: np.ndarray
    history: list = field(default_factory=list)
    moments: list = field(default_factory=list)


def run(h, L, nelec, eps0, max_iter=50, conv_tol=1e-8, nmom=1, fock_tol=1e-10,
        fock_max_cycle=50, diis_space=0, diis_start=2, mix=1.0, keep_moments=False, D0=None):
    """AGF2 from the HF reference (Eq. gf_hf).  With D0 (the reference
    density in the basis of h and L) the initial poles and couplings are the
    eigenpairs of F[D0]; without it the basis is that of the reference's
    canonical orbitals: poles e = eps0, C = I, D0 the aufbau density.

    Each iteration: moments from the current poles, DIIS on the stacked
    moments (U_<^(0), U_<^(1), U_>^(0), U_>^(1)) from iteration
    ``diis_start`` on, compression of each sector, Fock loop, energies."""
    N = h.shape[0]
    nocc = nelec // 2
    D = hf_density(N, nocc) if D0 is None else np.array(D0, dtype=np.float64)
    F = fock_matrix(h, L, D)
    E_hf = energy_1body(h, F, D)
    if D0 is None:
        e = np.array(eps0, dtype=np.float64)
        C = np.eye(N)
    else:
        e, C = np.linalg.eigh(F)
    mu = 0.5 * (e[nocc - 1] + e[nocc])
    hist = []
    moms = []
    diis_hist = []
    U_prev = None
    E_prev = E_hf
    converged = False
    rec = None
    it = 0
    for it in range(1, max_iter + 1):
        Uh, Up = build_moments(L, e, C, mu, nmom)
        if keep_moments:
            moms.append((Uh.copy(), Up.copy()))
        U = np.concatenate([Uh, Up])
        if U_prev is not None and it >= diis_start and diis_space > 1:
            diis_hist.append((U_prev, U - U_prev))
            if len(diis_hist) > diis_space:
                diis_hist.pop(0)
            if len(diis_hist) > 1:
                U = diis_extrapolate(diis_hist)
        elif U_prev is not None:
            U = U_prev + mix * (U - U_prev)
        U_prev = U
        Uh, Up = U[: nmom + 1], U[nmom + 1:]
        if nmom == 1:
            Eh, vh = compress(Uh[0], Uh[1])
            Ep, vp = compress(Up[0], Up[1])
        else:
            Eh, vh = compress_block_lanczos(Uh)
            Ep, vp = compress_block_lanczos(Up)
        E_se = np.concatenate([Eh, Ep])
        v_se = np.concatenate([vh, vp], axis=1)
        fr = fock_loop(h, L, nelec, E_se, v_se, D, tol_D=fock_tol, max_cycle=fock_max_cycle)
        D, e, C, mu = fr.D, fr.e, fr.C, fr.mu
        k = fr.nocc_qmo
        E1 = energy_1body(h, fr.F, D)
        nh = len(Eh)
        E2 = energy_2body(e[:k], C[:, :k], fr.E_shift[nh:], v_se[:, nh:])
        Et = E1 + E2
        rec = IterRecord(it, E1, E2, Et, -e[k - 1], -e[k], mu, fr.cycles)
        hist.append(rec)
        if abs(Et - E_prev) < conv_tol:
            converged = True
            break
        E_prev = Et
    return RunResult(E_hf, rec.E_1b, rec.E_2b, rec.E_tot, rec.ip, rec.ea, rec.mu,
                     it, converged, e, C, D, hist, moms)


def spectral_function(e, C, omega, eta):
    """A_p(w) = -(1/pi) Im G_pp(w + i eta) = (1/pi) sum_x C_px^2 eta / ((w - e_x)^2 + eta^2)
    for the physical orbitals p, and A(w) = sum_p A_p(w) (the trace; the
    broadened spectra of the paper's artemisinin figure).  Returns (A [nw], A_orb [N, nw])."""
    lor = eta / np.pi / ((omega[None, :] - e[:, None]) ** 2 + eta ** 2)   # [x, w]
    A_orb = (C * C) @ lor
    return A_orb.sum(axis=0), A_orb


def flops_moments(nmo, nocc_poles, nvir_poles, naux, nmom=1):
    """Algorithmic flop count of one moment build (both sectors)."""
    o, v = nocc_poles, nvir_poles
    return nmo * o * v * (o + v) * (2 * naux + 2 * (nmom + 1) * nmo)
