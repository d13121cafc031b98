"""FP64 CUDA path vs the FP64 oracle, through the C ABI (GPU only)."""
import numpy as np
import pytest

from oracle import agf2_oracle as O
from paper_2106_03508_gb300.synth import make_system, random_poles

pytestmark = pytest.mark.gpu
RTOL = 1e-10   # FP64 path: relative 1e-10 on moments and energies


def dev(x, dtype=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=dtype or np.float64)).cuda()


def empty(*shape):
    import torch
    return torch.empty(*shape, dtype=torch.float64, device="cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def gpu_moments(lib, h, L, e, C, mu, precision=0):
    naux, nmo, _ = L.shape
    nq = len(e)
    Ld, ed, Cd = dev(L), dev(e), dev(C)
    Uh, Up = empty(2, nmo, nmo), empty(2, nmo, nmo)
    lib.agf2_build_moments(h.h, Ld.data_ptr(), naux, nmo, ed.data_ptr(), Cd.data_ptr(), nq, mu, 1,
                           precision, Uh.data_ptr(), Up.data_ptr())
    return host(Uh), host(Up)


def test_hcore(cuda_handle, agf2_lib):
    s = make_system(37, 8, 70, 3)
    hc = empty(37, 37)
    L, eps = dev(s.L), dev(s.eps)
    agf2_lib.agf2_hcore_from_mo_energies(cuda_handle.h, L.data_ptr(), s.naux, s.nmo,
                                         eps.data_ptr(), s.nocc, hc.data_ptr())
    assert rel(host(hc), O.hcore_from_mo_energies(s.eps, s.L, s.nocc)) < 1e-12


@pytest.mark.parametrize("nmo,nq,no,naux,seed", [
    (24, 72, 29, 96, 1),      # c1-shaped, iteration >= 2 pole count
    (70, 150, 61, 150, 2),    # several 64-tiles in every GEMM dim, ragged tails
    (9, 20, 1, 5, 3),         # a single occupied pole
    (9, 20, 19, 1, 4),        # a single virtual pole, one auxiliary function
    (65, 130, 40, 33, 5),     # one past a tile edge
])
def test_moments_fp64_vs_oracle(cuda_handle, agf2_lib, nmo, nq, no, naux, seed):
    s = make_system(nmo, max(1, nmo // 5), naux, seed)
    e, C, mu = random_poles(nmo, nq, no, seed + 7)
    perm = np.random.default_rng(seed).permutation(nq)  # poles in arbitrary order
    e, C = e[perm], C[:, perm]
    Uh, Up = gpu_moments(agf2_lib, cuda_handle, s.L, e, C, mu)
    Rh, Rp = O.build_moments(s.L, e, C, mu)
    for n in range(2):
        assert rel(Uh[n], Rh[n]) < RTOL, n
        assert rel(Up[n], Rp[n]) < RTOL, n
        assert np.array_equal(Uh[n], Uh[n].T)


def test_moments_fp64_hf_reference(cuda_handle, agf2_lib):
    s = make_system(40, 8, 160, 9)
    mu = 0.5 * (s.eps[7] + s.eps[8])
    Uh, Up = gpu_moments(agf2_lib, cuda_handle, s.L, s.eps, np.eye(40), mu)
    Rh, Rp = O.build_moments(s.L, s.eps, np.eye(40), mu)
    assert rel(Uh, Rh) < RTOL and rel(Up, Rp) < RTOL


def test_moments_rejects_no_virtual(cuda_handle, agf2_lib):
    s = make_system(6, 2, 4, 1)
    e = np.linspace(-2, -1, 6)
    with pytest.raises(agf2_lib.AGF2Error) as ei:
        gpu_moments(agf2_lib, cuda_handle, s.L, e, np.eye(6), 0.0)
    assert ei.value.code == agf2_lib.AGF2_ERR_INVALID_ARG


def test_compress_vs_oracle(cuda_handle, agf2_lib):
    s = make_system(50, 10, 120, 13)
    e, C, mu = random_poles(50, 150, 60, 13)
    Rh, Rp = O.build_moments(s.L, e, C, mu)
    for U in (Rh, Rp):
        Ud = dev(U)
        E, v = empty(50), empty(50, 50)
        agf2_lib.agf2_compress(cuda_handle.h, Ud.data_ptr(), 50, E.data_ptr(), v.data_ptr())
        E, v = host(E), host(v)
        E0, v0 = O.compress(U[0], U[1])
        assert rel(E, E0) < RTOL
        sgn = np.sign(np.sum(v * v0, axis=0))
        assert rel(v * sgn, v0) < 1e-8
        assert rel(v @ v.T, U[0]) < 1e-11


def test_compress_not_pd(cuda_handle, agf2_lib):
    U = np.zeros((2, 4, 4))
    U[0] = np.diag([1.0, 2.0, -1e-3, 3.0])
    U[1] = np.eye(4)
    Ud = dev(U)
    E, v = empty(4), empty(4, 4)
    rc = agf2_lib.agf2_compress(cuda_handle.h, Ud.data_ptr(), 4, E.data_ptr(), v.data_ptr(),
                                allow=(agf2_lib.AGF2_ERR_NOT_PD,))
    assert rc == agf2_lib.AGF2_ERR_NOT_PD


def _first_iteration_self_energy(s, h):
    N, no = s.nmo, s.nocc
    Uh, Up = O.build_moments(s.L, s.eps, np.eye(N), 0.5 * (s.eps[no - 1] + s.eps[no]))
    Eh, vh = O.compress(Uh[0], Uh[1])
    Ep, vp = O.compress(Up[0], Up[1])
    return np.concatenate([Eh, Ep]), np.concatenate([vh, vp], 1)


@pytest.mark.parametrize("shift_mode", [0, 1])
def test_fock_loop_vs_oracle(cuda_handle, agf2_lib, shift_mode):
    """Same synthetic self-energy (drawn by the seeded generator) into both
    Fock loops; both shift modes reach the oracle's fixed point."""
    s = make_system(16, 4, 40, 5)
    h = O.hcore_from_mo_energies(s.eps, s.L, s.nocc)
    rng = np.random.default_rng(77)
    nse = 32
    E = np.sort(np.concatenate([rng.uniform(-4, -1, 16), rng.uniform(1, 5, 16)]))
    v = 0.3 * rng.standard_normal((16, nse))
    D0 = O.hf_density(16, 4)
    ref = O.fock_loop(h, s.L, s.nelec, E, v, D0, tol_D=1e-12, max_cycle=300)
    hd, Ld, Ed, vd, Dd = dev(h), dev(s.L), dev(E), dev(v), dev(D0)
    F, eq, Cq = empty(16, 16), empty(16 + nse), empty(16, 16 + nse)
    opts = agf2_lib.agf2_fock_opts_default()
    opts.shift_mode = shift_mode
    opts.max_cycle = 300
    opts.tol_D = 1e-12
    rc, info = agf2_lib.agf2_fock_loop(cuda_handle.h, hd.data_ptr(), Ld.data_ptr(), s.naux, 16,
                                       s.nelec, Ed.data_ptr(), vd.data_ptr(), nse, Dd.data_ptr(),
                                       F.data_ptr(), eq.data_ptr(), Cq.data_ptr(), opts)
    assert ref.converged and info.converged
    assert info.nocc_qmo == ref.nocc_qmo
    assert abs(info.mu - ref.mu) < 1e-10 * abs(ref.mu)
    assert rel(host(Dd), ref.D) < 1e-10
    assert rel(host(F), ref.F) < 1e-10
    assert rel(host(eq), ref.e) < 1e-10
    assert rel(host(Ed), ref.E_shift) < 1e-10
    Cg = host(Cq)
    k = ref.nocc_qmo
    assert abs(2 * np.sum(Cg[:, :k] ** 2) - s.nelec) < 1e-9


def run_gpu(lib, h, s, hcore, max_iter, precision=0, resume=0, tol_D=1e-10):
    L, hc, eps = dev(s.L), dev(hcore), dev(s.eps)
    o = lib.agf2_opts_default()
    o.max_iter = max_iter
    o.precision = precision
    o.resume = resume
    o.fock.tol_D = tol_D
    o.fock.max_cycle = 300
    rc, out = lib.agf2_run(h.h, hc.data_ptr(), L.data_ptr(), s.naux, s.nmo, s.nelec,
                           None, o)
    return out


def test_run_small_vs_oracle(cuda_handle, agf2_lib):
    """Whole AGF2 iterations (moments, compression, Fock loop, energies) on a
    small synthetic system with weaker coupling, iterated to convergence."""
    s = make_system(12, 3, 30, 8)
    s.L *= 0.5
    h = O.hcore_from_mo_energies(s.eps, s.L, s.nocc)
    # both Fock loops converge the density to 1e-12, so that their fixed points
    # agree well below the relative 1e-10 asserted on the energies
    ref = O.run(h, s.L, s.nelec, s.eps, max_iter=30, fock_tol=1e-12, fock_max_cycle=300)
    out = run_gpu(agf2_lib, cuda_handle, s, h, 30, tol_D=1e-12)
    assert out.iterations == ref.iterations
    assert out.converged == int(ref.converged)
    for a, b in ((out.E_hf, ref.E_hf), (out.E_tot, ref.E_tot), (out.E_1b, ref.E_1b),
                 (out.E_2b, ref.E_2b), (out.ip, ref.ip), (out.ea, ref.ea)):
        assert abs(a - b) <= 1e-10 * abs(b), (a, b)


def test_run_in_rotated_orbital_basis(cuda_handle, agf2_lib):
    """agf2_run takes its initial poles from eig(F[D0]) in whatever basis it is
    given (Eq. gf_hf): with hcore, every L^Q and the reference density D0
    rotated by one random orthogonal matrix, the iterations reproduce the
    canonical-basis run (and the oracle) -- energies, IP, EA and mu -- to a
    relative 1e-10."""
    import torch
    s = make_system(12, 3, 30, 8)
    s.L *= 0.5
    h = O.hcore_from_mo_energies(s.eps, s.L, s.nocc)
    rng = np.random.default_rng(44)
    Qm, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    hr = Qm.T @ h @ Qm
    Lr = np.ascontiguousarray(np.einsum("pi,Qpq,qj->Qij", Qm, s.L, Qm))
    D0r = Qm.T @ O.hf_density(12, 3) @ Qm
    out = {}
    for name, (hh, LL, D0) in (("canonical", (h, s.L, None)), ("rotated", (hr, Lr, D0r))):
        hd, Ld = dev(hh), dev(LL)
        D0d = dev(D0) if D0 is not None else None
        o = agf2_lib.agf2_opts_default()
        o.max_iter = 4
        o.conv_tol = 0.0
        o.fock.tol_D = 1e-12
        o.fock.max_cycle = 300
        rc, r = agf2_lib.agf2_run(cuda_handle.h, hd.data_ptr(), Ld.data_ptr(), s.naux, 12, s.nelec,
                                  None if D0d is None else D0d.data_ptr(), o)
        out[name] = r.as_dict()
    ref = O.run(h, s.L, s.nelec, s.eps, max_iter=4, fock_tol=1e-12, conv_tol=0.0,
                fock_max_cycle=300)
    bad = []
    for key in ("E_hf", "E_1b", "E_2b", "E_tot", "ip", "ea", "mu"):
        a, b, r = out["rotated"][key], out["canonical"][key], getattr(ref, key)
        # energies relative; the chemical potential and pole energies (mu is
        # -0.013 Ha here) against the Hartree scale
        scale = abs(b) if key.startswith("E") else max(1.0, abs(b))
        if abs(a - b) > 1e-10 * scale or abs(b - r) > 1e-10 * scale:
            bad.append((key, a, b, r))
    assert not bad, bad
