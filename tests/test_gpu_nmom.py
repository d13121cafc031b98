"""More conserved moments (AGF2(m,0), nmom = 2m+1) through the C ABI against
the FP64 oracle: the moment build for nmom = 3, 5 (FP64) and 3 (split
BF16), the block-Lanczos compression from the moments, and whole
iterations with nmom = 3 and 5."""
import numpy as np
import pytest

from oracle import agf2_oracle as O
from paper_2106_03508_gb300.synth import make_system, random_poles

from test_gpu_fp64 import RTOL, dev, empty, host, rel
from test_gpu_mixed import MIXED_RTOL

pytestmark = pytest.mark.gpu


def moments(lib, h, L, e, C, mu, nmom, precision=0):
    naux, nmo, _ = L.shape
    Ld, ed, Cd = dev(L), dev(e), dev(C)
    Uh, Up = empty(nmom + 1, nmo, nmo), empty(nmom + 1, nmo, nmo)
    lib.agf2_build_moments(h.h, Ld.data_ptr(), naux, nmo, ed.data_ptr(), Cd.data_ptr(), len(e),
                           mu, nmom, precision, Uh.data_ptr(), Up.data_ptr())
    return host(Uh), host(Up)


@pytest.mark.parametrize("nmom", [2, 3, 5])
@pytest.mark.parametrize("nmo,nq,no,naux,seed", [
    (24, 72, 29, 96, 1),      # c1-shaped
    (70, 150, 61, 150, 2),    # several 64-tiles, ragged tails
    (9, 20, 1, 5, 3),         # a single occupied pole
])
def test_moments_fp64_nmom(cuda_handle, agf2_lib, nmo, nq, no, naux, seed, nmom):
    s = make_system(nmo, max(1, nmo // 5), naux, seed)
    e, C, mu = random_poles(nmo, nq, no, seed + 7)
    Uh, Up = moments(agf2_lib, cuda_handle, s.L, e, C, mu, nmom)
    Rh, Rp = O.build_moments(s.L, e, C, mu, nmom)
    for n in range(nmom + 1):
        assert rel(Uh[n], Rh[n]) < RTOL, (n, rel(Uh[n], Rh[n]))
        assert rel(Up[n], Rp[n]) < RTOL, (n, rel(Up[n], Rp[n]))


@pytest.mark.parametrize("nmom", [2, 3])
@pytest.mark.parametrize("nmo,nq,no,naux,seed", [
    (24, 72, 29, 96, 1),
    (130, 260, 97, 200, 2),   # two p-tiles (ragged), inner counts past 128
    (9, 20, 19, 1, 4),        # one virtual pole, one auxiliary function
])
def test_moments_mixed_nmom(cuda_handle, agf2_lib, nmo, nq, no, naux, seed, nmom):
    s = make_system(nmo, max(1, nmo // 5), naux, seed)
    e, C, mu = random_poles(nmo, nq, no, seed + 7)
    Uh, Up = moments(agf2_lib, cuda_handle, s.L, e, C, mu, nmom, agf2_lib.AGF2_BF16X3)
    Rh, Rp = O.build_moments(s.L, e, C, mu, nmom)
    for n in range(nmom + 1):
        assert rel(Uh[n], Rh[n]) < MIXED_RTOL, (n, rel(Uh[n], Rh[n]))
        assert rel(Up[n], Rp[n]) < MIXED_RTOL, (n, rel(Up[n], Rp[n]))


def test_moments_mixed_rejects_nmom_4(cuda_handle, agf2_lib):
    s = make_system(9, 2, 5, 3)
    e, C, mu = random_poles(9, 20, 4, 10)
    with pytest.raises(agf2_lib.AGF2Error) as ei:
        moments(agf2_lib, cuda_handle, s.L, e, C, mu, 4, agf2_lib.AGF2_BF16X3)
    assert ei.value.code == agf2_lib.AGF2_ERR_UNSUPPORTED


def compress_gpu(lib, h, U, nmom):
    N = U.shape[1]
    na = (nmom + 1) // 2 * N
    Ud = dev(U[: nmom + 1])
    E, v = empty(na), empty(N, na)
    lib.agf2_compress_moments(h.h, Ud.data_ptr(), N, nmom, E.data_ptr(), v.data_ptr())
    return host(E), host(v)


@pytest.mark.parametrize("nmom", [1, 3, 5])
@pytest.mark.parametrize("sector", [0, 1])
def test_compress_moments_vs_oracle(cuda_handle, agf2_lib, nmom, sector):
    N = 20
    s = make_system(N, 5, 60, 21)
    e, C, mu = random_poles(N, 3 * N, 17, 22)
    U = O.build_moments(s.L, e, C, mu, nmom)[sector]
    E, v = compress_gpu(agf2_lib, cuda_handle, U, nmom)
    if nmom == 1:
        Er, vr = O.compress(U[0], U[1])
    else:
        Er, vr = O.compress_block_lanczos(U)
    assert E.shape == Er.shape and v.shape == vr.shape
    assert np.max(np.abs(E - Er)) < 1e-9 * max(1.0, np.max(np.abs(Er)))
    # eigenvector signs are free: compare sign-invariant products, and the
    # conserved moments v E^n v^T = U^(n), n = 0..nmom
    for n in range(nmom + 1):
        got = (v * E ** n) @ v.T
        assert rel(got, U[n]) < 1e-9, (n, rel(got, U[n]))
        assert rel(got, (vr * Er ** n) @ vr.T) < 1e-9
    assert rel(np.abs(v), np.abs(vr)) < 1e-7


def test_compress_moments_rejects(cuda_handle, agf2_lib):
    N = 6
    U = np.zeros((4, N, N))
    U[0] = -np.eye(N)
    with pytest.raises(agf2_lib.AGF2Error) as ei:
        compress_gpu(agf2_lib, cuda_handle, U, 3)
    assert ei.value.code == agf2_lib.AGF2_ERR_NOT_PD
    with pytest.raises(agf2_lib.AGF2Error) as ei:
        compress_gpu(agf2_lib, cuda_handle, U, 2)
    assert ei.value.code == agf2_lib.AGF2_ERR_INVALID_ARG


def run_gpu(lib, h, s, nmom, nit, precision=0, shift_mode=1):
    import torch
    L, eps = torch.from_numpy(s.L).cuda(), torch.from_numpy(s.eps).cuda()
    hc = torch.empty(s.nmo, s.nmo, dtype=torch.float64, device="cuda")
    lib.agf2_hcore_from_mo_energies(h.h, L.data_ptr(), s.naux, s.nmo, eps.data_ptr(), s.nocc,
                                    hc.data_ptr())
    o = lib.agf2_opts_default()
    o.precision = precision
    o.nmom = nmom
    o.max_iter = 1
    o.fock.max_cycle = 300
    o.fock.tol_D = 1e-12
    o.fock.shift_mode = shift_mode
    out = []
    for it in range(nit):
        o.resume = 1 if it else 0
        rc, r = lib.agf2_run(h.h, hc.data_ptr(), L.data_ptr(), s.naux, s.nmo, s.nelec,
                             None, o)
        out.append(r.as_dict())
    return out


# weakly coupled 16-orbital system: every Fock loop converges well inside the cap
WEAK = dict(nmo=16, nocc=4, naux=48, seed=11, scale=0.08)


@pytest.mark.parametrize("nmom,shift_mode", [(3, 0), (3, 1), (5, 1)])
def test_run_nmom_matches_oracle(cuda_handle, agf2_lib, nmom, shift_mode):
    s = make_system(**WEAK)
    nit = 4
    got = run_gpu(agf2_lib, cuda_handle, s, nmom, nit, shift_mode=shift_mode)
    h = O.hcore_from_mo_energies(s.eps, s.L, s.nocc)
    ref = O.run(h, s.L, s.nelec, s.eps, max_iter=nit, nmom=nmom, fock_max_cycle=300,
                conv_tol=0.0, fock_tol=1e-12)
    assert len(ref.history) == nit
    for g, r in zip(got, ref.history):
        assert g["fock_cycles"] < 300
        for key in ("E_1b", "E_2b", "E_tot", "ip", "ea", "mu"):
            assert abs(g[key] - getattr(r, key)) <= 1e-10 * abs(getattr(r, key)), (
                r.it, key, g[key], getattr(r, key))
    # the state holds nmo + (nmom+1) nmo poles
    nq = agf2_lib.agf2_get_state(cuda_handle.h)
    assert nq == s.nmo * (nmom + 2)
    e = empty(nq)
    agf2_lib.agf2_get_state(cuda_handle.h, e.data_ptr())
    assert np.max(np.abs(host(e) - ref.e)) < 1e-10 * np.max(np.abs(ref.e))


def test_run_nmom3_mixed_close_to_fp64(cuda_handle, agf2_lib):
    s = make_system(**WEAK)
    a = run_gpu(agf2_lib, cuda_handle, s, 3, 4, precision=agf2_lib.AGF2_BF16X3)
    b = run_gpu(agf2_lib, cuda_handle, s, 3, 4)
    for x, y in zip(a, b):
        assert abs(x["E_tot"] - y["E_tot"]) < 1e-6
        assert abs(x["ip"] - y["ip"]) < 1e-5 and abs(x["ea"] - y["ea"]) < 1e-5


def test_run_rejects_even_nmom(cuda_handle, agf2_lib):
    s = make_system(**WEAK)
    with pytest.raises(agf2_lib.AGF2Error) as ei:
        run_gpu(agf2_lib, cuda_handle, s, 2, 1)
    assert ei.value.code == agf2_lib.AGF2_ERR_INVALID_ARG
