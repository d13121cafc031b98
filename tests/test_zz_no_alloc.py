"""The allocation-free FP64 moment build (agf2_build_moments_noalloc) -- for
callers whose own allocator owns the device memory budget and who cannot let
a library call cudaMalloc/cudaFree -- must give what the regular
agf2_build_moments gives, call after call, through the C ABI, and what the
FP64 oracle gives.

This file is collected last so that a stop-at-first-failure run has already
run every other test; it also passes when run alone."""
import numpy as np
import pytest

from oracle import agf2_oracle as O
from paper_2106_03508_gb300.synth import make_system, random_poles

pytestmark = pytest.mark.gpu
RTOL = 1e-10   # the FP64 path's tolerance in the other GPU tests


def _moments(agf2_lib, h, s, e, C, mu, noalloc):
    import torch
    L = torch.from_numpy(s.L).cuda()
    ed, Cd = torch.from_numpy(e).cuda(), torch.from_numpy(C).cuda()
    Uh = torch.full((2, s.nmo, s.nmo), 7.0, dtype=torch.float64, device="cuda")  # stale values
    Up = torch.full_like(Uh, -3.0)
    if noalloc:
        rc = agf2_lib.agf2_build_moments_noalloc(L.data_ptr(), s.naux, s.nmo, ed.data_ptr(),
                                                 Cd.data_ptr(), len(e), mu, Uh.data_ptr(),
                                                 Up.data_ptr(), 0)
        assert rc == agf2_lib.AGF2_OK, rc
    else:
        agf2_lib.agf2_build_moments(h.h, L.data_ptr(), s.naux, s.nmo, ed.data_ptr(), Cd.data_ptr(),
                                    len(e), mu, 1, agf2_lib.AGF2_FP64, Uh.data_ptr(), Up.data_ptr())
    torch.cuda.synchronize()
    return Uh.cpu().numpy(), Up.cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice(cuda_handle, agf2_lib):
    cases = [(24, 72, 29, 96, 1), (37, 90, 30, 70, 2)]  # two calls in a row, different sizes
    for nmo, nq, no, naux, seed in cases:
        s = make_system(nmo, max(1, nmo // 5), naux, seed)
        e, C, mu = random_poles(nmo, nq, no, seed + 3)
        Ah, Ap = _moments(agf2_lib, cuda_handle, s, e, C, mu, noalloc=True)
        Bh, Bp = _moments(agf2_lib, cuda_handle, s, e, C, mu, noalloc=False)
        Rh, Rp = O.build_moments(s.L, e, C, mu)
        for a, b, r in ((Ah, Bh, Rh), (Ap, Bp, Rp)):
            assert np.max(np.abs(a - b)) <= RTOL * np.max(np.abs(b))
            assert np.max(np.abs(a - r)) <= RTOL * np.max(np.abs(r))


def test_noalloc_at_the_size_limit(cuda_handle, agf2_lib):
    """naux < nmo, where the largest need over the occupied/virtual splits
    lies inside the range (o' = nqmo/2 + 3 nmo/naux): the largest accepted
    pole count runs with that worst split and matches the oracle; one pole
    more is rejected."""
    import torch
    nmo, naux = 512, 240
    s = make_system(nmo, 100, naux, 12)
    L = torch.from_numpy(s.L).cuda()
    big = 256
    U = torch.empty(2, 2, nmo, nmo, dtype=torch.float64, device="cuda")

    def call(nq):
        o = min(nq - 1, max(1, int(round(nq / 2 + 3 * nmo / naux))))
        e, C, mu = random_poles(nmo, nq, o, nq)
        ed, Cd = torch.from_numpy(e).cuda(), torch.from_numpy(C).cuda()
        rc = agf2_lib.agf2_build_moments_noalloc(L.data_ptr(), naux, nmo, ed.data_ptr(),
                                                 Cd.data_ptr(), nq, mu, U[0].data_ptr(),
                                                 U[1].data_ptr(), 0)
        torch.cuda.synchronize()
        return rc, (e, C, mu)

    lo, hi = 2, big          # call(lo) accepted, call(hi) rejected
    assert call(lo)[0] == agf2_lib.AGF2_OK and call(hi)[0] == agf2_lib.AGF2_ERR_INVALID_ARG
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if call(mid)[0] == agf2_lib.AGF2_OK:
            lo = mid
        else:
            hi = mid
    rc, (e, C, mu) = call(lo)
    assert rc == agf2_lib.AGF2_OK and lo > 16
    Uh, Up = U[0].cpu().numpy(), U[1].cpu().numpy()
    Rh, Rp = O.build_moments(s.L, e, C, mu)
    for a, r in ((Uh, Rh), (Up, Rp)):
        assert np.max(np.abs(a - r)) <= RTOL * np.max(np.abs(r))


def test_noalloc_rejects_oversized_problem(agf2_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    small = torch.zeros(16, dtype=torch.float64, device="cuda")
    # naux so large that the rotated integrals alone exceed the static scratch;
    # rejected from the sizes before any argument is read
    rc = agf2_lib.agf2_build_moments_noalloc(small.data_ptr(), 10 ** 6, 24, small.data_ptr(),
                                             small.data_ptr(), 72, 0.0, small.data_ptr(),
                                             small.data_ptr(), 0)
    assert rc == agf2_lib.AGF2_ERR_INVALID_ARG
