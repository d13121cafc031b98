"""Split-BF16 (tcgen05) moment build vs the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import agf2_oracle as O
from paper_2106_03508_gb300.synth import make_system, random_poles

from test_gpu_fp64 import gpu_moments, rel

pytestmark = pytest.mark.gpu
# three-limb BF16 products with FP32 accumulation: ~2^-24 per product
MIXED_RTOL = 2e-6


@pytest.mark.parametrize("nmo,nq,no,naux,seed", [
    (24, 72, 29, 96, 1),      # c1-shaped, iteration >= 2
    (130, 260, 97, 200, 2),   # two p-tiles (ragged), inner counts past 128
    (9, 20, 1, 5, 3),         # one occupied pole, naux < 64
    (9, 20, 19, 1, 4),        # one virtual pole, one auxiliary function
    (70, 150, 61, 150, 5),
])
def test_moments_mixed_vs_oracle(cuda_handle, agf2_lib, nmo, nq, no, naux, seed):
    s = make_system(nmo, max(1, nmo // 5), naux, seed)
    e, C, mu = random_poles(nmo, nq, no, seed + 7)
    Uh, Up = gpu_moments(agf2_lib, cuda_handle, s.L, e, C, mu, precision=agf2_lib.AGF2_BF16X3)
    Rh, Rp = O.build_moments(s.L, e, C, mu)
    for n in range(2):
        assert rel(Uh[n], Rh[n]) < MIXED_RTOL, (n, rel(Uh[n], Rh[n]))
        assert rel(Up[n], Rp[n]) < MIXED_RTOL, (n, rel(Up[n], Rp[n]))


def test_moments_mixed_hf_reference(cuda_handle, agf2_lib):
    s = make_system(40, 8, 160, 9)
    mu = 0.5 * (s.eps[7] + s.eps[8])
    Uh, Up = gpu_moments(agf2_lib, cuda_handle, s.L, s.eps, np.eye(40), mu,
                         precision=agf2_lib.AGF2_BF16X3)
    Rh, Rp = O.build_moments(s.L, s.eps, np.eye(40), mu)
    assert rel(Uh, Rh) < MIXED_RTOL and rel(Up, Rp) < MIXED_RTOL


def test_moments_mixed_exact_integer_sums_flat_rows(cuda_handle, agf2_lib):
    """DF factors of constant magnitude (0.3 times random signs, no decay over
    Q) at naux = 2048 and the Hartree-Fock poles (C = I): the rotated rows are
    flat, so a row's integer limbs are all near the limb range, and the pair
    GEMM's h0 h0' sum of an orbital with itself reaches ~5e7 > 2^24 -- inexact
    in FP32 unless the row's unit is coarsened (the exactness certificate) or
    the sum is split.  The moments must still meet the split-precision
    tolerance."""
    nmo, nocc, naux = 24, 6, 2048
    s = make_system(nmo, nocc, naux, 21)
    L = 0.3 * np.sign(s.L)
    L = np.ascontiguousarray(0.5 * (L + L.transpose(0, 2, 1)))
    mu = 0.5 * (s.eps[nocc - 1] + s.eps[nocc])
    C = np.eye(nmo)
    Uh, Up = gpu_moments(agf2_lib, cuda_handle, L, s.eps, C, mu, precision=agf2_lib.AGF2_BF16X3)
    Rh, Rp = O.build_moments(L, s.eps, C, mu)
    for n in range(2):
        assert rel(Uh[n], Rh[n]) < MIXED_RTOL, (n, rel(Uh[n], Rh[n]))
        assert rel(Up[n], Rp[n]) < MIXED_RTOL, (n, rel(Up[n], Rp[n]))
