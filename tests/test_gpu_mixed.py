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


def test_moments_mixed_underflowing_row_units(cuda_handle, agf2_lib):
    """naux = 4000 with the generator's exp(-Q/24) decay: rows of the DF
    factors past Q ~ 2300 lie below 2^-142, so their FP32 slicing units
    underflow to zero in the rotation; those rows must contribute nothing
    (their true contribution is below 2^-140 relative) rather than enter the
    exponent arithmetic of the rotation's epilogue."""
    s = make_system(40, 8, 4000, 12)
    e, C, mu = random_poles(40, 120, 48, 19)
    Rh, Rp = O.build_moments(s.L, e, C, mu)
    for scale in (1.0, 1.0 / 16.0):
        Uh, Up = gpu_moments(agf2_lib, cuda_handle, s.L, e, C * scale, mu,
                             precision=agf2_lib.AGF2_BF16X3)
        for n in range(2):
            # (pi|ja) carries three pole couplings, so U scales as the sixth power
            assert rel(Uh[n] / scale ** 6, Rh[n]) < 1e-7, (scale, n, rel(Uh[n] / scale ** 6, Rh[n]))
            assert rel(Up[n] / scale ** 6, Rp[n]) < 1e-7, (scale, n, rel(Up[n] / scale ** 6, Rp[n]))


def test_moments_mixed_power_of_two_scaling(cuda_handle, agf2_lib):
    """Every unit of the split path is a power of two, so scaling the pole
    couplings by 2^-4 scales U (sixth order in the couplings: three per
    (pi|ja)) by exactly 2^-24 with unchanged limbs: the two builds agree to
    the FP64 atomics' summation-order rounding."""
    s = make_system(70, 14, 300, 21)
    e, C, mu = random_poles(70, 210, 83, 23)
    U1 = gpu_moments(agf2_lib, cuda_handle, s.L, e, C, mu, precision=agf2_lib.AGF2_BF16X3)
    U2 = gpu_moments(agf2_lib, cuda_handle, s.L, e, C / 16.0, mu, precision=agf2_lib.AGF2_BF16X3)
    for a, b in zip(U1, U2):
        assert np.max(np.abs(b * 2.0 ** 24 - a)) <= 1e-12 * np.max(np.abs(a))
