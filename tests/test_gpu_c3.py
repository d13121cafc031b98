"""Parity at the nmo = 500, naux = 2000 workload (the mixed-vs-FP64
accuracy configuration: synthetic system seed 2), through the same
agf2_build_moments launch configuration the iteration uses: sampled moment
elements from the oracle's one-element evaluation.

Iteration 1 starts from the Hartree-Fock poles (e = eps, C = I; 100 occupied,
400 virtual), where both precisions are affordable; from iteration 2 the
Green's function has 3 nmo poles, and a pole set of that shape (random
couplings, 1200 poles, 480 occupied) runs the split-BF16 path -- the FP64 path
would take ~20 GPU-minutes there (2.4e15 algorithmic flops at ~1.2 TFLOP/s)."""
import numpy as np
import pytest

from oracle import agf2_oracle as O
from paper_2106_03508_gb300.synth import make_config, random_poles

from test_gpu_fp64 import gpu_moments

pytestmark = pytest.mark.gpu
PQ = [(0, 0), (17, 17), (5, 123), (499, 64), (250, 251), (99, 100)]


@pytest.fixture(scope="module")
def c3():
    return make_config("c3")


def _check(U_h, U_p, ref_h, ref_p, rtol):
    for U, ref in ((U_h, ref_h), (U_p, ref_p)):
        for n in range(2):
            scale = np.max(np.abs(U[n]))
            for t, (p, q) in enumerate(PQ):
                assert abs(U[n, p, q] - ref[t, n]) <= rtol * scale, (n, p, q, U[n, p, q],
                                                                     ref[t, n])


@pytest.fixture(scope="module")
def hf_case(c3):
    s = c3
    mu = 0.5 * (s.eps[s.nocc - 1] + s.eps[s.nocc])
    C = np.eye(s.nmo)
    ref_h, ref_p = O.moment_elements(s.L, s.eps, C, mu, PQ)
    return s, C, mu, ref_h, ref_p


@pytest.mark.parametrize("prec,rtol", [(0, 1e-10), (1, 1e-7)])
def test_c3_iteration1_sampled_elements(cuda_handle, agf2_lib, hf_case, prec, rtol):
    s, C, mu, ref_h, ref_p = hf_case
    Uh, Up = gpu_moments(agf2_lib, cuda_handle, s.L, s.eps, C, mu, precision=prec)
    _check(Uh, Up, ref_h, ref_p, rtol)


def test_c3_steady_state_shape_mixed_sampled_elements(cuda_handle, agf2_lib, c3):
    s = c3
    e, C, mu = random_poles(s.nmo, 1200, 480, 13)
    ref_h, ref_p = O.moment_elements(s.L, e, C, mu, PQ)
    Uh, Up = gpu_moments(agf2_lib, cuda_handle, s.L, e, C, mu, precision=agf2_lib.AGF2_BF16X3)
    _check(Uh, Up, ref_h, ref_p, 1e-7)
