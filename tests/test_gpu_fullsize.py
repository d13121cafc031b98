"""Full-size parity at the bench's workload shape (c2: nmo=200, naux=800,
steady-state pole set of 600 poles, 240 occupied), through the same
agf2_build_moments launch configuration the bench times: sampled moment
elements from the oracle's one-element evaluation."""
import numpy as np
import pytest

from oracle import agf2_oracle as O
from paper_2106_03508_gb300.synth import make_config, random_poles

from test_gpu_fp64 import gpu_moments

pytestmark = pytest.mark.gpu
PQ = [(0, 0), (17, 17), (5, 123), (199, 64)]


@pytest.fixture(scope="module")
def c2_case():
    s = make_config("c2")
    e, C, mu = random_poles(s.nmo, 600, 240, 5)
    ref_h, ref_p = O.moment_elements(s.L, e, C, mu, PQ)
    return s, e, C, mu, ref_h, ref_p


def _check(U_h, U_p, ref_h, ref_p, rtol):
    for U, ref in ((U_h, ref_h), (U_p, ref_p)):
        for n in range(2):
            scale = np.max(np.abs(U[n]))
            for t, (p, q) in enumerate(PQ):
                assert abs(U[n, p, q] - ref[t, n]) <= rtol * scale, (n, p, q, U[n, p, q], ref[t, n])


def test_c2_mixed_sampled_elements(cuda_handle, agf2_lib, c2_case):
    s, e, C, mu, ref_h, ref_p = c2_case
    Uh, Up = gpu_moments(agf2_lib, cuda_handle, s.L, e, C, mu, precision=agf2_lib.AGF2_BF16X3)
    _check(Uh, Up, ref_h, ref_p, 1e-7)


def test_c2_fp64_sampled_elements(cuda_handle, agf2_lib, c2_case):
    s, e, C, mu, ref_h, ref_p = c2_case
    Uh, Up = gpu_moments(agf2_lib, cuda_handle, s.L, e, C, mu, precision=agf2_lib.AGF2_FP64)
    _check(Uh, Up, ref_h, ref_p, 1e-10)
