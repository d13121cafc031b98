"""Spectral function A(w) = -(1/pi) Im Tr G(w + i eta) through the C ABI vs the oracle."""
import numpy as np
import pytest

from oracle import agf2_oracle as O
from paper_2106_03508_gb300.synth import random_poles

from test_gpu_fp64 import dev, empty, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nmo,nq,nw", [(24, 72, 301), (65, 195, 1000), (3, 5, 1)])
def test_spectral_function_vs_oracle(cuda_handle, agf2_lib, nmo, nq, nw):
    e, C, _ = random_poles(nmo, nq, nq // 3, 17)
    w = np.linspace(-4.0, 4.0, nw)
    eta = 0.2 / 27.211386  # 0.2 eV in Ha
    A, Ao = O.spectral_function(e, C, w, eta)
    At, Aod = empty(nw), empty(nmo, nw)
    ed, Cd, wd = dev(e), dev(C), dev(w)
    agf2_lib.agf2_spectral_function(cuda_handle.h, ed.data_ptr(), Cd.data_ptr(), nmo, nq,
                                    wd.data_ptr(), nw, eta, At.data_ptr(), Aod.data_ptr())
    assert np.max(np.abs(host(At) - A)) <= 1e-12 * np.max(np.abs(A))
    assert np.max(np.abs(host(Aod) - Ao)) <= 1e-12 * np.max(np.abs(Ao))
