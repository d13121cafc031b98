"""A reached cap is a status, not a failure: agf2_fock_loop and agf2_run
return AGF2_ERR_NO_CONVERGENCE with their outputs filled."""
import numpy as np
import pytest

from oracle import agf2_oracle as O
from paper_2106_03508_gb300.synth import make_system

from test_gpu_fp64 import dev, empty, host

pytestmark = pytest.mark.gpu


def test_fock_loop_cycle_cap(cuda_handle, agf2_lib):
    s = make_system(16, 4, 40, 5)
    h = O.hcore_from_mo_energies(s.eps, s.L, s.nocc)
    rng = np.random.default_rng(77)
    nse = 32
    E = np.sort(np.concatenate([rng.uniform(-4, -1, 16), rng.uniform(1, 5, 16)]))
    v = 0.3 * rng.standard_normal((16, nse))
    D0 = O.hf_density(16, 4)
    hd, Ld, Ed, vd, Dd = dev(h), dev(s.L), dev(E), dev(v), dev(D0)
    F, eq, Cq = empty(16, 16), empty(16 + nse), empty(16, 16 + nse)
    opts = agf2_lib.agf2_fock_opts_default()
    opts.max_cycle = 1
    rc, info = agf2_lib.agf2_fock_loop(cuda_handle.h, hd.data_ptr(), Ld.data_ptr(), s.naux, 16,
                                       s.nelec, Ed.data_ptr(), vd.data_ptr(), nse, Dd.data_ptr(),
                                       F.data_ptr(), eq.data_ptr(), Cq.data_ptr(), opts)
    assert rc == agf2_lib.AGF2_ERR_NO_CONVERGENCE
    assert info.cycles == 1 and info.converged == 0
    e, D = host(eq), host(Dd)
    assert np.all(np.isfinite(e)) and np.all(np.diff(e) >= 0)
    assert np.array_equal(D, D.T) or np.max(np.abs(D - D.T)) < 1e-12
    assert 1 <= info.nocc_qmo < 16 + nse


def test_run_iteration_cap(cuda_handle, agf2_lib):
    s = make_system(16, 4, 48, 11, scale=0.08)
    hc = O.hcore_from_mo_energies(s.eps, s.L, s.nocc)
    L, hd, eps = dev(s.L), dev(hc), dev(s.eps)
    o = agf2_lib.agf2_opts_default()
    o.max_iter = 2
    o.conv_tol = 0.0  # |dE| < 0 never holds
    rc, out = agf2_lib.agf2_run(cuda_handle.h, hd.data_ptr(), L.data_ptr(), s.naux, s.nmo,
                                s.nelec, None, o)
    assert rc == agf2_lib.AGF2_ERR_NO_CONVERGENCE
    assert out.iterations == 2 and out.converged == 0
    assert np.isfinite(out.E_tot) and np.isfinite(out.ip) and np.isfinite(out.ea)

