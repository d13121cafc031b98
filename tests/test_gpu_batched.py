"""agf2_run_batched: uneven systems solved concurrently (worker threads with
their own streams) give each system's agf2_run / oracle result."""
import numpy as np
import pytest

from oracle import agf2_oracle as O
from paper_2106_03508_gb300.synth import make_system

pytestmark = pytest.mark.gpu


def test_batched_uneven_systems_match_oracle(cuda_handle, agf2_lib):
    import torch
    specs = [(10, 2, 24, 201), (13, 3, 30, 202), (8, 2, 20, 203), (12, 3, 28, 204),
             (9, 2, 18, 205)]
    systems, keep, refs = [], [], []
    for nmo, nocc, naux, seed in specs:
        s = make_system(nmo, nocc, naux, seed)
        s.L *= 0.5
        h = O.hcore_from_mo_energies(s.eps, s.L, s.nocc)
        refs.append(O.run(h, s.L, s.nelec, s.eps, max_iter=30, fock_max_cycle=300))
        L, hc, eps = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (s.L, h, s.eps))
        keep += [L, hc, eps]
        systems.append((hc.data_ptr(), L.data_ptr(), None, naux, nmo, s.nelec))
    o = agf2_lib.agf2_opts_default()
    o.max_iter = 30
    o.fock.max_cycle = 300
    rc, outs, st = agf2_lib.agf2_run_batched(cuda_handle.h, systems, o, nworkers=3)
    for out, ref, status in zip(outs, refs, st):
        assert status in (agf2_lib.AGF2_OK, agf2_lib.AGF2_ERR_NO_CONVERGENCE)
        assert out.iterations == ref.iterations
        for a, b in ((out.E_tot, ref.E_tot), (out.ip, ref.ip), (out.ea, ref.ea)):
            assert abs(a - b) <= 1e-9 * max(1.0, abs(b))


def test_batched_empty_and_bad_args(cuda_handle, agf2_lib):
    rc, outs, st = agf2_lib.agf2_run_batched(cuda_handle.h, [])
    assert rc == agf2_lib.AGF2_OK and outs == []
