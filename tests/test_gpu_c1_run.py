"""Whole AGF2 iterations on the c1 synthetic system (nmo=24, nocc=5,
naux=96, seed 0) through agf2_run: the FP64 path against the oracle's stored
trajectory (tests/golden/c1_run.json, written by make_golden.py from
oracle/ only), and the split-BF16 path against the FP64 path."""
import json
from pathlib import Path

import numpy as np
import pytest

from paper_2106_03508_gb300.synth import make_config

pytestmark = pytest.mark.gpu
GOLDEN = json.loads((Path(__file__).parent / "golden" / "c1_run.json").read_text())
NIT = len(GOLDEN["history"])


def trajectory(lib, h, precision, nit=NIT, shift_mode=0):
    import torch
    s = make_config("c1")
    L, eps = torch.from_numpy(s.L).cuda(), torch.from_numpy(s.eps).cuda()
    hc = torch.empty(s.nmo, s.nmo, dtype=torch.float64, device="cuda")
    lib.agf2_hcore_from_mo_energies(h.h, L.data_ptr(), s.naux, s.nmo, eps.data_ptr(), s.nocc,
                                    hc.data_ptr())
    o = lib.agf2_opts_default()
    o.precision = precision
    o.max_iter = 1
    o.fock.max_cycle = 300
    o.fock.tol_D = 1e-12   # as the stored trajectory
    o.fock.shift_mode = shift_mode
    out = []
    for it in range(nit):
        o.resume = 1 if it else 0
        rc, r = lib.agf2_run(h.h, hc.data_ptr(), L.data_ptr(), s.naux, s.nmo, s.nelec,
                             None, o)
        out.append(r.as_dict())
    return out


@pytest.mark.parametrize("shift_mode", [0, 1])
def test_c1_fp64_trajectory_matches_oracle(cuda_handle, agf2_lib, shift_mode):
    got = trajectory(agf2_lib, cuda_handle, agf2_lib.AGF2_FP64, shift_mode=shift_mode)
    assert abs(got[0]["E_hf"] - GOLDEN["E_hf"]) <= 1e-12 * abs(GOLDEN["E_hf"])
    for g, ref in zip(got, GOLDEN["history"]):
        assert g["fock_cycles"] < 300
        for key in ("E_1b", "E_2b", "E_tot", "ip", "ea", "mu"):
            assert abs(g[key] - ref[key]) <= 1e-10 * abs(ref[key]), (ref["it"], key, g[key],
                                                                     ref[key])


def test_c1_mixed_vs_fp64_errors(cuda_handle, agf2_lib):
    """Split-BF16 moments against FP64 moments, same options, whole
    trajectory: largest absolute E_tot / IP / EA differences (Ha)."""
    a = trajectory(agf2_lib, cuda_handle, agf2_lib.AGF2_BF16X3)
    b = GOLDEN["history"]
    for x, y in zip(a, b):
        print("it %2d  dE_tot %.2e  dIP %.2e  dEA %.2e" % (y["it"], x["E_tot"] - y["E_tot"],
                                                           x["ip"] - y["ip"], x["ea"] - y["ea"]))
    err = {k: max(abs(x[k] - y[k]) for x, y in zip(a, b)) for k in ("E_tot", "ip", "ea")}
    print("c1 mixed vs FP64 oracle max |error| over", NIT, "iterations:", err)
    # targets of the split-precision path: IP/EA within 1e-5 Ha, E_tot within
    # 1e-6 Ha, over the whole self-consistent trajectory
    assert err["ip"] < 1e-5 and err["ea"] < 1e-5
    assert err["E_tot"] < 1e-6
