"""Write tests/golden/c1_run.json: the FP64 oracle's AGF2 trajectory on the
c1 synthetic system (nmo=24, nocc=5, naux=96, seed 0), 12 outer iterations
from the Hartree-Fock reference, default options except a 300-cycle Fock
cap and a Fock-loop density tolerance of 1e-12 (every Fock loop then
converges, and tightly enough that energies can be compared at a relative
1e-10).  Calls only
oracle/ (and the seeded input generator).

    python tests/golden/make_golden.py
"""
import json
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import agf2_oracle as O  # noqa: E402
from paper_2106_03508_gb300.synth import make_config  # noqa: E402


def main():
    s = make_config("c1")
    h = O.hcore_from_mo_energies(s.eps, s.L, s.nocc)
    r = O.run(h, s.L, s.nelec, s.eps, max_iter=12, fock_max_cycle=300, fock_tol=1e-12)
    out = {
        "source": "oracle/agf2_oracle.py run(), defaults, max_iter=12, fock_max_cycle=300, fock_tol=1e-12",
        "system": {"nmo": s.nmo, "nocc": s.nocc, "naux": s.naux, "seed": s.seed},
        "E_hf": r.E_hf,
        "E_mp2": O.mp2_energy(s.L, s.eps, s.nocc),
        "history": [dict(it=x.it, E_1b=float(x.E_1b), E_2b=float(x.E_2b), E_tot=float(x.E_tot),
                         ip=float(x.ip), ea=float(x.ea), mu=float(x.mu),
                         fock_cycles=int(x.fock_cycles)) for x in r.history],
    }
    (Path(__file__).parent / "c1_run.json").write_text(json.dumps(out, indent=1) + "\n")


if __name__ == "__main__":
    main()
