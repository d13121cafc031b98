"""One timed moment build (Eqs. mp2_zeroth_moment / mp2_first_moment) on a
synthetic pole set of a chosen shape, through the C-ABI.

For profiling and for sizes where a whole AGF2 iteration is out of reach:

    python -m paper_2106_03508_gb300.moment_case --nmo 256 --naux 1024 \\
        --npoles 512 --nocc-poles 200 --repeat 1
    python -m paper_2106_03508_gb300.moment_case --config c5 --npoles 3000 \\
        --nocc-poles 1200

The DF factors come from ``synth.make_system`` (or a named workload), the poles
from ``synth.random_poles`` (the steady-state shape: a dense pole-coupling
matrix C, ``npoles`` poles of which ``nocc_poles`` are occupied), or with
``--hf-poles`` the first iteration's poles (e = orbital energies, C = I).
Prints one JSON line: seconds per build, algorithmic TFLOP/s
F_alg = N o v (o + v) (2 n_Q + 2 (nmom + 1) N), the tcgen05 kernels' CUDA-event
times and rates, and the device memory in use.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import agf2 as A
from .synth import make_config, make_system, random_poles


def main(argv=None) -> dict:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--config", default=None, help="named workload (c1/c2/c3/c5) for L")
    ap.add_argument("--nmo", type=int, default=256)
    ap.add_argument("--nocc", type=int, default=51, help="occupied orbitals of the system")
    ap.add_argument("--naux", type=int, default=1024)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--npoles", type=int, default=512)
    ap.add_argument("--nocc-poles", type=int, default=200)
    ap.add_argument("--pole-seed", type=int, default=3)
    ap.add_argument("--hf-poles", action="store_true",
                    help="poles of the first iteration: e = orbital energies, C = I")
    ap.add_argument("--nmom", type=int, default=1)
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp64"])
    ap.add_argument("--repeat", type=int, default=1)
    a = ap.parse_args(argv)
    if not torch.cuda.is_available():
        raise RuntimeError("moment_case needs a CUDA device")
    t0 = time.perf_counter()
    s = make_config(a.config) if a.config else make_system(a.nmo, a.nocc, a.naux, a.seed)
    t_gen = time.perf_counter() - t0
    N, naux = s.nmo, s.naux
    if a.hf_poles:
        e, C = s.eps, np.eye(N)
        mu = 0.5 * (s.eps[s.nocc - 1] + s.eps[s.nocc])
    else:
        e, C, mu = random_poles(N, a.npoles, a.nocc_poles, a.pole_seed)
    nq = e.shape[0]
    o = int(np.sum(e < mu))
    v = nq - o
    prec = A.AGF2_BF16X3 if a.precision == "bf16x3" else A.AGF2_FP64
    h = A.Handle(0)
    try:
        L = torch.from_numpy(s.L).cuda()
        ed = torch.from_numpy(np.ascontiguousarray(e)).cuda()
        Cd = torch.from_numpy(np.ascontiguousarray(C)).cuda()
        nm = a.nmom + 1
        Uh = torch.empty(nm, N, N, dtype=torch.float64, device="cuda")
        Up = torch.empty_like(Uh)
        A.agf2_set_profiling(h.h, True)
        times = []
        for _ in range(a.repeat):
            torch.cuda.synchronize()
            t = time.perf_counter()
            A.agf2_build_moments(h.h, L.data_ptr(), naux, N, ed.data_ptr(), Cd.data_ptr(), nq,
                                 mu, a.nmom, prec, Uh.data_ptr(), Up.data_ptr())
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t)
        st = {k: A.agf2_kernel_stats(h.h, k) for k in (0, 1)}
        A.agf2_set_profiling(h.h, False)
        free, total = torch.cuda.mem_get_info()
        F = N * o * v * (o + v) * (2.0 * naux + 2.0 * nm * N)
        sec = min(times)
        out = {
            "workload": a.config or f"nmo={N} nocc={s.nocc} naux={naux} seed={s.seed}",
            "nmo": N, "naux": naux, "o": o, "v": v, "nmom": a.nmom,
            "poles": "hf" if a.hf_poles else f"random_poles(seed={a.pole_seed})",
            "precision": a.precision, "repeat": a.repeat,
            "seconds_per_build": sec, "seconds_all": times,
            "tflops_algorithmic": F / sec / 1e12,
            "pair_gemm": {"launches": st[0][0], "ms": st[0][1],
                          "tflops": st[0][2] / st[0][1] / 1e9 if st[0][1] else None},
            "moment_gemm": {"launches": st[1][0], "ms": st[1][1],
                            "tflops": st[1][2] / st[1][1] / 1e9 if st[1][1] else None},
            "device_used_gb": (total - free) / 1e9,
            "torch_peak_gb": torch.cuda.max_memory_allocated() / 1e9,
            "generate_s": t_gen,
            "U_hole0_trace": float(torch.diagonal(Uh[0]).sum()),
        }
        print(json.dumps(out), flush=True)
        return out
    finally:
        h.close()


if __name__ == "__main__":
    main()
