"""Seeded synthetic inputs for AGF2 (closed-shell, density-fitted).

This module only draws random numbers; it holds none of the method's arithmetic
(no Fock build, no moments).  Both the CUDA path and the FP64 oracle start from
what it returns, so each side derives everything else (the one-body
Hamiltonian, the moments, ...) on its own.

Recipe (the synthetic stand-in for the paper's molecules, Sec. "parallel
speedup" / artemisinin: N orbitals, nocc doubly occupied, n_Q ~ 4N auxiliary
DF functions):

* ``rng = numpy.random.default_rng(seed)``; draws in this order:
  occupied energies ``U[-1.5, -0.3]`` (sorted), virtual energies ``U[0.1, 3.0]``
  (sorted), then ``G ~ N(0, 1)`` of shape ``[naux, nmo, nmo]``.
* ``L[Q] = 0.5 (G[Q] + G[Q]^T) * scale * exp(-Q / decay_len)`` with
  ``scale = 0.3`` and ``decay_len = 24`` for every size, so that
  ``(pq|rs) = sum_Q L[Q,p,q] L[Q,r,s]`` is a valid (positive semidefinite)
  density-fitted ERI tensor.
* Batched systems: system ``s`` uses ``seed = base + s``; its ``nmo`` is the
  first draw of that generator, uniform on ``[nmo_lo, nmo_hi]``, with
  ``nocc = nmo // 5`` and ``naux = 4 nmo``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Named workloads (sizes, seed).
CONFIGS = {
    "c1": dict(nmo=24, nocc=5, naux=96, seed=0),
    "c2": dict(nmo=200, nocc=40, naux=800, seed=1),
    "c3": dict(nmo=500, nocc=100, naux=2000, seed=2),
    "c5": dict(nmo=1000, nocc=200, naux=4000, seed=3),
}


@dataclass
class System:
    nmo: int
    nocc: int
    naux: int
    seed: int
    eps: np.ndarray  # [nmo] mean-field orbital energies, occupied first
    L: np.ndarray    # [naux, nmo, nmo] symmetric DF factors, float64, C order

    @property
    def nelec(self) -> int:
        return 2 * self.nocc


def make_system(nmo: int, nocc: int, naux: int, seed: int,
                scale: float = 0.3, decay_len: float = 24.0) -> System:
    if not (0 < nocc < nmo) or naux < 1:
        raise ValueError("need 0 < nocc < nmo and naux >= 1")
    rng = np.random.default_rng(seed)
    e_occ = np.sort(rng.uniform(-1.5, -0.3, size=nocc))
    e_vir = np.sort(rng.uniform(0.1, 3.0, size=nmo - nocc))
    G = rng.standard_normal(size=(naux, nmo, nmo))
    L = 0.5 * (G + G.transpose(0, 2, 1))
    L *= (scale * np.exp(-np.arange(naux, dtype=np.float64) / decay_len))[:, None, None]
    return System(nmo, nocc, naux, seed, np.concatenate([e_occ, e_vir]),
                  np.ascontiguousarray(L))


def make_config(name: str, **kw) -> System:
    return make_system(**CONFIGS[name], **kw)


def make_batched(nsys: int = 64, base_seed: int = 100, nmo_lo: int = 30,
                 nmo_hi: int = 150) -> list[System]:
    out = []
    for s in range(nsys):
        seed = base_seed + s
        nmo = int(np.random.default_rng(seed).integers(nmo_lo, nmo_hi + 1))
        out.append(make_system(nmo, nmo // 5, 4 * nmo, seed))
    return out


def random_poles(nmo: int, nqmo: int, nocc_poles: int, seed: int):
    """Random pole energies/couplings for unit tests of the moment build.

    Returns (e[nqmo] ascending, C[nmo, nqmo], mu) with exactly ``nocc_poles``
    energies below ``mu``.  C is a generic dense matrix (not unitary), the
    shape of the physical block of the extended-Hamiltonian eigenvectors.
    """
    rng = np.random.default_rng(seed)
    e_o = np.sort(rng.uniform(-2.0, -0.2, size=nocc_poles))
    e_v = np.sort(rng.uniform(0.2, 3.0, size=nqmo - nocc_poles))
    C = rng.standard_normal(size=(nmo, nqmo)) / np.sqrt(nqmo / nmo)
    return np.concatenate([e_o, e_v]), C, 0.0
