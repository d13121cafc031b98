"""Thin ctypes binding of the AGF2 C ABI (include/agf2.h).

Argument marshalling only: every step runs in ``libagf2.so``.  Functions
keep the C names and take device pointers (ints) exactly like the C ABI;
the ``tensor`` helpers below accept torch CUDA float64 tensors and pass their
``data_ptr()``.  Importing this module raises if the library is missing --
there is no fallback.
"""
from __future__ import annotations

import ctypes as ct
from pathlib import Path

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libagf2.so"

AGF2_OK = 0
AGF2_ERR_INVALID_ARG = 1
AGF2_ERR_CUDA = 2
AGF2_ERR_OOM = 3
AGF2_ERR_NOT_PD = 4
AGF2_ERR_NO_CONVERGENCE = 5
AGF2_ERR_TIMEOUT = 6
AGF2_ERR_UNSUPPORTED = 7

AGF2_FP64 = 0
AGF2_BF16X3 = 1

EXPORTED = [
    "agf2_create", "agf2_destroy", "agf2_set_stream", "agf2_last_error",
    "agf2_hcore_from_mo_energies", "agf2_build_moments", "agf2_compress",
    "agf2_fock_opts_default", "agf2_fock_loop", "agf2_opts_default", "agf2_run",
    "agf2_get_state", "agf2_set_profiling", "agf2_kernel_stats", "agf2_launch_count",
    "agf2_build_moments_noalloc", "agf2_run_batched", "agf2_spectral_function",
    "agf2_compress_moments", "agf2_eigh_physical",
]


class agf2_fock_opts(ct.Structure):
    _fields_ = [("tol_D", ct.c_double), ("max_cycle", ct.c_int), ("shift_tol", ct.c_double),
                ("damping", ct.c_double), ("diis_start", ct.c_int), ("diis_space", ct.c_int),
                ("shift_mode", ct.c_int)]


class agf2_fock_info(ct.Structure):
    _fields_ = [("cycles", ct.c_int), ("converged", ct.c_int), ("nocc_qmo", ct.c_int),
                ("shift_evals", ct.c_int), ("nerr", ct.c_double), ("mu", ct.c_double)]


class agf2_opts(ct.Structure):
    _fields_ = [("max_iter", ct.c_int), ("conv_tol", ct.c_double), ("nmom", ct.c_int),
                ("precision", ct.c_int), ("mix", ct.c_double), ("resume", ct.c_int),
                ("fock", agf2_fock_opts)]


class agf2_system(ct.Structure):
    _fields_ = [("hcore", ct.c_void_p), ("L", ct.c_void_p), ("D0", ct.c_void_p),
                ("naux", ct.c_int), ("nmo", ct.c_int), ("nelec", ct.c_int)]


class agf2_result(ct.Structure):
    _fields_ = [("E_hf", ct.c_double), ("E_1b", ct.c_double), ("E_2b", ct.c_double),
                ("E_tot", ct.c_double), ("ip", ct.c_double), ("ea", ct.c_double),
                ("mu", ct.c_double), ("iterations", ct.c_int), ("converged", ct.c_int),
                ("nocc_qmo", ct.c_int), ("fock_cycles", ct.c_int), ("t_moments", ct.c_double),
                ("t_compress", ct.c_double), ("t_fock", ct.c_double), ("t_energy", ct.c_double),
                ("flops_moments", ct.c_double), ("fock_converged", ct.c_int),
                ("fock_cycles_total", ct.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def _load():
    if not LIB_PATH.exists():
        raise ImportError(f"{LIB_PATH} not built: run __graft_entry__.build() "
                          "(python -m paper_2106_03508_gb300.build)")
    lib = ct.CDLL(str(LIB_PATH))
    P, I, D, V = ct.c_void_p, ct.c_int, ct.c_double, None
    sig = {
        "agf2_create": (I, [ct.POINTER(P), I]),
        "agf2_destroy": (I, [P]),
        "agf2_set_stream": (I, [P, P]),
        "agf2_last_error": (ct.c_char_p, [P]),
        "agf2_hcore_from_mo_energies": (I, [P, P, I, I, P, I, P]),
        "agf2_build_moments": (I, [P, P, I, I, P, P, I, D, I, I, P, P]),
        "agf2_compress": (I, [P, P, I, P, P]),
        "agf2_compress_moments": (I, [P, P, I, I, P, P]),
        "agf2_eigh_physical": (I, [P, P, I, I, P, P]),
        "agf2_fock_opts_default": (V, [ct.POINTER(agf2_fock_opts)]),
        "agf2_fock_loop": (I, [P, P, P, I, I, I, P, P, I, P, P, P, P,
                               ct.POINTER(agf2_fock_opts), ct.POINTER(agf2_fock_info)]),
        "agf2_opts_default": (V, [ct.POINTER(agf2_opts)]),
        "agf2_run": (I, [P, P, P, I, I, I, P, ct.POINTER(agf2_opts), ct.POINTER(agf2_result)]),
        "agf2_get_state": (I, [P, P, P, P, ct.POINTER(ct.c_int)]),
        "agf2_set_profiling": (I, [P, I]),
        "agf2_kernel_stats": (I, [P, I, ct.POINTER(ct.c_longlong), ct.POINTER(D),
                                  ct.POINTER(D)]),
        "agf2_launch_count": (ct.c_longlong, []),
        "agf2_build_moments_noalloc": (I, [P, I, I, P, P, I, D, P, P, P]),
        "agf2_run_batched": (I, [P, I, ct.POINTER(agf2_system), ct.POINTER(agf2_opts), I,
                                 ct.POINTER(agf2_result), ct.POINTER(ct.c_int)]),
        "agf2_spectral_function": (I, [P, P, P, I, I, P, I, D, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


class AGF2Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"AGF2 status {code}: {msg}")
        self.code = code


def _check(h, rc, allow=()):
    if rc != AGF2_OK and rc not in allow:
        raise AGF2Error(rc, agf2_last_error(h))
    return rc


# ---- raw C-named entry points (pointers as ints) ----
def agf2_create(device: int = 0):
    h = ct.c_void_p()
    rc = _lib.agf2_create(ct.byref(h), device)
    if rc != AGF2_OK:
        raise AGF2Error(rc, "agf2_create failed")
    return h


def agf2_destroy(h):
    return _lib.agf2_destroy(h)


def agf2_set_stream(h, stream_ptr: int):
    return _check(h, _lib.agf2_set_stream(h, ct.c_void_p(stream_ptr)))


def agf2_last_error(h) -> str:
    r = _lib.agf2_last_error(h)
    return r.decode() if r else ""


def agf2_hcore_from_mo_energies(h, L, naux, nmo, eps, nocc, hcore):
    return _check(h, _lib.agf2_hcore_from_mo_energies(h, L, naux, nmo, eps, nocc, hcore))


def agf2_build_moments(h, L, naux, nmo, e, C, nqmo, mu, nmom, precision, U_hole, U_part):
    return _check(h, _lib.agf2_build_moments(h, L, naux, nmo, e, C, nqmo, float(mu), nmom,
                                             precision, U_hole, U_part))


def agf2_compress(h, U, nmo, E_aux, v_aux, allow=()):
    return _check(h, _lib.agf2_compress(h, U, nmo, E_aux, v_aux), allow)


def agf2_compress_moments(h, U, nmo, nmom, E_aux, v_aux, allow=()):
    return _check(h, _lib.agf2_compress_moments(h, U, nmo, nmom, E_aux, v_aux), allow)


def agf2_eigh_physical(h, A, n, nphys, w, V):
    return _check(h, _lib.agf2_eigh_physical(h, A, n, nphys, w, V))



def agf2_fock_opts_default() -> agf2_fock_opts:
    o = agf2_fock_opts()
    _lib.agf2_fock_opts_default(ct.byref(o))
    return o


def agf2_fock_loop(h, hcore, L, naux, nmo, nelec, E_se, v_se, nse, D, F, e_qmo, C_qmo,
                   opts=None, allow=(AGF2_ERR_NO_CONVERGENCE,)):
    info = agf2_fock_info()
    rc = _lib.agf2_fock_loop(h, hcore, L, naux, nmo, nelec, E_se, v_se, nse, D, F, e_qmo, C_qmo,
                             ct.byref(opts) if opts is not None else None, ct.byref(info))
    _check(h, rc, allow)
    return rc, info


def agf2_opts_default() -> agf2_opts:
    o = agf2_opts()
    _lib.agf2_opts_default(ct.byref(o))
    return o


def agf2_run(h, hcore, L, naux, nmo, nelec, D0=None, opts=None,
             allow=(AGF2_ERR_NO_CONVERGENCE,)):
    out = agf2_result()
    rc = _lib.agf2_run(h, hcore, L, naux, nmo, nelec, D0,
                       ct.byref(opts) if opts is not None else None, ct.byref(out))
    _check(h, rc, allow)
    return rc, out


def agf2_run_batched(h, systems, opts=None, nworkers=0, allow=(AGF2_ERR_NO_CONVERGENCE,)):
    """systems: list of (hcore_ptr, L_ptr, D0_ptr or None, naux, nmo, nelec)."""
    n = len(systems)
    arr = (agf2_system * max(n, 1))(*[agf2_system(*sy) for sy in systems])
    out = (agf2_result * max(n, 1))()
    st = (ct.c_int * max(n, 1))()
    rc = _lib.agf2_run_batched(h, n, arr, ct.byref(opts) if opts is not None else None,
                               nworkers, out, st)
    _check(h, rc, allow)
    return rc, [out[i] for i in range(n)], [st[i] for i in range(n)]


def agf2_spectral_function(h, e, C, nmo, nqmo, omega, nomega, eta, A_total, A_orb=None):
    return _check(h, _lib.agf2_spectral_function(h, e, C, nmo, nqmo, omega, nomega, float(eta),
                                                 A_total, A_orb))


def agf2_get_state(h, e=None, C=None, D=None):
    nq = ct.c_int()
    _check(h, _lib.agf2_get_state(h, e, C, D, ct.byref(nq)))
    return nq.value


def agf2_set_profiling(h, enable: bool):
    return _check(h, _lib.agf2_set_profiling(h, 1 if enable else 0))


def agf2_kernel_stats(h, kind: int):
    n, ms, fl = ct.c_longlong(), ct.c_double(), ct.c_double()
    _check(h, _lib.agf2_kernel_stats(h, kind, ct.byref(n), ct.byref(ms), ct.byref(fl)))
    return n.value, ms.value, fl.value


def agf2_launch_count() -> int:
    return int(_lib.agf2_launch_count())


def agf2_build_moments_noalloc(L, naux, nmo, e, C, nqmo, mu, U_hole, U_part, stream_ptr=0):
    """FP64 moments without any device allocation (see include/agf2.h); returns the status."""
    return int(_lib.agf2_build_moments_noalloc(L, naux, nmo, e, C, nqmo, float(mu), U_hole,
                                               U_part, ct.c_void_p(stream_ptr)))


# ---- torch-tensor conveniences (marshalling only) ----
def ptr(t) -> int:
    """Device pointer of a contiguous CUDA float64/int tensor."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


class Handle:
    """RAII wrapper of an agf2_handle bound to a device and (optionally) the
    current torch stream."""

    def __init__(self, device: int = 0, stream_ptr: int | None = None):
        self.h = agf2_create(device)
        if stream_ptr is not None:
            agf2_set_stream(self.h, stream_ptr)

    def close(self):
        if self.h is not None:
            agf2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
