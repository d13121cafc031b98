"""The Fock loop's symmetric eigensolver (agf2_eigh_physical) against
numpy's LAPACK eigh: eigenvalues, orthogonality and residual of the full
eigenvectors, and the physical-row invariants the Fock loop uses (pole
weights and spectral projectors), on random, extended-Hamiltonian-shaped,
degenerate and structured matrices."""
import numpy as np
import pytest

from test_gpu_fp64 import dev, empty, host

pytestmark = pytest.mark.gpu


def eigh_gpu(lib, h, A, nphys=None):
    n = A.shape[0]
    nphys = n if nphys is None else nphys
    Ad = dev(np.ascontiguousarray(A))
    w, V = empty(n), empty(n, n)
    lib.agf2_eigh_physical(h.h, Ad.data_ptr(), n, nphys, w.data_ptr(), V.data_ptr())
    a_after = host(Ad)
    assert np.array_equal(a_after, A)  # input untouched
    return host(w), host(V).T[:nphys, :]   # V[p][x], physical rows


def extended(N, nse, seed, dup=True):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((N, N)) * 3.0
    F = 0.5 * (F + F.T)
    v = rng.standard_normal((N, nse)) * 0.4
    E = np.sort(rng.uniform(-25, 25, nse))
    if dup and nse > 20:
        E[5] = E[4] + 1e-13       # near-degenerate auxiliaries
        E[10:14] = E[10]          # exactly degenerate ones
    return np.block([[F, v], [v.T, np.diag(E)]])


def check_full(A, w, V):
    n = A.shape[0]
    wr = np.linalg.eigvalsh(A)
    scale = max(np.abs(wr).max(), 1e-300)
    assert np.abs(w - wr).max() <= 1e-12 * scale * max(1.0, np.sqrt(n) / 4)
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12 * max(1.0, np.sqrt(n) / 4)
    assert np.abs(A @ V - V * w).max() <= 1e-12 * scale * max(1.0, np.sqrt(n) / 4)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (17, 3), (64, 4), (200, 5), (601, 6)])
def test_random_symmetric(cuda_handle, agf2_lib, n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    A = 0.5 * (B + B.T)
    w, V = eigh_gpu(agf2_lib, cuda_handle, A)
    check_full(A, w, V)


@pytest.mark.parametrize("A_kind", ["identity", "two_level", "diagonal", "block_diagonal",
                                    "zero", "rank_one"])
def test_structured(cuda_handle, agf2_lib, A_kind):
    rng = np.random.default_rng(11)
    n = 48
    if A_kind == "identity":
        A = np.eye(n)
    elif A_kind == "two_level":
        A = np.diag(np.repeat([1.0, 2.0], n // 2))
    elif A_kind == "diagonal":
        A = np.diag(rng.uniform(-3, 3, n))
    elif A_kind == "block_diagonal":
        B1 = rng.standard_normal((20, 20)); B2 = rng.standard_normal((n - 20, n - 20))
        A = np.zeros((n, n)); A[:20, :20] = B1 + B1.T; A[20:, 20:] = B2 + B2.T
    elif A_kind == "zero":
        A = np.zeros((n, n))
    else:
        u = rng.standard_normal(n)
        A = np.outer(u, u)
    w, V = eigh_gpu(agf2_lib, cuda_handle, A)
    wr = np.linalg.eigvalsh(A)
    scale = max(np.abs(wr).max(), 1.0)
    assert np.abs(w - wr).max() <= 1e-12 * scale
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
    assert np.abs(A @ V - V * w).max() <= 1e-12 * scale


@pytest.mark.parametrize("N,mult,seed", [(24, 2, 7), (60, 2, 8), (200, 2, 9), (40, 4, 10)])
def test_extended_physical_rows(cuda_handle, agf2_lib, N, mult, seed):
    """nphys = N: eigenvalues, pole weights sum_p V_px^2 away from exact
    degeneracy, and the physical blocks of A^m = V w^m V^T (m = 0, 1, 2)
    and of the spectral projectors below every clear gap."""
    A = extended(N, mult * N, seed)
    n = A.shape[0]
    w, C = eigh_gpu(agf2_lib, cuda_handle, A, nphys=N)
    wr, Vr = np.linalg.eigh(A)
    Cr = Vr[:N, :]
    scale = np.abs(wr).max()
    assert np.abs(w - wr).max() <= 1e-12 * scale
    Am = np.eye(n)
    for m in range(3):
        got = (C * w ** m) @ C.T
        assert np.abs(got - Am[:N, :N]).max() <= 1e-11 * max(1.0, scale ** m), m
        Am = Am @ A
    gaps = np.where(np.diff(wr) > 1e-6 * scale)[0] + 1
    for k in gaps[:: max(1, len(gaps) // 25)]:
        P = C[:, :k] @ C[:, :k].T
        Pr = Cr[:, :k] @ Cr[:, :k].T
        assert np.abs(P - Pr).max() <= 1e-10, k
    iso = np.ones(n, dtype=bool)
    iso[1:] &= np.diff(wr) > 1e-6 * scale
    iso[:-1] &= np.diff(wr) > 1e-6 * scale
    wt, wtr = (C * C).sum(0), (Cr * Cr).sum(0)
    assert np.abs(wt[iso] - wtr[iso]).max() <= 1e-10


def test_c2_sized_extended(cuda_handle, agf2_lib):
    """The Fock loop's size at nmo = 200 (n = 600), twice in a row (the
    workspace is reused)."""
    A = extended(200, 400, 21, dup=False)
    for _ in range(2):
        w, C = eigh_gpu(agf2_lib, cuda_handle, A, nphys=200)
        wr, Vr = np.linalg.eigh(A)
        assert np.abs(w - wr).max() <= 1e-12 * np.abs(wr).max()
        k = 300
        assert np.abs(C[:, :k] @ C[:, :k].T - Vr[:200, :k] @ Vr[:200, :k].T).max() <= 1e-10


def test_rejects_bad_sizes(cuda_handle, agf2_lib):
    A = np.eye(4)
    with pytest.raises(agf2_lib.AGF2Error) as ei:
        eigh_gpu(agf2_lib, cuda_handle, A, nphys=5)
    assert ei.value.code == agf2_lib.AGF2_ERR_INVALID_ARG


def test_extended_global_rows(cuda_handle, agf2_lib):
    """n = 2000: too many rows per CTA for shared memory, so the
    tridiagonalisation keeps them in global memory (the variant of
    nmom = 3 at nmo = 500 and of nmo >= 1000)."""
    A = extended(400, 1600, 33, dup=False)
    w, C = eigh_gpu(agf2_lib, cuda_handle, A, nphys=400)
    wr = np.linalg.eigvalsh(A)
    scale = np.abs(wr).max()
    assert np.abs(w - wr).max() <= 1e-11 * scale
    assert np.abs(C @ C.T - np.eye(400)).max() <= 1e-10
    assert np.abs((C * w) @ C.T - A[:400, :400]).max() <= 1e-10 * scale


def test_extended_c5_shape_one_reflector_back_transformation(cuda_handle, agf2_lib):
    """n = 3000 with 1000 physical rows (nmo = 1000, AGF2(1,0)): the
    back-transformation's rows plus a block of eight reflectors exceed the
    shared memory of one CTA, so the physical rows are formed one reflector at
    a time (phys_rows_kernel) -- the path of every Fock cycle at nmo = 1000."""
    A = extended(1000, 2000, 35, dup=True)
    w, C = eigh_gpu(agf2_lib, cuda_handle, A, nphys=1000)
    wr, Vr = np.linalg.eigh(A)
    scale = np.abs(wr).max()
    assert np.abs(w - wr).max() <= 1e-11 * scale
    assert np.abs(C @ C.T - np.eye(1000)).max() <= 1e-10
    assert np.abs((C * w) @ C.T - A[:1000, :1000]).max() <= 1e-10 * scale
    gaps = np.nonzero(np.diff(wr) > 1e-6 * scale)[0] + 1
    for k in gaps[:: max(1, len(gaps) // 10)]:
        P = C[:, :k] @ C[:, :k].T
        Pr = Vr[:1000, :k] @ Vr[:1000, :k].T
        assert np.abs(P - Pr).max() <= 1e-9, k
