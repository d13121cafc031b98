/*
 * agf2.h -- C ABI of the GB300 AGF2 library (moment-truncated auxiliary
 * second-order Green's function theory, Backhouse, Santana-Bonilla & Booth,
 * arXiv 2106.03508).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Array arguments are row-major FP64 pointers to DEVICE memory of the
 *    handle's device unless stated otherwise.  The caller allocates them,
 *    owns them and keeps them alive until the call returns.  Calls are
 *    synchronous with respect to the host: outputs are complete on return.
 *  - The library owns only the workspace held by the handle (grown on
 *    demand, freed by agf2_destroy).  Work is issued on the handle's stream
 *    (agf2_set_stream; default: the legacy default stream); the AGF2_BF16X3
 *    moment build also forks part of its work onto a second stream owned by
 *    the handle and joins it back into the handle's stream with events
 *    before it returns.
 *  - Every function returns an int status (AGF2_OK = 0).  On failure the
 *    outputs are unspecified and agf2_last_error(handle) returns a message.
 *    No C++ exception crosses the ABI.
 *  - The DF tensor L is [naux][nmo][nmo], each L[Q] symmetric, defining the
 *    electron repulsion integrals (pq|rs) = sum_Q L[Q][p][q] L[Q][r][s].
 *  - A handle is not thread safe; use one handle per host thread.
 */
#ifndef AGF2_H
#define AGF2_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define AGF2_OK                 0
#define AGF2_ERR_INVALID_ARG    1   /* bad size, null pointer, bad option      */
#define AGF2_ERR_CUDA           2   /* a CUDA / cuSOLVER / cuBLAS call failed  */
#define AGF2_ERR_OOM            3   /* workspace allocation failed             */
#define AGF2_ERR_NOT_PD         4   /* U^(0) not positive definite (compress)  */
#define AGF2_ERR_NO_CONVERGENCE 5   /* an iteration cap was reached            */
#define AGF2_ERR_TIMEOUT        6   /* a bounded device wait gave up           */
#define AGF2_ERR_UNSUPPORTED    7   /* precision/size not supported here       */

/* ---- precision of the moment build ---- */
#define AGF2_FP64   0   /* FP64 throughout                                     */
#define AGF2_BF16X3 1   /* three-limb BF16 split products on tcgen05 tensor
                           cores, FP32 accumulation, FP64 reduction            */

typedef struct agf2_context* agf2_handle;

/* Create a handle bound to CUDA device `device`; *out receives it. */
int agf2_create(agf2_handle* out, int device);
/* Free the handle and its workspace (NULL is accepted). */
int agf2_destroy(agf2_handle h);
/* Issue all further work on `stream` (a cudaStream_t passed as void*). */
int agf2_set_stream(agf2_handle h, void* stream);
/* Message of the last failure on this handle ("" if none).  The string is
   owned by the handle and valid until its next call. */
const char* agf2_last_error(agf2_handle h);

/*
 * One-body Hamiltonian of the synthetic closed-shell systems: h such that
 * the Fock matrix of Eq. (fock_matrix) at the aufbau density
 * D0 = diag(2,..,2,0,..,0) (nocc doubly occupied orbitals) equals diag(eps):
 *     h = diag(eps) - (J[D0] - K[D0]/2).
 *   L     [naux][nmo][nmo]  in
 *   eps   [nmo]             in   orbital energies, occupied first
 *   hcore [nmo][nmo]        out
 */
int agf2_hcore_from_mo_energies(agf2_handle h, const double* L, int naux, int nmo,
                                const double* eps, int nocc, double* hcore);

/*
 * Self-energy moments, Eqs. (mp2_zeroth_moment), (mp2_first_moment) and
 * their greater (particle) analogue, over the current Green's-function
 * poles (the QMOs replace the MOs after the first iteration):
 *   U_<^(n)_pq = sum_{ija} (pi|ja)[2(qi|ja) - (qj|ia)] (e_i + e_j - e_a)^n
 *   U_>^(n)_pq = sum_{abi} (pa|bi)[2(qa|bi) - (qb|ai)] (e_a + e_b - e_i)^n
 * with (px|yz) = sum_Q (L^Q C)_px (C^T L^Q C)_yz.  This is the only
 * O(N^5) step of an AGF2 iteration.
 *   L      [naux][nmo][nmo]   in
 *   e      [nqmo]             in   pole energies; e < mu is occupied
 *   C      [nmo][nqmo]        in   physical-space couplings of the poles
 *   nmom   moment orders 0..nmom are produced (nmom >= 1; AGF2_BF16X3
 *          supports nmom <= 3, else AGF2_ERR_UNSUPPORTED)
 *   precision AGF2_FP64 or AGF2_BF16X3
 *   U_hole [nmom+1][nmo][nmo] out  (symmetrised)
 *   U_part [nmom+1][nmo][nmo] out  (symmetrised)
 * Needs at least one occupied and one virtual pole (else INVALID_ARG).
 * AGF2_BF16X3 holds the rotated integrals as three-limb BF16 planes,
 * 6 (nqmo nmo + o v) ceil32(naux) bytes (o, v the occupied / virtual pole
 * counts), plus the DF factors' four-limb planes and ~2 GB of pair-block
 * buffers; at nmo = 1000, naux = 4000, 3000 poles about 160 GB of workspace.
 */
int agf2_build_moments(agf2_handle h, const double* L, int naux, int nmo,
                       const double* e, const double* C, int nqmo, double mu,
                       int nmom, int precision, double* U_hole, double* U_part);

/*
 * Moment-conserving compression of one sector, Eq. (block_lanczos_chol_3)
 * and the M-block below it: T T^T = U^(0) (lower Cholesky),
 * M = T^-1 U^(1) T^-T, M = W diag(E) W^T, v = T W.  The nmo auxiliaries
 * (E, v) reproduce U^(0) = v v^T and U^(1) = v diag(E) v^T.
 *   U     [2][nmo][nmo]  in   U^(0), U^(1) of one sector
 *   E_aux [nmo]          out  ascending
 *   v_aux [nmo][nmo]     out  column k couples auxiliary k
 * Returns AGF2_ERR_NOT_PD if U^(0) is not positive definite.
 */
int agf2_compress(agf2_handle h, const double* U, int nmo, double* E_aux, double* v_aux);

/*
 * Compression that conserves the moments U^(0..nmom), nmom = 2m+1 odd: the
 * higher truncations of the compression paragraph (text before Eq.
 * post_compression_h), as m+1 steps of the block Lanczos recursion that
 * Eq. (block_lanczos_chol_3) starts, driven by the moments alone:
 *   U^(0) = B0 B0^T;  A_i = Q_i^T E Q_i;
 *   R_i = E Q_i - Q_i A_i - Q_{i-1} B_{i-1}^T,  R_i^T R_i = B_i^T B_i,
 *   Q_{i+1} = R_i B_i^-1,
 * with every Q_i^T E^s Q_j evaluated from U^(k+l+s).  The block-tridiagonal
 * matrix (diagonal A_0..A_m, sub-diagonal B_1..B_m) = W diag(E) W^T gives
 * the (m+1) nmo auxiliaries (E, B0 W[:nmo]); nmom = 1 is agf2_compress.
 *   U     [nmom+1][nmo][nmo]        in   moments of one sector
 *   E_aux [(nmom+1)/2 nmo]          out  ascending
 *   v_aux [nmo][(nmom+1)/2 nmo]     out  column k couples auxiliary k
 * Returns AGF2_ERR_NOT_PD if U^(0) or a Lanczos block R_i^T R_i is not
 * positive definite, AGF2_ERR_INVALID_ARG if nmom is even.
 */
int agf2_compress_moments(agf2_handle h, const double* U, int nmo, int nmom, double* E_aux,
                          double* v_aux);

/*
 * Eigenpairs of a real symmetric matrix, for the extended Hamiltonian
 * [[F, v], [v^T, diag(E)]] of Eqs. (dyson_eq_eig) / (post_compression_h)
 * whose eigenvalues are the Green's-function poles and whose eigenvectors'
 * physical rows are the pole couplings.  This is the eigensolver the Fock
 * loop uses: Householder tridiagonalisation in one cooperative kernel,
 * divide and conquer with Gu-Eisenstat eigenvectors, back-transformation of
 * the first nphys rows only.
 *   A [n][n]        in   symmetric (row- or column-major alike), unchanged
 *   w [n]           out  eigenvalues, ascending
 *   V [n][n]        out  column-major: eigenvector x in V[x n .. x n + n),
 *                        of which only the first nphys entries are written
 * Returns AGF2_ERR_INVALID_ARG unless 1 <= nphys <= n <= 7000, and
 * AGF2_ERR_TIMEOUT if the tridiagonalisation's grid barrier gave up.
 */
int agf2_eigh_physical(agf2_handle h, const double* A, int n, int nphys, double* w, double* V);

typedef struct {
    double tol_D;      /* convergence: max |D_new - D| (default 1e-10)        */
    int    max_cycle;  /* Fock cycles (default 50)                            */
    double shift_tol;  /* |n(delta) - nelec| target of the shift (1e-11)      */
    double damping;    /* linear mixing of F before DIIS starts (0.3)         */
    int    diis_start; /* first cycle whose pair enters DIIS (10)             */
    int    diis_space; /* DIIS history length (6)                             */
    int    shift_mode; /* 1 (default): one safeguarded Newton step on the shift
                          per cycle, one eigendecomposition per cycle;
                          0: solve the shift to shift_tol every cycle (Newton
                          with bracket, the same root as bisection).  Both stop
                          at the same fixed point: max|dD| < tol_D and
                          |n - nelec| < shift_tol                             */
} agf2_fock_opts;

typedef struct {
    int    cycles;     /* Fock cycles run                                     */
    int    converged;  /* 1 if max|dD| < tol_D                                */
    int    nocc_qmo;   /* occupied poles (aufbau count)                       */
    int    shift_evals;/* eigendecompositions spent on the shift, summed      */
    double nerr;       /* n - nelec of the last shift solve                   */
    double mu;         /* chemical potential (HOQMO/LUQMO midpoint)           */
} agf2_fock_info;

/* Fill `o` with the defaults listed above. */
void agf2_fock_opts_default(agf2_fock_opts* o);

/*
 * Fock loop (density relaxation with the chemical potential held so that the
 * non-idempotent density has nelec electrons; text after Eq. dyson_eq_eig):
 * each cycle shifts all auxiliary energies by a common delta with
 * n(delta) = nelec at fixed aufbau count, diagonalises the extended
 * Hamiltonian [[F, v],[v^T, diag(E)]] (Eq. post_compression_h), sets
 * D = 2 C_occ C_occ^T, and rebuilds F[D] by Eq. (fock_matrix).
 *   hcore [nmo][nmo]        in
 *   E_se  [nse]             in/out  auxiliary energies (returned shifted)
 *   v_se  [nmo][nse]        in      auxiliary couplings
 *   D     [nmo][nmo]        in/out  density
 *   F     [nmo][nmo]        out     F[D] of the returned D
 *   e_qmo [nmo+nse]         out     poles, ascending
 *   C_qmo [nmo][nmo+nse]    out     physical part of the eigenvectors
 *   opts  host pointer or NULL (defaults); info host pointer or NULL
 * Returns AGF2_ERR_NO_CONVERGENCE (outputs valid) if the cap is reached,
 * AGF2_ERR_INVALID_ARG if nmo + nse > 7000 (the eigensolver's limit).
 */
int agf2_fock_loop(agf2_handle h, const double* hcore, const double* L, int naux,
                   int nmo, int nelec, double* E_se, const double* v_se, int nse,
                   double* D, double* F, double* e_qmo, double* C_qmo,
                   const agf2_fock_opts* opts, agf2_fock_info* info);

typedef struct {
    int    max_iter;   /* outer AGF2 iterations (default 50)                  */
    double conv_tol;   /* |dE_tot| convergence (default 1e-8 Ha)              */
    int    nmom;       /* conserved moments 0..nmom, odd: AGF2(m,0) with
                          nmom = 2m+1 (default 1); (nmom+1)/2 nmo
                          auxiliaries per sector; AGF2_BF16X3: nmom <= 3    */
    int    precision;  /* AGF2_FP64 or AGF2_BF16X3                            */
    double mix;        /* moment mixing U <- U_prev + mix (U - U_prev) (1.0)  */
    int    resume;     /* 1: continue from the state kept in the handle       */
    agf2_fock_opts fock;
} agf2_opts;

typedef struct {
    double E_hf, E_1b, E_2b, E_tot;   /* Ha                                   */
    double ip, ea, mu;                /* ip = -e_HOQMO, ea = -e_LUQMO         */
    int    iterations;                /* outer iterations done in this call  */
    int    converged;
    int    nocc_qmo;
    int    fock_cycles;               /* of the last iteration                */
    double t_moments, t_compress, t_fock, t_energy;  /* seconds, summed      */
    double flops_moments;             /* algorithmic flops of the moment builds */
    int    fock_converged;            /* 1 if the last iteration's Fock loop met
                                         its density tolerance (else it stopped
                                         at max_cycle)                        */
    int    fock_cycles_total;         /* Fock cycles summed over the call      */
} agf2_result;

/* Fill `o` with the defaults listed above. */
void agf2_opts_default(agf2_opts* o);

/*
 * Full AGF2 iteration from the Hartree-Fock reference (Eq. gf_hf): the
 * reference density D0 gives F[D0] by Eq. (fock_matrix), and the initial
 * poles and couplings are its eigenpairs, e = eig(F[D0]) with C the
 * eigenvectors, in whatever orthonormal basis hcore, L and D0 are given.
 * Then moments -> moment mixing -> compression of each sector
 * (agf2_compress_moments) -> Fock loop over nmo + (nmom+1) nmo poles ->
 * energies, until |dE_tot| < conv_tol or max_iter.  E_hf = Tr[D0(h+F[D0])]/2,
 * E_1b = Tr[D(h+F)]/2; E_2b is the Galitskii-Migdal sum over occupied poles x
 * and particle-sector auxiliaries k of (C_x . v_k)^2 / (e_x - E_k).  The final
 * state (poles, self-energy, density, mixing history) stays in the handle;
 * with opts->resume = 1 the next call continues from it (D0 is then ignored).
 *   hcore [nmo][nmo], L [naux][nmo][nmo]: device pointers
 *   D0 [nmo][nmo]: device pointer to the reference density (2 x the
 *     projector onto the nelec/2 occupied orbitals), or NULL for the aufbau
 *     density of the first nelec/2 basis functions -- the basis of the
 *     reference's canonical orbitals, as for the synthetic systems
 *   opts, out: host pointers (opts NULL = defaults)
 * Returns AGF2_ERR_NO_CONVERGENCE (with *out filled) if max_iter is reached
 * before convergence and max_iter > 1, AGF2_ERR_INVALID_ARG if the extended
 * Hamiltonian would exceed the eigensolver's limit, nmo (nmom + 2) > 7000.
 */
int agf2_run(agf2_handle h, const double* hcore, const double* L, int naux, int nmo,
             int nelec, const double* D0, const agf2_opts* opts, agf2_result* out);

/* One system of a batch: device pointers as for agf2_run. */
typedef struct {
    const double* hcore;   /* [nmo][nmo]            */
    const double* L;       /* [naux][nmo][nmo]      */
    const double* D0;      /* [nmo][nmo] or NULL    */
    int naux, nmo, nelec;
} agf2_system;

/*
 * Many independent systems of uneven size (nmo, nocc, naux) in one call:
 * agf2_run (from the HF reference, opts->resume ignored) on each, with
 * `nworkers` host worker threads (0: 8), each owning a handle, a non-blocking
 * stream and its workspace on h's device, so that the small systems' kernels
 * run concurrently.  out[i] (host) receives system i's result and status[i]
 * (host, may be NULL) its status.  Returns AGF2_OK when every system returned
 * AGF2_OK or AGF2_ERR_NO_CONVERGENCE, else the first other error (message in
 * agf2_last_error(h)).  Systems are not graph-captured: each runs the same
 * host-sequenced iteration as agf2_run.
 */
int agf2_run_batched(agf2_handle h, int nsys, const agf2_system* systems, const agf2_opts* opts,
                     int nworkers, agf2_result* out, int* status);

/*
 * Copy the Green's function kept in the handle after agf2_run: nqmo poles
 * e [nqmo] and couplings C [nmo][nqmo] (device pointers sized for 3*nmo),
 * the density D [nmo][nmo].  *nqmo receives the pole count (host pointer).
 * Any output pointer may be NULL.
 */
int agf2_get_state(agf2_handle h, double* e, double* C, double* D, int* nqmo);

/*
 * Spectral function of the Green's function (the broadened spectra of the
 * paper's artemisinin figure, eta = 0.2 eV there):
 *   A_p(w) = -(1/pi) Im G_pp(w + i eta) = (1/pi) sum_x C[p][x]^2 eta / ((w - e_x)^2 + eta^2),
 *   A(w)   = sum_p A_p(w)  (the trace).
 *   e [nqmo], C [nmo][nqmo]: poles and couplings (e.g. from agf2_get_state)
 *   omega [nomega]: frequencies (Ha); eta > 0 (Ha)
 *   A_total [nomega] out; A_orb [nmo][nomega] out or NULL
 */
int agf2_spectral_function(agf2_handle h, const double* e, const double* C, int nmo, int nqmo,
                           const double* omega, int nomega, double eta, double* A_total,
                           double* A_orb);

/*
 * Opt-in timing with CUDA events on the handle's stream.  With enable = 1,
 * agf2_kernel_stats returns, since the last agf2_set_profiling call, the
 * number of timed regions of a kind, their summed duration (ms) and their
 * algorithmic flop count:
 *   kind 0: pair GEMM launches of the split-precision moment build (GEMM 1
 *           with its S/D and energy-weight epilogue; the ordered pole pairs'
 *           share of N o' v' (o'+v') 2 n_Q),
 *   kind 1: moment GEMM launches (GEMM 2 into U; 2 (nmom+1) N^2 per
 *           ordered pair and inner pole),
 *   kind 2: the FP64 GEMMs of each DF Fock build, Eq. (fock_matrix)
 *           (2 n^2 m n_Q for L C or L D, m = k or n, plus n (n+1) m n_Q for
 *           the symmetric half of K),
 *   kind 3: each extended-Hamiltonian eigendecomposition of the Fock loop
 *           (4/3 n^3 + 4 nmo n^2).
 * Timing adds event records and is off by default.
 */
int agf2_set_profiling(agf2_handle h, int enable);
int agf2_kernel_stats(agf2_handle h, int kind, long long* launches, double* ms, double* flops);

/*
 * Allocation-free FP64 moment build (the paper has no counterpart: this is a
 * deployment variant of agf2_build_moments with precision AGF2_FP64).
 * For callers that cannot let a library allocate device memory -- e.g. an
 * application whose own allocator owns the device budget, where cudaFree
 * would synchronise the device and a late cudaMalloc could fail.  It needs no
 * handle and calls no cudaMalloc/cudaFree: every intermediate lives in one
 * static device array of 64 MiB inside the library, held on every GPU that
 * loads the library until the process exits.  The intermediates take
 * 8 (nqmo nmo naux + o' v' naux + 6 nmo max(o', v')) bytes plus O(nqmo nmo)
 * (o', v': occupied and virtual pole counts); the call takes the largest of
 * this over every split o' + v' = nqmo and rejects sizes where it exceeds
 * 64 MiB with AGF2_ERR_INVALID_ARG before any argument is read, so an
 * accepted size fits whatever the pole energies are.
 *   Arguments and outputs as agf2_build_moments (nmom = 1); `stream` is a
 *   cudaStream_t passed as void* (NULL: legacy default stream).  Returns when
 *   the outputs are complete.
 * The first call on a device (with that device current) looks up the static
 * array's device address; make that call before any stream capture.  All
 * calls share the array: calls whose GPU work overlaps (other streams or host
 * threads) race on it.  Errors are reported by the return code only.
 */
int agf2_build_moments_noalloc(const double* L, int naux, int nmo, const double* e,
                               const double* C, int nqmo, double mu, double* U_hole,
                               double* U_part, void* stream);

/* Number of CUDA kernels this library has launched since it was loaded
   (all handles; counts kernels issued by cuSOLVER/cuBLAS calls as zero). */
long long agf2_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* AGF2_H */
