// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>

namespace agf2 {

// Number of kernels this library has launched (all devices, all handles).
void count_launch(long long n = 1);

// Per-kernel-kind timing of the split-precision kernels (opt-in): CUDA events
// bracket every launch; durations are summed when the stream is synchronised.
struct KernelStats {
  static constexpr int kKinds = 4;
  bool enabled = false;
  // 0: pair GEMM (GEMM 1 + epilogue), 1: moment GEMM, 2: FP64 Fock-build
  // GEMMs (per Fock build), 3: extended-Hamiltonian eigensolver (per call)
  long long launches[kKinds] = {0, 0, 0, 0};
  double ms[kKinds] = {0.0, 0.0, 0.0, 0.0};
  double flops[kKinds] = {0.0, 0.0, 0.0, 0.0};  // algorithmic flops of those launches
};

// Generic strided, two-level-batched FP64 GEMM:
//   C[z][m][n] = alpha * sum_k A[z][m][k] * B[z][k][n] + beta * C[z][m][n]
// with element (m,k) of A at A + off_A(z) + m*sAm + k*sAk (likewise B, C) and
// z = b1 * nb2 + b2, off_X(z) = b1*sX1 + b2*sX2.
struct DGemm {
  int M = 0, N = 0, K = 0;
  const double* A = nullptr; long long sAm = 0, sAk = 0, sA1 = 0, sA2 = 0;
  const double* B = nullptr; long long sBk = 0, sBn = 0, sB1 = 0, sB2 = 0;
  double* C = nullptr;       long long sCm = 0, sCn = 0, sC1 = 0, sC2 = 0;
  int nb1 = 1, nb2 = 1;
  double alpha = 1.0, beta = 0.0;
  bool atomic = false;  // C += alpha A B with atomicAdd (beta ignored)
  int ksplit = 1;       // split K over this many CTAs (requires atomic)
  bool upper = false;   // C is symmetric (M == N, one batch, sCn == 1): compute the
                        // tiles on and above the diagonal, then mirror the rest
};
cudaError_t dgemm(const DGemm& g, cudaStream_t s);
// Output tile edge dgemm uses for an M x N product (40 where it pads less than 64).
int dgemm_tile(int M, int N);
// K splits for an M x N product with a long K: about 1024 threads per SM.
int dgemm_split(int M, int N, long long K, bool upper);

// Moment epilogue of one block pair (I, J) of outer indices (FP64 path):
// from X_IJ[p][(ii*nJ+jj)*n_in + c] = (p x_ii | y_jj c) and
// X_JI[p][(jj*nI+ii)*n_in + c] (X_JI == X_IJ when diag) build
//   Y [p][k]  = sqrt(cS) S  (k < K1),  sqrt(cD) D  (K1 <= k < 2 K1)
//   Yw[p][k]  = Y[p][k] * (e_out[x] + e_out[y] - e_in[c])
// with S = X_IJ + X_JI, D = X_IJ - X_JI, (cS, cD) = (1/4, 3/4) on the
// diagonal block and (1/2, 3/2) off it; K1 = nI*nJ*n_in.
cudaError_t sd_epilogue_fp64(const double* XIJ, const double* XJI, int nmo, int nI, int nJ,
                             int n_in, const double* e_outI, const double* e_outJ,
                             const double* e_in, bool diag, double* Y, double* Yw,
                             cudaStream_t s);

// Z <- Z * w column-wise in the layout of sd_epilogue_fp64 (Y w^n -> Y w^(n+1)).
cudaError_t weight_columns_fp64(double* Z, int nmo, int nI, int nJ, int n_in, const double* e_outI,
                                const double* e_outJ, const double* e_in, cudaStream_t s);

// Small FP64 kernels.
cudaError_t gather_columns(const double* C, int nrow, int ncol_src, const int* idx, int n,
                           double* out, cudaStream_t s);                // out[r][t] = C[r][idx[t]]
cudaError_t gather_vec(const double* e, const int* idx, int n, double* out, cudaStream_t s);
cudaError_t symmetrize(double* U, int n, int nmat, cudaStream_t s);   // U <- (U+U^T)/2
// dst (column-major, leading dimension ld) <- Lc^T, zero below the diagonal,
// from a column-major lower Cholesky factor Lc [n x n]
cudaError_t upper_from_lower_t(const double* Lc, int n, double* dst, long long ld,
                               cudaStream_t s);
cudaError_t axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t s); // y = a*x + b*y
cudaError_t build_extended_h(const double* F, const double* E, const double* v, double delta,
                             int nmo, int nse, double* H, cudaStream_t s);
// weights[x] = sum_{p<nmo} V[x*ld + p]^2   (V column-major eigenvectors, ld = n)
cudaError_t column_weights(const double* V, int ld, int nmo, int ncol, double* w, cudaStream_t s);
// out[p][x] = V[x*ld + p] for p<nmo, x<ncol (physical block, row-major)
cudaError_t physical_block(const double* V, int ld, int nmo, int ncol, double* out, cudaStream_t s);
// sum of a[i]*b[i] into *out (device scalar), deterministic two-pass.
cudaError_t dot(const double* a, const double* b, long long n, double* out, double* scratch,
                cudaStream_t s);
// J_pq = sum_Q gamma_Q L[Q][p][q]
cudaError_t coulomb_from_gamma(const double* L, const double* gamma, int naux, int nmo, double* J,
                               cudaStream_t s);
// gamma_Q = 2 sum_{r,k} Cocc[r][k] Y[r][Q][k]
cudaError_t gamma_from_y(const double* Y, const double* Cocc, int nmo, int naux, int k,
                         double* gamma, cudaStream_t s);
// gamma_Q = sum_rs L[Q][r][s] D[r][s]
cudaError_t gamma_from_density(const double* L, const double* D, int naux, int n,
                               double* gamma, cudaStream_t s);
// F = h + J - K/2  (elementwise)
cudaError_t fock_combine(const double* h, const double* J, const double* K, long long n, double* F,
                         cudaStream_t s);
// GM: out = sum_{x<k, m<nse} V[x][m]^2 / (e[x] - E[m]), V = Cocc^T v (k x nse)
cudaError_t gm_energy(const double* V, const double* e, const double* E, int k, int nse,
                      double* out, double* scratch, cudaStream_t s);
// dn/d(delta) = 4 sum_{x<k,y} S[x][y]^2 / (w[k+y] - w[x]),  S = C_occ^T C_vir
cudaError_t shift_derivative(const double* S, const double* w, int k, int nv, double* out,
                             double* scratch, cudaStream_t s);
cudaError_t set_identity(double* A, int n, double scale, cudaStream_t s);
// lor[x][w] = eta/pi / ((w_j - e_x)^2 + eta^2);  out = a*a;  out[j] = sum_r M[r][j]
cudaError_t lorentzian(const double* e, int nq, const double* w, int nw, double eta, double* lor,
                       cudaStream_t s);
cudaError_t square(const double* a, long long n, double* out, cudaStream_t s);
cudaError_t column_sum(const double* M, int nrow, int ncol, double* out, cudaStream_t s);
cudaError_t diag_from_vec(const double* d, int n, double* A, cudaStream_t s);
// max |a - b| into *out (device)
cudaError_t max_abs_diff(const double* a, const double* b, long long n, double* out, double* scratch,
                         cudaStream_t s);
cudaError_t add_scalar(double* x, double a, int n, cudaStream_t s);

// Split-precision (BF16x3 / tcgen05) moment build: rotates L into the pole
// basis (occupied couplings Co [N][o], virtual Cv [N][v]) block by block
// straight into BF16 limb planes, then accumulates moments 0..nmom
// (nmom <= 3) into the zeroed U_hole, U_part [nmom+1][N][N] (upper tiles
// mirrored, not symmetrised).  Returns an AGF2 status; err receives a message.
int mixed_build_moments(const double* L, int naux, int N, const double* Co, const double* Cv,
                        int o, int v, const double* eo, const double* ev, int nmom,
                        double* U_hole, double* U_part, std::string& err, cudaStream_t s,
                        KernelStats* stats, void* workspace);
// Pole-basis rotation on the tensor cores (rotate.cu), four-limb split with
// exact chunk sums, FP64 results:
//   out[m sOm + b sOb + n] = sum_k A[a_row0 + m][k] B[b][n][k]
// from limb planes A [4][rowsA][Ks], B [4][nbatch][Nn][Ks] (Ks a multiple of
// 256) with row units unitA [rowsA], unitB [nbatch][Nn].
int rot_gemm4(const __nv_bfloat16* A, long long rowsA, int a_row0, int M, const float* unitA,
              const __nv_bfloat16* B, int Nn, int nbatch, const float* unitB, int Ks,
              double* out, long long sOm, long long sOb, int* derr, std::string& err,
              cudaStream_t s);
// FP64 rows (element (r, c) at src[r ld + c cs]) -> four integer BF16 limb
// planes [4][dst_rows][ncolp] with units (row r -> (r/grp) gstride + goff + r%grp).
int rot_limbs_slice4(const double* src, long long nrow, int ncol, long long ld, long long cs,
                     int ncolp, long long dst_rows, long long grp, long long gstride,
                     long long goff, __nv_bfloat16* dst, float* unit, cudaStream_t s);
// W [nx][nQ][N] -> three-limb planes of the rows (x, p) over Q, rows
// row0 + x N + p of [3][dst_rows][Qs], with certified units (stats: nx N doubles
// of scratch for the row units).
int rot_transpose_slice3(const double* W, int nx, int nQ, int N, int Qs, double* stats,
                         long long dst_rows, long long row0, __nv_bfloat16* dst, float* unit,
                         cudaStream_t s);
// Symmetric FP64 eigensolver (eigen.cu): eigenvalues ascending into w and
// the first nphys rows of the eigenvectors into V (column-major, column x at
// V + x n), n <= 7000.  A [n][n] symmetric is not modified.  Workspace: one per handle.
int eigh_phys(void* workspace, const double* A, int n, int nphys, double* w, double* V,
              cudaStream_t s, std::string& err);
void* eig_workspace_create();
void eig_workspace_destroy(void* w);
// Workspace of the split-precision path, one per handle.
void* mixed_workspace_create();
void mixed_workspace_destroy(void* w);

}  // namespace agf2
