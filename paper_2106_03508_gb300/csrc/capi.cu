// C ABI of the AGF2 library and the host-side sequencing of one AGF2
// iteration (moments -> compression -> Fock loop -> energies).  All array
// arithmetic runs in this library's CUDA kernels (fp64.cu, mixed.cu,
// eigen.cu: the Fock loop's extended-Hamiltonian eigensolver) or in
// cuSOLVER/cuBLAS for the small O(N^3) FP64 dense linear algebra of the
// compression (Cholesky, triangular solves, the N x N or (m+1)N x (m+1)N
// eigenproblem); the host only takes scalar decisions (aufbau count, shift
// step or bracket, DIIS coefficients, convergence).
#include <cublas_v2.h>
#include <cusolverDn.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/agf2.h"
#include "agf2_internal.h"

using namespace agf2;
namespace agf2 {
long long launch_count();
}

struct agf2_context {
  int device = 0;
  cudaStream_t stream = nullptr;
  cusolverDnHandle_t solver = nullptr;
  cublasHandle_t blas = nullptr;
  std::string err;
  struct Buf { void* p = nullptr; size_t bytes = 0; };
  std::map<std::string, Buf> bufs;
  int* dev_info = nullptr;
  // ---- state kept between agf2_run calls ----
  bool have_state = false;
  int nmo = 0, nq = 0, nq_max = 0;  // nq_max: leading dimension of the state C
  double mu = 0.0, E_prev = 0.0, E_hf = 0.0;
  bool have_uprev = false;
  int iter = 0;
  KernelStats stats;
  struct Pending { cudaEvent_t a, b; int kind; double flops; };
  std::vector<Pending> pending;  // timed regions not yet read back
  void* mixed_ws = nullptr;
  void* eig_ws = nullptr;
};

namespace {

struct Fail {
  int code;
};

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                        \
      throw Fail{AGF2_ERR_CUDA};                                                           \
    }                                                                                      \
  } while (0)
#define CKS(call)                                                                          \
  do {                                                                                     \
    cusolverStatus_t e_ = (call);                                                          \
    if (e_ != CUSOLVER_STATUS_SUCCESS) {                                                   \
      ctx->err = std::string(#call) + ": cusolver status " + std::to_string((int)e_);      \
      throw Fail{AGF2_ERR_CUDA};                                                           \
    }                                                                                      \
  } while (0)
#define CKB(call)                                                                          \
  do {                                                                                     \
    cublasStatus_t e_ = (call);                                                            \
    if (e_ != CUBLAS_STATUS_SUCCESS) {                                                     \
      ctx->err = std::string(#call) + ": cublas status " + std::to_string((int)e_);        \
      throw Fail{AGF2_ERR_CUDA};                                                           \
    }                                                                                      \
  } while (0)

void fail(agf2_context* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  throw Fail{code};
}

template <class T = double>
T* ws(agf2_context* ctx, const char* name, size_t count) {
  size_t bytes = std::max<size_t>(count * sizeof(T), 256);
  auto& b = ctx->bufs[name];
  if (b.bytes < bytes) {
    if (b.p) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(b.p);
      b.p = nullptr;
      b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->err = std::string("workspace '") + name + "' of " + std::to_string(bytes) +
                 " bytes: " + cudaGetErrorString(e);
      throw Fail{AGF2_ERR_OOM};
    }
    b.bytes = bytes;
  }
  return static_cast<T*>(b.p);
}

// Timed regions of kinds 2 and 3 (see KernelStats): events on the handle's
// stream, read back at the next synchronisation.
struct TimedRegion {
  agf2_context* ctx;
  cudaEvent_t a = nullptr, b = nullptr;
  int kind;
  double flops;
  TimedRegion(agf2_context* c, int k, double f) : ctx(c), kind(k), flops(f) {
    if (!ctx->stats.enabled) return;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, ctx->stream);
  }
  ~TimedRegion() {
    if (!a) return;
    cudaEventRecord(b, ctx->stream);
    ctx->pending.push_back({a, b, kind, flops});
  }
};

void flush_stats(agf2_context* ctx) {
  for (auto& p : ctx->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      ctx->stats.launches[p.kind] += 1;
      ctx->stats.ms[p.kind] += ms;
      ctx->stats.flops[p.kind] += p.flops;
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  ctx->pending.clear();
}

void sync(agf2_context* ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  if (!ctx->pending.empty()) flush_stats(ctx);
}

template <class T>
std::vector<T> to_host(agf2_context* ctx, const T* d, size_t n) {
  std::vector<T> h(n);
  if (n) {
    CK(cudaMemcpyAsync(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
    sync(ctx);
  }
  return h;
}

double scalar(agf2_context* ctx, const double* d) { return to_host(ctx, d, 1)[0]; }

void check_dev_ptr(agf2_context* ctx, const void* p, const char* name) {
  if (!p) fail(ctx, AGF2_ERR_INVALID_ARG, std::string(name) + " is NULL");
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(ctx, AGF2_ERR_INVALID_ARG, std::string(name) + ": not a CUDA pointer");
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    fail(ctx, AGF2_ERR_INVALID_ARG, std::string(name) + " must be device memory");
}

// NVTX range for the stages of one iteration (visible to profilers; a no-op
// unless a tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// ---------------------------------------------------------------------------
// Fock matrix, Eq. (fock_matrix), density fitted
// ---------------------------------------------------------------------------
// General D: J = sum_Q L^Q Tr(L^Q D),  K = sum_Q L^Q D L^Q.
void fock_general(agf2_context* ctx, const double* h, const double* L, int naux, int n,
                  const double* D, double* F) {
  cudaStream_t s = ctx->stream;
  const long long nn = (long long)n * n;
  double* Z = ws(ctx, "fock_Z", (size_t)naux * nn);
  double* J = ws(ctx, "fock_J", nn);
  double* K = ws(ctx, "fock_K", nn);
  double* gam = ws(ctx, "fock_gamma", naux);
  CK(gamma_from_density(L, D, naux, n, gam, s));
  CK(coulomb_from_gamma(L, gam, naux, n, J, s));
  // algorithmic flops: Z = L D (2 n^3 n_Q) and the symmetric half of K (n^2 (n+1) n_Q)
  TimedRegion tr(ctx, 2, (2.0 * n + (n + 1.0)) * (double)n * n * naux);
  // Z[p][Q][r] = sum_s L[Q][p][s] D[s][r]
  {
    DGemm g;
    g.M = n; g.N = n; g.K = n;
    g.A = L; g.sAm = n; g.sAk = 1; g.sA1 = nn;
    g.B = D; g.sBk = n; g.sBn = 1;
    g.C = Z; g.sCm = (long long)naux * n; g.sCn = 1; g.sC1 = n;
    g.nb1 = naux;
    CK(dgemm(g, s));
  }
  // K[p][q] = sum_{(Q,r)} Z[p][(Q,r)] L[(Q,r)][q]
  {
    DGemm g;
    g.M = n; g.N = n; g.K = naux * n;
    g.A = Z; g.sAm = (long long)naux * n; g.sAk = 1;
    g.B = L; g.sBk = n; g.sBn = 1;
    g.C = K; g.sCm = n; g.sCn = 1;
    g.atomic = true;
    g.upper = true;  // K is symmetric
    g.ksplit = dgemm_split(n, n, g.K, true);
    CK(cudaMemsetAsync(K, 0, nn * sizeof(double), s));
    CK(dgemm(g, s));
  }
  CK(fock_combine(h, J, K, nn, F, s));
}

// D = 2 Cocc Cocc^T with Cocc [n][k]:  J via gamma_Q = 2 sum Cocc . (L^Q Cocc),
// K = 2 sum_Q (L^Q Cocc)(L^Q Cocc)^T.  Cost 4 N^2 k naux instead of 4 N^3 naux.
void fock_cocc(agf2_context* ctx, const double* h, const double* L, int naux, int n,
               const double* Cocc, int k, double* F) {
  cudaStream_t s = ctx->stream;
  const long long nn = (long long)n * n;
  double* Y = ws(ctx, "fock_Y", (size_t)n * naux * k);
  double* J = ws(ctx, "fock_J", nn);
  double* K = ws(ctx, "fock_K", nn);
  double* gam = ws(ctx, "fock_gamma", naux);
  // algorithmic flops: Y = L Cocc (2 n^2 k n_Q) and the symmetric half of K (n (n+1) k n_Q)
  TimedRegion tr(ctx, 2, (2.0 * n + (n + 1.0)) * (double)n * k * naux);
  {
    DGemm g;  // Y[p][Q][c] = sum_r L[Q][p][r] Cocc[r][c]
    g.M = n; g.N = k; g.K = n;
    g.A = L; g.sAm = n; g.sAk = 1; g.sA1 = nn;
    g.B = Cocc; g.sBk = k; g.sBn = 1;
    g.C = Y; g.sCm = (long long)naux * k; g.sCn = 1; g.sC1 = k;
    g.nb1 = naux;
    CK(dgemm(g, s));
  }
  CK(gamma_from_y(Y, Cocc, n, naux, k, gam, s));
  CK(coulomb_from_gamma(L, gam, naux, n, J, s));
  {
    DGemm g;  // K = 2 Y Y^T over (Q, c), split over K with FP64 atomics
    g.M = n; g.N = n; g.K = naux * k;
    g.A = Y; g.sAm = (long long)naux * k; g.sAk = 1;
    g.B = Y; g.sBk = 1; g.sBn = (long long)naux * k;
    g.C = K; g.sCm = n; g.sCn = 1;
    g.alpha = 2.0;
    g.atomic = true;
    g.upper = true;
    g.ksplit = dgemm_split(n, n, g.K, true);
    CK(cudaMemsetAsync(K, 0, nn * sizeof(double), s));
    CK(dgemm(g, s));
  }
  CK(fock_combine(h, J, K, nn, F, s));
}

// F[D] for D = 2 Cocc Cocc^T (Cocc [n][k], D given as well): through the
// occupied couplings while k < n (about 3 n^2 k n_Q flops), else through D
// (about 3 n^3 n_Q flops); both form only the symmetric half of K.
void fock_density(agf2_context* ctx, const double* h, const double* L, int naux, int n,
                  const double* D, const double* Cocc, int k, double* F) {
  if (k < n)
    fock_cocc(ctx, h, L, naux, n, Cocc, k, F);
  else
    fock_general(ctx, h, L, naux, n, D, F);
}

// ---------------------------------------------------------------------------
// Moments, Eqs. (mp2_zeroth_moment), (mp2_first_moment): FP64 path
// ---------------------------------------------------------------------------
struct Sector {
  int n_out, n_in;
  const double* Lx_out;  // [n_out][N][Q]
  const double* Lpair;   // element (y, c, Q) at y*ys + c*cs + Q
  long long ys, cs;
  const double* e_out;
  const double* e_in;
};

void sector_fp64(agf2_context* ctx, const Sector& S, int N, int naux, int nmom, double* U) {
  cudaStream_t s = ctx->stream;
  const double budget_doubles = 2.0e8;  // 1.6 GB over the 6 block arrays
  int nb = (int)std::floor(std::sqrt(budget_doubles / 6.0 / ((double)N * S.n_in)));
  nb = std::max(1, std::min(nb, S.n_out));
  const size_t K1max = (size_t)nb * nb * S.n_in;
  double* XIJ = ws(ctx, "mom_XIJ", (size_t)N * K1max);
  double* XJI = ws(ctx, "mom_XJI", (size_t)N * K1max);
  double* Y = ws(ctx, "mom_Y", (size_t)N * 2 * K1max);
  double* Yw = ws(ctx, "mom_Yw", (size_t)N * 2 * K1max);
  const long long NQ = (long long)N * naux;
  for (int I0 = 0; I0 < S.n_out; I0 += nb) {
    const int nI = std::min(nb, S.n_out - I0);
    for (int J0 = I0; J0 < S.n_out; J0 += nb) {
      const int nJ = std::min(nb, S.n_out - J0);
      const bool diag = (I0 == J0);
      const long long K1 = (long long)nI * nJ * S.n_in;
      auto pair_gemm = [&](int A0, int nA, int B0, int nB, double* X) {
        DGemm g;  // X[p][(a*nB+b)*n_in + c] = sum_Q Lx_out[A0+a][p][Q] Lpair[B0+b][c][Q]
        g.M = N; g.N = S.n_in; g.K = naux;
        g.A = S.Lx_out + (long long)A0 * NQ; g.sAm = naux; g.sAk = 1; g.sA1 = NQ; g.sA2 = 0;
        g.B = S.Lpair + (long long)B0 * S.ys; g.sBk = 1; g.sBn = S.cs; g.sB1 = 0; g.sB2 = S.ys;
        g.C = X; g.sCm = K1; g.sCn = 1; g.sC1 = (long long)nB * S.n_in; g.sC2 = S.n_in;
        g.nb1 = nA; g.nb2 = nB;
        CK(dgemm(g, s));
      };
      pair_gemm(I0, nI, J0, nJ, XIJ);
      if (!diag) pair_gemm(J0, nJ, I0, nI, XJI);
      CK(sd_epilogue_fp64(XIJ, XJI, N, nI, nJ, S.n_in, S.e_out + I0, S.e_out + J0, S.e_in, diag, Y,
                          Yw, s));
      for (int n = 0; n <= nmom; ++n) {
        // U^(n) += Z Y^T, Z = Y w^n (Yw holds Y w^n for n >= 1), K = 2 K1, split over K
        if (n >= 2)
          CK(weight_columns_fp64(Yw, N, nI, nJ, S.n_in, S.e_out + I0, S.e_out + J0, S.e_in, s));
        DGemm g;
        g.M = N; g.N = N; g.K = (int)(2 * K1);
        g.A = n == 0 ? Y : Yw; g.sAm = 2 * K1; g.sAk = 1;
        g.B = Y; g.sBk = 1; g.sBn = 2 * K1;
        g.C = U + (long long)n * N * N; g.sCm = N; g.sCn = 1;
        g.atomic = true;
        g.upper = true;  // U^(n) = (Y w^n) Y^T is symmetric
        g.ksplit = dgemm_split(N, N, 2 * K1, true);
        CK(dgemm(g, s));
      }
    }
  }
}

struct PoleSplit {
  int o = 0, v = 0;
  std::vector<int> occ, vir;
};

PoleSplit split_poles(agf2_context* ctx, const double* e, int nq, double mu) {
  PoleSplit ps;
  std::vector<double> eh = to_host(ctx, e, nq);
  for (int x = 0; x < nq; ++x) {
    if (!std::isfinite(eh[x])) fail(ctx, AGF2_ERR_INVALID_ARG, "non-finite pole energy");
    if (eh[x] < mu) ps.occ.push_back(x); else ps.vir.push_back(x);
  }
  ps.o = (int)ps.occ.size();
  ps.v = (int)ps.vir.size();
  return ps;
}

void build_moments_impl(agf2_context* ctx, const double* L, int naux, int N, const double* e,
                        const double* C, int nq, double mu, int nmom, int precision,
                        double* Uh, double* Up) {
  Range rg("agf2_moments");
  cudaStream_t s = ctx->stream;
  PoleSplit ps = split_poles(ctx, e, nq, mu);
  if (ps.o < 1 || ps.v < 1) fail(ctx, AGF2_ERR_INVALID_ARG, "need occupied and virtual poles");
  const int o = ps.o, v = ps.v;
  int* idx = ws<int>(ctx, "mom_idx", nq);
  std::vector<int> all(ps.occ);
  all.insert(all.end(), ps.vir.begin(), ps.vir.end());
  CK(cudaMemcpyAsync(idx, all.data(), nq * sizeof(int), cudaMemcpyHostToDevice, s));
  double* Co = ws(ctx, "mom_Co", (size_t)N * o);
  double* Cv = ws(ctx, "mom_Cv", (size_t)N * v);
  double* eo = ws(ctx, "mom_eo", o);
  double* ev = ws(ctx, "mom_ev", v);
  CK(gather_columns(C, N, nq, idx, o, Co, s));
  CK(gather_columns(C, N, nq, idx + o, v, Cv, s));
  CK(gather_vec(e, idx, o, eo, s));
  CK(gather_vec(e, idx + o, v, ev, s));
  const long long NN = (long long)N * N;
  CK(cudaMemsetAsync(Uh, 0, (nmom + 1) * NN * sizeof(double), s));
  CK(cudaMemsetAsync(Up, 0, (nmom + 1) * NN * sizeof(double), s));
  if (precision == AGF2_BF16X3) {
    // rotation and moments in the split-precision path, block by block
    if (!ctx->mixed_ws) ctx->mixed_ws = mixed_workspace_create();
    int rc = mixed_build_moments(L, naux, N, Co, Cv, o, v, eo, ev, nmom, Uh, Up, ctx->err, s,
                                 &ctx->stats, ctx->mixed_ws);
    if (rc != AGF2_OK) throw Fail{rc};
  } else {
    const long long NQ = (long long)N * naux;
    double* Lxo = ws(ctx, "mom_Lxo", (size_t)o * NQ);
    double* Lxv = ws(ctx, "mom_Lxv", (size_t)v * NQ);
    double* Lov = ws(ctx, "mom_Lov", (size_t)o * v * naux);
    auto rot = [&](const double* Cx, int nx, double* out) {
      DGemm g;  // out[x][p][Q] = sum_r Cx[r][x] L[Q][r][p]
      g.M = nx; g.N = N; g.K = N;
      g.A = Cx; g.sAm = 1; g.sAk = nx;
      g.B = L; g.sBk = N; g.sBn = 1; g.sB1 = NN;
      g.C = out; g.sCm = NQ; g.sCn = naux; g.sC1 = 1;
      g.nb1 = naux;
      CK(dgemm(g, s));
    };
    rot(Co, o, Lxo);
    rot(Cv, v, Lxv);
    {
      DGemm g;  // Lov[j][a][Q] = sum_p Co[p][j] Lxv[a][p][Q]
      g.M = o; g.N = v; g.K = N;
      g.A = Co; g.sAm = 1; g.sAk = o;
      g.B = Lxv; g.sBk = naux; g.sBn = NQ; g.sB1 = 1;
      g.C = Lov; g.sCm = (long long)v * naux; g.sCn = naux; g.sC1 = 1;
      g.nb1 = naux;
      CK(dgemm(g, s));
    }
    Sector hole{o, v, Lxo, Lov, (long long)v * naux, (long long)naux, eo, ev};
    Sector part{v, o, Lxv, Lov, (long long)naux, (long long)v * naux, ev, eo};
    sector_fp64(ctx, hole, N, naux, nmom, Uh);
    sector_fp64(ctx, part, N, naux, nmom, Up);
  }
  CK(symmetrize(Uh, N, nmom + 1, s));
  CK(symmetrize(Up, N, nmom + 1, s));
  sync(ctx);
}

// ---------------------------------------------------------------------------
// Compression, Eq. (block_lanczos_chol_3): T T^T = U0, M = T^-1 U1 T^-T
// ---------------------------------------------------------------------------
void syevd(agf2_context* ctx, double* A, int n, double* w) {
  int lwork = 0;
  CKS(cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                  A, n, w, &lwork));
  double* work = ws(ctx, "syevd_work", (size_t)lwork);
  CKS(cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A, n, w,
                       work, lwork, ctx->dev_info));
  int info = 0;
  CK(cudaMemcpyAsync(&info, ctx->dev_info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  if (info != 0) fail(ctx, AGF2_ERR_CUDA, "syevd failed to converge, info " + std::to_string(info));
}

void compress_impl(agf2_context* ctx, const double* U, int n, double* E, double* v_rowmajor,
                   long long ldv) {
  Range rg("agf2_compress");
  cudaStream_t s = ctx->stream;
  const long long nn = (long long)n * n;
  double* T = ws(ctx, "cmp_T", nn);
  double* M = ws(ctx, "cmp_M", nn);
  double* W = ws(ctx, "cmp_W", nn);
  CK(cudaMemcpyAsync(T, U, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(M, U + nn, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  // column-major view: U0, U1 symmetric, so the arrays are their own transposes
  int lwork = 0;
  CKS(cusolverDnDpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_LOWER, n, T, n, &lwork));
  double* work = ws(ctx, "potrf_work", (size_t)lwork);
  CKS(cusolverDnDpotrf(ctx->solver, CUBLAS_FILL_MODE_LOWER, n, T, n, work, lwork, ctx->dev_info));
  int info = 0;
  CK(cudaMemcpyAsync(&info, ctx->dev_info, sizeof(int), cudaMemcpyDeviceToHost, s));
  sync(ctx);
  if (info != 0)
    fail(ctx, AGF2_ERR_NOT_PD,
         "U^(0) is not positive definite (potrf info " + std::to_string(info) + ")");
  const double one = 1.0;
  // M <- T^-1 U1, then M <- M T^-T
  CKB(cublasDtrsm(ctx->blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N,
                  CUBLAS_DIAG_NON_UNIT, n, n, &one, T, n, M, n));
  CKB(cublasDtrsm(ctx->blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T,
                  CUBLAS_DIAG_NON_UNIT, n, n, &one, T, n, M, n));
  CK(symmetrize(M, n, 1, s));
  syevd(ctx, M, n, E);
  // v = T W (column-major), W = eigenvectors in M
  CKB(cublasDtrmm(ctx->blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N,
                  CUBLAS_DIAG_NON_UNIT, n, n, &one, T, n, M, n, W, n));
  // row-major v[p][k] = W_cm[p + k n]  ->  physical_block does exactly this transpose
  if (ldv == n) {
    CK(physical_block(W, n, n, n, v_rowmajor, s));
  } else {
    double* tmp = ws(ctx, "cmp_vrm", nn);
    CK(physical_block(W, n, n, n, tmp, s));
    CK(cudaMemcpy2DAsync(v_rowmajor, ldv * sizeof(double), tmp, n * sizeof(double),
                         n * sizeof(double), n, cudaMemcpyDeviceToDevice, s));
  }
  sync(ctx);
}

// Moment-conserving compression for nmom = 2m + 1 (the higher truncations of
// the compression text before Eq. post_compression_h): m + 1 steps of
// block Lanczos in the auxiliary space, driven by the moments U^(0..2m+1)
// alone.  The Lanczos vectors are kept as coefficient lists, Q_i =
// sum_k E^k V C_i[k] (V = v^T), so that Q_i^T E^s Q_j = sum_kl C_i[k]^T
// U^(k+l+s) C_j[l]:
//   U^(0) = B0 B0^T, C_0 = [B0^-T];  A_i = Q_i^T E Q_i;
//   R_i = E Q_i - Q_i A_i - Q_{i-1} B_{i-1}^T,  R_i^T R_i = B_i^T B_i (B_i
//   upper);  Q_{i+1} = R_i B_i^-1.
// The block-tridiagonal H (diagonal A_i, sub-diagonal B_i) of order (m+1) N
// is diagonalised, H = W diag(E) W^T, and the auxiliaries are
// (E, B0 W[:N]), which conserve U^(0..2m+1).  m = 0 is compress_impl.
// All matrices column-major; U^(n) symmetric, so its row-major array is its
// own column-major view.  Output v row-major [n][(m+1) n] with row stride ldv.
void compress_lanczos_impl(agf2_context* ctx, const double* U, int n, int nmom, double* E,
                           double* v_rowmajor, long long ldv) {
  const int m = (nmom - 1) / 2, nb = m + 1;
  if (m == 0) {
    compress_impl(ctx, U, n, E, v_rowmajor, ldv);
    return;
  }
  Range rg("agf2_compress");
  cudaStream_t s = ctx->stream;
  const long long nn = (long long)n * n;
  const int nh = nb * n;
  auto Um = [&](int k) { return U + (long long)k * nn; };
  double* B0 = ws(ctx, "lz_B0", nn);
  double* tmp = ws(ctx, "lz_tmp", nn);
  double* A = ws(ctx, "lz_A", nn);
  double* S = ws(ctx, "lz_S", nn);
  double* Bprev = ws(ctx, "lz_Bprev", nn);
  double* Bcur = ws(ctx, "lz_Bcur", nn);
  double* H = ws(ctx, "lz_H", (size_t)nh * nh);
  double* pool[3] = {ws(ctx, "lz_pool0", (size_t)(nb + 1) * nn),
                     ws(ctx, "lz_pool1", (size_t)(nb + 1) * nn),
                     ws(ctx, "lz_pool2", (size_t)(nb + 1) * nn)};
  const double one = 1.0, mone = -1.0, zero = 0.0;
  auto potrf = [&](double* X, const char* what) {
    int lwork = 0;
    CKS(cusolverDnDpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_LOWER, n, X, n, &lwork));
    double* work = ws(ctx, "potrf_work", (size_t)lwork);
    CKS(cusolverDnDpotrf(ctx->solver, CUBLAS_FILL_MODE_LOWER, n, X, n, work, lwork,
                         ctx->dev_info));
    int info = 0;
    CK(cudaMemcpyAsync(&info, ctx->dev_info, sizeof(int), cudaMemcpyDeviceToHost, s));
    sync(ctx);
    if (info != 0)
      fail(ctx, AGF2_ERR_NOT_PD,
           std::string(what) + " is not positive definite (potrf info " + std::to_string(info) +
               ")");
  };
  auto mat = [&](double* base, int k) { return base + (long long)k * nn; };
  // out = sum_kl Ci[k]^T U^(k+l+shift) Cj[l]
  auto mom = [&](double* Ci, int ni, double* Cj, int nj, int shift, double* out) {
    bool first = true;
    for (int k = 0; k < ni; ++k)
      for (int l = 0; l < nj; ++l) {
        CKB(cublasDgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, Um(k + l + shift), n,
                        mat(Cj, l), n, &zero, tmp, n));
        CKB(cublasDgemm(ctx->blas, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n, &one, mat(Ci, k), n, tmp,
                        n, first ? &zero : &one, out, n));
        first = false;
      }
    CK(symmetrize(out, n, 1, s));
  };
  CK(cudaMemcpyAsync(B0, Um(0), nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  potrf(B0, "U^(0)");
  double *Ccur = pool[0], *Cprev = pool[1], *CR = pool[2];
  int ncur = 1, nprev = 0;
  CK(set_identity(Ccur, n, 1.0, s));  // C_0 = B0^-T: solve B0^T X = I
  CKB(cublasDtrsm(ctx->blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T,
                  CUBLAS_DIAG_NON_UNIT, n, n, &one, B0, n, Ccur, n));
  CK(cudaMemsetAsync(H, 0, (size_t)nh * nh * sizeof(double), s));
  for (int i = 0; i <= m; ++i) {
    mom(Ccur, ncur, Ccur, ncur, 1, A);
    CK(cudaMemcpy2DAsync(H + (long long)i * n + (long long)i * n * nh, nh * sizeof(double), A,
                         n * sizeof(double), n * sizeof(double), n, cudaMemcpyDeviceToDevice, s));
    if (i == m) break;
    // R_i = E Q_i - Q_i A_i - Q_{i-1} B_{i-1}^T as coefficients CR[0..ncur]
    CK(cudaMemsetAsync(CR, 0, (size_t)(ncur + 1) * nn * sizeof(double), s));
    for (int k = 0; k < ncur; ++k) {
      CKB(cublasDaxpy(ctx->blas, (int)nn, &one, mat(Ccur, k), 1, mat(CR, k + 1), 1));
      CKB(cublasDgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &mone, mat(Ccur, k), n, A, n,
                      &one, mat(CR, k), n));
    }
    for (int k = 0; k < nprev; ++k)
      CKB(cublasDgemm(ctx->blas, CUBLAS_OP_N, CUBLAS_OP_T, n, n, n, &mone, mat(Cprev, k), n,
                      Bprev, n, &one, mat(CR, k), n));
    mom(CR, ncur + 1, CR, ncur + 1, 0, S);
    potrf(S, "R^T R of a Lanczos block");
    CK(upper_from_lower_t(S, n, Bcur, n, s));
    CK(upper_from_lower_t(S, n, H + (long long)(i + 1) * n + (long long)i * n * nh, nh, s));
    // Q_{i+1} = R_i B_i^-1: solve X B_i = CR[k]
    for (int k = 0; k <= ncur; ++k)
      CKB(cublasDtrsm(ctx->blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N,
                      CUBLAS_DIAG_NON_UNIT, n, n, &one, Bcur, n, mat(CR, k), n));
    std::swap(Bprev, Bcur);
    double* old = Cprev;
    Cprev = Ccur;
    Ccur = CR;
    CR = old;
    nprev = ncur;
    ncur += 1;
  }
  syevd(ctx, H, nh, E);
  // v = B0 W[:n, :]
  double* Vc = ws(ctx, "lz_V", (size_t)n * nh);
  CKB(cublasDtrmm(ctx->blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N,
                  CUBLAS_DIAG_NON_UNIT, n, nh, &one, B0, n, H, nh, Vc, n));
  if (ldv == nh) {
    CK(physical_block(Vc, n, n, nh, v_rowmajor, s));
  } else {
    double* vr = ws(ctx, "lz_vrm", (size_t)n * nh);
    CK(physical_block(Vc, n, n, nh, vr, s));
    CK(cudaMemcpy2DAsync(v_rowmajor, ldv * sizeof(double), vr, nh * sizeof(double),
                         nh * sizeof(double), n, cudaMemcpyDeviceToDevice, s));
  }
  sync(ctx);
}

// ---------------------------------------------------------------------------
// Extended Hamiltonian, chemical potential and the Fock loop
// ---------------------------------------------------------------------------
struct Eig {
  double* V;  // column-major eigenvectors [n][n]
  double* w;  // eigenvalues
  int n;
};

Eig diag_extended(agf2_context* ctx, const double* F, const double* E, const double* v, double delta,
                  int nmo, int nse) {
  const int n = nmo + nse;
  double* H = ws(ctx, "ext_H", (size_t)n * n);
  Eig r{ws(ctx, "ext_V", (size_t)n * n), ws(ctx, "ext_w", n), n};
  CK(build_extended_h(F, E, v, delta, nmo, nse, H, ctx->stream));
  if (!ctx->eig_ws) ctx->eig_ws = eig_workspace_create();
  {
    // algorithmic flops: tridiagonalisation 4/3 n^3, physical rows 2 nmo n^2
    // and their product with the tridiagonal eigenvectors 2 nmo n^2
    TimedRegion tr(ctx, 3, (4.0 / 3.0) * n * (double)n * n + 4.0 * nmo * (double)n * n);
    const int rc = eigh_phys(ctx->eig_ws, H, n, nmo, r.w, r.V, ctx->stream, ctx->err);
    if (rc != AGF2_OK) throw Fail{rc};
  }
  return r;
}

std::vector<double> pole_weights(agf2_context* ctx, const Eig& eg, int nmo) {
  double* wt = ws(ctx, "ext_wt", eg.n);
  CK(column_weights(eg.V, eg.n, nmo, eg.n, wt, ctx->stream));
  return to_host(ctx, wt, eg.n);
}

struct Aufbau {
  int k;
  double mu, n;
};

Aufbau aufbau(const std::vector<double>& e, const std::vector<double>& wt, int nelec) {
  const int n = (int)e.size();
  double cum = 0.0, best = std::fabs(0.0 - nelec);
  int k = 0;
  std::vector<double> c(n + 1, 0.0);
  for (int x = 0; x < n; ++x) {
    cum += 2.0 * wt[x];
    c[x + 1] = cum;
  }
  for (int x = 1; x <= n; ++x) {
    const double d = std::fabs(c[x] - nelec);
    if (d < best) { best = d; k = x; }
  }
  k = std::min(std::max(k, 1), n - 1);
  return Aufbau{k, 0.5 * (e[k - 1] + e[k]), c[k]};
}

double nelec_fixed_k(const std::vector<double>& wt, int k) {
  double s = 0.0;
  for (int x = 0; x < k; ++x) s += wt[x];
  return 2.0 * s;
}

struct Shift {
  double delta, nerr;
  int evals;
  bool converged;
  bool last_is_best;  // the extended-Hamiltonian buffers hold the decomposition at delta
};

// dn/d(delta) at fixed aufbau count k from one decomposition:
// 4 sum_{x<k<=y} (C_x . C_y)^2 / (e_y - e_x), C = physical rows of the eigenvectors.
double count_derivative(agf2_context* ctx, const Eig& eg, int k, int nmo, double* red) {
  const int n = eg.n, nv = n - k;
  double* S = ws(ctx, "sh_S", (size_t)k * nv);
  DGemm g;  // S[x][y] = sum_p V[x n + p] V[(k + y) n + p]
  g.M = k; g.N = nv; g.K = nmo;
  g.A = eg.V; g.sAm = n; g.sAk = 1;
  g.B = eg.V + (long long)k * n; g.sBk = 1; g.sBn = n;
  g.C = S; g.sCm = nv; g.sCn = 1;
  CK(dgemm(g, ctx->stream));
  CK(shift_derivative(S, eg.w, k, nv, red + 512, red, ctx->stream));
  return scalar(ctx, red + 512);
}

// Common shift of the auxiliary energies so that n(delta; k) = nelec, with k
// the aufbau count at delta = 0.  n is increasing in delta with
//   dn/d(delta) = 4 sum_{x<k<=y} (C_x . C_y)^2 / (e_y - e_x)
// (first-order perturbation of the eigenvectors by the auxiliary-space
// projector), so the root is found by Newton steps safeguarded by a bracket
// (bisection whenever a step leaves it, expanding steps until one exists).
// It converges to the same root as plain bisection, in a few
// eigendecompositions instead of ~40.
Shift solve_shift(agf2_context* ctx, const double* F, const double* E, const double* v, int nmo,
                  int nse, int nelec, double tol) {
  const int n = nmo + nse;
  int k = -1;
  double* red = ws(ctx, "sh_red", 1024);
  auto eval = [&](double d, double& fp) -> double {
    Eig eg = diag_extended(ctx, F, E, v, d, nmo, nse);
    std::vector<double> wt = pole_weights(ctx, eg, nmo);
    if (k < 0) {
      std::vector<double> ev = to_host(ctx, eg.w, n);
      k = aufbau(ev, wt, nelec).k;
    }
    fp = count_derivative(ctx, eg, k, nmo, red);
    return nelec_fixed_k(wt, k) - nelec;
  };
  double fp = 0.0;
  double d = 0.0;
  double f = eval(0.0, fp);
  int evals = 1;
  if (std::fabs(f) < tol) return Shift{0.0, f, evals, true, true};
  bool has_lo = false, has_hi = false;
  double lo = 0.0, hi = 0.0;
  auto bracket = [&](double x, double fx) {
    if (fx < 0) { if (!has_lo || x > lo) lo = x; has_lo = true; }
    else { if (!has_hi || x < hi) hi = x; has_hi = true; }
  };
  bracket(d, f);
  double best = d, fbest = f;
  bool last_best = true;
  double expand = 1.0;
  for (int it = 0; it < 200; ++it) {
    double dn = (fp > 0.0 && std::isfinite(fp)) ? d - f / fp : NAN;
    if (has_lo && has_hi) {
      if (!(dn > lo && dn < hi)) dn = 0.5 * (lo + hi);
    } else if (!std::isfinite(dn) || std::fabs(dn - d) > expand) {
      dn = d + (f < 0 ? expand : -expand);
      expand *= 2.0;
    }
    d = dn;
    f = eval(d, fp);
    ++evals;
    bracket(d, f);
    last_best = std::fabs(f) < std::fabs(fbest);
    if (last_best) { best = d; fbest = f; }
    if (std::fabs(f) < tol) break;
    if (has_lo && has_hi && hi - lo < 1e-14) break;
    if (!has_lo || !has_hi) {
      if (expand > 1e6) break;
    }
  }
  return Shift{best, fbest, evals, std::fabs(fbest) < tol, last_best};
}

// Pulay extrapolation coefficients from B_ab = <r_a, r_b> (host solve of the
// bordered (m+1)x(m+1) system by Gaussian elimination with partial pivoting).
std::vector<double> diis_coeffs(const std::vector<double>& B, int m) {
  const int n = m + 1;
  std::vector<double> A((size_t)n * n, 0.0), b(n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[i * n + j] = B[i * m + j];
  for (int i = 0; i < m; ++i) { A[m * n + i] = 1.0; A[i * n + m] = 1.0; }
  b[m] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
    if (p != c) {
      for (int j = 0; j < n; ++j) std::swap(A[c * n + j], A[p * n + j]);
      std::swap(b[c], b[p]);
    }
    const double piv = A[c * n + c];
    if (piv == 0.0) continue;
    for (int r = c + 1; r < n; ++r) {
      const double f = A[r * n + c] / piv;
      if (f == 0.0) continue;
      for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
      b[r] -= f * b[c];
    }
  }
  std::vector<double> x(n, 0.0);
  for (int r = n - 1; r >= 0; --r) {
    double sacc = b[r];
    for (int j = r + 1; j < n; ++j) sacc -= A[r * n + j] * x[j];
    x[r] = A[r * n + r] != 0.0 ? sacc / A[r * n + r] : 0.0;
  }
  x.resize(m);
  return x;
}

struct FockOut {
  int cycles, converged, k, evals;
  double mu, nerr;
};

bool trace_on() {
  static int on = -1;
  if (on < 0) {
    const char* v = std::getenv("AGF2_TRACE");
    on = (v && v[0] && v[0] != '0') ? 1 : 0;
  }
  return on == 1;
}

// Fock loop: see agf2_fock_loop in agf2.h.  F_in holds the initial F[D] on
// entry; on exit D, F (= F[D]), e_qmo, C_qmo are written.
FockOut fock_loop_impl(agf2_context* ctx, const double* h, const double* L, int naux, int nmo,
                       int nelec, double* E, const double* v, int nse, double* D, double* F,
                       double* e_qmo, double* C_qmo, const agf2_fock_opts& o) {
  Range rg("agf2_fock_loop");
  cudaStream_t s = ctx->stream;
  const int n = nmo + nse;
  const long long nn = (long long)nmo * nmo;
  const int space = std::max(0, o.diis_space);
  double* Fin = ws(ctx, "fl_Fin", nn);
  double* Fout = ws(ctx, "fl_Fout", nn);
  double* Dn = ws(ctx, "fl_Dnew", nn);
  double* Cphys = ws(ctx, "fl_Cphys", (size_t)nmo * n);
  double* hF = ws(ctx, "fl_histF", (size_t)std::max(space, 1) * nn);
  double* hR = ws(ctx, "fl_histR", (size_t)std::max(space, 1) * nn);
  double* red = ws(ctx, "fl_red", 1024);
  double* dots = ws(ctx, "fl_dots", 64);
  CK(cudaMemcpyAsync(Fin, F, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int nh = 0, head = 0;  // ring buffer of history entries
  std::vector<int> order;
  FockOut out{0, 0, 0, 0, 0.0, 0.0};
  const bool tr = trace_on();
  for (int cyc = 1; cyc <= o.max_cycle; ++cyc) {
    out.cycles = cyc;
    auto tc0 = std::chrono::steady_clock::now();
    Shift sh{0.0, 0.0, 0, true, false};
    double joint_step = 0.0;
    Eig eg;
    if (o.shift_mode == 1) {
      // one decomposition per cycle; delta follows by one safeguarded Newton step
      eg = diag_extended(ctx, Fin, E, v, 0.0, nmo, nse);
      sh.evals = 1;
    } else {
      sh = solve_shift(ctx, Fin, E, v, nmo, nse, nelec, o.shift_tol);
      CK(add_scalar(E, sh.delta, nse, s));
      // the shift solve's last decomposition is the one at the chosen delta
      eg = sh.last_is_best ? Eig{ws(ctx, "ext_V", (size_t)n * n), ws(ctx, "ext_w", n), n}
                           : diag_extended(ctx, Fin, E, v, 0.0, nmo, nse);
    }
    const double t_shift = seconds_since(tc0);
    out.evals += sh.evals;
    std::vector<double> wt = pole_weights(ctx, eg, nmo);
    std::vector<double> ev = to_host(ctx, eg.w, n);
    Aufbau ab = aufbau(ev, wt, nelec);
    if (o.shift_mode == 1) {
      sh.nerr = ab.n - nelec;
      if (std::fabs(sh.nerr) >= o.shift_tol) {
        const double fp = count_derivative(ctx, eg, ab.k, nmo, red);
        const double lim = 4.0;
        joint_step = (fp > 0.0 && std::isfinite(fp)) ? -sh.nerr / fp : 0.0;
        joint_step = std::max(-lim, std::min(lim, joint_step));
      }
      sh.delta = joint_step;
    }
    out.nerr = sh.nerr;
    out.k = ab.k;
    out.mu = ab.mu;
    CK(physical_block(eg.V, n, nmo, n, Cphys, s));  // Cphys[p][x]
    CK(cudaMemcpyAsync(e_qmo, eg.w, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(C_qmo, Cphys, (size_t)nmo * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // occupied block Cocc[p][x<k] = Cphys with leading dimension n
    double* Cocc = ws(ctx, "fl_Cocc", (size_t)nmo * ab.k);
    CK(cudaMemcpy2DAsync(Cocc, ab.k * sizeof(double), Cphys, n * sizeof(double),
                         ab.k * sizeof(double), nmo, cudaMemcpyDeviceToDevice, s));
    {
      DGemm g;  // D_new = 2 Cocc Cocc^T
      g.M = nmo; g.N = nmo; g.K = ab.k;
      g.A = Cocc; g.sAm = ab.k; g.sAk = 1;
      g.B = Cocc; g.sBk = 1; g.sBn = ab.k;
      g.C = Dn; g.sCm = nmo; g.sCn = 1;
      g.alpha = 2.0;
      CK(dgemm(g, s));
    }
    auto tf0 = std::chrono::steady_clock::now();
    fock_density(ctx, h, L, naux, nmo, Dn, Cocc, ab.k, Fout);
    CK(max_abs_diff(Dn, D, nn, red + 512, red, s));
    const double dD = scalar(ctx, red + 512);
    if (tr)
      std::fprintf(stderr, "[agf2] fock cycle %d: shift evals %d (%.1f ms) delta %.3e nerr %.2e k %d "
                           "dD %.3e fock build %.1f ms cycle %.1f ms\n",
                   cyc, sh.evals, 1e3 * t_shift, sh.delta, sh.nerr, ab.k, dD,
                   1e3 * seconds_since(tf0), 1e3 * seconds_since(tc0));
    CK(cudaMemcpyAsync(D, Dn, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (dD < o.tol_D && std::fabs(out.nerr) < o.shift_tol) {
      out.converged = 1;
      break;
    }
    if (joint_step != 0.0) CK(add_scalar(E, joint_step, nse, s));
    if (cyc >= o.diis_start && space > 1) {
      // new entry (F_in, F_out - F_in) into the ring
      const int slot = (nh < space) ? nh : head;
      CK(cudaMemcpyAsync(hF + slot * nn, Fin, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(hR + slot * nn, Fout, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CK(axpby(hR + slot * nn, Fin, -1.0, 1.0, nn, s));
      if (nh < space) { order.push_back(slot); ++nh; }
      else { order.erase(order.begin()); order.push_back(slot); head = (head + 1) % space; }
    }
    if (nh > 1) {
      const int m = nh;
      for (int a = 0; a < m; ++a)
        for (int b = a; b < m; ++b)
          CK(dot(hR + order[a] * nn, hR + order[b] * nn, nn, dots + a * m + b, red, s));
      std::vector<double> Bh = to_host(ctx, dots, (size_t)m * m);
      for (int a = 0; a < m; ++a)
        for (int b = 0; b < a; ++b) Bh[a * m + b] = Bh[b * m + a];
      std::vector<double> c = diis_coeffs(Bh, m);
      CK(cudaMemsetAsync(Fin, 0, nn * sizeof(double), s));
      for (int a = 0; a < m; ++a) {
        CK(axpby(Fin, hF + order[a] * nn, c[a], 1.0, nn, s));
        CK(axpby(Fin, hR + order[a] * nn, c[a], 1.0, nn, s));
      }
    } else {
      // F_in <- F_in + damping (F_out - F_in)
      CK(axpby(Fin, Fout, o.damping, 1.0 - o.damping, nn, s));
    }
  }
  fock_density(ctx, h, L, naux, nmo, D, ws(ctx, "fl_Cocc", 1), out.k, F);
  sync(ctx);
  return out;
}

agf2_fock_opts fock_defaults() {
  agf2_fock_opts o;
  o.tol_D = 1e-10;
  o.max_cycle = 50;
  o.shift_tol = 1e-11;
  o.damping = 0.3;
  o.diis_start = 10;
  o.diis_space = 6;
  o.shift_mode = 1;
  return o;
}

template <class Fn>
int guarded(agf2_handle h, Fn&& fn) {
  if (!h) return AGF2_ERR_INVALID_ARG;
  agf2_context* ctx = h;
  ctx->err.clear();
  try {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) fail(ctx, AGF2_ERR_CUDA, cudaGetErrorString(e));
    fn(ctx);
    return AGF2_OK;
  } catch (const Fail& f) {
    return f.code;
  } catch (const std::exception& ex) {
    ctx->err = ex.what();
    return AGF2_ERR_CUDA;
  } catch (...) {
    ctx->err = "unknown exception";
    return AGF2_ERR_CUDA;
  }
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int agf2_create(agf2_handle* out, int device) {
  if (!out) return AGF2_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return AGF2_ERR_INVALID_ARG;
  }
  auto* ctx = new agf2_context();
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return AGF2_ERR_CUDA; }
  if (cusolverDnCreate(&ctx->solver) != CUSOLVER_STATUS_SUCCESS) { delete ctx; return AGF2_ERR_CUDA; }
  if (cublasCreate(&ctx->blas) != CUBLAS_STATUS_SUCCESS) {
    cusolverDnDestroy(ctx->solver);
    delete ctx;
    return AGF2_ERR_CUDA;
  }
  if (cudaMalloc(&ctx->dev_info, sizeof(int)) != cudaSuccess) {
    cublasDestroy(ctx->blas);
    cusolverDnDestroy(ctx->solver);
    delete ctx;
    return AGF2_ERR_OOM;
  }
  cusolverDnSetStream(ctx->solver, ctx->stream);
  cublasSetStream(ctx->blas, ctx->stream);
  *out = ctx;
  return AGF2_OK;
}

int agf2_destroy(agf2_handle h) {
  if (!h) return AGF2_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& kv : h->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  mixed_workspace_destroy(h->mixed_ws);
  eig_workspace_destroy(h->eig_ws);
  for (auto& p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  if (h->dev_info) cudaFree(h->dev_info);
  if (h->blas) cublasDestroy(h->blas);
  if (h->solver) cusolverDnDestroy(h->solver);
  delete h;
  return AGF2_OK;
}

int agf2_set_stream(agf2_handle h, void* stream) {
  return guarded(h, [&](agf2_context* ctx) {
    ctx->stream = static_cast<cudaStream_t>(stream);
    CKS(cusolverDnSetStream(ctx->solver, ctx->stream));
    CKB(cublasSetStream(ctx->blas, ctx->stream));
  });
}

const char* agf2_last_error(agf2_handle h) { return h ? h->err.c_str() : "null handle"; }

void agf2_fock_opts_default(agf2_fock_opts* o) {
  if (o) *o = fock_defaults();
}

void agf2_opts_default(agf2_opts* o) {
  if (!o) return;
  o->max_iter = 50;
  o->conv_tol = 1e-8;
  o->nmom = 1;
  o->precision = AGF2_FP64;
  o->mix = 1.0;
  o->resume = 0;
  o->fock = fock_defaults();
}

int agf2_hcore_from_mo_energies(agf2_handle h, const double* L, int naux, int nmo,
                                const double* eps, int nocc, double* hcore) {
  return guarded(h, [&](agf2_context* ctx) {
    if (naux < 1 || nmo < 2 || nocc < 1 || nocc >= nmo)
      fail(ctx, AGF2_ERR_INVALID_ARG, "need naux >= 1 and 0 < nocc < nmo");
    check_dev_ptr(ctx, L, "L");
    check_dev_ptr(ctx, eps, "eps");
    check_dev_ptr(ctx, hcore, "hcore");
    cudaStream_t s = ctx->stream;
    const long long nn = (long long)nmo * nmo;
    double* D0 = ws(ctx, "hc_D0", nn);
    double* Z = ws(ctx, "hc_zero", nn);
    double* F = ws(ctx, "hc_F", nn);
    std::vector<double> d(nmo, 0.0);
    for (int i = 0; i < nocc; ++i) d[i] = 2.0;
    double* dv = ws(ctx, "hc_d", nmo);
    CK(cudaMemcpyAsync(dv, d.data(), nmo * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(diag_from_vec(dv, nmo, D0, s));
    CK(cudaMemsetAsync(Z, 0, nn * sizeof(double), s));
    fock_general(ctx, Z, L, naux, nmo, D0, F);  // F = J - K/2
    CK(diag_from_vec(eps, nmo, hcore, s));
    CK(axpby(hcore, F, -1.0, 1.0, nn, s));
    sync(ctx);
  });
}

int agf2_build_moments(agf2_handle h, const double* L, int naux, int nmo, const double* e,
                       const double* C, int nqmo, double mu, int nmom, int precision,
                       double* U_hole, double* U_part) {
  return guarded(h, [&](agf2_context* ctx) {
    if (naux < 1 || nmo < 1 || nqmo < 2 || nmom < 1)
      fail(ctx, AGF2_ERR_INVALID_ARG, "bad sizes");
    if (precision != AGF2_FP64 && precision != AGF2_BF16X3)
      fail(ctx, AGF2_ERR_INVALID_ARG, "unknown precision");
    if (precision == AGF2_BF16X3 && nmom > 3)
      fail(ctx, AGF2_ERR_UNSUPPORTED, "AGF2_BF16X3 supports nmom <= 3");
    check_dev_ptr(ctx, L, "L");
    check_dev_ptr(ctx, e, "e");
    check_dev_ptr(ctx, C, "C");
    check_dev_ptr(ctx, U_hole, "U_hole");
    check_dev_ptr(ctx, U_part, "U_part");
    build_moments_impl(ctx, L, naux, nmo, e, C, nqmo, mu, nmom, precision, U_hole, U_part);
  });
}

int agf2_compress(agf2_handle h, const double* U, int nmo, double* E_aux, double* v_aux) {
  return guarded(h, [&](agf2_context* ctx) {
    if (nmo < 1) fail(ctx, AGF2_ERR_INVALID_ARG, "nmo < 1");
    check_dev_ptr(ctx, U, "U");
    check_dev_ptr(ctx, E_aux, "E_aux");
    check_dev_ptr(ctx, v_aux, "v_aux");
    compress_impl(ctx, U, nmo, E_aux, v_aux, nmo);
  });
}

int agf2_compress_moments(agf2_handle h, const double* U, int nmo, int nmom, double* E_aux,
                          double* v_aux) {
  return guarded(h, [&](agf2_context* ctx) {
    if (nmo < 1) fail(ctx, AGF2_ERR_INVALID_ARG, "nmo < 1");
    if (nmom < 1 || nmom % 2 == 0) fail(ctx, AGF2_ERR_INVALID_ARG, "nmom must be odd (2m+1)");
    check_dev_ptr(ctx, U, "U");
    check_dev_ptr(ctx, E_aux, "E_aux");
    check_dev_ptr(ctx, v_aux, "v_aux");
    compress_lanczos_impl(ctx, U, nmo, nmom, E_aux, v_aux, (long long)(nmom + 1) / 2 * nmo);
  });
}

int agf2_eigh_physical(agf2_handle h, const double* A, int n, int nphys, double* w, double* V) {
  return guarded(h, [&](agf2_context* ctx) {
    if (n < 1 || nphys < 1 || nphys > n) fail(ctx, AGF2_ERR_INVALID_ARG, "need 1 <= nphys <= n");
    check_dev_ptr(ctx, A, "A");
    check_dev_ptr(ctx, w, "w");
    check_dev_ptr(ctx, V, "V");
    if (!ctx->eig_ws) ctx->eig_ws = eig_workspace_create();
    const int rc = eigh_phys(ctx->eig_ws, A, n, nphys, w, V, ctx->stream, ctx->err);
    if (rc != AGF2_OK) throw Fail{rc};
  });
}

int agf2_fock_loop(agf2_handle h, const double* hcore, const double* L, int naux, int nmo,
                   int nelec, double* E_se, const double* v_se, int nse, double* D, double* F,
                   double* e_qmo, double* C_qmo, const agf2_fock_opts* opts,
                   agf2_fock_info* info) {
  int rc_conv = AGF2_OK;
  int rc = guarded(h, [&](agf2_context* ctx) {
    if (naux < 1 || nmo < 1 || nse < 0 || nelec < 1 || nelec > 2 * (nmo + nse))
      fail(ctx, AGF2_ERR_INVALID_ARG, "bad sizes");
    if (nmo + nse > 7000)
      fail(ctx, AGF2_ERR_INVALID_ARG, "nmo + nse > 7000: beyond the extended-Hamiltonian eigensolver");
    for (auto p : {(const void*)hcore, (const void*)L, (const void*)E_se, (const void*)v_se,
                   (const void*)D, (const void*)F, (const void*)e_qmo, (const void*)C_qmo})
      check_dev_ptr(ctx, p, "argument");
    agf2_fock_opts o = opts ? *opts : fock_defaults();
    if (o.max_cycle < 1) fail(ctx, AGF2_ERR_INVALID_ARG, "max_cycle < 1");
    fock_general(ctx, hcore, L, naux, nmo, D, F);
    FockOut fo = fock_loop_impl(ctx, hcore, L, naux, nmo, nelec, E_se, v_se, nse, D, F, e_qmo,
                                C_qmo, o);
    if (info) {
      info->cycles = fo.cycles;
      info->converged = fo.converged;
      info->nocc_qmo = fo.k;
      info->shift_evals = fo.evals;
      info->nerr = fo.nerr;
      info->mu = fo.mu;
    }
    if (!fo.converged) rc_conv = AGF2_ERR_NO_CONVERGENCE;
  });
  return rc != AGF2_OK ? rc : rc_conv;
}

int agf2_run(agf2_handle h, const double* hcore, const double* L, int naux, int nmo, int nelec,
             const double* D0_in, const agf2_opts* opts, agf2_result* out) {
  int rc_conv = AGF2_OK;
  int rc = guarded(h, [&](agf2_context* ctx) {
    if (!out) fail(ctx, AGF2_ERR_INVALID_ARG, "out is NULL");
    agf2_opts o;
    agf2_opts_default(&o);
    if (opts) o = *opts;
    if (naux < 1 || nmo < 2 || nelec < 2 || nelec % 2 || nelec >= 2 * nmo || o.max_iter < 1)
      fail(ctx, AGF2_ERR_INVALID_ARG, "bad sizes or options");
    if (o.nmom < 1 || o.nmom % 2 == 0)
      fail(ctx, AGF2_ERR_INVALID_ARG, "nmom must be odd (AGF2(m,0) uses nmom = 2m+1)");
    if (o.precision == AGF2_BF16X3 && o.nmom > 3)
      fail(ctx, AGF2_ERR_UNSUPPORTED, "AGF2_BF16X3 supports nmom <= 3");
    if ((long long)nmo * (o.nmom + 2) > 7000)
      fail(ctx, AGF2_ERR_INVALID_ARG,
           "nmo (nmom + 2) > 7000: beyond the extended-Hamiltonian eigensolver");
    check_dev_ptr(ctx, hcore, "hcore");
    check_dev_ptr(ctx, L, "L");
    cudaStream_t s = ctx->stream;
    const int nm = o.nmom + 1;          // moments per sector
    const int nb = nm / 2;              // auxiliaries per sector = nb * nmo
    const int N = nmo, nse = 2 * nb * nmo, nq_max = nmo + nse;
    const long long NN = (long long)N * N;
    double* e = ws(ctx, "st_e", nq_max);
    double* C = ws(ctx, "st_C", (size_t)N * nq_max);
    double* D = ws(ctx, "st_D", NN);
    double* F = ws(ctx, "st_F", NN);
    double* U = ws(ctx, "st_U", 2 * nm * NN);
    double* Uprev = ws(ctx, "st_Uprev", 2 * nm * NN);
    double* Ese = ws(ctx, "st_Ese", nse);
    double* vse = ws(ctx, "st_vse", (size_t)N * nse);
    double* eq = ws(ctx, "st_eq", nq_max);
    double* Cq = ws(ctx, "st_Cq", (size_t)N * nq_max);
    double* red = ws(ctx, "st_red", 1024);
    double* V = ws(ctx, "st_V", (size_t)nq_max * nb * N);
    const int nocc = nelec / 2;
    if (!o.resume || !ctx->have_state || ctx->nmo != N || ctx->nq_max != nq_max) {
      // reference density: the caller's, else the aufbau density of the first
      // nocc basis functions (the reference's canonical orbitals as basis)
      if (D0_in) {
        check_dev_ptr(ctx, D0_in, "D0");
        CK(cudaMemcpyAsync(D, D0_in, NN * sizeof(double), cudaMemcpyDeviceToDevice, s));
      } else {
        std::vector<double> d(N, 0.0);
        for (int i = 0; i < nocc; ++i) d[i] = 2.0;
        double* dv = ws(ctx, "st_d0", N);
        CK(cudaMemcpyAsync(dv, d.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(diag_from_vec(dv, N, D, s));
      }
      fock_general(ctx, hcore, L, naux, N, D, F);
      // initial Green's function: the mean-field poles e = eig(F[D0]) with the
      // eigenvectors as couplings C (Eq. gf_hf in the given basis)
      {
        if (!ctx->eig_ws) ctx->eig_ws = eig_workspace_create();
        double* V0 = ws(ctx, "st_V0", NN);
        const int rc = eigh_phys(ctx->eig_ws, F, N, N, e, V0, s, ctx->err);
        if (rc != AGF2_OK) throw Fail{rc};
        CK(physical_block(V0, N, N, N, C, s));  // C[p][x] = V0[x N + p]
      }
      std::vector<double> e0 = to_host(ctx, e, N);
      CK(dot(D, hcore, NN, red + 512, red, s));
      CK(dot(D, F, NN, red + 513, red, s));
      std::vector<double> tr = to_host(ctx, red + 512, 2);
      ctx->E_hf = 0.5 * (tr[0] + tr[1]);
      ctx->E_prev = ctx->E_hf;
      ctx->mu = 0.5 * (e0[nocc - 1] + e0[nocc]);
      ctx->nq = N;
      ctx->nmo = N;
      ctx->nq_max = nq_max;
      ctx->have_uprev = false;
      ctx->have_state = true;
      ctx->iter = 0;
    }
    std::memset(out, 0, sizeof(*out));
    out->E_hf = ctx->E_hf;
    bool conv = false;
    int it = 0;
    for (it = 1; it <= o.max_iter; ++it) {
      auto t0 = std::chrono::steady_clock::now();
      {
        PoleSplit ps = split_poles(ctx, e, ctx->nq, ctx->mu);
        out->flops_moments += (double)N * ps.o * ps.v * (double)(ps.o + ps.v) *
                              (2.0 * naux + 2.0 * (o.nmom + 1) * N);
      }
      build_moments_impl(ctx, L, naux, N, e, C, ctx->nq, ctx->mu, o.nmom, o.precision, U,
                         U + nm * NN);
      out->t_moments += seconds_since(t0);
      t0 = std::chrono::steady_clock::now();
      ctx->iter += 1;
      if (ctx->have_uprev) CK(axpby(U, Uprev, 1.0 - o.mix, o.mix, 2 * nm * NN, s));
      CK(cudaMemcpyAsync(Uprev, U, 2 * nm * NN * sizeof(double), cudaMemcpyDeviceToDevice, s));
      ctx->have_uprev = true;
      // hole auxiliaries first, then particle ones, nb * N each
      compress_lanczos_impl(ctx, U, N, o.nmom, Ese, vse, nse);
      compress_lanczos_impl(ctx, U + nm * NN, N, o.nmom, Ese + nb * N, vse + nb * N, nse);
      out->t_compress += seconds_since(t0);
      t0 = std::chrono::steady_clock::now();
      FockOut fo = fock_loop_impl(ctx, hcore, L, naux, N, nelec, Ese, vse, nse, D, F, eq, Cq, o.fock);
      out->t_fock += seconds_since(t0);
      t0 = std::chrono::steady_clock::now();
      CK(cudaMemcpyAsync(e, eq, nq_max * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(C, Cq, (size_t)N * nq_max * sizeof(double), cudaMemcpyDeviceToDevice, s));
      ctx->nq = nq_max;
      ctx->mu = fo.mu;
      const int k = fo.k;
      // energies
      CK(dot(D, hcore, NN, red + 512, red, s));
      CK(dot(D, F, NN, red + 513, red, s));
      {
        DGemm g;  // V[x][m] = sum_p C[p][x] v_>[p][m], m over the nb N particle auxiliaries
        g.M = k; g.N = nb * N; g.K = N;
        g.A = C; g.sAm = 1; g.sAk = nq_max;
        g.B = vse + nb * N; g.sBk = nse; g.sBn = 1;
        g.C = V; g.sCm = nb * N; g.sCn = 1;
        CK(dgemm(g, s));
      }
      CK(gm_energy(V, e, Ese + nb * N, k, nb * N, red + 514, red, s));
      std::vector<double> sc = to_host(ctx, red + 512, 3);
      std::vector<double> eh = to_host(ctx, e, nq_max);
      const double E1 = 0.5 * (sc[0] + sc[1]);
      const double E2 = sc[2];
      const double Et = E1 + E2;
      out->E_1b = E1;
      out->E_2b = E2;
      out->E_tot = Et;
      out->ip = -eh[k - 1];
      out->ea = -eh[k];
      out->mu = fo.mu;
      out->nocc_qmo = k;
      out->fock_cycles = fo.cycles;
      out->fock_converged = fo.converged;
      out->fock_cycles_total += fo.cycles;
      out->t_energy += seconds_since(t0);
      const double dE = std::fabs(Et - ctx->E_prev);
      ctx->E_prev = Et;
      if (dE < o.conv_tol) {
        conv = true;
        break;
      }
    }
    out->iterations = std::min(it, o.max_iter);
    out->converged = conv ? 1 : 0;
    if (!conv && o.max_iter > 1) rc_conv = AGF2_ERR_NO_CONVERGENCE;
  });
  return rc != AGF2_OK ? rc : rc_conv;
}

int agf2_spectral_function(agf2_handle h, const double* e, const double* C, int nmo, int nqmo,
                           const double* omega, int nomega, double eta, double* A_total,
                           double* A_orb) {
  return guarded(h, [&](agf2_context* ctx) {
    if (nmo < 1 || nqmo < 1 || nomega < 1 || !(eta > 0.0))
      fail(ctx, AGF2_ERR_INVALID_ARG, "need nmo, nqmo, nomega >= 1 and eta > 0");
    check_dev_ptr(ctx, e, "e");
    check_dev_ptr(ctx, C, "C");
    check_dev_ptr(ctx, omega, "omega");
    check_dev_ptr(ctx, A_total, "A_total");
    if (A_orb) check_dev_ptr(ctx, A_orb, "A_orb");
    cudaStream_t s = ctx->stream;
    double* lor = ws(ctx, "sp_lor", (size_t)nqmo * nomega);
    double* w2 = ws(ctx, "sp_w2", (size_t)nmo * nqmo);
    double* orb = A_orb ? A_orb : ws(ctx, "sp_orb", (size_t)nmo * nomega);
    CK(lorentzian(e, nqmo, omega, nomega, eta, lor, s));
    CK(square(C, (long long)nmo * nqmo, w2, s));
    DGemm g;  // A_orb[p][w] = sum_x C[p][x]^2 lor[x][w]
    g.M = nmo; g.N = nomega; g.K = nqmo;
    g.A = w2; g.sAm = nqmo; g.sAk = 1;
    g.B = lor; g.sBk = nomega; g.sBn = 1;
    g.C = orb; g.sCm = nomega; g.sCn = 1;
    CK(dgemm(g, s));
    CK(column_sum(orb, nmo, nomega, A_total, s));
    sync(ctx);
  });
}

int agf2_set_profiling(agf2_handle h, int enable) {
  return guarded(h, [&](agf2_context* ctx) {
    sync(ctx);
    ctx->stats = KernelStats();
    ctx->stats.enabled = enable != 0;
  });
}

int agf2_kernel_stats(agf2_handle h, int kind, long long* launches, double* ms, double* flops) {
  return guarded(h, [&](agf2_context* ctx) {
    if (kind < 0 || kind >= KernelStats::kKinds) fail(ctx, AGF2_ERR_INVALID_ARG, "kind must be 0..3");
    if (launches) *launches = ctx->stats.launches[kind];
    if (ms) *ms = ctx->stats.ms[kind];
    if (flops) *flops = ctx->stats.flops[kind];
  });
}

long long agf2_launch_count(void) { return launch_count(); }

int agf2_run_batched(agf2_handle h, int nsys, const agf2_system* systems, const agf2_opts* opts,
                     int nworkers, agf2_result* out, int* status) {
  if (!h) return AGF2_ERR_INVALID_ARG;
  h->err.clear();
  if (nsys < 0 || (nsys > 0 && (!systems || !out))) {
    h->err = "bad batch arguments";
    return AGF2_ERR_INVALID_ARG;
  }
  if (nsys == 0) return AGF2_OK;
  const int nw = std::max(1, std::min(nworkers > 0 ? nworkers : 8, nsys));
  std::vector<int> st(nsys, AGF2_OK);
  std::vector<std::string> msg(nsys);
  std::atomic<int> next{0};
  std::vector<int> worker_rc(nw, AGF2_OK);
  auto work = [&](int wi) {
    if (cudaSetDevice(h->device) != cudaSuccess) { worker_rc[wi] = AGF2_ERR_CUDA; return; }
    agf2_handle w = nullptr;
    cudaStream_t stream = nullptr;
    if (agf2_create(&w, h->device) != AGF2_OK ||
        cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
        agf2_set_stream(w, stream) != AGF2_OK) {
      cudaGetLastError();
      worker_rc[wi] = AGF2_ERR_CUDA;
      if (w) agf2_destroy(w);
      if (stream) cudaStreamDestroy(stream);
      return;
    }
    for (int i = next.fetch_add(1); i < nsys; i = next.fetch_add(1)) {
      const agf2_system& sy = systems[i];
      agf2_opts o;
      agf2_opts_default(&o);
      if (opts) o = *opts;
      o.resume = 0;
      st[i] = agf2_run(w, sy.hcore, sy.L, sy.naux, sy.nmo, sy.nelec, sy.D0, &o, &out[i]);
      if (st[i] != AGF2_OK) msg[i] = agf2_last_error(w);
    }
    agf2_destroy(w);
    cudaStreamDestroy(stream);
  };
  std::vector<std::thread> threads;
  for (int wi = 0; wi < nw; ++wi) threads.emplace_back(work, wi);
  for (auto& t : threads) t.join();
  int rc = AGF2_OK;
  for (int wi = 0; wi < nw; ++wi)
    if (worker_rc[wi] != AGF2_OK) { rc = worker_rc[wi]; h->err = "batch worker set-up failed"; }
  for (int i = 0; i < nsys; ++i) {
    if (status) status[i] = st[i];
    if (st[i] != AGF2_OK && st[i] != AGF2_ERR_NO_CONVERGENCE && rc == AGF2_OK) {
      rc = st[i];
      h->err = "system " + std::to_string(i) + ": " + msg[i];
    }
  }
  return rc;
}

int agf2_get_state(agf2_handle h, double* e, double* C, double* D, int* nqmo) {
  return guarded(h, [&](agf2_context* ctx) {
    if (!ctx->have_state) fail(ctx, AGF2_ERR_INVALID_ARG, "no state: call agf2_run first");
    const int N = ctx->nmo, nq = ctx->nq, nq_max = ctx->nq_max;
    cudaStream_t s = ctx->stream;
    if (nqmo) *nqmo = nq;
    if (e) CK(cudaMemcpyAsync(e, ws(ctx, "st_e", nq_max), nq * sizeof(double),
                              cudaMemcpyDeviceToDevice, s));
    if (C) {
      // state C has leading dimension nq_max once iterations ran, N before
      const int ld = (nq == N) ? N : nq_max;
      CK(cudaMemcpy2DAsync(C, nq * sizeof(double), ws(ctx, "st_C", (size_t)N * nq_max),
                           ld * sizeof(double), nq * sizeof(double), N, cudaMemcpyDeviceToDevice, s));
    }
    if (D) CK(cudaMemcpyAsync(D, ws(ctx, "st_D", (size_t)N * N), (size_t)N * N * sizeof(double),
                              cudaMemcpyDeviceToDevice, s));
    sync(ctx);
  });
}

}  // extern "C"
