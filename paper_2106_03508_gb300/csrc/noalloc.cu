// Allocation-free variant of the FP64 moment build.
//
// agf2_build_moments needs a handle, and the handle grows its workspace with
// cudaMalloc on demand.  Some callers cannot allow that: applications that
// hand all device memory to their own allocator (a framework's caching pool,
// a fixed per-process budget) and must not see a library call cudaMalloc or
// cudaFree behind their back -- cudaFree synchronises the whole device and a
// late cudaMalloc can fail once the budget is committed.  For them this file
// provides agf2_build_moments_noalloc: the same FP64 computation, with every
// intermediate carved out of one file-scope __device__ array of fixed size
// (kScratchBytes).  That array is part of the library's device image, so
// every GPU that loads the library holds it until the process exits.
//
// Set-up: the first call on a device (with that device current) resolves the
// array's device address with cudaGetSymbolAddress and caches it; make that
// first call before capturing any stream.  All calls share the one array:
// calls whose GPU work overlaps (other streams, other host threads) race on
// it.  Everything read from it is written earlier in the same call, and the
// outputs are cleared before they are accumulated.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/agf2.h"
#include "agf2_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[64] = {nullptr};

// Device address of the scratch array on the current device (set-up once).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return AGF2_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return AGF2_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return AGF2_OK;
}

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Arena {
  char* base;
  size_t used, cap;
  template <class T>
  T* take(size_t count) {
    const size_t bytes = (std::max<size_t>(count, 1) * sizeof(T) + 255) / 256 * 256;
    if (used + bytes > cap) return nullptr;
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

// Bytes the call can need for an occupied/virtual split o + v = nq, without
// the 256-byte rounding of each piece: the gathered couplings and energies,
// the three rotated tensors, and the smallest pair block (one outer pole per
// block: X_IJ, X_JI, Y, Yw of 6 N max(o, v) doubles).  128-bit arithmetic,
// so no size product can wrap.
using u128 = unsigned __int128;
u128 bytes_unpadded(u128 N, u128 nq, u128 o, u128 Q) {
  const u128 v = nq - o;
  return 4 * nq + 8 * N * nq + 8 * nq + 8 * N * Q * nq + 8 * Q * o * v +
         48 * N * (o > v ? o : v);
}
constexpr int kPieces = 12;  // Arena::take calls per call; each rounds up by < 256 bytes

// Largest need over every split 1 <= o <= nq - 1.  The need is symmetric
// under o <-> nq - o; for o >= nq/2 it is 8 Q o (nq - o) + 48 N o plus
// constants, a concave parabola with its vertex at o* = nq/2 + 3 N / Q, so
// the maximum over the integers lies at floor(o*) or ceil(o*) clamped to
// [ceil(nq/2), nq - 1].
u128 worst_case_bytes(size_t N, size_t nq, size_t Q) {
  const size_t half = (nq + 1) / 2;
  const double vertex = 0.5 * (double)nq + 3.0 * (double)N / (double)Q;
  u128 worst = 0;
  const double cands[4] = {(double)half, (double)(nq - 1), std::floor(vertex),
                           std::ceil(vertex)};
  for (double c : cands) {
    const double cl = std::min<double>(std::max<double>(c, (double)half), (double)(nq - 1));
    const u128 b = bytes_unpadded(N, nq, (u128)cl, Q);
    if (b > worst) worst = b;
  }
  return worst + (u128)kPieces * 256;
}

}  // namespace

using agf2::DGemm;

extern "C" int agf2_build_moments_noalloc(const double* L, int naux, int nmo, const double* e,
                                          const double* C, int nqmo, double mu, double* U_hole,
                                          double* U_part, void* stream) {
  if (!L || !e || !C || !U_hole || !U_part || naux < 1 || nmo < 1 || nqmo < 2)
    return AGF2_ERR_INVALID_ARG;
  const size_t N = nmo, nq = nqmo, Q = naux;
  // Size check before touching any argument: the worst split of nq poles.
  if (worst_case_bytes(N, nq, Q) > (u128)kScratchBytes) return AGF2_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* sp = nullptr;
  if (int rc = scratch_address(&sp)) return rc;
  Arena A{static_cast<char*>(sp), 0, kScratchBytes};

  std::vector<double> eh(nq);
  if (cudaMemcpyAsync(eh.data(), e, nq * sizeof(double), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return AGF2_ERR_CUDA;
  }
  std::vector<int> order;
  order.reserve(nq);
  for (size_t x = 0; x < nq; ++x) {
    if (!std::isfinite(eh[x])) return AGF2_ERR_INVALID_ARG;
    if (eh[x] < mu) order.push_back((int)x);
  }
  const int o = (int)order.size();
  for (size_t x = 0; x < nq; ++x)
    if (!(eh[x] < mu)) order.push_back((int)x);
  const int v = (int)nq - o;
  if (o < 1 || v < 1) return AGF2_ERR_INVALID_ARG;

  int* idx = A.take<int>(nq);
  double* Co = A.take<double>(N * o);
  double* Cv = A.take<double>(N * v);
  double* eo = A.take<double>(o);
  double* ev = A.take<double>(v);
  double* Lxo = A.take<double>((size_t)o * N * Q);
  double* Lxv = A.take<double>((size_t)v * N * Q);
  double* Lov = A.take<double>((size_t)o * v * Q);
  if (!idx || !Co || !Cv || !eo || !ev || !Lxo || !Lxv || !Lov) return AGF2_ERR_INVALID_ARG;

#define NA_CK(call)                \
  do {                             \
    if ((call) != cudaSuccess) {   \
      cudaGetLastError();          \
      return AGF2_ERR_CUDA;        \
    }                              \
  } while (0)

  const long long NN = (long long)N * N, NQ = (long long)N * Q;
  NA_CK(cudaMemcpyAsync(idx, order.data(), nq * sizeof(int), cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemsetAsync(U_hole, 0, 2 * NN * sizeof(double), s));
  NA_CK(cudaMemsetAsync(U_part, 0, 2 * NN * sizeof(double), s));
  NA_CK(agf2::gather_columns(C, (int)N, (int)nq, idx, o, Co, s));
  NA_CK(agf2::gather_columns(C, (int)N, (int)nq, idx + o, v, Cv, s));
  NA_CK(agf2::gather_vec(e, idx, o, eo, s));
  NA_CK(agf2::gather_vec(e, idx + o, v, ev, s));
  auto rot = [&](const double* Cx, int nx, double* out) {
    DGemm g;  // out[x][p][Q] = sum_r Cx[r][x] L[Q][r][p]
    g.M = nx; g.N = (int)N; g.K = (int)N;
    g.A = Cx; g.sAm = 1; g.sAk = nx;
    g.B = L; g.sBk = (long long)N; g.sBn = 1; g.sB1 = NN;
    g.C = out; g.sCm = NQ; g.sCn = (long long)Q; g.sC1 = 1;
    g.nb1 = (int)Q;
    return agf2::dgemm(g, s);
  };
  NA_CK(rot(Co, o, Lxo));
  NA_CK(rot(Cv, v, Lxv));
  {
    DGemm g;  // Lov[j][a][Q] = sum_p Co[p][j] Lxv[a][p][Q]
    g.M = o; g.N = v; g.K = (int)N;
    g.A = Co; g.sAm = 1; g.sAk = o;
    g.B = Lxv; g.sBk = (long long)Q; g.sBn = NQ; g.sB1 = 1;
    g.C = Lov; g.sCm = (long long)v * Q; g.sCn = (long long)Q; g.sC1 = 1;
    g.nb1 = (int)Q;
    NA_CK(agf2::dgemm(g, s));
  }
  // Pair blocks sized to what is left of the array (at least one outer pole
  // per block fits: the size check above covers the worst split).
  const int n_in_max = std::max(o, v);
  const size_t min_block = 48 * N * (size_t)n_in_max + 4 * 256;
  if (A.used > A.cap || A.cap - A.used < min_block) return AGF2_ERR_INVALID_ARG;
  const size_t left_doubles = (A.cap - A.used - 4 * 256) / 8;
  int nb = (int)std::floor(std::sqrt((double)left_doubles / (6.0 * N * n_in_max)));
  nb = std::max(1, nb);
  while (nb > 1 && 6 * N * (size_t)nb * nb * n_in_max > left_doubles) --nb;
  const size_t K1max = (size_t)nb * nb * n_in_max;
  double* XIJ = A.take<double>(N * K1max);
  double* XJI = A.take<double>(N * K1max);
  double* Y = A.take<double>(N * 2 * K1max);
  double* Yw = A.take<double>(N * 2 * K1max);
  if (!XIJ || !XJI || !Y || !Yw) return AGF2_ERR_INVALID_ARG;

  struct Sec {
    int n_out, n_in;
    const double* Lx;
    const double* Lp;
    long long ys, cs;
    const double* e_out;
    const double* e_in;
    double* U;
  } secs[2] = {{o, v, Lxo, Lov, (long long)v * (long long)Q, (long long)Q, eo, ev, U_hole},
               {v, o, Lxv, Lov, (long long)Q, (long long)v * (long long)Q, ev, eo, U_part}};
  for (const Sec& S : secs) {
    const int nbs = std::min(nb, S.n_out);
    for (int I0 = 0; I0 < S.n_out; I0 += nbs) {
      const int nI = std::min(nbs, S.n_out - I0);
      for (int J0 = I0; J0 < S.n_out; J0 += nbs) {
        const int nJ = std::min(nbs, S.n_out - J0);
        const bool diag = (I0 == J0);
        const long long K1 = (long long)nI * nJ * S.n_in;
        auto pair_gemm = [&](int A0, int nA, int B0, int nB, double* X) {
          DGemm g;  // X[p][(a*nB+b)*n_in + c] = sum_Q Lx[A0+a][p][Q] Lp[B0+b][c][Q]
          g.M = (int)N; g.N = S.n_in; g.K = (int)Q;
          g.A = S.Lx + (long long)A0 * NQ; g.sAm = (long long)Q; g.sAk = 1; g.sA1 = NQ;
          g.B = S.Lp + (long long)B0 * S.ys; g.sBk = 1; g.sBn = S.cs; g.sB2 = S.ys;
          g.C = X; g.sCm = K1; g.sCn = 1; g.sC1 = (long long)nB * S.n_in; g.sC2 = S.n_in;
          g.nb1 = nA; g.nb2 = nB;
          return agf2::dgemm(g, s);
        };
        NA_CK(pair_gemm(I0, nI, J0, nJ, XIJ));
        if (!diag) NA_CK(pair_gemm(J0, nJ, I0, nI, XJI));
        NA_CK(agf2::sd_epilogue_fp64(XIJ, XJI, (int)N, nI, nJ, S.n_in, S.e_out + I0,
                                     S.e_out + J0, S.e_in, diag, Y, Yw, s));
        for (int n = 0; n < 2; ++n) {
          DGemm g;  // U^(n) += Z Y^T with Z = Y or Yw, K = 2 K1, split over K
          g.M = (int)N; g.N = (int)N; g.K = (int)(2 * K1);
          g.A = n == 0 ? Y : Yw; g.sAm = 2 * K1; g.sAk = 1;
          g.B = Y; g.sBk = 1; g.sBn = 2 * K1;
          g.C = S.U + n * NN; g.sCm = (long long)N; g.sCn = 1;
          g.atomic = true;
          const int tiles = (int)(((N + 63) / 64) * ((N + 63) / 64));
          g.ksplit = std::max(1, std::min<int>((int)(2 * K1 / 256), (2 * 152 + tiles - 1) / tiles));
          NA_CK(agf2::dgemm(g, s));
        }
      }
    }
  }
  NA_CK(agf2::symmetrize(U_hole, (int)N, 2, s));
  NA_CK(agf2::symmetrize(U_part, (int)N, 2, s));
  NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
  return AGF2_OK;
}
