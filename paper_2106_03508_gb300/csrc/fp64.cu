// FP64 kernels of the AGF2 library: the strided-batched DGEMM used by the
// FP64 moment build (pole rotation, Eq. mp2_zeroth/first_moment GEMMs) and the
// Fock build, the 2J-K / energy-weight epilogue, and the small kernels of the
// compression / Fock loop / energy steps.
//
// GB300 executes FP64 at a small fraction of its BF16 tensor rate, so the
// GEMMs here are bound by the FP64 pipe, not by memory: a register-tiled SIMT
// tile (64x64 with 4x4 per thread, or 40x40 with 5x5 per thread where that
// pads the output less) keeps the pipe ~95-99% busy once enough CTAs run
// (split-K with FP64 atomics for long-K products, upper tiles only for
// symmetric outputs).
#include <algorithm>

#include "agf2_internal.h"

namespace agf2 {

namespace {

constexpr int BK = 16;

// Register-tiled FP64 GEMM tile: TB x TB outputs per CTA, R x R per thread,
// (TB/R)^2 threads.  TB = 64 (R = 4, 256 threads) for large operands, TB = 40
// (R = 5, 64 threads) where it pads less (e.g. 200 = 5 x 40 orbitals).
template <int TB, int R>
__global__ void __launch_bounds__((TB / R) * (TB / R)) dgemm_kernel(DGemm g) {
  constexpr int TT = TB / R;       // threads per tile edge
  constexpr int NT = TT * TT;
  __shared__ double As[BK][TB];
  __shared__ double Bs[BK][TB];
  const int z = blockIdx.z;
  const int b1 = z / g.nb2, b2 = z - b1 * g.nb2;
  const double* __restrict__ A = g.A + b1 * g.sA1 + b2 * g.sA2;
  const double* __restrict__ B = g.B + b1 * g.sB1 + b2 * g.sB2;
  double* C = g.C + b1 * g.sC1 + b2 * g.sC2;
  const int m0 = blockIdx.y * TB;
  const int nblk = (g.N + TB - 1) / TB;
  const int n0 = (blockIdx.x % nblk) * TB;
  if (g.upper && m0 > n0) return;  // symmetric C: the lower tiles are mirrored afterwards
  const int ks = blockIdx.x / nblk;  // K split index
  const int kchunk = ((g.K + g.ksplit - 1) / g.ksplit + BK - 1) / BK * BK;
  const int kbeg = ks * kchunk, kend = min(g.K, kbeg + kchunk);
  const int tid = threadIdx.x, tx = tid % TT, ty = tid / TT;
  const bool a_kc = (g.sAk == 1);
  const bool b_nc = (g.sBn == 1);
  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int e = tid; e < BK * TB; e += NT) {
      int mm, kk;
      if (a_kc) { mm = e / BK; kk = e % BK; } else { mm = e % TB; kk = e / TB; }
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < g.M && gk < kend) ? A[gm * g.sAm + gk * g.sAk] : 0.0;
      int nn;
      if (b_nc) { nn = e % TB; kk = e / TB; } else { nn = e / BK; kk = e % BK; }
      const int gn = n0 + nn, gk2 = k0 + kk;
      Bs[kk][nn] = (gn < g.N && gk2 < kend) ? B[gk2 * g.sBk + gn * g.sBn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[R], b[R];
#pragma unroll
      for (int i = 0; i < R; ++i) a[i] = As[kk][ty + TT * i];
#pragma unroll
      for (int j = 0; j < R; ++j) b[j] = Bs[kk][tx + TT * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int gm = m0 + ty + TT * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int gn = n0 + tx + TT * j;
      if (gn >= g.N) continue;
      double* c = C + gm * g.sCm + gn * g.sCn;
      const double v = g.alpha * acc[i][j];
      if (g.atomic) atomicAdd(c, v);
      else *c = (g.beta == 0.0) ? v : fma(g.beta, *c, v);
    }
  }
}

// C[p][q] <- C[q][p] for the lower tiles (p / tb > q / tb) an upper-tile GEMM skipped.
__global__ void mirror_lower_tiles_kernel(double* C, int n, long long ld, int tb) {
  const long long total = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(t / n), q = (int)(t % n);
    if (p / tb > q / tb) C[p * ld + q] = C[q * ld + p];
  }
}

__global__ void sd_epilogue_kernel(const double* __restrict__ XIJ, const double* __restrict__ XJI,
                                   int nmo, int nI, int nJ, int n_in,
                                   const double* __restrict__ eI, const double* __restrict__ eJ,
                                   const double* __restrict__ ein, double sS, double sD,
                                   double* __restrict__ Y, double* __restrict__ Yw) {
  const long long K1 = (long long)nI * nJ * n_in;
  const long long total = (long long)nmo * K1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long p = t / K1, k = t - p * K1;
    const int ii = (int)(k / ((long long)nJ * n_in));
    const int rem = (int)(k - (long long)ii * nJ * n_in);
    const int jj = rem / n_in, c = rem - jj * n_in;
    const double x1 = XIJ[t];
    const double x2 = XJI[p * K1 + ((long long)jj * nI + ii) * n_in + c];
    const double w = eI[ii] + eJ[jj] - ein[c];
    const double ys = sS * (x1 + x2), yd = sD * (x1 - x2);
    const long long row = p * 2 * K1;
    Y[row + k] = ys;
    Y[row + K1 + k] = yd;
    Yw[row + k] = ys * w;
    Yw[row + K1 + k] = yd * w;
  }
}

// Z[p][k] *= (e_out[x] + e_out[y] - e_in[c]) for the [S | D] layout of the
// FP64 epilogue (k mod K1 = (ii*nJ + jj)*n_in + c); turns Y w^n into Y w^(n+1).
__global__ void weight_columns_kernel(double* __restrict__ Z, int nmo, int nI, int nJ, int n_in,
                                      const double* __restrict__ eI, const double* __restrict__ eJ,
                                      const double* __restrict__ ein) {
  const long long K1 = (long long)nI * nJ * n_in;
  const long long total = (long long)nmo * 2 * K1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long k = t % (2 * K1);
    const long long k1 = k % K1;
    const int ii = (int)(k1 / ((long long)nJ * n_in));
    const int rem = (int)(k1 - (long long)ii * nJ * n_in);
    const int jj = rem / n_in, c = rem - jj * n_in;
    Z[t] *= eI[ii] + eJ[jj] - ein[c];
  }
}

inline int grid_for(long long n, int bs = 256) {
  long long g = (n + bs - 1) / bs;
  if (g > 152LL * 64) g = 152LL * 64;
  return (int)(g < 1 ? 1 : g);
}

__global__ void gather_columns_kernel(const double* __restrict__ C, int nrow, int ncol_src,
                                      const int* __restrict__ idx, int n, double* __restrict__ out) {
  const long long total = (long long)nrow * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / n;
    const int c = (int)(t - r * n);
    out[t] = C[r * ncol_src + idx[c]];
  }
}

__global__ void gather_vec_kernel(const double* __restrict__ e, const int* __restrict__ idx, int n,
                                  double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = e[idx[t]];
}

__global__ void symmetrize_kernel(double* U, int n, int nmat) {
  const long long total = (long long)nmat * n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long m = t / ((long long)n * n);
    const int r = (int)((t / n) % n), c = (int)(t % n);
    if (r < c) {
      double* B = U + m * n * n;
      const double s = 0.5 * (B[(long long)r * n + c] + B[(long long)c * n + r]);
      B[(long long)r * n + c] = s;
      B[(long long)c * n + r] = s;
    }
  }
}

__global__ void axpby_kernel(double* y, const double* x, double a, double b, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = (b == 0.0) ? a * x[t] : fma(a, x[t], b * y[t]);
}

__global__ void build_h_kernel(const double* __restrict__ F, const double* __restrict__ E,
                               const double* __restrict__ v, double delta, int nmo, int nse,
                               double* __restrict__ H) {
  const int n = nmo + nse;
  const long long total = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / n), c = (int)(t % n);
    double x;
    if (r < nmo && c < nmo) x = F[(long long)r * nmo + c];
    else if (r < nmo) x = v[(long long)r * nse + (c - nmo)];
    else if (c < nmo) x = v[(long long)c * nse + (r - nmo)];
    else x = (r == c) ? E[r - nmo] + delta : 0.0;
    H[t] = x;
  }
}

__global__ void column_weights_kernel(const double* __restrict__ V, int ld, int nmo, int ncol,
                                      double* __restrict__ w) {
  // one warp per column
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= ncol) return;
  const double* col = V + (long long)warp * ld;
  double s = 0.0;
  for (int p = lane; p < nmo; p += 32) s = fma(col[p], col[p], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) w[warp] = s;
}

__global__ void physical_block_kernel(const double* __restrict__ V, int ld, int nmo, int ncol,
                                      double* __restrict__ out) {
  const long long total = (long long)nmo * ncol;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(t / ncol), x = (int)(t % ncol);
    out[t] = V[(long long)x * ld + p];
  }
}

constexpr int RED_BLOCKS = 304, RED_THREADS = 256;

__device__ inline double block_sum(double s) {
  __shared__ double sh[RED_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  s = (threadIdx.x < RED_THREADS / 32) ? sh[threadIdx.x] : 0.0;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

// gamma_Q = sum_rs L[Q][r][s] D[r][s]: one block per Q (a pass over L at HBM rate)
__global__ void __launch_bounds__(RED_THREADS) gamma_density_kernel(const double* __restrict__ L,
                                                                     const double* __restrict__ D,
                                                                     long long nn,
                                                                     double* __restrict__ gam) {
  const double* LQ = L + (long long)blockIdx.x * nn;
  double s = 0.0;
  for (long long t = threadIdx.x; t < nn; t += blockDim.x) s = fma(LQ[t], D[t], s);
  s = block_sum(s);
  if (threadIdx.x == 0) gam[blockIdx.x] = s;
}

__device__ inline double block_max(double s) {
  __shared__ double sh[RED_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  s = (threadIdx.x < RED_THREADS / 32) ? sh[threadIdx.x] : 0.0;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  }
  return s;
}

__global__ void dot_partial(const double* __restrict__ a, const double* __restrict__ b, long long n,
                            double* __restrict__ part) {
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    s = fma(a[t], b[t], s);
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void maxdiff_partial(const double* __restrict__ a, const double* __restrict__ b,
                                long long n, double* __restrict__ part) {
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    s = fmax(s, fabs(a[t] - b[t]));
  s = block_max(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void final_sum(const double* __restrict__ part, int n, double* out) {
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += part[t];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

__global__ void final_max(const double* __restrict__ part, int n, double* out) {
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s = fmax(s, part[t]);
  s = block_max(s);
  if (threadIdx.x == 0) *out = s;
}

__global__ void coulomb_kernel(const double* __restrict__ L, const double* __restrict__ gamma,
                               int naux, long long nn, double* __restrict__ J) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int Q = 0; Q < naux; ++Q) s = fma(gamma[Q], L[(long long)Q * nn + t], s);
    J[t] = s;
  }
}

// gamma_Q = 2 sum_{r,k} Cocc[r][k] * Y[r][Q][k]; one block per Q.
__global__ void gamma_kernel(const double* __restrict__ Y, const double* __restrict__ Cocc, int nmo,
                             int naux, int k, double* __restrict__ gamma) {
  const int Q = blockIdx.x;
  double s = 0.0;
  const long long nk = (long long)nmo * k;
  for (long long t = threadIdx.x; t < nk; t += blockDim.x) {
    const long long r = t / k;
    const int c = (int)(t - r * k);
    s = fma(Cocc[t], Y[(r * naux + Q) * k + c], s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) gamma[Q] = 2.0 * s;
}

__global__ void fock_combine_kernel(const double* h, const double* J, const double* K, long long n,
                                   double* F) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    F[t] = h[t] + J[t] - 0.5 * K[t];
}

__global__ void gm_partial(const double* __restrict__ V, const double* __restrict__ e,
                           const double* __restrict__ E, int k, int nse, double* __restrict__ part) {
  double s = 0.0;
  const long long n = (long long)k * nse;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(t / nse), m = (int)(t % nse);
    const double vv = V[t];
    s += vv * vv / (e[x] - E[m]);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// 4 sum_{x<k, y<nv} S[x][y]^2 / (w[k+y] - w[x])
__global__ void deriv_partial(const double* __restrict__ S, const double* __restrict__ w, int k,
                              int nv, double* __restrict__ part) {
  double s = 0.0;
  const long long n = (long long)k * nv;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(t / nv), y = (int)(t % nv);
    const double sv = S[t];
    s += sv * sv / (w[k + y] - w[x]);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = 4.0 * s;
}

// lor[x][w] = eta / pi / ((omega_w - e_x)^2 + eta^2)
__global__ void lorentzian_kernel(const double* __restrict__ e, int nq, const double* __restrict__ w,
                                  int nw, double eta, double* __restrict__ lor) {
  const long long total = (long long)nq * nw;
  const double c = eta / 3.14159265358979323846;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(t / nw), j = (int)(t % nw);
    const double d = w[j] - e[x];
    lor[t] = c / fma(d, d, eta * eta);
  }
}

__global__ void square_kernel(const double* __restrict__ a, long long n, double* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = a[t] * a[t];
}

// out[j] = sum_r M[r][j]  (column sums, one thread per column)
__global__ void column_sum_kernel(const double* __restrict__ M, int nrow, int ncol,
                                  double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncol) return;
  double s = 0.0;
  for (int r = 0; r < nrow; ++r) s += M[(long long)r * ncol + j];
  out[j] = s;
}

__global__ void set_identity_kernel(double* A, int n, double scale) {
  const long long total = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    A[t] = ((t / n) == (t % n)) ? scale : 0.0;
}

__global__ void diag_from_vec_kernel(const double* d, int n, double* A) {
  const long long total = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    A[t] = ((t / n) == (t % n)) ? d[t / n] : 0.0;
}

__global__ void add_scalar_kernel(double* x, double a, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] += a;
}

}  // namespace

static long long g_launches = 0;
void count_launch(long long n) { __atomic_fetch_add(&g_launches, n, __ATOMIC_RELAXED); }
long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

cudaError_t dgemm(const DGemm& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.nb1 <= 0 || g.nb2 <= 0) return cudaSuccess;
  const long long nz = (long long)g.nb1 * g.nb2;
  if (g.ksplit > 1 && !g.atomic) return cudaErrorInvalidValue;
  if (g.upper && (g.M != g.N || nz != 1 || g.sCn != 1)) return cudaErrorInvalidValue;
  const int tb = dgemm_tile(g.M, g.N);
  dim3 grid(((g.N + tb - 1) / tb) * std::max(1, g.ksplit), (g.M + tb - 1) / tb, 1);
  // gridDim.z is limited to 65535: split large batches over several launches,
  // each covering whole b1 rows.
  const long long lim = (65535LL / g.nb2) * g.nb2;
  if (lim == 0) return cudaErrorInvalidValue;
  for (long long z0 = 0; z0 < nz;) {
    const long long chunk = std::min(nz - z0, lim);
    DGemm h = g;
    const long long b1_0 = z0 / g.nb2;
    h.A += b1_0 * g.sA1;
    h.B += b1_0 * g.sB1;
    h.C += b1_0 * g.sC1;
    h.nb1 = (int)(chunk / g.nb2);
    grid.z = (unsigned)chunk;
    if (tb == 40)
      dgemm_kernel<40, 5><<<grid, 64, 0, s>>>(h);
    else
      dgemm_kernel<64, 4><<<grid, 256, 0, s>>>(h);
    count_launch();
    z0 += chunk;
  }
  if (g.upper) {
    mirror_lower_tiles_kernel<<<grid_for((long long)g.M * g.M), 256, 0, s>>>(g.C, g.M, g.sCm, tb);
    count_launch();
  }
  return cudaGetLastError();
}

int dgemm_tile(int M, int N) {
  auto padded = [&](long long t) { return ((M + t - 1) / t * t) * ((N + t - 1) / t * t); };
  return padded(40) < padded(64) ? 40 : 64;
}

int dgemm_split(int M, int N, long long K, bool upper) {
  const int tb = dgemm_tile(M, N);
  const long long threads = tb == 40 ? 64 : 256;
  const long long tm = (M + tb - 1) / tb, tn = (N + tb - 1) / tb;
  const long long tiles = upper ? tm * (tm + 1) / 2 : tm * tn;
  const long long want = (152LL * 1024 / threads + tiles - 1) / tiles;
  return (int)std::max(1LL, std::min(want, K / 256));
}

cudaError_t sd_epilogue_fp64(const double* XIJ, const double* XJI, int nmo, int nI, int nJ,
                             int n_in, const double* e_outI, const double* e_outJ,
                             const double* e_in, bool diag, double* Y, double* Yw,
                             cudaStream_t s) {
  const double sS = diag ? 0.5 : sqrt(0.5);
  const double sD = diag ? sqrt(0.75) : sqrt(1.5);
  const long long total = (long long)nmo * nI * nJ * n_in;
  sd_epilogue_kernel<<<grid_for(total), 256, 0, s>>>(XIJ, diag ? XIJ : XJI, nmo, nI, nJ, n_in,
                                                      e_outI, e_outJ, e_in, sS, sD, Y, Yw);
  count_launch();
  return cudaGetLastError();
}

cudaError_t weight_columns_fp64(double* Z, int nmo, int nI, int nJ, int n_in, const double* e_outI,
                                const double* e_outJ, const double* e_in, cudaStream_t s) {
  const long long total = (long long)nmo * 2 * nI * nJ * n_in;
  weight_columns_kernel<<<grid_for(total), 256, 0, s>>>(Z, nmo, nI, nJ, n_in, e_outI, e_outJ, e_in);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gather_columns(const double* C, int nrow, int ncol_src, const int* idx, int n,
                           double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  gather_columns_kernel<<<grid_for((long long)nrow * n), 256, 0, s>>>(C, nrow, ncol_src, idx, n, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gather_vec(const double* e, const int* idx, int n, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  gather_vec_kernel<<<(n + 255) / 256, 256, 0, s>>>(e, idx, n, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t symmetrize(double* U, int n, int nmat, cudaStream_t s) {
  symmetrize_kernel<<<grid_for((long long)nmat * n * n), 256, 0, s>>>(U, n, nmat);
  count_launch();
  return cudaGetLastError();
}

cudaError_t axpby(double* y, const double* x, double a, double b, long long n, cudaStream_t s) {
  axpby_kernel<<<grid_for(n), 256, 0, s>>>(y, x, a, b, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t build_extended_h(const double* F, const double* E, const double* v, double delta,
                             int nmo, int nse, double* H, cudaStream_t s) {
  const long long n = nmo + nse;
  build_h_kernel<<<grid_for(n * n), 256, 0, s>>>(F, E, v, delta, nmo, nse, H);
  count_launch();
  return cudaGetLastError();
}

cudaError_t column_weights(const double* V, int ld, int nmo, int ncol, double* w, cudaStream_t s) {
  column_weights_kernel<<<(ncol * 32 + 255) / 256, 256, 0, s>>>(V, ld, nmo, ncol, w);
  count_launch();
  return cudaGetLastError();
}

// dst[r + c ld] = Lc(c, r) for r <= c, 0 below: the explicit upper factor
// B = Lc^T of a column-major lower Cholesky factor (upper part of Lc ignored).
__global__ void upper_from_lower_t_kernel(const double* __restrict__ Lc, int n,
                                          double* __restrict__ dst, long long ld) {
  const long long total = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / n), r = (int)(t % n);
    dst[r + c * ld] = (r <= c) ? Lc[c + (long long)r * n] : 0.0;
  }
}

cudaError_t upper_from_lower_t(const double* Lc, int n, double* dst, long long ld,
                               cudaStream_t s) {
  upper_from_lower_t_kernel<<<grid_for((long long)n * n), 256, 0, s>>>(Lc, n, dst, ld);
  count_launch();
  return cudaGetLastError();
}

cudaError_t physical_block(const double* V, int ld, int nmo, int ncol, double* out, cudaStream_t s) {
  physical_block_kernel<<<grid_for((long long)nmo * ncol), 256, 0, s>>>(V, ld, nmo, ncol, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gamma_from_density(const double* L, const double* D, int naux, int n,
                               double* gamma, cudaStream_t s) {
  gamma_density_kernel<<<naux, RED_THREADS, 0, s>>>(L, D, (long long)n * n, gamma);
  count_launch();
  return cudaGetLastError();
}

cudaError_t dot(const double* a, const double* b, long long n, double* out, double* scratch,
                cudaStream_t s) {
  dot_partial<<<RED_BLOCKS, RED_THREADS, 0, s>>>(a, b, n, scratch);
  count_launch();
  final_sum<<<1, RED_THREADS, 0, s>>>(scratch, RED_BLOCKS, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t max_abs_diff(const double* a, const double* b, long long n, double* out, double* scratch,
                         cudaStream_t s) {
  maxdiff_partial<<<RED_BLOCKS, RED_THREADS, 0, s>>>(a, b, n, scratch);
  count_launch();
  final_max<<<1, RED_THREADS, 0, s>>>(scratch, RED_BLOCKS, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t coulomb_from_gamma(const double* L, const double* gamma, int naux, int nmo, double* J,
                               cudaStream_t s) {
  const long long nn = (long long)nmo * nmo;
  coulomb_kernel<<<grid_for(nn), 256, 0, s>>>(L, gamma, naux, nn, J);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gamma_from_y(const double* Y, const double* Cocc, int nmo, int naux, int k,
                         double* gamma, cudaStream_t s) {
  gamma_kernel<<<naux, RED_THREADS, 0, s>>>(Y, Cocc, nmo, naux, k, gamma);
  count_launch();
  return cudaGetLastError();
}

cudaError_t fock_combine(const double* h, const double* J, const double* K, long long n, double* F,
                         cudaStream_t s) {
  fock_combine_kernel<<<grid_for(n), 256, 0, s>>>(h, J, K, n, F);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gm_energy(const double* V, const double* e, const double* E, int k, int nse,
                      double* out, double* scratch, cudaStream_t s) {
  gm_partial<<<RED_BLOCKS, RED_THREADS, 0, s>>>(V, e, E, k, nse, scratch);
  count_launch();
  final_sum<<<1, RED_THREADS, 0, s>>>(scratch, RED_BLOCKS, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t shift_derivative(const double* S, const double* w, int k, int nv, double* out,
                             double* scratch, cudaStream_t s) {
  deriv_partial<<<RED_BLOCKS, RED_THREADS, 0, s>>>(S, w, k, nv, scratch);
  count_launch();
  final_sum<<<1, RED_THREADS, 0, s>>>(scratch, RED_BLOCKS, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t lorentzian(const double* e, int nq, const double* w, int nw, double eta, double* lor,
                       cudaStream_t s) {
  lorentzian_kernel<<<grid_for((long long)nq * nw), 256, 0, s>>>(e, nq, w, nw, eta, lor);
  count_launch();
  return cudaGetLastError();
}

cudaError_t square(const double* a, long long n, double* out, cudaStream_t s) {
  square_kernel<<<grid_for(n), 256, 0, s>>>(a, n, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t column_sum(const double* M, int nrow, int ncol, double* out, cudaStream_t s) {
  column_sum_kernel<<<(ncol + 255) / 256, 256, 0, s>>>(M, nrow, ncol, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t set_identity(double* A, int n, double scale, cudaStream_t s) {
  set_identity_kernel<<<grid_for((long long)n * n), 256, 0, s>>>(A, n, scale);
  count_launch();
  return cudaGetLastError();
}

cudaError_t diag_from_vec(const double* d, int n, double* A, cudaStream_t s) {
  diag_from_vec_kernel<<<grid_for((long long)n * n), 256, 0, s>>>(d, n, A);
  count_launch();
  return cudaGetLastError();
}

cudaError_t add_scalar(double* x, double a, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  add_scalar_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, a, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace agf2
