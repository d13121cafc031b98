// Symmetric FP64 eigensolver for the Fock loop's extended Hamiltonian
// [[F, v], [v^T, diag(E)]] (Eqs. dyson_eq_eig / post_compression_h): all
// eigenvalues, and the eigenvectors' first nphys rows (the physical block the
// Fock loop reads: pole weights, the density, the shift derivative).
//
// Three stages, all on the GPU and without a host round trip:
//  1. Householder tridiagonalisation A = Q T Q^T in ONE cooperative kernel:
//     the matrix stays in L2, each CTA-warp owns fixed rows, and one grid
//     barrier per column separates the matrix-vector product from the
//     rank-2 update (the next pivot row is published before the barrier and
//     updated redundantly by every CTA).  A library sytrd spends most of its
//     time in per-column launches at these sizes (n = 3N .. 5N, a few
//     hundred to a few thousand).
//  2. Divide and conquer on T (Cuppen's split T = diag(T1, T2) + beta u u^T,
//     merged bottom-up by tree height): sort, deflation of negligible
//     z-components and of close pole pairs (Givens), the secular equation
//     1 + rho sum z_i^2 / (d_i - lambda) = 0 solved per root by safeguarded
//     Newton in the offset from the nearer pole, the Gu-Eisenstat
//     recomputation of z from the computed roots (which makes the
//     eigenvectors orthogonal to working precision), and the eigenvector
//     update Q_new = diag(Q1, Q2) M as tiled FP64 GEMMs.
//  3. The physical rows of Q (the reflectors applied to e_p^T, one warp per
//     row), then V_phys = Q[:nphys] Z with the library's FP64 GEMM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/agf2.h"
#include "agf2_internal.h"
#include "tc_core.cuh"

namespace agf2 {

namespace {

constexpr int SY_THREADS = 256;
// Limit of a grid-barrier wait, in ns of the global timer (a barrier that
// never completes).  The SM cycle counter is not used as the time base: the
// waiting warps sleep between polls, and a counter tied to the SM clock need
// not advance at its nominal rate then.
constexpr unsigned long long kSpinNs = 1000000000ULL;
constexpr int TILE = 40;                      // GEMM tile of the eigenvector update

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Arrival at step `step` of a flag barrier among the CTAs of a cooperative
// launch: every thread's prior global writes are made visible, then the
// CTA's own flag is raised (no shared counter, so no atomic contention).
__device__ __forceinline__ void flag_arrive(unsigned* flags, unsigned step) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // cumulative: the CTA's writes observed through the barrier come first
    volatile unsigned* f = flags + blockIdx.x;
    *f = step;
  }
}

// Wait until every CTA's flag reached `step` (warp 0 polls the flags in
// parallel); gives up after kSpinNs, setting *err and the abort flag.
__device__ bool flag_wait(unsigned* flags, unsigned step, int* err, int* abort_sh) {
  if (threadIdx.x < 32) {
    const unsigned long long t0 = tc::global_ns();
    bool ok = false;
    while (true) {
      bool mine = true;
      for (int g = threadIdx.x; g < (int)gridDim.x; g += 32)
        mine &= (*(volatile unsigned*)(flags + g) >= step);
      if (__all_sync(0xffffffffu, mine)) { ok = true; break; }
      // lane 0's clock decides, so the whole warp leaves the loop together
      // (a per-lane decision would strand the other lanes in __all_sync)
      if (__shfl_sync(0xffffffffu, (tc::global_ns() - t0 > kSpinNs) ? 1 : 0, 0)) break;
      __nanosleep(20);
    }
    if (!ok && threadIdx.x == 0) {
      atomicExch(err, 1);
      *abort_sh = 1;
    }
    __threadfence();
  }
  __syncthreads();
  return *abort_sh == 0;
}

// Householder tridiagonalisation (lower), A row-major n x n symmetric,
// destroyed.  Outputs d[n], e[n-1], tau[n-2] and the reflectors as rows of
// Vr (Vr[j][k] = v_j[k], v_j[j+1] = 1, zero for k <= j): A = Q T Q^T with
// Q = H_0 H_1 ... H_{n-3}, H_j = I - tau_j v_j v_j^T.
// CTA b owns rows b, b + G, b + 2G, ... (local row li = r / G, handled by warp
// li % warps); with ROWS_SMEM they live in shared memory for the whole
// reduction, else they stay in A.
// Step j, after the flag barrier: w_j = p_j + a v_j from the published p and
// partial sums; the pivot row j+1 (published by its owner before the
// barrier) gets step j's update in every CTA, which then forms v_{j+1}
// itself; one pass over each own row applies step j's rank-2 update and
// accumulates row . v_{j+1} for p_{j+1}.  The owner of row j+2 publishes
// it, and the CTA its partial v_{j+1} . p_{j+1}; then the next barrier.
// Scalar FP64 work is done by one warp: GB300's FP64 pipe is narrow and
// redundant per-warp copies of it cost more than the broadcast.
// Scratch: P [2][n], part [2][gridDim.x], nxt [2][n] (double-buffered by step
// parity so that a fast CTA's next step never overwrites what a slow CTA is
// still reading), bar [gridDim.x] step flags zeroed by the host.
template <bool ROWS_SMEM>
__global__ void __launch_bounds__(SY_THREADS) sytrd_kernel(double* A, int n, double* d,
                                                           double* e, double* tau, double* Vr,
                                                           double* P, double* part, double* nxt,
                                                           unsigned* bar, int* err) {
  extern __shared__ double sm[];
  double* piv = sm;          // pivot row, current
  double* va = sm + n;       // v of the current step
  double* vb = sm + 2 * n;   // v of the next step
  double* wv = sm + 3 * n;   // w of the current step
  double* rows_sm = sm + 4 * n;
  __shared__ double sc[4];   // broadcast scalars
  __shared__ double wpart[SY_THREADS / 32];
  __shared__ int abort_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int WPC = blockDim.x >> 5;
  const int G = gridDim.x, b = blockIdx.x;
  const int R = (n - b + G - 1) / G;  // rows of this CTA
  auto row_of = [&](int li) -> double* {
    return ROWS_SMEM ? rows_sm + (long long)li * n : A + (long long)(b + li * G) * n;
  };
  // reflector of step jj from piv[jj+1..n-1] into v (v[k] = 0 for k <= jj):
  // the norm and scalars in warp 0, the vector by the CTA
  auto householder = [&](int jj, double* v) {
    if (warp == 0) {
      double s2 = 0.0;
      for (int k = jj + 2 + lane; k < n; k += 32) s2 = fma(piv[k], piv[k], s2);
      s2 = warp_sum(s2);
      if (lane == 0) {
        const double alpha = piv[jj + 1];
        double t = 0.0, beta = alpha, scale = 0.0;
        if (s2 > 0.0) {
          beta = -copysign(sqrt(fma(alpha, alpha, s2)), alpha);
          t = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
        sc[0] = t;
        sc[1] = scale;
        if (b == 0) {
          d[jj] = piv[jj];
          e[jj] = beta;
          tau[jj] = t;
        }
      }
    }
    __syncthreads();
    const double scale = sc[1];
    for (int k = tid; k < n; k += blockDim.x)
      v[k] = k <= jj ? 0.0 : (k == jj + 1 ? 1.0 : piv[k] * scale);
    __syncthreads();
    if (b == 0)
      for (int k = tid; k < n; k += blockDim.x) Vr[(long long)jj * n + k] = v[k];
    return sc[0];
  };
  if (tid == 0) abort_sh = 0;
  for (int k = tid; k < n; k += blockDim.x) piv[k] = A[k];  // row 0 is never written
  if (ROWS_SMEM)
    for (long long t = tid; t < (long long)R * n; t += blockDim.x)
      rows_sm[t] = A[(long long)(b + (t / n) * G) * n + t % n];
  __syncthreads();
  double t_cur = 0.0;
  if (n > 2) {
    t_cur = householder(0, va);
    // p_0 over own rows r > 0, publish row 1
    double vp = 0.0;
    for (int li = warp; li < R; li += WPC) {
      const int r = b + li * G;
      if (r < 1) continue;
      const double* row = row_of(li);
      double a0 = 0.0, a1 = 0.0;
      int k = 1 + lane;
      for (; k + 32 < n; k += 64) {
        a0 = fma(row[k], va[k], a0);
        a1 = fma(row[k + 32], va[k + 32], a1);
      }
      if (k < n) a0 = fma(row[k], va[k], a0);
      const double pr = t_cur * warp_sum(a0 + a1);
      if (lane == 0) P[r] = pr;
      vp = fma(va[r], pr, vp);
      if (r == 1)
        for (int kk = 1 + lane; kk < n; kk += 32) nxt[kk] = row[kk];
    }
    if (lane == 0) wpart[warp] = vp;
    __syncthreads();
    if (tid == 0) {
      double sp = 0.0;
      for (int w = 0; w < WPC; ++w) sp += wpart[w];
      part[b] = sp;
    }
  }
  for (int j = 0; j + 2 < n; ++j) {
    const int buf = j & 1, nbuf = buf ^ 1;
    flag_arrive(bar, (unsigned)(j + 1));
    if (!flag_wait(bar, (unsigned)(j + 1), err, &abort_sh)) return;
    // w_j and the pivot row j+1, with the partial sums in the same round trip
    for (int k = j + 1 + tid; k < n; k += blockDim.x) {
      wv[k] = __ldcg(&P[buf * n + k]);
      piv[k] = __ldcg(&nxt[buf * n + k]);
    }
    if (warp == 0) {
      double sp = 0.0;
      for (int g = lane; g < G; g += 32) sp += __ldcg(&part[buf * G + g]);
      sp = warp_sum(sp);
      if (lane == 0) sc[2] = -0.5 * t_cur * sp;
    }
    __syncthreads();
    const double a2 = sc[2];
    for (int k = j + 1 + tid; k < n; k += blockDim.x) wv[k] = fma(a2, va[k], wv[k]);
    __syncthreads();
    for (int k = j + 1 + tid; k < n; k += blockDim.x)
      piv[k] = fma(-va[j + 1], wv[k], fma(-wv[j + 1], va[k], piv[k]));
    __syncthreads();
    const bool more = j + 3 < n;  // a reflector for step j+1 exists
    const double t_next = more ? householder(j + 1, vb) : 0.0;
    // one pass over own rows r > j: update by step j, dot with v_{j+1}
    double vp = 0.0;
    for (int li = warp; li < R; li += WPC) {
      const int r = b + li * G;
      if (r <= j) continue;
      double* row = row_of(li);
      const double vr = va[r], wr = wv[r];
      double a0 = 0.0;
      for (int k = j + 1 + lane; k < n; k += 32) {
        const double x = fma(-vr, wv[k], fma(-wr, va[k], row[k]));
        row[k] = x;
        a0 = fma(x, vb[k], a0);
      }
      if (more && r > j + 1) {
        const double pr = t_next * warp_sum(a0);
        if (lane == 0) P[nbuf * n + r] = pr;
        vp = fma(vb[r], pr, vp);
        if (r == j + 2)
          for (int kk = j + 2 + lane; kk < n; kk += 32) nxt[nbuf * n + kk] = row[kk];
      }
    }
    if (lane == 0) wpart[warp] = vp;
    __syncthreads();
    if (tid == 0 && more) {
      double sp = 0.0;
      for (int w = 0; w < WPC; ++w) sp += wpart[w];
      part[nbuf * G + b] = sp;
    }
    double* tmp = va;
    va = vb;
    vb = tmp;
    t_cur = t_next;
  }
  // the last 2 x 2: the pivot row n-2 is current in every CTA; row n-1's
  // owner holds its final diagonal
  if (n >= 2) {
    if (b == 0 && tid == 0) {
      d[n - 2] = piv[n - 2];
      e[n - 2] = piv[n - 1];
    }
    if ((n - 1) % G == b && tid == 0) d[n - 1] = row_of((n - 1 - b) / G)[n - 1];
  } else if (b == 0 && tid == 0) {
    d[0] = piv[0];
  }
}

// d'[i] = d[i] - beta(split at i) - beta(split at i+1); w = d', Q = I.
__global__ void dc_init_kernel(const double* __restrict__ d, const double* __restrict__ e,
                               const int* __restrict__ split, int n, double* __restrict__ w,
                               double* __restrict__ Q) {
  const long long total = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / n), c = (int)(t % n);
    Q[t] = (r == c) ? 1.0 : 0.0;
    if (r == c) {
      double x = d[r];
      if (split[r]) x -= e[r - 1];
      if (r + 1 < n && split[r + 1]) x -= e[r];
      w[r] = x;
    }
  }
}

// Per-position work arrays of one tree level (index s + local position).
struct DcArrays {
  double *dsrt, *zsrt, *dk, *zk, *rc, *rs, *tv, *zh, *inv, *mtmp;
  int *perm, *kept, *dpos, *ra, *rb, *org, *rank;
  double* mrho;   // per merge (at s): rho
  double* msgn;   // per merge (at s): +-1
  int *mk, *mrot; // per merge (at s): kept count, rotation count
};

// One merge per CTA.  The CTA stages the children's eigenvalues and the
// coupling vector z in shared memory; thread 0 then does the O(len)
// sequential parts (the sorted merge of the two runs, the deflation scan) on
// shared memory, and the CTA writes the results out.
// Shared memory: 2 len doubles + len ints (sorted values, z; the order).
__global__ void dc_deflate_kernel(const int* __restrict__ merges, const double* __restrict__ w,
                                  const double* __restrict__ Q, const double* __restrict__ e,
                                  int n, DcArrays a) {
  extern __shared__ double dsm[];
  const int s = merges[3 * blockIdx.x], h = merges[3 * blockIdx.x + 1],
            len = merges[3 * blockIdx.x + 2];
  double* wl = dsm;                                   // children's eigenvalues (local order)
  double* zl = dsm + len;                             // z (local order)
  int* order = reinterpret_cast<int*>(dsm + 2 * len); // sorted position -> local index
  const double beta = e[s + h - 1];
  const double sgn = beta < 0.0 ? -1.0 : 1.0;
  const double rho = fabs(2.0 * beta);
  const double r2 = 0.70710678118654752440;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    wl[i] = sgn * w[s + i];
    zl[i] = (i < h ? Q[(long long)(s + h - 1) * n + s + i] : Q[(long long)(s + h) * n + s + i]) * r2;
  }
  __syncthreads();
  __shared__ int kk_sh;
  if (threadIdx.x == 0) {
    // merge the two ascending (sgn > 0) or descending (sgn < 0) runs
    int i = sgn > 0 ? 0 : h - 1, j = sgn > 0 ? h : len - 1;
    const int di = sgn > 0 ? 1 : -1;
    for (int c = 0; c < len; ++c) {
      const bool lin = sgn > 0 ? i < h : i >= 0;
      const bool rin = sgn > 0 ? j < len : j >= h;
      int pick;
      if (!rin || (lin && wl[i] <= wl[j])) { pick = i; i += di; }
      else { pick = j; j += di; }
      order[c] = pick;
    }
  }
  __syncthreads();
  // sorted copies (reusing wl/zl would race: gather into the outputs first)
  for (int c = threadIdx.x; c < len; c += blockDim.x) {
    a.perm[s + c] = order[c];
    a.dsrt[s + c] = wl[order[c]];
    a.zsrt[s + c] = zl[order[c]];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < len; c += blockDim.x) {
    wl[c] = a.dsrt[s + c];
    zl[c] = a.zsrt[s + c];
  }
  __syncthreads();
  // tolerance, negligible-z flags and a pre-check of pair deflation between
  // consecutive non-negligible entries, in parallel
  __shared__ double red[8];
  __shared__ int anypair;
  double dm = 0.0;
  for (int c = threadIdx.x; c < len; c += blockDim.x) dm = fmax(dm, fabs(wl[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dm;
  if (threadIdx.x == 0) anypair = 0;
  __syncthreads();
  double dmax = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) dmax = fmax(dmax, red[i]);
  const double tol = 8.0 * 2.220446049250313e-16 * fmax(dmax, rho);
  int* tiny = a.rank + s;  // scratch flags (the ranks are computed by a later kernel)
  for (int c = threadIdx.x; c < len; c += blockDim.x) tiny[c] = rho * fabs(zl[c]) <= tol;
  __syncthreads();
  for (int c = threadIdx.x; c < len; c += blockDim.x) {
    if (tiny[c]) continue;
    int p = c - 1;
    while (p >= 0 && tiny[p]) --p;
    if (p < 0) continue;
    const double t = hypot(zl[p], zl[c]);
    if (fabs((wl[c] - wl[p]) * (zl[c] / t) * (zl[p] / t)) <= tol) anypair = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double* D = wl;
    double* Z = zl;
    int* kept = order;  // order[] is reused for the kept list
    int nrot = 0, k = 0, nd = 0, last = -1;
    if (!anypair) {
      // no pair can deflate (rotations only ever happen between consecutive
      // kept entries, and none of the original pairs qualifies): integer work only
      for (int c = 0; c < len; ++c) {
        if (tiny[c]) a.dpos[s + nd++] = c;
        else kept[k++] = c;
      }
    } else {
      for (int c = 0; c < len; ++c) {
        if (tiny[c]) { a.dpos[s + nd++] = c; continue; }
        if (last >= 0) {
          const double t = hypot(Z[last], Z[c]);
          const double cs = Z[c] / t, sn = -Z[last] / t;
          if (fabs((D[c] - D[last]) * cs * sn) <= tol) {
            a.rb[s + nrot] = c;
            a.rc[s + nrot] = cs;
            a.rs[s + nrot] = sn;
            a.ra[s + nrot] = last;
            ++nrot;
            const double dl_ = D[last], dc_ = D[c];
            D[last] = dl_ * cs * cs + dc_ * sn * sn;
            D[c] = dl_ * sn * sn + dc_ * cs * cs;
            Z[last] = 0.0;
            Z[c] = t;
            a.dpos[s + nd++] = last;
            --k;  // `last` was the newest kept entry
          }
        }
        kept[k++] = c;
        last = c;
      }
      // the kept list must stay ascending in D (a rotation moves D[c] towards
      // D[last]); insertion sort repairs the rare exception
      for (int i = 1; i < k; ++i) {
        const int x = kept[i];
        int j = i - 1;
        while (j >= 0 && D[kept[j]] > D[x]) { kept[j + 1] = kept[j]; --j; }
        kept[j + 1] = x;
      }
    }
    kk_sh = k;
    a.mrho[s] = rho;
    a.msgn[s] = sgn;
    a.mk[s] = k;
    a.mrot[s] = nrot;
  }
  __syncthreads();
  const int k = kk_sh;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    a.kept[s + i] = order[i];
    a.dk[s + i] = wl[order[i]];
    a.zk[s + i] = zl[order[i]];
  }
  // the deflated poles' rotated values
  for (int c = threadIdx.x; c < len; c += blockDim.x) a.dsrt[s + c] = wl[c];
}

// The per-root and per-pole kernels below run one warp per item, the lanes
// splitting the O(k) sums: GB300's FP64 pipe is narrow, so the divisions of
// a large merge must be spread over many SMs, not over the threads of a few.

// Root j of 1 + rho sum_i zk_i^2 / (dk_i - lambda) over the kept poles:
// lambda = dk[org] + tv with the origin the nearer pole of its interval.
__global__ void dc_secular_kernel(const int* __restrict__ owner, int n, DcArrays a) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n) return;
  const int s = owner[t];
  if (s < 0) return;
  const int j = t - s, k = a.mk[s];
  if (j >= k) return;
  const double* dk = a.dk + s;
  const double* zk = a.zk + s;
  const double rho = a.mrho[s];
  // f, f' and 1 + sum |terms| (the scale of f's rounding error) at offset tau from pole o
  auto f_and_df = [&](int o, double tau, double& df, double& fabs_sum) {
    double f = 0.0, g = 0.0, sa = 0.0;
    const double dor = dk[o];
    for (int i = lane; i < k; i += 32) {
      const double den = (dk[i] - dor) - tau;
      const double q = zk[i] / den;
      const double term = rho * zk[i] * q;   // rho z_i^2 / den
      f += term;
      sa += fabs(term);
      g = fma(rho * q, q, g);                // d/dtau: rho z_i^2 / den^2
    }
    f = 1.0 + warp_sum(f);
    df = warp_sum(g);
    fabs_sum = 1.0 + warp_sum(sa);
    return f;
  };
  int o;
  double lo, hi, tau;
  if (j + 1 < k) {
    // bracket half from the sign of f at the midpoint; first iterate from the
    // two-pole model c + a/(-t) + b/(width - t) = 0 (t from d_j), with c the
    // other poles' contribution at the midpoint
    const double width = dk[j + 1] - dk[j];
    const double mid = 0.5 * width;
    double df, sa;
    const double fm = f_and_df(j, mid, df, sa);
    const double a = rho * zk[j] * zk[j], b = rho * zk[j + 1] * zk[j + 1];
    const double c = fm + a / mid - b / (width - mid);
    const double B = c * width + a + b;
    const double t0 = 2.0 * a * width / (B + sqrt(fmax(0.0, B * B - 4.0 * a * c * width)));
    if (fm >= 0.0) { o = j; lo = 0.0; hi = mid; tau = t0; }
    else { o = j + 1; lo = mid - width; hi = 0.0; tau = t0 - width; }
  } else {
    double z2 = 0.0;
    for (int i = lane; i < k; i += 32) z2 = fma(zk[i], zk[i], z2);
    o = j;
    lo = 0.0;
    hi = rho * warp_sum(z2);
    double df, sa;
    const double fm = f_and_df(j, 0.5 * hi, df, sa);
    const double a = rho * zk[j] * zk[j];
    const double c = fm + a / (0.5 * hi);   // 1 + other poles at the midpoint
    tau = c > 0.0 ? a / c : 0.5 * hi;
  }
  if (!(tau > lo && tau < hi)) tau = 0.5 * (lo + hi);
  const double eps = 2.220446049250313e-16;
  for (int it = 0; it < 200; ++it) {
    double df, sa;
    const double f = f_and_df(o, tau, df, sa);
    // f is zero to within its own rounding error: tau is as good as the
    // data allow (the secular-equation stopping rule of LAPACK's dlaed4)
    if (fabs(f) <= 8.0 * eps * (double)k * sa) break;
    if (f > 0.0) hi = tau; else lo = tau;
    double tn = tau - f / df;
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    if (tn == tau || hi - lo <= 2.0 * eps * fmax(fabs(lo), fabs(hi))) { tau = tn; break; }
    tau = tn;
  }
  if (lane == 0) {
    a.org[s + j] = o;
    a.tv[s + j] = tau;
  }
}

__device__ __forceinline__ double warp_prod(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Gu-Eisenstat: zhat_i^2 = (lambda_i - d_i)/rho prod_{j != i} (lambda_j - d_i)/(d_j - d_i)
__global__ void dc_zhat_kernel(const int* __restrict__ owner, int n, DcArrays a) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n) return;
  const int s = owner[t];
  if (s < 0) return;
  const int i = t - s, k = a.mk[s];
  if (i >= k) return;
  const double* dk = a.dk + s;
  const double* tv = a.tv + s;
  const int* org = a.org + s;
  const double di = dk[i];
  double prod = 1.0;
  for (int j = lane; j < k; j += 32)
    prod *= (j == i) ? ((dk[org[i]] - di) + tv[i]) / a.mrho[s]
                     : ((dk[org[j]] - di) + tv[j]) / (dk[j] - di);
  prod = warp_prod(prod);
  if (lane == 0) a.zh[s + i] = copysign(sqrt(fabs(prod)), a.zk[s + i]);
}

// 1 / ||zhat_i / (d_i - lambda_j)||
__global__ void dc_norm_kernel(const int* __restrict__ owner, int n, DcArrays a) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n) return;
  const int s = owner[t];
  if (s < 0) return;
  const int j = t - s, k = a.mk[s];
  if (j >= k) return;
  const double* dk = a.dk + s;
  const double lo = dk[a.org[s + j]], tv = a.tv[s + j];
  double ss = 0.0;
  for (int i = lane; i < k; i += 32) {
    const double q = a.zh[s + i] / ((dk[i] - lo) - tv);
    ss = fma(q, q, ss);
  }
  ss = warp_sum(ss);
  if (lane == 0) a.inv[s + j] = 1.0 / sqrt(ss);
}

// Eigenvalue of column c of the merge (roots first, then deflated poles),
// its rank in ascending order, and the merged eigenvalues in place.
__global__ void dc_rank_kernel(const int* __restrict__ owner, const int* __restrict__ merges_len,
                               int n, DcArrays a, double* __restrict__ w) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n) return;
  const int s = owner[t];
  if (s < 0) return;
  const int c = t - s, len = merges_len[t], k = a.mk[s];
  const double sg = a.msgn[s];
  auto val = [&](int x) {
    return x < k ? sg * (a.dk[s + a.org[s + x]] + a.tv[s + x]) : sg * a.dsrt[s + a.dpos[s + x - k]];
  };
  const double v = val(c);
  int r = 0;
  for (int x = lane; x < len; x += 32) {
    const double u = val(x);
    r += (u < v || (u == v && x < c)) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  if (lane == 0) {
    a.rank[s + c] = r;
    w[s + r] = v;  // w is read by this level's deflation kernel only, which has finished
  }
}

// Column c of M = P R_1 ... R_r [X_roots | E_deflated], written to column
// rank[c] of the merge's block of Mout (rows in the children's local order).
// One warp per column; the column is built contiguously in mtmp row s + c.
__global__ void dc_column_kernel(const int* __restrict__ owner, const int* __restrict__ merges_len,
                                 int n, DcArrays a, double* __restrict__ Mout) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n) return;
  const int s = owner[t];
  if (s < 0) return;
  const int c = t - s, len = merges_len[t], k = a.mk[s], nrot = a.mrot[s];
  double* x = a.mtmp + (long long)(s + c) * n + s;
  for (int r = lane; r < len; r += 32) x[r] = 0.0;
  __syncwarp();
  if (c < k) {
    const double lam0 = a.dk[s + a.org[s + c]], tv = a.tv[s + c], inv = a.inv[s + c];
    for (int i = lane; i < k; i += 32)
      x[a.kept[s + i]] = a.zh[s + i] / ((a.dk[s + i] - lam0) - tv) * inv;
  } else if (lane == 0) {
    x[a.dpos[s + c - k]] = 1.0;
  }
  __syncwarp();
  if (lane == 0) {
    for (int r = nrot - 1; r >= 0; --r) {
      const int ia = a.ra[s + r], ib = a.rb[s + r];
      const double cs = a.rc[s + r], sn = a.rs[s + r];
      const double xa = x[ia], xb = x[ib];
      x[ia] = cs * xa - sn * xb;
      x[ib] = sn * xa + cs * xb;
    }
  }
  __syncwarp();
  const int col = s + a.rank[s + c];
  for (int r = lane; r < len; r += 32) Mout[(long long)(s + a.perm[s + r]) * n + col] = x[r];
}

// Qout[s+r][s+c] = sum_t Qin[s+r][s+t] M[s+t][s+c] over the half (t in
// [k0, k1)) that row r belongs to.  tiles: {s, r0, r1, k0, k1, c0, c1}.
__global__ void __launch_bounds__(64) dc_gemm_kernel(const int* __restrict__ tiles,
                                                     const double* __restrict__ Qin,
                                                     const double* __restrict__ M, int n,
                                                     double* __restrict__ Qout) {
  constexpr int BK = 16, R = 5, TT = 8;
  __shared__ double As[BK][TILE];
  __shared__ double Bs[BK][TILE];
  const int* tl = tiles + 7 * blockIdx.x;
  const int s = tl[0], r0 = tl[1], r1 = tl[2], k0 = tl[3], k1 = tl[4], c0 = tl[5], c1 = tl[6];
  const int tid = threadIdx.x, tx = tid % TT, ty = tid / TT;
  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;
  for (int kb = k0; kb < k1; kb += BK) {
    for (int e = tid; e < BK * TILE; e += 64) {
      const int mm = e / BK, kk = e % BK;
      const int gr = r0 + mm, gk = kb + kk;
      As[kk][mm] = (gr < r1 && gk < k1) ? Qin[(long long)(s + gr) * n + s + gk] : 0.0;
      const int nn = e % TILE, kk2 = e / TILE;
      const int gc = c0 + nn, gk2 = kb + kk2;
      Bs[kk2][nn] = (gc < c1 && gk2 < k1) ? M[(long long)(s + gk2) * n + s + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double av[R], bv[R];
#pragma unroll
      for (int i = 0; i < R; ++i) av[i] = As[kk][ty + TT * i];
#pragma unroll
      for (int j = 0; j < R; ++j) bv[j] = Bs[kk][tx + TT * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int gr = r0 + ty + TT * i;
    if (gr >= r1) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int gc = c0 + tx + TT * j;
      if (gc < c1) Qout[(long long)(s + gr) * n + s + gc] = acc[i][j];
    }
  }
}

// Copy the tiles' output region back: Qdst <- Qsrc.
__global__ void dc_copy_kernel(const int* __restrict__ tiles, const double* __restrict__ Qsrc,
                               int n, double* __restrict__ Qdst) {
  const int* tl = tiles + 7 * blockIdx.x;
  const int s = tl[0], r0 = tl[1], r1 = tl[2], c0 = tl[5], c1 = tl[6];
  const int w = c1 - c0;
  for (int e = threadIdx.x; e < (r1 - r0) * w; e += blockDim.x) {
    const long long idx = (long long)(s + r0 + e / w) * n + s + c0 + e % w;
    Qdst[idx] = Qsrc[idx];
  }
}

// Physical rows of Q: X[p] = e_p^T H_0 H_1 ... H_{n-3}, one warp per row p,
// the CTA's rows in shared memory; the reflectors are staged `ch` at a time
// (one barrier per chunk), then each warp applies them in order.
__global__ void phys_rows_kernel(const double* __restrict__ Vr, const double* __restrict__ tau,
                                 int n, int nphys, int ch, int wpb, double* __restrict__ X) {
  extern __shared__ double xs[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // warps >= wpb only help to stage the reflectors
  const int p = warp < wpb ? blockIdx.x * wpb + warp : nphys;
  double* vsm = xs + (long long)wpb * n;  // [ch][n]
  double* x = xs + (long long)min(warp, wpb - 1) * n;
  if (warp < wpb)
    for (int k = lane; k < n; k += 32) x[k] = (k == p) ? 1.0 : 0.0;
  const int nref = n - 2;
  for (int j0 = 0; j0 < nref; j0 += ch) {
    const int nc = min(ch, nref - j0);
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)nc * n; e += blockDim.x) {
      const int jj = (int)(e / n), k = (int)(e % n);
      if (k > j0 + jj) vsm[e] = Vr[(long long)(j0 + jj) * n + k];
    }
    __syncthreads();
    if (p < nphys) {
      for (int jj = 0; jj < nc; ++jj) {
        const int j = j0 + jj;
        const double t = tau[j];
        if (t == 0.0) continue;
        const double* v = vsm + (long long)jj * n;
        double d0 = 0.0, d1 = 0.0;
        int k = j + 1 + lane;
        for (; k + 32 < n; k += 64) {
          d0 = fma(x[k], v[k], d0);
          d1 = fma(x[k + 32], v[k + 32], d1);
        }
        if (k < n) d0 = fma(x[k], v[k], d0);
        const double dot = t * warp_sum(d0 + d1);
        for (int kk = j + 1 + lane; kk < n; kk += 32) x[kk] = fma(-dot, v[kk], x[kk]);
        __syncwarp();
      }
    }
  }
  if (p < nphys)
    for (int k = lane; k < n; k += 32) X[(long long)p * n + k] = x[k];
}

constexpr int WY = 8;  // reflectors per compact-WY block of the back-transformation

// T factors of the compact WY form, one CTA per block of WY reflectors
// j0 = c WY .. j0 + WY - 1 (missing ones count as tau = 0):
// H_{j0} H_{j0+1} ... = I - V T V^T with T upper triangular,
//   T[i][i] = tau_i,  T[0:i, i] = -tau_i T[0:i, 0:i] (V[:, 0:i]^T v_i).
__global__ void wy_t_kernel(const double* __restrict__ Vr, const double* __restrict__ tau, int n,
                            double* __restrict__ Tout) {
  __shared__ double Gm[WY][WY];
  const int c = blockIdx.x, j0 = c * WY, nref = n - 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int q = warp; q < WY * WY; q += nw) {
    const int l = q / WY, i = q % WY;
    if (l >= i) continue;  // warp-uniform
    double g = 0.0;
    if (j0 + i < nref) {
      const double* vl = Vr + (long long)(j0 + l) * n;
      const double* vi = Vr + (long long)(j0 + i) * n;
      for (int k = j0 + i + 1 + lane; k < n; k += 32) g = fma(vl[k], vi[k], g);
    }
    g = warp_sum(g);
    if (lane == 0) Gm[l][i] = g;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double T[WY][WY];
    for (int r = 0; r < WY; ++r)
      for (int i = 0; i < WY; ++i) T[r][i] = 0.0;
    for (int i = 0; i < WY; ++i) {
      const double ti = (j0 + i < nref) ? tau[j0 + i] : 0.0;
      double w[WY];
      for (int l = 0; l < i; ++l) w[l] = -ti * Gm[l][i];
      for (int r = 0; r < i; ++r) {
        double acc = 0.0;
        for (int l = r; l < i; ++l) acc = fma(T[r][l], w[l], acc);
        T[r][i] = acc;
      }
      T[i][i] = ti;
    }
    for (int r = 0; r < WY; ++r)
      for (int i = 0; i < WY; ++i) Tout[(long long)c * WY * WY + r * WY + i] = T[r][i];
  }
}

// Physical rows of Q block by block: x <- x (I - V T V^T) = x - ((x V) T) V^T,
// one warp per row (the CTA's rows and the block's reflectors and T in
// shared memory); the WY dot products and updates run side by side, so a
// row waits on one reduction per block instead of one per reflector.
__global__ void phys_rows_wy_kernel(const double* __restrict__ Vr, const double* __restrict__ Tall,
                                    int n, int nphys, int wpb, double* __restrict__ X) {
  extern __shared__ double xs[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = warp < wpb ? blockIdx.x * wpb + warp : nphys;  // other warps only stage
  double* vsm = xs + (long long)wpb * n;   // [WY][n]
  double* Tsm = vsm + (long long)WY * n;   // [WY][WY]
  double* x = xs + (long long)min(warp, wpb - 1) * n;
  if (warp < wpb)
    for (int k = lane; k < n; k += 32) x[k] = (k == p) ? 1.0 : 0.0;
  const int nref = n - 2, nblk = (nref + WY - 1) / WY;
  for (int c = 0; c < nblk; ++c) {
    const int j0 = c * WY;
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)WY * n; e += blockDim.x) {
      const int i = (int)(e / n), k = (int)(e % n), j = j0 + i;
      vsm[e] = (j < nref && k > j) ? Vr[(long long)j * n + k] : 0.0;
    }
    for (int e = threadIdx.x; e < WY * WY; e += blockDim.x) Tsm[e] = Tall[(long long)c * WY * WY + e];
    __syncthreads();
    if (p < nphys) {
      double y[WY];
#pragma unroll
      for (int i = 0; i < WY; ++i) y[i] = 0.0;
      for (int k = j0 + 1 + lane; k < n; k += 32) {
        const double xk = x[k];
#pragma unroll
        for (int i = 0; i < WY; ++i) y[i] = fma(xk, vsm[i * n + k], y[i]);
      }
#pragma unroll
      for (int i = 0; i < WY; ++i) y[i] = warp_sum(y[i]);
      double z[WY];
#pragma unroll
      for (int i = 0; i < WY; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int l = 0; l <= i; ++l) acc = fma(y[l], Tsm[l * WY + i], acc);
        z[i] = acc;
      }
      for (int k = j0 + 1 + lane; k < n; k += 32) {
        double a = x[k];
#pragma unroll
        for (int i = 0; i < WY; ++i) a = fma(-z[i], vsm[i * n + k], a);
        x[k] = a;
      }
      __syncwarp();
    }
  }
  if (p < nphys)
    for (int k = lane; k < n; k += 32) X[(long long)p * n + k] = x[k];
}

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

template <class T>
T* grow(Buf& b, size_t count, std::string& err) {
  const size_t bytes = std::max<size_t>(count * sizeof(T), 256);
  if (b.bytes < bytes) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      err = "eigensolver workspace allocation of " + std::to_string(bytes) + " bytes failed";
      return nullptr;
    }
    b.bytes = bytes;
  }
  return static_cast<T*>(b.p);
}

// The merge tree of one size n: merges grouped by height, the per-position
// owner map and GEMM tiles of every level, uploaded once.
struct Level {
  int nm = 0, ntiles = 0;
  int* merges = nullptr;  // device [nm][3] (s, h, len)
  int* owner = nullptr;   // device [n]: segment start of the merge owning position t, or -1
  int* lens = nullptr;    // device [n]: that merge's len
  int* tiles = nullptr;   // device [ntiles][7]
};

struct EigWs {
  int plan_n = -1;
  std::vector<Level> levels;
  Buf plan_mem;
  int* split = nullptr;  // device [n] split flags, inside plan_mem
  Buf A, d, e, tau, Vr, P, part, nxt, bar, err, w, Qa, Qb, M, X, Twy;
  Buf f_dsrt, f_zsrt, f_dk, f_zk, f_rc, f_rs, f_tv, f_zh, f_inv, f_mtmp, f_rho, f_sgn;
  Buf i_perm, i_kept, i_dpos, i_ra, i_rb, i_org, i_rank, i_k, i_rot;
};

int node(int s, int m, std::vector<std::vector<int>>& by_h) {
  if (m <= 1) return 0;
  const int h = m / 2;
  const int hl = node(s, h, by_h), hr = node(s + h, m - h, by_h);
  const int ht = std::max(hl, hr) + 1;
  if ((int)by_h.size() < ht) by_h.resize(ht);
  by_h[ht - 1].insert(by_h[ht - 1].end(), {s, h, m});
  return ht;
}

bool build_plan(EigWs& W, int n, cudaStream_t s, std::string& err) {
  if (W.plan_n == n) return true;
  std::vector<std::vector<int>> by_h;
  node(0, n, by_h);
  std::vector<int> host;  // all plan ints, then uploaded in one copy
  struct Off { size_t merges, owner, lens, tiles; int nm, ntiles; };
  std::vector<Off> offs;
  std::vector<int> split(n, 0);
  for (auto& L : by_h) {
    Off o{};
    o.nm = (int)L.size() / 3;
    std::vector<int> owner(n, -1), lens(n, 0), tiles;
    for (int m = 0; m < o.nm; ++m) {
      const int s0 = L[3 * m], h = L[3 * m + 1], len = L[3 * m + 2];
      split[s0 + h] = 1;
      for (int t = s0; t < s0 + len; ++t) { owner[t] = s0; lens[t] = len; }
      for (int half = 0; half < 2; ++half) {
        const int ra = half ? h : 0, rb = half ? len : h;
        for (int r0 = ra; r0 < rb; r0 += TILE)
          for (int c0 = 0; c0 < len; c0 += TILE)
            tiles.insert(tiles.end(), {s0, r0, std::min(rb, r0 + TILE), ra, rb, c0,
                                       std::min(len, c0 + TILE)});
      }
    }
    o.ntiles = (int)tiles.size() / 7;
    o.merges = host.size(); host.insert(host.end(), L.begin(), L.end());
    o.owner = host.size(); host.insert(host.end(), owner.begin(), owner.end());
    o.lens = host.size(); host.insert(host.end(), lens.begin(), lens.end());
    o.tiles = host.size(); host.insert(host.end(), tiles.begin(), tiles.end());
    offs.push_back(o);
  }
  const size_t split_off = host.size();
  host.insert(host.end(), split.begin(), split.end());
  int* dev = grow<int>(W.plan_mem, host.size(), err);
  if (!dev) return false;
  if (cudaMemcpyAsync(dev, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    err = "eigensolver plan upload failed";
    return false;
  }
  W.levels.clear();
  for (auto& o : offs) {
    Level L;
    L.nm = o.nm;
    L.ntiles = o.ntiles;
    L.merges = dev + o.merges;
    L.owner = dev + o.owner;
    L.lens = dev + o.lens;
    L.tiles = dev + o.tiles;
    W.levels.push_back(L);
  }
  W.split = dev + split_off;
  W.plan_n = n;
  return true;
}

}  // namespace

void* eig_workspace_create() { return new EigWs(); }

void eig_workspace_destroy(void* p) {
  if (!p) return;
  EigWs* W = static_cast<EigWs*>(p);
  for (Buf* b : {&W->plan_mem, &W->Twy, &W->A, &W->d, &W->e, &W->tau, &W->Vr, &W->P, &W->part, &W->nxt,
                 &W->bar, &W->err, &W->w, &W->Qa, &W->Qb, &W->M, &W->X, &W->f_dsrt, &W->f_zsrt,
                 &W->f_dk, &W->f_zk, &W->f_rc, &W->f_rs, &W->f_tv, &W->f_zh, &W->f_inv,
                 &W->f_mtmp, &W->f_rho, &W->f_sgn, &W->i_perm, &W->i_kept, &W->i_dpos, &W->i_ra,
                 &W->i_rb, &W->i_org, &W->i_rank, &W->i_k, &W->i_rot})
    if (b->p) cudaFree(b->p);
  delete W;
}

int eigh_phys(void* workspace, const double* Ain, int n, int nphys, double* w_out, double* V,
              cudaStream_t s, std::string& err) {
  EigWs& W = *static_cast<EigWs*>(workspace);
  // the tridiagonalisation keeps four length-n vectors in shared memory
  if (n < 1 || nphys < 1 || nphys > n || n > 7000) {
    err = "eigh_phys: need 1 <= nphys <= n <= 7000";
    return AGF2_ERR_INVALID_ARG;
  }
  const long long nn = (long long)n * n;
  double* A = grow<double>(W.A, nn, err);
  double* d = grow<double>(W.d, n, err);
  double* e = grow<double>(W.e, n, err);
  double* tau = grow<double>(W.tau, n, err);
  double* Vr = grow<double>(W.Vr, nn, err);
  double* P = grow<double>(W.P, 2 * (size_t)n, err);
  double* nxt = grow<double>(W.nxt, 2 * (size_t)n, err);
  unsigned* bar = grow<unsigned>(W.bar, 1024, err);  // step flags, one per CTA (G <= 1024)
  int* derr = grow<int>(W.err, 1, err);
  double* w = grow<double>(W.w, n, err);
  double* Qa = grow<double>(W.Qa, nn, err);
  double* Qb = grow<double>(W.Qb, nn, err);
  double* M = grow<double>(W.M, nn, err);
  double* X = grow<double>(W.X, (size_t)nphys * n, err);
  DcArrays a;
  a.dsrt = grow<double>(W.f_dsrt, n, err);
  a.zsrt = grow<double>(W.f_zsrt, n, err);
  a.dk = grow<double>(W.f_dk, n, err);
  a.zk = grow<double>(W.f_zk, n, err);
  a.rc = grow<double>(W.f_rc, n, err);
  a.rs = grow<double>(W.f_rs, n, err);
  a.tv = grow<double>(W.f_tv, n, err);
  a.zh = grow<double>(W.f_zh, n, err);
  a.inv = grow<double>(W.f_inv, n, err);
  a.mtmp = grow<double>(W.f_mtmp, nn, err);
  a.mrho = grow<double>(W.f_rho, n, err);
  a.msgn = grow<double>(W.f_sgn, n, err);
  a.perm = grow<int>(W.i_perm, n, err);
  a.kept = grow<int>(W.i_kept, n, err);
  a.dpos = grow<int>(W.i_dpos, n, err);
  a.ra = grow<int>(W.i_ra, n, err);
  a.rb = grow<int>(W.i_rb, n, err);
  a.org = grow<int>(W.i_org, n, err);
  a.rank = grow<int>(W.i_rank, n, err);
  a.mk = grow<int>(W.i_k, n, err);
  a.mrot = grow<int>(W.i_rot, n, err);
  for (void* p : {(void*)A, (void*)d, (void*)e, (void*)tau, (void*)Vr, (void*)P, (void*)nxt,
                  (void*)bar, (void*)derr, (void*)w, (void*)Qa, (void*)Qb, (void*)M, (void*)X,
                  (void*)a.dsrt, (void*)a.zsrt, (void*)a.dk, (void*)a.zk, (void*)a.rc,
                  (void*)a.rs, (void*)a.tv, (void*)a.zh, (void*)a.inv, (void*)a.mtmp,
                  (void*)a.mrho, (void*)a.msgn, (void*)a.perm, (void*)a.kept, (void*)a.dpos,
                  (void*)a.ra, (void*)a.rb, (void*)a.org, (void*)a.rank, (void*)a.mk,
                  (void*)a.mrot})
    if (!p) return AGF2_ERR_OOM;
  if (!build_plan(W, n, s, err)) return AGF2_ERR_OOM;
  const int* split = W.split;

  auto ck = [&](const char* what) {
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
      err = std::string(what) + ": " + cudaGetErrorString(ce);
      return false;
    }
    return true;
  };
  // 1. tridiagonalisation
  cudaMemcpyAsync(A, Ain, nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(bar, 0, 1024 * sizeof(unsigned), s);
  cudaMemsetAsync(derr, 0, sizeof(int), s);
  int dev = 0, nsm = 148, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // grid: more CTAs if the rows must fit in shared memory; global rows when
  // even one CTA per SM is too few
  const size_t base = 4 * (size_t)n * sizeof(double);
  const long long rmax = ((long long)smem_max - (long long)base - 1024) / (8LL * n);
  // about 4 rows per CTA: the per-step FP64 work (GB300's FP64 pipe is
  // narrow) spreads over up to all SMs, at the price of a wider barrier
  int G = std::min(nsm, std::max(1, (n + 3) / 4));
  bool rows_smem = rmax >= 1;
  if (rows_smem) {
    G = std::max<long long>(G, (n + rmax - 1) / rmax);
    if (G > nsm) { rows_smem = false; G = std::min(nsm, std::max(1, (n + 3) / 4)); }
  }
  const size_t smem = base + (rows_smem ? (size_t)((n + G - 1) / G) * n * sizeof(double) : 0);
  auto kern = rows_smem ? sytrd_kernel<true> : sytrd_kernel<false>;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    err = "eigh_phys: shared memory attribute";
    return AGF2_ERR_CUDA;
  }
  double* part = grow<double>(W.part, 2 * (size_t)G, err);
  if (!part) return AGF2_ERR_OOM;
  {
    void* args[] = {&A, (void*)&n, &d, &e, &tau, &Vr, &P, &part, &nxt, &bar, &derr};
    if (cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(SY_THREADS), args, smem, s) !=
        cudaSuccess) {
      ck("sytrd cooperative launch");
      return AGF2_ERR_CUDA;
    }
    count_launch();
    // a barrier that gave up left T unfinished: stop before the stages that read it
    int herr = 0;
    cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      ck("sytrd");
      return AGF2_ERR_CUDA;
    }
    if (herr) {
      err = "eigh_phys: tridiagonalisation barrier timed out";
      return AGF2_ERR_TIMEOUT;
    }
  }
  // 2. divide and conquer on T
  dc_init_kernel<<<(int)std::min<long long>((nn + 255) / 256, 152LL * 16), 256, 0, s>>>(
      d, e, split, n, w, Qa);
  count_launch();
  double* Qcur = Qa;
  const int wg = (n + 3) / 4;  // one warp per position, 4 warps per block
  // the deflation kernel's shared memory: 2 doubles + 1 int per position of
  // the largest merge (the root, len = n)
  const size_t dsm = (size_t)n * (2 * sizeof(double) + sizeof(int)) + 16;
  if (dsm > 48 * 1024 &&
      cudaFuncSetAttribute(dc_deflate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)dsm) != cudaSuccess) {
    err = "eigh_phys: shared memory attribute (deflation)";
    return AGF2_ERR_CUDA;
  }
  for (const Level& L : W.levels) {
    dc_deflate_kernel<<<L.nm, 256, dsm, s>>>(L.merges, w, Qcur, e, n, a);
    dc_secular_kernel<<<wg, 128, 0, s>>>(L.owner, n, a);
    dc_zhat_kernel<<<wg, 128, 0, s>>>(L.owner, n, a);
    dc_norm_kernel<<<wg, 128, 0, s>>>(L.owner, n, a);
    dc_rank_kernel<<<wg, 128, 0, s>>>(L.owner, L.lens, n, a, w);
    dc_column_kernel<<<(n + 7) / 8, 256, 0, s>>>(L.owner, L.lens, n, a, M);
    dc_gemm_kernel<<<L.ntiles, 64, 0, s>>>(L.tiles, Qcur, M, n, Qb);
    dc_copy_kernel<<<L.ntiles, 256, 0, s>>>(L.tiles, Qb, n, Qcur);
    count_launch(8);
  }
  if (!ck("divide and conquer")) return AGF2_ERR_CUDA;
  // 3. physical rows of Q, then V_phys = X Z (column-major output, ld n)
  {
    // rows per CTA: few, so that the rows' FP64 work spreads over the SMs
    const long long per = (long long)n * sizeof(double);
    const int wpb = std::max(1, std::min(4, (nphys + 2 * nsm - 1) / (2 * nsm)));
    const size_t wsm = (size_t)(wpb + WY) * per + WY * WY * sizeof(double);
    if (wsm + 1024 <= (size_t)smem_max) {
      // compact-WY blocks of 8 reflectors
      const int nblk = (n - 2 + WY - 1) / WY;
      double* Tw = grow<double>(W.Twy, (size_t)std::max(1, nblk) * WY * WY, err);
      if (!Tw) return AGF2_ERR_OOM;
      if (nblk > 0) {
        wy_t_kernel<<<nblk, 256, 0, s>>>(Vr, tau, n, Tw);
        count_launch();
      }
      if (wsm > 48 * 1024 &&
          cudaFuncSetAttribute(phys_rows_wy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)wsm) != cudaSuccess) {
        err = "eigh_phys: shared memory attribute (back-transformation)";
        return AGF2_ERR_CUDA;
      }
      phys_rows_wy_kernel<<<(nphys + wpb - 1) / wpb, 256, wsm, s>>>(Vr, Tw, n, nphys, wpb, X);
    } else {
      // one reflector at a time, staged `ch` per barrier (large n)
      const int ch = (int)std::max(1LL, std::min(8LL, ((long long)smem_max - 1024) / per - wpb));
      const size_t psm = (size_t)(wpb + ch) * per;
      if (psm > 48 * 1024 &&
          cudaFuncSetAttribute(phys_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)psm) != cudaSuccess) {
        err = "eigh_phys: shared memory attribute (back-transformation)";
        return AGF2_ERR_CUDA;
      }
      phys_rows_kernel<<<(nphys + wpb - 1) / wpb, 256, psm, s>>>(Vr, tau, n, nphys, ch, wpb, X);
    }
    count_launch();
    DGemm g;
    g.M = nphys; g.N = n; g.K = n;
    g.A = X; g.sAm = n; g.sAk = 1;
    g.B = Qcur; g.sBk = n; g.sBn = 1;
    g.C = V; g.sCm = 1; g.sCn = n;
    g.atomic = true;  // split over K: the product is tall in K for a short M
    g.ksplit = dgemm_split(nphys, n, n, false);
    cudaMemsetAsync(V, 0, (size_t)nn * sizeof(double), s);
    if (dgemm(g, s) != cudaSuccess) {
      ck("back-transformation");
      return AGF2_ERR_CUDA;
    }
  }
  cudaMemcpyAsync(w_out, w, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  int herr = 0;
  cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    ck("eigh_phys");
    return AGF2_ERR_CUDA;
  }
  if (herr) {
    err = "eigh_phys: tridiagonalisation barrier timed out";
    return AGF2_ERR_TIMEOUT;
  }
  return AGF2_OK;
}

}  // namespace agf2
