// Pole-basis rotation of the density-fitted integrals on the tcgen05 tensor
// cores (the rotation into the QMO basis that feeds Eqs. mp2_zeroth_moment /
// mp2_first_moment: (xi|Q) = sum_r C_ri L^Q_rx, text after Eq.
// mp2_first_moment), to FP64-class accuracy.
//
// Split: every operand row gets a power-of-two unit u with |x| < 128 u and
// four BF16 limbs holding integers,
//   x / u = a0 + a1 2^-8 + a2 2^-16 + a3 2^-24,  a0 in [-128, 128],
//   a1, a2, a3 in [-128, 128],
// so the representation error is below 2^-32 of the row's largest entry.
// The product sum_k x_k y_k keeps the limb products of order i + j <= 3 (ten
// tcgen05 MMAs per K = 16) in four tensor-memory accumulators, one per order:
//   acc_k = sum_{i + j = k} a_i b_j  (integers, weight 2^-8k).
// Over one chunk of 256 K entries every partial sum of every order is an
// integer of magnitude <= 2^24 (order 3: four products of at most 2^14 per
// K entry), so the tensor core adds each chunk EXACTLY.  The epilogue turns
// a chunk into acc0 + 2^-8 acc1 + 2^-16 acc2 + 2^-24 acc3 as an unevaluated
// FP32 pair (TwoSum) and sums the chunks of a tile in FP32 pairs (~48 bits);
// the products of order >= 4 that are left out are below 2^-31 relative.
// The result is written in FP64, scaled by the two rows' units.
//
// C[b][m][n] = sum_k A[m][k] B[b][n][k], out[m sOm + b sOb + n]:
//   A: limb planes [4][rowsA][Ks], rows a_row0 + m (3-D tensor map),
//   B: limb planes [4][nbatch][Nn][Ks] (4-D map (k, n, b, limb)).
// Tiles of 128 x 64 (MMA M = 128, N = 64): four order accumulators of 64
// columns are 256 TMEM columns, so two tiles' accumulators double-buffer in
// the 512 columns and a chunk's epilogue overlaps the next chunk's MMAs.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/agf2.h"
#include "agf2_internal.h"
#include "tc_core.cuh"

namespace agf2 {

namespace {

constexpr int RBM = 128;                 // MMA M (rows of A)
constexpr int RBN = 64;                  // MMA N (rows of B per tile)
constexpr int RBK = 32;                  // K per stage (64-byte rows, 64-byte swizzle)
constexpr int RNL = 4;                   // limbs
constexpr int RSTAGES = 4;
constexpr int R_TILE_A = RBM * RBK * 2;  // 8 KB per limb
constexpr int R_TILE_B = RBN * RBK * 2;  // 4 KB per limb
constexpr int R_STAGE = RNL * (R_TILE_A + R_TILE_B);  // 48 KB
constexpr int R_SMEM = RSTAGES * R_STAGE + 1024;
constexpr int R_CHUNK = 256 / RBK;       // stages per exactly-summed chunk
constexpr int R_NBUF = 2;
constexpr int R_BUF_COLS = 4 * RBN;      // four order accumulators
constexpr int R_THREADS = 320;           // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int R_EPI_COLS = RBN / 2;      // columns per epilogue thread

enum { R_DEV_OK = 0, R_DEV_TIMEOUT = 1 };

struct RotParams {
  int M, Nn, ksteps, nbatch;  // rows of this launch, columns, K steps (Ks / RBK), batches
  int a_row0;                 // first A row of this launch
  int m_tiles, n_tiles, ntiles;
  const float* unitA;         // [rowsA] (indexed a_row0 + m)
  const float* unitB;         // [nbatch][Nn]
  double* out;                // out[m sOm + b sOb + n]
  long long sOm, sOb;
  int* err;
};

__device__ __forceinline__ void rot_decode(const RotParams& P, int t, int& b, int& m0, int& n0) {
  const int mt = t % P.m_tiles;  // consecutive CTAs share the B tile
  int r = t / P.m_tiles;
  const int nt = r % P.n_tiles;
  b = r / P.n_tiles;
  m0 = mt * RBM;
  n0 = nt * RBN;
}

// exact sum hi + x as an unevaluated pair (s, e): s + e == hi + x
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float t = s - a;
  e = (a - (s - t)) + (b - t);
}

__global__ void __launch_bounds__(R_THREADS, 1)
rot4_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
            const RotParams P) {
  constexpr int N_EPI_WARPS = R_THREADS / 32 - 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[RSTAGES];
  __shared__ __align__(8) uint64_t empty_bar[RSTAGES];
  __shared__ __align__(8) uint64_t accf_bar[R_NBUF];
  __shared__ __align__(8) uint64_t acce_bar[R_NBUF];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  __shared__ int issued_sh, consumed_sh, committed_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort_flag = &abort_sh;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RSTAGES; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < R_NBUF; ++b) {
      tc::mbar_init(&accf_bar[b], 1);
      tc::mbar_init(&acce_bar[b], N_EPI_WARPS);
    }
    abort_sh = 0;
    issued_sh = consumed_sh = committed_sh = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_base_sh, R_NBUF * R_BUF_COLS);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    tc::tma_prefetch(&mapA);
    tc::tma_prefetch(&mapB);
    int t = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < P.ntiles && ok; tile += gridDim.x) {
      int b, m0, n0;
      rot_decode(P, tile, b, m0, n0);
      for (int ks = 0; ks < P.ksteps; ++ks, ++t) {
        const int st = t % RSTAGES;
        const uint32_t ph = (t / RSTAGES) & 1;
        if (!tc::mbar_wait(&empty_bar[st], ph ^ 1, abort_flag)) { ok = false; break; }
        uint8_t* base = smem + st * R_STAGE;
        tc::mbar_arrive_expect_tx(&full_bar[st], R_STAGE);
        for (int l = 0; l < RNL; ++l) {
          tc::tma_load_3d(base + l * R_TILE_A, &mapA, &full_bar[st], ks * RBK, P.a_row0 + m0, l);
          tc::tma_load_4d(base + RNL * R_TILE_A + l * R_TILE_B, &mapB, &full_bar[st], ks * RBK,
                          n0, b, l);
        }
        issued_sh = t + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t idesc = tc::idesc_bf16_f32(RBM, RBN);
    int t = 0, lt = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < P.ntiles && ok; tile += gridDim.x) {
      for (int kc = 0; kc < P.ksteps && ok; kc += R_CHUNK) {
        const int kce = min(P.ksteps, kc + R_CHUNK);
        const int buf = lt % R_NBUF;
        const uint32_t use = (uint32_t)(lt / R_NBUF);
        if (!tc::mbar_wait(&acce_bar[buf], (use & 1) ^ 1, abort_flag)) { ok = false; break; }
        tc::tc_fence_after();
        const uint32_t accb = tmem + buf * R_BUF_COLS;
        for (int ks = kc; ks < kce; ++ks, ++t) {
          const int st = t % RSTAGES;
          const uint32_t ph = (t / RSTAGES) & 1;
          if (!tc::mbar_wait(&full_bar[st], ph, abort_flag)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t base = tc::smem_u32(smem + st * R_STAGE);
#pragma unroll
          for (int kk = 0; kk < RBK / 16; ++kk) {
            const uint32_t first = (ks > kc || kk > 0) ? 1u : 0u;
            // limb products (i, j) of order i + j = 0..3, order by order; the
            // first product of an order in a chunk starts its accumulator
#pragma unroll
            for (int q = 0; q < 10; ++q) {
              const int o = q == 0 ? 0 : (q < 3 ? 1 : (q < 6 ? 2 : 3));
              const int i = q == 0 ? 0 : (q < 3 ? q - 1 : (q < 6 ? q - 3 : q - 6));
              const int j = o - i;
              const bool lead = (q == 0 || q == 1 || q == 3 || q == 6);
              const uint64_t ad = tc::sdesc_sw64(base + i * R_TILE_A + kk * 32);
              const uint64_t bd = tc::sdesc_sw64(base + RNL * R_TILE_A + j * R_TILE_B + kk * 32);
              tc::umma_bf16(accb + o * RBN, ad, bd, idesc, (first || !lead) ? 1u : 0u);
            }
          }
          tc::umma_commit(&empty_bar[st]);
          consumed_sh = t + 1;
        }
        if (!ok) break;
        tc::umma_commit(&accf_bar[buf]);
        committed_sh = lt + 1;
        ++lt;
      }
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int qd = warp & 3;                 // TMEM lane quarter
    const int half = (warp - 2) / 4;         // column half
    const int r = qd * 32 + lane;
    const int col0 = half * R_EPI_COLS;
    int lt = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < P.ntiles && ok; tile += gridDim.x) {
      int b, m0, n0;
      rot_decode(P, tile, b, m0, n0);
      float ah[R_EPI_COLS], al[R_EPI_COLS];
#pragma unroll
      for (int c = 0; c < R_EPI_COLS; ++c) ah[c] = al[c] = 0.f;
      for (int kc = 0; kc < P.ksteps; kc += R_CHUNK) {
        const int buf = lt % R_NBUF;
        const uint32_t use = (uint32_t)(lt / R_NBUF);
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&accf_bar[buf], use & 1, abort_flag))) { ok = false; break; }
        tc::tc_fence_after();
        const uint32_t trow = tmem + buf * R_BUF_COLS + ((uint32_t)(qd * 32) << 16);
#pragma unroll
        for (int g = 0; g < R_EPI_COLS; g += 8) {
          float a0[8], a1[8], a2[8], a3[8];
          tc::tmem_ld8(trow + 0 * RBN + col0 + g, a0);
          tc::tmem_ld8(trow + 1 * RBN + col0 + g, a1);
          tc::tmem_ld8(trow + 2 * RBN + col0 + g, a2);
          tc::tmem_ld8(trow + 3 * RBN + col0 + g, a3);
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            // chunk value a0 + 2^-8 a1 + 2^-16 a2 + 2^-24 a3 as (s, e), all
            // scalings exact (powers of two on integers below 2^24)
            float s, e;
            two_sum(a0[c], a1[c] * (1.0f / 256.0f), s, e);
            e += a2[c] * (1.0f / 65536.0f) + a3[c] * (1.0f / 16777216.0f);
            float s2, e2;
            two_sum(ah[g + c], s, s2, e2);
            ah[g + c] = s2;
            al[g + c] += e2 + e;
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acce_bar[buf]);
        ++lt;
      }
      if (!ok) break;
      const int m = m0 + r;
      if (m < P.M) {
        // (ah + al) u_a u_b: the power-of-two units as exponent shifts on the
        // integer pipe, one FP64 add per element
        const int ka = tc::pow2_exp(P.unitA[P.a_row0 + m]);
        const float* ub = P.unitB + (long long)b * P.Nn;
        double* o = P.out + (long long)m * P.sOm + (long long)b * P.sOb;
#pragma unroll
        for (int c = 0; c < R_EPI_COLS; ++c) {
          const int n = n0 + col0 + c;
          if (n < P.Nn) {
            const int k = ka + tc::pow2_exp(ub[n]);
            o[n] = tc::scale_to_double(ah[c], k) + tc::scale_to_double(al[c], k);
          }
        }
      }
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && abort_sh) {
    atomicExch(P.err, R_DEV_TIMEOUT);
    // let copies still in flight land before the shared memory goes away
    for (int t = consumed_sh; t < issued_sh; ++t) {
      const unsigned long long t0 = tc::global_ns();
      while (!tc::mbar_try_wait(&full_bar[t % RSTAGES], (t / RSTAGES) & 1) &&
             tc::global_ns() - t0 < tc::kWaitNs) {
      }
    }
  }
  if (warp == 1) {
    if (abort_sh && committed_sh > 0) {  // MMAs may still run: wait for the last commit
      const int lt = committed_sh - 1;
      const unsigned long long t0 = tc::global_ns();
      while (!tc::mbar_try_wait(&accf_bar[lt % R_NBUF], (uint32_t)((lt / R_NBUF) & 1)) &&
             tc::global_ns() - t0 < tc::kWaitNs) {
      }
    }
    __syncwarp();  // the bounded waits above may leave the lanes at different points
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, R_NBUF * R_BUF_COLS);
  }
}

// Rows of src (element (r, c) at src[r ld + c cs], c < ncol) -> four BF16
// limb planes [4][dst_rows][ncolp] of integers with the row's unit
// u = 2^(E - 7), |x| < 2^E (zero padded to ncolp); source row r lands in
// destination row (r / grp) gstride + goff + r % grp.  One warp per row.
__global__ void slice4_rows_kernel(const double* __restrict__ src, long long nrow, int ncol,
                                   long long ld, long long cs, int ncolp, long long dst_rows,
                                   long long grp, long long gstride, long long goff,
                                   __nv_bfloat16* __restrict__ dst, float* __restrict__ unit) {
  const long long plane = dst_rows * ncolp;
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; r < nrow;
       r += nwarps) {
    const double* row = src + r * ld;
    const long long dr = (r / grp) * gstride + goff + r % grp;
    unsigned long long mb = 0;  // max |x| on the integer pipe
    for (int c = lane; c < ncol; c += 32) mb = max(mb, tc::abs_bits(row[c * cs]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      mb = max(mb, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mb, o));
    const double u = tc::slice_unit(__longlong_as_double((long long)mb), 7);
    const int ku = tc::pow2_exp(u);
    __nv_bfloat16* d = dst + dr * ncolp;
    for (int c = lane; c < ncolp; c += 32) {
      // integer digits of x / u (integer pipe): |d0| <= 128, |d_l| <= 128
      int dg[RNL];
      tc::fixed_digits<RNL>((c < ncol) ? row[c * cs] : 0.0, ku, dg);
#pragma unroll
      for (int l = 0; l < RNL; ++l) d[l * plane + c] = __float2bfloat16_rn((float)dg[l]);
    }
    if (lane == 0) unit[dr] = (float)u;
  }
}

// Per (x, p): the certified unit (tc::certified_unit) of the row (x, p) over
// Q, from tc::RowStats (integer and FP32 pipes).  Block of 32 p x 8 Q-groups
// (coalesced over p), grid (ceil(N / 32), nx).
__global__ void col_stats_kernel(const double* __restrict__ W, int nQ, int N, int Qs,
                                 double* __restrict__ unit_out) {
  __shared__ unsigned long long smb[8][32];
  __shared__ float ss2[8][32], ss1[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + tx;
  const int x = blockIdx.y;
  tc::RowStats st;
  if (p < N) {
    const double* w = W + (long long)x * nQ * N + p;
    for (int Q = ty; Q < nQ; Q += 8) st.add(w[(long long)Q * N]);
  }
  smb[ty][tx] = st.mb;
  ss2[ty][tx] = st.s2;
  ss1[ty][tx] = st.s1;
  __syncthreads();
  if (ty != 0 || p >= N) return;
  for (int g = 1; g < 8; ++g) st.merge(smb[g][tx], ss2[g][tx], ss1[g][tx]);
  double u;
  if (!st.unit((double)Qs, u)) {  // a bound overflowed the float range: FP64 sums
    const double* w = W + (long long)x * nQ * N + p;
    double s2 = 0.0, s1 = 0.0;
    for (int Q = 0; Q < nQ; ++Q) {
      const double v = fabs(w[(long long)Q * N]);
      s2 = fma(v, v, s2);
      s1 += v;
    }
    u = tc::certified_unit(__longlong_as_double((long long)st.mb), s2, s1, (double)Qs);
  }
  unit_out[(long long)x * N + p] = u;
}

// W[x][Q][p] -> three BF16 limb planes of the rows (x, p) over Q (rows
// x0 N + x N + p of planes [3][dst_rows][Qs]) with the row units of
// col_stats_kernel (every h0 h0' partial sum of the pair GEMM exact).
// Block (32 x 8 threads) per (x, 32 p, 32 Q) tile, transposed through
// shared memory so both the reads (over p) and the writes (over Q) coalesce.
__global__ void transpose_slice3_kernel(const double* __restrict__ W, int nQ, int N, int Qs,
                                        const double* __restrict__ unit_in, long long dst_rows,
                                        long long row0, __nv_bfloat16* __restrict__ dst,
                                        float* __restrict__ unit) {
  __shared__ double tile[32][33];
  __shared__ int ku_sh[32];
  const int x = blockIdx.z;
  const int p0 = blockIdx.x * 32, Q0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const double* w = W + (long long)x * nQ * N;
  for (int j = ty; j < 32; j += 8) {
    const int Q = Q0 + j, p = p0 + tx;
    tile[j][tx] = (Q < nQ && p < N) ? w[(long long)Q * N + p] : 0.0;
  }
  if (ty == 0) {
    const int p = p0 + tx;
    ku_sh[tx] = (p < N) ? tc::pow2_exp(unit_in[(long long)x * N + p]) : 0;
  }
  __syncthreads();
  const long long plane = dst_rows * Qs;
  for (int j = ty; j < 32; j += 8) {
    const int p = p0 + j, Q = Q0 + tx;
    if (p >= N || Q >= Qs) continue;
    const long long dr = row0 + (long long)x * N + p;
    __nv_bfloat16 h0, h1, h2;
    tc::slice3_int(tile[tx][j], ku_sh[j], h0, h1, h2);
    __nv_bfloat16* d = dst + dr * Qs + Q;
    d[0] = h0;
    d[plane] = h1;
    d[2 * plane] = h2;
    if (Q == 0) unit[dr] = (float)unit_in[(long long)x * N + p];
  }
}

PFN_cuTensorMapEncodeTiled_v12000 rot_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool rot_map(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims,
             const cuuint64_t* strides_bytes, const cuuint32_t* box, std::string& err) {
  auto enc = rot_encode();
  if (!enc) {
    err = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, const_cast<void*>(base), dims,
                   strides_bytes, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

std::mutex g_rot_mu;
bool g_rot_attr[64] = {false};

}  // namespace

int rot_limbs_slice4(const double* src, long long nrow, int ncol, long long ld, long long cs,
                     int ncolp, long long dst_rows, long long grp, long long gstride,
                     long long goff, __nv_bfloat16* dst, float* unit, cudaStream_t s) {
  const long long blocks = std::min<long long>((nrow + 7) / 8, 152LL * 16);
  slice4_rows_kernel<<<(int)std::max(1LL, blocks), 256, 0, s>>>(
      src, nrow, ncol, ld, cs, ncolp, dst_rows, grp, gstride, goff, dst, unit);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? AGF2_OK : AGF2_ERR_CUDA;
}

int rot_transpose_slice3(const double* W, int nx, int nQ, int N, int Qs, double* stats,
                         long long dst_rows, long long row0, __nv_bfloat16* dst, float* unit,
                         cudaStream_t s) {
  col_stats_kernel<<<dim3((N + 31) / 32, nx), 256, 0, s>>>(W, nQ, N, Qs, stats);
  transpose_slice3_kernel<<<dim3((N + 31) / 32, (Qs + 31) / 32, nx), dim3(32, 8), 0, s>>>(
      W, nQ, N, Qs, stats, dst_rows, row0, dst, unit);
  count_launch(2);
  return cudaGetLastError() == cudaSuccess ? AGF2_OK : AGF2_ERR_CUDA;
}

int rot_gemm4(const __nv_bfloat16* A, long long rowsA, int a_row0, int M, const float* unitA,
              const __nv_bfloat16* B, int Nn, int nbatch, const float* unitB, int Ks,
              double* out, long long sOm, long long sOb, int* derr, std::string& err,
              cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(g_rot_mu);
    if (!g_rot_attr[dev & 63]) {
      if (cudaFuncSetAttribute(rot4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               R_SMEM) != cudaSuccess) {
        err = "cudaFuncSetAttribute(rot4 smem) failed";
        return AGF2_ERR_CUDA;
      }
      g_rot_attr[dev & 63] = true;
    }
  }
  if (Ks % 256 != 0) {
    err = "rotation GEMM: K padding must be a multiple of 256";
    return AGF2_ERR_INVALID_ARG;
  }
  CUtensorMap mapA, mapB;
  {
    cuuint64_t dims[3] = {(cuuint64_t)Ks, (cuuint64_t)rowsA, (cuuint64_t)RNL};
    cuuint64_t str[2] = {(cuuint64_t)Ks * 2, (cuuint64_t)rowsA * Ks * 2};
    cuuint32_t box[3] = {RBK, RBM, 1};
    if (!rot_map(&mapA, A, 3, dims, str, box, err)) return AGF2_ERR_CUDA;
  }
  {
    cuuint64_t dims[4] = {(cuuint64_t)Ks, (cuuint64_t)Nn, (cuuint64_t)nbatch, (cuuint64_t)RNL};
    cuuint64_t str[3] = {(cuuint64_t)Ks * 2, (cuuint64_t)Nn * Ks * 2,
                         (cuuint64_t)nbatch * Nn * Ks * 2};
    cuuint32_t box[4] = {RBK, RBN, 1, 1};
    if (!rot_map(&mapB, B, 4, dims, str, box, err)) return AGF2_ERR_CUDA;
  }
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  RotParams P{};
  P.M = M;
  P.Nn = Nn;
  P.ksteps = Ks / RBK;
  P.nbatch = nbatch;
  P.a_row0 = a_row0;
  P.m_tiles = (M + RBM - 1) / RBM;
  P.n_tiles = (Nn + RBN - 1) / RBN;
  P.ntiles = P.m_tiles * P.n_tiles * nbatch;
  P.unitA = unitA;
  P.unitB = unitB;
  P.out = out;
  P.sOm = sOm;
  P.sOb = sOb;
  P.err = derr;
  rot4_kernel<<<std::min(P.ntiles, nsm), R_THREADS, R_SMEM, s>>>(mapA, mapB, P);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("rotation kernel launch: ") + cudaGetErrorString(e);
    return AGF2_ERR_CUDA;
  }
  return AGF2_OK;
}

}  // namespace agf2
