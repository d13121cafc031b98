// Split-precision moment build on the tcgen05 tensor cores (AGF2_BF16X3).
//
// The self-energy moments of Eqs. (mp2_zeroth_moment), (mp2_first_moment)
// and their higher analogues (weights w^n, n <= nmom <= 3) are evaluated over
// unordered pole pairs (x <= y) of the summed outer index (i,j occupied for
// the hole sector; a,b virtual for the particle sector):
//
//   X_xy[p,c] = sum_Q Lx[x][p][Q] Lpair[y][c][Q]        (GEMM 1, K = n_Q)
//   S = X_xy + X_yx,  D = X_xy - X_yx,  w = e_x + e_y - e_c
//   Y  = [ sqrt(cS) S | sqrt(cD) D ]
//   U^(n) += (Y w^n) Y^T,  n = 0 .. nmom                 (GEMM 2, K = pairs x c)
//
// with (cS, cD) = (1/2, 3/2) for x < y and (1/4, 3/4) for x = y, which is
// the pair-symmetrised form of sum_{xyc} X_xy (2 X_xy - X_yx) w^n (the
// exchange partner X_yx of an ordered pair is the other ordered pair, so
// GEMM 1 runs once per ordered pair).
//
// Every operand row is sliced in fixed point with a per-row power-of-two unit
// into three BF16 limbs (x ~ unit (h0 + h1 + h2), h0 an integer, see
// tc_core.cuh).  Each GEMM keeps the six limb products h_a h_b (a + b <= 2)
// in two FP32 tensor-memory accumulators: h0 h0' alone (integer-valued, so
// the tensor core adds it exactly) and the five smaller products.  Separate
// accumulators matter: the tensor core truncates when it adds into an FP32
// accumulator, which over long K biases a single accumulator by ~2^-25 per
// instruction.  GEMM 2 drains its tiles into the FP64 moments.
//
// Kernels: slice_rows_kernel (FP64 rotated rows -> limb planes),
// gemm6_kernel<MODE_PAIR> (GEMM 1, writing X in FP32 for a block of pairs; its
// epilogue also takes the exact per-row maxima of every Y w^n),
// combine_kernel (S/D and energy weights; fixed-point limb planes of every
// Y w^n with the rows' units),
// gemm6_kernel<MODE_MOMENT> (GEMM 2 for every moment, upper tiles, split-K,
// FP64 atomics), mirror_tiles_kernel (the lower tiles).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/agf2.h"
#include "agf2_internal.h"
#include "tc_core.cuh"

namespace agf2 {

namespace {

constexpr int BM = 128;         // MMA M (rows of p)
constexpr int BN = 128;         // MMA N
constexpr int BK = 32;          // K elements per stage (64 B rows, 64-byte swizzle)
constexpr int STAGES = 4;       // 4 x 48 KB: three stages in flight while one is consumed
constexpr int TILE_A = BM * BK * 2;     // bytes of one A limb tile
constexpr int TILE_B = BN * BK * 2;     // bytes of one B limb tile
constexpr int STAGE_BYTES = 3 * TILE_A + 3 * TILE_B;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr int TMEM_COLS = 512;  // PAIR: (hi, lo) x (X_xy, X_yx) x BN; MOMENT: (hi, lo) x BN
constexpr int KCHUNK = 2 * BN;  // K entries of Y one PAIR tile writes: S and D of BN c's
constexpr int NTHREADS = 320;   // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue

enum { MODE_PAIR = 0, MODE_MOMENT = 1 };

// Device error codes (written to a device int).
enum { DEV_OK = 0, DEV_TIMEOUT = 1 };

constexpr int MAXM = 4;  // moments 0..3 on the split-precision path

// a + b for unevaluated float pairs (hi, lo), renormalised (Knuth's TwoSum on
// the high parts): about 2^-44 relative, so e_x + e_y - e_c rounds to FP32 as
// the FP64 sum would (within an ulp) at FP32 rather than FP64 throughput.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bb = s - a.x;
  const float e = (a.x - (s - bb)) + (b.x - bb);
  const float t = e + (a.y + b.y);
  const float hi = s + t;
  return make_float2(hi, t - (hi - s));
}

// e[i] -> (hi, lo) float pair with hi + lo = e[i] to about 2^-48 relative.
__global__ void float_pair_kernel(const double* __restrict__ e, int n, float2* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float hi = (float)e[i];
  out[i] = make_float2(hi, (float)(e[i] - (double)hi));
}

// Pair-symmetrised operand values for one (row, pair, inner pole): from
// X_xy = a0 and X_yx = a1 (a1 = a0 on a diagonal pair x = y),
//   Y_S = sqrt(cS) (a0 + a1), Y_D = sqrt(cD) (a0 - a1),
// (cS, cD) = (1/2, 3/2) off the diagonal and (1/4, 0) on it, with sqrt(cS),
// sqrt(cD) as unevaluated float pairs: a rounded FP32 constant would enter
// U^(0) = Y Y^T squared and bias its diagonal (~7e-8).  The pair GEMM's
// epilogue (row maxima) and the slicing pass call this same function on the
// same FP32 inputs, so both see bit-identical Y.
__device__ __forceinline__ void sd_values(float a0, float a1, bool diag, float& ys, float& yd) {
  const float sS = diag ? 0.5f : 0.7071067690849304f;
  const float sS_lo = diag ? 0.0f : 1.2101617485882343e-08f;
  const float sD = diag ? 0.0f : 1.2247449159622192f;
  const float sD_lo = diag ? 0.0f : -4.4570629853524224e-08f;
  const float sum = a0 + a1, dif = a0 - a1;
  ys = fmaf(sum, sS, sum * sS_lo);
  yd = fmaf(dif, sD, dif * sD_lo);
}

// Energy weight e_x + e_y - e_c rounded to FP32, from float pairs
// (ex = e_x + e_y already summed).
__device__ __forceinline__ float pair_weight(float2 ex, float2 ec) {
  const float2 w = df_add(ex, make_float2(-ec.x, -ec.y));
  return w.x + w.y;
}

struct Params {
  int N;            // physical orbitals (rows of U)
  int n_in;         // inner pole count (c index)
  int ksteps;       // K steps of GEMM 1 (Qs / BK) or of GEMM 2 in total
  int n_ptiles;     // ceil(N / BM)
  int n_cchunks;    // MODE_PAIR: ceil(n_in / BN)
  int n_qtiles;     // MODE_MOMENT: ceil(N / BN)
  int n_out;        // outer pole count (limb stride of the A map)
  int hole;         // MODE_PAIR: 1 -> B rows along map dim 1, 0 -> along dim 2
  int pair0;        // first pair of this block
  int ksplit;       // MODE_MOMENT: K steps per CTA
  int nsplit;       // MODE_MOMENT: K splits per (tile, moment)
  int ntiles;       // tiles of this launch (the persistent CTAs loop over them)
  const int2* pairs;
  const float2* e_out2;  // MODE_PAIR: pole energies as float pairs (outer, inner)
  const float2* e_in2;
  unsigned* maxbits;     // MODE_PAIR: [nm][N] row maxima of |Y w^n| (float bits)
  const float* unitA;   // MODE_PAIR: slicing unit of Lx rows [x][p]; MOMENT: [nm][N] of Y w^n rows
  const float* unitB;   // MODE_PAIR: unit of Lov rows [i][a];        MOMENT: of Y rows
  int nm;               // moments computed (nmom + 1)
  int v_stride;         // MODE_PAIR: v (row index of Lov rows is i * v + a)
  float* X;            // MODE_PAIR output: FP32 X_xy [N][np][2][ncp] (row stride Ks)
  int ncp;             // MODE_PAIR: n_cchunks * BN (padded inner count)
  long long Ks;
  long long plane;     // N * Ks
  double* U0;          // MODE_MOMENT: [nm][N][N]
  int* err;
};

// K steps of one moment-GEMM accumulation: KCHUNK = 256 entries.  With
// |h0| <= 256, every partial sum of a chunk's h0 h0' products is an integer
// of magnitude <= 2^24, exact in the FP32 accumulator, and the correction
// products see at most 16 instructions of FP32 accumulation; the epilogue
// sums the chunks of a tile in registers (round to nearest).
constexpr int CHUNK_STEPS = KCHUNK / BK;
// Chunks per moment-GEMM tile at most (bounds the register sum's rounding).
constexpr int MAX_TILE_CHUNKS = 8;

struct Segment {
  int a_row, a_idx;   // A tile: rows a_row.., outer index / plane a_idx
  int b_row, b_idx;   // B tile
  int acc_col;        // accumulator column offset
  int kbeg, kend;     // K steps
  int a_plane;        // MODE_MOMENT: moment n (A rows are Y w^n)
};

__device__ __forceinline__ void load_a(const CUtensorMap* mapA, uint8_t* dst, uint64_t* bar,
                                       const Params& P, const Segment& s, int ks, int limb) {
  if (P.n_out > 0)  // MODE_PAIR: A map dims (Qs, N, 3*n_out)
    tc::tma_load_3d(dst, mapA, bar, ks * BK, s.a_row, limb * P.n_out + s.a_idx);
  else              // MODE_MOMENT: map over [nm][3] planes of Y w^n, dims (K, N, 3 nm)
    tc::tma_load_3d(dst, mapA, bar, ks * BK, s.a_row, s.a_plane * 3 + limb);
}

// Work of one tile: one K segment into one accumulator set (nseg = 0: no
// work, the tile is skipped by every role).
struct TileWork {
  Segment seg[1];
  int nseg;
  int p0, c0, q0, moment, pair_local, orient;
  int2 pr;
};

template <int MODE>
__device__ __forceinline__ TileWork decode_tile(const Params& P, int t) {
  TileWork w;
  w.nseg = 1;
  w.p0 = w.c0 = w.q0 = w.moment = w.pair_local = w.orient = 0;
  w.pr = make_int2(0, 0);
  if (MODE == MODE_PAIR) {
    // ordered pair (x, y) (orient 0) or (y, x) (orient 1) of unordered pair
    // x <= y; the two orientations of one (pair, p-tile, chunk) are
    // consecutive tiles, taken by the same CTA (next_tile)
    w.orient = t & 1;
    int b = t >> 1;
    const int cc = b % P.n_cchunks; b /= P.n_cchunks;
    const int pt = b % P.n_ptiles; b /= P.n_ptiles;
    w.pair_local = b;
    w.pr = P.pairs[P.pair0 + w.pair_local];
    w.p0 = pt * BM;
    w.c0 = cc * BN;
    const int xa = w.orient ? w.pr.y : w.pr.x, yb = w.orient ? w.pr.x : w.pr.y;
    w.seg[0] = Segment{w.p0, xa, w.c0, yb, 0, 0, P.ksteps, 0};
    if (w.orient && w.pr.x == w.pr.y) w.nseg = 0;  // X_yx == X_xy on the diagonal
  } else {
    // U is symmetric: only tiles with qt >= pt (upper triangle of tiles).
    // Split-major order: the (tile, moment) items of one K split are
    // neighbours, so the CTAs that read the same K range of the Y planes run
    // together and share it through L2 instead of each fetching it from HBM.
    const int ntm = P.n_ptiles * (P.n_ptiles + 1) / 2 * P.nm;
    int b = t % ntm;
    const int sp = t / ntm;
    w.moment = b % P.nm; b /= P.nm;
    int pt = 0, qt = 0;
    for (int r = 0, left = b; r < P.n_ptiles; ++r) {
      const int row = P.n_ptiles - r;  // tiles qt = r .. n_ptiles - 1
      if (left < row) { pt = r; qt = r + left; break; }
      left -= row;
    }
    w.p0 = pt * BM;
    w.q0 = qt * BN;
    const int kb = sp * P.ksplit;
    const int ke = min(P.ksteps, kb + P.ksplit);
    w.seg[0] = Segment{w.p0, 0, w.q0, 0, 0, kb, ke, w.moment};
  }
  return w;
}

// Tile order of the persistent CTAs.  MODE_PAIR: CTA b takes tiles 2s and
// 2s + 1 (the two orientations of one pair tile) for s = b, b + grid, ..., so
// its epilogue still holds X_xy when X_yx arrives; MODE_MOMENT: b, b + grid, ...
template <int MODE>
__device__ __forceinline__ int first_tile() {
  return MODE == MODE_PAIR ? 2 * (int)blockIdx.x : (int)blockIdx.x;
}
template <int MODE>
__device__ __forceinline__ int next_tile(int t) {
  if (MODE == MODE_PAIR) return (t & 1) ? t + 2 * (int)gridDim.x - 1 : t + 1;
  return t + (int)gridDim.x;
}

// Persistent kernel: CTA b handles the tiles of first_tile / next_tile
//   warp 0: TMA producer (runs ahead across tiles through the smem ring)
//   warp 1: TMEM allocation + single-thread tcgen05.mma issue
//   warps 2..9: epilogue; warp w reads TMEM lane quarter w % 4 and column
//   half (w - 2) / 4 of each accumulator
// Each tile's accumulator set (h0h0 "hi" and correction "lo", BN columns each)
// takes 256 TMEM columns; two sets are double-buffered so a tile's epilogue
// overlaps the next tile's MMAs.
template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 1)
gemm6_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
             const Params P) {
  constexpr int NBUF = 2;
  constexpr int BUF_COLS = 2 * BN;
  constexpr int N_EPI_WARPS = (NTHREADS / 32) - 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t accf_bar[NBUF];   // MMA -> epilogue
  __shared__ __align__(8) uint64_t acce_bar[NBUF];   // epilogue -> MMA
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  __shared__ int issued_sh, consumed_sh, committed_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort_flag = &abort_sh;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      tc::mbar_init(&accf_bar[b], 1);
      tc::mbar_init(&acce_bar[b], N_EPI_WARPS);
    }
    abort_sh = 0;
    issued_sh = 0;
    consumed_sh = 0;
    committed_sh = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_base_sh, TMEM_COLS);
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
    for (int tile = first_tile<MODE>(); tile < P.ntiles && ok; tile = next_tile<MODE>(tile)) {
      const TileWork w = decode_tile<MODE>(P, tile);
      for (int si = 0; si < w.nseg && ok; ++si) {
        const Segment& s = w.seg[si];
        for (int ks = s.kbeg; ks < s.kend; ++ks, ++t) {
          const int st = t % STAGES;
          const uint32_t ph = (t / STAGES) & 1;
          if (!tc::mbar_wait(&empty_bar[st], ph ^ 1, abort_flag)) { ok = false; break; }
          uint8_t* base = smem + st * STAGE_BYTES;
          tc::mbar_arrive_expect_tx(&full_bar[st], STAGE_BYTES);
          for (int l = 0; l < 3; ++l) {
            if (MODE == MODE_PAIR) {
              load_a(&mapA, base + l * TILE_A, &full_bar[st], P, s, ks, l);
              if (P.hole)
                tc::tma_load_4d(base + 3 * TILE_A + l * TILE_B, &mapB, &full_bar[st], ks * BK,
                                s.b_row, s.b_idx, l);
              else
                tc::tma_load_4d(base + 3 * TILE_A + l * TILE_B, &mapB, &full_bar[st], ks * BK,
                                s.b_idx, s.b_row, l);
            } else {
              load_a(&mapA, base + l * TILE_A, &full_bar[st], P, s, ks, l);
              tc::tma_load_3d(base + 3 * TILE_A + l * TILE_B, &mapB, &full_bar[st], ks * BK,
                              s.b_row, l);
            }
          }
          issued_sh = t + 1;
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
    // correction products h_a h_b (a + b = 1, 2) into the lo accumulator
    const int pa[5] = {2, 1, 0, 1, 0};
    const int pb[5] = {0, 1, 2, 0, 1};
    int t = 0, lt = 0;
    bool ok = true;
    for (int tile = first_tile<MODE>(); tile < P.ntiles && ok; tile = next_tile<MODE>(tile)) {
      const TileWork w = decode_tile<MODE>(P, tile);
      if (w.nseg == 0) continue;
      const Segment& s = w.seg[0];
      // one accumulator use per chunk (MOMENT) or per tile (PAIR)
      const int span = (MODE == MODE_MOMENT) ? CHUNK_STEPS : (s.kend - s.kbeg);
      for (int kc = s.kbeg; kc < s.kend && ok; kc += span) {
        const int kce = min(s.kend, kc + span);
        const int buf = lt % NBUF;
        const uint32_t use = (uint32_t)(lt / NBUF);
        // wait until the epilogue has drained this accumulator set
        if (!tc::mbar_wait(&acce_bar[buf], (use & 1) ^ 1, abort_flag)) { ok = false; break; }
        tc::tc_fence_after();
        const uint32_t acc_hi = tmem + buf * BUF_COLS + s.acc_col;
        const uint32_t acc_lo = acc_hi + BN;
        for (int ks = kc; ks < kce; ++ks, ++t) {
          const int st = t % STAGES;
          const uint32_t ph = (t / STAGES) & 1;
          if (!tc::mbar_wait(&full_bar[st], ph, abort_flag)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t base = tc::smem_u32(smem + st * STAGE_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint32_t acc = (ks > kc || kk > 0) ? 1u : 0u;
#pragma unroll
            for (int pi = 0; pi < 5; ++pi) {
              const uint64_t ad = tc::sdesc_sw64(base + pa[pi] * TILE_A + kk * 32);
              const uint64_t bd = tc::sdesc_sw64(base + 3 * TILE_A + pb[pi] * TILE_B + kk * 32);
              tc::umma_bf16(acc_lo, ad, bd, idesc, (acc || pi > 0) ? 1u : 0u);
            }
            tc::umma_bf16(acc_hi, tc::sdesc_sw64(base + kk * 32),
                          tc::sdesc_sw64(base + 3 * TILE_A + kk * 32), idesc, acc);
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
    const int qd = warp & 3;                        // TMEM lane quarter of this warp
    const int half = (warp - 2) / 4;                // column half of each accumulator
    const int r = qd * 32 + lane;
    const int col0 = half * (BN / 2);
    int lt = 0;
    bool ok = true;
    for (int tile = first_tile<MODE>(); tile < P.ntiles && ok; tile = next_tile<MODE>(tile)) {
      const TileWork w = decode_tile<MODE>(P, tile);
      if (w.nseg == 0) continue;
      const int p = w.p0 + r;
      if (MODE == MODE_PAIR) {
        const int buf = lt % NBUF;
        const uint32_t use = (uint32_t)(lt / NBUF);
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&accf_bar[buf], use & 1, abort_flag))) break;
        tc::tc_fence_after();
        const uint32_t trow = tmem + buf * BUF_COLS + ((uint32_t)(qd * 32) << 16);
        // X[p][pair][orient][c] = (hi + lo) * unit(A row) * unit(B row), FP32
        const Segment& sg = w.seg[0];
        const bool prow = p < P.N;
        const float uA = prow ? P.unitA[(long long)sg.a_idx * P.N + p] : 0.f;
        float* xrow = P.X + (long long)p * P.Ks +
                      ((long long)w.pair_local * 2 + w.orient) * P.ncp + w.c0 + col0;
        // with both orders of the pair tile at hand (orient 1, or orient 0 of a
        // diagonal pair), the exact row maxima of |Y w^n| over this tile's
        // columns, folded into the block's per-row maxima; X_xy comes back
        // from this thread's own stores of the previous tile (same CTA)
        const bool diag = w.pr.x == w.pr.y;
        const bool take_max = prow && (w.orient == 1 || diag);
        float2 ex = make_float2(0.f, 0.f);
        if (take_max) ex = df_add(P.e_out2[w.pr.x], P.e_out2[w.pr.y]);
        float mx[MAXM];
#pragma unroll
        for (int n = 0; n < MAXM; ++n) mx[n] = 0.f;
#pragma unroll
        for (int cb = 0; cb < BN / 2; cb += 16) {
          float hi[16], lo[16], xv[16];
          tc::tmem_ld16(trow + col0 + cb, hi);
          tc::tmem_ld16(trow + BN + col0 + cb, lo);
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int ci = w.c0 + col0 + cb + c;
            float x = 0.f;
            if (prow && ci < P.n_in) {
              // B-row units: hole rows (y, c) -> y*v + c ; particle rows (c, y) -> c*v + y
              const long long rb = P.hole ? (long long)sg.b_idx * P.v_stride + ci
                                          : (long long)ci * P.v_stride + sg.b_idx;
              x = (hi[c] + lo[c]) * (uA * P.unitB[rb]);
            }
            xv[c] = x;
          }
          if (prow) {
#pragma unroll
            for (int g = 0; g < 16; g += 4)
              *reinterpret_cast<float4*>(xrow + cb + g) =
                  make_float4(xv[g], xv[g + 1], xv[g + 2], xv[g + 3]);
          }
          if (take_max) {
            float a0[16];  // X_xy
#pragma unroll
            for (int g = 0; g < 16; g += 4) {
              float4 t4 = diag ? make_float4(xv[g], xv[g + 1], xv[g + 2], xv[g + 3])
                               : *reinterpret_cast<const float4*>(xrow - P.ncp + cb + g);
              a0[g] = t4.x;
              a0[g + 1] = t4.y;
              a0[g + 2] = t4.z;
              a0[g + 3] = t4.w;
            }
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const int ci = w.c0 + col0 + cb + c;
              if (ci < P.n_in) {
                float ys, yd;
                sd_values(a0[c], xv[c], diag, ys, yd);
                const float wt = pair_weight(ex, P.e_in2[ci]);
#pragma unroll
                for (int n = 0; n < MAXM; ++n) {
                  if (n >= P.nm) break;
                  mx[n] = fmaxf(mx[n], fmaxf(fabsf(ys), fabsf(yd)));
                  ys *= wt;
                  yd *= wt;
                }
              }
            }
          }
        }
        // this accumulator set may be overwritten once every epilogue warp is done
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acce_bar[buf]);
        ++lt;
        if (take_max) {
#pragma unroll
          for (int n = 0; n < MAXM; ++n)
            if (n < P.nm) atomicMax(P.maxbits + (long long)n * P.N + p, __float_as_uint(mx[n]));
        }
      } else {
        // U^(n)[p][q] += u(p) u(q) sum over the tile's chunks of (hi + lo):
        // chunks summed in FP32 registers, one FP64 atomic per element
        const Segment& sg = w.seg[0];
        float acc[BN / 2];
#pragma unroll
        for (int c = 0; c < BN / 2; ++c) acc[c] = 0.f;
        for (int kc = sg.kbeg; kc < sg.kend; kc += CHUNK_STEPS) {
          const int buf = lt % NBUF;
          const uint32_t use = (uint32_t)(lt / NBUF);
          if (!__all_sync(0xffffffffu, tc::mbar_wait(&accf_bar[buf], use & 1, abort_flag))) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t trow = tmem + buf * BUF_COLS + ((uint32_t)(qd * 32) << 16);
#pragma unroll
          for (int g = 0; g < BN / 2; g += 16) {
            float hi[16], lo[16];
            tc::tmem_ld16(trow + col0 + g, hi);
            tc::tmem_ld16(trow + BN + col0 + g, lo);
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[g + c] += hi[c] + lo[c];
          }
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&acce_bar[buf]);
          ++lt;
        }
        if (!ok) break;
        if (p < P.N) {
          double* U = P.U0 + (long long)w.moment * P.N * P.N + (long long)p * P.N;
          // acc u(p) u(q) with power-of-two units: an exponent shift, formed
          // on the integer pipe (scale_to_double), then the FP64 atomic
          const int kA = tc::pow2_exp(P.unitA[(long long)w.moment * P.N + p]);
#pragma unroll
          for (int c = 0; c < BN / 2; ++c) {
            const int q = w.q0 + col0 + c;
            if (q < P.N && acc[c] != 0.f)
              atomicAdd(U + q, tc::scale_to_double(acc[c], kA + tc::pow2_exp(P.unitB[q])));
          }
        }
      }
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && abort_sh) {
    atomicExch(P.err, DEV_TIMEOUT);
    // let copies still in flight land before the shared memory goes away
    for (int t = consumed_sh; t < issued_sh; ++t) {
      const unsigned long long t0 = tc::global_ns();
      while (!tc::mbar_try_wait(&full_bar[t % STAGES], (t / STAGES) & 1) &&
             tc::global_ns() - t0 < tc::kWaitNs) {
      }
    }
  }
  if (warp == 1) {
    if (abort_sh && committed_sh > 0) {  // MMAs may still be running: wait for the last commit
      const int lt = committed_sh - 1;
      const unsigned long long t0 = tc::global_ns();
      while (!tc::mbar_try_wait(&accf_bar[lt % NBUF], (uint32_t)((lt / NBUF) & 1)) &&
             tc::global_ns() - t0 < tc::kWaitNs) {
      }
    }
    __syncwarp();  // the bounded waits above may leave the lanes at different points
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
}

// FP64 rows [nrow][ncol] (row stride ld) -> three BF16 limb planes
// [3][dst_rows][ncolp] (zero padded to ncolp) in fixed point with the row's
// certified power-of-two unit (tc::certified_unit: every h0 h0' partial sum of
// the pair GEMM, K = the whole row, is exact).  Source row r lands in
// destination row (r / grp) * gstride + goff + r % grp, which places a block
// of rotated rows inside the full limb planes.  One warp per row.
template <class T>
__global__ void slice_rows_kernel(const T* __restrict__ src, long long nrow, int ncol,
                                  long long ld, int ncolp, long long dst_rows, long long grp,
                                  long long gstride, long long goff,
                                  __nv_bfloat16* __restrict__ dst, float* __restrict__ unit) {
  const long long plane = dst_rows * ncolp;
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long r = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; r < nrow;
       r += nwarps) {
    const T* row = src + r * ld;
    const long long dr = (r / grp) * gstride + goff + r % grp;
    tc::RowStats st;  // integer and FP32 pipes only
    for (int c = lane; c < ncol; c += 32) st.add((double)row[c]);
    st.warp_reduce();
    double u;
    if (!st.unit((double)ncolp, u)) {  // a bound overflowed the float range: FP64 sums
      double s2 = 0.0, s1 = 0.0;
      for (int c = lane; c < ncol; c += 32) {
        const double x = fabs((double)row[c]);
        s2 = fma(x, x, s2);
        s1 += x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      }
      u = tc::certified_unit(__longlong_as_double((long long)st.mb), s2, s1, (double)ncolp);
    }
    const int ku = tc::pow2_exp(u);
    __nv_bfloat16* d = dst + dr * ncolp;
    for (int c = lane; c < ncolp; c += 32) {
      __nv_bfloat16 h0, h1, h2;
      tc::slice3_int((c < ncol) ? (double)row[c] : 0.0, ku, h0, h1, h2);
      d[c] = h0;
      d[plane + c] = h1;
      d[2 * plane + c] = h2;
    }
    if (lane == 0) unit[dr] = (float)u;
  }
}

// Slicing pass of GEMM 2's operands (Eqs. mp2_zeroth_moment /
// mp2_first_moment in S/D form): for unordered pair (x, y), inner pole c and
// row p, Y_S, Y_D from X_xy, X_yx (sd_values) and Yw^n = (e_x + e_y - e_c)^n Y,
// sliced in fixed point with each row's unit from the exact row maxima that
// the pair GEMM's epilogue took over the whole block, into the limb planes at
// K index pair * kpp + chunk * 256 + (S: c, D: 128 + c).  Exact maxima
// matter: a unit from a bound (e.g. sqrt(6) max|X|) coarsens the grid and the
// squared rounding error biases diag U^(0) (measured +1e-8 relative).  Four
// consecutive c per thread; grid = (blocks over pair x inner / 4, N rows).
struct Combine {
  const float* X;
  long long xrow;  // row stride of X
  int np, ncp, n_in, N, kpp, pair0, nm;
  const int2* pairs;
  const float2* e_out;  // pole energies as unevaluated float pairs (hi, lo)
  const float2* e_in;
  unsigned* maxbits;   // [nm][N]: max |Y w^n| per row
  __nv_bfloat16* Y;    // [nm][3][N][Ks] limb planes of Y w^n
  long long Ks, plane; // plane = N Ks
  float* unit;         // [nm][N]
};

__device__ __forceinline__ void store4(__nv_bfloat16* base, long long plane, long long k,
                                       const __nv_bfloat16 (&h)[3][4]) {
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    __nv_bfloat162 a = __halves2bfloat162(h[l][0], h[l][1]);
    __nv_bfloat162 b = __halves2bfloat162(h[l][2], h[l][3]);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&a);
    u.y = *reinterpret_cast<uint32_t*>(&b);
    *reinterpret_cast<uint2*>(base + l * plane + k) = u;
  }
}

__global__ void __launch_bounds__(256) combine_kernel(const Combine C) {
  const int p = blockIdx.y;
  const int nq = C.ncp / 4;  // groups of 4 inner poles per pair
  const int total = C.np * nq;
  float iu[MAXM];
#pragma unroll
  for (int n = 0; n < MAXM; ++n)
    iu[n] = n < C.nm
                ? 1.0f / tc::slice_unitf(__uint_as_float(C.maxbits[(long long)n * C.N + p]), 8)
                : 1.f;
  const float* xr = C.X + (long long)p * C.xrow;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int pl = e / nq, c0 = (e - pl * nq) * 4;
    const int2 pr = C.pairs[C.pair0 + pl];
    const bool diag = pr.x == pr.y;
    const float4 x0 = *reinterpret_cast<const float4*>(xr + (2LL * pl) * C.ncp + c0);
    const float4 x1 = diag ? x0 : *reinterpret_cast<const float4*>(xr + (2LL * pl + 1) * C.ncp + c0);
    const float2 ex = df_add(C.e_out[pr.x], C.e_out[pr.y]);
    const float a0[4] = {x0.x, x0.y, x0.z, x0.w};
    const float a1[4] = {x1.x, x1.y, x1.z, x1.w};
    float ys[4], yd[4], wt[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + j;
      ys[j] = yd[j] = wt[j] = 0.f;
      if (c < C.n_in) {
        sd_values(a0[j], a1[j], diag, ys[j], yd[j]);
        wt[j] = pair_weight(ex, C.e_in[c]);
      }
    }
    const long long k = (long long)pl * C.kpp + (c0 / BN) * KCHUNK + (c0 % BN);
#pragma unroll
    for (int n = 0; n < MAXM; ++n) {
      if (n >= C.nm) break;
      __nv_bfloat16 hs[3][4], hd[3][4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        tc::slice3f(ys[j] * iu[n], hs[0][j], hs[1][j], hs[2][j]);
        tc::slice3f(yd[j] * iu[n], hd[0][j], hd[1][j], hd[2][j]);
      }
      __nv_bfloat16* base = C.Y + (long long)n * 3 * C.plane + (long long)p * C.Ks;
      store4(base, C.plane, k, hs);
      store4(base, C.plane, k + BN, hd);
      // next power: Y w^(n+1)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        ys[j] *= wt[j];
        yd[j] *= wt[j];
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < C.nm)
    C.unit[(long long)threadIdx.x * C.N + p] =
        tc::slice_unitf(__uint_as_float(C.maxbits[(long long)threadIdx.x * C.N + p]), 8);
}

// Lower off-diagonal tiles of U (never computed) <- their upper mirror.
__global__ void mirror_tiles_kernel(double* U, int N, int nmat) {
  const long long total = (long long)nmat * N * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long m = t / ((long long)N * N);
    const int p = (int)((t / N) % N), q = (int)(t % N);
    if (p / BM > q / BN) U[m * N * N + (long long)p * N + q] = U[m * N * N + (long long)q * N + p];
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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

bool make_map(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims,
              const cuuint64_t* strides_bytes, const cuuint32_t* box, std::string& err) {
  auto enc = get_encode();
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

struct Buffers {
  void* p = nullptr;
  size_t bytes = 0;
};

struct MixedWs {
  Buffers lx_o, lx_v, l_ov, y, pairs, err;
  Buffers u_xo, u_xv, u_ov, u_y, x32, maxbits, rot;
  Buffers l4, u_l4, co4, cv4, u_co, u_cv, rot_stats, w4, u_w4, rot_ov, e2;
  Buffers y2, x32b, maxbits2, u_y2;  // second set of pair-block buffers
  cudaStream_t side = nullptr;       // slicing passes, overlapping the next pair GEMM
  cudaEvent_t ev_pair[2] = {nullptr, nullptr}, ev_comb[2] = {nullptr, nullptr};
};

std::mutex g_attr_mu;
bool g_attr_done[64] = {false};

template <class T>
T* grow(Buffers& b, size_t count, std::string& err) {
  const size_t bytes = std::max<size_t>(count * sizeof(T), 256);
  if (b.bytes < bytes) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      err = "mixed workspace allocation of " + std::to_string(bytes) + " bytes failed";
      return nullptr;
    }
    b.bytes = bytes;
  }
  return static_cast<T*>(b.p);
}


}  // namespace

void* mixed_workspace_create() { return new MixedWs(); }

void mixed_workspace_destroy(void* w) {
  if (!w) return;
  MixedWs* W = static_cast<MixedWs*>(w);
  for (Buffers* b : {&W->lx_o, &W->lx_v, &W->l_ov, &W->y, &W->pairs, &W->err, &W->u_xo,
                     &W->u_xv, &W->u_ov, &W->u_y, &W->x32, &W->maxbits, &W->rot, &W->l4, &W->u_l4, &W->co4,
                     &W->cv4, &W->u_co, &W->u_cv, &W->rot_stats, &W->w4, &W->u_w4, &W->rot_ov,
                     &W->e2, &W->y2, &W->x32b, &W->maxbits2, &W->u_y2})
    if (b->p) cudaFree(b->p);
  for (int i = 0; i < 2; ++i) {
    if (W->ev_pair[i]) cudaEventDestroy(W->ev_pair[i]);
    if (W->ev_comb[i]) cudaEventDestroy(W->ev_comb[i]);
  }
  if (W->side) cudaStreamDestroy(W->side);
  delete W;
}

#define CK_SIDE(call)                                                          \
  do {                                                                         \
    const cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) {                                                   \
      err = std::string(#call ": ") + cudaGetErrorString(e_);                  \
      if (W.side) cudaStreamSynchronize(W.side); /* no side work outlives us */ \
      return AGF2_ERR_CUDA;                                                    \
    }                                                                          \
  } while (0)

int mixed_build_moments(const double* L, int naux, int N, const double* Co, const double* Cv,
                        int o, int v, const double* eo, const double* ev, int nmom,
                        double* U_hole, double* U_part, std::string& err, cudaStream_t s,
                        KernelStats* stats, void* workspace) {
  // CUDA events around the tcgen05 launches when stats->enabled
  std::vector<cudaEvent_t> evs;
  std::vector<int> ev_kind;
  std::vector<double> ev_flops;
  auto mark = [&](int kind, double flops) {
    if (!stats || !stats->enabled) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    evs.push_back(a);
    evs.push_back(b);
    ev_kind.push_back(kind);
    ev_flops.push_back(flops);
    cudaEventRecord(a, s);
  };
  auto mark_end = [&]() {
    if (!stats || !stats->enabled) return;
    cudaEventRecord(evs.back(), s);
  };
  int dev = 0;
  cudaGetDevice(&dev);
  MixedWs& W = *static_cast<MixedWs*>(workspace);
  if (nmom < 1 || nmom + 1 > MAXM) {
    err = "the split-precision moment build supports nmom = 1..3";
    return AGF2_ERR_UNSUPPORTED;
  }
  {
    std::lock_guard<std::mutex> attr_lock(g_attr_mu);
    if (!g_attr_done[dev & 63]) {
      if (cudaFuncSetAttribute(gemm6_kernel<MODE_PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               SMEM_BYTES) != cudaSuccess ||
          cudaFuncSetAttribute(gemm6_kernel<MODE_MOMENT>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) != cudaSuccess) {
        err = "cudaFuncSetAttribute(smem) failed";
        return AGF2_ERR_CUDA;
      }
      g_attr_done[dev & 63] = true;
    }
  }
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int Qs = (naux + BK - 1) / BK * BK;
  const long long NQs = (long long)N * Qs;
  __nv_bfloat16* lxo = grow<__nv_bfloat16>(W.lx_o, 3LL * o * NQs, err);
  __nv_bfloat16* lxv = grow<__nv_bfloat16>(W.lx_v, 3LL * v * NQs, err);
  __nv_bfloat16* lov = grow<__nv_bfloat16>(W.l_ov, 3LL * o * v * Qs, err);
  int* derr = grow<int>(W.err, 1, err);
  if (!lxo || !lxv || !lov || !derr) return AGF2_ERR_OOM;
  cudaMemsetAsync(derr, 0, sizeof(int), s);
  float* u_xo = grow<float>(W.u_xo, (size_t)o * N, err);
  float* u_xv = grow<float>(W.u_xv, (size_t)v * N, err);
  float* u_ov = grow<float>(W.u_ov, (size_t)o * v, err);
  const int nm = nmom + 1;
  float* u_y = grow<float>(W.u_y, (size_t)nm * N, err);
  if (!u_xo || !u_xv || !u_ov || !u_y) return AGF2_ERR_OOM;
  // ---- a2: rotation into the pole basis on the tensor cores ----
  // Lxo[i][p][Q] = sum_r Co[r][i] L[Q][r][p] and Lxv likewise, one block of
  // outer poles at a time through W[x][Q][p] = sum_r Cx[r][x] L[Q][p][r]
  // (batched over Q, p contiguous), which a transposing slicer turns into the
  // limb planes of the rows (x, p) over Q; Lov[j][a][Q] = sum_p Co[p][j]
  // W_v[a][Q][p] (batched over a, Q contiguous).  Four-limb integer splits
  // with exactly summed 256-entry chunks (rotate.cu) keep the rotated values
  // FP64-class, so the three-limb slicing of the result stays the only
  // precision step before the pair GEMM.  Only the limbs of the three
  // rotated tensors are held whole.
  {
    const int Ns = (N + 255) / 256 * 256;  // K of the rotation GEMMs (r or p)
    const long long nQN = (long long)naux * N;
    __nv_bfloat16* l4 = grow<__nv_bfloat16>(W.l4, 4LL * nQN * Ns, err);
    float* u_l4 = grow<float>(W.u_l4, (size_t)nQN, err);
    __nv_bfloat16* co4 = grow<__nv_bfloat16>(W.co4, 4LL * o * Ns, err);
    __nv_bfloat16* cv4 = grow<__nv_bfloat16>(W.cv4, 4LL * v * Ns, err);
    float* u_co = grow<float>(W.u_co, (size_t)o, err);
    float* u_cv = grow<float>(W.u_cv, (size_t)v, err);
    if (!l4 || !u_l4 || !co4 || !cv4 || !u_co || !u_cv) return AGF2_ERR_OOM;
    int rc;
    // rows (Q, p) of L over r; rows x of C^T over r (C is [N][x])
    if ((rc = rot_limbs_slice4(L, nQN, N, N, 1, Ns, nQN, nQN, 0, 0, l4, u_l4, s)) ||
        (rc = rot_limbs_slice4(Co, o, N, 1, o, Ns, o, o, 0, 0, co4, u_co, s)) ||
        (rc = rot_limbs_slice4(Cv, v, N, 1, v, Ns, v, v, 0, 0, cv4, u_cv, s))) {
      err = "rotation slicing launch failed";
      return rc;
    }
    // per outer pole: W [nQ][N] FP64; per virtual pole also its four-limb
    // planes [nQ][Ns] and its Lov column block [o][nQ] FP64
    const size_t budget = size_t(4) << 30;
    const long long per_o = nQN * 8;
    const long long per_v = nQN * 8 + 4LL * naux * Ns * 2 + (long long)o * naux * 8;
    const int bi = (int)std::max<long long>(1, std::min<long long>(o, budget / per_o));
    const int ba = (int)std::max<long long>(1, std::min<long long>(v, budget / per_v));
    double* wtmp = grow<double>(W.rot, (size_t)std::max<long long>((long long)bi, ba) * nQN, err);
    double* stats = grow<double>(W.rot_stats, (size_t)std::max(bi, ba) * N, err);
    __nv_bfloat16* w4 = grow<__nv_bfloat16>(W.w4, 4LL * ba * naux * Ns, err);
    float* u_w4 = grow<float>(W.u_w4, (size_t)ba * naux, err);
    double* tmpov = grow<double>(W.rot_ov, (size_t)o * ba * naux, err);
    if (!wtmp || !stats || !w4 || !u_w4 || !tmpov) return AGF2_ERR_OOM;
    for (int i0 = 0; i0 < o; i0 += bi) {
      const int nb = std::min(bi, o - i0);
      if ((rc = rot_gemm4(co4, o, i0, nb, u_co, l4, N, naux, u_l4, Ns, wtmp, nQN, N, derr, err,
                          s)) ||
          (rc = rot_transpose_slice3(wtmp, nb, naux, N, Qs, stats, (long long)o * N,
                                     (long long)i0 * N, lxo, u_xo, s)))
        return rc ? rc : AGF2_ERR_CUDA;
    }
    for (int a0 = 0; a0 < v; a0 += ba) {
      const int nb = std::min(ba, v - a0);
      if ((rc = rot_gemm4(cv4, v, a0, nb, u_cv, l4, N, naux, u_l4, Ns, wtmp, nQN, N, derr, err,
                          s)) ||
          (rc = rot_transpose_slice3(wtmp, nb, naux, N, Qs, stats, (long long)v * N,
                                     (long long)a0 * N, lxv, u_xv, s)))
        return rc ? rc : AGF2_ERR_CUDA;
      // rows (a, Q) of W_v over p, then tmpov[j][a'][Q] = sum_p Co[p][j] W_v[a'][Q][p]
      const long long rows = (long long)nb * naux;
      if ((rc = rot_limbs_slice4(wtmp, rows, N, N, 1, Ns, rows, rows, 0, 0, w4, u_w4, s)) ||
          (rc = rot_gemm4(co4, o, 0, o, u_co, w4, naux, nb, u_w4, Ns, tmpov,
                          (long long)nb * naux, naux, derr, err, s)))
        return rc ? rc : AGF2_ERR_CUDA;
      // row (j, a') of the block is row j v + a0 + a' of the Lov planes
      const long long blocks = std::min<long long>(((long long)o * nb + 7) / 8, 152LL * 16);
      slice_rows_kernel<<<(int)std::max(1LL, blocks), 256, 0, s>>>(
          tmpov, (long long)o * nb, naux, naux, Qs, (long long)o * v, nb, v, a0, lov, u_ov);
      count_launch();
    }
  }
  if (cudaGetLastError() != cudaSuccess) {
    err = "slice kernel launch failed";
    return AGF2_ERR_CUDA;
  }
  // tensor maps of the rotated limb planes
  CUtensorMap map_xo, map_xv, map_b_hole, map_b_part;
  {
    cuuint64_t dims[3] = {(cuuint64_t)Qs, (cuuint64_t)N, (cuuint64_t)3 * o};
    cuuint64_t str[2] = {(cuuint64_t)Qs * 2, (cuuint64_t)NQs * 2};
    cuuint32_t box[3] = {BK, BM, 1};
    if (!make_map(&map_xo, lxo, 3, dims, str, box, err)) return AGF2_ERR_CUDA;
    dims[2] = (cuuint64_t)3 * v;
    if (!make_map(&map_xv, lxv, 3, dims, str, box, err)) return AGF2_ERR_CUDA;
  }
  {
    // Lov limbs [3][o][v][Qs]: dims (Q, a, i, limb)
    cuuint64_t dims[4] = {(cuuint64_t)Qs, (cuuint64_t)v, (cuuint64_t)o, 3};
    cuuint64_t str[3] = {(cuuint64_t)Qs * 2, (cuuint64_t)v * Qs * 2, (cuuint64_t)o * v * Qs * 2};
    cuuint32_t box_h[4] = {BK, BN, 1, 1};   // hole: rows a, fixed j
    cuuint32_t box_p[4] = {BK, 1, BN, 1};   // particle: rows i, fixed b
    if (!make_map(&map_b_hole, lov, 4, dims, str, box_h, err)) return AGF2_ERR_CUDA;
    if (!make_map(&map_b_part, lov, 4, dims, str, box_p, err)) return AGF2_ERR_CUDA;
  }

  const int n_ptiles = (N + BM - 1) / BM;
  // pole energies as float pairs for the combine pass's weights: [eo | ev]
  float2* e2 = grow<float2>(W.e2, (size_t)o + v, err);
  if (!e2) return AGF2_ERR_OOM;
  if (o > 0) float_pair_kernel<<<(o + 255) / 256, 256, 0, s>>>(eo, o, e2);
  if (v > 0) float_pair_kernel<<<(v + 255) / 256, 256, 0, s>>>(ev, v, e2 + o);
  count_launch((o > 0) + (v > 0));
  // the slicing pass of pair block b runs on a side stream while the pair GEMM
  // of block b + 1 runs on s (two sets of block buffers); every side-stream
  // launch is joined back into s by an event before the block's moment GEMM
  if (!W.side) {
    if (cudaStreamCreateWithFlags(&W.side, cudaStreamNonBlocking) != cudaSuccess) {
      err = "side stream creation failed";
      return AGF2_ERR_CUDA;
    }
    for (int i = 0; i < 2; ++i)
      if (cudaEventCreateWithFlags(&W.ev_pair[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&W.ev_comb[i], cudaEventDisableTiming) != cudaSuccess) {
        err = "event creation failed";
        return AGF2_ERR_CUDA;
      }
  }
  float* u_yb[2] = {u_y, grow<float>(W.u_y2, (size_t)nm * N, err)};
  if (!u_yb[1]) return AGF2_ERR_OOM;
  for (int sector = 0; sector < 2; ++sector) {
    const bool hole = (sector == 0);
    const int n_out = hole ? o : v;
    const int n_in = hole ? v : o;
    double* U = hole ? U_hole : U_part;
    const float2* e_out2 = hole ? e2 : e2 + o;
    const float2* e_in2 = hole ? e2 + o : e2;
    // unordered pairs x <= y
    std::vector<int2> pairs;
    pairs.reserve((size_t)n_out * (n_out + 1) / 2);
    for (int x = 0; x < n_out; ++x)
      for (int y = x; y < n_out; ++y) pairs.push_back(make_int2(x, y));
    int2* dpairs = grow<int2>(W.pairs, pairs.size(), err);
    if (!dpairs) return AGF2_ERR_OOM;
    cudaMemcpyAsync(dpairs, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    const int n_cchunks = (n_in + BN - 1) / BN;
    const int ncp = n_cchunks * BN;
    const long long kpp = (long long)n_cchunks * KCHUNK;
    // pairs per block: large enough that GEMM 2's split-K tiles are long (each
    // tile ends in a 128x128 FP64 drain) and launches few, about 1 GB of X + Y
    // + Yw (measured at nmo = 200 / 500: 0.26 / 0.25 GB blocks 15% / 10% slower
    // in GEMM 2, 2 GB no faster), and a whole number of waves of the
    // persistent CTAs
    const double per_pair = (double)N * (kpp * nm /*Y w^n*/ * 3 /*limbs*/ * 2 /*bytes*/ +
                                         2.0 * ncp * 4 /*X, both orders*/);
    const int tpp = 2 * n_ptiles * n_cchunks;  // tiles per unordered pair
    int bp = (int)std::max(1.0, std::floor(1.0e9 / per_pair));
    {
      int g = nsm, t = tpp / 2;  // a CTA takes both orientations of a pair tile
      while (t) { const int r = g % t; g = t; t = r; }  // gcd(nsm, tpp / 2)
      const int unit = nsm / g;                          // pairs per whole wave
      const int bp_lim = (int)std::floor(1.5e9 / per_pair);
      if (unit <= bp_lim) bp = std::max(unit, bp / unit * unit);
    }
    bp = std::max(1, std::min<int>(bp, (int)pairs.size()));
    const long long Ks = (long long)bp * kpp;
    const long long Kx = (long long)bp * 2 * ncp;  // row length of X
    __nv_bfloat16* yb[2] = {grow<__nv_bfloat16>(W.y, 3LL * nm * N * Ks, err),  // [nm][3][N][Ks]
                            grow<__nv_bfloat16>(W.y2, 3LL * nm * N * Ks, err)};
    float* xb[2] = {grow<float>(W.x32, (size_t)N * Kx, err), grow<float>(W.x32b, (size_t)N * Kx, err)};
    unsigned* mb[2] = {grow<unsigned>(W.maxbits, (size_t)nm * N, err),
                       grow<unsigned>(W.maxbits2, (size_t)nm * N, err)};
    if (!yb[0] || !yb[1] || !xb[0] || !xb[1] || !mb[0] || !mb[1]) return AGF2_ERR_OOM;
    // block whose moment GEMM is launched after the next block's pair GEMM
    struct Pending {
      bool valid = false;
      int buf = 0;
      long long K = 0;
      long long ordered = 0;
    } pend;
    auto launch_moment = [&](const Pending& pb) -> int {
      CK_SIDE(cudaStreamWaitEvent(s, W.ev_comb[pb.buf], 0));
      __nv_bfloat16* y = yb[pb.buf];
      const long long K = pb.K;
      // GEMM 2 over this block's K = np * kpp
      CUtensorMap map_y;  // all [nm][3] planes; plane index = moment * 3 + limb
      cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)N, (cuuint64_t)3 * nm};
      cuuint64_t str[2] = {(cuuint64_t)Ks * 2, (cuuint64_t)N * Ks * 2};
      cuuint32_t box[3] = {BK, BM, 1};
      if (!make_map(&map_y, y, 3, dims, str, box, err)) return AGF2_ERR_CUDA;
      Params M{};
      M.N = N;
      M.n_ptiles = n_ptiles;
      M.n_qtiles = (N + BN - 1) / BN;
      M.ksteps = (int)((K + BK - 1) / BK);
      M.nm = nm;
      const int tiles = M.n_ptiles * (M.n_ptiles + 1) / 2 * nm;  // upper tiles x moments
      // about two tiles per persistent CTA, so each tile's atomics overlap the
      // next tile's MMAs; splits on chunk boundaries, at most MAX_TILE_CHUNKS each
      const int nchunks = M.ksteps / CHUNK_STEPS;  // K is a whole number of chunks
      int nsplit = std::max(1, (nsm * 2 + tiles - 1) / tiles);
      nsplit = std::max(nsplit, (nchunks + MAX_TILE_CHUNKS - 1) / MAX_TILE_CHUNKS);
      nsplit = std::min(nsplit, nchunks);
      M.ksplit = (nchunks + nsplit - 1) / nsplit * CHUNK_STEPS;
      M.nsplit = (M.ksteps + M.ksplit - 1) / M.ksplit;  // every split non-empty
      M.ntiles = tiles * M.nsplit;
      M.n_out = 0;
      M.unitA = u_yb[pb.buf];
      M.unitB = u_yb[pb.buf];
      M.U0 = U;
      M.err = derr;
      // algorithmic flops: every moment over the ordered pairs, 2 N^2 per (pair, c)
      mark(1, 2.0 * nm * (double)N * N * (double)n_in * (double)pb.ordered);
      gemm6_kernel<MODE_MOMENT><<<std::min(M.ntiles, nsm), NTHREADS, SMEM_BYTES, s>>>(map_y,
                                                                                      map_y, M);
      mark_end();
      count_launch();
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        err = std::string("tcgen05 kernel launch: ") + cudaGetErrorString(e);
        return AGF2_ERR_CUDA;
      }
      return AGF2_OK;
    };
    int bi = 0;
    for (size_t b0 = 0; b0 < pairs.size(); b0 += bp, ++bi) {
      const int cur = bi & 1;
      const int np = (int)std::min<size_t>(bp, pairs.size() - b0);
      const long long K = (long long)np * kpp;
      float* x32 = xb[cur];
      unsigned* maxbits = mb[cur];
      Params P{};
      P.N = N;
      P.n_in = n_in;
      P.ksteps = Qs / BK;
      P.n_ptiles = n_ptiles;
      P.n_cchunks = n_cchunks;
      P.n_out = n_out;
      P.hole = hole ? 1 : 0;
      P.pair0 = (int)b0;
      P.pairs = dpairs;
      P.e_out2 = e_out2;
      P.e_in2 = e_in2;
      P.maxbits = maxbits;
      P.nm = nm;
      P.unitA = hole ? u_xo : u_xv;
      P.unitB = u_ov;
      P.v_stride = v;
      P.X = x32;
      P.ncp = ncp;
      P.Ks = Kx;
      P.err = derr;
      P.ntiles = np * tpp;

      const int grid1 = std::min(P.ntiles / 2, nsm);  // tpp is even: whole orientation pairs
      // algorithmic flops: GEMM 1 for the ordered pairs of this block
      long long ordered = 0;
      for (int t = 0; t < np; ++t) ordered += (pairs[b0 + t].x == pairs[b0 + t].y) ? 1 : 2;
      mark(0, 2.0 * N * (double)naux * n_in * (double)ordered);
      // the epilogue folds each pair tile's row maxima of |Y w^n| into maxbits
      cudaMemsetAsync(maxbits, 0, (size_t)nm * N * sizeof(unsigned), s);
      gemm6_kernel<MODE_PAIR><<<grid1, NTHREADS, SMEM_BYTES, s>>>(
          hole ? map_xo : map_xv, hole ? map_b_hole : map_b_part, P);
      mark_end();
      count_launch();
      CK_SIDE(cudaEventRecord(W.ev_pair[cur], s));
      // S/D and energy weights, then fixed-point limbs with each row's exact
      // unit, on the side stream (overlaps the next block's pair GEMM)
      CK_SIDE(cudaStreamWaitEvent(W.side, W.ev_pair[cur], 0));
      Combine C{x32, Kx, np, ncp, n_in, N, (int)kpp, (int)b0, nm, dpairs, e_out2, e_in2, maxbits,
                yb[cur], Ks, (long long)N * Ks, u_yb[cur]};
      const long long per_row = (long long)np * ncp / 4;
      const dim3 gc((unsigned)std::max(1LL, std::min<long long>((per_row + 1023) / 1024, 64)),
                    (unsigned)N);
      combine_kernel<<<gc, 256, 0, W.side>>>(C);
      count_launch();
      CK_SIDE(cudaEventRecord(W.ev_comb[cur], W.side));
      if (pend.valid) {
        const int rc = launch_moment(pend);
        if (rc != AGF2_OK) {
          cudaStreamSynchronize(W.side);  // the slicing passes still queued there
          return rc;
        }
      }
      pend.valid = true;
      pend.buf = cur;
      pend.K = K;
      pend.ordered = ordered;
    }
    if (pend.valid) {
      const int rc = launch_moment(pend);
      if (rc != AGF2_OK) {
        cudaStreamSynchronize(W.side);
        return rc;
      }
    }
  }
  {
    const long long tot = (long long)nm * N * N;
    const int g = (int)std::min<long long>((tot + 255) / 256, 152LL * 32);
    mirror_tiles_kernel<<<g, 256, 0, s>>>(U_hole, N, nm);
    mirror_tiles_kernel<<<g, 256, 0, s>>>(U_part, N, nm);
    count_launch(2);
  }
  int herr = 0;
  cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    err = std::string("mixed moment build: ") + cudaGetErrorString(e);
    return AGF2_ERR_CUDA;
  }
  for (size_t i = 0; i < ev_kind.size(); ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, evs[2 * i], evs[2 * i + 1]);
    stats->launches[ev_kind[i]] += 1;
    stats->ms[ev_kind[i]] += ms;
    stats->flops[ev_kind[i]] += ev_flops[i];
  }
  for (auto e2 : evs) cudaEventDestroy(e2);
  if (herr == DEV_TIMEOUT) {
    err = "tcgen05 pipeline wait timed out";
    return AGF2_ERR_TIMEOUT;
  }
  return AGF2_OK;
}

}  // namespace agf2
