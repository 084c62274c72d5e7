// A8: batched statistical-equilibrium solves (Sec. 2.2; Sec. 2.3.2 for the
// photoexcitation and detailed-balance photodeexcitation rates).
//
// One persistent launch serves every (cell, ion) system, longest first (a
// work list sorted by level count, taken from an atomic counter), one CTA per
// system at a time:
//   assemble  the FP64 rate matrix of the system in the CTA's global
//             workspace: collisions for every level pair (Boltzmann factors
//             per level, detailed balance), radiative lines (A beta_S,
//             photoexcitation, stimulated emission) by atomics, beta_S from
//             the fixed-point exponential, the non-thermal term into the
//             ground level, the diagonal as minus the total out-rate (column
//             sums), the ground-level equation replaced by sum n = n_z;
//   factor    blocked right-looking LU with partial pivoting: the CTA factors
//             each panel of nb columns in shared memory (a warp finds each
//             pivot), then swaps rows, solves for the panel's U rows and
//             updates the trailing matrix through L2 (rank-nb update from
//             shared memory);
//   solve     blocked forward/back substitution;
//   refine    (FP32 path) the matrix scaled by powers of two near the warm
//             start (columns) and the row maxima is factored in FP32;
//             residuals and updates are FP64 until the error every level keeps
//             is below tol (a ratio test on successive corrections); a system
//             that does not converge, or whose FP32 factor meets a zero pivot,
//             is solved again in FP64.
// Newton mode repeats assemble..refine on the Jacobian of the rate equations
// with beta_S taken from the iterate (Sec. 2.2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fixexp.cuh"
#include "tc.cuh"
#include "xt_internal.cuh"

namespace xt {

constexpr int kSeThreads = 256;   // CTA of the large systems
constexpr int kSeMaxL = 320;      // levels per system
constexpr int kSmallThreads = 64; // CTA of the systems with at most kSmallL levels
constexpr int kSmallL = 64;
constexpr int kSeNbMax = 32;      // panel width
// panel buffer: [maxl][nb + 1] of the factor type, or of doubles with nb <= 16
__host__ __device__ constexpr size_t se_pan_bytes(int maxl) {
  return (size_t)maxl * (kSeNbMax + 1) * 4 > (size_t)maxl * 17 * 8 ? (size_t)maxl * (kSeNbMax + 1) * 4
                                                                    : (size_t)maxl * 17 * 8;
}

struct SeArgs {
  Geometry g;
  int nlev, n_ion, nline;
  const int* __restrict__ level_off;
  const double* __restrict__ E;
  const double* __restrict__ glev;
  const double* __restrict__ nion;      // [row][n_ion]
  const double* __restrict__ Te;        // row order
  const double* __restrict__ ne;
  const double* __restrict__ dep;
  const double* __restrict__ pops;      // [row][nlev]: optical depths, estimator f_corr
  const double* __restrict__ warm;      // [row][nlev] warm start, or nullptr for Boltzmann
  double* __restrict__ pops_out;        // [row][nlev]
  int* __restrict__ status;             // [cell * n_ion + z] natural cell order
  const double* __restrict__ lines;     // packed sorted: nu, K, g_l/g_u, (lo | up << 32)
  const double* __restrict__ A;         // sorted
  const int* __restrict__ down_off;     // [nlev + 1] lines by upper level
  const int* __restrict__ down_line;
  const int* __restrict__ low_off;      // [nlev + 1] lines by lower level,
  const int* __restrict__ low_line;     //   as positions k in down_line
  const double* __restrict__ S;         // estimators (net photons) [row][sorted line]
  const int* __restrict__ crow;         // compact store: the cell's row in S, -1 none (nullptr: dense)
  const double* __restrict__ Rj;        // photoexcitation per sorted line (Jbar model)
  int rates;
  double V;                             // cell volume of the cube (a spherical grid's: g.vol[row])
  const double* __restrict__ ups;       // per ion [L_z][L_z]
  const int64_t* __restrict__ ups_off;
  const int* __restrict__ levels_used;  // [cell * n_ion + z] or nullptr
  const int* __restrict__ work;         // cell * 16 + ion, longest first
  int64_t n_work;
  unsigned long long* __restrict__ counter;
  double* __restrict__ W64;             // per CTA: L_max^2 doubles
  void* __restrict__ WT;                // per CTA: L_max^2 of the factor type
  int64_t wlen;                         // L_max^2
  int precision;
  double tol, eta;
  int max_iter;
  int nb_bucket[8];                     // panel width per 64-level bucket
  double* __restrict__ iters;           // [cell * n_ion + z] refinement (or Newton) steps
  int tmem_cols;                        // > 0: FP32 factors' trailing updates on the tensor cores
  unsigned long long* __restrict__ tc_err;   //   (TMEM columns per CTA; CTAs that gave up)
  int tc_bf16;                          //   with BF16 operands, else TF32
  int newton_max;                       // 0: linear solve with beta_S from pops
  double newton_tol, newton_maxvar;
  FixExpTables fx;                      // e^-tau tables (fixed point)
};

// Newton: the derivative of a line's net downward flow F = A beta n_u -
// beta B J_ext (n_l - g_l/g_u n_u) through beta_S, t = beta'(tau) K (A n_u -
// B J_ext net); F enters row l with +, row u with - (so dF/dn_l = t and dF/dn_u
// = -g_l/g_u t).  Lr is the line's packed record (nu, K, g_l/g_u, lo | up).
__device__ __forceinline__ double line_jac_t(const SeArgs& a, const FixExpTables& fx, const double* Lr,
                                             int s, double n_lo, double n_up) {
  const double net = n_lo - Lr[2] * n_up;
  const double tau = Lr[1] * net;
  double db;
  sobolev_beta_fix(fx, tau, &db);
  if (db == 0.0) return 0.0;
  const double BJ = a.rates == XT_RATES_JBAR ? a.Rj[s] : 0.0;
  return db * Lr[1] * (a.A[s] * n_up - BJ * net);
}

__device__ __forceinline__ void block_sync() { __syncthreads(); }

// Tensor-core state of a CTA (shared memory): the TMEM accumulator (ncols
// columns), the mbarrier that MMA completions arrive on and its phase; ok = 0
// once a bounded wait ran out (the CTA then keeps to the CUDA cores).
struct TcState {
  uint64_t bar;
  uint32_t taddr, phase;
  int ncols, ok;
  int bf16;                    // operands in BF16 (kind::f16), else TF32
  unsigned long long* err;     // global count of CTAs that gave up on the tensor cores
};
constexpr long long kTcSpin = 1ll << 24;   // polls of an MMA completion before giving up
// Byte offset of the TcState in the U12 buffer (kSeNbMax x kSeMaxL floats): an
// FP32 panel step uses kb x n2 <= kSeNbMax x (kSeMaxL - kSeNbMax) of it
// (panels of 32 columns; 16-column panels use half the rows), and the operand B
// of the tensor cores <= (kSeMaxL - kSeNbMax) rows of 128 bytes, the same.
constexpr size_t kTcStateOff = (size_t)kSeNbMax * (kSeMaxL - kSeNbMax) * 4;
static_assert(kTcStateOff + sizeof(TcState) <= (size_t)kSeNbMax * kSeMaxL * 4, "TcState in the U12 buffer");
static_assert(kTcStateOff % 8 == 0, "TcState alignment");
static_assert((size_t)8 * (kSeMaxL - 8) * 8 <= kTcStateOff, "FP64 fallback panels below the TcState");

// ---- blocked LU with partial pivoting of the L x L row-major matrix A (global)
// Panels of nb columns are staged in shared memory with row stride nb + 1 (no
// bank conflicts between consecutive rows).  Every step of a panel column uses
// the whole CTA: pivot search (warp reductions, then across warps), row swap,
// multipliers and the rank-1 update of the panel, one thread per row.  Then
// the CTA applies the swaps to the other columns, solves for the panel's U
// rows and updates the trailing matrix through L2 (rank-nb update).
// A22 -= L21 U12 of one panel step on the tensor cores (see lu_factor); false
// if an MMA completion was not seen within its bounded wait (the CTA then
// stops using the tensor cores and the factor is treated as singular, which
// sends the system to the FP64 solve).
__device__ __noinline__ bool lu_trailing_tc(float* __restrict__ A, int L, int k0, int kb, int kbp, int m2, int n2, int Npad,
                               float* pan, float* u12, TcState* tc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char* const Bs = reinterpret_cast<unsigned char*>(u12);
  unsigned char* const As = reinterpret_cast<unsigned char*>(pan + kb * kbp);   // L21's first row
  const bool bf = tc->bf16 != 0;
  if (bf) {
    // operand B: U12 rounded to BF16, zero outside kb x n2, in the 16-bit
    // layout; each thread converts 16-byte groups of 8 K elements (two of the
    // 32-bit chunks) through registers, since the new tile overwrites the old
    constexpr int kGroups = (kSeMaxL * 4 + 255) / 256;   // Npad <= kSeMaxL rows of 4 groups
    uint4 gv[kGroups];
#pragma unroll
    for (int q = 0; q < kGroups; ++q) {
      const int gi = tid + 256 * q, n = gi >> 2, k8 = (gi & 3) << 3;
      uint4 o = make_uint4(0u, 0u, 0u, 0u);
      if (gi < Npad * 4 && n < n2) {
        const float4 lo = *reinterpret_cast<const float4*>(Bs + tc::tile_off(n, k8, Npad));
        const float4 hi = *reinterpret_cast<const float4*>(Bs + tc::tile_off(n, k8 + 4, Npad));
        o.x = tc::pack_bf16(k8 < kb ? lo.x : 0.f, k8 + 1 < kb ? lo.y : 0.f);
        o.y = tc::pack_bf16(k8 + 2 < kb ? lo.z : 0.f, k8 + 3 < kb ? lo.w : 0.f);
        o.z = tc::pack_bf16(k8 + 4 < kb ? hi.x : 0.f, k8 + 5 < kb ? hi.y : 0.f);
        o.w = tc::pack_bf16(k8 + 6 < kb ? hi.z : 0.f, k8 + 7 < kb ? hi.w : 0.f);
      }
      gv[q] = o;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kGroups; ++q) {
      const int gi = tid + 256 * q;
      if (gi < Npad * 4) *reinterpret_cast<uint4*>(Bs + tc::tile_off16(gi >> 2, (gi & 3) << 3, Npad)) = gv[q];
    }
  } else {
    // operand B: U12 rounded to TF32, zero outside kb x n2
    for (int e = tid; e < Npad * 32; e += blockDim.x) {
      const int n = e >> 5, k = e & 31;
      uint32_t* q = reinterpret_cast<uint32_t*>(Bs + tc::tile_off(n, k, Npad));
      *q = (n < n2 && k < kb) ? tc::to_tf32(__uint_as_float(*q)) : 0u;
    }
  }
  const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
  const int nmax = tc->ncols < 256 ? tc->ncols : 256;
  const uint32_t taddr = tc->taddr;
  uint32_t ph = tc->phase;
  bool ok = true;
  for (int t0 = 0; t0 < m2 && ok; t0 += 128) {
    // operand A: rows t0..t0+127 of L21, through registers (the region they
    // are written to holds the first rows themselves)
    float av[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = tid + 256 * q, r = e >> 5, k = e & 31;
      av[q] = (t0 + r < m2 && k < kb) ? pan[(kb + t0 + r) * kbp + k] : 0.f;
    }
    __syncthreads();
    if (bf) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int e = tid + 256 * q, r = e >> 5, k = e & 31;
        *reinterpret_cast<uint16_t*>(As + tc::tile_off16(r, k, 128)) = tc::to_bf16(av[q]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int e = tid + 256 * q, r = e >> 5, k = e & 31;
        *reinterpret_cast<uint32_t*>(As + tc::tile_off(r, k, 128)) = tc::to_tf32(av[q]);
      }
    }
    tc::fence_smem_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    for (int n0 = 0; n0 < Npad; n0 += nmax) {
      const int Nc = min(nmax, Npad - n0);
      if (tid == 0) {
        // one MMA per 32 bytes of K (two 16-byte chunks): 4 in TF32, 2 in BF16
        for (int k = 0; k < (bf ? 2 : 4); ++k) {
          const uint64_t ad = tc::smem_desc(a0 + (uint32_t)(k * 4096), 2048, 128);
          const uint64_t bd = tc::smem_desc(b0 + (uint32_t)((2 * k * (Npad >> 3) + (n0 >> 3)) * 128),
                                            (uint32_t)(Npad >> 3) * 128, 128);
          if (bf) tc::mma_bf16(taddr, ad, bd, tc::idesc_bf16(128, Nc), k > 0);
          else tc::mma_tf32(taddr, ad, bd, tc::idesc_tf32(128, Nc), k > 0);
        }
        tc::commit(&tc->bar);
      }
      const bool got = tc::bar_wait(&tc->bar, ph, kTcSpin);
      ph ^= 1u;
      if (!__syncthreads_and(got)) { ok = false; break; }
      tc::fence_after();
      // D rows 32 (warp % 4) + lane of the tile, half (warp / 4) of the columns
      const int q4 = warp & 3, half = Nc >> 1, c0 = (warp >> 2) * half;
      const int r = t0 + 32 * q4 + lane;
      for (int c = 0; c < half; c += 16) {
        float v[16];
        tc::ld16(taddr + ((uint32_t)(32 * q4) << 16) + (uint32_t)(c0 + c), v);
        if (r < m2) {
          float* Ar = A + (int64_t)(k0 + kb + r) * L + k0 + kb + n0 + c0 + c;
          const int nv = n2 - (n0 + c0 + c);
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (q < nv) Ar[q] -= v[q];
        }
      }
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
    }
  }
  if (tid == 0) {
    tc->phase = ph;
    if (!ok) {
      tc->ok = 0;
      atomicAdd(tc->err, 1ull);
    }
  }
  __syncthreads();
  return ok;
}

// With tc (FP32 factors, 256 threads, panels of 32 columns), trailing updates
// of at least kTcMinRows rows run on the tensor cores (tcgen05, kind::tf32,
// or kind::f16 with BF16 operands): U12 is solved straight into the canonical
// 32-bit operand layout of tc.cuh in the u12 buffer (40 KB: 320 rows x 32 K),
// then rounded to TF32 in place, or to BF16 into the 16-bit layout at the
// buffer's start, and zero-padded; each tile of 128 rows of L21 is read from
// the panel into registers and written in the operand layout at the start of
// L21's own rows in the panel buffer (128 rows of 33 floats hold its 16 KB, or
// 8 KB in BF16, so no row still to be read is overwritten); the MMAs
// accumulate L21 U12 in TMEM (FP32), and the CTA subtracts it from A22
// through tcgen05 loads (a warp per 32 rows and half the columns).
constexpr int kTcMinRows = 32;

template <typename T>
__device__ bool lu_factor(T* __restrict__ A, int L, int nb, int* piv, T* pan, T* u12,
                          TcState* tc = nullptr) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int sing, spiv;
  if (tid == 0) sing = 0;
  const int kbp = nb + 1;
  for (int k0 = 0; k0 < L; k0 += nb) {
    const int kb = min(nb, L - k0);
    const int rows = L - k0;                       // panel rows k0..L-1
    for (int e = tid; e < rows * kb; e += blockDim.x) {
      const int r = e / kb, cc = e - r * kb;
      pan[r * kbp + cc] = A[(int64_t)(k0 + r) * L + k0 + cc];
    }
    block_sync();
    // Column j: warp 0 applies the previous column's row exchange and finds the
    // pivot row p; then every thread eliminates its rows (all r >= j but p)
    // with row p, and the exchange of rows j and p follows in the next step
    // (eliminating with row p in place and exchanging afterwards gives the
    // same factor as exchanging first).  Two barriers per column.
    int prev = -1;                                 // previous column and its pivot row
    for (int j = 0; j < kb; ++j) {
      if (warp == 0) {
        if (j > 0 && prev != j - 1 && prev >= 0 && lane < kb) {
          const T t = pan[(j - 1) * kbp + lane];
          pan[(j - 1) * kbp + lane] = pan[prev * kbp + lane];
          pan[prev * kbp + lane] = t;
        }
        __syncwarp();
        // argmax |pan[r][j]| over r >= j, ties to the lowest row
        T best = 0;
        int bi = j;
        for (int r = j + lane; r < rows; r += 32) {
          const T v = pan[r * kbp + j] < 0 ? -pan[r * kbp + j] : pan[r * kbp + j];
          if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const T ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
          piv[k0 + j] = k0 + bi;
          if (best == 0) sing = 1;
          spiv = best == 0 ? -1 : bi;
        }
      }
      block_sync();
      const int pr = spiv;
      prev = pr < 0 ? j : pr;                      // a zero column exchanges nothing
      if (pr >= 0) {
        const T inv = T(1) / pan[pr * kbp + j];
        const T* prow = pan + pr * kbp;
        for (int r = j + tid; r < rows; r += blockDim.x) {
          if (r == pr) continue;
          T* row = pan + r * kbp;
          const T l = row[j] * inv;
          row[j] = l;
          for (int cc = j + 1; cc < kb; ++cc) row[cc] -= l * prow[cc];
        }
      }
      block_sync();
    }
    // the last column's exchange
    if (warp == 0 && prev != kb - 1 && prev >= 0 && lane < kb) {
      const T t = pan[(kb - 1) * kbp + lane];
      pan[(kb - 1) * kbp + lane] = pan[prev * kbp + lane];
      pan[prev * kbp + lane] = t;
    }
    block_sync();
    // write the panel back; apply its row swaps to the other columns
    for (int e = tid; e < rows * kb; e += blockDim.x) {
      const int r = e / kb, cc = e - r * kb;
      A[(int64_t)(k0 + r) * L + k0 + cc] = pan[r * kbp + cc];
    }
    // each thread applies the panel's exchanges in order to its own columns (the
    // exchanges of one column depend on each other, different columns do not)
    for (int cc = tid; cc < L; cc += blockDim.x) {
      if (cc >= k0 && cc < k0 + kb) continue;
      for (int j = 0; j < kb; ++j) {
        const int p = piv[k0 + j];
        if (p != k0 + j) {
          const T tmp = A[(int64_t)(k0 + j) * L + cc];
          A[(int64_t)(k0 + j) * L + cc] = A[(int64_t)p * L + cc];
          A[(int64_t)p * L + cc] = tmp;
        }
      }
    }
    block_sync();
    const int n2 = L - k0 - kb;                     // trailing columns
    if (n2 > 0) {
      bool use_tc = false;
      int Npad = 0;
      if constexpr (sizeof(T) == 4) {
        use_tc = tc != nullptr && tc->ok && n2 >= kTcMinRows && kb == 32 && blockDim.x == 256 &&
                 ((tc::smem_u32(pan + kb * kbp) | tc::smem_u32(u12)) & 15) == 0;   // operand alignment
        Npad = (n2 + 31) & ~31;
      }
      // U12 = L11^-1 A12 (unit lower), one column per thread, kept in shared
      // memory: the column's kb entries are loaded first (independent loads in
      // flight together), then solved in place; row-major [kb][n2], or for the
      // tensor cores as operand B (row cc, K r)
      if (use_tc) {
        unsigned char* const ub = reinterpret_cast<unsigned char*>(u12);
        for (int cc = tid; cc < n2; cc += blockDim.x) {
          for (int r = 0; r < kb; ++r)
            *reinterpret_cast<T*>(ub + tc::tile_off(cc, r, Npad)) = A[(int64_t)(k0 + r) * L + k0 + kb + cc];
          for (int r = 0; r < kb; ++r) {
            T v = *reinterpret_cast<T*>(ub + tc::tile_off(cc, r, Npad));
            for (int s = 0; s < r; ++s) v -= pan[r * kbp + s] * *reinterpret_cast<T*>(ub + tc::tile_off(cc, s, Npad));
            *reinterpret_cast<T*>(ub + tc::tile_off(cc, r, Npad)) = v;
            A[(int64_t)(k0 + r) * L + k0 + kb + cc] = v;
          }
        }
      } else {
        for (int cc = tid; cc < n2; cc += blockDim.x)
          for (int r = 0; r < kb; ++r) u12[r * n2 + cc] = A[(int64_t)(k0 + r) * L + k0 + kb + cc];
        for (int cc = tid; cc < n2; cc += blockDim.x) {
          for (int r = 0; r < kb; ++r) {
            T v = u12[r * n2 + cc];
            for (int s = 0; s < r; ++s) v -= pan[r * kbp + s] * u12[s * n2 + cc];
            u12[r * n2 + cc] = v;
            A[(int64_t)(k0 + r) * L + k0 + kb + cc] = v;
          }
        }
      }
      block_sync();
      const int m2 = L - k0 - kb;                   // trailing rows
      if constexpr (sizeof(T) == 4) {
        if (use_tc && !lu_trailing_tc(A, L, k0, kb, kbp, m2, n2, Npad, pan, u12, tc)) sing = 1;
      }
      if (use_tc) continue;
      // A22 -= L21 U12: 4 x 4 register tiles
      const int tr = (m2 + 3) / 4, tcl = (n2 + 3) / 4;
      for (int t = tid; t < tr * tcl; t += blockDim.x) {
        const int bi = (t / tcl) * 4, bj = (t % tcl) * 4;
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = 0;
        for (int k = 0; k < kb; ++k) {
          T lv[4], uv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) lv[a] = (bi + a < m2) ? pan[(kb + bi + a) * kbp + k] : T(0);
#pragma unroll
          for (int b = 0; b < 4; ++b) uv[b] = (bj + b < n2) ? u12[k * n2 + bj + b] : T(0);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += lv[a] * uv[b];
        }
        // the tile's 16 loads first, then its stores
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (bi + a < m2 && bj + b < n2)
              acc[a][b] = A[(int64_t)(k0 + kb + bi + a) * L + k0 + kb + bj + b] - acc[a][b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (bi + a < m2 && bj + b < n2)
              A[(int64_t)(k0 + kb + bi + a) * L + k0 + kb + bj + b] = acc[a][b];
      }
      block_sync();
    }
  }
  block_sync();
  return sing == 0;
}

// The row permutation of lu_factor's pivots as a gather: row i of P b is b[perm[i]].
__device__ void lu_perm(const int* piv, int L, int* perm) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < L; ++i) perm[i] = i;
    for (int k = 0; k < L; ++k) {
      const int p = piv[k];
      if (p != k) { const int t = perm[k]; perm[k] = perm[p]; perm[p] = t; }
    }
  }
  block_sync();
}

// ---- solve L U x = y in place (x in shared memory, type T, already permuted)
// Each 32-row diagonal block is solved by one warp with the block's rows in
// registers (one row per lane) and the solved values passed by shuffles; the
// rows outside the block are updated by the whole CTA, one row per thread.
template <typename T>
__device__ void lu_solve(const T* __restrict__ A, int L, T* x) {
  const int tid = threadIdx.x, lane = tid & 31;
  // forward, unit lower
  for (int r0 = 0; r0 < L; r0 += 32) {
    const int rb = min(32, L - r0);
    if (tid < 32) {
      const bool on = lane < rb;
      const T* Ar = A + (int64_t)(r0 + (on ? lane : 0)) * L + r0;
      T a[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) a[c] = (on && c < lane) ? Ar[c] : T(0);
      T xv = on ? x[r0 + lane] : T(0);
#pragma unroll
      for (int c = 0; c < 31; ++c) {
        const T xc = __shfl_sync(0xffffffffu, xv, c);
        xv -= a[c] * xc;                           // a[c] = 0 for c >= lane
      }
      if (on) x[r0 + lane] = xv;
    }
    block_sync();
    for (int i = r0 + rb + tid; i < L; i += blockDim.x) {
      T s = 0;
      for (int c = 0; c < rb; ++c) s += A[(int64_t)i * L + r0 + c] * x[r0 + c];
      x[i] -= s;
    }
    block_sync();
  }
  // backward, upper
  for (int r1 = L; r1 > 0; r1 -= 32) {
    const int r0 = max(0, r1 - 32), rb = r1 - r0;
    if (tid < 32) {
      const bool on = lane < rb;
      const T* Ar = A + (int64_t)(r0 + (on ? lane : 0)) * L + r0;
      T a[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) a[c] = (on && c > lane && c < rb) ? Ar[c] : T(0);
      const T d = on ? Ar[lane] : T(1);
      T xv = on ? x[r0 + lane] : T(0);
#pragma unroll
      for (int c = 31; c >= 0; --c) {
        if (c < rb) {                              // uniform across the warp
          if (lane == c) xv = xv / d;
          const T xc = __shfl_sync(0xffffffffu, xv, c);
          xv -= a[c] * xc;                         // a[c] = 0 for c <= lane
        }
      }
      if (on) x[r0 + lane] = xv;
    }
    block_sync();
    for (int i = tid; i < r0; i += blockDim.x) {
      T s = 0;
      for (int c = 0; c < rb; ++c) s += A[(int64_t)i * L + r0 + c] * x[r0 + c];
      x[i] -= s;
    }
    block_sync();
  }
}

// MAXL: largest level count the CTA takes (the large kernel 320 with 256
// threads, the small one 64 with 64 threads: short block-wide steps cost few
// warps, and several CTAs share an SM).
// TC: the tensor-core instance (TF32 factors of the large systems).  A kernel
// that holds tcgen05 instructions ran one CTA per SM where the same kernel
// without them ran two (measured: the CUDA occupancy query reports 1 at any
// shared-memory size), so the FP32 and FP64 instances carry none.
template <typename T, int MAXL, int THREADS, bool TC = false>
__global__ void __launch_bounds__(THREADS) k_se(const SeArgs a) {
  extern __shared__ double sm[];
  double* sE = sm;                       // per-level vectors (MAXL each)
  double* sG = sE + MAXL;
  double* sW = sG + MAXL;                // g_i exp(-E_i / k Te)
  double* sX0 = sW + MAXL;               // warm start (column scale)
  double* sR = sX0 + MAXL;               // row scale
  double* sN = sR + MAXL;                // solution (FP64)
  double* sRes = sN + MAXL;              // residual
  double* sB = sRes + MAXL;              // right-hand side (b, or -G for a Newton step)
  double* sNk = sB + MAXL;               // Newton iterate
  double* sQ = sNk + MAXL;               // collisional factor of upward rates (per lower level)
  int* sPiv = (int*)(sQ + MAXL);
  int* sPerm = sPiv + MAXL;              // the pivots as a gather
  T* sVec = (T*)(sPerm + MAXL);          // right-hand side in the factor type
  T* sPan = sVec + MAXL;                 // panel [L][nb + 1]
  T* sU12 = (T*)((char*)sPan + se_pan_bytes(MAXL));   // [nb][L]
  __shared__ unsigned long long item;
  __shared__ double red[32];
  __shared__ int flag;
  __shared__ FixExpTables sfx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;
  // the tensor-core leg (TF32 factors of the large systems): TMEM for the
  // accumulator, allocated for the whole persistent launch (the host sizes it
  // so that the CTAs resident on an SM never ask for more than its 512
  // columns); the CTA's state sits in the tail of the U12 buffer, which no
  // FP32 panel reaches (a static variable would cost the SM its second CTA)
  TcState* tcp = nullptr;
  if constexpr (TC && sizeof(T) == 4 && MAXL > kSmallL && THREADS == 256) {
    if (a.tmem_cols > 0) {
      TcState* const ts = reinterpret_cast<TcState*>(reinterpret_cast<unsigned char*>(sU12) + kTcStateOff);
      if (warp == 0) tc::tmem_alloc(&ts->taddr, (uint32_t)a.tmem_cols);
      if (tid == 0) {
        tc::bar_init(&ts->bar, 1);
        ts->phase = 0;
        ts->ncols = a.tmem_cols;
        ts->ok = 1;
        ts->bf16 = a.tc_bf16;
        ts->err = a.tc_err;
      }
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      tcp = ts;
    }
  }
  for (int k = tid; k < (int)(sizeof(FixExpTables) / 8); k += blockDim.x)
    reinterpret_cast<uint64_t*>(&sfx)[k] = reinterpret_cast<const uint64_t*>(&a.fx)[k];
  double* W = a.W64 + (int64_t)blockIdx.x * a.wlen;
  // each CTA owns L_max^2 doubles of WT, used as T (factor) or double (fallback)
  T* WT = (T*)((double*)a.WT + (int64_t)blockIdx.x * a.wlen);
  const double kB = 1.380649e-16;
  for (;;) {
    if (tid == 0) item = atomicAdd(a.counter, 1ull);
    block_sync();
    if (item >= (unsigned long long)a.n_work) break;
    const int w = a.work[item];
    const int cell = w >> 4, z = w & 15;
    const int ix = cell % a.g.nx, iy = (cell / a.g.nx) % a.g.ny, iz = cell / (a.g.nx * a.g.ny);
    const int64_t row = row_of(a.g, ix, iy, iz);
    const int off = a.level_off[z], Lz = a.level_off[z + 1] - off;
    const int L = a.levels_used ? min(a.levels_used[cell * a.n_ion + z], Lz) : Lz;
    const double Te = a.Te[row], ne = a.ne[row], dep = a.dep ? a.dep[row] : 0.0;
    const double nz = a.nion[row * a.n_ion + z];
    const double* pc = a.pops + row * a.nlev;
    const double* ups = a.ups + a.ups_off[z];
    const double sqT = sqrt(Te), kT = kB * Te;
    const bool newton = a.newton_max > 0;
    if (!(nz > 0.0)) {
      // no atoms of this ion here: zero populations, nothing to solve
      double* out = a.pops_out + row * a.nlev + off;
      for (int i = tid; i < Lz; i += blockDim.x) out[i] = 0.0;
      if (tid == 0) {
        if (a.status) a.status[cell * a.n_ion + z] = XT_SE_OK;
        if (a.iters) a.iters[cell * a.n_ion + z] = 0;
      }
      block_sync();
      continue;
    }
    // per-level data; warm start
    for (int i = tid; i < L; i += blockDim.x) {
      sE[i] = a.E[off + i];
      sG[i] = a.glev[off + i];
      sW[i] = sG[i] * exp(-(sE[i] - a.E[off]) / kT);
    }
    block_sync();
    if (a.warm) {
      for (int i = tid; i < L; i += blockDim.x) sX0[i] = a.warm[row * a.nlev + off + i];
    } else {
      double s = 0;
      for (int i = tid; i < L; i += blockDim.x) s += sW[i];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if ((tid & 31) == 0) red[tid >> 5] = s;
      block_sync();
      if (tid == 0) { double t = 0; for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k]; red[0] = t; }
      block_sync();
      const double tot = red[0];
      for (int i = tid; i < L; i += blockDim.x) sX0[i] = nz * sW[i] / tot;
    }
    block_sync();
    // Newton iterate: the warm start, kept positive
    if (newton)
      for (int i = tid; i < L; i += blockDim.x) sNk[i] = fmax(sX0[i], 1e-280 * nz);
    // collisional rate factors of the system, with w_i = g_i e^{-(E_i - E_0)/kT}:
    // down j -> i (j > i) = Y_ij cfac / g_j; up j -> i (j < i) = Y_ji cfac / g_j
    // e^{-(E_i - E_j)/kT} = Y_ji (cfac / w_j) (w_i / g_i)
    const double cfac = 8.629e-6 * ne / sqT;
    for (int i = tid; i < L; i += blockDim.x) {
      const double gi = a.glev[off + i], wi = sW[i];
      sQ[i] = cfac / wi;
      sG[i] = cfac / gi;          // from here on: the downward factor
      sW[i] = wi / gi;            // from here on: e^{-(E_i - E_0)/kT}
    }
    block_sync();
    const int nb = a.nb_bucket[min(L >> 6, 7)];
    int st = XT_SE_OK, iters = 0, nsteps = 0;
    bool ok = true;
    for (;;) {
      // optical depths from the iterate (Newton) or from the context's populations
      const double* nbeta = newton ? sNk : pc + off;
      // ---- assemble M (row-major, M[i][j] = rate j -> i) : collisions, a warp
      // per row (the collision strengths are stored symmetric)
      for (int i = warp; i < L; i += nwarp) {
        const double* ur = ups + (int64_t)i * Lz;
        double* Wr = W + (int64_t)i * L;
        const double ei = sW[i];
        for (int j = lane; j < L; j += 32) {
          const double y = ur[j];
          Wr[j] = j > i ? y * sG[j] : j < i ? y * (sQ[j] * ei) : 0.0;
        }
      }
      block_sync();
      // radiative lines of the kept levels (the lines of upper levels 1..L-1,
      // positions kA..kB-1 of down_line): each line's two rate terms, a thread
      // per line, into the panel buffer (free until the factor); then a thread
      // per upper level adds its lines' terms in a fixed order, so that every
      // entry is summed in the same order on every run (a line u -> lo writes
      // only column u and row u, which no other upper level's lines touch).
      // Without room in the buffer the thread per upper level computes them.
      const int kA = a.down_off[off + 1], kB = a.down_off[off + L], nk = kB - kA;
      double* const lbuf = (double*)sPan;
      const bool lbuffered = 2 * (size_t)nk * sizeof(double) <= se_pan_bytes(MAXL);
      auto line_terms = [&](int k, double& down, double& up_rate) {
        const int s = a.down_line[k];
        const double* Lr = a.lines + 4 * (int64_t)s;
        const int64_t lu = __double_as_longlong(Lr[3]);
        const int lo = (int)(lu & 0xFFFFFFFF) - off, u = (int)(lu >> 32) - off;
        const double tau = Lr[1] * (nbeta[lo] - Lr[2] * nbeta[u]);
        const double beta = sobolev_beta_fix(sfx, tau, nullptr);
        double Rlu = 0.0;
        if (a.rates == XT_RATES_JBAR) {
          Rlu = a.Rj[s] * beta;   // external field, Sobolev-absorbed part
        } else if (a.rates == XT_RATES_ESTIMATORS) {
          // fixed per atom: the populations of the transport pass set it
          const double net = pc[off + lo] - Lr[2] * pc[off + u];
          const int64_t sr = a.crow ? (int64_t)a.crow[row] : (int64_t)row;
          const double Sv = sr < 0 ? 0.0 : a.S[sr * a.nline + s];
          if (net > 0.0 && Sv > 0.0) Rlu = div_pos(Sv, net * (a.g.vol ? a.g.vol[row] : a.V));
        }
        down = a.A[s] * beta + Lr[2] * Rlu;                           // u -> lo
        up_rate = Rlu;                                                // lo -> u
      };
      if (lbuffered) {
        for (int k = kA + tid; k < kB; k += blockDim.x) line_terms(k, lbuf[k - kA], lbuf[nk + k - kA]);
        block_sync();
      }
      for (int u = 1 + tid; u < L; u += blockDim.x) {
        const int k0 = a.down_off[off + u], k1 = a.down_off[off + u + 1];
        for (int k = k0; k < k1; ++k) {
          const int lo = (int)(__double_as_longlong(a.lines[4 * (int64_t)a.down_line[k] + 3]) & 0xFFFFFFFF) - off;
          double down, up_rate;
          if (lbuffered) { down = lbuf[k - kA]; up_rate = lbuf[nk + k - kA]; }
          else line_terms(k, down, up_rate);
          W[(int64_t)lo * L + u] += down;
          W[(int64_t)u * L + lo] += up_rate;
        }
      }
      // non-thermal excitation from the ground level
      if (dep > 0.0 && nz > 0.0 && L > 1) {
        double s = 0;
        for (int u = 1 + tid; u < L; u += blockDim.x) s += ups[u] * (sE[u] - sE[0]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((tid & 31) == 0) red[tid >> 5] = s;
        block_sync();
        if (tid == 0) { double t = 0; for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k]; red[0] = t; }
        block_sync();
        const double denom = nz * red[0];
        if (denom > 0.0)
          for (int u = 1 + tid; u < L; u += blockDim.x) W[(int64_t)u * L] += a.eta * dep * ups[u] / denom;
      }
      block_sync();
      // diagonal: minus the total rate out of each level (column sums), 128
      // columns at a time: a warp per row, 4 columns per lane, then across warps
      {
        double* part = (double*)sPan;              // [nwarp][128], free until the factor
        for (int c0 = 0; c0 < L; c0 += 128) {
          double cs[4] = {0.0, 0.0, 0.0, 0.0};
          for (int j = warp; j < L; j += nwarp) {
            const double* Wr = W + (int64_t)j * L + c0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int i = c0 + lane + 32 * q;
              if (i < L && i != j) cs[q] += Wr[lane + 32 * q];
            }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) part[warp * 128 + lane + 32 * q] = cs[q];
          block_sync();
          for (int i = tid; i < 128 && c0 + i < L; i += blockDim.x) {
            double s = 0.0;
            for (int w = 0; w < nwarp; ++w) s += part[w * 128 + i];
            sRes[c0 + i] = -s;
          }
          block_sync();
        }
      }
      for (int i = tid; i < L; i += blockDim.x) W[(int64_t)i * L + i] = sRes[i];
      block_sync();
      for (int j = tid; j < L; j += blockDim.x) W[j] = 1.0;   // ground-level equation -> sum n = n_z
      block_sync();
      if (newton) {
        // right-hand side -G = b - M n (FP64), then the Jacobian: for every line
        // the derivative of its net downward flow F = A beta n_u - beta B J_ext
        // (n_l - g_l/g_u n_u) through beta: dF/dn_l = t, dF/dn_u = -g_l/g_u t,
        // t = beta'(tau) K (A n_u - B J_ext net); +F in row l, -F in row u
        for (int i = warp; i < L; i += nwarp) {
          const double* Wr = W + (int64_t)i * L;
          double s = 0.0;
          for (int j = lane; j < L; j += 32) s += Wr[j] * sNk[j];
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (lane == 0) sB[i] = (i == 0 ? nz : 0.0) - s;
        }
        block_sync();
        // each line's t, a thread per line, into the panel buffer (without
        // room there it is computed where it is used); then a thread per upper
        // level writes its lines' entries of column u and row u (no other
        // thread's), and a thread per lower level adds the t of the lines
        // below it to its diagonal, both in fixed line order
        const bool tbuffered = (size_t)nk * sizeof(double) <= se_pan_bytes(MAXL);
        auto line_t = [&](int k) {
          const int s = a.down_line[k];
          const double* Lr = a.lines + 4 * (int64_t)s;
          const int64_t lu = __double_as_longlong(Lr[3]);
          return line_jac_t(a, sfx, Lr, s, sNk[(int)(lu & 0xFFFFFFFF) - off], sNk[(int)(lu >> 32) - off]);
        };
        if (tbuffered) {
          for (int k = kA + tid; k < kB; k += blockDim.x) lbuf[k - kA] = line_t(k);
          block_sync();
        }
        for (int u = 1 + tid; u < L; u += blockDim.x) {
          const int k0 = a.down_off[off + u], k1 = a.down_off[off + u + 1];
          double du = 0.0;
          for (int k = k0; k < k1; ++k) {
            const double t = tbuffered ? lbuf[k - kA] : line_t(k);
            if (t == 0.0) continue;
            const double* Lr = a.lines + 4 * (int64_t)a.down_line[k];
            const int lo = (int)(__double_as_longlong(Lr[3]) & 0xFFFFFFFF) - off;
            if (lo != 0) W[(int64_t)lo * L + u] += -Lr[2] * t;
            W[(int64_t)u * L + lo] += -t;
            du += Lr[2] * t;
          }
          W[(int64_t)u * L + u] += du;
        }
        block_sync();
        for (int lo = 1 + tid; lo < L; lo += blockDim.x) {
          const int q0 = a.low_off[off + lo], q1 = a.low_off[off + lo + 1];
          double dl = 0.0;
          for (int q = q0; q < q1; ++q) {
            const int k = a.low_line[q];
            if (k >= kB) continue;                      // upper level not kept
            dl += tbuffered ? lbuf[k - kA] : line_t(k);
          }
          W[(int64_t)lo * L + lo] += dl;
        }
        // the column scale of the FP32 factor: the iterate (levels below
        // 1e-30 n_z need no relative accuracy)
        for (int i = tid; i < L; i += blockDim.x) sX0[i] = fmax(sNk[i], 1e-30 * nz);
      } else {
        for (int i = tid; i < L; i += blockDim.x) sB[i] = i == 0 ? nz : 0.0;
      }
      block_sync();
      // ---- solve W x = sB into sN
      int it_ir = 0;
      if (sizeof(T) == 8 || a.precision == XT_PREC_FP64) {
        // plain FP64: factor, solve
        double* Wd = (double*)WT;
        for (int e = tid; e < L * L; e += blockDim.x) Wd[e] = W[e];
        block_sync();
        ok = lu_factor<double>(Wd, L, min(nb, 16), sPiv, (double*)sPan, (double*)sU12);
        lu_perm(sPiv, L, sPerm);
        for (int i = tid; i < L; i += blockDim.x) sN[i] = sB[sPerm[i]];
        block_sync();
        if (ok) lu_solve<double>(Wd, L, sN);
        else st = XT_SE_SINGULAR;
      } else {
        // FP32 factor of diag(r) W diag(x0), FP64 refinement
        for (int i = tid; i < L; i += blockDim.x) sX0[i] = sX0[i] > 1e-300 ? sX0[i] : 1e-300;
        block_sync();
        if constexpr (sizeof(T) == 4) {
          // powers of two as scales: column j by 2^ex_j (x0_j rounded down to
          // one), row i by 2^er_i with er_i = -max_j (ew_ij + ex_j), so the row
          // maxima lie in [1, 2); the scaling is then exact and, with the
          // rounding to FP32, done on the integer pipe (scaled_f32)
          for (int i = warp; i < L; i += nwarp) {
            const double* Wr = W + (int64_t)i * L;
            int mx = -1 << 20;
            for (int j = lane; j < L; j += 32) {
              const int ew = (int)((__double_as_longlong(Wr[j]) >> 52) & 0x7FF);
              if (ew) mx = max(mx, ew + (int)(__double_as_longlong(sX0[j]) >> 52));
            }
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const int er = mx > -(1 << 19) ? min(max(2046 - mx, -1022), 1023) : 0;   // unbiased
            T* Tr = WT + (int64_t)i * L;
            for (int j = lane; j < L; j += 32)
              Tr[j] = scaled_f32(Wr[j], (int)(__double_as_longlong(sX0[j]) >> 52) - 1023 + er);
            if (lane == 0) sR[i] = __longlong_as_double((long long)(er + 1023) << 52);
          }
          block_sync();
          // the column scale of the refinement: x0 rounded down to a power of two
          for (int i = tid; i < L; i += blockDim.x)
            sX0[i] = __longlong_as_double(__double_as_longlong(sX0[i]) & 0x7FF0000000000000ll);
        } else {
          for (int i = warp; i < L; i += nwarp) {
            const double* Wr = W + (int64_t)i * L;
            double mx = 0;
            for (int j = lane; j < L; j += 32) mx = fmax(mx, fabs(Wr[j] * sX0[j]));
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const double r = mx > 0 ? 1.0 / mx : 1.0;
            T* Tr = WT + (int64_t)i * L;
            for (int j = lane; j < L; j += 32) Tr[j] = (T)(Wr[j] * sX0[j] * r);
            if (lane == 0) sR[i] = r;
          }
        }
        block_sync();
        // a factor that meets an exactly zero pivot (entries of the scaled matrix
        // below the FP32 range count as zero) goes to the FP64 solve below
        ok = lu_factor<T>(WT, L, nb, sPiv, sPan, sU12, tcp);
        lu_perm(sPiv, L, sPerm);
        for (int i = tid; i < L; i += blockDim.x) { sN[i] = 0.0; sRes[i] = sB[i]; }
        block_sync();
        bool conv = false;
        for (it_ir = 0; ok && it_ir < a.max_iter; ++it_ir) {
          for (int i = tid; i < L; i += blockDim.x) { const int q = sPerm[i]; sVec[i] = (T)(sRes[q] * sR[q]); }
          block_sync();
          lu_solve<T>(WT, L, sVec);
          // the error each level keeps after this correction d_k: refinement
          // contracts it by about rho = |d_k| / |d_(k-1)| per step, so about
          // d_k^2 / |d_(k-1)| where the level's corrections halve or better, else
          // |d_k| (the previous corrections sit in the panel buffer, free here);
          // relative to the solution, or for a Newton correction to its level's
          // population (the step needs it resolved below the Newton tolerance:
          // the fixed point is set by the FP64 right-hand side, not by the step)
          double dmax = 0;
          double* dprev_i = (double*)sPan;
          for (int i = tid; i < L; i += blockDim.x) {
            const double d = (double)sVec[i] * sX0[i];
            sN[i] += d;
            double e = fabs(d);
            if (it_ir > 0) {
              const double q = fabs(dprev_i[i]);
              if (e < 0.5 * q) e = e * (e / q);
            }
            dprev_i[i] = d;
            dmax = fmax(dmax, e / (newton ? sX0[i] : fmax(fabs(sN[i]), 1e-30 * nz)));
          }
          for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
          if ((tid & 31) == 0) red[tid >> 5] = dmax;
          block_sync();
          if (tid == 0) {
            double t = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmax(t, red[k]);
            flag = t < (newton ? fmax(a.tol, 1e-2 * a.newton_tol) : a.tol);
          }
          block_sync();
          if (flag && it_ir > 0) { conv = true; ++it_ir; break; }
          // residual sB - W x in FP64
          for (int i = warp; i < L; i += nwarp) {
            const double* Wr = W + (int64_t)i * L;
            double s = 0.0;
            for (int j = lane; j < L; j += 32) s += Wr[j] * sN[j];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) sRes[i] = sB[i] - s;
          }
          block_sync();
        }
        if (!conv) {
          // not converged, or no FP32 factor: the plain FP64 solve decides
          st |= XT_SE_FALLBACK;
          double* Wd = (double*)a.WT + (int64_t)blockIdx.x * a.wlen;   // reuse (FP64 sized)
          for (int e = tid; e < L * L; e += blockDim.x) Wd[e] = W[e];
          block_sync();
          // (8-column panels where the tensor-core state sits in the U12 tail:
          // 8 x 312 doubles stay clear of it)
          ok = lu_factor<double>(Wd, L, tcp ? 8 : 16, sPiv, (double*)sPan, (double*)sU12);
          lu_perm(sPiv, L, sPerm);
          for (int i = tid; i < L; i += blockDim.x) sN[i] = sB[sPerm[i]];
          block_sync();
          if (ok) lu_solve<double>(Wd, L, sN);
          else st = XT_SE_SINGULAR;
        }
      }
      block_sync();
      if (!newton) { iters = it_ir; break; }
      if (!ok) break;
      // ---- Newton step: r = max |d_i| / n_i over the levels that count; every
      // level moves by the factor 1 + lam d_i / n_i within [1/max_var, max_var]
      // (Sec. 2.2 bounds the change per step); lam = 1 once r <= 0.1, before
      // that the damping of the step (Sec. 2.2)
      {
        double r = 0.0;
        for (int i = tid; i < L; i += blockDim.x)
          if (sNk[i] >= 1e-30 * nz) r = fmax(r, fabs(sN[i]) / sNk[i]);
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
        if ((tid & 31) == 0) red[tid >> 5] = r;
        block_sync();
        if (tid == 0) { double t = 0.0; for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmax(t, red[k]); red[0] = t; }
        block_sync();
        const double rmax = red[0];
        block_sync();
        const double lam = rmax <= 0.1 ? 1.0
                         : nsteps < 10 ? 0.95 : nsteps < 35 ? 0.75 : nsteps < 50 ? 0.5 : nsteps < 90 ? 0.25 : 0.05;
        const double vmax = a.newton_maxvar, vmin = 1.0 / a.newton_maxvar;
        for (int i = tid; i < L; i += blockDim.x)
          sNk[i] *= fmin(fmax(1.0 + lam * sN[i] / sNk[i], vmin), vmax);
        block_sync();
        ++nsteps;
        if (rmax <= a.newton_tol) break;
        if (nsteps >= a.newton_max) { st |= XT_SE_NOCONV; break; }
      }
    }
    if (newton) {
      iters = nsteps;
      for (int i = tid; i < L; i += blockDim.x) sN[i] = sNk[i];
    }
    block_sync();
    double* out = a.pops_out + row * a.nlev + off;
    for (int i = tid; i < Lz; i += blockDim.x) out[i] = i < L ? sN[i] : 0.0;
    if (tid == 0) {
      if (a.status) a.status[cell * a.n_ion + z] = st;
      if (a.iters) a.iters[cell * a.n_ion + z] = iters;
    }
    block_sync();
  }
  if constexpr (TC) {
    if (tcp) {                           // every thread left the loop together
      tc::fence_before();
      __syncthreads();
      if (warp == 0) tc::tmem_free(tcp->taddr, (uint32_t)a.tmem_cols);
    }
  }
}

// Boltzmann populations of the kept levels (XT_WARM_LTE for transport use).
__global__ void k_lte(Geometry g, int nlev, int n_ion, const int* __restrict__ level_off,
                      const double* __restrict__ E, const double* __restrict__ glev,
                      const double* __restrict__ nion, const double* __restrict__ Te,
                      const int* __restrict__ levels_used, double* __restrict__ out) {
  const int64_t n = g.ncell * n_ion;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = e / n_ion;
    const int z = (int)(e - cell * n_ion);
    const int ix = (int)(cell % g.nx), iy = (int)((cell / g.nx) % g.ny), iz = (int)(cell / ((int64_t)g.nx * g.ny));
    const int64_t row = row_of(g, ix, iy, iz);
    const int off = level_off[z], Lz = level_off[z + 1] - off;
    const int L = levels_used ? min(levels_used[e], Lz) : Lz;
    const double kT = 1.380649e-16 * Te[row];
    double s = 0;
    for (int i = 0; i < L; ++i) s += glev[off + i] * exp(-(E[off + i] - E[off]) / kT);
    const double nz = nion[row * n_ion + z];
    for (int i = 0; i < Lz; ++i)
      out[row * nlev + off + i] = i < L ? nz * glev[off + i] * exp(-(E[off + i] - E[off]) / kT) / s : 0.0;
  }
}

int lte_fill(xt_ctx* c, const int* levels_used_dev, double* out) {
  const int64_t n = c->geo.ncell * c->n_ion;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  k_lte<<<std::max(blocks, 1), 256, 0, c->stream>>>(c->geo, c->nlev, c->n_ion, c->d_level_off, c->d_E, c->d_g,
                                                  c->d_nion, c->d_Te, levels_used_dev, out);
  XT_CUDA(c, cudaGetLastError());
  return XT_OK;
}

static size_t se_smem(size_t tsize, int maxl) {
  return 10 * (size_t)maxl * sizeof(double) + 2 * (size_t)maxl * sizeof(int) + (size_t)maxl * tsize +
         se_pan_bytes(maxl) + (size_t)kSeNbMax * maxl * tsize;
}

}  // namespace xt

using namespace xt;

extern "C" int solve_nlte(xt_ctx* c, const xt_nlte_params* p, double* pops_out, int32_t* status_out,
                          xt_nlte_stats* stats) {
  if (!c || !p) return fail(c, XT_EINVAL, "solve_nlte: null argument");
  if (!c->have_pops || !c->have_atoms) return fail(c, XT_ESTATE, "solve_nlte: load_atomic_data and set_populations first");
  if (!c->d_nion) return fail(c, XT_ESTATE, "solve_nlte: n_ion_density was not given to load_atomic_data");
  if (c->n_ion > 16) return fail(c, XT_EINVAL, "solve_nlte: at most 16 ions");
  if (p->precision != XT_PREC_FP64 && p->precision != XT_PREC_FP32_IR && p->precision != XT_PREC_TF32_IR &&
      p->precision != XT_PREC_BF16_IR)
    return fail(c, XT_EINVAL, "solve_nlte: precision");
  if (p->rates == XT_RATES_ESTIMATORS && !c->have_S)
    return fail(c, XT_ESTATE, "solve_nlte: estimator rates need a transport pass with the current populations");
  if (p->rates == XT_RATES_JBAR && !(p->jbar_W > 0 && p->jbar_TR > 0)) return fail(c, XT_EINVAL, "solve_nlte: jbar_W, jbar_TR > 0");
  if (!p->upsilon) return fail(c, XT_EINVAL, "solve_nlte: upsilon is required");
  if (p->warm == XT_WARM_GIVEN && !p->warm_in) return fail(c, XT_EINVAL, "solve_nlte: warm_in required");
  if (p->warm < XT_WARM_CURRENT || p->warm > XT_WARM_SURROGATE) return fail(c, XT_EINVAL, "solve_nlte: warm");
  if (p->precision != XT_PREC_FP64 && (p->max_iter < 1 || !(p->tol > 0))) return fail(c, XT_EINVAL, "solve_nlte: max_iter >= 1, tol > 0");
  if (p->newton_max < 0 || (p->newton_max > 0 && (!(p->newton_tol > 0) || !(p->newton_maxvar > 1))))
    return fail(c, XT_EINVAL, "solve_nlte: newton_max >= 0, newton_tol > 0, newton_maxvar > 1");
  cudaSetDevice(c->device);
  const Geometry& G = c->geo;
  int Lmax = 0;
  for (int z = 0; z < c->n_ion; ++z) Lmax = std::max(Lmax, c->h_level_off[z + 1] - c->h_level_off[z]);
  if (Lmax > kSeMaxL) return fail(c, XT_EINVAL, "solve_nlte: more than 320 levels in an ion");
  int rc;
  const int64_t nsys = G.ncell * c->n_ion;
  // levels kept and the longest-first work list (counting sort by L)
  std::vector<int> used(nsys);
  if (p->levels_used) {
    if ((rc = copy(c, used.data(), p->levels_used, nsys * sizeof(int), "levels_used"))) return rc;
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  std::vector<int64_t> cnt(Lmax + 2, 0);
  for (int64_t e = 0; e < nsys; ++e) {
    const int z = (int)(e % c->n_ion);
    const int Lz = c->h_level_off[z + 1] - c->h_level_off[z];
    int L = p->levels_used ? used[e] : Lz;
    if (L < 1 || L > Lz) return fail(c, XT_EINVAL, "solve_nlte: levels_used out of range at " + std::to_string(e));
    used[e] = L;
    cnt[L]++;
  }
  // bucket of L starts after every longer bucket: start[L] = sum_{L' > L} cnt[L']
  std::vector<int64_t> start(Lmax + 2, 0);
  for (int L = Lmax - 1; L >= 1; --L) start[L] = start[L + 1] + cnt[L + 1];
  std::vector<int> work(nsys);
  // estimator rates from a host-held store: the systems go group by group
  // (each group's cells are a contiguous natural range), longest first within
  // a group, and each group's launch reads its staged slab
  const bool grouped = c->S_groups > 0 && p->rates == XT_RATES_ESTIMATORS;
  const int NG = grouped ? c->S_groups : 1;
  std::vector<int64_t> g_begin(NG + 1, 0), g_big(NG, 0);
  if (!grouped) {
    std::vector<int64_t> fill(start);
    for (int64_t e = 0; e < nsys; ++e) {
      const int64_t cell = e / c->n_ion;
      const int z = (int)(e % c->n_ion);
      work[fill[used[e]]++] = (int)(cell * 16 + z);
    }
  } else {
    const int64_t per_g = nsys / NG;                // systems of a group (cells x ions)
    for (int g = 0; g < NG; ++g) {
      const int64_t e0 = (int64_t)g * per_g, e1 = e0 + per_g;
      std::vector<int64_t> cg(Lmax + 2, 0), sg(Lmax + 2, 0);
      for (int64_t e = e0; e < e1; ++e) cg[used[e]]++;
      for (int L = Lmax - 1; L >= 1; --L) sg[L] = sg[L + 1] + cg[L + 1];
      for (int64_t e = e0; e < e1; ++e) {
        const int64_t cell = e / c->n_ion;
        const int z = (int)(e % c->n_ion);
        work[e0 + sg[used[e]]++] = (int)(cell * 16 + z);
      }
      g_begin[g] = e0;
      g_big[g] = 0;
      for (int L = Lmax; L > kSmallL; --L) g_big[g] += cg[L];
    }
    g_begin[NG] = nsys;
  }
  // buffers of the solve, kept in the context between calls
  auto& B = c->se;
  std::vector<int64_t> ups_off(c->n_ion + 1, 0);
  for (int z = 0; z < c->n_ion; ++z) {
    const int64_t Lz = c->h_level_off[z + 1] - c->h_level_off[z];
    ups_off[z + 1] = ups_off[z] + Lz * Lz;
  }
  const size_t ups_n = (size_t)ups_off[c->n_ion];
  const int pi = p->precision == XT_PREC_FP64 ? 0 : 1;           // kernel type: double / float
  const bool tcore = p->precision == XT_PREC_TF32_IR || p->precision == XT_PREC_BF16_IR;
  const int ti = tcore ? 2 : pi;                                   // tuning slot
  const size_t tsz = pi == 0 ? sizeof(double) : sizeof(float);
  // systems with more than kSmallL levels go to the large kernel, the rest
  // (the tail of the longest-first list) to the small one
  const int64_t n_big = Lmax > kSmallL ? start[kSmallL] : 0, n_small = nsys - n_big;
  const size_t smem = se_smem(tsz, kSeMaxL), smem_s = se_smem(tsz, kSmallL);
  int per_sm = 0, per_sm_s = 0;
  if (pi == 0) {
    cudaFuncSetAttribute(k_se<double, kSeMaxL, kSeThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_se<double, kSeMaxL, kSeThreads>, kSeThreads, smem);
    cudaFuncSetAttribute(k_se<double, kSmallL, kSmallThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, k_se<double, kSmallL, kSmallThreads>, kSmallThreads, smem_s);
  } else if (ti == 2) {
    // the occupancy query reports one CTA per SM for the instance that holds
    // tcgen05 code, but the SM runs two (measured: 1.55x faster launched at
    // two per SM); the launch takes the residency of the same kernel without
    // that code (same shared memory, more registers)
    cudaFuncSetAttribute(k_se<float, kSeMaxL, kSeThreads, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_se<float, kSeMaxL, kSeThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_se<float, kSeMaxL, kSeThreads>, kSeThreads, smem);
    cudaFuncSetAttribute(k_se<float, kSmallL, kSmallThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, k_se<float, kSmallL, kSmallThreads>, kSmallThreads, smem_s);
  } else {
    cudaFuncSetAttribute(k_se<float, kSeMaxL, kSeThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_se<float, kSeMaxL, kSeThreads>, kSeThreads, smem);
    cudaFuncSetAttribute(k_se<float, kSmallL, kSmallThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, k_se<float, kSmallL, kSmallThreads>, kSmallThreads, smem_s);
  }
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * sms, n_big));
  const int grid_s = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(per_sm_s, 1) * sms, n_small));
  const int64_t wlen = (int64_t)Lmax * Lmax, wlen_s = (int64_t)kSmallL * kSmallL;
  const size_t wbytes = ((size_t)grid * wlen + (size_t)grid_s * wlen_s) * sizeof(double);
  const size_t pops_n = (size_t)G.ncell * c->nlev;
#define SE_GROW(ptr, have, need, elt, what)                                           \
  do {                                                                                \
    if ((have) < (need)) {                                                            \
      (have) = 0;                                                                     \
      if ((rc = alloc(c, (void**)&(ptr), (size_t)(need) * (elt), what))) return rc;   \
      (have) = (need);                                                                \
    }                                                                                 \
  } while (0)
  SE_GROW(B.ups, B.ups_n, ups_n, sizeof(double), "upsilon");
  if (!B.upsoff && (rc = alloc(c, (void**)&B.upsoff, 17 * sizeof(int64_t), "upsilon offsets"))) return rc;
  if (B.nsys < nsys) {
    B.nsys = 0;
    if ((rc = alloc(c, (void**)&B.work, nsys * sizeof(int), "work list"))) return rc;
    if ((rc = alloc(c, (void**)&B.used, nsys * sizeof(int), "levels used"))) return rc;
    if ((rc = alloc(c, (void**)&B.iters, nsys * sizeof(double), "iterations"))) return rc;
    if ((rc = alloc(c, (void**)&B.status, nsys * sizeof(int), "status"))) return rc;
    B.nsys = nsys;
  }
  if (!B.cnt && (rc = alloc(c, (void**)&B.cnt, 8 * sizeof(unsigned long long), "counter"))) return rc;
  SE_GROW(B.pops_new, B.pops_n, pops_n, sizeof(double), "new populations");
  if (B.wbytes < wbytes) {
    B.wbytes = 0;
    if ((rc = alloc(c, (void**)&B.W64, wbytes, "workspace"))) return rc;
    if ((rc = alloc(c, (void**)&B.WT, wbytes, "workspace"))) return rc;
    B.wbytes = wbytes;
  }
  {
    // the kernel reads the collision strengths by rows: store them symmetric
    std::vector<double> ups(ups_n);
    if ((rc = copy(c, ups.data(), p->upsilon, ups_n * sizeof(double), "upsilon"))) return rc;
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int z = 0; z < c->n_ion; ++z) {
      const int64_t Lz = c->h_level_off[z + 1] - c->h_level_off[z];
      double* u = ups.data() + ups_off[z];
      for (int64_t i = 0; i < Lz; ++i)
        for (int64_t j = 0; j < i; ++j) u[i * Lz + j] = u[j * Lz + i];
    }
    if ((rc = copy(c, B.ups, ups.data(), ups_n * sizeof(double), "upsilon"))) return rc;
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  if ((rc = copy(c, B.upsoff, ups_off.data(), ups_off.size() * sizeof(int64_t), "upsilon offsets"))) return rc;
  if ((rc = copy(c, B.work, work.data(), nsys * sizeof(int), "work list"))) return rc;
  if ((rc = copy(c, B.used, used.data(), nsys * sizeof(int), "levels used"))) return rc;
  if (p->levels_used) {
    if (!B.used_nat || B.used_nat_n < nsys) {
      if ((rc = alloc(c, (void**)&B.used_nat, nsys * sizeof(int), "levels used"))) return rc;
      B.used_nat_n = nsys;
    }
    if ((rc = copy(c, B.used_nat, p->levels_used, nsys * sizeof(int), "levels used"))) return rc;
  }
  if (p->rates == XT_RATES_JBAR) {
    // R_lu = B_lu W B_nu(T_R), B_lu = 4 pi K / (h c t) with K = (pi e^2 / m_e c) f lambda t
    std::vector<double> packed(4 * (size_t)c->nline), Rj(c->nline);
    XT_CUDA(c, cudaMemcpyAsync(packed.data(), c->d_lines, packed.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int s = 0; s < c->nline; ++s) {
      const double nu = packed[4 * s], K = packed[4 * s + 1];
      const double Bl = 4.0 * kPi * K / (kH * kC * c->t);
      const double x = kH * nu / (1.380649e-16 * p->jbar_TR);
      Rj[s] = Bl * p->jbar_W * 2.0 * kH * nu * nu * nu / (kC * kC) / std::expm1(x);
    }
    SE_GROW(B.Rj, B.Rj_n, c->nline, sizeof(double), "jbar rates");
    if ((rc = copy(c, B.Rj, Rj.data(), c->nline * sizeof(double), "jbar rates"))) return rc;
  }
  const double* warm = c->d_pops;
  if (p->warm == XT_WARM_GIVEN) {
    SE_GROW(B.warm, B.warm_n, pops_n, sizeof(double), "warm start");
    if ((rc = ensure_scratch(c, pops_n * sizeof(double)))) return rc;
    if ((rc = copy(c, c->d_scratch, p->warm_in, pops_n * sizeof(double), "warm start"))) return rc;
    if ((rc = nat_to_row(c, (const double*)c->d_scratch, B.warm, c->nlev))) return rc;
    warm = B.warm;
  } else if (p->warm == XT_WARM_LTE) {
    warm = nullptr;
  } else if (p->warm == XT_WARM_SURROGATE) {
    SE_GROW(B.warm, B.warm_n, pops_n, sizeof(double), "warm start");
    int* d_lu = nullptr;
    if (p->levels_used) d_lu = B.used_nat;
    if ((rc = surrogate_warm(c, p->rates, p->jbar_W, p->jbar_TR, d_lu, B.warm))) return rc;
    warm = B.warm;
  }
  SeArgs a;
  std::memset(&a, 0, sizeof(a));
  fixexp_tables(&a.fx);
  a.g = G; a.nlev = c->nlev; a.n_ion = c->n_ion; a.nline = c->nline;
  a.level_off = c->d_level_off; a.E = c->d_E; a.glev = c->d_g; a.nion = c->d_nion;
  a.Te = c->d_Te; a.ne = c->d_ne; a.dep = c->d_dep; a.pops = c->d_pops; a.warm = warm;
  a.pops_out = B.pops_new; a.status = B.status; a.lines = c->d_lines; a.A = c->d_A;
  a.down_off = c->d_down_off; a.down_line = c->d_down_line; a.S = c->d_S; a.Rj = B.Rj;
  a.crow = c->S_compact ? c->d_crow : nullptr;
  a.low_off = c->d_low_off; a.low_line = c->d_low_line;
  a.rates = p->rates; a.V = G.dx * G.dy * G.dz; a.ups = B.ups; a.ups_off = B.upsoff;
  a.levels_used = B.used; a.work = B.work; a.n_work = n_big; a.counter = B.cnt;
  a.W64 = B.W64; a.WT = B.WT; a.wlen = wlen; a.precision = p->precision; a.tol = p->tol;
  a.eta = p->eta_nt; a.max_iter = p->max_iter; a.iters = B.iters;
  a.newton_max = p->newton_max; a.newton_tol = p->newton_tol; a.newton_maxvar = p->newton_maxvar;
  // TF32 or BF16 factors: the large systems' trailing updates on the tensor cores, with
  // TMEM columns such that the CTAs resident on an SM fit its 512 (a CTA's
  // allocation would otherwise wait for one that never frees it)
  if (tcore) {
    // residency bound by shared memory (1 KB per CTA reserved by the system),
    // whatever the launch assumed: TMEM columns x resident CTAs <= 512
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device);
    cudaFuncAttributes fa_tc;
    cudaFuncGetAttributes(&fa_tc, k_se<float, kSeMaxL, kSeThreads, true>);
    const int res_smem = std::max(1, (int)((size_t)smem_sm / (smem + fa_tc.sharedSizeBytes + 1024)));
    const int cols = 512 / std::max(std::max(per_sm, res_smem), 1);
    int pw = 32;
    while (pw * 2 <= cols && pw < 256) pw *= 2;
    a.tmem_cols = cols >= 32 ? pw : 0;
    a.tc_err = B.cnt + 7;
    a.tc_bf16 = p->precision == XT_PREC_BF16_IR;
  }
  SeArgs as = a;                         // the small systems: own work range, counter, workspace
  as.tmem_cols = 0;
  as.work = B.work + n_big; as.n_work = n_small; as.counter = B.cnt + 1;
  as.W64 = B.W64 + (size_t)grid * wlen; as.WT = B.WT + (size_t)grid * wlen; as.wlen = wlen_s;
  // one kernel (small = the 64-level one) on a work range
  auto launch_one = [&](const SeArgs& args, bool small, int g_, cudaStream_t s_) {
    if (args.n_work <= 0) return;
    if (small) {
      if (pi == 0) k_se<double, kSmallL, kSmallThreads><<<g_, kSmallThreads, smem_s, s_>>>(args);
      else k_se<float, kSmallL, kSmallThreads><<<g_, kSmallThreads, smem_s, s_>>>(args);
    } else {
      if (pi == 0) k_se<double, kSeMaxL, kSeThreads><<<g_, kSeThreads, smem, s_>>>(args);
      else if (ti == 2) k_se<float, kSeMaxL, kSeThreads, true><<<g_, kSeThreads, smem, s_>>>(args);
      else k_se<float, kSeMaxL, kSeThreads><<<g_, kSeThreads, smem, s_>>>(args);
    }
  };
  auto launch_on = [&](const SeArgs& big, const SeArgs& small, cudaStream_t s_) {
    cudaMemsetAsync(B.cnt, 0, 2 * sizeof(unsigned long long), s_);   // the two work counters
    launch_one(big, false, grid, s_);
    launch_one(small, true, grid_s, s_);
  };
  // ---- autotuner: panel width per 64-level bucket, timed on a sample of each
  // (the tensor-core leg keeps panels of 32 columns, the width its operand tiles take)
  if (p->autotune && !B.tuned[ti] && !grouped && ti != 2) {
    const int cand[3] = {8, 16, 32};
    for (int b = 0; b < 8; ++b) {
      // systems with L in [64 b, 64 b + 63] are contiguous in the longest-first list
      int64_t lo = -1, hi = -1;
      for (int L = std::min(64 * b + 63, Lmax); L >= std::max(1, 64 * b); --L)
        if (cnt[L] > 0) { if (lo < 0 || start[L] < lo) lo = start[L]; hi = std::max(hi, start[L] + cnt[L]); }
      if (lo < 0) continue;
      const int64_t n = std::min<int64_t>(hi - lo, 2048);
      float best = 1e30f;
      for (int k = 0; k < 3; ++k) {
        if (pi == 0 && cand[k] > 16) continue;
        const bool small = lo >= n_big;               // the sample lies in the small range
        SeArgs t_ = small ? as : a;
        t_.work = B.work + lo;
        t_.n_work = n;
        for (int q = 0; q < 8; ++q) t_.nb_bucket[q] = cand[k];
        const int g_ = (int)std::min<int64_t>(small ? grid_s : grid, n);
        cudaMemsetAsync(B.cnt, 0, 8 * sizeof(unsigned long long), c->stream);
        launch_one(t_, small, g_, c->stream);           // warm
        cudaMemsetAsync(B.cnt, 0, 8 * sizeof(unsigned long long), c->stream);
        XT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
        launch_one(t_, small, g_, c->stream);
        XT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
        XT_CUDA(c, cudaEventSynchronize(c->ev1));
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        if (ms < best) { best = ms; B.nb[ti][b] = cand[k]; }
      }
    }
    B.tuned[ti] = true;
  }
  for (int k = 0; k < 8; ++k) a.nb_bucket[k] = as.nb_bucket[k] = B.nb[ti][k];
  XT_CUDA(c, cudaMemsetAsync(B.cnt + 7, 0, sizeof(unsigned long long), c->stream));   // tensor-core give-ups
  XT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  if (grouped) {
    const int64_t cells_g = G.ncell / NG;
    const size_t slab_n = (size_t)cells_g * c->nline;
    for (int g = 0; g < NG; ++g) {
      if (c->S_valid.size() == (size_t)NG && c->S_valid[g])
        XT_CUDA(c, cudaMemcpyAsync(c->d_S, c->h_S + (size_t)g * slab_n, slab_n * sizeof(double),
                                   cudaMemcpyHostToDevice, c->stream));
      else
        XT_CUDA(c, cudaMemsetAsync(c->d_S, 0, slab_n * sizeof(double), c->stream));
      SeArgs ag = a, asg = as;
      ag.S = asg.S = c->d_S - (int64_t)g * (int64_t)slab_n;   // row r of the group at S + r nline
      ag.work = B.work + g_begin[g];
      ag.n_work = g_big[g];
      asg.work = B.work + g_begin[g] + g_big[g];
      asg.n_work = g_begin[g + 1] - g_begin[g] - g_big[g];
      launch_on(ag, asg, c->stream);
    }
  } else if (p->use_graph) {
    // one captured pair of launches per argument set, replayed on later calls
    std::vector<unsigned char> key(2 * sizeof(a) + 3 * sizeof(int));
    std::memcpy(key.data(), &a, sizeof(a));
    std::memcpy(key.data() + sizeof(a), &as, sizeof(as));
    std::memcpy(key.data() + 2 * sizeof(a), &grid, sizeof(int));
    std::memcpy(key.data() + 2 * sizeof(a) + sizeof(int), &grid_s, sizeof(int));
    std::memcpy(key.data() + 2 * sizeof(a) + 2 * sizeof(int), &pi, sizeof(int));
    int gi = -1;
    for (size_t k = 0; k < B.graph_keys.size(); ++k) if (B.graph_keys[k] == key) gi = (int)k;
    if (gi < 0) {
      // captured on the context's own stream (the caller's may be the legacy
      // default stream, which cannot be captured); replayed on the caller's
      cudaGraph_t graph;
      XT_CUDA(c, cudaStreamSynchronize(c->stream));
      XT_CUDA(c, cudaStreamBeginCapture(c->side, cudaStreamCaptureModeThreadLocal));
      launch_on(a, as, c->side);
      XT_CUDA(c, cudaStreamEndCapture(c->side, &graph));
      cudaGraphExec_t ex;
      XT_CUDA(c, cudaGraphInstantiate(&ex, graph, 0));
      cudaGraphDestroy(graph);
      if (B.graphs.size() >= 4) { cudaGraphExecDestroy(B.graphs.front()); B.graphs.erase(B.graphs.begin()); B.graph_keys.erase(B.graph_keys.begin()); }
      B.graphs.push_back(ex);
      B.graph_keys.push_back(key);
      gi = (int)B.graphs.size() - 1;
    }
    XT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
    XT_CUDA(c, cudaGraphLaunch(B.graphs[gi], c->stream));
  } else {
    launch_on(a, as, c->stream);
  }
  XT_CUDA(c, cudaGetLastError());
  XT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  std::vector<int> status(nsys);
  std::vector<double> iters(nsys);
  XT_CUDA(c, cudaMemcpyAsync(status.data(), B.status, nsys * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  XT_CUDA(c, cudaMemcpyAsync(iters.data(), B.iters, nsys * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  float ms = 0;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  // the new populations replace the context's (estimators refer to the old ones);
  // the old buffer becomes the next call's output
  std::swap(c->d_pops, B.pops_new);
  c->have_S = false;
  if (c->qoff_mode == XT_EMIT_LINES) c->qoff_N = -1;
  int64_t nfb = 0, nsing = 0, nnc = 0;
  double itmax = 0, itsum = 0, flops_lu = 0, flops_as = 0;
  for (int64_t e = 0; e < nsys; ++e) {
    if (status[e] & XT_SE_FALLBACK) ++nfb;
    if (status[e] & XT_SE_SINGULAR) ++nsing;
    if (status[e] & XT_SE_NOCONV) ++nnc;
    itmax = std::max(itmax, iters[e]);
    itsum += iters[e];
    const double L = used[e];
    const double solves = p->newton_max > 0 ? std::max(iters[e], 1.0) : 1.0;   // factorizations
    flops_lu += solves * 2.0 / 3.0 * L * L * L;
    flops_as += solves * 4.0 * L * L;
  }
  if (status_out) {
    if ((rc = copy(c, status_out, status.data(), nsys * sizeof(int), "status"))) return rc;
  }
  if (pops_out) {
    if ((rc = get_populations(c, pops_out, (size_t)G.ncell * c->nlev))) return rc;
  }
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->systems = (double)nsys;
    stats->fp64_fallbacks = (double)nfb;
    stats->singular = (double)nsing;
    stats->max_iter_used = itmax;
    stats->mean_iter = nsys ? itsum / nsys : 0;
    stats->solve_ms = ms;
    stats->assemble_flops = flops_as;
    stats->lu_flops = flops_lu;
    for (int k = 0; k < 8; ++k) stats->panel_width[k] = a.nb_bucket[k];
    stats->not_converged = (double)nnc;
  }
  if (tcore) {
    unsigned long long gave_up = 0;
    XT_CUDA(c, cudaMemcpy(&gave_up, B.cnt + 7, sizeof(gave_up), cudaMemcpyDeviceToHost));
    if (gave_up > 0)
      return fail(c, XT_ETIMEOUT, "solve_nlte: " + std::to_string(gave_up) +
                                      " CTAs did not see a tensor-core MMA complete within the bounded wait");
  }
  if (nsing > 0) return fail(c, XT_ENOTCONV, "solve_nlte: " + std::to_string(nsing) + " singular systems");
  return XT_OK;
}
