// Packet transport through the homologous Cartesian grid (A2-A6).
//
// Kernels per chunk of packets (Secs. 2.3, 2.3.2 of the paper); in attenuation
// mode without subdomain rounds the trace kernel emits each packet itself when
// a lane takes it (no pool round trip), otherwise k_emit fills the pool first:
//   k_emit     one thread per packet, all lanes doing the same work: emitting
//              cell from the integer packet quota, position uniform in the
//              cell, isotropic direction, comoving frequency from the cell's
//              emission (flat-nu band, or lines weighted by A dE beta N_u,
//              Eq. (thin_emissivity)); lab frequency nu_cmf / (1 - n.r/ct); the
//              cell-walk state (distance to the next wall along each axis and
//              the distance between walls).  Written to a packet pool (SoA).
//              The quotients and the direction's square root run on the
//              integer pipe (fixexp.cuh), and the searches for the emitting
//              cell and the first line start from guide tables.
//   k_trace    persistent: every lane owns one packet; a lane whose packet ends
//              takes the next pool entry at once (warp-aggregated counter), so
//              warps never wait for their longest-lived packet.  One loop
//              iteration is one cell segment: the comoving frequency at the wall,
//              nu0 - (nu_lab/ct) s_wall, bounds the lines met in the cell (every
//              line with nu_end < nu_line <= current nu, in descending order).
//              Lines with tau_S > tau_min (Eq. (tau_Sobolev)) attenuate the
//              packet by 1 - e^-tau and add dN / f_corr to the estimator; the
//              packet stops once its photon energy at the line is below e_cut of
//              its starting energy.  Scatter mode absorbs the whole packet with
//              probability 1 - e^-tau and re-emits it in a down-line of the upper
//              level (weights A beta) or destroys it collisionally.
//   k_escape   escaped packets: lab energy into (viewing direction, log-lambda
//              bin), done apart so that the trace loop carries no trigonometry.
// With subdomain rounds (Sec. 2.4.1) a packet that crosses into another
// subdomain stops and is queued; the queue is sorted by destination subdomain
// and traced again in the next round, until no packet is left.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "fixexp.cuh"
#include "philox.cuh"
#include "quota.h"
#include "raysched.h"
#include "xt_internal.cuh"

namespace xt {

enum PoolField { F_R0X, F_R0Y, F_R0Z, F_NX, F_NY, F_NZ, F_TMX, F_TMY, F_TMZ, F_TDX, F_TDY, F_TDZ,
                 F_NULAB, F_NU0, F_N, F_T, F_SPI, NF };   // F_SPI: start of the photoionization segment

struct Pool {           // structure of arrays, capacity cap
  int64_t cap;
  double* f;            // [NF][cap]
  int* cell;            // current cell, packed ix | iy << 10 | iz << 20
  int* cursor;          // next sorted line to test
  int* events;
  int* ndraw;           // scatter draws used
  int* inter;           // scatter interactions
  int64_t* pid;         // packet id
  __device__ __forceinline__ double& F(int k, int64_t i) const { return f[(int64_t)k * cap + i]; }
};

// Guide tables of the emission's two inversions (Chen & Asau's guide-table
// method for discrete inverse transforms): the emitting cell of packet p lies
// between the cells of packets (p >> 6) 2^6 and ((p >> 6) + 1) 2^6, and the
// first line below a band frequency nu_lo + u span between the first lines
// below the edges of u's bucket of width 2^-16; the binary searches then run
// over a few entries instead of the whole tables.
constexpr int kQGuideShift = 6;
constexpr int kNuGuideShift = 37;                 // 2^16 buckets of the 53-bit uniform
constexpr int kNuGuideN = (1 << (53 - kNuGuideShift)) + 1;

// The RAYS sampler's tables (Sec. 2.3): ray r = (emitting-cell rank, emitting
// bin rank, viewer) in row-major order.
struct RayTables {
  int64_t nbin, nview;
  const int* __restrict__ rcell;       // natural index of each emitting cell
  const double* __restrict__ bin_nu;   // [nbin] comoving start frequency (the bin's reddest feature)
  const int* __restrict__ bin_cursor;  // [nbin] first line its rays test
  const double* __restrict__ bin_frac; // band: [nbin] the bin's share of the band
  const double* __restrict__ Ebin;     // lines: [row][nbin] the cell's emission in the bin
  const double* __restrict__ view;     // [nview][4] direction of the viewer's centre, dOmega / 4 pi
  const int* __restrict__ win_len;     // [nbin] lines a ray of the bin can reach (staged window)
};

struct EmitArgs {
  Geometry g;
  const int64_t* __restrict__ qoff;   // natural [ncell+1]
  const int* __restrict__ qguide;     // cell of packet j 2^6 (nullptr: search all of qoff)
  const int* __restrict__ nuguide;    // band: first line with nu <= the bucket edges (or nullptr)
  const double* __restrict__ Epk;     // natural [ncell] packet energy L_c / n_c
  const double* __restrict__ Eph;     // natural [ncell] packet energy / h
  const double* __restrict__ cdf;     // [row][caller line] (line emission)
  const double* __restrict__ Lc;      // natural [ncell]
  const int* __restrict__ sorted_of;
  const double* __restrict__ nu_tab;  // sorted
  int nline, emission;
  uint64_t seed;
  double nu_lo, nu_hi, nu_span, e_cut;   // nu_span = nu_hi - nu_lo
  const double* __restrict__ wall;    // lower cell walls -R + i d per axis [nx + ny + nz], or null
  int64_t p_begin, n;
  Pool pool;
  double* __restrict__ ledger;
  double* __restrict__ records;       // record of packet p at (p - rec_base)
  int64_t rec_base;
  FixTrigTables trig;
  int rays;                           // the RAYS sampler instead of Monte Carlo packets
  RayTables ray;
};

struct TraceArgs {
  Geometry g;
  const double2* __restrict__ lines;  // per sorted line: nu, K, gratio, (lo, up)
  int nline, nlev;
  const double* __restrict__ pops;    // [row][nlev]
  double* __restrict__ S;             // [row][sorted line]
  const double* __restrict__ A;       // sorted
  const int* __restrict__ down_off;
  const int* __restrict__ down_line;
  const double* __restrict__ Te;      // row order
  const double* __restrict__ ne;
  const double* __restrict__ ups_down;
  const double* __restrict__ glev;
  Pool pool;
  const int* __restrict__ list;       // pool indices to trace (nullptr: 0..n_list-1)
  int64_t n_list;
  unsigned long long* __restrict__ counter;
  int* __restrict__ esc;              // escaped pool indices
  unsigned long long* __restrict__ n_esc;
  int* __restrict__ out;              // queued pool indices (subdomain rounds)
  unsigned long long* __restrict__ n_out;
  int rounds;                         // 0: no subdomain boundaries
  uint64_t seed;
  double tau_min, ct, inv_ct;
  int64_t max_events;
  double* __restrict__ ledger;
  double* __restrict__ records;
  int64_t rec_base;
  FixExpTables fx;
  FixTrigTables trig;
  const int* __restrict__ rtab;       // [nx + ny + nz] separable blocked-row offsets
  int64_t* __restrict__ slotlog;      // touched estimator slots: one segment per block
  int64_t* __restrict__ seg_n;        // entries per segment (kept across launches)
  int64_t seg_len;
  unsigned long long* __restrict__ log_overflow;
  int fused;                          // attenuation without rounds: emit packets in the refill
  EmitArgs em;                        // (packet p = em.p_begin + pool slot)
  int64_t row0;                       // first row held by S (a streamed group's slab; else 0)
  int grp_nz;                         // rounds == 2: cells along z per streamed group
  int dom_zlo, dom_zhi;               // rounds == 3: the domain's z layers
  const int* __restrict__ crow;       // compact store: the cell's row in S, -1 none (nullptr: dense)
  // photoionization (the PI instance): levels sorted by threshold frequency,
  // descending; per-cell suffix sums and accumulators (see pi_segment)
  int npi;
  const double* __restrict__ pi_nuth;  // [npi] Hz
  const double* __restrict__ pi_sig;   // [npi] sigma = sig lambda^3
  const int* __restrict__ pi_lev;      // [npi]
  const double* __restrict__ kappa;    // [row][npi+1]
  double* __restrict__ piG;            // [row][npi+1]
  double* __restrict__ piD;            // [row][npi]
  double* __restrict__ piH;            // [row]
};

struct EscArgs {
  Pool pool;
  const int* __restrict__ esc;
  int64_t n_esc;
  double* __restrict__ spec;
  int n_theta, n_phi, nbins;
  double lam0, log1p_dlog;
  double* __restrict__ ledger;
  double* __restrict__ records;
  int64_t rec_base;
};

__device__ __forceinline__ long long bits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double dabs_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll);
}

// 32-byte line record: x = nu, y = K, z = g_l/g_u, w = (lo | up << 32) bit pattern
struct LineRec { double x, y, z, w; };
__device__ __forceinline__ LineRec ldline(const double2* __restrict__ t, int s) {
  const double2 a = __ldg(t + 2 * s), b = __ldg(t + 2 * s + 1);
  return LineRec{a.x, a.y, b.x, b.y};
}

// Isotropic direction: mu = 2u - 1, phi = 2 pi u', from the 53-bit integers of
// the two uniforms, on the integer pipe (isotropic_fix).
__device__ __forceinline__ void isotropic(const FixTrigTables& T, uint64_t Umu, uint64_t Uphi,
                                          double n[3]) {
  isotropic_fix(T, Umu, Uphi, n);
}

__device__ __forceinline__ double sobolev_beta(double tau) {
  return tau <= 0.0 ? 1.0 : -expm1(-tau) / tau;   // no trapping for tau <= 0
}

// Distance to the next wall along each axis and between walls, from r in cell idx.
// The three reciprocals 1/n_k come from one division, 1/(n_x n_y n_z).
__device__ __forceinline__ void walk_init(const Geometry& g, const int idx[3], const double r[3],
                                          const double n[3], double tm[3], double td[3]) {
  const double d[3] = {g.dx, g.dy, g.dz};
  double inv[3];
  const double pxy = n[0] * n[1], pall = pxy * n[2];
  if (fabs(pall) > 1e-280) {
    const double q = 1.0 / pall;
    inv[0] = q * (n[1] * n[2]); inv[1] = q * (n[0] * n[2]); inv[2] = q * pxy;
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) inv[k] = n[k] != 0.0 ? 1.0 / n[k] : 0.0;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (n[k] > 0.0) {
      tm[k] = fmax(((-g.R + (idx[k] + 1) * d[k]) - r[k]) * inv[k], 0.0);
      td[k] = d[k] * inv[k];
    } else if (n[k] < 0.0) {
      tm[k] = fmax(((-g.R + idx[k] * d[k]) - r[k]) * inv[k], 0.0);
      td[k] = -d[k] * inv[k];
    } else {
      tm[k] = INFINITY;
      td[k] = INFINITY;
    }
  }
}

template <int W>
__device__ __forceinline__ void warp_flush(double (&acc)[W], double* ledger, const int (&slot)[W]) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(ledger + slot[k], v);
  }
}

// Warp-aggregated append of `idx` by the lanes of the current active set that
// have `want`; returns nothing, writes buf[slot].
__device__ __forceinline__ void warp_append(bool want, int idx, int* buf, unsigned long long* n) {
  const unsigned act = __activemask();
  const unsigned m = __ballot_sync(act, want);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(n, (unsigned long long)__popc(m));
  base = __shfl_sync(act, base, leader);
  if (want) buf[base + __popc(m & ((1u << lane) - 1u))] = idx;
}

// Estimator increment with a warp-level pre-reduction by slot: the lanes of the
// current active set that add to the same slot are found with one match, every
// lane of such a group sums its peers' values (in lane order, one shuffle per
// further member of the largest group), and only the lowest lane of each group
// issues the FP64 atomic and logs the slot.  Returns whether this lane did.
// (Opt-in, XT_FLAG_WARP_REDUCE: measured on GB300 it made the trace kernel 1
// to 3 % slower on every workload tried, the collision-heavy one included;
// the hardware's own handling of same-address atomics leaves it nothing to
// gain, and its code costs instruction-cache room.)
__device__ __forceinline__ bool warp_add_slot(double* __restrict__ S, int64_t slot, double v,
                                              bool reduce) {
  if (!reduce) {
    atomicAdd(S + slot, v);
    return true;
  }
  const unsigned act = __activemask();
  const int lane = threadIdx.x & 31;
  const unsigned m = __match_any_sync(act, (unsigned long long)slot);
  const unsigned gmax = __reduce_max_sync(act, (unsigned)__popc(m));
  double sum = v;
  if (gmax > 1) {
    unsigned others = m & ~(1u << lane);
    for (unsigned k = 1; k < gmax; ++k) {
      const int src = others ? __ffs(others) - 1 : lane;
      const double x = __shfl_sync(act, v, src);
      if (others) {
        sum += x;
        others &= others - 1;
      }
    }
  }
  if (lane != __ffs(m) - 1) return false;
  atomicAdd(S + slot, sum);
  return true;
}

// Clear the slots listed in each block's log segment.  Eight slot indices are
// loaded before their stores, so that a thread keeps eight loads in flight
// instead of waiting on each (the kernel is bound by that latency).
__global__ void k_unlog(double* __restrict__ S, const int64_t* __restrict__ log,
                        const int64_t* __restrict__ seg_n, int64_t seg_len) {
  const int64_t n = seg_n[blockIdx.x];
  const int64_t* l = log + (int64_t)blockIdx.x * seg_len;
  const int64_t B = blockDim.x;
  int64_t k = threadIdx.x;
  for (; k + 7 * B < n; k += 8 * B) {
    int64_t a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = __ldcs(l + k + q * B);
#pragma unroll
    for (int q = 0; q < 8; ++q) S[a[q]] = 0.0;
  }
  for (; k < n; k += B) S[l[k]] = 0.0;
}

// ---------------------------------------------------------------- emission
template <class T>
__device__ __forceinline__ void stage(T& dst, const T& src) {
  for (int k = threadIdx.x; k < (int)(sizeof(T) / 8); k += blockDim.x)
    reinterpret_cast<uint64_t*>(&dst)[k] = reinterpret_cast<const uint64_t*>(&src)[k];
}

// One packet of the emission: emitting cell from the integer quota, position,
// direction, comoving and lab frequency, photon number, first resonance cursor
// and the cell-walk state (td carries the sign of the direction).
struct EmitOut {
  int64_t c;
  int idx[3];
  double E0, r[3], n[3], nu_cmf, nu_lab, N, tm[3], td[3];
  int cursor;
};

// Ray r of the RAYS sampler (Sec. 2.3): from the middle of its cell along its
// viewer's centre direction, at its bin's start frequency, with the bin's
// emission times dOmega_k / 4 pi.  E0 = 0 marks an empty ray (the cell has no
// emission in the bin), which is not traced.  The walls are half a cell away.
// The ray id a lane takes at id v of the launch's range, for the spherical
// walk's refill: within every cell's block of nbin x nview ids that the
// launch holds whole, the lanes take the rays of one viewer after another,
// bin by bin, so that a warp's rays share their start point and direction and
// cross the same faces together, and their neighbouring frequencies give them
// line-test loops of similar length; ids in a block the launch holds only in
// part are taken in order.  A bijection of the launch's range onto itself:
// every ray is traced once and keeps its id.  (Bins spread across the band
// instead, 1.7x slower; the same order on the cube, whose cell walk is cheap,
// 1.8x slower than ids in order.)
__device__ __forceinline__ int64_t ray_id_of(const EmitArgs& a, int64_t v) {
  return ray_id_in_range(v, a.p_begin, a.n, a.ray.nbin, a.ray.nview);
}

__device__ __forceinline__ void emit_ray(const EmitArgs& a, int64_t rid, EmitOut& o) {
  const Geometry& g = a.g;
  const RayTables& T = a.ray;
  const int64_t per_cell = T.nbin * T.nview;
  const int64_t ci = rid / per_cell;
  const int64_t rem = rid - ci * per_cell;
  const int64_t jb = rem / T.nview;
  const int k = (int)(rem - jb * T.nview);
  const int64_t c = T.rcell[ci];
  o.c = c;
  {
    const uint32_t c32 = (uint32_t)c, nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
    const uint32_t cy = c32 / nx;
    o.idx[0] = (int)(c32 - cy * nx); o.idx[1] = (int)(cy % ny); o.idx[2] = (int)(cy / ny);
  }
  const double2 v01 = __ldg(reinterpret_cast<const double2*>(T.view) + 2 * k);
  const double2 v23 = __ldg(reinterpret_cast<const double2*>(T.view) + 2 * k + 1);
  const double E_bin = T.Ebin ? T.Ebin[row_of(g, o.idx[0], o.idx[1], o.idx[2]) * T.nbin + jb]
                              : a.Lc[c] * T.bin_frac[jb];
  o.E0 = E_bin * v23.y;
  if (!(o.E0 > 0.0)) return;
  const double d[3] = {g.dx, g.dy, g.dz};
  o.n[0] = v01.x; o.n[1] = v01.y; o.n[2] = v23.x;
#pragma unroll
  for (int q = 0; q < 3; ++q)   // (-R + i d) + d / 2, rounded step by step
    o.r[q] = __dadd_rn(__dadd_rn(-g.R, __dmul_rn((double)o.idx[q], d[q])), 0.5 * d[q]);
  o.nu_cmf = T.bin_nu[jb];
  o.cursor = T.bin_cursor[jb];
  const double* n = o.n;
  const double* r = o.r;
  o.nu_lab = div_pos(o.nu_cmf, 1.0 - (n[0] * r[0] + n[1] * r[1] + n[2] * r[2]) * g.inv_ct);
  o.N = div_pos(o.E0, kH * o.nu_cmf);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const long long nb = __double_as_longlong(n[q]);
    if ((nb << 1) != 0) {
      const double t = div_pos(d[q], __longlong_as_double(nb & 0x7FFFFFFFFFFFFFFFll));
      o.tm[q] = 0.5 * t;
      o.td[q] = nb > 0 ? t : neg_bits(t);
    } else {
      o.tm[q] = INFINITY;
      o.td[q] = INFINITY;
    }
  }
}

// The emitting cell of packet p: the last c with qoff[c] <= p.
__device__ __forceinline__ int64_t quota_cell(const EmitArgs& a, int64_t p) {
  int64_t lo = 0, hi = a.g.ncell;
  if (a.qguide) {                         // qoff[lo] <= p < qoff[hi]
    const int64_t j = p >> kQGuideShift;
    lo = a.qguide[j];
    hi = (int64_t)a.qguide[j + 1] + 1;
  }
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (a.qoff[mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

// Comoving frequency and first line to test of a packet of cell c (natural
// index, cell indices idx) from its uniform draw xv1: flat in nu over the
// band, or a line picked by its share of the cell's line emission (the packet
// then starts past that line).
__device__ __forceinline__ void emit_frequency(const EmitArgs& a, uint64_t xv1, int64_t c, const int idx[3],
                                               double& nu_cmf, int& cursor) {
  const double v1 = u01(xv1);
  if (a.emission == XT_EMIT_BAND) {
    nu_cmf = fma(v1, a.nu_span, a.nu_lo);   // the guide's edges use the same fma
    int l0 = 0, l1 = a.nline;             // first sorted line with nu <= nu_cmf
    if (a.nuguide) {                      // nu_cmf lies between its bucket's edges
      const int j = (int)((xv1 >> 11) >> kNuGuideShift);
      l0 = a.nuguide[j + 1];
      l1 = a.nuguide[j];
    }
    const long long nb = bits(nu_cmf);
    while (l0 < l1) {
      const int mid = (l0 + l1) >> 1;
      if (bits(a.nu_tab[mid]) <= nb) l1 = mid; else l0 = mid + 1;
    }
    cursor = l0;
  } else {
    const double* cdf = a.cdf + row_of(a.g, idx[0], idx[1], idx[2]) * a.nline;
    const double x = v1 * a.Lc[c];
    int l0 = 0, l1 = a.nline;             // first caller line with x < cdf
    while (l0 < l1) {
      const int mid = (l0 + l1) >> 1;
      if (x < cdf[mid]) l1 = mid; else l0 = mid + 1;
    }
    const int s = a.sorted_of[l0 < a.nline ? l0 : a.nline - 1];
    nu_cmf = a.nu_tab[s];
    cursor = s + 1;
  }
}

__device__ __forceinline__ void emit_packet(const EmitArgs& a, const FixTrigTables& trig, int64_t p,
                                            EmitOut& o) {
  const Geometry& g = a.g;
  const int64_t c = quota_cell(a, p);
  o.c = c;
  {                                       // cell indices in 32-bit arithmetic (ncell < 2^30)
    const uint32_t c32 = (uint32_t)c, nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
    const uint32_t cy = c32 / nx;
    o.idx[0] = (int)(c32 - cy * nx); o.idx[1] = (int)(cy % ny); o.idx[2] = (int)(cy / ny);
  }
  const double d[3] = {g.dx, g.dy, g.dz};
  o.E0 = a.Epk[c];
  uint64_t xu[4], xv[4];
  draw_raw(a.seed, p, 0, xu);
  draw_raw(a.seed, p, 1, xv);
  double uu[3];
  const int woff[3] = {0, g.nx, g.nx + g.ny};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uu[k] = u01(xu[k]);
    const double w0 = a.wall ? a.wall[woff[k] + o.idx[k]] : fma((double)o.idx[k], d[k], -g.R);
    o.r[k] = w0 + uu[k] * d[k];
  }
  isotropic(trig, xu[3] >> 11, xv[0] >> 11, o.n);
  emit_frequency(a, xv[1], c, o.idx, o.nu_cmf, o.cursor);
  const double* n = o.n;
  const double* r = o.r;
  // the quotients on the integer pipe (div_pos, within 0.51 ulp): GB300's FP64
  // pipe is the scarce one, and it would spend about as much on these three
  // divisions as on the rest of the emission
  o.nu_lab = div_pos(o.nu_cmf, 1.0 - (n[0] * r[0] + n[1] * r[1] + n[2] * r[2]) * g.inv_ct);
  o.N = div_pos(a.Eph[c], o.nu_cmf);                // E0 / (h nu_cmf)
  // cell walk from the position inside the cell: walls d / |n_k| apart, the
  // nearest one (1 - u) d / |n_k| ahead for n_k > 0 and u d / |n_k| for n_k < 0;
  // td carries the sign of n_k (sign and zero tests on the bit patterns)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const long long nb = bits(n[k]);
    if ((nb << 1) != 0) {
      const double t = div_pos(d[k], __longlong_as_double(nb & 0x7FFFFFFFFFFFFFFFll));
      const uint64_t U = xu[k] >> 11;                // uu[k] = U 2^-53, 1 - uu[k] exact below
      o.tm[k] = (nb > 0 ? q63_to_double((1ull << 53) - U, 10) : uu[k]) * t;
      o.td[k] = nb > 0 ? t : neg_bits(t);
    } else {
      o.tm[k] = INFINITY;
      o.td[k] = INFINITY;
    }
  }
}

// qguide[j] = the cell of packet j 2^6: the last c with qoff[c] <= j 2^6.
__global__ void k_q_guide(const int64_t* __restrict__ qoff, int64_t ncell, int64_t nj,
                          int* __restrict__ out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nj) return;
  const int64_t x = j << kQGuideShift;
  int64_t lo = 0, hi = ncell;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (qoff[mid] <= x) lo = mid; else hi = mid;
  }
  out[j] = (int)lo;
}

// nuguide[j] = first sorted line with nu <= fma(j 2^-16, span, nu_lo), the
// lower edge of bucket j of the band emission's uniform (j = 0..2^16).
__global__ void k_nu_guide(const double* __restrict__ nu, int nline, double nu_lo, double nu_span,
                           int* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kNuGuideN) return;
  const double v = (double)((uint64_t)j << kNuGuideShift) * 0x1p-53;   // exact
  const long long eb = bits(fma(v, nu_span, nu_lo));
  int l0 = 0, l1 = nline;
  while (l0 < l1) {
    const int mid = (l0 + l1) >> 1;
    if (bits(nu[mid]) <= eb) l1 = mid; else l0 = mid + 1;
  }
  out[j] = l0;
}

__global__ void __launch_bounds__(256) k_emit(const EmitArgs a) {
  __shared__ FixTrigTables trig;
  stage(trig, a.trig);
  __syncthreads();
  double acc[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = a.p_begin + i;
    EmitOut o;
    emit_packet(a, trig, p, o);
    const Pool& P = a.pool;
    P.F(F_R0X, i) = o.r[0]; P.F(F_R0Y, i) = o.r[1]; P.F(F_R0Z, i) = o.r[2];
    P.F(F_NX, i) = o.n[0]; P.F(F_NY, i) = o.n[1]; P.F(F_NZ, i) = o.n[2];
    P.F(F_TMX, i) = o.tm[0]; P.F(F_TMY, i) = o.tm[1]; P.F(F_TMZ, i) = o.tm[2];
    P.F(F_TDX, i) = o.td[0]; P.F(F_TDY, i) = o.td[1]; P.F(F_TDZ, i) = o.td[2];
    // stop once N nu_line < e_cut E0 / h (the photon energy at the line below e_cut E0)
    P.F(F_NULAB, i) = o.nu_lab; P.F(F_NU0, i) = o.nu_cmf; P.F(F_N, i) = o.N;
    P.F(F_T, i) = a.e_cut * a.Eph[o.c];
    P.F(F_SPI, i) = 0.0;
    P.cell[i] = o.idx[0] | (o.idx[1] << 10) | (o.idx[2] << 20);
    P.cursor[i] = o.cursor; P.events[i] = 0; P.ndraw[i] = 0; P.inter[i] = 0;
    P.pid[i] = p;
    acc[0] += o.N;
    acc[1] += o.E0;
    if (a.records) {
      double* rec = a.records + (p - a.rec_base) * XT_PKT_FIELDS;
      rec[7] = (double)o.c; rec[8] = o.N; rec[9] = o.nu_cmf;
    }
  }
  const int slots[2] = {LG_EMIT_N, LG_EMIT_E};
  warp_flush(acc, a.ledger, slots);
}

// ---------------------------------------------------------------- photoionization
// Photoionization on one path segment (Sec. 2.3.1), s0..s1 along the ray (s
// from the emission point, comoving frequency nu0 - aslope s).  Every level
// whose threshold lies below the photon energy at the segment start takes
// part over the whole length d = s1 - s0, or up to where the falling comoving
// frequency reaches its threshold; sigma_k = sig_k lambda^3 with the
// wavelength at the segment start (Eq. sigma_OTSPI).  So
//   tau = lambda^3 (d kappa[b] + sum_{crossed k} sig_k n_k d_k),
// kappa[b] the cell's suffix sum of sig n over the levels that keep the whole
// length (sorted positions >= b).  The packet loses N (1 - e^-tau); level k's
// share N_abs tau_k / tau is X sig_k n_k d_k with X = N beta(tau) lambda^3,
// beta = (1 - e^-tau) / tau, so the cell keeps X d at G[b] and X d_k at D[k]
// for the crossed levels (one atomic for the common part), and N_abs nu for
// the heating.  pcur is the first level still active at s0 and moves past the
// crossed ones.  Returns whether the photon energy at s1 fell below the cut.
__device__ __forceinline__ bool pi_segment(const TraceArgs& a, const FixExpTables& fx,
                                           const double* s_nuth, const double* s_sig, const int* s_lev,
                                           int row, const double* prow, double s0, double s1,
                                           double nu0, double aslope, double inv_as, int& pcur,
                                           double& N, double& N_pi, double& E_pi, double Tq) {
  double d = s1 - s0;
  if (bits(d) <= 0) d = 0.0;                        // (rounding can put s1 just before s0)
  const double nu_a = fma(-aslope, s0, nu0);
  const double nu_b = fma(-aslope, bits(d) > 0 ? s1 : s0, nu0);
  int kb = pcur;
  double tc = 0.0;
  while (kb < a.npi && s_nuth[kb] >= nu_b) {        // thresholds crossed inside the segment
    tc = fma(s_sig[kb] * prow[s_lev[kb]], (nu_a - s_nuth[kb]) * inv_as, tc);
    ++kb;
  }
  const int64_t rb = (int64_t)row * (a.npi + 1);
  const double lam = div_pos(kC, nu_a);
  const double l3 = lam * lam * lam;
  const double tau = l3 * fma(a.kappa[rb + kb], d, tc);
  if (bits(tau) > 0) {
    double ex, ome, beta;
    if (bits(tau) < bits(0x1p-10)) {                // series: keeps 1 - e^-tau exact for tiny tau
      beta = sobolev_beta_fix(fx, tau, nullptr);
      ome = tau * beta;
      ex = 1.0 - ome;
    } else {
      expneg(fx, tau, ex, ome);
      beta = div_pos(ome, tau);
    }
    const double X = N * beta * l3;
    if (kb < a.npi && bits(d) > 0) atomicAdd(a.piG + rb + kb, X * d);
    for (int k = pcur; k < kb; ++k)
      atomicAdd(a.piD + (int64_t)row * a.npi + k, X * ((nu_a - s_nuth[k]) * inv_as));
    const double Nabs = N * ome;
    N_pi += Nabs;
    E_pi += Nabs * nu_a;
    atomicAdd(a.piH + row, Nabs * nu_a);
    N = N * ex;
  }
  pcur = kb;
  return bits(N * nu_b) < bits(Tq);
}

// ---------------------------------------------------------------- trace
// Per-lane ledger: integer counters, FP64 sums.
enum { T_ABS, T_DROP, T_ABSE, T_REEM, T_THERM, T_EMITN, T_EMITE, T_NACC, T_PIN = T_NACC, T_PIE };
constexpr int kMaxSteps = 4;      // walls crossed per search before the lane yields
constexpr int kRefillLanes = 24;  // empty lanes of a warp that trigger a refill with emission
// Rays on the spherical grid: a warp is refilled only once all its lanes are
// empty, so that it keeps walking one cell's and viewer's rays together
// (ray_id_of)
constexpr int kRayRefillLanes = 32;
constexpr int kLogSegments = 4096; // touched-slot log segments (>= trace blocks per launch)

template <int MODE, bool PI = false, bool RAYS = false, bool WR = false>
__global__ void __launch_bounds__(256, (MODE == XT_MODE_ATTEN && !PI) ? 4 : 2) k_trace(const TraceArgs a) {
  __shared__ FixExpTables fx;
  __shared__ FixTrigTables trig;
  __shared__ int rtab[3 * 1024];
  constexpr int kPiS = PI ? XT_PI_MAX : 1;          // photoionization tables (PI instance)
  __shared__ double s_nuth[kPiS], s_sig[kPiS];
  __shared__ int s_lev[kPiS];
  stage(fx, a.fx);
  if (MODE == XT_MODE_SCATTER || a.fused) stage(trig, a.trig);
  const int nt = a.g.nx + a.g.ny + a.g.nz;
  for (int k = threadIdx.x; k < nt; k += blockDim.x) rtab[k] = a.rtab[k];
  if constexpr (PI) {
    for (int k = threadIdx.x; k < a.npi; k += blockDim.x) {
      s_nuth[k] = a.pi_nuth[k]; s_sig[k] = a.pi_sig[k]; s_lev[k] = a.pi_lev[k];
    }
  }
  __syncthreads();
  const int* RX = rtab;
  const int* RY = rtab + a.g.nx;
  const int* RZ = rtab + a.g.nx + a.g.ny;
  __shared__ unsigned long long blk_log;          // entries in this block's log segment
  if (threadIdx.x == 0) blk_log = (unsigned long long)a.seg_n[blockIdx.x];
  __syncthreads();
  int64_t* const my_log = a.slotlog + (int64_t)blockIdx.x * a.seg_len;
  const Geometry& g = a.g;
  const Pool& P = a.pool;
  const int lane = threadIdx.x & 31;
  const long long taumin_bits = __double_as_longlong(a.tau_min);
  constexpr int kAcc = PI ? T_PIE + 1 : T_NACC;
  double acc[kAcc];
#pragma unroll
  for (int k = 0; k < kAcc; ++k) acc[k] = 0.0;
  unsigned n_tests = 0, n_events = 0, n_guard = 0, n_inter = 0;

  bool have = false, seg_new = true;
  int i = 0;                             // pool slot
  int ix = 0, iy = 0, iz = 0, sx = 1, sy = 1, sz = 1, cursor = 0, events = 0, axis = 0;
  int rx = 0, ry = 0, rz = 0;            // row = rx + ry + rz (separable blocked layout)
  int box_lo = 0, box_hi = 0;            // current subdomain box, packed like the cell
  int row = 0;
  long long end_bits = 0;
  double tmx = 0, tmy = 0, tmz = 0, tdx = 0, tdy = 0, tdz = 0, nu0 = 0, aslope = 0;
  double N = 0, N_in = 0, Tq = 0;
  // photoionization state (PI instance): segment start, 1 / aslope, the
  // packet's photoionized photons, first level still active, the wall ahead
  double s_pi = 0, inv_as = 0, N_pi = 0, s_wall = 0;
  int pcur = 0;

  bool drained = false;                  // the packet list is used up (warp-uniform)
  for (;;) {
    // ---- refill lanes whose packet ended (warp-aggregated).  The loop runs
    // warp-synchronously: with emission in the refill (FP64-heavy) the empty
    // lanes are refilled together, once at least kRefillLanes are empty, so
    // the emission runs with most lanes; busy lanes trace on meanwhile.
    __syncwarp();
    {
      const unsigned act = 0xffffffffu;
      const unsigned m0 = __ballot_sync(act, !have);
      if (m0 == act && drained) break;
      const unsigned m = (drained || (a.fused && m0 != act && __popc(m0) < kRefillLanes)) ? 0u : m0;
      if (m) {
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(a.counter, (unsigned long long)__popc(m));
        base = __shfl_sync(act, base, leader);
        if (base + __popc(m) >= (unsigned long long)a.n_list) drained = true;
        if (!have) {
          const unsigned long long my = base + __popc(m & ((1u << lane) - 1u));
          if (my < (unsigned long long)a.n_list && MODE == XT_MODE_ATTEN && a.fused) {
            // emit the packet here: its state goes to registers; the pool keeps
            // what the escape tallies read (direction, lab frequency, id)
            i = (int)my;
            const int64_t p = a.em.p_begin + (int64_t)my;
            EmitOut o;
            if constexpr (RAYS) emit_ray(a.em, p, o);
            else emit_packet(a.em, trig, p, o);
            if (RAYS && !(o.E0 > 0.0)) {           // an empty ray: recorded, not traced
              if (a.records) {
                double* rec = a.records + (p - a.rec_base) * XT_PKT_FIELDS;
                rec[0] = 4.0; rec[1] = 0.0; rec[2] = 0.0; rec[3] = 0.0; rec[4] = -1.0; rec[5] = -1.0;
                rec[6] = 0.0; rec[7] = (double)o.c; rec[8] = 0.0; rec[9] = 0.0; rec[10] = 0.0;
              }
              continue;
            }
            ix = o.idx[0]; iy = o.idx[1]; iz = o.idx[2];
            tmx = o.tm[0]; tmy = o.tm[1]; tmz = o.tm[2];
            sx = bits(o.td[0]) < 0 ? -1 : 1; sy = bits(o.td[1]) < 0 ? -1 : 1; sz = bits(o.td[2]) < 0 ? -1 : 1;
            tdx = dabs_bits(o.td[0]); tdy = dabs_bits(o.td[1]); tdz = dabs_bits(o.td[2]);
            nu0 = o.nu_cmf;
            aslope = o.nu_lab * a.inv_ct;
            N = o.N;
            N_in = N;
            if constexpr (RAYS) Tq = (a.em.e_cut * o.E0) * (1.0 / kH);
            else Tq = a.em.e_cut * a.em.Eph[o.c];
            cursor = o.cursor;
            events = 0;
            if constexpr (PI) {
              s_pi = 0.0;
              N_pi = 0.0;
              inv_as = div_pos(a.ct, o.nu_lab);
              pcur = 0;
              while (pcur < a.npi && s_nuth[pcur] >= nu0) ++pcur;
            }
            P.F(F_NX, i) = o.n[0]; P.F(F_NY, i) = o.n[1]; P.F(F_NZ, i) = o.n[2];
            P.F(F_NULAB, i) = o.nu_lab;
            P.pid[i] = p;
            acc[T_EMITN] += o.N;
            acc[T_EMITE] += o.E0;
            if (a.records) {
              P.inter[i] = 0;
              double* rec = a.records + (p - a.rec_base) * XT_PKT_FIELDS;
              rec[7] = (double)o.c; rec[8] = o.N; rec[9] = o.nu_cmf;
            }
            rx = RX[ix]; ry = RY[iy]; rz = RZ[iz];
            row = rx + ry + rz;
            seg_new = true;
            have = true;
          } else if (my < (unsigned long long)a.n_list) {
            i = a.list ? a.list[my] : (int)my;
            const int cs = P.cell[i];
            ix = cs & 1023; iy = (cs >> 10) & 1023; iz = cs >> 20;
            tmx = P.F(F_TMX, i); tmy = P.F(F_TMY, i); tmz = P.F(F_TMZ, i);
            tdx = P.F(F_TDX, i); tdy = P.F(F_TDY, i); tdz = P.F(F_TDZ, i);
            sx = bits(tdx) < 0 ? -1 : 1; sy = bits(tdy) < 0 ? -1 : 1; sz = bits(tdz) < 0 ? -1 : 1;
            tdx = dabs_bits(tdx); tdy = dabs_bits(tdy); tdz = dabs_bits(tdz);
            nu0 = P.F(F_NU0, i);
            aslope = P.F(F_NULAB, i) * a.inv_ct;
            N = P.F(F_N, i);
            N_in = N;
            Tq = P.F(F_T, i);
            cursor = P.cursor[i];
            events = P.events[i];
            if constexpr (PI) {
              s_pi = P.F(F_SPI, i);
              N_pi = 0.0;
              inv_as = div_pos(a.ct, P.F(F_NULAB, i));
              const double nu_s = fma(-aslope, s_pi, nu0);
              pcur = 0;
              while (pcur < a.npi && s_nuth[pcur] >= nu_s) ++pcur;
            }
            rx = RX[ix]; ry = RY[iy]; rz = RZ[iz];
            row = rx + ry + rz;
            if (a.rounds == 3) {          // a process's domain: whole x-y layers
              box_lo = a.dom_zlo << 20;
              box_hi = (g.nx - 1) | ((g.ny - 1) << 10) | ((a.dom_zhi - 1) << 20);
            } else if (a.rounds == 2) {   // a streamed group: whole x-y layers of z cells
              const int z0 = (iz / a.grp_nz) * a.grp_nz;
              box_lo = z0 << 20;
              box_hi = (g.nx - 1) | ((g.ny - 1) << 10) | ((z0 + a.grp_nz - 1) << 20);
            } else if (a.rounds) {        // the packet's subdomain (bounds inclusive)
              const int x0 = (ix / g.bx) * g.bx, y0 = (iy / g.by) * g.by, z0 = (iz / g.bz) * g.bz;
              box_lo = x0 | (y0 << 10) | (z0 << 20);
              box_hi = (x0 + g.bx - 1) | ((y0 + g.by - 1) << 10) | ((z0 + g.bz - 1) << 20);
            }
            seg_new = true;
            have = true;
          }
        }
      }
    }
    if (!have) continue;

    // ---- search: test lines and walk cells until an interaction point is met,
    // the packet leaves the grid or its subdomain, or kMaxSteps walls are crossed
    // (so that no lane keeps its warp waiting long); the event code below then
    // runs for all lanes that found one together.
    const double* prow = a.pops + (int64_t)row * a.nlev;
    bool found = false, escaped = false, queued = false, pi_drop = false;
    LineRec L;
    double n_l = 0.0, n_u = 0.0, tau = 0.0;
    // the record of the next line to test is loaded one test ahead, so that its
    // fetch overlaps the population loads of the current one
    LineRec Ln{0.0, 0.0, 0.0, 0.0};
    if (cursor < a.nline) Ln = ldline(a.lines, cursor);
    long long next_bits = cursor < a.nline ? bits(Ln.x) : 0;
    for (int steps = 0;;) {
      if (seg_new) {       // nearest wall and the comoving frequency there
        double sw = tmx;
        axis = 0;
        if (bits(tmy) < bits(sw)) { sw = tmy; axis = 1; }   // ties to the lowest axis
        if (bits(tmz) < bits(sw)) { sw = tmz; axis = 2; }
        end_bits = bits(nu0 - aslope * sw);
        if constexpr (PI) s_wall = sw;
        seg_new = false;
      }
      while (cursor < a.nline && next_bits > end_bits) {
        L = Ln;
        ++n_tests;
        n_l = prow[__double2loint(L.w)];
        n_u = prow[__double2hiint(L.w)];
        const int cn = cursor + 1;
        if (cn < a.nline) Ln = ldline(a.lines, cn);
        tau = L.y * (n_l - L.z * n_u);
        if (bits(tau) > taumin_bits) { found = true; break; }
        cursor = cn;
        next_bits = cn < a.nline ? bits(Ln.x) : 0;
      }
      if (found) break;
      if constexpr (PI) {      // photoionization up to the wall (Sec. 2.3.1)
        if (pi_segment(a, fx, s_nuth, s_sig, s_lev, row, prow, s_pi, s_wall, nu0, aslope, inv_as, pcur,
                       N, N_pi, acc[T_PIE], Tq)) {
          pi_drop = true;
          break;
        }
        if (bits(s_wall) > bits(s_pi)) s_pi = s_wall;
      }
      // no further line in this cell: step into the next one (branch-free in axis)
      const bool a0 = axis == 0, a1 = axis == 1, a2 = axis == 2;
      const int coord = (a0 ? ix : a1 ? iy : iz) + (a0 ? sx : a1 ? sy : sz);
      const double tnew = (a0 ? tmx : a1 ? tmy : tmz) + (a0 ? tdx : a1 ? tdy : tdz);
      ix = a0 ? coord : ix; iy = a1 ? coord : iy; iz = a2 ? coord : iz;
      tmx = a0 ? tnew : tmx; tmy = a1 ? tnew : tmy; tmz = a2 ? tnew : tmz;
      seg_new = true;
      if (coord < 0 || coord >= (a0 ? g.nx : a1 ? g.ny : g.nz)) { escaped = true; break; }
      const int rnew = rtab[(a0 ? 0 : a1 ? g.nx : g.nx + g.ny) + coord];
      rx = a0 ? rnew : rx; ry = a1 ? rnew : ry; rz = a2 ? rnew : rz;
      row = rx + ry + rz;
      prow = a.pops + (int64_t)row * a.nlev;
      if (a.rounds && (ix < (box_lo & 1023) || ix > (box_hi & 1023) ||
                       iy < ((box_lo >> 10) & 1023) || iy > ((box_hi >> 10) & 1023) ||
                       iz < (box_lo >> 20) || iz > (box_hi >> 20))) {
        queued = true;
        break;
      }
      if (++steps >= kMaxSteps) break;
    }
    int fate = -1;                        // -1 alive
    if constexpr (PI) {
      if (found) {             // the ray moves to the resonance point, photoionizing on the way
        const double s_l = (nu0 - L.x) * inv_as;
        if (pi_segment(a, fx, s_nuth, s_sig, s_lev, row, prow, s_pi, s_l, nu0, aslope, inv_as, pcur,
                       N, N_pi, acc[T_PIE], Tq)) {
          pi_drop = true;
          found = false;
        }
        if (bits(s_l) > bits(s_pi)) s_pi = s_l;
      }
      if (pi_drop) { acc[T_DROP] += N; fate = 1; }
    }
    if (found) {
      // ---- line event (lanes that found one run this together)
      ++events;
      ++n_events;
      double ex, ome;
      expneg(fx, tau, ex, ome);
      if (MODE == XT_MODE_ATTEN) {
        // net photons (divided by f_corr at readout), pre-reduced over the lanes
        // of the warp that hit the same slot; the adding lane logs the slot
        const int64_t slot = (a.crow ? (int64_t)a.crow[row] : (int64_t)(row - a.row0)) * a.nline + cursor;
        if (warp_add_slot(a.S, slot, N * ome, WR)) {
          const unsigned long long k = atomicAdd(&blk_log, 1ull);
          if (k < (unsigned long long)a.seg_len) my_log[k] = slot;
        }
        N = N * ex;
        if (bits(N * L.x) < bits(Tq)) { acc[T_DROP] += N; fate = 1; }
        ++cursor;
      } else {
        const int64_t p = P.pid[i];
        const int nd = P.ndraw[i];
        P.ndraw[i] = nd + 1;
        uint64_t xw[4];
        draw_raw(a.seed, p, 2 + (uint64_t)nd, xw);
        const U4 w{{u01(xw[0]), u01(xw[1]), u01(xw[2]), u01(xw[3])}};
        const int64_t slot = (a.crow ? (int64_t)a.crow[row] : (int64_t)(row - a.row0)) * a.nline + cursor;
        {   // every event's slot is logged (interaction or not), as before the draw
          const unsigned long long k = atomicAdd(&blk_log, 1ull);
          if (k < (unsigned long long)a.seg_len) my_log[k] = slot;
        }
        if (w.u[0] < ome) {
          P.inter[i] += 1;
          ++n_inter;
          warp_add_slot(a.S, slot, N, WR);
          acc[T_ABS] += N;                    // the whole packet is absorbed
          const double Ecmf = N * kH * L.x;
          acc[T_ABSE] += Ecmf;
          const int up = __double2hiint(L.w);
          const int k0 = a.down_off[up], k1 = a.down_off[up + 1];
          double Wtot = 8.629e-6 * a.ne[row] * a.ups_down[up] / (a.glev[up] * sqrt(a.Te[row]));
          for (int k = k0; k < k1; ++k) {
            const int m = a.down_line[k];
            const LineRec M = ldline(a.lines, m);
            Wtot += a.A[m] * sobolev_beta_fix(fx, M.y * (prow[__double2loint(M.w)] - M.z * n_u), nullptr);
          }
          const double x = w.u[1] * Wtot;
          double run = 0.0;
          int pick = -1;
          for (int k = k0; k < k1; ++k) {
            const int m = a.down_line[k];
            const LineRec M = ldline(a.lines, m);
            run += a.A[m] * sobolev_beta_fix(fx, M.y * (prow[__double2loint(M.w)] - M.z * n_u), nullptr);
            if (x < run) { pick = m; break; }
          }
          if (pick < 0) {
            acc[T_THERM] += Ecmf;
            fate = 2;
          } else {
            // move to the resonance point, re-emit isotropically in line `pick`
            double r[3] = {P.F(F_R0X, i), P.F(F_R0Y, i), P.F(F_R0Z, i)};
            double n[3] = {P.F(F_NX, i), P.F(F_NY, i), P.F(F_NZ, i)};
            const double nu_lab = P.F(F_NULAB, i);
            const double s_l = a.ct * (1.0 - L.x / nu_lab) - (n[0] * r[0] + n[1] * r[1] + n[2] * r[2]);
#pragma unroll
            for (int k = 0; k < 3; ++k) r[k] = r[k] + s_l * n[k];
            isotropic(trig, xw[2] >> 11, xw[3] >> 11, n);
            const double nu_new = ldline(a.lines, pick).x;
            N = Ecmf / (kH * nu_new);
            N_in = N;
            acc[T_REEM] += Ecmf;
            const double nl_new = nu_new / (1.0 - (n[0] * r[0] + n[1] * r[1] + n[2] * r[2]) * a.inv_ct);
            const int idx[3] = {ix, iy, iz};
            double tm[3], td[3];
            walk_init(g, idx, r, n, tm, td);
            tmx = tm[0]; tmy = tm[1]; tmz = tm[2]; tdx = td[0]; tdy = td[1]; tdz = td[2];   // |d / n|
            sx = n[0] > 0.0 ? 1 : -1; sy = n[1] > 0.0 ? 1 : -1; sz = n[2] > 0.0 ? 1 : -1;
            P.F(F_R0X, i) = r[0]; P.F(F_R0Y, i) = r[1]; P.F(F_R0Z, i) = r[2];
            P.F(F_NX, i) = n[0]; P.F(F_NY, i) = n[1]; P.F(F_NZ, i) = n[2];
            P.F(F_NULAB, i) = nl_new;
            nu0 = nu_new;
            aslope = nl_new * a.inv_ct;
            cursor = pick + 1;
            seg_new = true;
          }
        } else {
          ++cursor;
        }
      }
      if (fate < 0 && events >= a.max_events) { ++n_guard; fate = 3; }
    }
    // ---- packet leaves this lane: escaped, finished, or handed to another subdomain
    if (escaped || queued || fate >= 0) {
      P.F(F_N, i) = N;
      P.events[i] = events;
      if (MODE == XT_MODE_ATTEN) {
        if constexpr (PI) {
          acc[T_ABS] += (N_in - N) - N_pi;               // photons the lines absorbed
          acc[T_PIN] += N_pi;
        } else {
          acc[T_ABS] += N_in - N;                        // photons this lane absorbed
        }
      }
      if (queued || (MODE == XT_MODE_SCATTER && escaped)) {
        P.F(F_TMX, i) = tmx; P.F(F_TMY, i) = tmy; P.F(F_TMZ, i) = tmz;
        P.F(F_TDX, i) = sx < 0 ? neg_bits(tdx) : tdx;
        P.F(F_TDY, i) = sy < 0 ? neg_bits(tdy) : tdy;
        P.F(F_TDZ, i) = sz < 0 ? neg_bits(tdz) : tdz;
        P.F(F_NU0, i) = nu0;
        P.cursor[i] = cursor;
        P.cell[i] = ix | (iy << 10) | (iz << 20);
        if constexpr (PI) P.F(F_SPI, i) = s_pi;
      }
      if (fate >= 0 && a.records) {
        double* rec = a.records + (P.pid[i] - a.rec_base) * XT_PKT_FIELDS;
        rec[0] = fate; rec[1] = events; rec[2] = N; rec[3] = 0.0; rec[4] = -1.0; rec[5] = -1.0;
        rec[6] = P.inter[i]; rec[10] = P.F(F_NULAB, i);
      }
      have = false;
    }
    warp_append(escaped, i, a.esc, a.n_esc);
    warp_append(queued, i, a.out, a.n_out);
  }
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long nb = blk_log;
    if (nb > (unsigned long long)a.seg_len) atomicAdd(a.log_overflow, 1ull);
    a.seg_n[blockIdx.x] = (int64_t)(nb < (unsigned long long)a.seg_len ? nb : a.seg_len);
  }
  double cnt[4] = {(double)n_tests, (double)n_events, (double)n_guard, (double)n_inter};
  const int cslots[4] = {LG_TESTS, LG_EVENTS, LG_GUARD, LG_INTERACT};
  warp_flush(cnt, a.ledger, cslots);
  const int all_slots[T_PIE + 1] = {LG_ABS_N, LG_DROP_N, LG_ABS_E_CMF, LG_REEMIT_E_CMF, LG_THERMAL_E,
                                    LG_EMIT_N, LG_EMIT_E, LG_PI_N, LG_PI_E};
  int slots[kAcc];
#pragma unroll
  for (int k = 0; k < kAcc; ++k) slots[k] = all_slots[k];
  warp_flush(acc, a.ledger, slots);
}

// ---------------------------------------------------------------- staged rays
// The RAYS sampler with the line list staged in shared memory.  The rays of
// one (cell, bin) group start in the same cell at the same comoving frequency
// nu_j and only ever test lines below it, down to where the largest Doppler
// drift across the grid can take them; that frequency window of the sorted
// line records is copied into shared memory by the bulk-copy engine
// (cp.async.bulk, completion on an mbarrier) once per group, and every ray of
// the group reads its line records from there (beyond the window, from global
// memory).  A CTA takes a batch of rays of consecutive bins of one cell at a
// time (their windows overlap); a thread traces a ray to its end.  Attenuation
// mode, no photoionization; the event logic is k_trace's.  Opt-in
// (XT_FLAG_RAYS_STAGED): with the line list resident in L2 the plain trace
// kernel measured faster.
constexpr int kStageLines = 1536;              // window capacity: 48 KB of 32-byte records
constexpr int kStageRays = 512;                // rays per batch (consecutive bins of one cell)
constexpr long long kStageSpin = 1ll << 26;    // bound of the wait for a window

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__global__ void __launch_bounds__(256, 3) k_trace_rays_staged(const TraceArgs a, const int* __restrict__ win_len,
                                                             int64_t p_end, unsigned long long* __restrict__ err) {
  extern __shared__ __align__(128) double2 s_lines[];      // kStageLines x 2 double2
  __shared__ FixExpTables fx;
  __shared__ int rtab[3 * 1024];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ unsigned long long blk_log;
  __shared__ int s_abort, s_next;
  stage(fx, a.fx);
  const int nt = a.g.nx + a.g.ny + a.g.nz;
  for (int k = threadIdx.x; k < nt; k += blockDim.x) rtab[k] = a.rtab[k];
  if (threadIdx.x == 0) {
    blk_log = (unsigned long long)a.seg_n[blockIdx.x];
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
  }
  __syncthreads();
  const int* RX = rtab;
  const int* RY = rtab + a.g.nx;
  const int* RZ = rtab + a.g.nx + a.g.ny;
  int64_t* const my_log = a.slotlog + (int64_t)blockIdx.x * a.seg_len;
  const Geometry& g = a.g;
  const Pool& P = a.pool;
  const RayTables& T = a.em.ray;
  const long long taumin_bits = __double_as_longlong(a.tau_min);
  double acc[T_NACC];
#pragma unroll
  for (int k = 0; k < T_NACC; ++k) acc[k] = 0.0;
  unsigned n_tests = 0, n_events = 0, n_guard = 0;
  // a batch: up to kStageRays rays of consecutive bins of one cell, whose
  // windows overlap (the bins' start frequencies fall with the bin index)
  const int64_t rays_per_group = T.nview;
  const int64_t gpb = max((int64_t)1, (int64_t)kStageRays / rays_per_group);   // groups per batch
  const int64_t bpc = (T.nbin + gpb - 1) / gpb;                                 // batches per cell
  const int64_t p_begin = a.em.p_begin;
  const int64_t c_first = p_begin / (rays_per_group * T.nbin);
  const int64_t c_last = (p_end + rays_per_group * T.nbin - 1) / (rays_per_group * T.nbin);
  uint32_t phase = 0;
  for (int64_t bt = c_first * bpc + blockIdx.x; bt < c_last * bpc; bt += gridDim.x) {
    const int64_t ci = bt / bpc, j0 = (bt - ci * bpc) * gpb, j1 = min(j0 + gpb, T.nbin);
    const int64_t r0 = max(p_begin, (ci * T.nbin + j0) * rays_per_group);
    const int64_t r1 = min(p_end, (ci * T.nbin + j1) * rays_per_group);
    if (r1 <= r0) continue;                          // (uniform over the CTA)
    const int base = T.bin_cursor[j0];
    int hi = base;
    for (int64_t j = j0; j < j1; ++j) hi = max(hi, T.bin_cursor[j] + win_len[j]);
    const int wl = min(hi - base, kStageLines);
    __syncthreads();                                   // the previous window is no longer read
    if (threadIdx.x == 0) s_next = 0;
    if (threadIdx.x == 0 && wl > 0) {
      const uint32_t bytes = (uint32_t)wl * 32u;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   ::"r"(smem_addr(&bar)), "r"(bytes) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   ::"r"(smem_addr(s_lines)), "l"(a.lines + 2 * (int64_t)base), "r"(bytes), "r"(smem_addr(&bar))
                   : "memory");
    }
    if (wl > 0) {
      // every thread waits for the window (bounded: a copy that never lands
      // sets the error flag and ends the kernel)
      uint32_t done = 0;
      for (long long it = 0; it < kStageSpin && !done; ++it)
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(smem_addr(&bar)), "r"(phase) : "memory");
      if (!done) atomicExch(&s_abort, 1);
      phase ^= 1u;
    }
    __syncthreads();
    if (s_abort) {
      if (threadIdx.x == 0) atomicAdd(err, 1ull);
      break;
    }
    const int nr = (int)(r1 - r0);
    for (;;) {
      const int k = atomicAdd(&s_next, 1);           // the next ray of the batch
      if (k >= nr) break;
      const int64_t rid = r0 + k;
      const int i = (int)(rid - p_begin);
      EmitOut o;
      emit_ray(a.em, rid, o);
      if (!(o.E0 > 0.0)) {
        if (a.records) {
          double* rec = a.records + (rid - a.rec_base) * XT_PKT_FIELDS;
          rec[0] = 4.0; rec[1] = 0.0; rec[2] = 0.0; rec[3] = 0.0; rec[4] = -1.0; rec[5] = -1.0;
          rec[6] = 0.0; rec[7] = (double)o.c; rec[8] = 0.0; rec[9] = 0.0; rec[10] = 0.0;
        }
        continue;
      }
      int ix = o.idx[0], iy = o.idx[1], iz = o.idx[2];
      double tmx = o.tm[0], tmy = o.tm[1], tmz = o.tm[2];
      const int sx = bits(o.td[0]) < 0 ? -1 : 1, sy = bits(o.td[1]) < 0 ? -1 : 1, sz = bits(o.td[2]) < 0 ? -1 : 1;
      const double tdx = dabs_bits(o.td[0]), tdy = dabs_bits(o.td[1]), tdz = dabs_bits(o.td[2]);
      const double nu0 = o.nu_cmf, aslope = o.nu_lab * a.inv_ct;
      double N = o.N;
      const double N_in = N, Tq = (a.em.e_cut * o.E0) * (1.0 / kH);
      int cursor = o.cursor, events = 0;
      P.F(F_NX, i) = o.n[0]; P.F(F_NY, i) = o.n[1]; P.F(F_NZ, i) = o.n[2];
      P.F(F_NULAB, i) = o.nu_lab;
      P.pid[i] = rid;
      acc[T_EMITN] += o.N;
      acc[T_EMITE] += o.E0;
      if (a.records) {
        double* rec = a.records + (rid - a.rec_base) * XT_PKT_FIELDS;
        rec[7] = (double)o.c; rec[8] = o.N; rec[9] = o.nu_cmf;
      }
      int row = RX[ix] + RY[iy] + RZ[iz];
      int fate = -1;
      bool escaped = false;
      for (;;) {
        double sw = tmx;
        int axis = 0;
        if (bits(tmy) < bits(sw)) { sw = tmy; axis = 1; }
        if (bits(tmz) < bits(sw)) { sw = tmz; axis = 2; }
        const long long end_bits = bits(nu0 - aslope * sw);
        const double* prow = a.pops + (int64_t)row * a.nlev;
        for (;;) {
          if (cursor >= a.nline) break;
          const int wi = cursor - base;
          const LineRec L = (wi >= 0 && wi < wl)
                                ? LineRec{s_lines[2 * wi].x, s_lines[2 * wi].y, s_lines[2 * wi + 1].x, s_lines[2 * wi + 1].y}
                                : ldline(a.lines, cursor);
          if (bits(L.x) <= end_bits) break;
          ++n_tests;
          const double n_l = prow[__double2loint(L.w)], n_u = prow[__double2hiint(L.w)];
          const double tau = L.y * (n_l - L.z * n_u);
          if (bits(tau) > taumin_bits) {
            ++events;
            ++n_events;
            double ex, ome;
            expneg(fx, tau, ex, ome);
            const int64_t slot = (a.crow ? (int64_t)a.crow[row] : (int64_t)row) * a.nline + cursor;
            atomicAdd(a.S + slot, N * ome);
            const unsigned long long kk = atomicAdd(&blk_log, 1ull);
            if (kk < (unsigned long long)a.seg_len) my_log[kk] = slot;
            N = N * ex;
            if (bits(N * L.x) < bits(Tq)) { acc[T_DROP] += N; fate = 1; break; }
            if (events >= a.max_events) { ++n_guard; fate = 3; break; }
          }
          ++cursor;
        }
        if (fate >= 0) break;
        const bool a0 = axis == 0, a1 = axis == 1;
        const int coord = (a0 ? ix : a1 ? iy : iz) + (a0 ? sx : a1 ? sy : sz);
        const double tnew = (a0 ? tmx : a1 ? tmy : tmz) + (a0 ? tdx : a1 ? tdy : tdz);
        if (a0) { ix = coord; tmx = tnew; } else if (a1) { iy = coord; tmy = tnew; } else { iz = coord; tmz = tnew; }
        if (coord < 0 || coord >= (a0 ? g.nx : a1 ? g.ny : g.nz)) { escaped = true; break; }
        row = RX[ix] + RY[iy] + RZ[iz];
      }
      P.F(F_N, i) = N;
      P.events[i] = events;
      acc[T_ABS] += N_in - N;
      if (fate >= 0 && a.records) {
        double* rec = a.records + (rid - a.rec_base) * XT_PKT_FIELDS;
        rec[0] = fate; rec[1] = events; rec[2] = N; rec[3] = 0.0; rec[4] = -1.0; rec[5] = -1.0;
        rec[6] = 0.0; rec[10] = o.nu_lab;
      }
      if (escaped) {
        P.inter[i] = 0;
        a.esc[atomicAdd(a.n_esc, 1ull)] = i;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long nb = blk_log;
    if (nb > (unsigned long long)a.seg_len) atomicAdd(a.log_overflow, 1ull);
    a.seg_n[blockIdx.x] = (int64_t)(nb < (unsigned long long)a.seg_len ? nb : a.seg_len);
  }
  double cnt[3] = {(double)n_tests, (double)n_events, (double)n_guard};
  const int cslots[3] = {LG_TESTS, LG_EVENTS, LG_GUARD};
  warp_flush(cnt, a.ledger, cslots);
  const int slots[T_NACC] = {LG_ABS_N, LG_DROP_N, LG_ABS_E_CMF, LG_REEMIT_E_CMF, LG_THERMAL_E,
                             LG_EMIT_N, LG_EMIT_E};
  warp_flush(acc, a.ledger, slots);
}

// ---------------------------------------------------------------- spherical grid
// The attenuation pass on a spherical grid (Sec. 2: radial shells, polar and
// azimuthal sectors).  The walk's coordinate is the path s from the emission
// point p0 along n; every face crossing is a root of a quadratic (a sphere or
// a polar cone) or a linear equation (the equatorial plane, an azimuthal
// half-plane) in s whose coefficients come from p0 and n alone (b = p0.n,
// pp = p0.p0 per packet), solved by one routine, so that a face solved again
// gives exactly the path at which it was crossed and is excluded by s > s_cur:
// no nudging and no accumulated error.  The three families of faces (shells,
// polar edges, azimuthal edges) keep their next crossing; crossing a face
// changes only its own family's faces, so only that family is solved again.
// Within a family one face is solved first: along a straight line phi is
// monotonic (the side is the sign of (p0 x n)_z), d cos(theta) / ds changes sign
// at most once (its numerator nz pp - z0 b + s (nz b - z0) is linear in s),
// and a shell's inner sphere can only be met while r decreases (s < -b); the
// other face of the family is solved only when the first has no crossing.
// The persistent warp loop follows k_trace: a lane walks its packet one face
// per iteration, testing the lines between the comoving frequency now and at
// that face (as in k_trace), and empty lanes are refilled together with fresh
// packets (emission: cell from the quota, a point uniform in the cell's volume,
// isotropic direction, comoving frequency as on the cube).  Escaped packets go
// to k_escape through the pool.
constexpr int kSphRefill = 16;   // empty lanes of a warp that trigger a refill

enum { SF_INNER, SF_OUTER, SF_CONE, SF_PLANE, SF_HALF };

// Next crossing s > s_cur (s_cur >= 0) of face family fam (0 shells, 1 polar
// edges, 2 azimuthal edges) from cell (ir, it, ip), and the face (kind 0 outer
// sphere, 1 inner sphere, 2 lower polar edge, 3 upper polar edge, 4 lower
// azimuthal edge, 5 upper azimuthal edge; -1 and INFINITY for none).  Every
// face is A s^2 + 2 B s + C = 0 (a sphere A = 1, B = b, C = pp - R^2; a cone;
// A = 0 for a plane), solved with one square root and one reciprocal for all
// of them, so that the lanes of a warp on different families stay together;
// comparisons are on the bit patterns (integer pipe: the FP64 pipe, 2 lanes
// per SM and cycle, is the scarce one).  For a sphere the reciprocal is 1 and
// the roots are -b -/+ sqrt(disc) exactly.  Not inlined: every crossing of the
// kernel is solved by this one code.
__device__ __noinline__ double sph_next(const double* __restrict__ tab, int tnx, int tny, int tnz, int fam,
                                        double p0x, double p0y, double p0z, double nx_, double ny_,
                                        double nz_, double b, double pp, int ir, int it, int ip,
                                        double s_cur, int* kind_out) {
  const double* sR = tab;
  const double* cth = sR + tnx + 1;
  const double* cph = cth + tny + 1;
  const double* sph = cph + tnz + 1;
  const long long scb = bits(s_cur);
  const long long infb = bits(INFINITY);
  int k;
  if (fam == 0) {
    k = (ir > 0 && bits(-b) > scb) ? 1 : 0;                          // r decreasing: s < -b
  } else if (fam == 1) {
    const double g = nz_ * pp - p0z * b + s_cur * (nz_ * b - p0z);   // sign of d cos(theta) / ds
    k = bits(g) > 0 ? 2 : 3;
    const int j = it + k - 2;
    if (j == 0 || j == tny) k = 5 - k;                                // the polar axis is no face
    const int j2 = it + k - 2;
    if (j2 == 0 || j2 == tny) k = -1;
  } else {
    k = tnz < 2 ? -1 : (bits(p0x * ny_ - p0y * nx_) > 0 ? 5 : 4);
  }
  for (int att = 0; att < 2 && k >= 0; ++att) {
    double A, B, C, u = 0.0, v = 0.0;
    int side;
    if (k <= 1) {
      const double R = sR[ir + 1 - k];
      A = 1.0; B = b; C = pp - R * R;
      side = k == 1 ? SF_INNER : SF_OUTER;
    } else if (k <= 3) {
      const double c = cth[it + k - 2];
      if ((bits(c) << 1) == 0) {                                      // the plane z = 0
        A = 0.0; B = 0.5 * nz_; C = p0z;
        side = SF_PLANE;
      } else {
        const double c2 = c * c;
        A = nz_ * nz_ - c2; B = p0z * nz_ - c2 * b; C = p0z * p0z - c2 * pp;
        side = SF_CONE;
        u = c;
      }
    } else {
      const int e = ip + k - 4;
      u = cph[e]; v = sph[e];
      A = 0.0; B = 0.5 * (ny_ * u - nx_ * v); C = p0y * u - p0x * v;
      side = SF_HALF;
    }
    const bool lin = (bits(A) << 1) == 0;
    const double disc = B * B - A * C;
    const long long db = bits(disc);
    const double sq = db > 0 ? sqrt(disc) : 0.0;
    const double inv = 1.0 / (lin ? B + B : A);
    double r0 = INFINITY, r1 = INFINITY;
    if (lin) {
      if ((bits(B) << 1) != 0) r0 = -C * inv;
    } else if (db > 0 || ((db << 1) == 0 && side == SF_CONE)) {
      const double sa = (-B - sq) * inv, sb = (-B + sq) * inv;
      const bool apos = bits(A) > 0;                                  // then sa <= sb
      r0 = apos ? sa : sb;
      r1 = apos ? sb : sa;
      if (side == SF_INNER) r1 = INFINITY;                            // the nearer crossing only
      else if (side == SF_OUTER) { r0 = r1; r1 = INFINITY; }          // the farther only
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const double r = q == 0 ? r0 : r1;
      const long long rb = bits(r);
      if (rb <= scb || rb >= infb) continue;                          // r > s_cur, finite
      bool on = true;
      if (side == SF_CONE) on = bits((p0z + r * nz_) * u) > 0;        // its own nappe
      else if (side == SF_HALF) on = bits((p0x + r * nx_) * u + (p0y + r * ny_) * v) > 0;  // its own side
      if (on) { *kind_out = k; return r; }
    }
    if (att == 0) {                                                   // the family's other face
      if (fam == 0) k = k == 1 ? 0 : -1;
      else if (fam == 1) {
        k = 5 - k;
        const int j = it + k - 2;
        if (j == 0 || j == tny) k = -1;
      } else k = 9 - k;
    }
  }
  *kind_out = -1;
  return INFINITY;
}

// DOM: one domain of a spatial decomposition across processes (Sec. 2.4.1,
// rounds == 3): work items below em.n are the domain's own packets, emitted
// here; the rest resume from the pool (states received from other domains).
// A packet that enters a cell outside the domain's phi slices [dom_zlo,
// dom_zhi) leaves: its state (emission point, direction, lab and comoving
// frequency, photons, energy cut, path s, cursor, events, cell) goes to the
// pool and its slot to the out list.
// RAYS: the rays of the RAYS sampler instead of Monte Carlo packets.
// PI: photoionization on every segment (Sec. 2.3.1, pi_segment as in k_trace:
// up to each line's resonance point before the line acts, then up to the
// exit face), the path coordinate being the walk's own.
template <bool DOM, bool RAYS = false, bool PI = false>
__global__ void __launch_bounds__(256) k_trace_sph(const TraceArgs a) {
  __shared__ FixExpTables fx;
  __shared__ FixTrigTables trig;
  __shared__ unsigned long long blk_log;
  constexpr int kPiS = PI ? XT_PI_MAX : 1;          // photoionization tables (PI instance)
  __shared__ double s_nuth[kPiS], s_sig[kPiS];
  __shared__ int s_lev[kPiS];
  stage(fx, a.fx);
  stage(trig, a.trig);
  if constexpr (PI) {
    for (int k = threadIdx.x; k < a.npi; k += blockDim.x) {
      s_nuth[k] = a.pi_nuth[k]; s_sig[k] = a.pi_sig[k]; s_lev[k] = a.pi_lev[k];
    }
  }
  if (threadIdx.x == 0) blk_log = (unsigned long long)a.seg_n[blockIdx.x];
  __syncthreads();
  int64_t* const my_log = a.slotlog + (int64_t)blockIdx.x * a.seg_len;
  const Geometry& g = a.g;
  const EmitArgs& em = a.em;
  const Pool& P = a.pool;
  const double* const sR = g.sph;
  const double* const cth = sR + g.nx + 1;
  const double* const phe = cth + g.ny + 1 + 2 * (g.nz + 1);
  const double* const the = phe + g.nz + 1;
  const int* RX = a.rtab;
  const int* RY = a.rtab + g.nx;
  const int* RZ = a.rtab + g.nx + g.ny;
  const long long taumin_bits = bits(a.tau_min);
  const int lane = threadIdx.x & 31;
  // a straight path meets each sphere and cone at most twice, each half-plane once
  const int max_faces = 2 * (g.nx + g.ny) + g.nz + 8;
  constexpr int kAcc = PI ? T_PIE + 1 : T_NACC;
  double acc[kAcc];
#pragma unroll
  for (int k = 0; k < kAcc; ++k) acc[k] = 0.0;
  unsigned n_tests = 0, n_events = 0, n_guard = 0;

  bool have = false, drained = false;
  int i = 0, ix = 0, iy = 0, iz = 0, row = 0, cursor = 0, events = 0, faces = 0;
  int k_r = -1, k_t = -1, k_p = -1;
  double p0x = 0, p0y = 0, p0z = 0, nxv = 0, nyv = 0, nzv = 0, b = 0, pp = 0, s = 0;
  double s_r = 0, s_t = 0, s_p = 0, nu_cmf = 0, aslope = 0, N = 0, N_in = 0, Tq = 0;
  // photoionization: segment start, 1 / aslope, the packet's photoionized
  // photons, first level still active
  double s_pi = 0, inv_as = 0, N_pi = 0;
  int pcur = 0;
  for (;;) {
    __syncwarp();
    {
      const unsigned full = 0xffffffffu;
      const unsigned m0 = __ballot_sync(full, !have);
      if (m0 == full && drained) break;
      const unsigned m =
          (drained || (m0 != full && __popc(m0) < (RAYS ? kRayRefillLanes : kSphRefill))) ? 0u : m0;
      if (m) {
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(a.counter, (unsigned long long)__popc(m));
        base = __shfl_sync(full, base, leader);
        if (base + __popc(m) >= (unsigned long long)a.n_list) drained = true;
        const unsigned long long my = base + __popc(m & ((1u << lane) - 1u));
        if (DOM && !have && my < (unsigned long long)a.n_list && my >= (unsigned long long)em.n) {
          // ---- a packet handed on by another domain resumes
          i = (int)my;
          const int cs = P.cell[i];
          ix = cs & 1023; iy = (cs >> 10) & 1023; iz = cs >> 20;
          p0x = P.F(F_R0X, i); p0y = P.F(F_R0Y, i); p0z = P.F(F_R0Z, i);
          nxv = P.F(F_NX, i); nyv = P.F(F_NY, i); nzv = P.F(F_NZ, i);
          nu_cmf = P.F(F_NU0, i);
          aslope = P.F(F_NULAB, i) * a.inv_ct;
          N = P.F(F_N, i);
          N_in = N;
          Tq = P.F(F_T, i);
          s = P.F(F_TMX, i);
          cursor = P.cursor[i];
          events = P.events[i];
          faces = 0;
          if constexpr (PI) {
            s_pi = P.F(F_SPI, i);
            N_pi = 0.0;
            inv_as = div_pos(a.ct, P.F(F_NULAB, i));
            const double nu_s = fma(-aslope, s_pi, nu_cmf);
            pcur = 0;
            while (pcur < a.npi && s_nuth[pcur] >= nu_s) ++pcur;
          }
          b = nxv * p0x + nyv * p0y + nzv * p0z;
          pp = p0x * p0x + p0y * p0y + p0z * p0z;
          row = RX[ix] + RY[iy] + RZ[iz];
          s_r = sph_next(g.sph, g.nx, g.ny, g.nz, 0, p0x, p0y, p0z, nxv, nyv, nzv, b, pp, ix, iy, iz, s, &k_r);
          s_t = sph_next(g.sph, g.nx, g.ny, g.nz, 1, p0x, p0y, p0z, nxv, nyv, nzv, b, pp, ix, iy, iz, s, &k_t);
          s_p = sph_next(g.sph, g.nx, g.ny, g.nz, 2, p0x, p0y, p0z, nxv, nyv, nzv, b, pp, ix, iy, iz, s, &k_p);
          have = true;
        } else if (!have && my < (unsigned long long)a.n_list) {
          // ---- emission
          i = (int)my;
          const int64_t p = RAYS ? ray_id_of(em, em.p_begin + (int64_t)my) : em.p_begin + (int64_t)my;
          int64_t c;
          int idx[3];
          double E0;
          bool live = true;
          if constexpr (RAYS) {
            // ray p (Sec. 2.3): (emitting-cell rank, bin rank, viewer), from the
            // middle of the cell's r, theta and phi ranges along the viewer's
            // centre direction, carrying the bin's emission times dOmega / 4 pi
            const RayTables& T = em.ray;
            const int64_t per_cell = T.nbin * T.nview;
            const int64_t ci = p / per_cell, rem = p - ci * per_cell, jb = rem / T.nview;
            const int kv = (int)(rem - jb * T.nview);
            c = T.rcell[ci];
            {
              const uint32_t c32 = (uint32_t)c, gx = (uint32_t)g.nx, gy = (uint32_t)g.ny;
              const uint32_t cy = c32 / gx;
              idx[0] = (int)(c32 - cy * gx); idx[1] = (int)(cy % gy); idx[2] = (int)(cy / gy);
            }
            const double2 v01 = __ldg(reinterpret_cast<const double2*>(T.view) + 2 * kv);
            const double2 v23 = __ldg(reinterpret_cast<const double2*>(T.view) + 2 * kv + 1);
            const double E_bin = T.Ebin ? T.Ebin[row_of(g, idx[0], idx[1], idx[2]) * T.nbin + jb]
                                        : em.Lc[c] * T.bin_frac[jb];
            E0 = E_bin * v23.y;
            if (!(E0 > 0.0)) {                 // an empty ray: recorded, not traced
              if (a.records) {
                double* rec = a.records + (p - a.rec_base) * XT_PKT_FIELDS;
                rec[0] = 4.0; rec[1] = 0.0; rec[2] = 0.0; rec[3] = 0.0; rec[4] = -1.0; rec[5] = -1.0;
                rec[6] = 0.0; rec[7] = (double)c; rec[8] = 0.0; rec[9] = 0.0; rec[10] = 0.0;
              }
              live = false;                    // (the lane stays empty; no early continue: every
            }                                  //  lane reaches the warp-wide ballot below)
            nxv = v01.x; nyv = v01.y; nzv = v23.x;
            const double* const mid = the + g.ny + 1 + 3 * c;   // the cell's middle, tabulated
            p0x = mid[0]; p0y = mid[1]; p0z = mid[2];
            nu_cmf = T.bin_nu[jb];
            cursor = T.bin_cursor[jb];
          } else {
          c = quota_cell(em, p);
          E0 = em.Epk[c];
          {
            const uint32_t c32 = (uint32_t)c, gx = (uint32_t)g.nx, gy = (uint32_t)g.ny;
            const uint32_t cy = c32 / gx;
            idx[0] = (int)(c32 - cy * gx); idx[1] = (int)(cy % gy); idx[2] = (int)(cy / gy);
          }
          uint64_t xu[4], xv[4];
          draw_raw(em.seed, p, 0, xu);
          draw_raw(em.seed, p, 1, xv);
          {   // uniform in the cell's volume: r^3, cos theta and phi uniform
            const double R0 = sR[idx[0]], R1 = sR[idx[0] + 1];
            const double R03 = R0 * R0 * R0, R13 = R1 * R1 * R1;
            const double rr = cbrt(R03 + u01(xu[0]) * (R13 - R03));
            const double c0 = cth[idx[1]], c1 = cth[idx[1] + 1];
            const double ct = c0 - u01(xu[1]) * (c0 - c1);
            const double ph0 = phe[idx[2]], ph1 = phe[idx[2] + 1];
            const double ph = ph0 + u01(xu[2]) * (ph1 - ph0);
            double sp, cp;
            sincos(ph, &sp, &cp);
            const double q = 1.0 - ct * ct;
            const double st = bits(q) > 0 ? sqrt(q) : 0.0;
            p0x = rr * st * cp; p0y = rr * st * sp; p0z = rr * ct;
          }
          double n[3];
          isotropic(trig, xu[3] >> 11, xv[0] >> 11, n);
          nxv = n[0]; nyv = n[1]; nzv = n[2];
          emit_frequency(em, xv[1], c, idx, nu_cmf, cursor);
          }
          if (live) {
            b = nxv * p0x + nyv * p0y + nzv * p0z;
            pp = p0x * p0x + p0y * p0y + p0z * p0z;
            const double nu_lab = div_pos(nu_cmf, 1.0 - b * a.inv_ct);
            aslope = nu_lab * a.inv_ct;                      // d nu_cmf / ds
            if constexpr (RAYS) {
              N = div_pos(E0, kH * nu_cmf);
              Tq = (em.e_cut * E0) * (1.0 / kH);
            } else {
              N = div_pos(em.Eph[c], nu_cmf);                // E0 / (h nu_cmf)
              Tq = em.e_cut * em.Eph[c];
            }
            N_in = N;
            if constexpr (PI) {
              s_pi = 0.0;
              N_pi = 0.0;
              inv_as = div_pos(a.ct, nu_lab);
              pcur = 0;
              while (pcur < a.npi && s_nuth[pcur] >= nu_cmf) ++pcur;
            }
            P.F(F_NX, i) = nxv; P.F(F_NY, i) = nyv; P.F(F_NZ, i) = nzv;
            P.F(F_NULAB, i) = nu_lab;
            P.pid[i] = p;
            acc[T_EMITN] += N;
            acc[T_EMITE] += E0;
            if (a.records) {
              P.inter[i] = 0;
              double* rec = a.records + (p - a.rec_base) * XT_PKT_FIELDS;
              rec[7] = (double)c; rec[8] = N; rec[9] = nu_cmf;
            }
            ix = idx[0]; iy = idx[1]; iz = idx[2];
            row = RX[ix] + RY[iy] + RZ[iz];
            s = 0.0;
            events = 0;
            faces = 0;
            s_r = sph_next(g.sph, g.nx, g.ny, g.nz, 0, p0x, p0y, p0z, nxv, nyv, nzv, b, pp, ix, iy, iz, 0.0,
                             &k_r);
            s_t = sph_next(g.sph, g.nx, g.ny, g.nz, 1, p0x, p0y, p0z, nxv, nyv, nzv, b, pp, ix, iy, iz, 0.0,
                             &k_t);
            s_p = sph_next(g.sph, g.nx, g.ny, g.nz, 2, p0x, p0y, p0z, nxv, nyv, nzv, b, pp, ix, iy, iz, 0.0,
                             &k_p);
            have = true;
          }
        }
      }
    }
    const unsigned busy = __ballot_sync(0xffffffffu, have);
    if (!have) continue;

    // ---- one face: the lines up to it, then across it
    double s_exit = s_r;                                // (all >= 0: compared as bit patterns)
    int kind = k_r;
    if (bits(s_t) < bits(s_exit)) { s_exit = s_t; kind = k_t; }   // ties to the lower kind
    if (bits(s_p) < bits(s_exit)) { s_exit = s_p; kind = k_p; }
    int fate = -1, fam = 0;
    bool escaped = false, queued = false;
    if (kind < 0 || ++faces > max_faces) {
      ++n_guard;
      fate = 3;
    } else {
      const long long end_bits = bits(nu_cmf - aslope * s_exit);
      const double* prow = a.pops + (int64_t)row * a.nlev;
      while (cursor < a.nline) {
        const LineRec L = ldline(a.lines, cursor);
        if (bits(L.x) <= end_bits) break;
        ++n_tests;
        const double n_l = prow[__double2loint(L.w)], n_u = prow[__double2hiint(L.w)];
        const double tau = L.y * (n_l - L.z * n_u);
        if (bits(tau) > taumin_bits) {
          if constexpr (PI) {    // to the resonance point, photoionizing on the way
            const double s_l = (nu_cmf - L.x) * inv_as;
            if (pi_segment(a, fx, s_nuth, s_sig, s_lev, row, prow, s_pi, s_l, nu_cmf, aslope, inv_as, pcur, N,
                           N_pi, acc[T_PIE], Tq)) {
              acc[T_DROP] += N;
              fate = 1;
              break;
            }
            if (bits(s_l) > bits(s_pi)) s_pi = s_l;
          }
          ++events;
          ++n_events;
          double ex, ome;
          expneg(fx, tau, ex, ome);
          const int64_t slot = (a.crow ? (int64_t)a.crow[row] : (int64_t)row) * a.nline + cursor;
          atomicAdd(a.S + slot, N * ome);
          const unsigned long long k = atomicAdd(&blk_log, 1ull);
          if (k < (unsigned long long)a.seg_len) my_log[k] = slot;
          N = N * ex;
          if (bits(N * L.x) < bits(Tq)) { acc[T_DROP] += N; fate = 1; }
          else if (events >= a.max_events) { ++n_guard; fate = 3; }
        }
        ++cursor;
        if (fate >= 0) break;
      }
      if constexpr (PI) {      // photoionization up to the exit face
        if (fate < 0) {
          if (pi_segment(a, fx, s_nuth, s_sig, s_lev, row, prow, s_pi, s_exit, nu_cmf, aslope, inv_as, pcur,
                         N, N_pi, acc[T_PIE], Tq)) {
            acc[T_DROP] += N;
            fate = 1;
          } else if (bits(s_exit) > bits(s_pi)) {
            s_pi = s_exit;
          }
        }
      }
      if (fate < 0) {
        s = s_exit;
        if (kind <= 1) {
          fam = 0;
          if (kind == 0) escaped = ++ix == g.nx;
          else --ix;
        } else if (kind <= 3) {
          fam = 1;
          iy += kind == 2 ? -1 : 1;
        } else {
          fam = 2;
          iz = kind == 4 ? (iz == 0 ? g.nz - 1 : iz - 1) : (iz == g.nz - 1 ? 0 : iz + 1);
        }
        if (!escaped) row = RX[ix] + RY[iy] + RZ[iz];
        if (DOM && !escaped && (iz < a.dom_zlo || iz >= a.dom_zhi)) {
          // ---- the packet enters another domain's slices: its state goes on
          queued = true;
          P.F(F_R0X, i) = p0x; P.F(F_R0Y, i) = p0y; P.F(F_R0Z, i) = p0z;
          P.F(F_NU0, i) = nu_cmf;
          P.F(F_T, i) = Tq;
          P.F(F_TMX, i) = s;
          if constexpr (PI) P.F(F_SPI, i) = s_pi;
          P.cursor[i] = cursor;
          P.cell[i] = ix | (iy << 10) | (iz << 20);
        }
      }
    }
    // ---- the crossed family's next face, solved by every busy lane of the
    // warp together after the divergent line tests (a lane without a face to
    // solve passes cell (0, 0, 0) and drops the result): measured 1.5x faster
    // than solving inside the lanes' own branches
    __syncwarp(busy);
    {
      const bool solve = fate < 0 && !escaped && !queued;
      int kn;
      const double sn = sph_next(g.sph, g.nx, g.ny, g.nz, fam, p0x, p0y, p0z, nxv, nyv, nzv, b, pp,
                                 solve ? ix : 0, solve ? iy : 0, solve ? iz : 0, s, &kn);
      if (solve) {
        if (fam == 0) { s_r = sn; k_r = kn; }
        else if (fam == 1) { s_t = sn; k_t = kn; }
        else { s_p = sn; k_p = kn; }
      }
    }
    // ---- the packet leaves the lane
    if (escaped || queued || fate >= 0) {
      P.F(F_N, i) = N;
      P.events[i] = events;
      if constexpr (PI) {
        acc[T_ABS] += (N_in - N) - N_pi;               // photons the lines absorbed
        acc[T_PIN] += N_pi;
      } else {
        acc[T_ABS] += N_in - N;
      }
      if (fate >= 0 && a.records) {
        double* rec = a.records + (P.pid[i] - a.rec_base) * XT_PKT_FIELDS;
        rec[0] = fate; rec[1] = events; rec[2] = N; rec[3] = 0.0; rec[4] = -1.0; rec[5] = -1.0;
        rec[6] = 0.0; rec[10] = P.F(F_NULAB, i);
      }
      have = false;
    }
    warp_append(escaped, i, a.esc, a.n_esc);
    if (DOM) warp_append(queued, i, a.out, a.n_out);
  }
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long nb = blk_log;
    if (nb > (unsigned long long)a.seg_len) atomicAdd(a.log_overflow, 1ull);
    a.seg_n[blockIdx.x] = (int64_t)(nb < (unsigned long long)a.seg_len ? nb : a.seg_len);
  }
  double cnt[3] = {(double)n_tests, (double)n_events, (double)n_guard};
  const int cslots[3] = {LG_TESTS, LG_EVENTS, LG_GUARD};
  warp_flush(cnt, a.ledger, cslots);
  const int all_slots[T_PIE + 1] = {LG_ABS_N, LG_DROP_N, LG_ABS_E_CMF, LG_REEMIT_E_CMF, LG_THERMAL_E,
                                    LG_EMIT_N, LG_EMIT_E, LG_PI_N, LG_PI_E};
  int slots[kAcc];
#pragma unroll
  for (int k = 0; k < kAcc; ++k) slots[k] = all_slots[k];
  warp_flush(acc, a.ledger, slots);
}

// ---------------------------------------------------------------- escape
__global__ void __launch_bounds__(256) k_escape(const EscArgs a) {
  double acc[3] = {0.0, 0.0, 0.0};
  const Pool& P = a.pool;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.n_esc;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = a.esc[j];
    const double N = P.F(F_N, i), nu_lab = P.F(F_NULAB, i);
    const double n[3] = {P.F(F_NX, i), P.F(F_NY, i), P.F(F_NZ, i)};
    const double E = N * kH * nu_lab;
    acc[0] += N;
    acc[1] += E;
    const double th = acos(n[2]);
    double ph = atan2(n[1], n[0]);
    if (ph < 0.0) ph += 2.0 * kPi;
    int it = (int)floor(th / (kPi / a.n_theta)), ip = (int)floor(ph / (2.0 * kPi / a.n_phi));
    it = min(max(it, 0), a.n_theta - 1);
    ip = min(max(ip, 0), a.n_phi - 1);
    const int vbin = it * a.n_phi + ip;
    int64_t lbin = -1;
    const double lam = kC / nu_lab * 1e8;
    if (lam >= a.lam0) {
      const double kb = floor(log(lam / a.lam0) / a.log1p_dlog);
      if (kb < (double)a.nbins) lbin = (int64_t)kb;
    }
    if (lbin >= 0) atomicAdd(a.spec + (int64_t)vbin * a.nbins + lbin, E);
    else acc[2] += E;
    if (a.records) {
      double* rec = a.records + (P.pid[i] - a.rec_base) * XT_PKT_FIELDS;
      rec[0] = 0.0; rec[1] = P.events[i]; rec[2] = N; rec[3] = E; rec[4] = vbin;
      rec[5] = (double)lbin; rec[6] = P.inter[i]; rec[10] = nu_lab;
    }
  }
  const int slots[3] = {LG_ESC_N, LG_ESC_E, LG_OOB_E};
  warp_flush(acc, a.ledger, slots);
}

// ---------------------------------------------------------------- subdomain queue sort
__global__ void k_sd_hist(Geometry g, const int* __restrict__ cell, const int* __restrict__ q,
                          int64_t n, int* __restrict__ key, unsigned* __restrict__ hist) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int cs = cell[q[j]];
    const int ix = cs & 1023, iy = (cs >> 10) & 1023, iz = cs >> 20;
    const int sd = ((iz / g.bz) * g.sy + iy / g.by) * g.sx + ix / g.bx;
    key[j] = sd;
    atomicAdd(hist + sd, 1u);
  }
}

// streamed groups: key = the group of the packet's cell (grp_nz cells along z per group)
__global__ void k_grp_hist(const int* __restrict__ cell, const int* __restrict__ q, int64_t n, int grp_nz,
                           int* __restrict__ key, unsigned* __restrict__ hist) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int g = (cell[q ? q[j] : j] >> 20) / grp_nz;
    key[j] = g;
    atomicAdd(hist + g, 1u);
  }
}

// Packets that left a streamed group: those now in group `next` go to `carry`
// (traced later in the same sweep), the others to `pend` (the next sweep).
__global__ void k_grp_split(const int* __restrict__ cell, const int* __restrict__ q, int64_t n, int grp_nz,
                            int next, int* __restrict__ carry, unsigned long long* __restrict__ n_carry,
                            int* __restrict__ pend, unsigned long long* __restrict__ n_pend) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int i = q[j];
    if ((cell[i] >> 20) / grp_nz == next) carry[atomicAdd(n_carry, 1ull)] = i;
    else pend[atomicAdd(n_pend, 1ull)] = i;
  }
}

__global__ void k_iota(int* __restrict__ out, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    out[j] = (int)j;
}

// Bundles of packets handed between domains: pool entry <-> XT_BUNDLE_FIELDS
// doubles (the NF state fields, then cell, cursor, events, draws,
// interactions and id; integers exactly).
static_assert(NF + 6 <= XT_BUNDLE_FIELDS && NF == XT_BUNDLE_CELL, "bundle layout");
// Received packet states into the pool; entries whose cell lies outside the
// grid or whose line cursor lies outside [0, nline] are counted in *bad (the
// caller refuses the bundle before any trace kernel reads the pool).
__global__ void k_bundle_in(Pool P, const double* __restrict__ in, int64_t n, int64_t base, Geometry g,
                            int nline, unsigned long long* __restrict__ bad) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double* e = in + j * XT_BUNDLE_FIELDS;
    const int64_t i = base + j;
#pragma unroll
    for (int k = 0; k < NF; ++k) P.F(k, i) = e[k];
    const double cd = e[NF], ud = e[NF + 1];
    const bool ok = cd >= 0.0 && cd < 1073741824.0 && ud >= 0.0 && ud <= (double)nline;
    const int cs = ok ? (int)cd : 0;
    const int cx = cs & 1023, cy = (cs >> 10) & 1023, cz = cs >> 20;
    if (!ok || cx >= g.nx || cy >= g.ny || cz >= g.nz) atomicAdd(bad, 1ull);
    P.cell[i] = cs; P.cursor[i] = ok ? (int)ud : 0; P.events[i] = (int)e[NF + 2];
    P.ndraw[i] = (int)e[NF + 3]; P.inter[i] = (int)e[NF + 4]; P.pid[i] = (int64_t)e[NF + 5];
  }
}

__global__ void k_bundle_out(Pool P, const int* __restrict__ q, int64_t n, double* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    double* e = out + j * XT_BUNDLE_FIELDS;
    const int i = q[j];
#pragma unroll
    for (int k = 0; k < NF; ++k) e[k] = P.F(k, i);
    e[NF] = (double)P.cell[i]; e[NF + 1] = (double)P.cursor[i]; e[NF + 2] = (double)P.events[i];
    e[NF + 3] = (double)P.ndraw[i]; e[NF + 4] = (double)P.inter[i]; e[NF + 5] = (double)P.pid[i];
    for (int k = NF + 6; k < XT_BUNDLE_FIELDS; ++k) e[k] = 0.0;
  }
}

__global__ void k_sd_scatter(const int* __restrict__ q, const int* __restrict__ key, int64_t n,
                             unsigned* __restrict__ fill, int* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    out[atomicAdd(fill + key[j], 1u)] = q[j];
}

// ---------------------------------------------------------------- line emission weights
// A_ul dE_ul beta_S N_u, Eq. (thin_emissivity), as an inclusive prefix over the
// caller's line order per cell; Lc = the total.
__global__ void k_line_emission(Geometry g, const double2* __restrict__ lines,
                                const double* __restrict__ A, int nline, int nlev,
                                const double* __restrict__ pops, const int* __restrict__ sorted_of,
                                double V, double* __restrict__ cdf, double* __restrict__ Lc) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(c % g.nx), iy = (int)((c / g.nx) % g.ny), iz = (int)(c / ((int64_t)g.nx * g.ny));
    const int64_t row = row_of(g, ix, iy, iz);
    const double* pc = pops + row * nlev;
    double* cr = cdf + row * nline;
    const double Vc = g.vol ? g.vol[row] : V;
    double run = 0.0;
    for (int l = 0; l < nline; ++l) {
      const int s = sorted_of[l];
      const LineRec L = ldline(lines, s);
      const double nu_ = pc[__double2hiint(L.w)];
      const double tau = L.y * (pc[__double2loint(L.w)] - L.z * nu_);
      run += A[s] * (kH * L.x) * sobolev_beta(tau) * nu_ * Vc;
      cr[l] = run;
    }
    Lc[c] = run;
  }
}


// Compact store: 1 for the rows whose populations are not all zero.
__global__ void k_row_flags(int64_t nrows, int nlev, const double* __restrict__ pops, int* __restrict__ flag) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < nrows;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const double* pr = pops + r * nlev;
    bool any = false;
    for (int l = lane; l < nlev; l += 32) any |= pr[l] != 0.0;
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) flag[r] = any ? 1 : 0;
  }
}

// Photoionization: per cell the suffix sums kappa[b] = sum_{k >= b} sig_k n_k
// over the levels sorted by threshold frequency (descending), kappa[npi] = 0.
__global__ void k_pi_kappa(int64_t nrows, int npi, int nlev, const double* __restrict__ pops,
                           const double* __restrict__ sig, const int* __restrict__ lev,
                           double* __restrict__ kappa) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double* pr = pops + r * nlev;
    double* kr = kappa + r * (npi + 1);
    double run = 0.0;
    kr[npi] = 0.0;
    for (int k = npi - 1; k >= 0; --k) {
      run += sig[k] * pr[lev[k]];
      kr[k] = run;
    }
  }
}

// The RAYS sampler with line emission: per cell the emission of every line,
// A_ul h nu beta_S N_u (Eq. thin_emissivity), summed into the cell's
// wavelength bins (caller line order, so each bin's sum runs in ascending
// line index) and in total (Lc, natural order).
__global__ void k_ray_line_bins(Geometry g, const double2* __restrict__ lines, const double* __restrict__ A,
                                int nline, int nlev, const double* __restrict__ pops,
                                const int* __restrict__ sorted_of, const int* __restrict__ bin_of_line,
                                int64_t nbin, double V, double* __restrict__ Ebin, double* __restrict__ Lc) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(c % g.nx), iy = (int)((c / g.nx) % g.ny), iz = (int)(c / ((int64_t)g.nx * g.ny));
    const int64_t row = row_of(g, ix, iy, iz);
    const double* pc = pops + row * nlev;
    double* er = Ebin + row * nbin;
    for (int64_t j = 0; j < nbin; ++j) er[j] = 0.0;
    double run = 0.0;
    for (int l = 0; l < nline; ++l) {
      const int s = sorted_of[l];
      const LineRec L = ldline(lines, s);
      const double nu_ = pc[__double2hiint(L.w)];
      const double tau = L.y * (pc[__double2loint(L.w)] - L.z * nu_);
      const double w = A[s] * (kH * L.x) * sobolev_beta(tau) * nu_ * (g.vol ? g.vol[row] : V);
      run += w;
      er[bin_of_line[l]] += w;
    }
    Lc[c] = run;
  }
}

static int sm_count() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

static int blocks_for(int64_t n, int threads, int per_sm) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * per_sm));
}

}  // namespace xt

using namespace xt;

// Run `fill(dev_out)` writing `bytes` and deliver them to `user` (host or
// device memory).
template <class F>
static int deliver(xt_ctx* c, void* user, size_t bytes, F fill) {
  if (is_device_ptr(user)) {
    fill(user);
    XT_CUDA(c, cudaGetLastError());
    return XT_OK;
  }
  int rc = ensure_scratch(c, bytes);
  if (rc) return rc;
  fill(c->d_scratch);
  XT_CUDA(c, cudaGetLastError());
  return copy(c, user, c->d_scratch, bytes, "device-to-host copy");
}

// Packet pool (NF doubles, 9 ints, one id per slot), counters and the
// subdomain histogram, grown on demand and kept in the context.
static int ensure_buffers(xt_ctx* c, int64_t cap, int nsd) {
  int rc;
  if (c->pool_cap < cap) {
    c->pool_cap = 0;
    if ((rc = alloc(c, (void**)&c->d_pool_f, (size_t)cap * NF * sizeof(double), "packet pool"))) return rc;
    if ((rc = alloc(c, (void**)&c->d_pool_i, (size_t)cap * 9 * sizeof(int), "packet pool"))) return rc;
    if ((rc = alloc(c, (void**)&c->d_pool_pid, (size_t)cap * sizeof(int64_t), "packet pool"))) return rc;
    c->pool_cap = cap;
  }
  if (!c->d_counters && (rc = alloc(c, (void**)&c->d_counters, 8 * sizeof(unsigned long long), "counters"))) return rc;
  if (c->hist_n < nsd) {
    c->hist_n = 0;
    if ((rc = alloc(c, (void**)&c->d_hist, (size_t)2 * nsd * sizeof(unsigned), "subdomain histogram"))) return rc;
    c->hist_n = nsd;
  }
  return XT_OK;
}

// Tables of the RAYS sampler (Sec. 2.3) for this pass: emitting cells, the
// emitting bins of the output grid with their start frequency and first line,
// the band share of each bin or the cells' emission per bin (line emission),
// the viewers' centre directions and solid-angle shares.  Returns the number
// of rays in *n_rays.
static int build_rays(xt_ctx* c, const xt_transport_params* p, RayTables& T, const double*& Lc_nat,
                      int64_t* n_rays, std::vector<int>* rcell_out) {
  const Geometry& G = c->geo;
  const int nb = p->spec_nbins;
  const double lam0 = p->spec_lam0_A, dlog = p->spec_dlog;
  const int nl = c->nline;
  std::vector<double> bnu, bfrac;
  std::vector<int> bcur, bin_of_line;
  const std::vector<double>& snu = c->h_nu_sorted;
  auto cursor_at = [&](double nu) {      // first sorted line with nu <= the given one
    int lo = 0, hi = nl;
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (snu[mid] <= nu) hi = mid; else lo = mid + 1;
    }
    return lo;
  };
  if (p->emission == XT_EMIT_BAND) {
    const double nu_lo = kC / (c->band_hi_A * 1e-8), nu_hi = kC / (c->band_lo_A * 1e-8);
    for (int j = 0; j < nb; ++j) {
      const double l0 = lam0 * std::pow(1.0 + dlog, (double)j);
      const double l1 = lam0 * std::pow(1.0 + dlog, (double)(j + 1));
      const double a = l0 > c->band_lo_A ? l0 : c->band_lo_A;
      const double b = l1 < c->band_hi_A ? l1 : c->band_hi_A;
      if (!(b > a)) continue;
      const double nu_red = kC / (b * 1e-8), nu_blue = kC / (a * 1e-8);
      bnu.push_back(nu_red);
      bcur.push_back(cursor_at(nu_red));
      bfrac.push_back((nu_blue - nu_red) / (nu_hi - nu_lo));
    }
  } else {
    std::vector<int> jmap(nb, -1), best(nb, -1), bin_j(nl);
    for (int l = 0; l < nl; ++l) {
      const double la = c->h_lam_caller[l];
      int64_t j = -1;
      if (la >= lam0) {
        const double k = std::floor(std::log(la / lam0) / std::log1p(dlog));
        if (k < (double)nb) j = (int64_t)k;
      }
      if (j < 0) return fail(c, XT_EINVAL, "run_transport: line " + std::to_string(l) +
                                               " lies outside the output grid (RAYS sampler, line emission)");
      bin_j[l] = (int)j;
      const int s = c->h_sorted_of[l];
      if (best[j] < 0 || s > best[j]) best[j] = s;
    }
    int nbin = 0;
    for (int j = 0; j < nb; ++j)
      if (best[j] >= 0) {
        jmap[j] = nbin++;
        bnu.push_back(snu[best[j]]);
        bcur.push_back(best[j] + 1);
      }
    bin_of_line.resize(nl);
    for (int l = 0; l < nl; ++l) bin_of_line[l] = jmap[bin_j[l]];
  }
  const int64_t nbin = (int64_t)bnu.size();
  // the lines a ray of a bin can reach: its comoving frequency falls by at most
  // nu_lab s_max / ct with s_max <= 2 sqrt(3) R (the cube's diagonal) and
  // nu_lab <= nu_j / (1 - sqrt(3) R / ct); a little margin on top
  std::vector<int> wlen(nbin);
  {
    const double b = c->v_max / kC, r3 = std::sqrt(3.0);
    const double drop = 2.0 * r3 * b / (1.0 - r3 * b) * 1.01 + 1e-9;
    for (int64_t j = 0; j < nbin; ++j) {
      const double nu_min = bnu[j] * (1.0 - drop);
      int lo = bcur[j], hi = nl;                     // first line below nu_min
      while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (snu[mid] < nu_min) hi = mid; else lo = mid + 1;
      }
      wlen[j] = lo - bcur[j];
    }
  }
  const int nview = p->n_theta * p->n_phi;
  std::vector<double> view(4 * (size_t)nview);
  for (int it = 0; it < p->n_theta; ++it)
    for (int ip = 0; ip < p->n_phi; ++ip) {
      const int k = it * p->n_phi + ip;
      const double th = kPi * (it + 0.5) / p->n_theta, ph = 2.0 * kPi * (ip + 0.5) / p->n_phi;
      const double th0 = kPi * it / p->n_theta, th1 = kPi * (it + 1) / p->n_theta;
      view[4 * k] = std::sin(th) * std::cos(ph);
      view[4 * k + 1] = std::sin(th) * std::sin(ph);
      view[4 * k + 2] = std::cos(th);
      view[4 * k + 3] = (2.0 * kPi / p->n_phi) * (std::cos(th0) - std::cos(th1)) / (4.0 * kPi);
    }
  // one device allocation, carved: view | bin_nu | bin_frac | Lc | Ebin | bin_cursor | bin_of_line | rcell
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const bool lines = p->emission == XT_EMIT_LINES;
  const size_t o_view = 0, o_nu = al(o_view + 32 * (size_t)nview), o_frac = al(o_nu + 8 * nbin);
  const size_t o_Lc = al(o_frac + 8 * nbin), o_E = al(o_Lc + 8 * (size_t)G.ncell);
  const size_t o_cur = al(o_E + (lines ? 8 * (size_t)G.ncell * nbin : 0));
  const size_t o_bol = al(o_cur + 4 * nbin), o_rc = al(o_bol + 4 * (size_t)nl);
  const size_t o_wl = al(o_rc + 4 * (size_t)G.ncell);
  const size_t total = al(o_wl + 4 * (size_t)nbin);
  int rc;
  if (c->rays_bytes < total) {
    c->rays_bytes = 0;
    if ((rc = alloc(c, &c->d_rays, total, "ray tables"))) return rc;
    c->rays_bytes = total;
  }
  char* B = (char*)c->d_rays;
  if ((rc = copy(c, B + o_view, view.data(), view.size() * 8, "ray tables"))) return rc;
  if (nbin > 0) {
    if ((rc = copy(c, B + o_nu, bnu.data(), 8 * nbin, "ray tables"))) return rc;
    if ((rc = copy(c, B + o_cur, bcur.data(), 4 * nbin, "ray tables"))) return rc;
    if ((rc = copy(c, B + o_wl, wlen.data(), 4 * nbin, "ray tables"))) return rc;
    if (!lines && (rc = copy(c, B + o_frac, bfrac.data(), 8 * nbin, "ray tables"))) return rc;
  }
  std::vector<double> Lnat;
  if (lines) {
    if ((rc = copy(c, B + o_bol, bin_of_line.data(), 4 * (size_t)nl, "ray tables"))) return rc;
    k_ray_line_bins<<<blocks_for(G.ncell, 128, 16), 128, 0, c->stream>>>(
        G, (const double2*)c->d_lines, c->d_A, nl, c->nlev, c->d_pops, c->d_orig, (const int*)(B + o_bol),
        nbin, G.dx * G.dy * G.dz, (double*)(B + o_E), (double*)(B + o_Lc));
    XT_CUDA(c, cudaGetLastError());
    Lnat.resize(G.ncell);
    XT_CUDA(c, cudaMemcpyAsync(Lnat.data(), B + o_Lc, G.ncell * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
  } else {
    Lnat = c->h_L;
    if ((rc = copy(c, B + o_Lc, Lnat.data(), G.ncell * sizeof(double), "ray tables"))) return rc;
  }
  std::vector<int> rcell;
  for (int64_t k = 0; k < G.ncell; ++k)
    if (Lnat[k] > 0.0) rcell.push_back((int)k);
  if (!rcell.empty() && (rc = copy(c, B + o_rc, rcell.data(), 4 * rcell.size(), "ray tables"))) return rc;
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  T.nbin = nbin;
  T.nview = nview;
  if (rcell_out) *rcell_out = rcell;
  T.rcell = (const int*)(B + o_rc);
  T.bin_nu = (const double*)(B + o_nu);
  T.bin_cursor = (const int*)(B + o_cur);
  T.bin_frac = (const double*)(B + o_frac);
  T.Ebin = lines ? (const double*)(B + o_E) : nullptr;
  T.view = (const double*)(B + o_view);
  T.win_len = (const int*)(B + o_wl);
  Lc_nat = (const double*)(B + o_Lc);
  *n_rays = (int64_t)rcell.size() * nbin * nview;
  return XT_OK;
}

extern "C" int run_transport(xt_ctx* c, const xt_transport_params* p, xt_transport_stats* out) {
  if (!c || !p) return fail(c, XT_EINVAL, "run_transport: null argument");
  if (!c->have_pops) return fail(c, XT_ESTATE, "run_transport: set_populations first");
  cudaSetDevice(c->device);
  const Geometry& G = c->geo;
  const bool rays = p->sampler == XT_SAMPLER_RAYS;
  if (p->sampler != XT_SAMPLER_MC && !rays) return fail(c, XT_EINVAL, "run_transport: sampler");
  if (rays && (p->mode != XT_MODE_ATTEN || p->subdomain_rounds || c->S_groups > 0))
    return fail(c, XT_EINVAL, "run_transport: the RAYS sampler runs in attenuation mode without subdomain "
                              "rounds, with the estimator store on the device");
  if (p->n_packets < 0) return fail(c, XT_EINVAL, "run_transport: n_packets < 0");
  if (p->n_theta < 1 || p->n_phi < 1 || p->spec_nbins < 1 || !(p->spec_lam0_A > 0) || !(p->spec_dlog > 0))
    return fail(c, XT_EINVAL, "run_transport: spectrum grid (n_theta, n_phi, spec_nbins, spec_lam0_A, spec_dlog)");
  if (p->emission != XT_EMIT_BAND && p->emission != XT_EMIT_LINES) return fail(c, XT_EINVAL, "run_transport: emission");
  const bool sph = c->geometry == XT_GEOM_SPHERICAL;
  if (sph && (p->mode != XT_MODE_ATTEN || p->subdomain_rounds || c->S_groups > 0))
    return fail(c, XT_EINVAL, "run_transport: a spherical grid takes attenuation mode, without subdomain "
                              "rounds, with the estimator store on the device");
  RayTables rtab_rays{};
  std::vector<int> ray_cells;          // the emitting cells, natural order (rays)
  const double* ray_Lc = nullptr;
  int64_t n_total = p->n_packets;
  if (rays) {
    if (c->nline < 1) return fail(c, XT_ESTATE, "run_transport: no lines loaded");
    if (p->emission == XT_EMIT_BAND && !c->d_L) return fail(c, XT_ESTATE, "run_transport: band emission needs L_cell in init_grid");
    int rcr = build_rays(c, p, rtab_rays, ray_Lc, &n_total, &ray_cells);
    if (rcr) return rcr;
  }
  const int64_t count_all = p->packet_count < 0 ? n_total - p->packet_begin : p->packet_count;
  if (p->packet_begin < 0 || count_all < 0 || p->packet_begin + count_all > n_total)
    return fail(c, XT_EINVAL, rays ? "run_transport: ray range outside [0, rays)"
                                   : "run_transport: packet range outside [0, n_packets)");
  const bool dom = c->dom.active;
  if (dom && ((rays && !sph) || p->mode != XT_MODE_ATTEN || p->subdomain_rounds || c->S_groups > 0 ||
              p->packet_records))
    return fail(c, XT_EINVAL, "run_transport_domain: attenuation mode with Monte Carlo packets (or rays on "
                              "a spherical grid), the store on the device, no subdomain rounds and no "
                              "packet records");
  int64_t count = count_all;
  if (p->mode != XT_MODE_ATTEN && p->mode != XT_MODE_SCATTER) return fail(c, XT_EINVAL, "run_transport: mode");
  if (p->emission != XT_EMIT_BAND && p->emission != XT_EMIT_LINES) return fail(c, XT_EINVAL, "run_transport: emission");
  if (p->emission == XT_EMIT_BAND && !c->d_L) return fail(c, XT_ESTATE, "run_transport: band emission needs L_cell in init_grid");
  if (p->n_theta < 1 || p->n_phi < 1 || p->spec_nbins < 1 || !(p->spec_lam0_A > 0) || !(p->spec_dlog > 0))
    return fail(c, XT_EINVAL, "run_transport: spectrum grid (n_theta, n_phi, spec_nbins, spec_lam0_A, spec_dlog)");
  if (p->max_events < 1) return fail(c, XT_EINVAL, "run_transport: max_events must be >= 1");
  if (!(p->tau_min > 0) || !(p->e_cut >= 0)) return fail(c, XT_EINVAL, "run_transport: tau_min > 0 and e_cut >= 0 required");
  if (c->nline < 1) return fail(c, XT_ESTATE, "run_transport: no lines loaded");
  const bool pi = c->npi > 0;
  if (pi && p->mode != XT_MODE_ATTEN)
    return fail(c, XT_EINVAL, "run_transport: photoionization is part of the attenuation mode only");
  if (G.ncell >= (int64_t)1 << 31) return fail(c, XT_EINVAL, "run_transport: more than 2^31 cells");
  if (G.nx > 1024 || G.ny > 1024 || G.nz > 1024) return fail(c, XT_EINVAL, "run_transport: more than 1024 cells along an axis");
  int rc;
  // estimator store: on the device, or (host groups) in pinned host memory with
  // one group's slab on the device at a time
  const bool host_store = c->S_groups > 0;
  const int NG = host_store ? c->S_groups : 1;
  if (c->S_compact) {
    // rows only for the cells with populations: the map from this pass's
    // populations; a new map starts from a zeroed store
    std::vector<int> flag(G.ncell);
    {
      int* d_flag = nullptr;
      if ((rc = ensure_scratch(c, G.ncell * sizeof(int)))) return rc;
      d_flag = (int*)c->d_scratch;
      k_row_flags<<<blocks_for(G.ncell * 32, 256, 16), 256, 0, c->stream>>>(G.ncell, c->nlev, c->d_pops, d_flag);
      XT_CUDA(c, cudaGetLastError());
      XT_CUDA(c, cudaMemcpyAsync(flag.data(), d_flag, G.ncell * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      XT_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    std::vector<int> crow(G.ncell);
    int64_t nr = 0;
    for (int64_t r = 0; r < G.ncell; ++r) crow[r] = flag[r] ? (int)nr++ : -1;
    if (crow != c->h_crow) {
      if (p->accumulate && !c->h_crow.empty())
        return fail(c, XT_ESTATE, "run_transport: the cells with populations changed within an accumulating sequence");
      if (!c->d_crow || (int64_t)c->h_crow.size() != G.ncell) {
        if ((rc = alloc(c, (void**)&c->d_crow, G.ncell * sizeof(int), "store row map"))) return rc;
      }
      if ((rc = copy(c, c->d_crow, crow.data(), G.ncell * sizeof(int), "store row map"))) return rc;
      c->h_crow = crow;
      c->n_crow = nr;
      release((void**)&c->d_S);      // reallocated (and zeroed) below for the new map
      c->S_bytes = 0;
    }
  }
  const size_t Sb = (size_t)(c->S_compact ? c->n_crow : G.ncell) * c->nline * sizeof(double);
  const size_t slab_b = Sb / NG;
  if (host_store) {
    if (!c->d_S || c->S_bytes != slab_b) {
      if ((rc = alloc(c, (void**)&c->d_S, slab_b, "estimator slab"))) return rc;
      c->S_bytes = slab_b;
    }
    if (c->h_S_bytes != Sb) {
      if (c->h_S) cudaFreeHost(c->h_S);
      c->h_S = nullptr;
      c->h_S_bytes = 0;
      const cudaError_t e = cudaHostAlloc((void**)&c->h_S, Sb, cudaHostAllocDefault);
      if (e != cudaSuccess) {
        cudaGetLastError();
        c->h_S = nullptr;
        return fail(c, XT_ENOMEM, "run_transport: pinned host estimator store (" + std::to_string(Sb) + " bytes)");
      }
      c->h_S_bytes = Sb;
      c->S_valid.assign(NG, 0);
    }
    if (!p->accumulate) c->S_valid.assign(NG, 0);   // every group starts at zero
  } else if (!c->d_S || c->S_bytes != Sb) {
    if ((rc = alloc(c, (void**)&c->d_S, Sb, "estimator store"))) return rc;
    c->S_bytes = Sb;
    XT_CUDA(c, cudaMemsetAsync(c->d_S, 0, Sb, c->stream));
    c->slotlog_valid = true;        // the store is all zero
    c->slotlog_n = 0;
  }
  if (!c->d_slotlog) {
    const int64_t want = std::min<int64_t>(std::max<int64_t>(4 * count, (int64_t)1 << 22), (int64_t)1 << 29);
    if ((rc = alloc(c, (void**)&c->d_slotlog, (size_t)want * sizeof(int64_t), "slot log"))) return rc;
    c->slotlog_cap = want;
  }
  if (!c->d_seg_n) {
    if ((rc = alloc(c, (void**)&c->d_seg_n, (kLogSegments + 1) * sizeof(int64_t), "log segments"))) return rc;
    XT_CUDA(c, cudaMemsetAsync(c->d_seg_n, 0, (kLogSegments + 1) * sizeof(int64_t), c->stream));
  }
  // spectrum
  const int views = p->n_theta * p->n_phi;
  const size_t spec_b = (size_t)views * p->spec_nbins * sizeof(double);
  if (!c->d_spec || views != c->spec_views || p->spec_nbins != c->spec_bins ||
      p->spec_lam0_A != c->spec_lam0 || p->spec_dlog != c->spec_dlog) {
    if ((rc = alloc(c, (void**)&c->d_spec, spec_b, "spectrum"))) return rc;
    c->spec_views = views; c->spec_bins = p->spec_nbins; c->n_theta = p->n_theta; c->n_phi = p->n_phi;
    c->spec_lam0 = p->spec_lam0_A; c->spec_dlog = p->spec_dlog;
    XT_CUDA(c, cudaMemsetAsync(c->d_spec, 0, spec_b, c->stream));
  }
  // emission: cell luminosities, packet quota, packet energy per cell
  if (!rays && (c->qoff_N != p->n_packets || c->qoff_mode != p->emission)) {
    std::vector<double> Lnat;
    if (c->Lc_n != G.ncell) {
      c->Lc_n = 0;
      if ((rc = alloc(c, (void**)&c->d_Lc, G.ncell * sizeof(double) * 3, "Lc"))) return rc;
      c->Lc_n = G.ncell;
    }
    if (p->emission == XT_EMIT_BAND) {
      Lnat = c->h_L;
    } else {
      const size_t wb = (size_t)G.ncell * c->nline * sizeof(double);
      if (!c->d_wline || c->wline_bytes != wb) {
        if ((rc = alloc(c, (void**)&c->d_wline, wb, "line emission"))) return rc;
        c->wline_bytes = wb;
      }
      k_line_emission<<<blocks_for(G.ncell, 128, 16), 128, 0, c->stream>>>(
          G, (const double2*)c->d_lines, c->d_A, c->nline, c->nlev, c->d_pops, c->d_orig,
          G.dx * G.dy * G.dz, c->d_wline, c->d_Lc);
      XT_CUDA(c, cudaGetLastError());
      Lnat.resize(G.ncell);
      XT_CUDA(c, cudaMemcpyAsync(Lnat.data(), c->d_Lc, G.ncell * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      XT_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    std::vector<int64_t> q;
    packet_quota(Lnat, p->n_packets, q);
    std::vector<double> hv(3 * G.ncell, 0.0);     // [Lc | E per packet | E per packet / h]
    for (int64_t k = 0; k < G.ncell; ++k) {
      hv[k] = Lnat[k];
      const int64_t nq = q[k + 1] - q[k];
      hv[G.ncell + k] = nq > 0 ? Lnat[k] / (double)nq : 0.0;
      hv[2 * G.ncell + k] = hv[G.ncell + k] / kH;
    }
    if ((rc = copy(c, c->d_Lc, hv.data(), hv.size() * sizeof(double), "Lc"))) return rc;
    if (c->qoff_n != (int64_t)q.size()) {
      c->qoff_n = 0;
      if ((rc = alloc(c, (void**)&c->d_qoff, q.size() * sizeof(int64_t), "quota"))) return rc;
      c->qoff_n = (int64_t)q.size();
    }
    if ((rc = copy(c, c->d_qoff, q.data(), q.size() * sizeof(int64_t), "quota"))) return rc;
    c->h_qoff = q;
    // guide of the packet -> cell inversion: the cell of packet j 2^6 for
    // j = 0..(N-1)/2^6 + 1 (ids past N map to the last cell)
    if (p->n_packets > 0) {
      const int64_t nj = ((p->n_packets - 1) >> kQGuideShift) + 2;
      if (c->qguide_n < nj) {
        c->qguide_n = 0;
        if ((rc = alloc(c, (void**)&c->d_qguide, (size_t)nj * sizeof(int), "packet guide"))) return rc;
        c->qguide_n = nj;
      }
      k_q_guide<<<(int)((nj + 255) / 256), 256, 0, c->stream>>>(c->d_qoff, G.ncell, nj, c->d_qguide);
      XT_CUDA(c, cudaGetLastError());
    }
    if (p->emission == XT_EMIT_BAND && c->nline > 0) {
      if (!c->d_nuguide &&
          (rc = alloc(c, (void**)&c->d_nuguide, kNuGuideN * sizeof(int), "band guide"))) return rc;
      const double nu_lo = kC / (c->band_hi_A * 1e-8), nu_hi = kC / (c->band_lo_A * 1e-8);
      k_nu_guide<<<(kNuGuideN + 255) / 256, 256, 0, c->stream>>>(c->d_nu, c->nline, nu_lo,
                                                                  nu_hi - nu_lo, c->d_nuguide);
      XT_CUDA(c, cudaGetLastError());
    }
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->qoff_N = p->n_packets;
    c->qoff_mode = p->emission;
  }
  // packet pool and queues
  const int nsd = c->sx * c->sy * c->sz;
  // a process's domain: its own packets are those of its cells (whole z
  // layers, a contiguous id range of the quota), then the bundle it receives
  int64_t dom_e0 = 0, dom_emit = 0;
  if (dom) {
    const int64_t nxy = (int64_t)G.nx * G.ny;
    int64_t q0, q1;
    if (rays) {
      // the rays of the domain's emitting cells: a contiguous range of the
      // cells' blocks of nbin x nview ids (whole z layers are a contiguous
      // range of natural cell indices)
      const int64_t per_cell = rtab_rays.nbin * rtab_rays.nview;
      const int64_t r0 = std::lower_bound(ray_cells.begin(), ray_cells.end(), (int)(c->dom.z_lo * nxy)) - ray_cells.begin();
      const int64_t r1 = std::lower_bound(ray_cells.begin(), ray_cells.end(), (int)(c->dom.z_hi * nxy)) - ray_cells.begin();
      q0 = r0 * per_cell;
      q1 = r1 * per_cell;
    } else {
      q0 = c->h_qoff[(size_t)(c->dom.z_lo * nxy)];
      q1 = c->h_qoff[(size_t)(c->dom.z_hi * nxy)];
    }
    dom_e0 = std::max<int64_t>(q0, p->packet_begin);
    const int64_t e1 = std::min<int64_t>(q1, p->packet_begin + count_all);
    dom_emit = c->dom.emit && e1 > dom_e0 ? e1 - dom_e0 : 0;
    count = dom_emit + c->dom.n_in;
    if (count > ((int64_t)1 << 27))
      return fail(c, XT_EINVAL, "run_transport_domain: more than 2^27 packets in one call");
  }
  // one chunk of up to 2^27 packets (23 GB of pool): the whole emission of a
  // paper-scale pass runs while the estimator store is being cleared; rays
  // in chunks of whole cells' blocks of ids where a block fits (the spherical
  // walk hands a warp the rays of one cell and viewer only within blocks a
  // launch holds whole)
  int64_t chunk = std::min<int64_t>(std::max<int64_t>(count, 1), (int64_t)1 << 27);
  if (rays && count > chunk) {
    const int64_t per_cell = rtab_rays.nbin * rtab_rays.nview;
    if (per_cell > 0 && per_cell <= chunk) chunk = (chunk / per_cell) * per_cell;
  }
  if ((rc = ensure_buffers(c, chunk, nsd))) return rc;
  const int64_t cap = c->pool_cap;
  if (host_store && c->stream_q_cap < cap) {      // out, carry in, carry out queues
    c->stream_q_cap = 0;
    if ((rc = alloc(c, (void**)&c->d_stream_q, (size_t)cap * 3 * sizeof(int), "group queues"))) return rc;
    c->stream_q_cap = cap;
  }
  int* const I = c->d_pool_i;
  Pool P;
  P.cap = cap; P.f = c->d_pool_f;
  P.cell = I; P.cursor = I + cap; P.events = I + 2 * cap; P.ndraw = I + 3 * cap;
  P.inter = I + 4 * cap; P.pid = c->d_pool_pid;
  int* esc = I + 5 * cap;
  int* qA = I + 6 * cap;
  int* qB = I + 7 * cap;
  int* key = I + 8 * cap;
  unsigned long long* const counters = c->d_counters;
  unsigned* const hist = c->d_hist;

  double* d_rec = nullptr;
  const size_t rec_bytes = (size_t)count * XT_PKT_FIELDS * sizeof(double);
  bool rec_host = false;
  if (p->packet_records) {
    if (is_device_ptr(p->packet_records)) {
      d_rec = p->packet_records;
    } else {
      if ((rc = ensure_scratch(c, rec_bytes))) return rc;
      d_rec = (double*)c->d_scratch;
      rec_host = true;
    }
  }

  // photoionization: per-cell arrays, the cell's suffix sums from the populations
  if (pi) {
    const int64_t rows = G.ncell;
    if (c->pi_rows != rows || c->pi_npi != c->npi) {
      c->pi_rows = 0;
      if ((rc = alloc(c, (void**)&c->d_kappa, (size_t)rows * (c->npi + 1) * sizeof(double), "pi kappa"))) return rc;
      if ((rc = alloc(c, (void**)&c->d_piG, (size_t)rows * (c->npi + 1) * sizeof(double), "pi G"))) return rc;
      if ((rc = alloc(c, (void**)&c->d_piD, (size_t)rows * c->npi * sizeof(double), "pi D"))) return rc;
      if ((rc = alloc(c, (void**)&c->d_piH, (size_t)rows * sizeof(double), "pi H"))) return rc;
      XT_CUDA(c, cudaMemsetAsync(c->d_piG, 0, (size_t)rows * (c->npi + 1) * sizeof(double), c->stream));
      XT_CUDA(c, cudaMemsetAsync(c->d_piD, 0, (size_t)rows * c->npi * sizeof(double), c->stream));
      XT_CUDA(c, cudaMemsetAsync(c->d_piH, 0, (size_t)rows * sizeof(double), c->stream));
      c->pi_rows = rows;
      c->pi_npi = c->npi;
    }
    k_pi_kappa<<<blocks_for(rows, 128, 8), 128, 0, c->stream>>>(rows, c->npi, c->nlev, c->d_pops, c->d_pi_sig,
                                                                c->d_pi_lev, c->d_kappa);
    XT_CUDA(c, cudaGetLastError());
    if (!p->accumulate) {
      XT_CUDA(c, cudaMemsetAsync(c->d_piG, 0, (size_t)rows * (c->npi + 1) * sizeof(double), c->stream));
      XT_CUDA(c, cudaMemsetAsync(c->d_piD, 0, (size_t)rows * c->npi * sizeof(double), c->stream));
      XT_CUDA(c, cudaMemsetAsync(c->d_piH, 0, (size_t)rows * sizeof(double), c->stream));
    }
  }
  c->have_pi = pi;

  int occ = 0;
  if (sph && pi)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace_sph<false, false, true>, 256, 0);
  else if (sph)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace_sph<false>, 256, 0);
  else if (rays && pi)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace<XT_MODE_ATTEN, true, true>, 256, 0);
  else if (rays)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace<XT_MODE_ATTEN, false, true>, 256, 0);
  else if (p->mode == XT_MODE_ATTEN && pi)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace<XT_MODE_ATTEN, true>, 256, 0);
  else if (p->mode == XT_MODE_ATTEN)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace<XT_MODE_ATTEN>, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace<XT_MODE_SCATTER>, 256, 0);
  occ = std::max(occ, 1);
  // trace blocks per launch = touched-slot log segments
  int grid_max = (int)std::min<int64_t>((int64_t)sm_count() * occ, kLogSegments);
  if (p->accumulate && c->log_nseg > 0) grid_max = std::min(grid_max, c->log_nseg);
  XT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  // Clear the estimator store: only the slots the previous passes wrote (the
  // touched-slot log) when the log is complete, else the whole store.
  int kernels_clear = 0;
  if (!p->accumulate) {
    if (host_store) {
      // groups are zeroed when first staged
    } else if (c->slotlog_valid) {
      if (c->slotlog_n > 0) {
        k_unlog<<<c->log_nseg, 256, 0, c->stream>>>(c->d_S, c->d_slotlog, c->d_seg_n, c->log_seglen);
        XT_CUDA(c, cudaGetLastError());
        ++kernels_clear;
      }
    } else {
      XT_CUDA(c, cudaMemsetAsync(c->d_S, 0, Sb, c->stream));
    }
    XT_CUDA(c, cudaMemsetAsync(c->d_seg_n, 0, (kLogSegments + 1) * sizeof(int64_t), c->stream));
    c->slotlog_n = 0;
    c->slotlog_valid = true;
    c->log_nseg = grid_max;
    c->log_seglen = c->slotlog_cap / grid_max;
    XT_CUDA(c, cudaMemsetAsync(c->d_spec, 0, spec_b, c->stream));
    XT_CUDA(c, cudaMemsetAsync(c->d_ledger, 0, LG_N * sizeof(double), c->stream));
  }
  XT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  // per-kernel timing: pairs of events around each launch, summed at the end
  std::vector<std::pair<int, int>> timed;      // (kind, first event index)
  size_t nev = 0;
  auto tick = [&](int kind) -> int {
    if (nev + 2 > c->ev_pool.size()) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      c->ev_pool.push_back(e0);
      c->ev_pool.push_back(e1);
    }
    timed.push_back({kind, (int)nev});
    cudaEventRecord(c->ev_pool[nev], c->stream);
    nev += 2;
    return (int)nev - 1;
  };
  auto tock = [&](int slot) { cudaEventRecord(c->ev_pool[slot], c->stream); };
  int kernels = kernels_clear;

  EmitArgs ea;
  ea.g = G; ea.qoff = c->d_qoff; ea.Lc = c->d_Lc; ea.Epk = c->d_Lc + G.ncell;
  ea.qguide = c->d_qguide;
  // (built with the quota for band emission over a non-empty line list)
  ea.nuguide = (p->emission == XT_EMIT_BAND && c->nline > 0) ? c->d_nuguide : nullptr;
  ea.Eph = c->d_Lc + 2 * G.ncell; ea.cdf = c->d_wline;
  ea.sorted_of = c->d_orig; ea.nu_tab = c->d_nu; ea.nline = c->nline; ea.emission = p->emission;
  ea.seed = p->seed;
  ea.nu_lo = c->band_hi_A > 0 ? kC / (c->band_hi_A * 1e-8) : 0.0;
  ea.nu_hi = c->band_lo_A > 0 ? kC / (c->band_lo_A * 1e-8) : 0.0;
  ea.nu_span = ea.nu_hi - ea.nu_lo;
  {
    // lower wall of every cell index per axis, fma(i, d, -R) as the device computes it
    std::vector<double> wl(G.nx + G.ny + G.nz);
    for (int x = 0; x < G.nx; ++x) wl[x] = std::fma((double)x, G.dx, -G.R);
    for (int y = 0; y < G.ny; ++y) wl[G.nx + y] = std::fma((double)y, G.dy, -G.R);
    for (int z = 0; z < G.nz; ++z) wl[G.nx + G.ny + z] = std::fma((double)z, G.dz, -G.R);
    if (c->wall_n != (int64_t)wl.size()) {
      c->wall_n = 0;
      if ((rc = alloc(c, (void**)&c->d_wall, wl.size() * sizeof(double), "wall table"))) return rc;
      c->wall_n = (int64_t)wl.size();
    }
    if ((rc = copy(c, c->d_wall, wl.data(), wl.size() * sizeof(double), "wall table"))) return rc;
  }
  ea.wall = c->d_wall;
  ea.rays = rays ? 1 : 0;
  ea.ray = rtab_rays;
  if (rays) ea.Lc = ray_Lc;
  ea.e_cut = p->e_cut; ea.pool = P; ea.ledger = c->d_ledger; ea.records = d_rec;
  ea.rec_base = p->packet_begin;
  fixtrig_tables(&ea.trig);

  TraceArgs ta;
  ta.g = G; ta.lines = (const double2*)c->d_lines; ta.nline = c->nline; ta.nlev = c->nlev;
  ta.pops = c->d_pops; ta.S = c->d_S; ta.A = c->d_A; ta.down_off = c->d_down_off;
  ta.down_line = c->d_down_line; ta.Te = c->d_Te; ta.ne = c->d_ne; ta.ups_down = c->d_ups_down;
  ta.glev = c->d_g; ta.pool = P; ta.counter = counters; ta.esc = esc; ta.n_esc = counters + 1;
  ta.n_out = counters + 2; ta.rounds = p->subdomain_rounds ? 1 : 0; ta.seed = p->seed;
  ta.tau_min = p->tau_min; ta.ct = G.ct; ta.inv_ct = G.inv_ct; ta.max_events = p->max_events;
  ta.ledger = c->d_ledger; ta.records = d_rec; ta.rec_base = p->packet_begin;
  fixexp_tables(&ta.fx);
  ta.trig = ea.trig;
  {
    // separable blocked-row offsets: row = RX[ix] + RY[iy] + RZ[iz]
    const int B = G.bx * G.by * G.bz;
    std::vector<int> rt(G.nx + G.ny + G.nz);
    for (int x = 0; x < G.nx; ++x) rt[x] = (x / G.bx) * B + x % G.bx;
    for (int y = 0; y < G.ny; ++y) rt[G.nx + y] = (y / G.by) * G.sx * B + (y % G.by) * G.bx;
    for (int z = 0; z < G.nz; ++z)
      rt[G.nx + G.ny + z] = (z / G.bz) * G.sy * G.sx * B + (z % G.bz) * G.by * G.bx;
    if (c->rtab_n != (int64_t)rt.size()) {
      c->rtab_n = 0;
      if ((rc = alloc(c, (void**)&c->d_rtab, rt.size() * sizeof(int), "row tables"))) return rc;
      c->rtab_n = (int64_t)rt.size();
    }
    if ((rc = copy(c, c->d_rtab, rt.data(), rt.size() * sizeof(int), "row tables"))) return rc;
  }
  ta.rtab = c->d_rtab;
  ta.slotlog = c->d_slotlog;
  ta.seg_n = c->d_seg_n;
  if (c->log_nseg <= 0) {         // first pass of an accumulating sequence
    c->log_nseg = grid_max;
    c->log_seglen = c->slotlog_cap / grid_max;
  }
  ta.seg_len = c->log_seglen;
  ta.log_overflow = (unsigned long long*)(c->d_seg_n + kLogSegments);
  // attenuation without subdomain rounds: the trace kernel emits its packets
  ta.fused = (p->mode == XT_MODE_ATTEN && !p->subdomain_rounds && !host_store && !dom) ? 1 : 0;
  ta.row0 = 0;
  ta.grp_nz = G.nz / NG;
  const bool wr = (p->flags & XT_FLAG_WARP_REDUCE) != 0 && p->mode == XT_MODE_ATTEN && !pi && !rays;
  const bool staged = rays && !pi && (p->flags & XT_FLAG_RAYS_STAGED) != 0;
  if (staged) {
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
      XT_CUDA(c, cudaFuncSetAttribute(k_trace_rays_staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kStageLines * 32));
      attr_set[dev] = true;
    }
    XT_CUDA(c, cudaMemsetAsync(counters + 5, 0, sizeof(unsigned long long), c->stream));
  }
  ta.npi = pi ? c->npi : 0;
  ta.crow = c->S_compact ? c->d_crow : nullptr;
  ta.pi_nuth = c->d_pi_nuth; ta.pi_sig = c->d_pi_sig; ta.pi_lev = c->d_pi_lev;
  ta.kappa = c->d_kappa; ta.piG = c->d_piG; ta.piD = c->d_piD; ta.piH = c->d_piH;
  if (host_store) ta.rounds = 2;

  EscArgs xa;
  xa.pool = P; xa.esc = esc; xa.spec = c->d_spec; xa.n_theta = p->n_theta; xa.n_phi = p->n_phi;
  xa.nbins = p->spec_nbins; xa.lam0 = p->spec_lam0_A; xa.log1p_dlog = std::log1p(p->spec_dlog);
  xa.ledger = c->d_ledger; xa.records = d_rec; xa.rec_base = p->packet_begin;

  const int max_rounds = 1 << 20;
  int64_t rounds = 0, queued_total = 0;
  if (dom) {
    // one launch: the domain's own packets and the received bundle, traced
    // until they end or leave the domain; those are written out as a bundle
    int sl;
    ea.p_begin = dom_e0;
    ea.n = dom_emit;
    ta.em = ea;                        // (the spherical walk emits the domain's packets itself)
    if (dom_emit > 0 && !sph) {
      sl = tick(0);
      k_emit<<<blocks_for(dom_emit, 256, 16), 256, 0, c->stream>>>(ea);
      XT_CUDA(c, cudaGetLastError());
      tock(sl);
      ++kernels;
    }
    const int64_t n_in = c->dom.n_in;
    const size_t in_b = (size_t)n_in * XT_BUNDLE_FIELDS * sizeof(double);
    if (n_in > 0) {
      const double* src = c->dom.in;
      if (!is_device_ptr(src)) {
        if ((rc = ensure_scratch(c, in_b))) return rc;
        if ((rc = copy(c, c->d_scratch, src, in_b, "bundle in"))) return rc;
        src = (const double*)c->d_scratch;
      }
      XT_CUDA(c, cudaMemsetAsync(counters + 6, 0, sizeof(unsigned long long), c->stream));
      k_bundle_in<<<blocks_for(n_in, 256, 8), 256, 0, c->stream>>>(P, src, n_in, dom_emit, G, c->nline,
                                                                    counters + 6);
      XT_CUDA(c, cudaGetLastError());
      ++kernels;
      unsigned long long bad = 0;
      XT_CUDA(c, cudaMemcpyAsync(&bad, counters + 6, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
      XT_CUDA(c, cudaStreamSynchronize(c->stream));
      if (bad > 0)
        return fail(c, XT_EINVAL, "run_transport_domain: " + std::to_string(bad) +
                                      " bundle_in entries with a cell outside the grid or a line cursor "
                                      "outside [0, nline]");
    }
    c->dom.n_out = 0;
    if (count > 0) {
      XT_CUDA(c, cudaMemsetAsync(counters, 0, 3 * sizeof(unsigned long long), c->stream));
      ta.rounds = 3;
      ta.dom_zlo = c->dom.z_lo;
      ta.dom_zhi = c->dom.z_hi;
      ta.list = nullptr;
      ta.n_list = count;
      ta.out = qA;
      const int grid = (int)std::min<int64_t>(grid_max, (count + 255) / 256);
      sl = tick(1);
      if (sph && rays && pi) k_trace_sph<true, true, true><<<grid, 256, 0, c->stream>>>(ta);
      else if (sph && rays) k_trace_sph<true, true><<<grid, 256, 0, c->stream>>>(ta);
      else if (sph && pi) k_trace_sph<true, false, true><<<grid, 256, 0, c->stream>>>(ta);
      else if (sph) k_trace_sph<true><<<grid, 256, 0, c->stream>>>(ta);
      else if (pi) k_trace<XT_MODE_ATTEN, true><<<grid, 256, 0, c->stream>>>(ta);
      else if (wr) k_trace<XT_MODE_ATTEN, false, false, true><<<grid, 256, 0, c->stream>>>(ta);
      else k_trace<XT_MODE_ATTEN><<<grid, 256, 0, c->stream>>>(ta);
      XT_CUDA(c, cudaGetLastError());
      tock(sl);
      ++kernels;
      unsigned long long cnt[4];
      XT_CUDA(c, cudaMemcpyAsync(cnt, counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
      XT_CUDA(c, cudaStreamSynchronize(c->stream));
      ++rounds;
      if (cnt[1] > 0) {
        xa.n_esc = (int64_t)cnt[1];
        sl = tick(2);
        k_escape<<<blocks_for(xa.n_esc, 256, 8), 256, 0, c->stream>>>(xa);
        XT_CUDA(c, cudaGetLastError());
        tock(sl);
        ++kernels;
      }
      const int64_t nq = (int64_t)cnt[2];
      c->dom.n_out = nq;
      queued_total = nq;
      const int64_t nw = std::min<int64_t>(nq, c->dom.out_cap);
      if (nw > 0 && c->dom.out) {
        rc = deliver(c, c->dom.out, (size_t)nw * XT_BUNDLE_FIELDS * sizeof(double), [&](void* d) {
          k_bundle_out<<<blocks_for(nw, 256, 8), 256, 0, c->stream>>>(P, qA, nw, (double*)d);
        });
        if (rc) return rc;
        ++kernels;
      }
    }
  }
  for (int64_t off = 0; !dom && off < count; off += chunk) {
    const int64_t n = std::min(chunk, count - off);
    ea.p_begin = p->packet_begin + off;
    ea.n = n;
    ta.em = ea;
    int sl;
    if (!ta.fused) {
      sl = tick(0);
      k_emit<<<blocks_for(n, 256, 16), 256, 0, c->stream>>>(ea);
      XT_CUDA(c, cudaGetLastError());
      tock(sl);
      ++kernels;
    }

    if (host_store) {
      // streamed groups, in sweeps over the groups alternately up and down in
      // z: each group's slab is staged (from host memory, or zeros on its
      // first visit in the pass), its pending packets traced, then the packets
      // that entered it from the previous group of the sweep; packets leaving
      // into the next group of the sweep follow it, the others wait for the
      // next sweep (a straight path needs at most two sweeps).  The slab is
      // written back after each visit.
      const int64_t rows_g = G.ncell / NG;
      const size_t slab_n = (size_t)rows_g * c->nline;
      int* const out_tmp = c->d_stream_q;
      int* carry_in = c->d_stream_q + cap;
      int* carry_out = c->d_stream_q + 2 * cap;
      k_iota<<<blocks_for(n, 256, 8), 256, 0, c->stream>>>(qA, n);
      XT_CUDA(c, cudaGetLastError());
      ++kernels;
      int64_t n_pend = n;
      int dir = 1;
      for (int sweep = 0; n_pend > 0; ++sweep, dir = -dir) {
        if (sweep >= max_rounds) return fail(c, XT_ETIMEOUT, "run_transport: streamed sweeps did not drain");
        // pending packets (in qA) sorted by group into qB; qA then collects the next sweep's
        XT_CUDA(c, cudaMemsetAsync(hist, 0, (size_t)NG * sizeof(unsigned), c->stream));
        k_grp_hist<<<blocks_for(n_pend, 256, 8), 256, 0, c->stream>>>(P.cell, qA, n_pend, ta.grp_nz, key, hist);
        XT_CUDA(c, cudaGetLastError());
        std::vector<unsigned> h(NG), start(NG);
        XT_CUDA(c, cudaMemcpyAsync(h.data(), hist, NG * sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
        XT_CUDA(c, cudaStreamSynchronize(c->stream));
        unsigned run = 0;
        for (int g = 0; g < NG; ++g) { start[g] = run; run += h[g]; }
        XT_CUDA(c, cudaMemcpyAsync(hist + NG, start.data(), NG * sizeof(unsigned), cudaMemcpyHostToDevice, c->stream));
        k_sd_scatter<<<blocks_for(n_pend, 256, 8), 256, 0, c->stream>>>(qA, key, n_pend, hist + NG, qB);
        XT_CUDA(c, cudaGetLastError());
        kernels += 2;
        XT_CUDA(c, cudaMemsetAsync(counters + 3, 0, 2 * sizeof(unsigned long long), c->stream));  // carry, pend
        int64_t n_carry = 0;
        for (int k = 0; k < NG; ++k) {
          const int g = dir > 0 ? k : NG - 1 - k;
          if (h[g] == 0 && n_carry == 0) continue;
          double* hs = c->h_S + (size_t)g * slab_n;
          if (c->S_valid[g]) XT_CUDA(c, cudaMemcpyAsync(c->d_S, hs, slab_b, cudaMemcpyHostToDevice, c->stream));
          else XT_CUDA(c, cudaMemsetAsync(c->d_S, 0, slab_b, c->stream));
          ta.row0 = (int64_t)g * rows_g;
          XT_CUDA(c, cudaMemsetAsync(counters + 3, 0, sizeof(unsigned long long), c->stream));  // carry out
          const int* lists[2] = {qB + start[g], carry_in};
          const int64_t lens[2] = {(int64_t)h[g], n_carry};
          for (int part = 0; part < 2; ++part) {
            if (lens[part] == 0) continue;
            XT_CUDA(c, cudaMemsetAsync(counters, 0, 3 * sizeof(unsigned long long), c->stream));
            ta.list = lists[part];
            ta.n_list = lens[part];
            ta.out = out_tmp;
            const int grid = (int)std::min<int64_t>(grid_max, (lens[part] + 255) / 256);
            sl = tick(1);
            if (pi) k_trace<XT_MODE_ATTEN, true><<<grid, 256, 0, c->stream>>>(ta);
            else if (wr) k_trace<XT_MODE_ATTEN, false, false, true><<<grid, 256, 0, c->stream>>>(ta);
            else if (p->mode == XT_MODE_ATTEN) k_trace<XT_MODE_ATTEN><<<grid, 256, 0, c->stream>>>(ta);
            else k_trace<XT_MODE_SCATTER><<<grid, 256, 0, c->stream>>>(ta);
            XT_CUDA(c, cudaGetLastError());
            tock(sl);
            ++kernels;
            unsigned long long cnt[4];
            XT_CUDA(c, cudaMemcpyAsync(cnt, counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
            XT_CUDA(c, cudaStreamSynchronize(c->stream));
            ++rounds;
            if (cnt[1] > 0) {
              xa.n_esc = (int64_t)cnt[1];
              sl = tick(2);
              k_escape<<<blocks_for(xa.n_esc, 256, 8), 256, 0, c->stream>>>(xa);
              XT_CUDA(c, cudaGetLastError());
              tock(sl);
              ++kernels;
            }
            if (cnt[2] > 0) {
              queued_total += (int64_t)cnt[2];
              k_grp_split<<<blocks_for((int64_t)cnt[2], 256, 8), 256, 0, c->stream>>>(
                  P.cell, out_tmp, (int64_t)cnt[2], ta.grp_nz, g + dir, carry_out, counters + 3, qA, counters + 4);
              XT_CUDA(c, cudaGetLastError());
              ++kernels;
            }
          }
          XT_CUDA(c, cudaMemcpyAsync(hs, c->d_S, slab_b, cudaMemcpyDeviceToHost, c->stream));
          c->S_valid[g] = 1;
          unsigned long long nco = 0;
          XT_CUDA(c, cudaMemcpyAsync(&nco, counters + 3, sizeof(nco), cudaMemcpyDeviceToHost, c->stream));
          XT_CUDA(c, cudaStreamSynchronize(c->stream));
          std::swap(carry_in, carry_out);
          n_carry = (int64_t)nco;
        }
        unsigned long long np = 0;
        XT_CUDA(c, cudaMemcpyAsync(&np, counters + 4, sizeof(np), cudaMemcpyDeviceToHost, c->stream));
        XT_CUDA(c, cudaStreamSynchronize(c->stream));
        if (n_carry > 0)      // (a straight path leaves the grid past the last group)
          XT_CUDA(c, cudaMemcpyAsync(qA + np, carry_in, (size_t)n_carry * sizeof(int), cudaMemcpyDeviceToDevice, c->stream));
        n_pend = (int64_t)np + n_carry;
        ta.row0 = 0;
      }
      XT_CUDA(c, cudaStreamSynchronize(c->stream));
      continue;
    }
    const int* list = nullptr;
    int64_t n_list = n;
    for (int round = 0; n_list > 0; ++round) {
      if (round >= max_rounds) return fail(c, XT_ETIMEOUT, "run_transport: subdomain rounds did not drain");
      XT_CUDA(c, cudaMemsetAsync(counters, 0, 3 * sizeof(unsigned long long), c->stream));
      ta.list = list;
      ta.n_list = n_list;
      ta.out = (list == qA) ? qB : qA;
      const int grid = (int)std::min<int64_t>(grid_max, (n_list + 255) / 256);
      sl = tick(1);
      if (sph && rays && pi) k_trace_sph<false, true, true><<<grid, 256, 0, c->stream>>>(ta);
      else if (sph && rays) k_trace_sph<false, true><<<grid, 256, 0, c->stream>>>(ta);
      else if (sph && pi) k_trace_sph<false, false, true><<<grid, 256, 0, c->stream>>>(ta);
      else if (sph) k_trace_sph<false><<<grid, 256, 0, c->stream>>>(ta);
      else if (rays && pi) k_trace<XT_MODE_ATTEN, true, true><<<grid, 256, 0, c->stream>>>(ta);
      else if (rays && staged) {
        const int64_t gpb = std::max<int64_t>(1, kStageRays / ea.ray.nview);
        const int64_t per_cell = ea.ray.nview * ea.ray.nbin;
        const int64_t batches = ((ea.p_begin + n + per_cell - 1) / per_cell - ea.p_begin / per_cell) *
                                ((ea.ray.nbin + gpb - 1) / gpb);
        const int sgrid = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)grid_max, (int64_t)sm_count() * 3, batches}));
        k_trace_rays_staged<<<sgrid, 256, kStageLines * 32, c->stream>>>(ta, ea.ray.win_len, ea.p_begin + n,
                                                                           counters + 5);
      } else if (rays) k_trace<XT_MODE_ATTEN, false, true><<<grid, 256, 0, c->stream>>>(ta);
      else if (pi) k_trace<XT_MODE_ATTEN, true><<<grid, 256, 0, c->stream>>>(ta);
      else if (wr) k_trace<XT_MODE_ATTEN, false, false, true><<<grid, 256, 0, c->stream>>>(ta);
      else if (p->mode == XT_MODE_ATTEN) k_trace<XT_MODE_ATTEN><<<grid, 256, 0, c->stream>>>(ta);
      else k_trace<XT_MODE_SCATTER><<<grid, 256, 0, c->stream>>>(ta);
      XT_CUDA(c, cudaGetLastError());
      tock(sl);
      ++kernels;
      unsigned long long cnt[4];
      XT_CUDA(c, cudaMemcpyAsync(cnt, counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
      XT_CUDA(c, cudaStreamSynchronize(c->stream));
      ++rounds;
      if (cnt[1] > 0) {
        xa.n_esc = (int64_t)cnt[1];
        sl = tick(2);
        k_escape<<<blocks_for(xa.n_esc, 256, 8), 256, 0, c->stream>>>(xa);
        XT_CUDA(c, cudaGetLastError());
        tock(sl);
        ++kernels;
      }
      n_list = (int64_t)cnt[2];
      queued_total += n_list;
      if (n_list > 0) {
        // bundle the queued packets by destination subdomain (counting sort)
        int* q = ta.out;
        int* sorted = (q == qA) ? qB : qA;
        XT_CUDA(c, cudaMemsetAsync(hist, 0, (size_t)nsd * sizeof(unsigned), c->stream));
        kernels += 2;
        k_sd_hist<<<blocks_for(n_list, 256, 8), 256, 0, c->stream>>>(G, P.cell, q, n_list, key, hist);
        XT_CUDA(c, cudaGetLastError());
        std::vector<unsigned> h(nsd);
        XT_CUDA(c, cudaMemcpyAsync(h.data(), hist, nsd * sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
        XT_CUDA(c, cudaStreamSynchronize(c->stream));
        std::vector<unsigned> start(nsd);
        unsigned run = 0;
        for (int s = 0; s < nsd; ++s) { start[s] = run; run += h[s]; }
        XT_CUDA(c, cudaMemcpyAsync(hist + nsd, start.data(), nsd * sizeof(unsigned), cudaMemcpyHostToDevice, c->stream));
        k_sd_scatter<<<blocks_for(n_list, 256, 8), 256, 0, c->stream>>>(q, key, n_list, hist + nsd, sorted);
        XT_CUDA(c, cudaGetLastError());
        list = sorted;
      }
    }
  }
  XT_CUDA(c, cudaEventRecord(c->ev2, c->stream));
  double led[LG_N];
  XT_CUDA(c, cudaMemcpyAsync(led, c->d_ledger, sizeof(led), cudaMemcpyDeviceToHost, c->stream));
  unsigned long long nover = 0;
  XT_CUDA(c, cudaMemcpyAsync(&nover, c->d_seg_n + kLogSegments, sizeof(nover), cudaMemcpyDeviceToHost, c->stream));
  if (rec_host) XT_CUDA(c, cudaMemcpyAsync(p->packet_records, d_rec, rec_bytes, cudaMemcpyDeviceToHost, c->stream));
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  c->have_S = true;
  c->slotlog_n += (int64_t)led[LG_EVENTS] + 1;      // nonzero once anything was logged
  if (nover > 0 && !host_store) {
    // a segment overflowed: the next pass clears the whole store; grow the log
    c->slotlog_valid = false;
    const int64_t want = std::min<int64_t>(4 * c->slotlog_cap, (int64_t)1 << 31);
    if (want > c->slotlog_cap && alloc(c, (void**)&c->d_slotlog, (size_t)want * sizeof(int64_t), "slot log") == XT_OK)
      c->slotlog_cap = want;
    else if (!c->d_slotlog)
      c->slotlog_cap = 0;
    c->log_nseg = 0;
    c->err.clear();
  }
  if (out) {
    double* o = &out->emitted_N;
    for (int k = 0; k < LG_STATS; ++k) o[k] = led[k];
    out->photoionized_N = led[LG_PI_N];
    out->photoionized_E = kH * led[LG_PI_E];
    out->rays = rays ? (double)n_total : 0.0;
    float ms_all = 0, ms_clear = 0;
    cudaEventElapsedTime(&ms_all, c->ev0, c->ev2);
    cudaEventElapsedTime(&ms_clear, c->ev0, c->ev1);
    out->zero_ms = ms_clear;
    out->transport_ms = ms_all;
    out->rounds = (double)rounds;
    out->queued = (double)queued_total;
    double kind_ms[3] = {0, 0, 0};
    for (auto& tp : timed) {
      float ms = 0;
      cudaEventElapsedTime(&ms, c->ev_pool[tp.second], c->ev_pool[tp.second + 1]);
      kind_ms[tp.first] += ms;
    }
    out->emit_ms = kind_ms[0];
    out->trace_ms = kind_ms[1];
    out->escape_ms = kind_ms[2];
    out->kernels = kernels;
  }
  if (staged) {
    unsigned long long stage_err = 0;
    XT_CUDA(c, cudaMemcpyAsync(&stage_err, counters + 5, sizeof(stage_err), cudaMemcpyDeviceToHost, c->stream));
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (stage_err) return fail(c, XT_ETIMEOUT, "run_transport: a staged line window did not arrive in time");
  }
  if (led[LG_GUARD] > 0)
    return fail(c, XT_ETIMEOUT, "run_transport: " + std::to_string((long long)led[LG_GUARD]) +
                                    (sph ? " packets hit max_events or the walk's face limit" : " packets hit max_events"));
  return XT_OK;
}


extern "C" int run_transport_domain(xt_ctx* c, const xt_transport_params* p, int32_t z_lo, int32_t z_hi,
                                    int32_t emit, const double* bundle_in, int64_t n_in, double* bundle_out,
                                    int64_t out_cap, int64_t* n_out, xt_transport_stats* out) {
  if (!c || !p || !n_out) return fail(c, XT_EINVAL, "run_transport_domain: null argument");
  if (!c->have_grid) return fail(c, XT_ESTATE, "run_transport_domain: init_grid first");
  if (z_lo < 0 || z_hi > c->geo.nz || z_lo >= z_hi)
    return fail(c, XT_EINVAL, "run_transport_domain: need 0 <= z_lo < z_hi <= nz");
  if (n_in < 0 || (n_in > 0 && !bundle_in) || out_cap < 0 || (out_cap > 0 && !bundle_out))
    return fail(c, XT_EINVAL, "run_transport_domain: bundle arguments");
  c->dom.active = true;
  c->dom.z_lo = z_lo; c->dom.z_hi = z_hi; c->dom.emit = emit ? 1 : 0;
  c->dom.in = bundle_in; c->dom.n_in = n_in; c->dom.out = bundle_out; c->dom.out_cap = out_cap;
  c->dom.n_out = 0;
  const int rc = run_transport(c, p, out);
  c->dom.active = false;
  *n_out = c->dom.n_out;
  if (rc) return rc;
  if (c->dom.n_out > out_cap)
    return fail(c, XT_EINVAL, "run_transport_domain: " + std::to_string(c->dom.n_out) +
                                  " packets leave the domain, bundle_out holds " + std::to_string(out_cap));
  return XT_OK;
}

// ============================================================================
// Transport without device allocation.
//
// Some callers cannot call cudaMalloc: programs whose device memory is carved
// up once at start-up by another framework's allocator, or embedders that must
// keep a fixed device-memory budget.  run_transport_noalloc gives them one
// attenuation-mode transport pass that allocates nothing: its working memory
// (line table, packet quota, packet pool, escape list, counters, ledger) lives
// in the file-scope array below, of fixed size, which every GPU that loads the
// library holds until the process exits.  The kernels are the ones
// run_transport launches; only where their scratch lives differs.
// ============================================================================
namespace xt {

constexpr size_t kNaScratch = (size_t)XT_NOALLOC_SCRATCH_BYTES;
constexpr int64_t kNaChunk = XT_NOALLOC_CHUNK;
constexpr int kNaMaxCells = XT_NOALLOC_MAX_CELLS;
constexpr int kNaMaxLines = XT_NOALLOC_MAX_LINES;
constexpr int kNaSegs = 4096;

// byte offsets of the parts of the scratch array (all 256-byte aligned)
constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kNaLines = 0;                                               // 4 doubles per line
constexpr size_t kNaNu = na_align(kNaLines + 32ull * kNaMaxLines);           // sorted nu
constexpr size_t kNaSorted = na_align(kNaNu + 8ull * kNaMaxLines);           // caller -> sorted
constexpr size_t kNaQoff = na_align(kNaSorted + 4ull * kNaMaxLines);         // [ncell+1]
constexpr size_t kNaCellE = na_align(kNaQoff + 8ull * (kNaMaxCells + 1));    // Lc | Epk | Eph
constexpr size_t kNaRtab = na_align(kNaCellE + 24ull * kNaMaxCells);         // [nx+ny+nz]
constexpr size_t kNaCount = na_align(kNaRtab + 4ull * 3 * 1024);             // 8 counters
constexpr size_t kNaLedger = na_align(kNaCount + 64);                        // [LG_N]
constexpr size_t kNaSegN = na_align(kNaLedger + 8ull * LG_N);                // [kNaSegs + 1]
constexpr size_t kNaLog = na_align(kNaSegN + 8ull * (kNaSegs + 1));          // 256 B dummy
constexpr size_t kNaPoolF = na_align(kNaLog + 256);                          // NF doubles x chunk
constexpr size_t kNaPoolI = na_align(kNaPoolF + 8ull * NF * kNaChunk);       // 9 ints x chunk
constexpr size_t kNaPoolP = na_align(kNaPoolI + 4ull * 9 * kNaChunk);        // packet ids
constexpr size_t kNaEnd = na_align(kNaPoolP + 8ull * kNaChunk);
static_assert(kNaEnd <= kNaScratch, "no-allocation scratch layout exceeds its array");

static __device__ __align__(256) unsigned char g_na_scratch[kNaScratch];
static void* g_na_ptr[64];            // device address of g_na_scratch, per device

// Device address of the scratch array on the current device.  Looked up once
// per device with that device current (host code must not use the symbol's
// name as an address).
static int na_scratch(void** out, std::string& err) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    err = "run_transport_noalloc: no current CUDA device (or device index >= 64)";
    return XT_ECUDA;
  }
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("run_transport_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return XT_ECUDA;
    }
    g_na_ptr[dev] = p;
  }
  *out = g_na_ptr[dev];
  return XT_OK;
}

// Estimators of one row from descending-frequency order to the caller's line
// order, and from net photons to photons divided by f_corr (in place; the row
// is staged in shared memory).
__global__ void k_na_finish(double* __restrict__ S, const double* __restrict__ pops,
                            const double* __restrict__ lines, const int* __restrict__ sorted_of,
                            int nline, int nlev) {
  extern __shared__ double srow[];
  double* row = S + (int64_t)blockIdx.x * nline;
  const double* pc = pops + (int64_t)blockIdx.x * nlev;
  for (int s = threadIdx.x; s < nline; s += blockDim.x) srow[s] = row[s];
  __syncthreads();
  for (int l = threadIdx.x; l < nline; l += blockDim.x) {
    const int s = sorted_of[l];
    const double v = srow[s];
    double out = 0.0;
    if (v != 0.0) {
      const double* L = lines + 4 * (int64_t)s;
      const int64_t lu = __double_as_longlong(L[3]);
      const double nl = pc[(int)(lu & 0xFFFFFFFF)], nu = pc[(int)(lu >> 32)];
      out = v * nl / (nl - L[2] * nu);
    }
    row[l] = out;
  }
}

// host staging, fixed size (no heap allocation on this path)
static double h_na_L[kNaMaxCells], h_na_cellE[3 * kNaMaxCells];
static int64_t h_na_q[kNaMaxCells + 1];
static double h_na_frac[kNaMaxCells];
static int64_t h_na_qord[kNaMaxCells];
static int h_na_ord[kNaMaxLines];
static double h_na_lam[kNaMaxLines], h_na_f[kNaMaxLines], h_na_nu[kNaMaxLines];
static int h_na_lo[kNaMaxLines], h_na_up[kNaMaxLines], h_na_sorted[kNaMaxLines];
static double h_na_g[1 << 16];
static double h_na_lines[4 * kNaMaxLines], h_na_nus[kNaMaxLines];
static int h_na_rtab[3 * 1024];

}  // namespace xt

extern "C" int run_transport_noalloc(const xt_noalloc_transport* a, void* cuda_stream,
                                     xt_transport_stats* out, char* errbuf, size_t errlen) {
  using namespace xt;
  std::string err;
  auto bad = [&](int code, const std::string& m) {
    if (errbuf && errlen) { std::snprintf(errbuf, errlen, "%s", m.c_str()); }
    return code;
  };
  if (!a) return bad(XT_EINVAL, "run_transport_noalloc: null argument");
  const int64_t ncell = (int64_t)a->nx * a->ny * a->nz;
  if (a->nx < 1 || a->ny < 1 || a->nz < 1 || a->nx > 1024 || a->ny > 1024 || a->nz > 1024)
    return bad(XT_EINVAL, "run_transport_noalloc: nx, ny, nz must be in 1..1024");
  if (ncell > kNaMaxCells)
    return bad(XT_EINVAL, "run_transport_noalloc: " + std::to_string(ncell) + " cells exceed the maximum " +
                              std::to_string(kNaMaxCells));
  if (a->nline < 1 || a->nline > kNaMaxLines)
    return bad(XT_EINVAL, "run_transport_noalloc: nline must be in 1.." + std::to_string(kNaMaxLines));
  if (a->nlev < 2 || a->nlev > (1 << 16))
    return bad(XT_EINVAL, "run_transport_noalloc: nlev must be in 2..65536");
  if (!a->L_cell || !a->g_level || !a->lo || !a->up || !a->lambda_A || !a->f_lu || !a->pops || !a->S || !a->spec)
    return bad(XT_EINVAL, "run_transport_noalloc: every array argument is required");
  if (!is_device_ptr(a->pops) || !is_device_ptr(a->S) || !is_device_ptr(a->spec))
    return bad(XT_EINVAL, "run_transport_noalloc: pops, S and spec must be device memory");
  if (a->n_packets < 0 || !(a->v_max > 0) || !(a->t > 0) || !(a->band_hi_A > a->band_lo_A) || !(a->band_lo_A > 0))
    return bad(XT_EINVAL, "run_transport_noalloc: n_packets >= 0, v_max > 0, t > 0, 0 < band_lo_A < band_hi_A");
  if (a->n_theta < 1 || a->n_phi < 1 || a->spec_nbins < 1 || !(a->spec_lam0_A > 0) || !(a->spec_dlog > 0) ||
      !(a->tau_min > 0) || !(a->e_cut >= 0) || a->max_events < 1)
    return bad(XT_EINVAL, "run_transport_noalloc: spectrum grid, tau_min, e_cut or max_events");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  void* base = nullptr;
  if (int rc = na_scratch(&base, err)) return bad(rc, err);
  unsigned char* B = (unsigned char*)base;
  const int nl = a->nline, nlev = a->nlev;
#define NA_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return bad(XT_ECUDA, std::string("run_transport_noalloc: ") + #call + ": " + cudaGetErrorString(e_)); \
  } while (0)
  // ---- inputs to host staging (the caller's arrays may be host or device memory)
  NA_CUDA(cudaMemcpyAsync(h_na_L, a->L_cell, ncell * sizeof(double), cudaMemcpyDefault, st));
  NA_CUDA(cudaMemcpyAsync(h_na_g, a->g_level, nlev * sizeof(double), cudaMemcpyDefault, st));
  NA_CUDA(cudaMemcpyAsync(h_na_lo, a->lo, nl * sizeof(int), cudaMemcpyDefault, st));
  NA_CUDA(cudaMemcpyAsync(h_na_up, a->up, nl * sizeof(int), cudaMemcpyDefault, st));
  NA_CUDA(cudaMemcpyAsync(h_na_lam, a->lambda_A, nl * sizeof(double), cudaMemcpyDefault, st));
  NA_CUDA(cudaMemcpyAsync(h_na_f, a->f_lu, nl * sizeof(double), cudaMemcpyDefault, st));
  NA_CUDA(cudaStreamSynchronize(st));
  for (int l = 0; l < nl; ++l) {
    if (h_na_lo[l] < 0 || h_na_up[l] >= nlev || h_na_lo[l] >= h_na_up[l] || !(h_na_lam[l] > 0) || !(h_na_f[l] > 0))
      return bad(XT_EINVAL, "run_transport_noalloc: line " + std::to_string(l) + " needs 0 <= lo < up < nlev, lambda > 0, f > 0");
    h_na_nu[l] = kC / (h_na_lam[l] * 1e-8);
  }
  for (int64_t k = 0; k < ncell; ++k)
    if (!(h_na_L[k] >= 0.0) || !std::isfinite(h_na_L[k]))
      return bad(XT_EINVAL, "run_transport_noalloc: L_cell must be finite and >= 0");
  // ---- line table in descending frequency (ties: ascending caller index)
  for (int l = 0; l < nl; ++l) h_na_ord[l] = l;
  std::sort(h_na_ord, h_na_ord + nl, [](int x, int y) {
    return h_na_nu[x] > h_na_nu[y] || (h_na_nu[x] == h_na_nu[y] && x < y);
  });
  const double pie2mc = kPi * kE * kE / (kMe * kC);
  for (int s = 0; s < nl; ++s) {
    const int l = h_na_ord[s];
    h_na_sorted[l] = s;
    h_na_nus[s] = h_na_nu[l];
    h_na_lines[4 * s] = h_na_nu[l];
    h_na_lines[4 * s + 1] = pie2mc * h_na_f[l] * (h_na_lam[l] * 1e-8) * a->t;
    h_na_lines[4 * s + 2] = h_na_g[h_na_lo[l]] / h_na_g[h_na_up[l]];
    const int64_t lu = (int64_t)(uint32_t)h_na_lo[l] | ((int64_t)h_na_up[l] << 32);
    std::memcpy(&h_na_lines[4 * s + 3], &lu, sizeof(lu));
  }
  // ---- packet quota by largest remainder (the routine run_transport uses, on
  // the fixed staging buffers), packet energies
  packet_quota(h_na_L, ncell, a->n_packets, h_na_q, h_na_frac, h_na_qord);
  for (int64_t k = 0; k < ncell; ++k) {
    const int64_t nq = h_na_q[k + 1] - h_na_q[k];
    h_na_cellE[k] = h_na_L[k];
    h_na_cellE[ncell + k] = nq > 0 ? h_na_L[k] / (double)nq : 0.0;
    h_na_cellE[2 * ncell + k] = h_na_cellE[ncell + k] / kH;
  }
  for (int x = 0; x < a->nx; ++x) h_na_rtab[x] = x;
  for (int y = 0; y < a->ny; ++y) h_na_rtab[a->nx + y] = y * a->nx;
  for (int z = 0; z < a->nz; ++z) h_na_rtab[a->nx + a->ny + z] = z * a->nx * a->ny;
  // ---- staged tables into the scratch array; outputs and counters cleared
  NA_CUDA(cudaMemcpyAsync(B + kNaLines, h_na_lines, 32ull * nl, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(B + kNaNu, h_na_nus, 8ull * nl, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(B + kNaSorted, h_na_sorted, 4ull * nl, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(B + kNaQoff, h_na_q, 8ull * (ncell + 1), cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(B + kNaCellE, h_na_cellE, 24ull * ncell, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(B + kNaRtab, h_na_rtab, 4ull * (a->nx + a->ny + a->nz), cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemsetAsync(B + kNaLedger, 0, 8ull * LG_N, st));
  NA_CUDA(cudaMemsetAsync(B + kNaSegN, 0, 8ull * (kNaSegs + 1), st));
  const size_t Sb = (size_t)ncell * nl * sizeof(double);
  const int views = a->n_theta * a->n_phi;
  NA_CUDA(cudaMemsetAsync(a->S, 0, Sb, st));
  NA_CUDA(cudaMemsetAsync(a->spec, 0, (size_t)views * a->spec_nbins * sizeof(double), st));
  // ---- the same kernels as run_transport, with their scratch in the array
  Geometry G;
  G.nx = a->nx; G.ny = a->ny; G.nz = a->nz; G.bx = a->nx; G.by = a->ny; G.bz = a->nz; G.sx = 1; G.sy = 1;
  G.ncell = ncell; G.R = a->v_max * a->t;
  G.dx = 2.0 * G.R / a->nx; G.dy = 2.0 * G.R / a->ny; G.dz = 2.0 * G.R / a->nz;
  G.ct = kC * a->t; G.inv_ct = 1.0 / G.ct;
  unsigned long long* counters = (unsigned long long*)(B + kNaCount);
  double* ledger = (double*)(B + kNaLedger);
  int* I = (int*)(B + kNaPoolI);
  Pool P;
  P.cap = kNaChunk; P.f = (double*)(B + kNaPoolF);
  P.cell = I; P.cursor = I + kNaChunk; P.events = I + 2 * kNaChunk; P.ndraw = I + 3 * kNaChunk;
  P.inter = I + 4 * kNaChunk; P.pid = (int64_t*)(B + kNaPoolP);
  int* esc = I + 5 * kNaChunk;
  double* cellE = (double*)(B + kNaCellE);
  EmitArgs ea{};
  ea.g = G; ea.qoff = (const int64_t*)(B + kNaQoff); ea.Lc = cellE; ea.Epk = cellE + ncell;
  ea.qguide = nullptr; ea.nuguide = nullptr;
  ea.Eph = cellE + 2 * ncell; ea.cdf = nullptr; ea.sorted_of = (const int*)(B + kNaSorted);
  ea.nu_tab = (const double*)(B + kNaNu); ea.nline = nl; ea.emission = XT_EMIT_BAND; ea.seed = a->seed;
  ea.nu_lo = kC / (a->band_hi_A * 1e-8); ea.nu_hi = kC / (a->band_lo_A * 1e-8); ea.e_cut = a->e_cut;
  ea.nu_span = ea.nu_hi - ea.nu_lo; ea.wall = nullptr;
  ea.pool = P; ea.ledger = ledger; ea.records = nullptr; ea.rec_base = 0;
  fixtrig_tables(&ea.trig);
  TraceArgs ta{};
  ta.g = G; ta.lines = (const double2*)(B + kNaLines); ta.nline = nl; ta.nlev = nlev; ta.pops = a->pops;
  ta.S = a->S; ta.pool = P; ta.list = nullptr; ta.counter = counters; ta.esc = esc; ta.n_esc = counters + 1;
  ta.out = nullptr; ta.n_out = counters + 2; ta.rounds = 0; ta.seed = a->seed; ta.tau_min = a->tau_min;
  ta.ct = G.ct; ta.inv_ct = G.inv_ct; ta.max_events = a->max_events; ta.ledger = ledger;
  ta.records = nullptr; ta.rec_base = 0;
  fixexp_tables(&ta.fx);
  ta.trig = ea.trig;
  ta.rtab = (const int*)(B + kNaRtab);
  ta.slotlog = (int64_t*)(B + kNaLog); ta.seg_n = (int64_t*)(B + kNaSegN); ta.seg_len = 0;
  ta.log_overflow = (unsigned long long*)(B + kNaSegN + 8ull * kNaSegs);
  EscArgs xa{};
  xa.pool = P; xa.esc = esc; xa.spec = a->spec; xa.n_theta = a->n_theta; xa.n_phi = a->n_phi;
  xa.nbins = a->spec_nbins; xa.lam0 = a->spec_lam0_A; xa.log1p_dlog = std::log1p(a->spec_dlog);
  xa.ledger = ledger; xa.records = nullptr; xa.rec_base = 0;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trace<XT_MODE_ATTEN>, 256, 0);
  const int grid_max = (int)std::min<int64_t>((int64_t)sm_count() * std::max(occ, 1), kNaSegs);
  int kernels = 0;
  for (int64_t off = 0; off < a->n_packets; off += kNaChunk) {
    const int64_t n = std::min(kNaChunk, a->n_packets - off);
    ea.p_begin = off;
    ea.n = n;
    k_emit<<<blocks_for(n, 256, 16), 256, 0, st>>>(ea);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaMemsetAsync(counters, 0, 3 * sizeof(unsigned long long), st));
    ta.n_list = n;
    k_trace<XT_MODE_ATTEN><<<(int)std::min<int64_t>(grid_max, (n + 255) / 256), 256, 0, st>>>(ta);
    NA_CUDA(cudaGetLastError());
    unsigned long long cnt[3];
    NA_CUDA(cudaMemcpyAsync(cnt, counters, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    kernels += 2;
    if (cnt[1] > 0) {
      xa.n_esc = (int64_t)cnt[1];
      k_escape<<<blocks_for(xa.n_esc, 256, 8), 256, 0, st>>>(xa);
      NA_CUDA(cudaGetLastError());
      ++kernels;
    }
  }
  // ---- estimators to the caller's line order, divided by f_corr
  const size_t smem = (size_t)nl * sizeof(double);
  NA_CUDA(cudaFuncSetAttribute(k_na_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_na_finish<<<(unsigned)ncell, 256, smem, st>>>(a->S, a->pops, (const double*)(B + kNaLines),
                                                  (const int*)(B + kNaSorted), nl, nlev);
  NA_CUDA(cudaGetLastError());
  ++kernels;
  double led[LG_N];
  NA_CUDA(cudaMemcpyAsync(led, ledger, sizeof(led), cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaStreamSynchronize(st));
#undef NA_CUDA
  if (out) {
    std::memset(out, 0, sizeof(*out));
    double* o = &out->emitted_N;
    for (int k = 0; k < LG_STATS; ++k) o[k] = led[k];
    out->rounds = 1;
    out->kernels = kernels;
  }
  if (led[LG_GUARD] > 0) return bad(XT_ETIMEOUT, "run_transport_noalloc: packets hit max_events");
  return XT_OK;
}
