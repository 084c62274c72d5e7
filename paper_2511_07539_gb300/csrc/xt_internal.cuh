// Internal declarations of the GB300 transport library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/extrass.h"

namespace xt {

// cgs constants (CODATA exact or recommended values)
constexpr double kC = 2.99792458e10;
constexpr double kH = 6.62607015e-27;
constexpr double kE = 4.80320471e-10;
constexpr double kMe = 9.1093837015e-28;
constexpr double kPi = 3.14159265358979323846;

// Per-packet ledger slots (device accumulators), same order as xt_transport_stats.
// The first LG_STATS slots map one to one onto the leading fields of
// xt_transport_stats; the photoionization slots onto its last two (LG_PI_E
// holds photons x Hz, times h on the host).
enum Ledger {
  LG_EMIT_N, LG_ESC_N, LG_ABS_N, LG_DROP_N, LG_EMIT_E, LG_ESC_E, LG_OOB_E, LG_EVENTS,
  LG_TESTS, LG_GUARD, LG_THERMAL_E, LG_INTERACT, LG_ABS_E_CMF, LG_REEMIT_E_CMF,
  LG_STATS, LG_PI_N = LG_STATS, LG_PI_E, LG_N
};

// Read-only view of everything the transport kernel needs (passed by value).
struct Geometry {
  int nx, ny, nz;        // cells per axis
  int bx, by, bz;        // cells per subdomain per axis
  int sx, sy;            // subdomains per axis (x, y)
  int64_t ncell;
  double R, dx, dy, dz, ct, inv_ct;
  // spherical grid (both nullptr for the cube): cell volumes [row], and the
  // walk's tables [shell radii (nx+1) | cos theta (ny+1), exactly 0 for an
  // equatorial edge | cos phi (nz+1) | sin phi (nz+1) | phi (nz+1) | theta
  // (ny+1) | the middle of every cell's r, theta and phi ranges as x, y, z
  // (3 ncell, natural order)], edge nz of the azimuthal tables being edge 0
  // again for cos and sin
  const double* vol = nullptr;
  const double* sph = nullptr;
};

struct LineTable {        // lines in descending-frequency ("sorted") order
  int nline, nlev;
  const double* nu;       // Hz
  const double* K;        // (pi e^2 / m_e c) f lambda t  [cm^3]
  const double* gratio;   // g_l / g_u
  const double* hnu;      // h nu [erg]
  const double* A;        // Einstein A_ul [s^-1]
  const int* lo;          // global lower level
  const int* up;          // global upper level
  const int* down_off;    // [nlev+1] CSR of radiative down-lines per upper level
  const int* down_line;   //   (sorted line indices, ascending caller order)
};

// Map natural (ix,iy,iz) to the subdomain-blocked storage row.
__host__ __device__ inline int64_t row_of(const Geometry& g, int ix, int iy, int iz) {
  int qx = ix / g.bx, qy = iy / g.by, qz = iz / g.bz;
  int64_t sd = ((int64_t)qz * g.sy + qy) * g.sx + qx;
  int64_t loc = ((int64_t)(iz - qz * g.bz) * g.by + (iy - qy * g.by)) * g.bx + (ix - qx * g.bx);
  return sd * ((int64_t)g.bx * g.by * g.bz) + loc;
}

}  // namespace xt

struct xt_mlp;

struct xt_ctx {
  xt_mlp* mlp = nullptr;             // population surrogate (mlp.cu)
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  std::unordered_map<void*, size_t> alloc_bytes;   // size of every buffer alloc() made
  // grid
  bool have_grid = false;
  xt::Geometry geo{};
  int sx = 1, sy = 1, sz = 1;
  double v_max = 0, t = 0, band_lo_A = 0, band_hi_A = 0;
  std::vector<double> h_L;           // natural order, for the packet quota
  double* d_Te = nullptr;            // row order
  double* d_ne = nullptr;
  double* d_rho = nullptr;
  double* d_dep = nullptr;
  double* d_L = nullptr;             // row order
  int geometry = XT_GEOM_CARTESIAN;
  double* d_vol = nullptr;           // spherical grid: cell volumes, row order
  double* d_sph = nullptr;           //   and the walk's tables (Geometry::sph)
  std::vector<double> h_sph;
  // atoms
  bool have_atoms = false;
  int n_ion = 0, nlev = 0, nline = 0;
  std::vector<int> h_level_off;
  std::vector<double> h_g, h_E;
  std::vector<int> h_sorted_of;      // caller line -> sorted position
  std::vector<int> h_orig_of;        // sorted position -> caller line
  std::vector<double> h_nu_sorted;   // line frequencies, sorted (descending)
  std::vector<double> h_lam_caller;  // line wavelengths (A), caller order
  int* d_level_off = nullptr;
  double* d_g = nullptr;
  double* d_E = nullptr;
  double *d_nu = nullptr, *d_K = nullptr, *d_gratio = nullptr, *d_hnu = nullptr, *d_A = nullptr;
  double* d_invB = nullptr;          // 1 / B_lu (sorted)
  int *d_lo = nullptr, *d_up = nullptr, *d_orig = nullptr;
  int *d_down_off = nullptr, *d_down_line = nullptr;
  int *d_low_off = nullptr, *d_low_line = nullptr;   // lines by lower level (positions in d_down_line)
  double* d_nion = nullptr;          // [row][n_ion]
  double* d_ups_down = nullptr;      // [nlev]
  // photoionizing levels, sorted by threshold frequency (descending; ties in
  // the caller's order k)
  int npi = 0;
  std::vector<int> h_pi_sorted_of;   // caller k -> sorted position
  double* d_pi_nuth = nullptr;       // [npi] threshold frequency (Hz)
  double* d_pi_sig = nullptr;        // [npi] sigma = sig lambda^3 (lambda in cm)
  double* d_pi_chi = nullptr;        // [npi] threshold energy (erg)
  int* d_pi_lev = nullptr;           // [npi] global level
  int* d_pi_sorted_of = nullptr;     // [npi] caller k -> sorted position
  double* d_kappa = nullptr;         // [row][npi+1] suffix sums of sig n_level per cell
  double* d_piG = nullptr;           // [row][npi+1] segment weights by first full-length level
  double* d_piD = nullptr;           // [row][npi]   weights of levels whose threshold a segment crossed
  double* d_piH = nullptr;           // [row] absorbed photons x frequency
  int64_t pi_rows = 0;               // rows the per-cell photoionization arrays hold
  int pi_npi = 0;                    //   for this many levels
  bool have_pi = false;              // the last pass photoionized
  // spatial decomposition: the domain of the current run_transport_domain call
  struct Domain {
    bool active = false;
    int z_lo = 0, z_hi = 0, emit = 0;
    const double* in = nullptr; int64_t n_in = 0;
    double* out = nullptr; int64_t out_cap = 0, n_out = 0;
  } dom;
  std::vector<int64_t> h_qoff;       // the packet quota (natural order prefix) on the host
  void* d_rays = nullptr;            // the RAYS sampler's tables (one allocation, carved)
  size_t rays_bytes = 0;
  // state
  bool have_pops = false;
  double* d_pops = nullptr;          // [row][nlev]
  double* d_S = nullptr;             // [row][sorted line] (host groups: one group's slab)
  size_t S_bytes = 0;
  bool S_compact = false;            // the store holds rows only for cells with populations:
  int* d_crow = nullptr;             //   [row] its row in the store, or -1
  int64_t n_crow = 0;
  std::vector<int> h_crow;
  int S_groups = 0;                  // > 0: the store lives in pinned host memory in this
  double* h_S = nullptr;             //   many groups of subdomain z-layers (rows contiguous)
  size_t h_S_bytes = 0;
  std::vector<char> S_valid;         // group written by the current pass (else all zero)
  int* d_stream_q = nullptr;         // host store: out, carry-in, carry-out packet queues
  int64_t stream_q_cap = 0;
  bool have_S = false;
  // emission
  int64_t* d_qoff = nullptr;         // natural order [ncell+1]
  int64_t qoff_n = 0, qguide_n = 0, Lc_n = 0;   // allocated entries (cells for d_Lc)
  int* d_qguide = nullptr;           // cell of packet j 2^6, j = 0..(N-1)/2^6 + 1
  int* d_nuguide = nullptr;          // band emission: first sorted line below each of 2^16 + 1 edges
  int64_t qoff_N = -1;               // N the quota was built for
  int qoff_mode = -1;
  double* d_Lc = nullptr;            // natural order cell luminosity used by the quota
  double* d_wline = nullptr;         // [row][sorted line] line emission weights (XT_EMIT_LINES)
  size_t wline_bytes = 0;
  // spectrum
  double* d_spec = nullptr;
  int spec_views = 0, spec_bins = 0, n_theta = 20, n_phi = 20;
  double spec_lam0 = 0, spec_dlog = 1e-3;
  // ledger
  double* d_ledger = nullptr;        // [LG_N]
  double* d_lines = nullptr;         // [sorted line] packed nu, K, gratio, (lo, up): 32 B
  int* d_rtab = nullptr;             // separable blocked-row offsets [nx + ny + nz]
  double* d_wall = nullptr;          // lower cell walls per axis [nx + ny + nz]
  int64_t rtab_n = 0, wall_n = 0;    // their lengths (reallocated when the grid changes)
  // touched-slot log: every estimator slot written by the last pass, so the
  // next pass clears those slots instead of the whole store
  int64_t* d_slotlog = nullptr;
  int64_t* d_seg_n = nullptr;        // entries per log segment, then an overflow counter
  int log_nseg = 0;                  // segments (trace blocks) of the current log layout
  int64_t log_seglen = 0;
  int64_t slotlog_cap = 0;
  int64_t slotlog_n = 0;             // entries of the last pass (may exceed cap)
  bool slotlog_valid = false;        // every nonzero slot of the store is in the log
  // transport buffers
  double* d_pool_f = nullptr;
  int* d_pool_i = nullptr;
  int64_t* d_pool_pid = nullptr;
  int64_t pool_cap = 0;
  unsigned long long* d_counters = nullptr;
  unsigned* d_hist = nullptr;
  int hist_n = 0;
  // scratch
  void* d_scratch = nullptr;
  size_t scratch_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
  // statistical-equilibrium solve: buffers kept between calls, tuned panel
  // widths per precision and 64-level bucket, captured launches
  struct SeBufs {
    double* ups = nullptr; size_t ups_n = 0;
    int64_t* upsoff = nullptr;
    int* work = nullptr; int* used = nullptr; int64_t nsys = 0;
    unsigned long long* cnt = nullptr;
    double* iters = nullptr; int* status = nullptr;
    double* pops_new = nullptr; size_t pops_n = 0;
    double* W64 = nullptr; double* WT = nullptr; size_t wbytes = 0;
    double* Rj = nullptr; int Rj_n = 0;
    double* warm = nullptr; size_t warm_n = 0;
    int* used_nat = nullptr; int64_t used_nat_n = 0;
    int nb[3][8] = {{16, 16, 16, 16, 16, 16, 16, 16}, {32, 32, 32, 32, 32, 32, 32, 32},
                    {32, 32, 32, 32, 32, 32, 32, 32}};   // FP64, FP32, TF32
    bool tuned[3] = {false, false, false};
    std::vector<std::vector<unsigned char>> graph_keys;
    std::vector<cudaGraphExec_t> graphs;
  } se;
  cudaStream_t side = nullptr;       // second stream: store clear overlapping emission
  cudaEvent_t ev_side0 = nullptr, ev_side1 = nullptr;
  std::vector<cudaEvent_t> ev_pool;  // per-kernel timing events
};

namespace xt {
int fail(xt_ctx* c, int code, const std::string& msg);
int cuda_fail(xt_ctx* c, cudaError_t e, const char* what);
bool is_device_ptr(const void* p);
// Copy n bytes between any host/device pointers on the context stream.
int copy(xt_ctx* c, void* dst, const void* src, size_t n, const char* what);
int ensure_scratch(xt_ctx* c, size_t bytes);
int alloc(xt_ctx* c, void** p, size_t bytes, const char* what);
void release(void** p);
// natural-order [ncell][W] device array -> blocked rows (device), on the context stream
int nat_to_row(xt_ctx* c, const double* src, double* dst, int64_t W);
void mlp_destroy(xt_mlp* n);
// Surrogate warm start: populations [row][nlev] predicted for every cell
// (levels beyond levels_used zero), into `out` (device).
int surrogate_warm(xt_ctx* c, int rates, double jbar_W, double jbar_TR, const int* levels_used_dev,
                   double* out);
// Boltzmann populations [row][nlev] of the kept levels into `out` (device).
int lte_fill(xt_ctx* c, const int* levels_used_dev, double* out);
}  // namespace xt

#define XT_CUDA(ctx, call)                                        \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return xt::cuda_fail(ctx, e_, #call);  \
  } while (0)
