// Context, data upload, A1 (Sobolev tau/beta), A7 (rates) and A5 (spectrum
// normalisation) of the GB300 transport library.  See include/extrass.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "fixexp.cuh"
#include "linesort.h"
#include "xt_internal.cuh"

namespace xt {

int fail(xt_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(xt_ctx* c, cudaError_t e, const char* what) {
  return fail(c, XT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) { cudaGetLastError(); return false; }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int copy(xt_ctx* c, void* dst, const void* src, size_t n, const char* what) {
  if (n == 0) return XT_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  return XT_OK;
}

// (Re)allocate *p to `bytes` of device memory.  A buffer of exactly that size
// is kept (reloading a workload of the same shape allocates nothing); any
// other is freed first.  Contents are undefined either way.
int alloc(xt_ctx* c, void** p, size_t bytes, const char* what) {
  if (*p) {
    const auto it = c->alloc_bytes.find(*p);
    if (bytes > 0 && it != c->alloc_bytes.end() && it->second == bytes) return XT_OK;
    if (it != c->alloc_bytes.end()) c->alloc_bytes.erase(it);
    cudaFree(*p);
    *p = nullptr;
  }
  if (bytes == 0) return XT_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, XT_ENOMEM, std::string("cudaMalloc failed for ") + what + " (" +
                                  std::to_string(bytes) + " bytes)");
  }
  c->alloc_bytes[*p] = bytes;
  return XT_OK;
}

void release(void** p) {
  if (*p) cudaFree(*p);
  *p = nullptr;
}

int ensure_scratch(xt_ctx* c, size_t bytes) {
  if (bytes <= c->scratch_bytes) return XT_OK;
  cudaStreamSynchronize(c->stream);
  int rc = alloc(c, &c->d_scratch, bytes, "scratch");
  c->scratch_bytes = rc == XT_OK ? bytes : 0;
  return rc;
}

// dst[row(c)][j] = src[c][j]  (natural -> blocked rows), width W
__global__ void k_nat_to_row(Geometry g, const double* __restrict__ src, double* __restrict__ dst,
                             int64_t W) {
  int64_t n = g.ncell * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = i / W, j = i - c * W;
    int ix = (int)(c % g.nx), iy = (int)((c / g.nx) % g.ny), iz = (int)(c / ((int64_t)g.nx * g.ny));
    dst[row_of(g, ix, iy, iz) * W + j] = src[i];
  }
}

__global__ void k_row_to_nat(Geometry g, const double* __restrict__ src, double* __restrict__ dst,
                             int64_t W) {
  int64_t n = g.ncell * W;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = i / W, j = i - c * W;
    int ix = (int)(c % g.nx), iy = (int)((c / g.nx) % g.ny), iz = (int)(c / ((int64_t)g.nx * g.ny));
    dst[i] = src[row_of(g, ix, iy, iz) * W + j];
  }
}

static int grid_blocks(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (int)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 32);
}

int nat_to_row(xt_ctx* c, const double* src, double* dst, int64_t W) {
  k_nat_to_row<<<grid_blocks(c->geo.ncell * W, 256), 256, 0, c->stream>>>(c->geo, src, dst, W);
  XT_CUDA(c, cudaGetLastError());
  return XT_OK;
}

// Upload a natural-order [ncell][W] array (host or device) into blocked rows.
static int upload_rows(xt_ctx* c, const double* src, double** dst, int64_t W, const char* what) {
  size_t bytes = (size_t)c->geo.ncell * W * sizeof(double);
  int rc = alloc(c, (void**)dst, bytes, what);
  if (rc) return rc;
  const double* dsrc = src;
  if (!is_device_ptr(src)) {
    if ((rc = ensure_scratch(c, bytes))) return rc;
    if ((rc = copy(c, c->d_scratch, src, bytes, what))) return rc;
    dsrc = (const double*)c->d_scratch;
  }
  k_nat_to_row<<<grid_blocks(c->geo.ncell * W, 256), 256, 0, c->stream>>>(c->geo, dsrc, *dst, W);
  XT_CUDA(c, cudaGetLastError());
  return XT_OK;
}

// Run `fill(dev_out)` writing `bytes` and deliver them to `user` (host or device).
template <class F>
static int deliver(xt_ctx* c, void* user, size_t bytes, F fill) {
  if (!user) return XT_OK;
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

template <class T>
static int to_host(xt_ctx* c, const T* src, size_t n, std::vector<T>& out, const char* what) {
  out.resize(n);
  if (n == 0) return XT_OK;
  cudaError_t e = cudaMemcpyAsync(out.data(), src, n * sizeof(T), cudaMemcpyDefault, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  return XT_OK;
}

template <class T>
static int to_device(xt_ctx* c, const std::vector<T>& v, T** dst, const char* what) {
  int rc = alloc(c, (void**)dst, v.size() * sizeof(T), what);
  if (rc) return rc;
  return copy(c, *dst, v.data(), v.size() * sizeof(T), what);
}

// ---- A1: tau_S, Eq. (tau_Sobolev), and beta_S, Eq. (beta_Sobolev) ----------
__device__ __forceinline__ double beta_sobolev(double tau) {
  return tau <= 0.0 ? 1.0 : -expm1(-tau) / tau;   // no trapping for tau <= 0
}

__global__ void k_tau_beta(Geometry g, LineTable L, const double* __restrict__ pops,
                           const int* __restrict__ sorted_of, int64_t c0, int64_t nc,
                           double* __restrict__ tau_out, double* __restrict__ beta_out) {
  int64_t n = nc * L.nline;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t cl = i / L.nline;
    int l = (int)(i - cl * L.nline);
    int64_t c = c0 + cl;
    int ix = (int)(c % g.nx), iy = (int)((c / g.nx) % g.ny), iz = (int)(c / ((int64_t)g.nx * g.ny));
    const double* pc = pops + row_of(g, ix, iy, iz) * L.nlev;
    int s = sorted_of[l];
    double tau = L.K[s] * (pc[L.lo[s]] - L.gratio[s] * pc[L.up[s]]);
    if (tau_out) tau_out[i] = tau;
    if (beta_out) beta_out[i] = beta_sobolev(tau);
  }
}

// ---- A7: rates from estimators -------------------------------------------
__global__ void k_rates(Geometry g, LineTable L, const double* __restrict__ pops,
                        const double* __restrict__ S, const double* __restrict__ invB,
                        const int* __restrict__ sorted_of, int64_t c0, int64_t nc, double V,
                        int which, double* __restrict__ out, const int* __restrict__ crow) {
  // a block per cell at a time: the cell's row found once, its lines spread
  // over the threads (output in caller line order, coalesced)
  for (int64_t cl = blockIdx.x; cl < nc; cl += gridDim.x) {
    const int64_t c = c0 + cl;
    const int ix = (int)(c % g.nx), iy = (int)((c / g.nx) % g.ny), iz = (int)(c / ((int64_t)g.nx * g.ny));
    const int64_t row = row_of(g, ix, iy, iz);
    const int64_t sr = crow ? (int64_t)crow[row] : row;    // the cell's row in the store (-1: none)
    const double* Sr = S + (sr < 0 ? 0 : sr) * L.nline;
    const double* pr = pops + row * L.nlev;
    double* o = out + cl * L.nline;
    const double Vc = g.vol ? g.vol[row] : V;
    for (int l = threadIdx.x; l < L.nline; l += blockDim.x) {
      const int s = sorted_of[l];
      // the store holds net photons absorbed; gross = net / f_corr, f_corr = net_pop / n_l
      const double Snet = sr < 0 ? 0.0 : Sr[s];
      double v = 0.0;
      if (Snet != 0.0) {
        const double nl = pr[L.lo[s]];
        const double net = nl - L.gratio[s] * pr[L.up[s]];
        if (which == 0) {
          v = Snet * nl / net;
        } else {
          const double R = Snet / (net * Vc);        // S / (n_l V)
          v = which == 1 ? R : which == 2 ? L.gratio[s] * R : R * invB[s];
        }
      }
      o[l] = v;
    }
  }
}

// ---- A5: spectrum normalisation -------------------------------------------
__global__ void k_spectrum(const double* __restrict__ E, int n_theta, int n_phi, int nb,
                           double lam0, double dlog, int kind, double* __restrict__ out) {
  int views = n_theta * n_phi;
  int64_t n = kind == 2 ? nb : (int64_t)views * nb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int b = (int)(i % nb);
    double e0 = lam0 * pow(1.0 + dlog, (double)b), e1 = lam0 * pow(1.0 + dlog, (double)(b + 1));
    double dlam = e1 - e0;
    if (kind == 2) {
      double s = 0.0;
      for (int k = 0; k < views; ++k) s += E[(int64_t)k * nb + b];
      out[i] = s / dlam;
    } else {
      int k = (int)(i / nb);
      double th0 = kPi * (k / n_phi) / n_theta, th1 = kPi * (k / n_phi + 1) / n_theta;
      double dOm = (2.0 * kPi / n_phi) * (cos(th0) - cos(th1));
      out[i] = kind == 0 ? E[i] : 4.0 * kPi / dOm * E[i] / dlam;
    }
  }
}

__global__ void k_selftest_fixed(int kind, FixExpTables T, FixTrigTables R,
                                 const double* __restrict__ x, int64_t n, double* y0, double* y1,
                                 double* r0, double* r1) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (kind == 0) {
      expneg(T, x[i], y0[i], y1[i]);
      r0[i] = exp(-x[i]);
      r1[i] = -expm1(-x[i]);
    } else if (kind == 1) {
      const uint64_t U = (uint64_t)(x[i] * 9007199254740992.0);   // exact for u = U 2^-53
      sincos_2pi(R, U, y0[i], y1[i]);
      sincos(2.0 * kPi * x[i], &r0[i], &r1[i]);
    } else if (kind == 2) {
      y0[i] = div_pos(x[2 * i], x[2 * i + 1]);
      r0[i] = x[2 * i] / x[2 * i + 1];
      y1[i] = 0.0;
      r1[i] = 0.0;
    } else {
      double n[3];
      isotropic_fix(R, (uint64_t)(x[2 * i] * 9007199254740992.0),
                    (uint64_t)(x[2 * i + 1] * 9007199254740992.0), n);
      y0[i] = n[0];
      y1[i] = n[1];
      r0[i] = n[2];
      r1[i] = 0.0;
    }
  }
}

}  // namespace xt

using namespace xt;

extern "C" {

int xt_create(xt_ctx** out, int device, void* cuda_stream) {
  if (!out) return XT_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return XT_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return XT_ECUDA;
  xt_ctx* c = new xt_ctx();
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  cudaEventCreate(&c->ev0);
  cudaEventCreate(&c->ev1);
  cudaEventCreate(&c->ev2);
  cudaEventCreate(&c->ev_side0);
  cudaEventCreate(&c->ev_side1);
  cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (alloc(c, (void**)&c->d_ledger, LG_N * sizeof(double), "ledger")) { delete c; return XT_ENOMEM; }
  *out = c;
  return XT_OK;
}

void xt_destroy(xt_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  void** ptrs[] = {(void**)&c->d_Te, (void**)&c->d_ne, (void**)&c->d_rho, (void**)&c->d_dep,
                   (void**)&c->d_L, (void**)&c->d_level_off, (void**)&c->d_g, (void**)&c->d_E,
                   (void**)&c->d_nu, (void**)&c->d_K, (void**)&c->d_gratio, (void**)&c->d_hnu,
                   (void**)&c->d_A, (void**)&c->d_invB, (void**)&c->d_lo, (void**)&c->d_up,
                   (void**)&c->d_orig, (void**)&c->d_down_off, (void**)&c->d_down_line,
                   (void**)&c->d_nion, (void**)&c->d_ups_down, (void**)&c->d_pops, (void**)&c->d_S,
                   (void**)&c->d_qoff, (void**)&c->d_qguide, (void**)&c->d_nuguide, (void**)&c->d_Lc, (void**)&c->d_wline, (void**)&c->d_spec,
                   (void**)&c->d_ledger, (void**)&c->d_scratch, (void**)&c->d_lines,
                   (void**)&c->d_pool_f, (void**)&c->d_pool_i, (void**)&c->d_pool_pid,
                   (void**)&c->d_counters, (void**)&c->d_hist, (void**)&c->d_rtab, (void**)&c->d_wall, (void**)&c->d_stream_q, (void**)&c->d_slotlog, (void**)&c->d_seg_n,
                   (void**)&c->d_pi_nuth, (void**)&c->d_pi_sig, (void**)&c->d_pi_chi, (void**)&c->d_pi_lev,
                   (void**)&c->d_pi_sorted_of, (void**)&c->d_kappa, (void**)&c->d_piG, (void**)&c->d_piD,
                   (void**)&c->d_piH, (void**)&c->d_rays, (void**)&c->d_low_off, (void**)&c->d_low_line,
                   (void**)&c->d_crow, (void**)&c->d_vol, (void**)&c->d_sph};
  for (void** p : ptrs) release(p);
  if (c->h_S) cudaFreeHost(c->h_S);
  c->h_S = nullptr;
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->ev2) cudaEventDestroy(c->ev2);
  if (c->ev_side0) cudaEventDestroy(c->ev_side0);
  if (c->ev_side1) cudaEventDestroy(c->ev_side1);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  {
    auto& s = c->se;
    void** sp[] = {(void**)&s.ups, (void**)&s.upsoff, (void**)&s.work, (void**)&s.used, (void**)&s.cnt,
                   (void**)&s.iters, (void**)&s.status, (void**)&s.pops_new, (void**)&s.W64, (void**)&s.used_nat,
                   (void**)&s.WT, (void**)&s.Rj, (void**)&s.warm};
    for (void** q : sp) release(q);
    for (cudaGraphExec_t g : s.graphs) cudaGraphExecDestroy(g);
  }
  if (c->side) cudaStreamDestroy(c->side);
  if (c->mlp) mlp_destroy(c->mlp);
  delete c;
}

const char* xt_last_error(const xt_ctx* c) { return c ? c->err.c_str() : "null context"; }

int init_grid(xt_ctx* c, const xt_grid_desc* g) {
  if (!c || !g) return fail(c, XT_EINVAL, "init_grid: null argument");
  cudaSetDevice(c->device);
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(c, XT_EINVAL, "init_grid: nx, ny, nz must be >= 1");
  if (g->sx < 1 || g->sy < 1 || g->sz < 1 || g->nx % g->sx || g->ny % g->sy || g->nz % g->sz)
    return fail(c, XT_EINVAL, "init_grid: sx, sy, sz must be >= 1 and divide nx, ny, nz");
  if (!(g->v_max > 0) || !(g->t > 0)) return fail(c, XT_EINVAL, "init_grid: v_max and t must be > 0");
  if (!g->Te || !g->ne) return fail(c, XT_EINVAL, "init_grid: Te and ne are required");
  if (g->L_cell && !(g->band_hi_A > g->band_lo_A && g->band_lo_A > 0))
    return fail(c, XT_EINVAL, "init_grid: band_lo_A < band_hi_A required with L_cell");
  if (g->geometry != XT_GEOM_CARTESIAN && g->geometry != XT_GEOM_SPHERICAL)
    return fail(c, XT_EINVAL, "init_grid: geometry must be XT_GEOM_CARTESIAN or XT_GEOM_SPHERICAL");
  const bool sph = g->geometry == XT_GEOM_SPHERICAL;
  // spherical grid: edges checked before anything of the context changes
  std::vector<double> re, te, pe, tab, vol_nat;
  if (sph) {
    if (!g->r_edges || !g->theta_edges || !g->phi_edges)
      return fail(c, XT_EINVAL, "init_grid: a spherical grid needs r_edges, theta_edges and phi_edges");
    re.resize(g->nx + 1); te.resize(g->ny + 1); pe.resize(g->nz + 1);
    int rc0;
    if ((rc0 = copy(c, re.data(), g->r_edges, re.size() * sizeof(double), "r_edges"))) return rc0;
    if ((rc0 = copy(c, te.data(), g->theta_edges, te.size() * sizeof(double), "theta_edges"))) return rc0;
    if ((rc0 = copy(c, pe.data(), g->phi_edges, pe.size() * sizeof(double), "phi_edges"))) return rc0;
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
    auto increasing = [](const std::vector<double>& e, double last) {
      if (e[0] != 0.0) return false;
      for (size_t i = 1; i < e.size(); ++i)
        if (!(e[i] > e[i - 1]) || !std::isfinite(e[i])) return false;
      return std::fabs(e.back() - last) <= 1e-12 * last;
    };
    if (!increasing(re, g->v_max))
      return fail(c, XT_EINVAL, "init_grid: r_edges must increase strictly from 0 to v_max");
    if (!increasing(te, kPi))
      return fail(c, XT_EINVAL, "init_grid: theta_edges must increase strictly from 0 to pi");
    if (!increasing(pe, 2.0 * kPi))
      return fail(c, XT_EINVAL, "init_grid: phi_edges must increase strictly from 0 to 2 pi");
  }
  Geometry& G = c->geo;
  G.nx = g->nx; G.ny = g->ny; G.nz = g->nz;
  G.bx = g->nx / g->sx; G.by = g->ny / g->sy; G.bz = g->nz / g->sz;
  G.sx = g->sx; G.sy = g->sy;
  G.ncell = (int64_t)g->nx * g->ny * g->nz;
  G.R = g->v_max * g->t;
  G.dx = 2.0 * G.R / g->nx; G.dy = 2.0 * G.R / g->ny; G.dz = 2.0 * G.R / g->nz;
  G.ct = kC * g->t;
  G.inv_ct = 1.0 / G.ct;
  c->sx = g->sx; c->sy = g->sy; c->sz = g->sz;
  c->v_max = g->v_max; c->t = g->t;
  c->band_lo_A = g->band_lo_A; c->band_hi_A = g->band_hi_A;
  int rc;
  G.vol = nullptr;
  G.sph = nullptr;
  c->geometry = g->geometry;
  if (!sph) {
    release((void**)&c->d_vol);
    release((void**)&c->d_sph);
    c->h_sph.clear();
  } else {
    // the walk's tables (shell radii, cos theta with equatorial edges exactly
    // 0, cos and sin phi with edge nz taken as edge 0, phi) and the volumes
    // (r1^3 - r0^3) / 3 (cos theta0 - cos theta1) (phi1 - phi0), natural order
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    tab.assign((size_t)(nx + 1) + 2 * (size_t)(ny + 1) + 3 * (size_t)(nz + 1) + 3 * (size_t)G.ncell, 0.0);
    double* sR = tab.data();
    double* cth = sR + nx + 1;
    double* cph = cth + ny + 1;
    double* sphi = cph + nz + 1;
    double* phe = sphi + nz + 1;
    double* the = phe + nz + 1;
    double* mid = the + ny + 1;
    for (int j = 0; j <= ny; ++j) the[j] = te[j];
    std::vector<double> ct_raw(ny + 1);
    for (int i = 0; i <= nx; ++i) sR[i] = re[i] * g->t;
    for (int j = 0; j <= ny; ++j) {
      ct_raw[j] = std::cos(te[j]);
      cth[j] = std::fabs(ct_raw[j]) < 1e-12 ? 0.0 : ct_raw[j];
    }
    for (int k = 0; k <= nz; ++k) {
      const double ph = pe[k == nz ? 0 : k];
      cph[k] = std::cos(ph);
      sphi[k] = std::sin(ph);
      phe[k] = pe[k];
    }
    vol_nat.resize(G.ncell);
    for (int64_t cc = 0; cc < G.ncell; ++cc) {
      const int ir = (int)(cc % nx), it = (int)((cc / nx) % ny), ip = (int)(cc / ((int64_t)nx * ny));
      vol_nat[cc] = (sR[ir + 1] * sR[ir + 1] * sR[ir + 1] - sR[ir] * sR[ir] * sR[ir]) / 3.0 *
                    (ct_raw[it] - ct_raw[it + 1]) * (pe[ip + 1] - pe[ip]);
      // the middle of the cell's r, theta and phi ranges (where its rays start)
      const double rm = 0.5 * (sR[ir] + sR[ir + 1]);
      const double tm = 0.5 * (te[it] + te[it + 1]), pm = 0.5 * (pe[ip] + pe[ip + 1]);
      mid[3 * cc] = rm * std::sin(tm) * std::cos(pm);
      mid[3 * cc + 1] = rm * std::sin(tm) * std::sin(pm);
      mid[3 * cc + 2] = rm * std::cos(tm);
    }
    if ((rc = alloc(c, (void**)&c->d_sph, tab.size() * sizeof(double), "spherical tables"))) return rc;
    if ((rc = copy(c, c->d_sph, tab.data(), tab.size() * sizeof(double), "spherical tables"))) return rc;
    if ((rc = upload_rows(c, vol_nat.data(), &c->d_vol, 1, "cell volumes"))) return rc;
    c->h_sph = tab;
    G.vol = c->d_vol;
    G.sph = c->d_sph;
  }
  if ((rc = upload_rows(c, g->Te, &c->d_Te, 1, "Te"))) return rc;
  if ((rc = upload_rows(c, g->ne, &c->d_ne, 1, "ne"))) return rc;
  if (g->rho && (rc = upload_rows(c, g->rho, &c->d_rho, 1, "rho"))) return rc;
  if (g->deposition && (rc = upload_rows(c, g->deposition, &c->d_dep, 1, "deposition"))) return rc;
  c->h_L.assign(G.ncell, 0.0);
  if (g->L_cell) {
    if ((rc = copy(c, c->h_L.data(), g->L_cell, G.ncell * sizeof(double), "L_cell"))) return rc;
    if ((rc = upload_rows(c, g->L_cell, &c->d_L, 1, "L_cell"))) return rc;
  }
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int64_t i = 0; i < G.ncell; ++i)
    if (!(c->h_L[i] >= 0.0) || !std::isfinite(c->h_L[i]))
      return fail(c, XT_EINVAL, "init_grid: L_cell must be finite and >= 0 (cell " + std::to_string(i) + ")");
  c->have_grid = true;
  c->have_atoms = c->have_pops = c->have_S = false;
  c->qoff_N = -1;
  return XT_OK;
}

// Photoionizing levels of load_atomic_data (Sec. 2.3.1, Eq. sigma_OTSPI):
// thresholds, the cross section's constant factor sig (sigma = sig lambda^3),
// sorted by threshold frequency, descending (ties in the caller's order).
static int load_photoionization(xt_ctx* c, const xt_atom_desc* a, const std::vector<int>& off,
                                const std::vector<double>& E) {
  c->npi = 0;
  c->have_pi = false;
  c->h_pi_sorted_of.clear();
  const int given = (a->chi_ion != nullptr) + (a->charge != nullptr) + (a->pi_nlev != nullptr);
  if (given == 0) return XT_OK;
  if (given != 3) return fail(c, XT_EINVAL, "load_atomic_data: chi_ion, charge and pi_nlev go together");
  int rc;
  const int nz = a->n_ion;
  std::vector<double> chi(nz);
  std::vector<int> ch(nz), np(nz);
  if ((rc = copy(c, chi.data(), a->chi_ion, nz * sizeof(double), "chi_ion"))) return rc;
  if ((rc = copy(c, ch.data(), a->charge, nz * sizeof(int), "charge"))) return rc;
  if ((rc = copy(c, np.data(), a->pi_nlev, nz * sizeof(int), "pi_nlev"))) return rc;
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<double> nuth, sig, thr;
  std::vector<int> lev;
  for (int z = 0; z < nz; ++z) {
    if (np[z] < 0 || np[z] > off[z + 1] - off[z])
      return fail(c, XT_EINVAL, "load_atomic_data: pi_nlev[" + std::to_string(z) + "] outside 0..levels of the ion");
    if (ch[z] < 0) return fail(c, XT_EINVAL, "load_atomic_data: charge[" + std::to_string(z) + "] < 0");
    for (int i = 0; i < np[z]; ++i) {
      const int l = off[z] + i;
      const double x = chi[z] - E[l];                       // threshold energy
      if (!(x > 0) || !std::isfinite(chi[z]))
        return fail(c, XT_EINVAL, "load_atomic_data: photoionization threshold chi_ion - E_u <= 0 (ion " +
                                      std::to_string(z) + ", level " + std::to_string(i) + ")");
      const double inv_lam_ion = x / (kH * kC);             // 1 / lambda_ion [cm^-1]
      const double q = (double)(ch[z] + 1);
      sig.push_back(7.9e-18 * inv_lam_ion * inv_lam_ion * inv_lam_ion / std::sqrt(1.0 - E[l] / chi[z]) / (q * q));
      nuth.push_back(x / kH);
      thr.push_back(x);
      lev.push_back(l);
    }
  }
  const int n = (int)lev.size();
  if (n > XT_PI_MAX)
    return fail(c, XT_EINVAL, "load_atomic_data: " + std::to_string(n) + " photoionizing levels exceed XT_PI_MAX");
  std::vector<int> ord(n);
  for (int k = 0; k < n; ++k) ord[k] = k;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return nuth[x] > nuth[y]; });
  std::vector<double> s_nu(n), s_sig(n), s_chi(n);
  std::vector<int> s_lev(n);
  c->h_pi_sorted_of.assign(n, 0);
  for (int s = 0; s < n; ++s) {
    const int k = ord[s];
    s_nu[s] = nuth[k]; s_sig[s] = sig[k]; s_chi[s] = thr[k]; s_lev[s] = lev[k];
    c->h_pi_sorted_of[k] = s;
  }
  c->npi = n;
  if (n == 0) return XT_OK;
  if ((rc = to_device(c, s_nu, &c->d_pi_nuth, "pi thresholds"))) return rc;
  if ((rc = to_device(c, s_sig, &c->d_pi_sig, "pi cross sections"))) return rc;
  if ((rc = to_device(c, s_chi, &c->d_pi_chi, "pi threshold energies"))) return rc;
  if ((rc = to_device(c, s_lev, &c->d_pi_lev, "pi levels"))) return rc;
  if ((rc = to_device(c, c->h_pi_sorted_of, &c->d_pi_sorted_of, "pi order"))) return rc;
  return XT_OK;
}

int load_atomic_data(xt_ctx* c, const xt_atom_desc* a) {
  if (!c || !a) return fail(c, XT_EINVAL, "load_atomic_data: null argument");
  if (!c->have_grid) return fail(c, XT_ESTATE, "load_atomic_data: call init_grid first");
  cudaSetDevice(c->device);
  if (a->n_ion < 1 || a->nline < 0 || !a->level_off || !a->E_level || !a->g_level)
    return fail(c, XT_EINVAL, "load_atomic_data: n_ion >= 1, level_off, E_level, g_level required");
  if (a->nline > 0 && (!a->lo || !a->up || !a->lambda_A || !a->f_lu))
    return fail(c, XT_EINVAL, "load_atomic_data: lo, up, lambda_A, f_lu required");
  int rc;
  std::vector<int> off(a->n_ion + 1);
  if ((rc = copy(c, off.data(), a->level_off, off.size() * sizeof(int), "level_off"))) return rc;
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  if (off[0] != 0) return fail(c, XT_EINVAL, "load_atomic_data: level_off[0] must be 0");
  for (int z = 0; z < a->n_ion; ++z)
    if (off[z + 1] <= off[z]) return fail(c, XT_EINVAL, "load_atomic_data: level_off must increase (ion " + std::to_string(z) + ")");
  int nlev = off[a->n_ion], nl = a->nline;
  std::vector<double> E(nlev), g(nlev), lam(nl), f(nl), ups;
  std::vector<int> lo(nl), up(nl);
  if ((rc = copy(c, E.data(), a->E_level, nlev * sizeof(double), "E_level"))) return rc;
  if ((rc = copy(c, g.data(), a->g_level, nlev * sizeof(double), "g_level"))) return rc;
  if ((rc = copy(c, lo.data(), a->lo, nl * sizeof(int), "lo"))) return rc;
  if ((rc = copy(c, up.data(), a->up, nl * sizeof(int), "up"))) return rc;
  if ((rc = copy(c, lam.data(), a->lambda_A, nl * sizeof(double), "lambda_A"))) return rc;
  if ((rc = copy(c, f.data(), a->f_lu, nl * sizeof(double), "f_lu"))) return rc;
  if (a->ups_down) {
    ups.resize(nlev);
    if ((rc = copy(c, ups.data(), a->ups_down, nlev * sizeof(double), "ups_down"))) return rc;
  } else {
    ups.assign(nlev, 0.0);
  }
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<int> ion_of(nlev);
  for (int z = 0; z < a->n_ion; ++z)
    for (int i = off[z]; i < off[z + 1]; ++i) ion_of[i] = z;
  for (int i = 0; i < nlev; ++i)
    if (!(g[i] > 0)) return fail(c, XT_EINVAL, "load_atomic_data: g_level must be > 0 (level " + std::to_string(i) + ")");
  for (int l = 0; l < nl; ++l) {
    if (lo[l] < 0 || up[l] >= nlev || lo[l] >= up[l] || ion_of[lo[l]] != ion_of[up[l]])
      return fail(c, XT_EINVAL, "load_atomic_data: line " + std::to_string(l) + " needs 0 <= lo < up < nlev in one ion");
    if (!(lam[l] > 0) || !(f[l] > 0))
      return fail(c, XT_EINVAL, "load_atomic_data: lambda_A and f_lu must be > 0 (line " + std::to_string(l) + ")");
  }
  // descending frequency, ties in ascending caller index
  std::vector<double> nu(nl);
  for (int l = 0; l < nl; ++l) nu[l] = kC / (lam[l] * 1e-8);
  std::vector<int> order(nl);
  sort_lines_by_frequency(nu.data(), nl, order.data());
  c->h_orig_of = order;
  c->h_sorted_of.assign(nl, 0);
  for (int s = 0; s < nl; ++s) c->h_sorted_of[order[s]] = s;
  const double pie2mc = kPi * kE * kE / (kMe * kC);
  std::vector<double> s_nu(nl), s_K(nl), s_gr(nl), s_hnu(nl), s_A(nl), s_invB(nl);
  std::vector<int> s_lo(nl), s_up(nl);
  for (int s = 0; s < nl; ++s) {
    int l = order[s];
    double lc = lam[l] * 1e-8;
    s_nu[s] = nu[l];
    s_K[s] = pie2mc * f[l] * lc * c->t;
    s_gr[s] = g[lo[l]] / g[up[l]];
    s_hnu[s] = kH * nu[l];
    s_A[s] = 8.0 * kPi * kPi * kE * kE / (kMe * kC * lc * lc) * s_gr[s] * f[l];
    s_invB[s] = kH * nu[l] / (4.0 * kPi * pie2mc * f[l]);
    s_lo[s] = lo[l];
    s_up[s] = up[l];
  }
  // radiative down-lines per upper level, ascending caller index
  std::vector<int> doff(nlev + 1, 0), dline(nl);
  for (int l = 0; l < nl; ++l) doff[up[l] + 1]++;
  for (int u = 0; u < nlev; ++u) doff[u + 1] += doff[u];
  std::vector<int> fill(nlev, 0), dpos(nl);
  for (int l = 0; l < nl; ++l) {
    dpos[l] = doff[up[l]] + fill[up[l]]++;
    dline[dpos[l]] = c->h_sorted_of[l];
  }
  // radiative lines per lower level, ascending caller index, as their
  // positions in the down-line lists
  std::vector<int> loff(nlev + 1, 0), lline(nl);
  for (int l = 0; l < nl; ++l) loff[lo[l] + 1]++;
  for (int i = 0; i < nlev; ++i) loff[i + 1] += loff[i];
  std::vector<int> lfill(nlev, 0);
  for (int l = 0; l < nl; ++l) lline[loff[lo[l]] + lfill[lo[l]]++] = dpos[l];
  c->n_ion = a->n_ion; c->nlev = nlev; c->nline = nl;
  c->h_nu_sorted = s_nu;
  c->h_lam_caller = lam;
  c->h_level_off = off; c->h_g = g; c->h_E = E;
  if ((rc = to_device(c, off, &c->d_level_off, "level_off"))) return rc;
  if ((rc = to_device(c, g, &c->d_g, "g"))) return rc;
  if ((rc = to_device(c, E, &c->d_E, "E"))) return rc;
  std::vector<double> packed(4 * (size_t)nl);
  for (int s = 0; s < nl; ++s) {
    packed[4 * s] = s_nu[s];
    packed[4 * s + 1] = s_K[s];
    packed[4 * s + 2] = s_gr[s];
    int64_t lu = (int64_t)(uint32_t)s_lo[s] | ((int64_t)s_up[s] << 32);
    std::memcpy(&packed[4 * s + 3], &lu, sizeof(lu));
  }
  if ((rc = to_device(c, packed, &c->d_lines, "line table"))) return rc;
  if ((rc = to_device(c, s_nu, &c->d_nu, "nu"))) return rc;
  if ((rc = to_device(c, s_K, &c->d_K, "K"))) return rc;
  if ((rc = to_device(c, s_gr, &c->d_gratio, "gratio"))) return rc;
  if ((rc = to_device(c, s_hnu, &c->d_hnu, "hnu"))) return rc;
  if ((rc = to_device(c, s_A, &c->d_A, "A"))) return rc;
  if ((rc = to_device(c, s_invB, &c->d_invB, "invB"))) return rc;
  if ((rc = to_device(c, s_lo, &c->d_lo, "lo"))) return rc;
  if ((rc = to_device(c, s_up, &c->d_up, "up"))) return rc;
  if ((rc = to_device(c, c->h_sorted_of, &c->d_orig, "sorted_of"))) return rc;
  if ((rc = to_device(c, doff, &c->d_down_off, "down_off"))) return rc;
  if ((rc = to_device(c, dline, &c->d_down_line, "down_line"))) return rc;
  if ((rc = to_device(c, loff, &c->d_low_off, "low_off"))) return rc;
  if ((rc = to_device(c, lline, &c->d_low_line, "low_line"))) return rc;
  if ((rc = to_device(c, ups, &c->d_ups_down, "ups_down"))) return rc;
  if (a->n_ion_density && (rc = upload_rows(c, a->n_ion_density, &c->d_nion, a->n_ion, "n_ion_density")))
    return rc;
  if ((rc = load_photoionization(c, a, off, E))) return rc;
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  c->have_atoms = true;
  c->have_pops = c->have_S = false;
  c->qoff_N = -1;
  return XT_OK;
}

int set_populations(xt_ctx* c, const double* pops) {
  if (!c || !pops) return fail(c, XT_EINVAL, "set_populations: null argument");
  if (!c->have_atoms) return fail(c, XT_ESTATE, "set_populations: load_atomic_data first");
  cudaSetDevice(c->device);
  int rc;
  // sized for the current grid and atoms (alloc keeps a buffer of that size;
  // a context reloaded with another grid gets a new one)
  if ((rc = upload_rows(c, pops, &c->d_pops, c->nlev, "pops"))) return rc;
  c->have_pops = true;
  c->have_S = false;     // estimators refer to the populations of their transport pass
  if (c->qoff_mode == XT_EMIT_LINES) c->qoff_N = -1;
  return XT_OK;
}

int get_populations(xt_ctx* c, double* pops, size_t n_cap) {
  if (!c || !pops) return fail(c, XT_EINVAL, "get_populations: null argument");
  if (!c->have_pops) return fail(c, XT_ESTATE, "get_populations: no populations");
  size_t n = (size_t)c->geo.ncell * c->nlev;
  if (n_cap < n) return fail(c, XT_EINVAL, "get_populations: n_cap < ncell*nlev");
  cudaSetDevice(c->device);
  int rc = deliver(c, pops, n * sizeof(double), [&](void* d) {
    k_row_to_nat<<<grid_blocks((int64_t)n, 256), 256, 0, c->stream>>>(c->geo, c->d_pops, (double*)d, c->nlev);
  });
  if (rc) return rc;
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  return XT_OK;
}

static LineTable line_table(xt_ctx* c) {
  LineTable L;
  L.nline = c->nline; L.nlev = c->nlev;
  L.nu = c->d_nu; L.K = c->d_K; L.gratio = c->d_gratio; L.hnu = c->d_hnu; L.A = c->d_A;
  L.lo = c->d_lo; L.up = c->d_up; L.down_off = c->d_down_off; L.down_line = c->d_down_line;
  return L;
}

static int check_range(xt_ctx* c, int64_t c0, int64_t nc, const char* who) {
  if (c0 < 0 || nc < 0 || c0 + nc > c->geo.ncell)
    return fail(c, XT_EINVAL, std::string(who) + ": cell range outside the grid");
  return XT_OK;
}

int get_sobolev_tau(xt_ctx* c, int64_t c0, int64_t nc, double* tau, double* beta) {
  if (!c) return XT_EINVAL;
  if (!c->have_pops) return fail(c, XT_ESTATE, "get_sobolev_tau: set_populations first");
  int rc = check_range(c, c0, nc, "get_sobolev_tau");
  if (rc) return rc;
  cudaSetDevice(c->device);
  LineTable L = line_table(c);
  size_t bytes = (size_t)nc * c->nline * sizeof(double);
  int64_t n = nc * c->nline;
  if (tau && (rc = deliver(c, tau, bytes, [&](void* d) {
        k_tau_beta<<<grid_blocks(n, 256), 256, 0, c->stream>>>(c->geo, L, c->d_pops, c->d_orig, c0, nc, (double*)d, nullptr);
      }))) return rc;
  if (beta) {
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
    if ((rc = deliver(c, beta, bytes, [&](void* d) {
          k_tau_beta<<<grid_blocks(n, 256), 256, 0, c->stream>>>(c->geo, L, c->d_pops, c->d_orig, c0, nc, nullptr, (double*)d);
        }))) return rc;
  }
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  return XT_OK;
}

static int rates_common(xt_ctx* c, int64_t c0, int64_t nc, double* out, int which) {
  LineTable L = line_table(c);
  double V = c->geo.dx * c->geo.dy * c->geo.dz;
  if (c->S_groups > 0) {
    // host-held store: a group's cells are a contiguous natural range (whole
    // x-y layers) and its rows a contiguous slab; stage each group the range
    // touches on the device and read it with the slab's rows offset
    const Geometry& G = c->geo;
    const int NG = c->S_groups;
    const int64_t cells_g = G.ncell / NG;
    const size_t slab_n = (size_t)cells_g * c->nline;
    int rc;
    for (int g = (int)(c0 / cells_g); g < NG && (int64_t)g * cells_g < c0 + nc; ++g) {
      const int64_t a = std::max<int64_t>(c0, (int64_t)g * cells_g);
      const int64_t b = std::min<int64_t>(c0 + nc, (int64_t)(g + 1) * cells_g);
      if (c->S_valid.size() == (size_t)NG && c->S_valid[g])
        XT_CUDA(c, cudaMemcpyAsync(c->d_S, c->h_S + (size_t)g * slab_n, slab_n * sizeof(double),
                                   cudaMemcpyHostToDevice, c->stream));
      else
        XT_CUDA(c, cudaMemsetAsync(c->d_S, 0, slab_n * sizeof(double), c->stream));
      const double* Sg = c->d_S - (int64_t)g * (int64_t)slab_n;   // row r of the slab at S + r nline
      double* o = out + (size_t)(a - c0) * c->nline;
      const int64_t n = (b - a) * c->nline;
      rc = deliver(c, o, (size_t)n * sizeof(double), [&](void* d) {
        k_rates<<<(int)std::max<int64_t>(1, std::min<int64_t>(b - a, 152 * 16)), 256, 0, c->stream>>>(
            G, L, c->d_pops, Sg, c->d_invB, c->d_orig, a, b - a, V, which, (double*)d, nullptr);
      });
      if (rc) return rc;
      XT_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return XT_OK;
  }
  size_t bytes = (size_t)nc * c->nline * sizeof(double);
  int rc = deliver(c, out, bytes, [&](void* d) {
    k_rates<<<(int)std::max<int64_t>(1, std::min<int64_t>(nc, 152 * 16)), 256, 0, c->stream>>>(
        c->geo, L, c->d_pops, c->d_S, c->d_invB, c->d_orig, c0, nc, V, which, (double*)d,
        c->S_compact ? c->d_crow : nullptr);
  });
  if (rc) return rc;
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  return XT_OK;
}

int set_estimator_store(xt_ctx* c, int32_t host_groups) {
  if (!c) return XT_EINVAL;
  if (!c->have_grid || !c->have_atoms) return fail(c, XT_ESTATE, "set_estimator_store: init_grid and load_atomic_data first");
  if (host_groups < XT_STORE_COMPACT_ROWS)
    return fail(c, XT_EINVAL, "set_estimator_store: host_groups >= 0 or XT_STORE_COMPACT_ROWS");
  if (host_groups > 0 && (c->sz % host_groups != 0))
    return fail(c, XT_EINVAL, "set_estimator_store: host_groups must divide the subdomains along z (" +
                                  std::to_string(c->sz) + ")");
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  release((void**)&c->d_S);
  c->S_bytes = 0;
  if (c->h_S) cudaFreeHost(c->h_S);
  c->h_S = nullptr;
  c->h_S_bytes = 0;
  c->S_valid.clear();
  c->S_compact = host_groups == XT_STORE_COMPACT_ROWS;
  c->S_groups = host_groups > 0 ? host_groups : 0;
  c->h_crow.clear();
  c->n_crow = 0;
  c->have_S = false;
  c->slotlog_valid = true;
  c->slotlog_n = 0;
  c->log_nseg = 0;
  return XT_OK;
}

int get_estimators(xt_ctx* c, int64_t c0, int64_t nc, double* S) {
  if (!c || !S) return fail(c, XT_EINVAL, "get_estimators: null argument");
  if (!c->have_S) return fail(c, XT_ESTATE, "get_estimators: run_transport first");
  int rc = check_range(c, c0, nc, "get_estimators");
  if (rc) return rc;
  cudaSetDevice(c->device);
  return rates_common(c, c0, nc, S, 0);
}

int get_photoexcitation_rates(xt_ctx* c, int64_t c0, int64_t nc, double* R_lu, double* R_ul, double* Jbar) {
  if (!c) return XT_EINVAL;
  if (!c->have_S) return fail(c, XT_ESTATE, "get_photoexcitation_rates: run_transport first");
  int rc = check_range(c, c0, nc, "get_photoexcitation_rates");
  if (rc) return rc;
  cudaSetDevice(c->device);
  if (R_lu && (rc = rates_common(c, c0, nc, R_lu, 1))) return rc;
  if (R_ul && (rc = rates_common(c, c0, nc, R_ul, 2))) return rc;
  if (Jbar && (rc = rates_common(c, c0, nc, Jbar, 3))) return rc;
  return XT_OK;
}

// Photoionization rates Gamma_k = N_abs,k / (n_k V) and heating per cell
// (Sec. 2.3.1) from the pass's per-cell accumulators: a segment that
// photoionized over length d added X d (X = N beta(tau) lambda^3, beta =
// (1 - e^-tau) / tau) to G[row][b], b its first level with the whole length,
// and X d_k to D[row][k] for a level k whose threshold it crossed after d_k;
// level k (sorted) then absorbed N_abs,k = sig_k n_k (sum_{b <= k} G[b] + D[k]).
// Heating = h sum (N_abs nu) - sum_k N_abs,k chi_k.  A thread per cell.
__global__ void k_pi_rates(Geometry g, int npi, const double* __restrict__ pops, int nlev,
                           const double* __restrict__ G, const double* __restrict__ D,
                           const double* __restrict__ H, const double* __restrict__ sig,
                           const double* __restrict__ chi, const int* __restrict__ lev,
                           int64_t c0, int64_t nc, double V, double* __restrict__ Gamma,
                           double* __restrict__ heat) {
  for (int64_t cl = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cl < nc;
       cl += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = c0 + cl;
    const int ix = (int)(c % g.nx), iy = (int)((c / g.nx) % g.ny), iz = (int)(c / ((int64_t)g.nx * g.ny));
    const int64_t row = row_of(g, ix, iy, iz);
    const double* Gr = G + row * (npi + 1);
    const double* Dr = D + row * npi;
    const double* pr = pops + row * nlev;
    double run = 0.0, absorbed = 0.0;
    for (int s = 0; s < npi; ++s) {
      run += Gr[s];
      const double n = pr[lev[s]];
      const double Nabs = sig[s] * n * (run + Dr[s]);
      absorbed += Nabs * chi[s];
      if (Gamma) Gamma[cl * npi + s] = n > 0.0 ? Nabs / (n * (g.vol ? g.vol[row] : V)) : 0.0;
    }
    if (heat) heat[cl] = kH * H[row] - absorbed;
  }
}

// Sorted level order to the caller's, row by row (in place through a copy).
__global__ void k_pi_reorder(const double* __restrict__ in, const int* __restrict__ sorted_of, int npi,
                             int64_t nc, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc * npi;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cl = i / npi;
    const int k = (int)(i - cl * npi);
    out[i] = in[cl * npi + sorted_of[k]];
  }
}

int get_photoionization_rates(xt_ctx* c, int64_t c0, int64_t nc, double* Gamma, double* heating) {
  if (!c) return XT_EINVAL;
  if (!c->have_pi || !c->have_S)
    return fail(c, XT_ESTATE, "get_photoionization_rates: no attenuation pass with photoionization data");
  int rc = check_range(c, c0, nc, "get_photoionization_rates");
  if (rc) return rc;
  cudaSetDevice(c->device);
  const Geometry& G = c->geo;
  const double V = G.dx * G.dy * G.dz;
  const int npi = c->npi;
  const int blocks = grid_blocks(std::max<int64_t>(nc, 1), 128);
  // Gamma: sorted order into the first half of the scratch, then reordered
  const size_t gb = (size_t)nc * npi * sizeof(double), hb = (size_t)nc * sizeof(double);
  if (Gamma) {
    if ((rc = ensure_scratch(c, 2 * gb + hb))) return rc;
    double* tmp = (double*)c->d_scratch;
    k_pi_rates<<<blocks, 128, 0, c->stream>>>(G, npi, c->d_pops, c->nlev, c->d_piG, c->d_piD, c->d_piH,
                                             c->d_pi_sig, c->d_pi_chi, c->d_pi_lev, c0, nc, V, tmp,
                                             nullptr);
    XT_CUDA(c, cudaGetLastError());
    double* dst = is_device_ptr(Gamma) ? Gamma : tmp + (size_t)nc * npi;
    k_pi_reorder<<<grid_blocks(std::max<int64_t>(nc * npi, 1), 256), 256, 0, c->stream>>>(
        tmp, c->d_pi_sorted_of, npi, nc, dst);
    XT_CUDA(c, cudaGetLastError());
    if (dst != Gamma && (rc = copy(c, Gamma, dst, gb, "photoionization rates"))) return rc;
  }
  if (heating) {
    rc = deliver(c, heating, hb, [&](void* d) {
      k_pi_rates<<<blocks, 128, 0, c->stream>>>(G, npi, c->d_pops, c->nlev, c->d_piG, c->d_piD, c->d_piH,
                                               c->d_pi_sig, c->d_pi_chi, c->d_pi_lev, c0, nc, V, nullptr,
                                               (double*)d);
    });
    if (rc) return rc;
  }
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  return XT_OK;
}

int get_spectrum(xt_ctx* c, int32_t kind, double* out, size_t n_cap) {
  if (!c || !out) return fail(c, XT_EINVAL, "get_spectrum: null argument");
  if (!c->d_spec) return fail(c, XT_ESTATE, "get_spectrum: run_transport first");
  if (kind < 0 || kind > 2) return fail(c, XT_EINVAL, "get_spectrum: kind must be 0, 1 or 2");
  size_t n = kind == 2 ? (size_t)c->spec_bins : (size_t)c->spec_views * c->spec_bins;
  if (n_cap < n) return fail(c, XT_EINVAL, "get_spectrum: n_cap too small");
  cudaSetDevice(c->device);
  int rc = deliver(c, out, n * sizeof(double), [&](void* d) {
    k_spectrum<<<grid_blocks((int64_t)n, 256), 256, 0, c->stream>>>(c->d_spec, c->n_theta, c->n_phi, c->spec_bins, c->spec_lam0, c->spec_dlog, kind, (double*)d);
  });
  if (rc) return rc;
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  return XT_OK;
}

int xt_selftest_fixed(int32_t kind, const double* x, int64_t n, double* y0, double* y1,
                      double* r0, double* r1) {
  if (!x || n < 0 || !y0 || !y1 || kind < 0 || kind > 3) return XT_EINVAL;
  const int64_t nin = kind >= 2 ? 2 * n : n;       // kinds 2 and 3 read pairs
  FixExpTables T;
  fixexp_tables(&T);
  FixTrigTables R;
  fixtrig_tables(&R);
  const size_t b = (size_t)n * sizeof(double);
  double* d = nullptr;
  if (cudaMalloc(&d, 6 * b + 8) != cudaSuccess) { cudaGetLastError(); return XT_ENOMEM; }
  cudaMemcpy(d, x, (size_t)nin * sizeof(double), cudaMemcpyDefault);
  double* o = d + nin;
  k_selftest_fixed<<<grid_blocks(n, 256), 256>>>(kind, T, R, d, n, o, o + n, o + 2 * n, o + 3 * n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) {
    cudaMemcpy(y0, o, b, cudaMemcpyDefault);
    cudaMemcpy(y1, o + n, b, cudaMemcpyDefault);
    if (r0) cudaMemcpy(r0, o + 2 * n, b, cudaMemcpyDefault);
    if (r1) cudaMemcpy(r1, o + 3 * n, b, cudaMemcpyDefault);
  }
  cudaFree(d);
  return e == cudaSuccess ? XT_OK : XT_ECUDA;
}

int get_sizes(xt_ctx* c, xt_sizes* o) {
  if (!c || !o) return XT_EINVAL;
  o->ncell = c->geo.ncell; o->nlev = c->nlev; o->nline = c->nline; o->n_ion = c->n_ion;
  o->spec_views = c->spec_views; o->spec_bins = c->spec_bins;
  o->store_bytes = (int64_t)c->S_bytes;
  o->n_pi = c->npi;
  return XT_OK;
}

}  // extern "C"
