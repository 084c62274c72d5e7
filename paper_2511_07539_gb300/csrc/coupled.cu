// A10: the coupled NLTE / transport loop (Sec. 2: the NLTE solver and the ray
// tracing alternate; Sec. 2.2: populations from the rates with the transport's
// photoexcitation held fixed; Sec. 2.3.2: those rates from the estimators).
//
// One outer step: a transport pass from the context's populations n_k, the
// statistical-equilibrium solve with its estimator rates (s_k), then on the
// device n_{k+1} = n_k^(1-alpha) s_k^alpha and the largest relative change
// over the levels that count, of which only that one double comes back to the
// host.  The loop ends when the change is at most tol.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "xt_internal.cuh"

namespace xt {

// n_new <- relax(n_old, n_new); *change = max |n_new - n_old| / n_old over the
// levels with max(n_old, n_new) >= floor n_z (n_z > 0, n_old > 0).  Rows in
// the blocked order of both arrays; the change is a non-negative double kept
// as its bit pattern, whose integer order is its numeric order.
__global__ void k_relax(int64_t ncell, int nlev, int n_ion, const int* __restrict__ level_off,
                        const double* __restrict__ nion, const double* __restrict__ old,
                        double* __restrict__ nw, double alpha, double floor,
                        unsigned long long* __restrict__ change) {
  __shared__ int s_off[17];
  __shared__ double red[32];
  if (threadIdx.x <= n_ion) s_off[threadIdx.x] = level_off[threadIdx.x];
  __syncthreads();
  const int64_t n = ncell * nlev;
  double ch = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / nlev;
    const int lev = (int)(e - row * nlev);
    int z = 0;
    while (z + 1 < n_ion && s_off[z + 1] <= lev) ++z;
    const double nz = nion[row * n_ion + z];
    const double o = old[e], s = nw[e];
    double m = s;
    if (alpha != 1.0 && o > 0.0 && s > 0.0) m = exp((1.0 - alpha) * log(o) + alpha * log(s));
    nw[e] = m;
    if (nz > 0.0 && o > 0.0 && fmax(o, m) >= floor * nz) ch = fmax(ch, fabs(m - o) / o);
  }
  for (int k = 16; k > 0; k >>= 1) ch = fmax(ch, __shfl_xor_sync(0xffffffffu, ch, k));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ch;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmax(t, red[k]);
    atomicMax(change, (unsigned long long)__double_as_longlong(t));
  }
}

}  // namespace xt

using namespace xt;

extern "C" int run_coupled(xt_ctx* c, const xt_coupled_params* p, xt_coupled_stats* out) {
  if (!c || !p || !p->transport || !p->nlte) return fail(c, XT_EINVAL, "run_coupled: null argument");
  if (!c->have_grid || !c->have_atoms || !c->d_nion) return fail(c, XT_ESTATE, "run_coupled: init_grid and load_atomic_data (with n_ion_density) first");
  if (!(p->alpha > 0 && p->alpha <= 1) || !(p->tol > 0) || !(p->floor >= 0) || p->max_outer < 1)
    return fail(c, XT_EINVAL, "run_coupled: 0 < alpha <= 1, tol > 0, floor >= 0, max_outer >= 1");
  if (p->start < XT_WARM_CURRENT || p->start > XT_WARM_SURROGATE) return fail(c, XT_EINVAL, "run_coupled: start");
  if (p->start == XT_WARM_GIVEN && !p->start_in) return fail(c, XT_EINVAL, "run_coupled: start_in required");
  if (p->start == XT_WARM_CURRENT && !c->have_pops) return fail(c, XT_ESTATE, "run_coupled: no current populations");
  if (p->start == XT_WARM_SURROGATE && !(p->nlte->jbar_W > 0 && p->nlte->jbar_TR > 0))
    return fail(c, XT_EINVAL, "run_coupled: the surrogate start reads its Jbar inputs from nlte->jbar_W, jbar_TR");
  if (c->n_ion > 16) return fail(c, XT_EINVAL, "run_coupled: at most 16 ions");
  cudaSetDevice(c->device);
  const auto t0 = std::chrono::steady_clock::now();
  const Geometry& G = c->geo;
  const size_t pops_n = (size_t)G.ncell * c->nlev;
  int rc;
  xt_coupled_stats st;
  std::memset(&st, 0, sizeof(st));
  // levels kept, on the device, for the start populations
  int* d_used = nullptr;
  if (p->nlte->levels_used && p->start != XT_WARM_CURRENT && p->start != XT_WARM_GIVEN) {
    const size_t nb = (size_t)G.ncell * c->n_ion * sizeof(int);
    if ((rc = alloc(c, (void**)&d_used, nb, "levels used"))) return rc;
    if ((rc = copy(c, d_used, p->nlte->levels_used, nb, "levels used"))) { release((void**)&d_used); return rc; }
  }
  auto finish = [&](int code) {
    release((void**)&d_used);
    return code;
  };
  // ---- start populations
  if (p->start == XT_WARM_GIVEN) {
    if ((rc = set_populations(c, p->start_in))) return finish(rc);
  } else if (p->start == XT_WARM_LTE || p->start == XT_WARM_SURROGATE) {
    // sized for the current grid and atoms (alloc keeps a buffer of that size)
    if ((rc = alloc(c, (void**)&c->d_pops, pops_n * sizeof(double), "pops"))) return finish(rc);
    if (p->start == XT_WARM_LTE) rc = lte_fill(c, d_used, c->d_pops);
    else rc = surrogate_warm(c, XT_RATES_JBAR, p->nlte->jbar_W, p->nlte->jbar_TR, d_used, c->d_pops);
    if (rc) return finish(rc);
    c->have_pops = true;
    c->have_S = false;
    if (c->qoff_mode == XT_EMIT_LINES) c->qoff_N = -1;
  }
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  st.start_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  unsigned long long* d_change = nullptr;
  if ((rc = alloc(c, (void**)&d_change, sizeof(unsigned long long), "change"))) return finish(rc);
  auto finish2 = [&](int code) {
    release((void**)&d_change);
    return finish(code);
  };
  xt_transport_params tp = *p->transport;
  tp.accumulate = 0;
  xt_nlte_params np = *p->nlte;
  np.rates = XT_RATES_ESTIMATORS;
  np.warm = XT_WARM_CURRENT;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)(pops_n + 255) / 256, (int64_t)sms * 8));
  for (int k = 0; k < p->max_outer; ++k) {
    xt_transport_stats ts;
    if ((rc = run_transport(c, &tp, &ts))) return finish2(rc);
    xt_nlte_stats ns;
    // the solve swaps buffers: afterwards d_pops holds s_k, se.pops_new n_k
    if ((rc = solve_nlte(c, &np, nullptr, nullptr, &ns))) return finish2(rc);
    XT_CUDA(c, cudaMemsetAsync(d_change, 0, sizeof(unsigned long long), c->stream));
    XT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
    k_relax<<<blocks, 256, 0, c->stream>>>(G.ncell, c->nlev, c->n_ion, c->d_level_off, c->d_nion,
                                           c->se.pops_new, c->d_pops, p->alpha, p->floor, d_change);
    XT_CUDA(c, cudaGetLastError());
    XT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
    unsigned long long bits = 0;
    XT_CUDA(c, cudaMemcpyAsync(&bits, d_change, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
    float ms = 0;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    double ch;
    std::memcpy(&ch, &bits, sizeof(ch));
    c->have_S = false;                       // the estimators belong to n_k
    if (c->qoff_mode == XT_EMIT_LINES) c->qoff_N = -1;
    st.transport_ms += ts.transport_ms;
    st.solve_ms += ns.solve_ms;
    st.mix_ms += ms;
    st.newton_steps += ns.mean_iter;
    st.max_newton_steps = std::max(st.max_newton_steps, ns.max_iter_used);
    st.not_converged += ns.not_converged;
    st.fp64_fallbacks += ns.fp64_fallbacks;
    if (k < 64) st.change[k] = ch;
    st.outer = k + 1;
    st.last_change = ch;
    if (ch <= p->tol) { st.converged = 1; break; }
  }
  st.wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (out) *out = st;
  return finish2(XT_OK);
}
