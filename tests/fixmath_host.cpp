// The library's fixed-point routines (fixexp.cuh), its Philox generator and
// its packet quota compiled for the host, with C entry points for a CPU test.
// Test infrastructure only.
#define XT_FIXEXP_HOST
#include "fixexp.cuh"
#include "philox.cuh"
#include "quota.h"
#include "linesort.h"
#include "raysched.h"

using namespace xt;

extern "C" {

void h_div_pos(const double* a, const double* b, double* q, long n) {
  for (long i = 0; i < n; ++i) q[i] = div_pos(a[i], b[i]);
}

void h_expneg(const double* tau, double* ex, double* ome, long n) {
  FixExpTables T;
  fixexp_tables(&T);
  for (long i = 0; i < n; ++i) expneg(T, tau[i], ex[i], ome[i]);
}

void h_sincos(const uint64_t* U, double* s, double* c, long n) {
  FixTrigTables T;
  fixtrig_tables(&T);
  for (long i = 0; i < n; ++i) sincos_2pi(T, U[i], s[i], c[i]);
}

void h_isotropic(const uint64_t* Umu, const uint64_t* Uphi, double* nx, double* ny, double* nz, long n) {
  FixTrigTables T;
  fixtrig_tables(&T);
  for (long i = 0; i < n; ++i) {
    double v[3];
    isotropic_fix(T, Umu[i], Uphi[i], v);
    nx[i] = v[0]; ny[i] = v[1]; nz[i] = v[2];
  }
}

void h_beta(const double* tau, double* beta, double* dbeta, long n) {
  FixExpTables T;
  fixexp_tables(&T);
  for (long i = 0; i < n; ++i) beta[i] = sobolev_beta_fix(T, tau[i], &dbeta[i]);
}

void h_scaled_f32(const double* w, const int* k, float* out, long n) {
  for (long i = 0; i < n; ++i) out[i] = scaled_f32(w[i], k[i]);
}

void h_philox(const uint64_t* ctr, const uint64_t* key, uint64_t* out, long n) {
  for (long i = 0; i < n; ++i)
    philox4x64_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], key[2 * i], key[2 * i + 1],
                  out + 4 * i);
}

void h_u01(const uint64_t* x, double* out, long n) {
  for (long i = 0; i < n; ++i) out[i] = u01(x[i]);
}

void h_linesort(const double* nu, int n, int* order) { sort_lines_by_frequency(nu, n, order); }

void h_rayids(int64_t p_begin, int64_t n, int64_t nbin, int64_t nview, int64_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = ray_id_in_range(p_begin + i, p_begin, n, nbin, nview);
}

void h_quota(const double* L, long nc, long N, int64_t* qoff) {
  std::vector<double> Lv(L, L + nc);
  std::vector<int64_t> q;
  packet_quota(Lv, (int64_t)N, q);
  for (long i = 0; i <= nc; ++i) qoff[i] = q[i];
}

}  // extern "C"
