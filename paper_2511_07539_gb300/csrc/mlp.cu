// A9: the population surrogate network (not in the paper; it warm-starts the
// statistical-equilibrium solves).  Input: log10 n_e, log10 Te, log10 of the
// deposition, per ion the mean log10 Jbar of its lines in 32 log-lambda bins,
// and per ion log10 n_z / 10 (it sets the optical depths); output: log10(n_i / n_z) / 10 of every level (clipped at -30 in
// log10, masked beyond the kept levels).  Hidden layers GELU (tanh form,
// Hendrycks & Gimpel 2016), linear output; masked mean squared error; Adam
// (Kingma & Ba 2015) on FP32 master weights.  Training runs in the fused
// kernel of mlp_train.cu (tcgen05 MMAs, every step in one launch); this file
// holds the network's setup, the training loop's batches and the prediction
// forward pass, whose products (batches of up to every cell) run in BF16
// with FP32 accumulation (warp-level mma.sync m16n8k16).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "mlp.cuh"
#include "philox.cuh"
#include "xt_internal.cuh"

namespace xt {

// ---------------------------------------------------------------- BF16 GEMM
// C[m][n] = sum_k A(m, k) B(k, n), A(m, k) = A[m sam + k sak], B(k, n) =
// B[k sbk + n sbn] (bf16), C fp32 row-major [M][ldc].  Epilogue: optional
// bias[n], optional GELU written as bf16 to H (the FP32 pre-activation to C).
constexpr int GBM = 64, GBN = 64, GBK = 32;

struct GemmArgs {
  const __nv_bfloat16* A; int64_t sam, sak;
  const __nv_bfloat16* B; int64_t sbk, sbn;
  float* C; int64_t ldc;
  const float* bias;
  __nv_bfloat16* H; int64_t ldh;   // GELU(C + bias) as bf16 (optional)
  int M, N, K;
};

__device__ __forceinline__ float gelu_f(float z) {
  const float u = 0.7978845608028654f * (z + 0.044715f * z * z * z);
  return 0.5f * z * (1.0f + tanhf(u));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__global__ void __launch_bounds__(128) k_gemm_bf16(const GemmArgs g) {
  __shared__ __nv_bfloat16 As[GBM][GBK + 8];
  __shared__ __nv_bfloat16 Bs[GBK][GBN + 8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < g.K; k0 += GBK) {
    for (int e = tid; e < GBM * GBK; e += 128) {
      const int r = e / GBK, kk = e - r * GBK;
      const int m = m0 + r, k = k0 + kk;
      As[r][kk] = (m < g.M && k < g.K) ? g.A[m * g.sam + k * g.sak] : zero;
    }
    for (int e = tid; e < GBK * GBN; e += 128) {
      const int kk = e / GBN, c = e - kk * GBN;
      const int k = k0 + kk, n = n0 + c;
      Bs[kk][c] = (k < g.K && n < g.N) ? g.B[k * g.sbk + n * g.sbn] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + gid;
        af[i][0] = pack2(As[r][ks + 2 * tig], As[r][ks + 2 * tig + 1]);
        af[i][1] = pack2(As[r + 8][ks + 2 * tig], As[r + 8][ks + 2 * tig + 1]);
        af[i][2] = pack2(As[r][ks + 2 * tig + 8], As[r][ks + 2 * tig + 9]);
        af[i][3] = pack2(As[r + 8][ks + 2 * tig + 8], As[r + 8][ks + 2 * tig + 9]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + gid;
        bfr[j][0] = pack2(Bs[ks + 2 * tig][c], Bs[ks + 2 * tig + 1][c]);
        bfr[j][1] = pack2(Bs[ks + 2 * tig + 8][c], Bs[ks + 2 * tig + 9][c]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
              "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]),
                "r"(bfr[j][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + i * 16 + gid + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + 2 * tig + (q & 1);
        if (m < g.M && n < g.N) {
          float v = acc[i][j][q] + (g.bias ? g.bias[n] : 0.f);
          g.C[(int64_t)m * g.ldc + n] = v;
          if (g.H) g.H[(int64_t)m * g.ldh + n] = __float2bfloat16(gelu_f(v));
        }
      }
}

__global__ void k_to_bf16(const float* __restrict__ x, int64_t n, __nv_bfloat16* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

__global__ void k_init_w(float* w, int64_t n, float scale, uint64_t seed, uint64_t stream) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t x[4];
    philox4x64_10((uint64_t)i, stream, 0, 0, seed, 0x5375727261ull, x);
    // Box-Muller from two uniforms
    const double u1 = ((double)(x[0] >> 11) + 0.5) * 0x1.0p-53, u2 = (double)(x[1] >> 11) * 0x1.0p-53;
    w[i] = (float)(scale * sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2));
  }
}

static int gb(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 152 * 16); }

}  // namespace xt

using namespace xt;

int xt_mlp_step(xt_ctx* c, int64_t B, double msum, double lr, int update, float* grads_out,
                double* loss_out);

static void mlp_free(xt_mlp* n) {
  if (!n) return;
  void** ps[] = {(void**)&n->w,     (void**)&n->m,     (void**)&n->v,     (void**)&n->g,
                 (void**)&n->wb,    (void**)&n->wp,    (void**)&n->wt,    (void**)&n->X,
                 (void**)&n->dz[0], (void**)&n->dz[1], (void**)&n->T,     (void**)&n->M,
                 (void**)&n->dzT[0], (void**)&n->dzT[1],
                 (void**)&n->loss,  (void**)&n->msum1, (void**)&n->st,    (void**)&n->bar};
  for (void** p : ps) release(p);
  for (auto& p : n->Z) release((void**)&p);
  for (auto& p : n->H) release((void**)&p);
  for (auto& p : n->hp) release((void**)&p);
  for (auto& p : n->zp) release((void**)&p);
  for (auto& p : n->hT) release((void**)&p);
}

namespace xt {
void mlp_destroy(xt_mlp* n) {
  mlp_free(n);
  delete n;
}
}  // namespace xt

// Prediction buffers for batches of up to B rows.
static int mlp_ensure_batch(xt_ctx* c, xt_mlp* n, int64_t B) {
  if (B <= n->cap) return XT_OK;
  int rc;
  const int L = (int)n->sizes.size() - 1;
  for (auto& q : n->Z) release((void**)&q);
  for (auto& q : n->H) release((void**)&q);
  n->Z.assign(L + 1, nullptr);
  n->H.assign(L + 1, nullptr);
  for (int k = 0; k <= L; ++k) {
    if (k > 0 && (rc = alloc(c, (void**)&n->Z[k], (size_t)B * n->sizes[k] * 4, "mlp activations"))) return rc;
    if ((rc = alloc(c, (void**)&n->H[k], (size_t)B * n->sizes[k] * 2, "mlp activations"))) return rc;
  }
  if ((rc = alloc(c, (void**)&n->X, (size_t)B * n->sizes[0] * 4, "mlp input"))) return rc;
  n->cap = B;
  return XT_OK;
}

static void gemm(cudaStream_t s, const __nv_bfloat16* A, int64_t sam, int64_t sak, const __nv_bfloat16* B,
                 int64_t sbk, int64_t sbn, float* C, int64_t ldc, const float* bias, __nv_bfloat16* H,
                 int64_t ldh, int M, int N, int K) {
  GemmArgs g{A, sam, sak, B, sbk, sbn, C, ldc, bias, H, ldh, M, N, K};
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
  k_gemm_bf16<<<grid, 128, 0, s>>>(g);
}

// Forward on n->H[0] (bf16 input, B rows); output fp32 in n->Z[L].
static void mlp_forward(xt_ctx* c, xt_mlp* n, int64_t B) {
  const int L = (int)n->sizes.size() - 1;
  for (int k = 1; k <= L; ++k) {
    const int fi = n->sizes[k - 1], fo = n->sizes[k];
    gemm(c->stream, n->H[k - 1], fi, 1, n->wb + n->woff[k - 1], fo, 1, n->Z[k], fo,
         n->w + n->boff[k - 1], k < L ? n->H[k] : nullptr, fo, (int)B, fo, fi);
  }
}

extern "C" {

int surrogate_init(xt_ctx* c, const int32_t* sizes, int32_t n_sizes, uint64_t seed) {
  if (!c || !sizes || n_sizes < 2) return fail(c, XT_EINVAL, "surrogate_init: sizes");
  cudaSetDevice(c->device);
  xt_mlp*& n = c->mlp;
  if (n) { mlp_destroy(n); n = nullptr; }
  n = new xt_mlp();
  n->sizes.assign(sizes, sizes + n_sizes);
  for (int s : n->sizes) if (s < 1 || s > 8192) return fail(c, XT_EINVAL, "surrogate_init: layer sizes 1..8192");
  int64_t o = 0;
  for (int k = 0; k + 1 < n_sizes; ++k) {
    n->woff.push_back(o); o += (int64_t)n->sizes[k] * n->sizes[k + 1];
    n->boff.push_back(o); o += n->sizes[k + 1];
  }
  n->nparam = o;
  int rc;
  if ((rc = mlp_layout_copies(c, n))) return rc;
  if ((rc = alloc(c, (void**)&n->w, o * 4, "mlp weights"))) return rc;
  if ((rc = alloc(c, (void**)&n->m, o * 4, "mlp adam"))) return rc;
  if ((rc = alloc(c, (void**)&n->v, o * 4, "mlp adam"))) return rc;
  if ((rc = alloc(c, (void**)&n->g, o * 4, "mlp grads"))) return rc;
  if ((rc = alloc(c, (void**)&n->wb, o * 2, "mlp weights"))) return rc;
  if ((rc = alloc(c, (void**)&n->st, sizeof(int64_t), "mlp step count"))) return rc;
  XT_CUDA(c, cudaMemsetAsync(n->st, 0, sizeof(int64_t), c->stream));
  XT_CUDA(c, cudaMemsetAsync(n->w, 0, o * 4, c->stream));
  XT_CUDA(c, cudaMemsetAsync(n->m, 0, o * 4, c->stream));
  XT_CUDA(c, cudaMemsetAsync(n->v, 0, o * 4, c->stream));
  for (int k = 0; k + 1 < n_sizes; ++k) {   // He-style normal init, zero biases
    const int64_t cnt = (int64_t)n->sizes[k] * n->sizes[k + 1];
    k_init_w<<<gb(cnt), 256, 0, c->stream>>>(n->w + n->woff[k], cnt, (float)std::sqrt(2.0 / n->sizes[k]), seed, (uint64_t)k);
  }
  mlp_sync_copies(c, n);
  XT_CUDA(c, cudaGetLastError());
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  return XT_OK;
}

int surrogate_weights(xt_ctx* c, int32_t set, float* flat, size_t n_cap) {
  if (!c || !c->mlp || !flat) return fail(c, XT_ESTATE, "surrogate_weights: surrogate_init first");
  xt_mlp* n = c->mlp;
  if (n_cap < (size_t)n->nparam) return fail(c, XT_EINVAL, "surrogate_weights: n_cap too small");
  cudaSetDevice(c->device);
  int rc;
  if (set) {
    if ((rc = copy(c, n->w, flat, n->nparam * 4, "weights"))) return rc;
    mlp_sync_copies(c, n);
    XT_CUDA(c, cudaGetLastError());
  } else if ((rc = copy(c, flat, n->w, n->nparam * 4, "weights"))) {
    return rc;
  }
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  return XT_OK;
}

// One forward + backward pass on a batch (host or device arrays, fp32):
// X [B][n_in], T and mask [B][n_out]; optional Adam update; gradients of the
// flat parameter vector to grads_out (optional) and the loss to loss_out.
int surrogate_train_step(xt_ctx* c, const float* X, const float* T, const float* mask, int64_t B,
                         double lr, int32_t update, float* grads_out, double* loss_out) {
  if (!c || !c->mlp) return fail(c, XT_ESTATE, "surrogate_train_step: surrogate_init first");
  if (!X || !T || !mask || B < 1) return fail(c, XT_EINVAL, "surrogate_train_step: X, T, mask, B");
  cudaSetDevice(c->device);
  xt_mlp* n = c->mlp;
  int rc;
  if ((rc = mlp_ensure_batch(c, n, B)) || (rc = mlp_train_buffers(c, n, B))) return rc;
  const int L = (int)n->sizes.size() - 1;
  const int nin = n->sizes[0], nout = n->sizes[L];
  if ((rc = copy(c, n->X, X, B * nin * 4, "X"))) return rc;
  if ((rc = copy(c, n->T, T, B * nout * 4, "T"))) return rc;
  if ((rc = copy(c, n->M, mask, B * nout * 4, "mask"))) return rc;
  std::vector<float> hm(B * nout);
  if ((rc = copy(c, hm.data(), n->M, B * nout * 4, "mask"))) return rc;
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  double msum = 0;
  for (float v : hm) msum += v;
  if (!(msum > 0)) return fail(c, XT_EINVAL, "surrogate_train_step: empty mask");
  return xt_mlp_step(c, B, msum, lr, update, grads_out, loss_out);
}

int surrogate_predict(xt_ctx* c, const float* X, int64_t B, float* Y) {
  if (!c || !c->mlp) return fail(c, XT_ESTATE, "surrogate_predict: surrogate_init first");
  if (!X || !Y || B < 1) return fail(c, XT_EINVAL, "surrogate_predict: X, Y, B");
  cudaSetDevice(c->device);
  xt_mlp* n = c->mlp;
  int rc;
  if ((rc = mlp_ensure_batch(c, n, B))) return rc;
  const int L = (int)n->sizes.size() - 1;
  if ((rc = copy(c, n->X, X, B * n->sizes[0] * 4, "X"))) return rc;
  k_to_bf16<<<gb(B * n->sizes[0]), 256, 0, c->stream>>>(n->X, B * n->sizes[0], n->H[0]);
  mlp_forward(c, n, B);
  XT_CUDA(c, cudaGetLastError());
  if ((rc = copy(c, Y, n->Z[L], B * n->sizes[L] * 4, "Y"))) return rc;
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  return XT_OK;
}

}  // extern "C"

// One step of the fused training kernel on the batch already in n->X / n->T
// / n->M (surrogate_train_step).
int xt_mlp_step(xt_ctx* c, int64_t B, double msum, double lr, int update, float* grads_out,
                double* loss_out) {
  (void)msum;   // the kernel sums the mask itself
  xt_mlp* n = c->mlp;
  XT_CUDA(c, cudaMemsetAsync(n->loss, 0, 8, c->stream));
  XT_CUDA(c, cudaMemsetAsync(n->msum1, 0, 8, c->stream));
  int rc;
  if ((rc = mlp_train_run(c, n, B, TrainSrc{n->X, n->T, n->M, nullptr}, 1, n->msum1, n->loss, lr, update != 0)))
    return rc;
  if (grads_out && (rc = copy(c, grads_out, n->g, n->nparam * 4, "grads"))) return rc;
  double l = 0;
  XT_CUDA(c, cudaMemcpyAsync(&l, n->loss, 8, cudaMemcpyDeviceToHost, c->stream));
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  if (loss_out) *loss_out = l;
  return XT_OK;
}

// ---------------------------------------------------------------- features
namespace xt {

struct FeatArgs {
  Geometry g;
  int n_ion, nlev, nline, nbin;
  const int* __restrict__ level_off;
  const double* __restrict__ ne;   // row order
  const double* __restrict__ Te;
  const double* __restrict__ dep;
  const double* __restrict__ nion; // [row][n_ion]
  const double* __restrict__ pops; // [row][nlev] targets (may be null)
  const int* __restrict__ levels_used;   // [cell*n_ion] natural, or null
  const double* __restrict__ lines;      // packed sorted
  const double* __restrict__ S;          // estimators (net) [row][sorted]
  const double* __restrict__ Jline;      // Jbar per sorted line (model), or null
  const double* __restrict__ invB;       // 1 / B_lu per sorted line
  const int* __restrict__ line_ion;      // ion of each sorted line
  const int* __restrict__ line_bin;      // log-lambda bin of each sorted line within its ion
  float* __restrict__ X;                 // [ncell][n_in] natural cell order
  float* __restrict__ T;                 // [ncell][nlev]
  float* __restrict__ M;                 // [ncell][nlev]
  double V;
  const int* __restrict__ crow;          // compact store: the cell's row in S, -1 none
};

// One block per cell: x = ((log10 ne - 7), (log10 Te - 3.7)/0.3, (log10 D + 14),
// per ion and bin the mean log10 Jbar + 9 of its lines (empty bins -5));
// targets log10(n_i/n_z)/10 clipped at -3, mask 1 on the kept levels.
__global__ void k_features(const FeatArgs a) {
  const int64_t cell = blockIdx.x;
  const int ix = (int)(cell % a.g.nx), iy = (int)((cell / a.g.nx) % a.g.ny), iz = (int)(cell / ((int64_t)a.g.nx * a.g.ny));
  const int64_t row = row_of(a.g, ix, iy, iz);
  const int nin = 3 + a.n_ion * (a.nbin + 1);
  float* x = a.X + cell * nin;
  extern __shared__ float sh[];
  float* sum = sh;                       // [n_ion * nbin]
  float* cnt = sh + a.n_ion * a.nbin;
  for (int k = threadIdx.x; k < a.n_ion * a.nbin; k += blockDim.x) { sum[k] = 0.f; cnt[k] = 0.f; }
  __syncthreads();
  for (int s = threadIdx.x; s < a.nline; s += blockDim.x) {
    double J;
    if (a.Jline) {
      J = a.Jline[s];
    } else {
      const int64_t sr = a.crow ? (int64_t)a.crow[row] : (int64_t)row;
      const double Snet = sr < 0 ? 0.0 : a.S[sr * a.nline + s];
      const double* L = a.lines + 4 * (int64_t)s;
      const int64_t lu = __double_as_longlong(L[3]);
      const double net = a.pops[row * a.nlev + (int)(lu & 0xFFFFFFFF)] - L[2] * a.pops[row * a.nlev + (int)(lu >> 32)];
      const double Vc = a.g.vol ? a.g.vol[row] : a.V;
      J = (Snet != 0.0 && net > 0.0) ? Snet / (net * Vc) * a.invB[s] : 0.0;
    }
    if (J > 0.0) {
      const int k = a.line_ion[s] * a.nbin + a.line_bin[s];
      atomicAdd(sum + k, (float)log10(J));
      atomicAdd(cnt + k, 1.f);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    x[0] = (float)(log10(fmax(a.ne[row], 1e-30)) - 7.0);
    x[1] = (float)((log10(fmax(a.Te[row], 1.0)) - 3.7) / 0.3);
    x[2] = (float)(log10(fmax(a.dep ? a.dep[row] : 0.0, 1e-30)) + 14.0);
  }
  for (int k = threadIdx.x; k < a.n_ion * a.nbin; k += blockDim.x)
    x[3 + k] = cnt[k] > 0.f ? sum[k] / cnt[k] + 9.f : -5.f;
  // the density of every ion: it sets the optical depths of its lines
  for (int z = threadIdx.x; z < a.n_ion; z += blockDim.x)
    x[3 + a.n_ion * a.nbin + z] = (float)(log10(fmax(a.nion[row * a.n_ion + z], 1e-30)) / 10.0);
  if (a.T) {
    for (int z = 0; z < a.n_ion; ++z) {
      const int off = a.level_off[z], Lz = a.level_off[z + 1] - off;
      const int L = a.levels_used ? min(a.levels_used[cell * a.n_ion + z], Lz) : Lz;
      const double nz = a.nion[row * a.n_ion + z];
      for (int i = threadIdx.x; i < Lz; i += blockDim.x) {
        const double r = nz > 0.0 ? a.pops[row * a.nlev + off + i] / nz : 0.0;
        a.T[cell * a.nlev + off + i] = (float)(log10(fmax(r, 1e-30)) / 10.0);
        a.M[cell * a.nlev + off + i] = (i < L && nz > 0.0) ? 1.f : 0.f;
      }
    }
  }
}

// warm populations from predictions: n_i = n_z 10^(10 y_i) over the kept
// levels, renormalised to sum n_z (one block per cell)
__global__ void k_warm_from_pred(Geometry g, int n_ion, int nlev, const int* __restrict__ level_off,
                                 const double* __restrict__ nion, const int* __restrict__ levels_used,
                                 const float* __restrict__ Y, double* __restrict__ out) {
  const int64_t cell = blockIdx.x;
  const int ix = (int)(cell % g.nx), iy = (int)((cell / g.nx) % g.ny), iz = (int)(cell / ((int64_t)g.nx * g.ny));
  const int64_t row = row_of(g, ix, iy, iz);
  __shared__ double red[32];
  for (int z = 0; z < n_ion; ++z) {
    const int off = level_off[z], Lz = level_off[z + 1] - off;
    const int L = levels_used ? min(levels_used[cell * n_ion + z], Lz) : Lz;
    double s = 0;
    for (int i = threadIdx.x; i < L; i += blockDim.x) s += exp10(10.0 * (double)Y[cell * nlev + off + i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) { double t = 0; for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k]; red[0] = t; }
    __syncthreads();
    const double scale = red[0] > 0.0 ? nion[row * n_ion + z] / red[0] : 0.0;
    for (int i = threadIdx.x; i < Lz; i += blockDim.x)
      out[row * nlev + off + i] = i < L ? scale * exp10(10.0 * (double)Y[cell * nlev + off + i]) : 0.0;
    __syncthreads();
  }
}

}  // namespace xt

constexpr int kJbarBins = 32;

// Feature matrix of every cell (and targets from the context's populations).
static int build_features(xt_ctx* c, int rates, double jbar_W, double jbar_TR, const int* levels_used_dev,
                          float* X, float* T, float* M) {
  const Geometry& G = c->geo;
  int rc;
  // per sorted line: ion, bin, model Jbar, 1/B
  std::vector<double> packed(4 * (size_t)c->nline);
  if ((rc = copy(c, packed.data(), c->d_lines, packed.size() * sizeof(double), "lines"))) return rc;
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<int> ion(c->nline), bin(c->nline);
  std::vector<double> Jm(c->nline);
  std::vector<double> lmin(c->n_ion, 1e300), lmax(c->n_ion, 0);
  for (int s = 0; s < c->nline; ++s) {
    int64_t lu;
    std::memcpy(&lu, &packed[4 * s + 3], 8);
    const int lo = (int)(lu & 0xFFFFFFFF);
    int z = 0;
    while (z + 1 < c->n_ion && c->h_level_off[z + 1] <= lo) ++z;
    ion[s] = z;
    const double lam = kC / packed[4 * s];
    lmin[z] = std::min(lmin[z], lam);
    lmax[z] = std::max(lmax[z], lam);
    const double x = kH * packed[4 * s] / (1.380649e-16 * (jbar_TR > 0 ? jbar_TR : 1.0));
    Jm[s] = jbar_W * 2.0 * kH * std::pow(packed[4 * s], 3) / (kC * kC) / std::expm1(x);
  }
  for (int s = 0; s < c->nline; ++s) {
    const int z = ion[s];
    const double lam = kC / packed[4 * s];
    const double span = std::log(lmax[z] / lmin[z]);
    int b = span > 0 ? (int)(std::log(lam / lmin[z]) / span * kJbarBins) : 0;
    bin[s] = std::min(std::max(b, 0), kJbarBins - 1);
  }
  int *d_ion = nullptr, *d_bin = nullptr;
  double* d_J = nullptr;
  if ((rc = alloc(c, (void**)&d_ion, c->nline * sizeof(int), "features"))) return rc;
  if ((rc = alloc(c, (void**)&d_bin, c->nline * sizeof(int), "features"))) { cudaFree(d_ion); return rc; }
  if ((rc = alloc(c, (void**)&d_J, c->nline * sizeof(double), "features"))) { cudaFree(d_ion); cudaFree(d_bin); return rc; }
  copy(c, d_ion, ion.data(), c->nline * sizeof(int), "features");
  copy(c, d_bin, bin.data(), c->nline * sizeof(int), "features");
  copy(c, d_J, Jm.data(), c->nline * sizeof(double), "features");
  FeatArgs a;
  a.g = G; a.n_ion = c->n_ion; a.nlev = c->nlev; a.nline = c->nline; a.nbin = kJbarBins;
  a.level_off = c->d_level_off; a.ne = c->d_ne; a.Te = c->d_Te; a.dep = c->d_dep; a.nion = c->d_nion;
  a.pops = c->d_pops; a.levels_used = levels_used_dev; a.lines = c->d_lines; a.S = c->d_S;
  a.crow = c->S_compact ? c->d_crow : nullptr;
  a.Jline = rates == XT_RATES_ESTIMATORS ? nullptr : d_J; a.invB = c->d_invB;
  a.line_ion = d_ion; a.line_bin = d_bin; a.X = X; a.T = T; a.M = M;
  a.V = G.dx * G.dy * G.dz;
  const size_t sh = 2 * (size_t)c->n_ion * kJbarBins * sizeof(float);
  k_features<<<(unsigned)G.ncell, 256, sh, c->stream>>>(a);
  cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(c->stream);
  cudaFree(d_ion); cudaFree(d_bin); cudaFree(d_J);
  if (e != cudaSuccess) return cuda_fail(c, e, "k_features");
  return XT_OK;
}

namespace xt {
int surrogate_warm(xt_ctx* c, int rates, double jbar_W, double jbar_TR, const int* levels_used_dev,
                   double* out) {
  if (!c->mlp) return fail(c, XT_ESTATE, "surrogate warm start: surrogate_init / train_surrogate first");
  xt_mlp* n = c->mlp;
  const int nin = 3 + c->n_ion * (kJbarBins + 1);
  if (n->sizes.front() != nin || n->sizes.back() != c->nlev)
    return fail(c, XT_EINVAL, "surrogate warm start: network sizes do not match the context");
  const int64_t N = c->geo.ncell;
  int rc;
  float* X = nullptr;
  if ((rc = alloc(c, (void**)&X, (size_t)N * nin * 4, "features"))) return rc;
  if ((rc = build_features(c, rates, jbar_W, jbar_TR, levels_used_dev, X, nullptr, nullptr))) { cudaFree(X); return rc; }
  const int64_t chunk = 8192;
  if ((rc = mlp_ensure_batch(c, n, chunk))) { cudaFree(X); return rc; }
  const int L = (int)n->sizes.size() - 1;
  float* Y = nullptr;
  if ((rc = alloc(c, (void**)&Y, (size_t)N * c->nlev * 4, "predictions"))) { cudaFree(X); return rc; }
  for (int64_t o = 0; o < N; o += chunk) {
    const int64_t B = std::min(chunk, N - o);
    k_to_bf16<<<gb(B * nin), 256, 0, c->stream>>>(X + o * nin, B * nin, n->H[0]);
    mlp_forward(c, n, B);
    cudaMemcpyAsync(Y + o * c->nlev, n->Z[L], B * c->nlev * 4, cudaMemcpyDeviceToDevice, c->stream);
  }
  k_warm_from_pred<<<(unsigned)N, 256, 0, c->stream>>>(c->geo, c->n_ion, c->nlev, c->d_level_off, c->d_nion,
                                                     levels_used_dev, Y, out);
  cudaError_t e = cudaGetLastError();
  cudaStreamSynchronize(c->stream);
  cudaFree(X);
  cudaFree(Y);
  if (e != cudaSuccess) return cuda_fail(c, e, "surrogate warm start");
  return XT_OK;
}
}  // namespace xt

extern "C" int train_surrogate(xt_ctx* c, const xt_train_params* p, xt_train_stats* out) {
  if (!c || !p) return fail(c, XT_EINVAL, "train_surrogate: null argument");
  if (!c->have_pops || !c->d_nion) return fail(c, XT_ESTATE, "train_surrogate: populations and n_ion_density needed");
  if (p->rates == XT_RATES_ESTIMATORS && !c->have_S) return fail(c, XT_ESTATE, "train_surrogate: no estimators for these populations");
  if (p->rates == XT_RATES_ESTIMATORS && c->S_groups > 0) return fail(c, XT_ESTATE, "train_surrogate: estimator inputs from a host-held store are not supported");
  if (p->epochs < 0 || p->batch < 1 || !(p->lr > 0)) return fail(c, XT_EINVAL, "train_surrogate: epochs >= 0, batch >= 1, lr > 0");
  cudaSetDevice(c->device);
  const int nin = 3 + c->n_ion * (kJbarBins + 1), nout = c->nlev;
  int rc;
  if (!c->mlp || c->mlp->sizes.front() != nin || c->mlp->sizes.back() != nout) {
    std::vector<int> sz{nin};
    for (int k = 0; k < p->n_layers; ++k) sz.push_back(p->n_hidden);
    sz.push_back(nout);
    if ((rc = surrogate_init(c, sz.data(), (int)sz.size(), p->seed))) return rc;
  }
  xt_mlp* n = c->mlp;
  const int64_t N = c->geo.ncell;
  int* d_used = nullptr;
  if (p->levels_used) {
    if ((rc = alloc(c, (void**)&d_used, N * c->n_ion * sizeof(int), "levels used"))) return rc;
    copy(c, d_used, p->levels_used, N * c->n_ion * sizeof(int), "levels used");
  }
  float *X = nullptr, *T = nullptr, *M = nullptr;
  int* d_idx = nullptr;
  double *d_msum = nullptr, *d_loss = nullptr;
  auto cleanup = [&]() {
    void* ps[] = {d_used, X, T, M, d_idx, d_msum, d_loss};
    for (void* q : ps) if (q) cudaFree(q);
  };
  if ((rc = alloc(c, (void**)&X, (size_t)N * nin * 4, "features")) ||
      (rc = alloc(c, (void**)&T, (size_t)N * nout * 4, "targets")) ||
      (rc = alloc(c, (void**)&M, (size_t)N * nout * 4, "mask"))) { cleanup(); return rc; }
  if ((rc = build_features(c, p->rates, p->jbar_W, p->jbar_TR, d_used, X, T, M))) { cleanup(); return rc; }
  // cells with matter only
  std::vector<double> nion(N * c->n_ion);
  std::vector<int> cells;
  {
    std::vector<double> rowv((size_t)N * c->n_ion);
    if ((rc = copy(c, rowv.data(), c->d_nion, rowv.size() * sizeof(double), "n_ion"))) { cleanup(); return rc; }
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
    const Geometry& G = c->geo;
    for (int64_t cell = 0; cell < N; ++cell) {
      const int ix = (int)(cell % G.nx), iy = (int)((cell / G.nx) % G.ny), iz = (int)(cell / ((int64_t)G.nx * G.ny));
      const int64_t row = row_of(G, ix, iy, iz);
      double s = 0;
      for (int z = 0; z < c->n_ion; ++z) s += rowv[row * c->n_ion + z];
      if (s > 0) cells.push_back((int)cell);
    }
  }
  if (cells.empty()) { cleanup(); return fail(c, XT_EINVAL, "train_surrogate: no cell with matter"); }
  const int64_t B = std::min<int64_t>(p->batch, (int64_t)cells.size());
  // The steps run in blocks of whole epochs: the host shuffles the cells of
  // each epoch of a block (a step takes the next B of them; an epoch's tail
  // short of B is left out), uploads the block's batch indices, and one launch
  // of the fused kernel runs all of the block's steps; the block's mask sums
  // and losses come back at its end.
  const int64_t per_epoch = (int64_t)cells.size() / B;
  const int64_t block_epochs = std::max<int64_t>(
      1, std::min<int64_t>(p->epochs, ((int64_t)64 << 20) / std::max<int64_t>(per_epoch * B * 4, 1)));
  const int64_t block_steps = block_epochs * per_epoch;
  if ((rc = alloc(c, (void**)&d_idx, (size_t)block_steps * B * sizeof(int), "batch index")) ||
      (rc = alloc(c, (void**)&d_msum, (size_t)block_steps * 8, "mask sums")) ||
      (rc = alloc(c, (void**)&d_loss, (size_t)block_steps * 8, "losses"))) { cleanup(); return rc; }
  uint64_t rng = p->seed * 0x9E3779B97F4A7C15ull + 1;
  auto next = [&]() { rng ^= rng << 13; rng ^= rng >> 7; rng ^= rng << 17; return rng; };
  double first = -1, last = 0;
  int64_t steps = 0;
  std::vector<int> hidx((size_t)block_steps * B);
  std::vector<double> hms(block_steps), hl(block_steps);
  cudaEventRecord(c->ev0, c->stream);
  for (int64_t ep0 = 0; ep0 < p->epochs; ep0 += block_epochs) {
    const int64_t ne = std::min<int64_t>(block_epochs, p->epochs - ep0), ns = ne * per_epoch;
    for (int64_t e = 0; e < ne; ++e) {
      for (int64_t k = (int64_t)cells.size() - 1; k > 0; --k) std::swap(cells[k], cells[next() % (k + 1)]);
      std::copy(cells.begin(), cells.begin() + per_epoch * B, hidx.begin() + e * per_epoch * B);
    }
    if (ns == 0) continue;
    if ((rc = copy(c, d_idx, hidx.data(), (size_t)ns * B * sizeof(int), "batch index"))) { cleanup(); return rc; }
    XT_CUDA(c, cudaMemsetAsync(d_msum, 0, (size_t)ns * 8, c->stream));
    XT_CUDA(c, cudaMemsetAsync(d_loss, 0, (size_t)ns * 8, c->stream));
    if ((rc = mlp_train_run(c, n, B, TrainSrc{X, T, M, d_idx}, ns, d_msum, d_loss, p->lr, true))) {
      cleanup();
      return rc;
    }
    if ((rc = copy(c, hms.data(), d_msum, (size_t)ns * 8, "mask sums")) ||
        (rc = copy(c, hl.data(), d_loss, (size_t)ns * 8, "losses"))) { cleanup(); return rc; }
    XT_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int64_t t = 0; t < ns; ++t) {
      if (!(hms[t] > 0)) continue;             // an empty mask: no step
      if (first < 0) first = hl[t];
      last = hl[t];
      ++steps;
    }
  }
  cudaEventRecord(c->ev1, c->stream);
  cudaEventSynchronize(c->ev1);
  float ms = 0;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  cleanup();
  if (out) {
    out->first_loss = first;
    out->last_loss = last;
    out->steps = (double)steps;
    out->samples = (double)cells.size();
    out->train_ms = ms;
  }
  return XT_OK;
}
