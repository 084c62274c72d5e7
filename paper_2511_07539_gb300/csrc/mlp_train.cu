// The surrogate's training steps fused into one persistent kernel: every
// step (batch gather, forward, masked-MSE loss, backward, Adam) runs in one
// cooperative launch, the phases separated by a grid barrier, so a training
// loop of thousands of small steps costs no launches and no host round trips.
// Every matrix product is a tcgen05 MMA (kind::f16, BF16 operands, FP32
// accumulation in TMEM) of M = 128 rows by N = 32 columns:
//   forward  Z_k = H_(k-1) W_k + b_k      rows = batch, K = s_(k-1)
//   backward dW_k = H_(k-1)^T dZ_k         rows = inputs i, K = batch; an extra
//            row of ones in H^T gives the bias gradient sum_b dZ_k in row s_(k-1)
//            dH_(k-1) = dZ_k W_k^T          rows = batch, K = s_k
// The epilogues write every activation and output gradient twice, by rows
// ([b][i]) and transposed ([i][b]), so that each product's operands are rows
// with K contiguous; the CTA stages them through registers into the canonical
// K-major layout of tc.cuh, in chunks of 256 K, and reads the accumulator with
// tcgen05.ld.  Hidden activations GELU (tanh form, Hendrycks & Gimpel 2016),
// masked mean squared error, Adam (Kingma & Ba 2015) on FP32 master weights.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "mlp.cuh"
#include "tc.cuh"

namespace xt {

constexpr int kTrThreads = 256;
constexpr int kTrKC = 256;                     // K elements staged per chunk
constexpr int kTrN = 32;                       // output columns per tile
constexpr int kTrMaxL = 8;                     // layers
constexpr size_t kTrSmemA = 128 * kTrKC * 2;   // 64 KB
constexpr size_t kTrSmemB = kTrN * kTrKC * 2;  // 16 KB
constexpr long long kTrMmaSpin = 1ll << 24;    // polls of an MMA completion
constexpr long long kTrBarSpin = 1ll << 24;    // polls of a grid barrier (64 ns sleeps: about a second)

struct TrainArgs {
  int L, B, nout, dzld;
  int s[kTrMaxL + 1], ps[kTrMaxL + 1];          // layer sizes and their 16-padded row lengths
  const float* X; const float* Tsrc; const float* Msrc; const int* idx;
  float* Tb; float* Mb;                          // the batch's targets and mask
  __nv_bfloat16* hp[kTrMaxL]; float* zp[kTrMaxL]; __nv_bfloat16* dz[2];
  __nv_bfloat16* hT[kTrMaxL]; __nv_bfloat16* dzT[2]; int bT;   // transposed copies, rows of bT = P(B)
  __nv_bfloat16* wp; __nv_bfloat16* wt; int64_t wpo[kTrMaxL], wto[kTrMaxL];
  float* w; float* m; float* v; float* g; __nv_bfloat16* wb;
  int64_t woff[kTrMaxL], boff[kTrMaxL];
  float lr, b1, b2, eps; int update;
  double* msumv; double* lossv; int64_t nsteps; int64_t* st;
  unsigned* bar;                                 // arrivals, generation, error
};

__device__ __forceinline__ float tr_gelu(float z) {
  const float u = 0.7978845608028654f * (z + 0.044715f * z * z * z);
  return 0.5f * z * (1.0f + tanhf(u));
}

__device__ __forceinline__ float tr_gelu_grad(float z) {
  const float u = 0.7978845608028654f * (z + 0.044715f * z * z * z);
  const float th = tanhf(u);
  const float du = 0.7978845608028654f * (1.0f + 3.0f * 0.044715f * z * z);
  return 0.5f * (1.0f + th) + 0.5f * z * (1.0f - th * th) * du;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of a cooperative launch with bounded waits: false (and the
// error flag set) if some CTA did not arrive within about a second or another
// CTA already gave up; a CTA that sees the flag set does not arrive.  The
// arrival is an acquire-release add (it publishes the CTA's writes, ordered
// before it by the block barrier; the last arrival thereby sees every CTA's),
// the last arrival advances the generation with a release, and the others
// wait on it with acquires.
__device__ bool grid_barrier(unsigned* bar) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = ld_acquire(bar + 2) == 0;
    if (ok) {
      const unsigned g0 = ld_acquire(bar + 1);
      unsigned old;
      asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
      if (old == gridDim.x - 1) {
        asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
      } else {
        long long i = 0;
        while (ld_acquire(bar + 1) == g0) {
          if (ld_acquire(bar + 2) != 0 || ++i > kTrBarSpin) { atomicExch(bar + 2, 1u); ok = 0; break; }
          __nanosleep(64);
        }
      }
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Operand rows r < R (128 or 32) of a K chunk, element (r, k) =
// src[(r0 + r) ld + kc + k], zero for r0 + r >= nrows; k < kn (a multiple of
// 16 with kc + kn <= ld, ld a multiple of 16), in 16-byte pieces.  A warp
// takes 8 rows x 4 pieces (lane % 8 the row, lane / 8 the piece): each row's
// pieces are 64 contiguous bytes of the source, and every 8 lanes store 128
// contiguous bytes of the tile (no bank conflicts).
template <int R>
__device__ __forceinline__ void stage_rows(unsigned char* dst, const __nv_bfloat16* __restrict__ src, int ld,
                                           int r0, int nrows, int kc, int kn) {
  constexpr int kGroups = R / 8;
  constexpr int kMax = R * (kTrKC / 8) / kTrThreads;
  const int per_row = kn >> 3;
  uint4 val[kMax];
#pragma unroll
  for (int q = 0; q < kMax; ++q) {
    const int sl = threadIdx.x + kTrThreads * q, lane = sl & 31, w = sl >> 5;
    const int r = (w % kGroups) * 8 + (lane & 7), c8 = (w / kGroups) * 4 + (lane >> 3);
    val[q] = make_uint4(0u, 0u, 0u, 0u);
    if (c8 < per_row && r0 + r < nrows)
      val[q] = *reinterpret_cast<const uint4*>(src + (int64_t)(r0 + r) * ld + kc + 8 * c8);
  }
#pragma unroll
  for (int q = 0; q < kMax; ++q) {
    const int sl = threadIdx.x + kTrThreads * q, lane = sl & 31, w = sl >> 5;
    const int r = (w % kGroups) * 8 + (lane & 7), c8 = (w / kGroups) * 4 + (lane >> 3);
    if (c8 < per_row) *reinterpret_cast<uint4*>(dst + tc::tile_off16(r, 8 * c8, R)) = val[q];
  }
}

struct TcCta {
  uint64_t* bar;
  uint32_t taddr, ph;
};

// D (TMEM: 128 lanes x 32 FP32 columns) = A B^T over kpad (a multiple of 16),
// the operands staged chunk by chunk by stA(kc, kn), stB(kc, kn); false if an
// MMA completion was not seen within its bounded wait.
template <typename SA, typename SB>
__device__ bool mma_tile(TcCta& t, unsigned char* sa, unsigned char* sb, int kpad, SA stA, SB stB) {
  for (int kc = 0; kc < kpad; kc += kTrKC) {
    const int kn = min(kTrKC, kpad - kc);
    stA(kc, kn);
    stB(kc, kn);
    tc::fence_smem_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (threadIdx.x == 0) {
      const uint32_t a0 = tc::smem_u32(sa), b0 = tc::smem_u32(sb);
      for (int j = 0; j < kn / 16; ++j) {
        const uint64_t ad = tc::smem_desc(a0 + (uint32_t)(2 * j * (128 / 8) * 128), (128 / 8) * 128, 128);
        const uint64_t bd = tc::smem_desc(b0 + (uint32_t)(2 * j * (kTrN / 8) * 128), (kTrN / 8) * 128, 128);
        tc::mma_bf16(t.taddr, ad, bd, tc::idesc_bf16(128, kTrN), kc > 0 || j > 0);
      }
      tc::commit(t.bar);
    }
    const bool got = tc::bar_wait(t.bar, t.ph, kTrMmaSpin);
    t.ph ^= 1u;
    if (!__syncthreads_and(got)) return false;
    tc::fence_after();
  }
  return true;
}

// This thread's 16 accumulator columns: row 32 (warp % 4) + lane of the tile,
// columns 16 (warp / 4) + 0..15; then every thread's loads are done before the
// next tile's MMAs overwrite the accumulator.
template <typename EPI>
__device__ __forceinline__ void epilogue(const TcCta& t, EPI epi) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float v[16];
  tc::ld16(t.taddr + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(16 * (w >> 2)), v);
  epi(32 * (w & 3) + lane, 16 * (w >> 2), v);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
}

// Block-wide sum of one double per thread, added to *out by thread 0.
__device__ __forceinline__ void block_add(double x, double* out) {
  __shared__ double red[kTrThreads / 32];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < kTrThreads / 32; ++k) t += red[k];
    if (t != 0.0) atomicAdd(out, t);
  }
  __syncthreads();
}

// Step t's batch: input rows as BF16 (padded with zeros), targets and mask
// (gathered, or already the batch's), and the mask sum to msumv[t].
__device__ void phase_gather(const TrainArgs& a, int64_t t) {
  const int B = a.B, nin = a.s[0], pin = a.ps[0], nout = a.nout;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  const int* idx = a.idx ? a.idx + t * B : nullptr;
  for (int64_t e = tid; e < (int64_t)B * pin; e += nth) {
    const int b = (int)(e / pin), j = (int)(e - (int64_t)b * pin);
    const int64_t r = idx ? idx[b] : b;
    const __nv_bfloat16 x = __float2bfloat16(j < nin ? a.X[r * nin + j] : 0.f);
    a.hp[0][e] = x;
    if (j < nin) a.hT[0][(int64_t)j * a.bT + b] = x;
  }
  // the row of ones after each layer's inputs (bias gradients), once per launch
  if (t == 0)
    for (int k = 0; k < a.L; ++k)
      for (int64_t b = tid; b < B; b += nth) a.hT[k][(int64_t)a.s[k] * a.bT + b] = __float2bfloat16(1.f);
  double ms = 0;
  for (int64_t e = tid; e < (int64_t)B * nout; e += nth) {
    float mv;
    if (idx) {
      const int b = (int)(e / nout), j = (int)(e - (int64_t)b * nout);
      const int64_t r = idx[b];
      a.Tb[e] = a.Tsrc[r * nout + j];
      mv = a.Msrc[r * nout + j];
      a.Mb[e] = mv;
    } else {
      mv = a.Mb[e];
    }
    ms += mv;
  }
  block_add(ms, a.msumv + t);
}

// Adam on the FP32 master weights after step t (nothing if its mask was
// empty; `count` the steps taken, the same in every CTA), writing the BF16
// copies: flat (prediction) and both operand layouts.  The flat vector is one
// range (per layer W_k then b_k), walked four parameters at a time per thread
// so that their loads are in flight together.
__device__ void phase_adam(const TrainArgs& a, int64_t t, int64_t& count) {
  if (!a.update || !(a.msumv[t] > 0)) return;
  ++count;
  const float c1 = 1.f - powf(a.b1, (float)count), c2 = 1.f - powf(a.b2, (float)count);
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t np = a.boff[a.L - 1] + a.s[a.L];
  for (int64_t e0 = tid; e0 < np; e0 += 4 * nth) {
    float gi[4], mi[4], vi[4], wi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t q = e0 + u * nth;
      if (q < np) { gi[u] = a.g[q]; mi[u] = a.m[q]; vi[u] = a.v[q]; wi[u] = a.w[q]; }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t q = e0 + u * nth;
      if (q >= np) break;
      const float m1 = a.b1 * mi[u] + (1.f - a.b1) * gi[u], v1 = a.b2 * vi[u] + (1.f - a.b2) * gi[u] * gi[u];
      a.m[q] = m1;
      a.v[q] = v1;
      const float w1 = wi[u] - a.lr * (m1 / c1) / (sqrtf(v1 / c2) + a.eps);
      a.w[q] = w1;
      const __nv_bfloat16 wh = __float2bfloat16(w1);
      a.wb[q] = wh;
      int k = 0;
      while (k + 1 < a.L && q >= a.woff[k + 1]) ++k;
      if (q < a.boff[k]) {
        const int so = a.s[k + 1];
        const int64_t e = q - a.woff[k];
        const int i = (int)(e / so), o = (int)(e - (int64_t)i * so);
        a.wp[a.wpo[k] + (int64_t)i * a.ps[k + 1] + o] = wh;
        a.wt[a.wto[k] + (int64_t)o * a.ps[k] + i] = wh;
      }
    }
  }
}

// Forward through layer k (1..L): tiles of 128 batch rows x 32 outputs.
// Hidden layers store Z (FP32) and GELU(Z) (BF16, zero in the row padding);
// the output layer turns Y straight into the loss gradient
// dY = 2 M (Y - T) / sum M (BF16) and adds M (Y - T)^2 / sum M to lossv[t].
__device__ bool phase_forward(const TrainArgs& a, int k, int64_t t, TcCta& tc_, unsigned char* sa,
                              unsigned char* sb) {
  const int B = a.B, so = a.s[k], pi = a.ps[k - 1], po = a.ps[k];
  const int nt = (so + kTrN - 1) / kTrN, tiles = ((B + 127) / 128) * nt;
  const bool last = k == a.L;
  const double ms = a.msumv[t];
  const double inv = ms > 0 ? 1.0 / ms : 0.0;
  const float* bias = a.w + a.boff[k - 1];
  const __nv_bfloat16* H = a.hp[k - 1];
  const __nv_bfloat16* Wt = a.wt + a.wto[k - 1];
  double loss = 0;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int m0 = (tile / nt) * 128, n0 = (tile % nt) * kTrN;
    const bool ok = mma_tile(
        tc_, sa, sb, pi, [&](int kc, int kn) { stage_rows<128>(sa, H, pi, m0, B, kc, kn); },
        [&](int kc, int kn) { stage_rows<kTrN>(sb, Wt, pi, n0, so, kc, kn); });
    if (!ok) return false;
    epilogue(tc_, [&](int row, int c0, const float* v) {
      const int b = m0 + row, o0 = n0 + c0;
      if (b >= B || o0 >= po) return;           // (po a multiple of 16: the 16 columns are in the row)
      uint32_t hw[8];
      if (!last) {
        float z[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int o = o0 + q;
          z[q] = o < so ? v[q] + bias[o] : 0.f;
          const __nv_bfloat16 h = __float2bfloat16(o < so ? tr_gelu(z[q]) : 0.f);
          if (o < so) a.hT[k][(int64_t)o * a.bT + b] = h;
          const uint32_t hb = __bfloat16_as_ushort(h);
          hw[q >> 1] = (q & 1) ? (hw[q >> 1] | (hb << 16)) : hb;
        }
        float4* zr = reinterpret_cast<float4*>(a.zp[k] + (int64_t)b * po + o0);
#pragma unroll
        for (int q = 0; q < 4; ++q) zr[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
        uint4* hr = reinterpret_cast<uint4*>(a.hp[k] + (int64_t)b * po + o0);
        hr[0] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        hr[1] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int o = o0 + q;
          __nv_bfloat16 gy = __float2bfloat16(0.f);
          if (o < so) {
            const float y = v[q] + bias[o];
            const float d = y - a.Tb[(int64_t)b * so + o];
            const float r = a.Mb[(int64_t)b * so + o] * d;
            loss += (double)r * (double)d;
            gy = __float2bfloat16((float)(2.0 * inv) * r);
            a.dzT[k & 1][(int64_t)o * a.bT + b] = gy;
          }
          const uint32_t gb = __bfloat16_as_ushort(gy);
          hw[q >> 1] = (q & 1) ? (hw[q >> 1] | (gb << 16)) : gb;
        }
        uint4* dr = reinterpret_cast<uint4*>(a.dz[k & 1] + (int64_t)b * a.dzld + o0);
        dr[0] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        dr[1] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
      }
    });
  }
  if (last) block_add(loss * inv, a.lossv + t);
  return true;
}

// Backward through layer k (L..1): the weight and bias gradients (tiles of
// 128 inputs, the row of ones last, x 32 outputs; K = the batch, from the
// transposed copies) and, for
// k > 1, dZ_(k-1) = (dZ_k W_k^T) GELU'(Z_(k-1)) (tiles of 128 batch rows x 32
// inputs; K = s_k), in one set of tiles.
__device__ bool phase_backward(const TrainArgs& a, int k, TcCta& tc_, unsigned char* sa, unsigned char* sb) {
  const int B = a.B, si = a.s[k - 1], so = a.s[k], pi = a.ps[k - 1], po = a.ps[k];
  const int nt1 = (so + kTrN - 1) / kTrN, t1 = ((si + 1 + 127) / 128) * nt1;
  const int nt2 = (si + kTrN - 1) / kTrN, t2 = k > 1 ? ((B + 127) / 128) * nt2 : 0;
  const __nv_bfloat16* dZ = a.dz[k & 1];
  const __nv_bfloat16* dZT = a.dzT[k & 1];
  const __nv_bfloat16* HT = a.hT[k - 1];
  const __nv_bfloat16* Wp = a.wp + a.wpo[k - 1];
  float* gW = a.g + a.woff[k - 1];
  float* gb = a.g + a.boff[k - 1];
  for (int tile = blockIdx.x; tile < t1 + t2; tile += gridDim.x) {
    if (tile < t1) {
      const int m0 = (tile / nt1) * 128, n0 = (tile % nt1) * kTrN;
      const bool ok = mma_tile(
          tc_, sa, sb, a.bT, [&](int kc, int kn) { stage_rows<128>(sa, HT, a.bT, m0, si + 1, kc, kn); },
          [&](int kc, int kn) { stage_rows<kTrN>(sb, dZT, a.bT, n0, so, kc, kn); });
      if (!ok) return false;
      epilogue(tc_, [&](int row, int c0, const float* v) {
        const int i = m0 + row;
        if (i > si) return;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int o = n0 + c0 + q;
          if (o < so) {
            if (i < si) gW[(int64_t)i * so + o] = v[q];
            else gb[o] = v[q];
          }
        }
      });
    } else {
      const int tt = tile - t1, m0 = (tt / nt2) * 128, n0 = (tt % nt2) * kTrN;
      const bool ok = mma_tile(
          tc_, sa, sb, po, [&](int kc, int kn) { stage_rows<128>(sa, dZ, a.dzld, m0, B, kc, kn); },
          [&](int kc, int kn) { stage_rows<kTrN>(sb, Wp, po, n0, si, kc, kn); });
      if (!ok) return false;
      __nv_bfloat16* dZn = a.dz[(k - 1) & 1];
      __nv_bfloat16* dZnT = a.dzT[(k - 1) & 1];
      const float* Z = a.zp[k - 1];
      epilogue(tc_, [&](int row, int c0, const float* v) {
        const int b = m0 + row, i0 = n0 + c0;
        if (b >= B || i0 >= pi) return;          // (pi a multiple of 16: the 16 columns are in the row)
        const float4* zr = reinterpret_cast<const float4*>(Z + (int64_t)b * pi + i0);
        float z[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 f = zr[q];
          z[4 * q] = f.x; z[4 * q + 1] = f.y; z[4 * q + 2] = f.z; z[4 * q + 3] = f.w;
        }
        uint32_t dw[8];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int i = i0 + q;
          const __nv_bfloat16 d = __float2bfloat16(i < si ? v[q] * tr_gelu_grad(z[q]) : 0.f);
          if (i < si) dZnT[(int64_t)i * a.bT + b] = d;
          const uint32_t db = __bfloat16_as_ushort(d);
          dw[q >> 1] = (q & 1) ? (dw[q >> 1] | (db << 16)) : db;
        }
        uint4* dr = reinterpret_cast<uint4*>(dZn + (int64_t)b * a.dzld + i0);
        dr[0] = make_uint4(dw[0], dw[1], dw[2], dw[3]);
        dr[1] = make_uint4(dw[4], dw[5], dw[6], dw[7]);
      });
    }
  }
  return true;
}

__device__ __forceinline__ void raise_error(unsigned* bar) {
  if (threadIdx.x == 0) atomicExch(bar + 2, 1u);
}

// The persistent training kernel: one CTA per SM (cooperative launch), TMEM
// for one 128 x 32 FP32 accumulator per CTA.  Per step: batch gather (with
// the previous step's Adam) | forward per layer | backward per layer, a grid
// barrier after each phase.
__global__ void __launch_bounds__(kTrThreads, 1) k_train(const TrainArgs a) {
  extern __shared__ __align__(1024) unsigned char trsm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  unsigned char* const sa = trsm;
  unsigned char* const sb = trsm + kTrSmemA;
  if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&tslot, 32);
  if (threadIdx.x == 0) tc::bar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  TcCta tcs{&mbar, tslot, 0u};
  int64_t count = *a.st;
  bool ok = true;
  for (int64_t t = 0; ok && t < a.nsteps; ++t) {
    phase_gather(a, t);
    if (t > 0) phase_adam(a, t - 1, count);
    ok = grid_barrier(a.bar);
    for (int k = 1; ok && k <= a.L; ++k) {
      if (!phase_forward(a, k, t, tcs, sa, sb)) raise_error(a.bar);
      ok = grid_barrier(a.bar);
    }
    for (int k = a.L; ok && k >= 1; --k) {
      if (!phase_backward(a, k, tcs, sa, sb)) raise_error(a.bar);
      ok = grid_barrier(a.bar);
    }
  }
  if (ok && a.nsteps > 0) phase_adam(a, a.nsteps - 1, count);
  if (ok && blockIdx.x == 0 && threadIdx.x == 0) *a.st = count;
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if ((threadIdx.x >> 5) == 0) tc::tmem_free(tslot, 32);
}

// The BF16 copies of every weight (flat, and the two operand layouts).
__global__ void k_sync_copies(const TrainArgs a) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int k = 1; k <= a.L; ++k) {
    const int si = a.s[k - 1], so = a.s[k];
    const int64_t nw = (int64_t)si * so;
    for (int64_t e = tid; e < nw + so; e += nth) {
      const int64_t q = e < nw ? a.woff[k - 1] + e : a.boff[k - 1] + (e - nw);
      const __nv_bfloat16 wh = __float2bfloat16(a.w[q]);
      a.wb[q] = wh;
      if (e < nw) {
        const int i = (int)(e / so), o = (int)(e - (int64_t)i * so);
        a.wp[a.wpo[k - 1] + (int64_t)i * a.ps[k] + o] = wh;
        a.wt[a.wto[k - 1] + (int64_t)o * a.ps[k - 1] + i] = wh;
      }
    }
  }
}

static void fill_layers(const xt_mlp* n, TrainArgs& a) {
  a.L = (int)n->sizes.size() - 1;
  for (int k = 0; k <= a.L; ++k) { a.s[k] = n->sizes[k]; a.ps[k] = pad16(n->sizes[k]); }
  for (int k = 0; k < a.L; ++k) {
    a.woff[k] = n->woff[k]; a.boff[k] = n->boff[k]; a.wpo[k] = n->wpo[k]; a.wto[k] = n->wto[k];
  }
  a.wp = n->wp; a.wt = n->wt; a.w = n->w; a.m = n->m; a.v = n->v; a.g = n->g; a.wb = n->wb;
}

int mlp_layout_copies(xt_ctx* c, xt_mlp* n) {
  const int L = (int)n->sizes.size() - 1;
  if (L > kTrMaxL) return fail(c, XT_EINVAL, "surrogate_init: at most " + std::to_string(kTrMaxL) + " layers");
  n->wpo.assign(L, 0);
  n->wto.assign(L, 0);
  int64_t op = 0, ot = 0;
  for (int k = 1; k <= L; ++k) {
    n->wpo[k - 1] = op; op += (int64_t)n->sizes[k - 1] * pad16(n->sizes[k]);
    n->wto[k - 1] = ot; ot += (int64_t)n->sizes[k] * pad16(n->sizes[k - 1]);
  }
  int rc;
  if ((rc = alloc(c, (void**)&n->wp, (size_t)op * 2, "mlp weights"))) return rc;
  if ((rc = alloc(c, (void**)&n->wt, (size_t)ot * 2, "mlp weights"))) return rc;
  XT_CUDA(c, cudaMemsetAsync(n->wp, 0, (size_t)op * 2, c->stream));
  XT_CUDA(c, cudaMemsetAsync(n->wt, 0, (size_t)ot * 2, c->stream));
  return XT_OK;
}

void mlp_sync_copies(xt_ctx* c, xt_mlp* n) {
  TrainArgs a{};
  fill_layers(n, a);
  k_sync_copies<<<152 * 8, 256, 0, c->stream>>>(a);
}

int mlp_train_buffers(xt_ctx* c, xt_mlp* n, int64_t B) {
  if (B <= n->tcap) return XT_OK;
  const int L = (int)n->sizes.size() - 1;
  for (auto& q : n->hp) release((void**)&q);
  for (auto& q : n->zp) release((void**)&q);
  for (auto& q : n->hT) release((void**)&q);
  release((void**)&n->dz[0]); release((void**)&n->dz[1]);
  release((void**)&n->dzT[0]); release((void**)&n->dzT[1]);
  release((void**)&n->T); release((void**)&n->M);
  n->hp.assign(L, nullptr);
  n->zp.assign(L, nullptr);
  n->hT.assign(L, nullptr);
  const size_t bT = (size_t)pad16((int)B);
  int smax = 0;
  for (int s : n->sizes) smax = std::max(smax, pad16(s));
  int rc;
  for (int k = 0; k < L; ++k) {
    const size_t hb = (size_t)B * pad16(n->sizes[k]) * 2;
    if ((rc = alloc(c, (void**)&n->hp[k], hb, "mlp activations"))) return rc;
    XT_CUDA(c, cudaMemsetAsync(n->hp[k], 0, hb, c->stream));
    if (k > 0 && (rc = alloc(c, (void**)&n->zp[k], (size_t)B * pad16(n->sizes[k]) * 4, "mlp activations"))) return rc;
    if ((rc = alloc(c, (void**)&n->hT[k], (size_t)(n->sizes[k] + 1) * bT * 2, "mlp activations"))) return rc;
  }
  for (int j = 0; j < 2; ++j) {
    if ((rc = alloc(c, (void**)&n->dz[j], (size_t)B * smax * 2, "mlp gradients"))) return rc;
    XT_CUDA(c, cudaMemsetAsync(n->dz[j], 0, (size_t)B * smax * 2, c->stream));
    if ((rc = alloc(c, (void**)&n->dzT[j], (size_t)smax * bT * 2, "mlp gradients"))) return rc;
  }
  if ((rc = alloc(c, (void**)&n->T, (size_t)B * n->sizes[L] * 4, "mlp targets"))) return rc;
  if ((rc = alloc(c, (void**)&n->M, (size_t)B * n->sizes[L] * 4, "mlp mask"))) return rc;
  if (!n->loss && (rc = alloc(c, (void**)&n->loss, 8, "mlp loss"))) return rc;
  if (!n->msum1 && (rc = alloc(c, (void**)&n->msum1, 8, "mlp mask sum"))) return rc;
  if (!n->bar && (rc = alloc(c, (void**)&n->bar, 4 * sizeof(unsigned), "mlp barrier"))) return rc;
  n->tcap = B;
  return XT_OK;
}

int mlp_train_run(xt_ctx* c, xt_mlp* n, int64_t B, const TrainSrc& src, int64_t nsteps, double* msumv,
                  double* lossv, double lr, bool update) {
  const int L = (int)n->sizes.size() - 1;
  if (L > kTrMaxL) return fail(c, XT_EINVAL, "surrogate training: at most " + std::to_string(kTrMaxL) + " layers");
  if (B < 1 || B > (1 << 24)) return fail(c, XT_EINVAL, "surrogate training: batch size");
  if (nsteps <= 0) return XT_OK;
  int rc;
  if ((rc = mlp_train_buffers(c, n, B))) return rc;
  TrainArgs a{};
  fill_layers(n, a);
  a.B = (int)B;
  a.nout = n->sizes[L];
  int smax = 0;
  for (int s : n->sizes) smax = std::max(smax, pad16(s));
  a.dzld = smax;
  a.X = src.X; a.Tsrc = src.T; a.Msrc = src.M; a.idx = src.idx;
  a.Tb = n->T; a.Mb = n->M;
  for (int k = 0; k < L; ++k) { a.hp[k] = n->hp[k]; a.zp[k] = n->zp[k]; }
  a.dz[0] = n->dz[0]; a.dz[1] = n->dz[1];
  // the transposed copies in rows of P(B), zero beyond the batch (a launch
  // with another batch size may have left values there)
  a.bT = pad16((int)B);
  for (int k = 0; k < L; ++k) {
    a.hT[k] = n->hT[k];
    XT_CUDA(c, cudaMemsetAsync(n->hT[k], 0, (size_t)(n->sizes[k] + 1) * a.bT * 2, c->stream));
  }
  for (int j = 0; j < 2; ++j) {
    a.dzT[j] = n->dzT[j];
    XT_CUDA(c, cudaMemsetAsync(n->dzT[j], 0, (size_t)smax * a.bT * 2, c->stream));
  }
  a.lr = (float)lr; a.b1 = 0.9f; a.b2 = 0.999f; a.eps = 1e-8f; a.update = update ? 1 : 0;
  a.msumv = msumv; a.lossv = lossv; a.nsteps = nsteps; a.st = n->st; a.bar = n->bar;
  const size_t smem = kTrSmemA + kTrSmemB;
  XT_CUDA(c, cudaFuncSetAttribute(k_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, nsm = 0;
  XT_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_train, kTrThreads, smem));
  XT_CUDA(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  if (per_sm < 1) return fail(c, XT_ECUDA, "surrogate training: the kernel does not fit an SM");
  // one CTA per SM: the phases have up to a few dozen tiles, and the
  // elementwise work (gather, Adam) takes every thread the launch has (fewer
  // CTAs, sized to the largest phase, measured slower)
  const int grid = nsm;
  XT_CUDA(c, cudaMemsetAsync(n->bar, 0, 4 * sizeof(unsigned), c->stream));
  void* args[] = {(void*)&a};
  XT_CUDA(c, cudaLaunchCooperativeKernel((const void*)k_train, dim3(grid), dim3(kTrThreads), args, smem, c->stream));
  unsigned err = 0;
  XT_CUDA(c, cudaMemcpyAsync(&err, n->bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  XT_CUDA(c, cudaStreamSynchronize(c->stream));
  if (err) return fail(c, XT_ETIMEOUT, "surrogate training: a grid barrier or an MMA completion wait ran out");
  return XT_OK;
}

}  // namespace xt
