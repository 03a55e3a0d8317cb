// Fourier-neural-operator surrogate kernels: BF16 tensor-core GEMM with fused
// epilogues, truncated spectral transforms, channel mixing, GELU, loss and Adam.
//
// The surrogate maps the normalised fundamental on an N^3 focal box (2 channels) to the
// normalised harmonics 2..5 (8 channels); see include/vp_fno.h for the architecture.
// Activations are [voxel][channel] (x slowest, z, then channel fastest); a "line" is
// one (x, y) column of N voxels along z.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "vp.h"
#include "vp_fno.h"

namespace {

using bf16 = __nv_bfloat16;

// ---- BF16 tensor-core GEMM (mma.sync m16n8k16, FP32 accumulate) ---------------------
// C[b][m][n] = sum_k A[b][m][k] B[b][k][n] (+ epilogue), general strides.
struct Gemm {
  int M, N, K, batch, ksplit;
  const bf16* A;
  long long a_rs, a_cs, a_bs;
  const bf16* B;
  long long b_rs, b_cs, b_bs;
  float* C;  // FP32 result (pre-activation when gelu), may be null if only Cb is wanted
  long long c_rs, c_cs, c_bs;
  bf16* Cb;  // optional BF16 copy of the (activated) result, same strides as C
  const float* bias;    // [N] or null
  const float* addend;  // same layout as C, or null
  int gelu;        // 1: Cb = GELU(result)
  int accumulate;  // 1: C += result (atomic when ksplit > 1)
  int a_mode, b_mode;  // tile loaders, set by gemm()
  // Optional row grouping of A: row m lives at (m / a_group) * a_gstride + (m % a_group) * a_rs
  // (a_group = 0: plain rows m * a_rs).  Lets per-line products over all lines run as
  // one GEMM whose rows are (line, channel).
  int a_group;
  long long a_gstride;
  // Optional second contraction added to the same tile (batch 1 only): rows are
  // (line, z) with line = m / rows_per_line, z = m % rows_per_line, and
  //   C[m][n] += sum_{j < K2} A2[z][j] B2[line][j][n]
  // (A2 row-major with row stride a2_rs, B2 row stride b2_rs, line stride b2_line).
  // Needs rows_per_line % BM == 0 and 16-byte aligned, contiguous rows.
  const bf16* A2;
  long long a2_rs;
  const bf16* B2;
  long long b2_rs, b2_line;
  int K2, rows_per_line;
};

// The K slices of the main product and of the optional second contraction form one
// pipeline of stages: the next stage's tiles are loaded while the current one computes.
// (BK = 64, one stage for K <= 64, measured slower: more registers, fewer resident CTAs.)
constexpr int BM = 64, BN = 64, BK = 32, KP = BK + 8;  // padded rows: conflict-free fragments
constexpr int kChunks = BM * BK / 8 / 128;             // 16-byte chunks per thread per tile

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * __expf(-0.5f * x * x);
  return cdf + x * pdf;
}

// Tile loaders.  Vector modes move 16-byte chunks (8 BF16 values) and are chosen on
// the host only when every chunk is either wholly inside the operand or wholly outside
// and 16-byte aligned:  A: 1 = k contiguous, 2 = m contiguous;  B: 1 = n contiguous,
// 2 = k contiguous;  0 = element by element.  Each thread moves two chunks per tile.
struct TileRegs {
  uint4 a[kChunks], b[kChunks];
};

__device__ __forceinline__ long long a_row(const Gemm& g, int m) {
  if (g.a_group == 0) return (long long)m * g.a_rs;
  const int q = m / g.a_group;
  return (long long)q * g.a_gstride + (long long)(m - q * g.a_group) * g.a_rs;
}

__device__ __forceinline__ void load_tiles(const Gemm& g, const bf16* A, const bf16* B, int m0, int n0, int k0,
                                           int k_end, int tid, TileRegs& r) {
  const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
  constexpr int KC = BK / 8;  // chunks along k in a row of the tile
#pragma unroll
  for (int c = 0; c < kChunks; ++c) {
    const int e = tid + c * 128;
    if (g.a_mode == 1) {
      const int m = e / KC, kc = (e % KC) * 8;
      const int gm = m0 + m, gk = k0 + kc;
      r.a[c] = (gm < g.M && gk < k_end) ? *reinterpret_cast<const uint4*>(A + a_row(g, gm) + gk) : z4;
    } else if (g.a_mode == 2) {
      const int mc = (e & 7) * 8, k = e >> 3;
      const int gm = m0 + mc, gk = k0 + k;
      r.a[c] = (gm < g.M && gk < k_end) ? *reinterpret_cast<const uint4*>(A + a_row(g, gm) + (long long)gk * g.a_cs) : z4;
    }
    if (g.b_mode == 1) {
      const int nc = (e & 7) * 8, k = e >> 3;
      const int gn = n0 + nc, gk = k0 + k;
      r.b[c] = (gn < g.N && gk < k_end) ? *reinterpret_cast<const uint4*>(B + (long long)gk * g.b_rs + gn) : z4;
    } else if (g.b_mode == 2) {
      const int n = e / KC, kc = (e % KC) * 8;
      const int gn = n0 + n, gk = k0 + kc;
      r.b[c] = (gn < g.N && gk < k_end) ? *reinterpret_cast<const uint4*>(B + gk + (long long)gn * g.b_cs) : z4;
    }
  }
}

__device__ __forceinline__ void store_tiles(const Gemm& g, const bf16* A, const bf16* B, int m0, int n0, int k0,
                                            int k_end, int tid, const TileRegs& r, bf16 (*As)[KP],
                                            bf16 (*Bs)[KP]) {
  const bf16 zero = __float2bfloat16(0.f);
  constexpr int KC = BK / 8;
#pragma unroll
  for (int c = 0; c < kChunks; ++c) {
    const int e = tid + c * 128;
    if (g.a_mode == 1) {
      *reinterpret_cast<uint4*>(&As[e / KC][(e % KC) * 8]) = r.a[c];
    } else if (g.a_mode == 2) {
      const bf16* v = reinterpret_cast<const bf16*>(&r.a[c]);
      const int mc = (e & 7) * 8, k = e >> 3;
#pragma unroll
      for (int i = 0; i < 8; ++i) As[mc + i][k] = v[i];
    }
    if (g.b_mode == 1) {
      const bf16* v = reinterpret_cast<const bf16*>(&r.b[c]);
      const int nc = (e & 7) * 8, k = e >> 3;
#pragma unroll
      for (int i = 0; i < 8; ++i) Bs[nc + i][k] = v[i];
    } else if (g.b_mode == 2) {
      *reinterpret_cast<uint4*>(&Bs[e / KC][(e % KC) * 8]) = r.b[c];
    }
  }
  if (g.a_mode == 0) {
    const bool a_kfast = g.a_cs == 1;
    for (int e = tid; e < BM * BK; e += 128) {
      int m, k;
      if (a_kfast) { k = e % BK; m = e / BK; } else { m = e % BM; k = e / BM; }
      const int gm = m0 + m, gk = k0 + k;
      As[m][k] = (gm < g.M && gk < k_end) ? A[a_row(g, gm) + (long long)gk * g.a_cs] : zero;
    }
  }
  if (g.b_mode == 0) {
    const bool b_nfast = g.b_cs == 1;
    for (int e = tid; e < BK * BN; e += 128) {
      int n, k;
      if (b_nfast) { n = e % BN; k = e / BN; } else { k = e % BK; n = e / BK; }
      const int gn = n0 + n, gk = k0 + k;
      Bs[n][k] = (gn < g.N && gk < k_end) ? B[(long long)gk * g.b_rs + (long long)gn * g.b_cs] : zero;
    }
  }
}

// One BK slice of the CTA tile: each warp's 32 x 32 block by mma.sync m16n8k16.
__device__ __forceinline__ void mma_slice(const bf16 (*As)[KP], const bf16 (*Bs)[KP], int wm, int wn, int gq,
                                          int tq, float (&acc)[2][4][4]) {
#pragma unroll
  for (int kk = 0; kk < BK; kk += 16) {
    unsigned af[2][4], bfr[4][2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = wm + i * 16 + gq;
      af[i][0] = *reinterpret_cast<const unsigned*>(&As[r][kk + 2 * tq]);
      af[i][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][kk + 2 * tq]);
      af[i][2] = *reinterpret_cast<const unsigned*>(&As[r][kk + 2 * tq + 8]);
      af[i][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][kk + 2 * tq + 8]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = wn + j * 8 + gq;
      bfr[j][0] = *reinterpret_cast<const unsigned*>(&Bs[c][kk + 2 * tq]);
      bfr[j][1] = *reinterpret_cast<const unsigned*>(&Bs[c][kk + 2 * tq + 8]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
            : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]), "r"(bfr[j][1]));
  }
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const Gemm g) {
  __shared__ __align__(16) bf16 As[BM][KP];
  __shared__ __align__(16) bf16 Bs[BN][KP];  // n-major: Bs[n][k]
  const int b = blockIdx.z / g.ksplit;
  const int ks = blockIdx.z - b * g.ksplit;
  const int kchunk = ((g.K + g.ksplit - 1) / g.ksplit + BK - 1) / BK * BK;
  const int k_begin = ks * kchunk;
  const int k_end = min(g.K, k_begin + kchunk);
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const bf16* A = g.A + (long long)b * g.a_bs;
  const bf16* B = g.B + (long long)b * g.b_bs;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gq = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  // stages: the K slices of the main product, then those of the second contraction
  Gemm g2 = g;
  const bf16* A2 = nullptr;
  const bf16* B2 = nullptr;
  int n1 = k_begin < k_end ? (k_end - k_begin + BK - 1) / BK : 0, n2 = 0;
  if (g.A2 && ks == 0) {
    g2.M = min(BM, g.M - m0);
    g2.K = g.K2;
    g2.a_rs = g.a2_rs; g2.a_cs = 1; g2.a_mode = 1; g2.a_group = 0;
    g2.b_rs = g.b2_rs; g2.b_cs = 1; g2.b_mode = 1;
    const int line = m0 / g.rows_per_line, z0 = m0 - line * g.rows_per_line;
    A2 = g.A2 + (long long)z0 * g.a2_rs;
    B2 = g.B2 + (long long)line * g.b2_line;
    n2 = (g2.K + BK - 1) / BK;
  }
  auto load_stage = [&](int st, TileRegs& r) {
    if (st < n1) load_tiles(g, A, B, m0, n0, k_begin + st * BK, k_end, tid, r);
    else load_tiles(g2, A2, B2, 0, n0, (st - n1) * BK, g2.K, tid, r);
  };
  auto store_stage = [&](int st, const TileRegs& r) {
    if (st < n1) store_tiles(g, A, B, m0, n0, k_begin + st * BK, k_end, tid, r, As, Bs);
    else store_tiles(g2, A2, B2, 0, n0, (st - n1) * BK, g2.K, tid, r, As, Bs);
  };
  TileRegs regs;
  const int nst = n1 + n2;
  if (nst > 0) load_stage(0, regs);
  for (int st = 0; st < nst; ++st) {
    store_stage(st, regs);
    __syncthreads();
    if (st + 1 < nst) load_stage(st + 1, regs);
    mma_slice(As, Bs, wm, wn, gq, tq, acc);
    __syncthreads();
  }
  // epilogue: column pairs (n, n + 1) go out as one 8-byte / 4-byte store when the
  // output rows are contiguous and even-aligned
  const bool pair = g.c_cs == 1 && g.c_rs % 2 == 0 && g.c_bs % 2 == 0 && g.N % 2 == 0 && !g.accumulate &&
                    !g.addend;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int m = m0 + wm + i * 16 + gq + h2 * 8;
        const int n = n0 + wn + j * 8 + 2 * tq;
        if (m >= g.M || n >= g.N) continue;
        const long long off = (long long)b * g.c_bs + (long long)m * g.c_rs + (long long)n * g.c_cs;
        float v0 = acc[i][j][2 * h2], v1 = acc[i][j][2 * h2 + 1];
        if (pair) {
          if (g.bias && ks == 0) {
            v0 += g.bias[n];
            v1 += g.bias[n + 1];
          }
          if (g.C) *reinterpret_cast<float2*>(g.C + off) = make_float2(v0, v1);
          if (g.Cb) {
            const float a0 = g.gelu ? gelu_f(v0) : v0, a1 = g.gelu ? gelu_f(v1) : v1;
            *reinterpret_cast<__nv_bfloat162*>(g.Cb + off) = __floats2bfloat162_rn(a0, a1);
          }
          continue;
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          if (n + r >= g.N) break;
          const long long o = off + r * g.c_cs;
          float v = r == 0 ? v0 : v1;
          if (ks == 0) {
            if (g.bias) v += g.bias[n + r];
            if (g.addend) v += g.addend[o];
          }
          if (g.accumulate) {
            if (g.ksplit > 1) atomicAdd(&g.C[o], v);
            else g.C[o] += v;
            continue;
          }
          if (g.C) g.C[o] = v;
          if (g.Cb) g.Cb[o] = __float2bfloat16(g.gelu ? gelu_f(v) : v);
        }
      }
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

cudaError_t gemm(const Gemm& g0, cudaStream_t s) {
  Gemm g = g0;
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.ksplit > 1 && !(g.accumulate && g.batch == 1)) return cudaErrorInvalidValue;
  const bool abs8 = g.batch == 1 || g.a_bs % 8 == 0, bbs8 = g.batch == 1 || g.b_bs % 8 == 0;
  g.a_mode = 0;
  const bool grp8 = g.a_group == 0 || (g.a_group % 8 == 0 && g.a_gstride % 8 == 0);
  if (al16(g.A) && abs8) {
    if (g.a_cs == 1 && g.K % 8 == 0 && g.a_rs % 8 == 0 && (g.a_group == 0 || g.a_gstride % 8 == 0)) g.a_mode = 1;
    else if (g.a_rs == 1 && g.M % 8 == 0 && g.a_cs % 8 == 0 && grp8) g.a_mode = 2;
  }
  g.b_mode = 0;
  if (al16(g.B) && bbs8) {
    if (g.b_cs == 1 && g.N % 8 == 0 && g.b_rs % 8 == 0) g.b_mode = 1;
    else if (g.b_rs == 1 && g.K % 8 == 0 && g.b_cs % 8 == 0) g.b_mode = 2;
  }
  if (g.A2) {
    if (g.batch != 1 || g.rows_per_line % BM != 0 || g.K2 % 8 != 0 || g.N % 8 != 0 || !al16(g.A2) ||
        !al16(g.B2) || g.a2_rs % 8 != 0 || g.b2_rs % 8 != 0 || g.b2_line % 8 != 0)
      return cudaErrorInvalidValue;
  }
  const dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch * g.ksplit);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
  return cudaGetLastError();
}

Gemm gemm_base() {
  Gemm g;
  std::memset(&g, 0, sizeof(g));
  g.batch = 1;
  g.ksplit = 1;
  return g;
}

// ---- elementwise / spectral kernels --------------------------------------------------

int grid1(long long n, int t) {
  long long b = (n + t - 1) / t;
  if (b > 152LL * 32) b = 152LL * 32;
  return (int)(b < 1 ? 1 : b);
}

// Input features of one voxel: Re, Im of q^k, k = 1..VP_FNO_POWERS, for q = x0 + i x1.
__device__ __forceinline__ void features(const float* __restrict__ x, long long v, float* f) {
  const float qr = x[2 * v], qi = x[2 * v + 1];
  float pr = qr, pi = qi;
#pragma unroll
  for (int k = 0; k < VP_FNO_POWERS; ++k) {
    f[2 * k] = pr;
    f[2 * k + 1] = pi;
    const float nr = pr * qr - pi * qi;
    pi = pr * qi + pi * qr;
    pr = nr;
  }
}

// h0[v][c] = sum_f feat[v][f] P[f][c] + bP[c]: one thread per (voxel, 8 channels), the
// features once per thread, one 16-byte store (W % 8 == 0; else one channel per thread)
__global__ void lift_kernel(const float* __restrict__ x, const float* __restrict__ P, const float* __restrict__ bP,
                            bf16* __restrict__ h, long long V, int W) {
  if (W % 8 == 0) {
    const int groups = W / 8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V * groups;
         i += (long long)gridDim.x * blockDim.x) {
      const long long v = i / groups;
      const int c0 = (int)(i - v * groups) * 8;
      float f[VP_FNO_IN];
      features(x, v, f);
      __align__(16) bf16 out[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float acc = bP[c0 + j];
#pragma unroll
        for (int k = 0; k < VP_FNO_IN; ++k) acc = fmaf(f[k], P[k * W + c0 + j], acc);
        out[j] = __float2bfloat16(acc);
      }
      *reinterpret_cast<uint4*>(h + v * W + c0) = *reinterpret_cast<const uint4*>(out);
    }
    return;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V * W; i += (long long)gridDim.x * blockDim.x) {
    const long long v = i / W;
    const int c = (int)(i - v * W);
    float f[VP_FNO_IN];
    features(x, v, f);
    float acc = bP[c];
#pragma unroll
    for (int k = 0; k < VP_FNO_IN; ++k) acc = fmaf(f[k], P[k * W + c], acc);
    h[i] = __float2bfloat16(acc);
  }
}

// dP += feat^T dh, dbP += sum dh  (dh: fp32 [V][W]); each thread owns one channel c
// for a slice of voxels, then atomics.
__global__ void lift_grad_kernel(const float* __restrict__ x, const float* __restrict__ dh, float* __restrict__ dP,
                                 float* __restrict__ dbP, long long V, int W) {
  const int c = threadIdx.x % W;
  const int lane_group = threadIdx.x / W;
  const int groups = blockDim.x / W;
  float s[VP_FNO_IN], sb = 0.f;
#pragma unroll
  for (int k = 0; k < VP_FNO_IN; ++k) s[k] = 0.f;
  for (long long v = (long long)blockIdx.x * groups + lane_group; v < V; v += (long long)gridDim.x * groups) {
    const float d = dh[v * W + c];
    float f[VP_FNO_IN];
    features(x, v, f);
#pragma unroll
    for (int k = 0; k < VP_FNO_IN; ++k) s[k] = fmaf(f[k], d, s[k]);
    sb += d;
  }
  if (lane_group < groups) {
#pragma unroll
    for (int k = 0; k < VP_FNO_IN; ++k) atomicAdd(&dP[k * W + c], s[k]);
    atomicAdd(&dbP[c], sb);
  }
}

// Truncated DFT along one axis of interleaved complex FP32 data [outer][n_in][inner]:
//   mode 0 (full axis -> kept):  out[o][j][q] = sum_{i<N} in[o][i][q] w(k_j, i)
//   mode 1 (kept -> full axis):  out[o][j][q] = sum_{i<m} in[o][i][q] w(k_i, j)
// with w(k, pos) = exp(sign 2 pi i k pos / N) and the kept frequency of slot s equal
// to s for s < m/2, else N - m + s.  Used for the y and x transforms of the spectral
// convolution and their adjoints.  Block: DFT_Q threads along q, DFT_J outputs j per
// thread (twiddles of its DFT_J outputs staged in shared memory), one outer index.
constexpr int DFT_Q = 128, DFT_J = 8, DFT_MAXN = 256;

__global__ void __launch_bounds__(DFT_Q) axis_dft_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                         int N, int m, int inner, int sign, int mode, float scale,
                                                         int accumulate) {
  __shared__ float2 root[DFT_MAXN];
  __shared__ float2 tw[DFT_MAXN][DFT_J];
  const int nin = mode == 0 ? N : m;
  const int nout = mode == 0 ? m : N;
  const int o = blockIdx.z;
  const int j0 = blockIdx.y * DFT_J;
  const int q = blockIdx.x * DFT_Q + threadIdx.x;
  for (int t = threadIdx.x; t < N; t += DFT_Q) {
    float sn, cs;
    sincospif(2.f * (float)t / (float)N, &sn, &cs);
    root[t] = make_float2(cs, (float)sign * sn);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nin * DFT_J; e += DFT_Q) {
    const int i = e / DFT_J, jj = e - i * DFT_J;
    const int j = j0 + jj;
    float2 w = make_float2(0.f, 0.f);
    if (j < nout) {
      const int slot = mode == 0 ? j : i;
      const int pos = mode == 0 ? i : j;
      const int k = slot < m / 2 ? slot : N - m + slot;
      w = root[(k * pos) % N];
    }
    tw[i][jj] = w;
  }
  __syncthreads();
  if (q >= inner) return;
  float ar[DFT_J], ai[DFT_J];
#pragma unroll
  for (int jj = 0; jj < DFT_J; ++jj) ar[jj] = ai[jj] = 0.f;
  const float2* src = in + (long long)o * nin * inner + q;
#pragma unroll 4
  for (int i = 0; i < nin; ++i) {
    const float2 v = __ldg(src + (long long)i * inner);
#pragma unroll
    for (int jj = 0; jj < DFT_J; ++jj) {
      const float2 w = tw[i][jj];
      ar[jj] = fmaf(v.x, w.x, fmaf(-v.y, w.y, ar[jj]));
      ai[jj] = fmaf(v.x, w.y, fmaf(v.y, w.x, ai[jj]));
    }
  }
  float2* dst = out + (long long)o * nout * inner + q;
#pragma unroll
  for (int jj = 0; jj < DFT_J; ++jj) {
    const int j = j0 + jj;
    if (j >= nout) break;
    float2* d = dst + (long long)j * inner;
    if (accumulate) {
      d->x += scale * ar[jj];
      d->y += scale * ai[jj];
    } else {
      *d = make_float2(scale * ar[jj], scale * ai[jj]);
    }
  }
}

// axis_dft_kernel over a grid of (inner columns, output rows, outer index).
cudaError_t axis_dft(const float2* in, float2* out, int outer, int N, int m, int inner, int sign, int mode,
                     float scale, int accumulate, cudaStream_t s) {
  if (N > DFT_MAXN || outer > 65535) return cudaErrorInvalidValue;
  const int nout = mode == 0 ? m : N;
  const dim3 grid((inner + DFT_Q - 1) / DFT_Q, (nout + DFT_J - 1) / DFT_J, outer);
  axis_dft_kernel<<<grid, DFT_Q, 0, s>>>(in, out, N, m, inner, sign, mode, scale, accumulate);
  return cudaGetLastError();
}

// Per-mode channel mixing O[mode][o] = sum_c H[mode][c] R[mode][c][o] (complex), with
// H laid out [mode][c] interleaved complex and R [mode][c][o] complex (Re, Im).
// One thread per (mode, o): for each c the threads of a mode read one contiguous row.
__global__ void mix_kernel(const float2* __restrict__ in, const float2* __restrict__ R, float2* __restrict__ out,
                           int modes, int W) {
  const long long total = (long long)modes * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t % W);
    const long long md = t / W;
    const float2* h = in + md * W;
    const float2* r = R + md * W * W + j;
    float ar = 0.f, ai = 0.f;
    for (int i = 0; i < W; ++i) {
      const float2 v = h[i];
      const float2 w = __ldg(r + (long long)i * W);
      ar = fmaf(v.x, w.x, fmaf(-v.y, w.y, ar));
      ai = fmaf(v.x, w.y, fmaf(v.y, w.x, ai));
    }
    out[t] = make_float2(ar, ai);
  }
}

// Adjoint of the mixing: dH[mode][c] = sum_o dO[mode][o] conj(R[mode][c][o]).  One warp
// per (mode, c): the lanes read the contiguous row R[mode][c][:] and reduce by shuffles.
__global__ void mix_adjoint_kernel(const float2* __restrict__ dO, const float2* __restrict__ R,
                                   float2* __restrict__ dH, int modes, int W) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)modes * W;
  for (long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; wid < warps;
       wid += ((long long)gridDim.x * blockDim.x) >> 5) {
    const long long md = wid / W;
    const float2* r = R + wid * W;
    const float2* g = dO + md * W;
    float ar = 0.f, ai = 0.f;
    for (int o = lane; o < W; o += 32) {
      const float2 w = __ldg(r + o), v = g[o];
      ar = fmaf(v.x, w.x, fmaf(v.y, w.y, ar));
      ai = fmaf(v.y, w.x, fmaf(-v.x, w.y, ai));
    }
    for (int k = 16; k > 0; k >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, k);
      ai += __shfl_xor_sync(0xffffffffu, ai, k);
    }
    if (lane == 0) dH[wid] = make_float2(ar, ai);
  }
}

// dR[mode][c][o] += conj(H[mode][c]) dO[mode][o]
__global__ void mix_grad_kernel(const float2* __restrict__ H, const float2* __restrict__ dO, float* __restrict__ dR,
                                int modes, int W) {
  const long long total = (long long)modes * W * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(t % W);
    const long long r = t / W;
    const int c = (int)(r % W);
    const long long md = r / W;
    const float2 h = H[md * W + c], g = dO[md * W + o];
    dR[2 * t] += h.x * g.x + h.y * g.y;
    dR[2 * t + 1] += h.x * g.y - h.y * g.x;
  }
}

// [line][c][2mz] (FP32, from the z GEMM) -> [line][kz][c] interleaved complex
__global__ void z_to_mode_major(const float* __restrict__ in, float2* __restrict__ out, long long lines, int W,
                                int mz) {
  const long long total = lines * mz * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t % W);
    const long long r = t / W;
    const int kz = (int)(r % mz);
    const long long l = r / mz;
    const float* src = in + (l * W + c) * 2 * mz + 2 * kz;
    out[t] = make_float2(src[0], src[1]);
  }
}

// [line][kz][c] complex -> BF16 [line][2mz][c] (rows kz-major, re then im) for the
// inverse z GEMM operand
__global__ void mode_to_gemm_bf16(const float2* __restrict__ in, bf16* __restrict__ out, long long lines, int W,
                                  int mz) {
  const long long total = lines * mz * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t % W);
    const long long r = t / W;
    const int kz = (int)(r % mz);
    const long long l = r / mz;
    const float2 v = in[t];
    out[(l * 2 * mz + 2 * kz) * W + c] = __float2bfloat16(v.x);
    out[(l * 2 * mz + 2 * kz + 1) * W + c] = __float2bfloat16(v.y);
  }
}

// dt = dh * GELU'(t) (FP32 t; apply = 0: dt = dh) written in BF16 for the GEMMs that
// read it, and the column sums of dt (the bias gradient) added to dbias.  Threads
// cover cols consecutive channels of blockDim / cols rows at a time.
__global__ void __launch_bounds__(512) gelu_back_sum_kernel(const float* __restrict__ dh, const float* __restrict__ t,
                                                            bf16* __restrict__ dtb, float* __restrict__ dbias,
                                                            long long rows, int cols, int apply) {
  const int c = threadIdx.x % cols;
  const int grp = threadIdx.x / cols, groups = blockDim.x / cols;
  if (grp >= groups) return;
  float sum = 0.f;
  for (long long r = (long long)blockIdx.x * groups + grp; r < rows; r += (long long)gridDim.x * groups) {
    const long long i = r * cols + c;
    const float v = apply ? dh[i] * gelu_grad(t[i]) : dh[i];
    dtb[i] = __float2bfloat16(v);
    sum += v;
  }
  atomicAdd(&dbias[c], sum);
}

__global__ void col_sum_kernel(const float* __restrict__ a, float* __restrict__ out, long long rows, int cols) {
  const int c = threadIdx.x % cols;
  const int grp = threadIdx.x / cols, groups = blockDim.x / cols;
  if (grp >= groups) return;
  float s = 0.f;
  for (long long r = (long long)blockIdx.x * groups + grp; r < rows; r += (long long)gridDim.x * groups)
    s += a[r * cols + c];
  atomicAdd(&out[c], s);
}

// relative squared L2 per harmonic: sums over voxels of |y - q|^2 and |q|^2 (4 pairs);
// warp shuffles, then one shared-memory reduction and 8 atomics per block
__global__ void __launch_bounds__(256) loss_sums_kernel(const float* __restrict__ y, const float* __restrict__ q,
                                                        float* __restrict__ sums, long long V) {
  __shared__ float part[8][8];
  float d[4] = {0, 0, 0, 0}, t[4] = {0, 0, 0, 0};
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const float2 yy = *reinterpret_cast<const float2*>(y + 8 * v + 2 * n);
      const float2 qq = *reinterpret_cast<const float2*>(q + 8 * v + 2 * n);
      const float a = yy.x - qq.x, b = yy.y - qq.y;
      d[n] += a * a + b * b;
      t[n] += qq.x * qq.x + qq.y * qq.y;
    }
  }
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    for (int o = 16; o > 0; o >>= 1) {
      d[n] += __shfl_xor_sync(0xffffffffu, d[n], o);
      t[n] += __shfl_xor_sync(0xffffffffu, t[n], o);
    }
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      part[warp][n] = d[n];
      part[warp][4 + n] = t[n];
    }
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    float acc = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += part[w][threadIdx.x];
    atomicAdd(&sums[threadIdx.x], acc);
  }
}

// dy = (1/4) * 2 (y - q) / ||q_n||^2, as FP32 and BF16
__global__ void loss_grad_kernel(const float* __restrict__ y, const float* __restrict__ q, const float* __restrict__ sums,
                                 float* __restrict__ dy, bf16* __restrict__ dyb, long long V) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V * 8;
       i += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(i % 8) / 2;
    const float g = 0.5f * (y[i] - q[i]) / fmaxf(sums[4 + n], 1e-30f);
    dy[i] = g;
    dyb[i] = __float2bfloat16(g);
  }
}

__global__ void adam_kernel(float* __restrict__ w, bf16* __restrict__ wb, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2, float clip) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float gi = g[i] * clip;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] -= upd;
    wb[i] = __float2bfloat16(w[i]);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ a, bf16* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16(a[i]);
}

// Fused projection for inference: y = GELU(h Q1 + bQ1) Q2 + bQ2 on 64-voxel tiles
// (one warp per 16 voxels), Q1 and Q2 staged once per CTA, the hidden activation kept
// in shared memory.  Needs W, H multiples of 16 with W <= 64, H <= 128.
constexpr int PJ_ROWS = 64, PJ_MAXW = 64, PJ_MAXH = 128;
constexpr int PJ_WP = PJ_MAXW + 8, PJ_HP = PJ_MAXH + 8;  // padded rows: conflict-free fragments

constexpr size_t proj_smem_bytes() {
  return sizeof(bf16) * ((size_t)PJ_MAXH * PJ_WP + 8 * PJ_HP + PJ_ROWS * PJ_WP + PJ_ROWS * PJ_HP);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(128) proj_kernel(const bf16* __restrict__ h, const bf16* __restrict__ Q1,
                                                   const float* __restrict__ bQ1, const bf16* __restrict__ Q2,
                                                   const float* __restrict__ bQ2, float* __restrict__ y,
                                                   long long V, int W, int H) {
  extern __shared__ __align__(16) unsigned char pj_smem[];
  bf16(*q1s)[PJ_WP] = reinterpret_cast<bf16(*)[PJ_WP]>(pj_smem);                    // [H][W]: Q1^T
  bf16(*q2s)[PJ_HP] = reinterpret_cast<bf16(*)[PJ_HP]>(q1s + PJ_MAXH);              // [8][H]: Q2^T
  bf16(*hs)[PJ_WP] = reinterpret_cast<bf16(*)[PJ_WP]>(q2s + 8);                     // [64][W]
  bf16(*gs)[PJ_HP] = reinterpret_cast<bf16(*)[PJ_HP]>(hs + PJ_ROWS);                // [64][H]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
  for (int e = tid; e < W * H; e += 128) q1s[e % H][e / H] = Q1[e];
  for (int e = tid; e < H * 8; e += 128) q2s[e & 7][e >> 3] = Q2[e];
  const int r0 = warp * 16;
  const int wc = W / 8;
  for (long long tile = blockIdx.x; tile * PJ_ROWS < V; tile += gridDim.x) {
    const long long v0 = tile * PJ_ROWS;
    __syncthreads();  // staged weights ready / previous tile's reads done
    for (int e = tid; e < PJ_ROWS * wc; e += 128) {
      const int r = e / wc, c = e - r * wc;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (v0 + r < V) val = *reinterpret_cast<const uint4*>(h + (v0 + r) * W + c * 8);
      *reinterpret_cast<uint4*>(&hs[r][c * 8]) = val;
    }
    __syncthreads();
    float acc[PJ_MAXH / 8][4];
#pragma unroll
    for (int j = 0; j < PJ_MAXH / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int kk = 0; kk < W; kk += 16) {
      unsigned a[4];
      a[0] = *reinterpret_cast<const unsigned*>(&hs[r0 + gq][kk + 2 * tq]);
      a[1] = *reinterpret_cast<const unsigned*>(&hs[r0 + gq + 8][kk + 2 * tq]);
      a[2] = *reinterpret_cast<const unsigned*>(&hs[r0 + gq][kk + 2 * tq + 8]);
      a[3] = *reinterpret_cast<const unsigned*>(&hs[r0 + gq + 8][kk + 2 * tq + 8]);
#pragma unroll
      for (int j = 0; j < PJ_MAXH / 8; ++j) {
        if (j * 8 < H) {
          const unsigned b0 = *reinterpret_cast<const unsigned*>(&q1s[j * 8 + gq][kk + 2 * tq]);
          const unsigned b1 = *reinterpret_cast<const unsigned*>(&q1s[j * 8 + gq][kk + 2 * tq + 8]);
          mma16816(acc[j], a, b0, b1);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < PJ_MAXH / 8; ++j) {
      if (j * 8 < H) {
        const int col = j * 8 + 2 * tq;
        const float b0 = bQ1[col], b1 = bQ1[col + 1];
        gs[r0 + gq][col] = __float2bfloat16(gelu_f(acc[j][0] + b0));
        gs[r0 + gq][col + 1] = __float2bfloat16(gelu_f(acc[j][1] + b1));
        gs[r0 + gq + 8][col] = __float2bfloat16(gelu_f(acc[j][2] + b0));
        gs[r0 + gq + 8][col + 1] = __float2bfloat16(gelu_f(acc[j][3] + b1));
      }
    }
    __syncwarp();
    float o[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kk = 0; kk < H; kk += 16) {
      unsigned a[4];
      a[0] = *reinterpret_cast<const unsigned*>(&gs[r0 + gq][kk + 2 * tq]);
      a[1] = *reinterpret_cast<const unsigned*>(&gs[r0 + gq + 8][kk + 2 * tq]);
      a[2] = *reinterpret_cast<const unsigned*>(&gs[r0 + gq][kk + 2 * tq + 8]);
      a[3] = *reinterpret_cast<const unsigned*>(&gs[r0 + gq + 8][kk + 2 * tq + 8]);
      const unsigned b0 = *reinterpret_cast<const unsigned*>(&q2s[gq][kk + 2 * tq]);
      const unsigned b1 = *reinterpret_cast<const unsigned*>(&q2s[gq][kk + 2 * tq + 8]);
      mma16816(o, a, b0, b1);
    }
    const int col = 2 * tq;
    const long long ra = v0 + r0 + gq, rb = ra + 8;
    if (ra < V) *reinterpret_cast<float2*>(y + ra * 8 + col) = make_float2(o[0] + bQ2[col], o[1] + bQ2[col + 1]);
    if (rb < V) *reinterpret_cast<float2*>(y + rb * 8 + col) = make_float2(o[2] + bQ2[col], o[3] + bQ2[col + 1]);
  }
}

// ---- layout of parameters and workspace ----------------------------------------------

struct Layout {
  long long P, bP, R[VP_FNO_MAX_LAYERS], W[VP_FNO_MAX_LAYERS], b[VP_FNO_MAX_LAYERS], Q1, bQ1, Q2, bQ2, total;
  long long modes;
};

bool desc_ok(const vp_fno_desc* d) {
  if (!d) return false;
  const int N = d->n;
  return N >= 4 && N <= 256 && d->width >= 1 && d->width <= 256 && d->hidden >= 1 && d->hidden <= 512 &&
         d->layers >= 1 && d->layers <= VP_FNO_MAX_LAYERS && d->modes[0] >= 2 && d->modes[0] % 2 == 0 &&
         d->modes[0] <= N && d->modes[1] >= 2 && d->modes[1] % 2 == 0 && d->modes[1] <= N && d->modes[2] >= 1 &&
         d->modes[2] <= N / 2;
}

Layout layout(const vp_fno_desc* d) {
  Layout L;
  std::memset(&L, 0, sizeof(L));
  const long long W = d->width, H = d->hidden;
  L.modes = (long long)d->modes[0] * d->modes[1] * d->modes[2];
  long long o = 0;
  L.P = o; o += VP_FNO_IN * W;
  L.bP = o; o += W;
  for (int l = 0; l < d->layers; ++l) {
    L.R[l] = o; o += L.modes * W * W * 2;
    L.W[l] = o; o += W * W;
    L.b[l] = o; o += W;
  }
  L.Q1 = o; o += W * H;
  L.bQ1 = o; o += H;
  L.Q2 = o; o += H * 8;
  L.bQ2 = o; o += 8;
  L.total = o;
  return L;
}

// Workspace (bytes) for one sample: every activation the backward pass needs.
struct Work {
  long long V, lines, W, H, mz, modes2d;
  // offsets in bytes
  long long hb[VP_FNO_MAX_LAYERS + 1];  // bf16 activations h_0 .. h_L  [V][W]
  long long t[VP_FNO_MAX_LAYERS];       // fp32 pre-activations [V][W]
  long long hz[VP_FNO_MAX_LAYERS];      // fp32 complex [line][kz][c] after the z transform
  long long hx[VP_FNO_MAX_LAYERS];      // fp32 complex [kx][ky][kz][c] (mixing input)
  long long u, gb, y;                   // projection: u fp32 [V][H], g bf16 [V][H], y fp32 [V][8]
  long long fz, gz;                     // bf16 DFT matrices: forward [N][2mz], inverse [N][2mz]
  long long zgemm;                      // fp32 [line][c][2mz] scratch
  long long cplx_a, cplx_b;             // fp32 complex scratch (largest spectral buffer)
  long long s;                          // fp32 [V][W] spectral branch output / gradient scratch
  long long bfa;                        // bf16 [V][max(W,H)] scratch
  long long dh, dh2;                    // fp32 [V][max(W,H)] gradients
  long long sums;                       // fp32 [8]
  long long total;
};

Work work(const vp_fno_desc* d) {
  Work w;
  std::memset(&w, 0, sizeof(w));
  const long long N = d->n;
  w.V = N * N * N;
  w.lines = N * N;
  w.W = d->width;
  w.H = d->hidden;
  w.mz = d->modes[2];
  const long long mx = d->modes[0], my = d->modes[1];
  const long long WH = w.W > w.H ? w.W : w.H;
  long long o = 0;
  auto take = [&](long long bytes) {
    const long long at = o;
    o += (bytes + 255) / 256 * 256;
    return at;
  };
  for (int l = 0; l <= d->layers; ++l) w.hb[l] = take(w.V * w.W * 2);
  for (int l = 0; l < d->layers; ++l) {
    w.t[l] = take(w.V * w.W * 4);
    w.hz[l] = take(w.lines * w.mz * w.W * 8);
    w.hx[l] = take(mx * my * w.mz * w.W * 8);
  }
  w.u = take(w.V * w.H * 4);
  w.gb = take(w.V * w.H * 2);
  w.y = take(w.V * 8 * 4);
  w.fz = take(N * 2 * w.mz * 2);
  w.gz = take(N * 2 * w.mz * 2);
  w.zgemm = take(w.lines * w.W * 2 * w.mz * 4);
  const long long cpl = (N * my > mx * my ? N * my : mx * my) * w.mz * w.W * 8;
  const long long cpl2 = w.lines * w.mz * w.W * 8;
  w.cplx_a = take(cpl > cpl2 ? cpl : cpl2);
  w.cplx_b = take(cpl > cpl2 ? cpl : cpl2);
  w.s = take(w.V * w.W * 4);
  w.bfa = take(w.V * WH * 2);
  w.dh = take(w.V * WH * 4);
  w.dh2 = take(w.V * WH * 4);
  w.sums = take(8 * 4);
  w.total = o;
  return w;
}

template <typename T>
T* at(void* base, long long off) {
  return reinterpret_cast<T*>(reinterpret_cast<char*>(base) + off);
}

__global__ void dft_tables_kernel(bf16* fz, bf16* gz, int N, int mz) {
  // fz[z][2kz + r]: forward  cos(2 pi kz z / N), -sin(...)
  // gz[z][2kz + r]: inverse real output weights c_kz cos(.), -c_kz sin(.), divided by N^3
  const int total = N * 2 * mz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int z = i / (2 * mz);
    const int c = i - z * 2 * mz;
    const int kz = c / 2, r = c & 1;
    double s, co;
    sincospi(2.0 * (double)((kz * z) % N) / (double)N, &s, &co);
    const double f = r == 0 ? co : -s;
    fz[i] = __float2bfloat16((float)f);
    const double ck = kz == 0 ? 1.0 : 2.0;
    const double N3 = (double)N * N * N;
    gz[i] = __float2bfloat16((float)(ck * f / N3));
  }
}

int st(cudaError_t e) { return e == cudaSuccess ? VP_OK : VP_ERR_CUDA; }

// Z[line][c][j] = sum_z A[line][z][c] T[z][j] for every line (A BF16 [lines][N][W],
// T BF16 [N][2mz], Z FP32 [lines][W][2mz]): one GEMM with rows (line, c).
cudaError_t z_transform(const bf16* A, const bf16* T, float* Z, long long lines, int N, int W, int mz,
                        cudaStream_t s) {
  if (lines * W > 0x7fffffffLL) return cudaErrorInvalidValue;
  Gemm g = gemm_base();
  g.M = (int)(lines * W); g.N = 2 * mz; g.K = N;
  g.A = A; g.a_rs = 1; g.a_cs = W; g.a_group = W; g.a_gstride = (long long)N * W;
  g.B = T; g.b_rs = 2 * mz; g.b_cs = 1;
  g.C = Z; g.c_rs = 2 * mz; g.c_cs = 1;
  return gemm(g, s);
}

// Forward pass.  train = true keeps every activation the backward pass reads (FP32
// pre-activations t_l and u, BF16 h_l, the truncated spectra) and leaves y in ws;
// train = false writes only what the next step reads (BF16 h in two alternating
// buffers) and fuses the projection.  Where N is a multiple of the GEMM tile height
// the inverse z transform of the spectral branch is a second contraction inside the
// pointwise GEMM, so the branch output never goes to memory.
int forward_impl(const vp_fno_desc* d, const float* params, const bf16* pb, const float* x, float* y, void* ws,
                 cudaStream_t s, bool train) {
  const Layout L = layout(d);
  const Work w = work(d);
  const int N = d->n, W = d->width, H = d->hidden, mx = d->modes[0], my = d->modes[1], mz = d->modes[2];
  cudaError_t e;
  dft_tables_kernel<<<16, 256, 0, s>>>(at<bf16>(ws, w.fz), at<bf16>(ws, w.gz), N, mz);
  lift_kernel<<<grid1(w.V * W, 256), 256, 0, s>>>(x, params + L.P, params + L.bP, at<bf16>(ws, w.hb[0]), w.V, W);
  if ((e = cudaGetLastError()) != cudaSuccess) return st(e);
  const bool fused = N % BM == 0 && (2 * mz) % 8 == 0 && W % 8 == 0;
  for (int l = 0; l < d->layers; ++l) {
    const bf16* h = at<bf16>(ws, w.hb[train ? l : (l & 1)]);
    bf16* h_next = at<bf16>(ws, w.hb[train ? l + 1 : ((l + 1) & 1)]);
    float2* hz = at<float2>(ws, w.hz[train ? l : 0]);
    float2* hx = at<float2>(ws, w.hx[train ? l : 0]);
    // z transform of every line as one GEMM over rows (line, c):
    //   Z[line][c][kz r] = sum_z h[line][z][c] fz[z][kz r]
    if ((e = z_transform(h, at<bf16>(ws, w.fz), at<float>(ws, w.zgemm), w.lines, N, W, mz, s)) != cudaSuccess)
      return st(e);
    z_to_mode_major<<<grid1(w.lines * mz * W, 256), 256, 0, s>>>(at<float>(ws, w.zgemm), hz, w.lines, W, mz);
    // y then x transforms to the kept modes: [x][y][kz c] -> [x][ky][kz c] -> [kx][ky][kz c]
    float2* ca = at<float2>(ws, w.cplx_a);
    if ((e = axis_dft(hz, ca, N, N, my, mz * W, -1, 0, 1.f, 0, s)) != cudaSuccess) return st(e);
    if ((e = axis_dft(ca, hx, 1, N, mx, my * mz * W, -1, 0, 1.f, 0, s)) != cudaSuccess) return st(e);
    // mixing
    float2* cb = at<float2>(ws, w.cplx_b);
    mix_kernel<<<grid1((long long)mx * my * mz * W, 256), 256, 0, s>>>(
        hx, reinterpret_cast<const float2*>(params + L.R[l]), cb, mx * my * mz, W);
    // inverse x then y (kept -> full), scaled later by the z inverse weights (1/N^3)
    if ((e = axis_dft(cb, ca, 1, N, mx, my * mz * W, 1, 1, 1.f, 0, s)) != cudaSuccess) return st(e);
    if ((e = axis_dft(ca, cb, N, N, my, mz * W, 1, 1, 1.f, 0, s)) != cudaSuccess) return st(e);
    bf16* ob = at<bf16>(ws, w.bfa);
    mode_to_gemm_bf16<<<grid1(w.lines * mz * W, 256), 256, 0, s>>>(cb, ob, w.lines, W, mz);
    if ((e = cudaGetLastError()) != cudaSuccess) return st(e);
    // t = h W_l + b_l + s with s[(line, z)][o] = sum_(kz, r) gz[z][kz r] O[line][kz r][o];
    // h_{l+1} = GELU(t) (not after the last layer)
    Gemm gl = gemm_base();
    gl.M = (int)w.V; gl.N = W; gl.K = W;
    gl.A = h; gl.a_rs = W; gl.a_cs = 1;
    gl.B = pb + L.W[l]; gl.b_rs = W; gl.b_cs = 1;
    gl.C = train ? at<float>(ws, w.t[l]) : nullptr; gl.c_rs = W; gl.c_cs = 1;
    gl.Cb = h_next;
    gl.bias = params + L.b[l];
    gl.gelu = l < d->layers - 1;
    if (fused) {
      gl.A2 = at<bf16>(ws, w.gz); gl.a2_rs = 2 * mz;
      gl.B2 = ob; gl.b2_rs = W; gl.b2_line = 2LL * mz * W;
      gl.K2 = 2 * mz; gl.rows_per_line = N;
    } else {
      Gemm gi = gemm_base();
      gi.M = N; gi.N = W; gi.K = 2 * mz; gi.batch = (int)w.lines;
      gi.A = at<bf16>(ws, w.gz); gi.a_rs = 2 * mz; gi.a_cs = 1; gi.a_bs = 0;
      gi.B = ob; gi.b_rs = W; gi.b_cs = 1; gi.b_bs = 2LL * mz * W;
      gi.C = at<float>(ws, w.s); gi.c_rs = W; gi.c_cs = 1; gi.c_bs = (long long)N * W;
      if ((e = gemm(gi, s)) != cudaSuccess) return st(e);
      gl.addend = at<float>(ws, w.s);
    }
    if ((e = gemm(gl, s)) != cudaSuccess) return st(e);
  }
  const bf16* hL = at<bf16>(ws, w.hb[train ? d->layers : (d->layers & 1)]);
  if (!train && W % 16 == 0 && H % 16 == 0 && W <= PJ_MAXW && H <= PJ_MAXH) {
    const long long tiles = (w.V + PJ_ROWS - 1) / PJ_ROWS;
    const int grid = (int)std::min<long long>(tiles, 152LL * 4);
    proj_kernel<<<grid, 128, proj_smem_bytes(), s>>>(hL, pb + L.Q1, params + L.bQ1, pb + L.Q2, params + L.bQ2, y,
                                                    w.V, W, H);
    return st(cudaGetLastError());
  }
  // projection as two GEMMs
  Gemm g1 = gemm_base();
  g1.M = (int)w.V; g1.N = H; g1.K = W;
  g1.A = hL; g1.a_rs = W; g1.a_cs = 1;
  g1.B = pb + L.Q1; g1.b_rs = H; g1.b_cs = 1;
  g1.C = train ? at<float>(ws, w.u) : nullptr; g1.c_rs = H; g1.c_cs = 1;
  g1.Cb = at<bf16>(ws, w.gb);
  g1.bias = params + L.bQ1;
  g1.gelu = 1;
  if ((e = gemm(g1, s)) != cudaSuccess) return st(e);
  Gemm g2 = gemm_base();
  g2.M = (int)w.V; g2.N = 8; g2.K = H;
  g2.A = at<bf16>(ws, w.gb); g2.a_rs = H; g2.a_cs = 1;
  g2.B = pb + L.Q2; g2.b_rs = 8; g2.b_cs = 1;
  g2.C = train ? at<float>(ws, w.y) : y; g2.c_rs = 8; g2.c_cs = 1;
  g2.bias = params + L.bQ2;
  if ((e = gemm(g2, s)) != cudaSuccess) return st(e);
  if (train && y) {
    e = cudaMemcpyAsync(y, at<float>(ws, w.y), w.V * 8 * 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return st(e);
  }
  return st(cudaGetLastError());
}


}  // namespace

extern "C" {

VP_API long long vp_fno_param_count(const vp_fno_desc* d) { return desc_ok(d) ? layout(d).total : -1; }

VP_API int vp_fno_param_offsets(const vp_fno_desc* d, long long* off) {
  if (!desc_ok(d) || !off) return VP_ERR_ARG;
  const Layout L = layout(d);
  int k = 0;
  off[k++] = L.P;
  off[k++] = L.bP;
  for (int l = 0; l < d->layers; ++l) {
    off[k++] = L.R[l];
    off[k++] = L.W[l];
    off[k++] = L.b[l];
  }
  off[k++] = L.Q1;
  off[k++] = L.bQ1;
  off[k++] = L.Q2;
  off[k++] = L.bQ2;
  off[k++] = L.total;
  return VP_OK;
}

VP_API long long vp_fno_workspace_bytes(const vp_fno_desc* d) { return desc_ok(d) ? work(d).total : -1; }

VP_API int vp_fno_forward(const vp_fno_desc* d, const float* params, const void* params_bf16, const float* x,
                          float* y, void* ws, vp_stream_t stream) {
  if (!desc_ok(d) || !params || !params_bf16 || !x || !ws) return VP_ERR_ARG;
  return forward_impl(d, params, (const bf16*)params_bf16, x, y, ws, (cudaStream_t)stream, true);
}

VP_API int vp_fno_infer(const vp_fno_desc* d, const float* params, const void* params_bf16, const float* x, float* y,
                        void* ws, vp_stream_t stream) {
  if (!desc_ok(d) || !params || !params_bf16 || !x || !y || !ws) return VP_ERR_ARG;
  return forward_impl(d, params, (const bf16*)params_bf16, x, y, ws, (cudaStream_t)stream, false);
}

VP_API int vp_fno_loss(const vp_fno_desc* d, const float* target, float* sums8, void* ws, vp_stream_t stream) {
  if (!desc_ok(d) || !target || !ws) return VP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Work w = work(d);
  float* sums = at<float>(ws, w.sums);
  cudaError_t e = cudaMemsetAsync(sums, 0, 8 * 4, s);
  if (e != cudaSuccess) return st(e);
  loss_sums_kernel<<<grid1(w.V, 256), 256, 0, s>>>(at<float>(ws, w.y), target, sums, w.V);
  if ((e = cudaGetLastError()) != cudaSuccess) return st(e);
  if (sums8) e = cudaMemcpyAsync(sums8, sums, 8 * 4, cudaMemcpyDeviceToDevice, s);
  return st(e);
}

VP_API int vp_fno_backward(const vp_fno_desc* d, const float* params, const void* params_bf16, const float* x,
                           const float* target, float* grads, void* ws, vp_stream_t stream) {
  if (!desc_ok(d) || !params || !params_bf16 || !x || !target || !grads || !ws) return VP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const Layout L = layout(d);
  const Work w = work(d);
  const int N = d->n, W = d->width, H = d->hidden, mx = d->modes[0], my = d->modes[1], mz = d->modes[2];
  const bf16* pb = (const bf16*)params_bf16;
  cudaError_t e;
  // loss gradient dy (uses the sums of vp_fno_loss)
  float* dy = at<float>(ws, w.dh);
  bf16* dyb = at<bf16>(ws, w.bfa);
  loss_grad_kernel<<<grid1(w.V * 8, 256), 256, 0, s>>>(at<float>(ws, w.y), target, at<float>(ws, w.sums), dy, dyb, w.V);
  // Q2: dQ2 += g^T dy, dbQ2 += sum dy
  // weight gradients contract over every voxel: split K so that ~8 CTAs per SM are busy
  const int ksplit_v = (int)std::max<long long>(1, std::min<long long>(152LL * 8, w.V / 256));
  const bool fused = N % BM == 0 && (2 * mz) % 8 == 0 && W % 8 == 0;
  Gemm g = gemm_base();
  g.M = H; g.N = 8; g.K = (int)w.V; g.ksplit = ksplit_v; g.accumulate = 1;
  g.A = at<bf16>(ws, w.gb); g.a_rs = 1; g.a_cs = H;
  g.B = dyb; g.b_rs = 8; g.b_cs = 1;
  g.C = grads + L.Q2; g.c_rs = 8; g.c_cs = 1;
  if ((e = gemm(g, s)) != cudaSuccess) return st(e);
  col_sum_kernel<<<152 * 8, 256, 0, s>>>(dy, grads + L.bQ2, w.V, 8);
  // dg = dy Q2^T ; du = dg * GELU'(u)
  float* dg = at<float>(ws, w.dh2);
  g = gemm_base();
  g.M = (int)w.V; g.N = H; g.K = 8;
  g.A = dyb; g.a_rs = 8; g.a_cs = 1;
  g.B = pb + L.Q2; g.b_rs = 1; g.b_cs = 8;
  g.C = dg; g.c_rs = H; g.c_cs = 1;
  if ((e = gemm(g, s)) != cudaSuccess) return st(e);
  bf16* dub = at<bf16>(ws, w.bfa);
  gelu_back_sum_kernel<<<152 * 8, H <= 256 ? 256 : 512, 0, s>>>(dg, at<float>(ws, w.u), dub, grads + L.bQ1, w.V,
                                                                H, 1);
  // dQ1 += h_L^T du, dbQ1 += sum du, dh_L = du Q1^T
  g = gemm_base();
  g.M = W; g.N = H; g.K = (int)w.V; g.ksplit = ksplit_v; g.accumulate = 1;
  g.A = at<bf16>(ws, w.hb[d->layers]); g.a_rs = 1; g.a_cs = W;
  g.B = dub; g.b_rs = H; g.b_cs = 1;
  g.C = grads + L.Q1; g.c_rs = H; g.c_cs = 1;
  if ((e = gemm(g, s)) != cudaSuccess) return st(e);
  float* dh = at<float>(ws, w.dh2);
  g = gemm_base();
  g.M = (int)w.V; g.N = W; g.K = H;
  g.A = dub; g.a_rs = H; g.a_cs = 1;
  g.B = pb + L.Q1; g.b_rs = 1; g.b_cs = H;
  g.C = dh; g.c_rs = W; g.c_cs = 1;
  if ((e = gemm(g, s)) != cudaSuccess) return st(e);
  for (int l = d->layers - 1; l >= 0; --l) {
    // dt = dh (* GELU'(t) if activated) in BF16, bias gradient = column sums of dt
    bf16* dtb = at<bf16>(ws, w.bfa);
    gelu_back_sum_kernel<<<152 * 8, W <= 256 ? 256 : 512, 0, s>>>(dh, at<float>(ws, w.t[l]), dtb,
                                                                  grads + L.b[l], w.V, W, l < d->layers - 1);
    // dW_l += h_l^T dt
    g = gemm_base();
    g.M = W; g.N = W; g.K = (int)w.V; g.ksplit = ksplit_v; g.accumulate = 1;
    g.A = at<bf16>(ws, w.hb[l]); g.a_rs = 1; g.a_cs = W;
    g.B = dtb; g.b_rs = W; g.b_cs = 1;
    g.C = grads + L.W[l]; g.c_rs = W; g.c_cs = 1;
    if ((e = gemm(g, s)) != cudaSuccess) return st(e);
    // spectral branch adjoint: dO[line][o][kz r] = sum_z dt[line][z][o] gz[z][kz r]
    if ((e = z_transform(dtb, at<bf16>(ws, w.gz), at<float>(ws, w.zgemm), w.lines, N, W, mz, s)) != cudaSuccess)
      return st(e);
    float2* ca = at<float2>(ws, w.cplx_a);
    float2* cb = at<float2>(ws, w.cplx_b);
    z_to_mode_major<<<grid1(w.lines * mz * W, 256), 256, 0, s>>>(at<float>(ws, w.zgemm), cb, w.lines, W, mz);
    // adjoints of the inverse y and x transforms (full -> kept, conjugate phase)
    if ((e = axis_dft(cb, ca, N, N, my, mz * W, -1, 0, 1.f, 0, s)) != cudaSuccess) return st(e);
    if ((e = axis_dft(ca, cb, 1, N, mx, my * mz * W, -1, 0, 1.f, 0, s)) != cudaSuccess) return st(e);
    // mixing: dR += conj(H) dO, dH = dO conj(R)^T
    const float2* hx = at<float2>(ws, w.hx[l]);
    mix_grad_kernel<<<grid1((long long)mx * my * mz * W * W, 256), 256, 0, s>>>(hx, cb, grads + L.R[l], mx * my * mz, W);
    mix_adjoint_kernel<<<grid1((long long)mx * my * mz * W * 32, 256), 256, 0, s>>>(
        cb, reinterpret_cast<const float2*>(params + L.R[l]), ca, mx * my * mz, W);
    // adjoints of the forward x and y transforms (kept -> full, conjugate phase)
    if ((e = axis_dft(ca, cb, 1, N, mx, my * mz * W, 1, 1, 1.f, 0, s)) != cudaSuccess) return st(e);
    if ((e = axis_dft(cb, ca, N, N, my, mz * W, 1, 1, 1.f, 0, s)) != cudaSuccess) return st(e);
    // dZ as BF16 [line][kz r][c]; dt (BF16) is still needed by the next GEMM
    bf16* dzb = at<bf16>(ws, w.dh);  // FP32 scratch of [V][max(W, H)]: free during the layer loop
    mode_to_gemm_bf16<<<grid1(w.lines * mz * W, 256), 256, 0, s>>>(ca, dzb, w.lines, W, mz);
    // dh_l = dt W_l^T + (z-transform adjoint: sum_(kz r) fz[z][kz r] dZ[line][kz r][c])
    float* dhn = at<float>(ws, w.dh2);
    g = gemm_base();
    g.M = (int)w.V; g.N = W; g.K = W;
    g.A = dtb; g.a_rs = W; g.a_cs = 1;
    g.B = pb + L.W[l]; g.b_rs = 1; g.b_cs = W;
    g.C = dhn; g.c_rs = W; g.c_cs = 1;
    if (fused) {
      g.A2 = at<bf16>(ws, w.fz); g.a2_rs = 2 * mz;
      g.B2 = dzb; g.b2_rs = W; g.b2_line = 2LL * mz * W;
      g.K2 = 2 * mz; g.rows_per_line = N;
      if ((e = gemm(g, s)) != cudaSuccess) return st(e);
    } else {
      if ((e = gemm(g, s)) != cudaSuccess) return st(e);
      g = gemm_base();
      g.M = N; g.N = W; g.K = 2 * mz; g.batch = (int)w.lines; g.accumulate = 1;
      g.A = at<bf16>(ws, w.fz); g.a_rs = 2 * mz; g.a_cs = 1; g.a_bs = 0;
      g.B = dzb; g.b_rs = W; g.b_cs = 1; g.b_bs = 2LL * mz * W;
      g.C = dhn; g.c_rs = W; g.c_cs = 1; g.c_bs = (long long)N * W;
      if ((e = gemm(g, s)) != cudaSuccess) return st(e);
    }
    dh = dhn;
  }
  lift_grad_kernel<<<152 * 8, 256, 0, s>>>(x, dh, grads + L.P, grads + L.bP, w.V, W);
  return st(cudaGetLastError());
}

}  // extern "C"

extern "C" {

VP_API int vp_fno_adam(long long n, float* params, void* params_bf16, const float* grads, float* m, float* v,
                       float lr, float b1, float b2, float eps, float c1, float c2, float grad_scale,
                       vp_stream_t stream) {
  if (n < 1 || !params || !params_bf16 || !grads || !m || !v) return VP_ERR_ARG;
  adam_kernel<<<grid1(n, 256), 256, 0, (cudaStream_t)stream>>>(params, (bf16*)params_bf16, grads, m, v, n, lr, b1,
                                                                b2, eps, c1, c2, grad_scale);
  return st(cudaGetLastError());
}

VP_API int vp_fno_to_bf16(long long n, const float* src, void* dst, vp_stream_t stream) {
  if (n < 1 || !src || !dst) return VP_ERR_ARG;
  to_bf16_kernel<<<grid1(n, 256), 256, 0, (cudaStream_t)stream>>>(src, (bf16*)dst, n);
  return st(cudaGetLastError());
}

}  // extern "C"
