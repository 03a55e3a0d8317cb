// Fourier-neural-operator surrogate kernels: BF16 tensor-core GEMM with fused
// epilogues, truncated spectral transforms, channel mixing, GELU, loss and Adam.
//
// The surrogate maps the normalised fundamental on an N^3 focal box (2 channels) to the
// normalised harmonics 2..5 (8 channels); see include/vp_fno.h for the architecture.
// Activations are [voxel][channel] (x slowest, z, then channel fastest); a "line" is
// one (x, y) column of N voxels along z.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
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
};

constexpr int BM = 64, BN = 64, BK = 32, KP = BK + 8;  // padded rows: conflict-free fragments

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * __expf(-0.5f * x * x);
  return cdf + x * pdf;
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
  const bool a_kfast = g.a_cs == 1;
  const bool b_nfast = g.b_cs == 1;
  const bf16 zero = __float2bfloat16(0.f);
  for (int k0 = k_begin; k0 < k_end; k0 += BK) {
    // A tile: BM x BK
    for (int e = tid; e < BM * BK; e += 128) {
      int m, k;
      if (a_kfast) { k = e % BK; m = e / BK; } else { m = e % BM; k = e / BM; }
      const int gm = m0 + m, gk = k0 + k;
      As[m][k] = (gm < g.M && gk < k_end) ? A[(long long)gm * g.a_rs + (long long)gk * g.a_cs] : zero;
    }
    // B tile: BK x BN, stored n-major
    for (int e = tid; e < BK * BN; e += 128) {
      int n, k;
      if (b_nfast) { n = e % BN; k = e / BN; } else { k = e % BK; n = e / BK; }
      const int gn = n0 + n, gk = k0 + k;
      Bs[n][k] = (gn < g.N && gk < k_end) ? B[(long long)gk * g.b_rs + (long long)gn * g.b_cs] : zero;
    }
    __syncthreads();
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
    __syncthreads();
  }
  // epilogue
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + i * 16 + gq + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + 2 * tq + (r & 1);
        if (m >= g.M || n >= g.N) continue;
        const long long off = (long long)b * g.c_bs + (long long)m * g.c_rs + (long long)n * g.c_cs;
        float v = acc[i][j][r];
        if (ks == 0) {
          if (g.bias) v += g.bias[n];
          if (g.addend) v += g.addend[off];
        }
        if (g.accumulate) {
          if (g.ksplit > 1) atomicAdd(&g.C[off], v);
          else g.C[off] += v;
          continue;
        }
        if (g.C) g.C[off] = v;
        if (g.Cb) g.Cb[off] = __float2bfloat16(g.gelu ? gelu_f(v) : v);
      }
}

cudaError_t gemm(const Gemm& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.ksplit > 1 && !(g.accumulate && g.batch == 1)) return cudaErrorInvalidValue;
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

// h0[v][c] = x[v][0] P[0][c] + x[v][1] P[1][c] + bP[c]
__global__ void lift_kernel(const float* __restrict__ x, const float* __restrict__ P, const float* __restrict__ bP,
                            bf16* __restrict__ h, long long V, int W) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V * W; i += (long long)gridDim.x * blockDim.x) {
    const long long v = i / W;
    const int c = (int)(i - v * W);
    h[i] = __float2bfloat16(fmaf(x[2 * v], P[c], fmaf(x[2 * v + 1], P[W + c], bP[c])));
  }
}

// dP += x^T dh, dbP += sum dh  (dh: fp32 [V][W]); one thread per (c) accumulates a
// slice of voxels, then atomics.
__global__ void lift_grad_kernel(const float* __restrict__ x, const float* __restrict__ dh, float* __restrict__ dP,
                                 float* __restrict__ dbP, long long V, int W) {
  const int c = threadIdx.x % W;
  const int lane_group = threadIdx.x / W;
  const int groups = blockDim.x / W;
  float s0 = 0.f, s1 = 0.f, sb = 0.f;
  for (long long v = (long long)blockIdx.x * groups + lane_group; v < V; v += (long long)gridDim.x * groups) {
    const float d = dh[v * W + c];
    s0 = fmaf(x[2 * v], d, s0);
    s1 = fmaf(x[2 * v + 1], d, s1);
    sb += d;
  }
  if (lane_group < groups) {
    atomicAdd(&dP[c], s0);
    atomicAdd(&dP[W + c], s1);
    atomicAdd(&dbP[c], sb);
  }
}

// y (complex, [rows][...]) : out[x][ko][inner] = sum_i in[x][i][inner] w(i, k_o) with
// w = exp(sign 2 pi i k i / N) for the kept frequencies k_o of an axis.  Data are
// interleaved complex FP32 with `inner` complex values per (x, i).  Used for the y and
// x transforms of the truncated spectrum and their adjoints (kept -> full axis too).
// mode 0: full axis (N) -> kept (m);  mode 1: kept (m) -> full axis (N).
__global__ void axis_dft_kernel(const float2* __restrict__ in, float2* __restrict__ out, int outer, int N, int m,
                                int inner, int sign, int mode, float scale, int accumulate) {
  const int nin = mode == 0 ? N : m;
  const int nout = mode == 0 ? m : N;
  const long long total = (long long)outer * nout * inner;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t % inner);
    const long long r = t / inner;
    const int jo = (int)(r % nout);
    const int o = (int)(r / nout);
    // frequency of kept slot j: j < m/2 -> j, else N - m + j
    float ar = 0.f, ai = 0.f;
    for (int ji = 0; ji < nin; ++ji) {
      const int pos = mode == 0 ? ji : jo;
      const int slot = mode == 0 ? jo : ji;
      const int k = slot < m / 2 ? slot : N - m + slot;
      const int ph = (int)(((long long)k * pos) % N);
      float sn, cs;
      sincospif(2.f * (float)ph / (float)N, &sn, &cs);
      sn *= (float)sign;
      const float2 v = in[((long long)o * nin + ji) * inner + q];
      ar += v.x * cs - v.y * sn;
      ai += v.x * sn + v.y * cs;
    }
    float2* dst = &out[t];
    if (accumulate) {
      dst->x += scale * ar;
      dst->y += scale * ai;
    } else {
      *dst = make_float2(scale * ar, scale * ai);
    }
  }
}

// Per-mode channel mixing O[mode][o] = sum_c H[mode][c] R[mode][c][o] (complex), with
// H laid out [mode][c] interleaved complex and R [mode][c][o][2] FP32.
// adjoint = 1: dH[mode][c] = sum_o dO[mode][o] conj(R[mode][c][o]).
__global__ void mix_kernel(const float2* __restrict__ in, const float* __restrict__ R, float2* __restrict__ out,
                           int modes, int W, int adjoint) {
  const long long total = (long long)modes * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t % W);
    const long long md = t / W;
    const float2* h = in + md * W;
    const float* r = R + md * W * W * 2;
    float ar = 0.f, ai = 0.f;
    for (int i = 0; i < W; ++i) {
      const float2 v = h[i];
      float rr, ri;
      if (!adjoint) {
        rr = r[(i * W + j) * 2];
        ri = r[(i * W + j) * 2 + 1];
        ar += v.x * rr - v.y * ri;
        ai += v.x * ri + v.y * rr;
      } else {
        rr = r[(j * W + i) * 2];
        ri = r[(j * W + i) * 2 + 1];
        ar += v.x * rr + v.y * ri;
        ai += v.y * rr - v.x * ri;
      }
    }
    out[t] = make_float2(ar, ai);
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

// [line][c][2mz] FP32 (gradient w.r.t. the forward z transform's output, as the GEMM
// laid it out) from the complex [line][kz][c] gradient, in BF16 for the adjoint GEMM
__global__ void mode_to_zgrad_bf16(const float2* __restrict__ in, bf16* __restrict__ out, long long lines, int W,
                                   int mz) {
  const long long total = lines * mz * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t % W);
    const long long r = t / W;
    const int kz = (int)(r % mz);
    const long long l = r / mz;
    const float2 v = in[t];
    out[(l * W + c) * 2 * mz + 2 * kz] = __float2bfloat16(v.x);
    out[(l * W + c) * 2 * mz + 2 * kz + 1] = __float2bfloat16(v.y);
  }
}

// [line][2mz][o] real pairs (re row, im row per kz) -> complex [line][kz][o]
__global__ void pairs_to_complex(const float* __restrict__ in, float2* __restrict__ out, long long lines, int W,
                                 int mz) {
  const long long total = lines * mz * W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int o = (int)(t % W);
    const long long r = t / W;
    const int kz = (int)(r % mz);
    const long long l = r / mz;
    out[t] = make_float2(in[(l * 2 * mz + 2 * kz) * W + o], in[(l * 2 * mz + 2 * kz + 1) * W + o]);
  }
}

// dt = dh * GELU'(t) (FP32 t), written as FP32 and BF16
__global__ void gelu_back_kernel(const float* __restrict__ dh, const float* __restrict__ t, float* __restrict__ dt,
                                 bf16* __restrict__ dtb, long long n, int apply) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = apply ? dh[i] * gelu_grad(t[i]) : dh[i];
    dt[i] = v;
    dtb[i] = __float2bfloat16(v);
  }
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

// relative squared L2 per harmonic: sums over voxels of |y - q|^2 and |q|^2 (4 pairs)
__global__ void loss_sums_kernel(const float* __restrict__ y, const float* __restrict__ q, float* __restrict__ sums,
                                 long long V) {
  float d[4] = {0, 0, 0, 0}, t[4] = {0, 0, 0, 0};
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      const float a = y[8 * v + 2 * n] - q[8 * v + 2 * n], b = y[8 * v + 2 * n + 1] - q[8 * v + 2 * n + 1];
      d[n] += a * a + b * b;
      t[n] += q[8 * v + 2 * n] * q[8 * v + 2 * n] + q[8 * v + 2 * n + 1] * q[8 * v + 2 * n + 1];
    }
  }
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    for (int o = 16; o > 0; o >>= 1) {
      d[n] += __shfl_xor_sync(0xffffffffu, d[n], o);
      t[n] += __shfl_xor_sync(0xffffffffu, t[n], o);
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      atomicAdd(&sums[n], d[n]);
      atomicAdd(&sums[4 + n], t[n]);
    }
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
  L.P = o; o += 2 * W;
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
  cudaStream_t s = (cudaStream_t)stream;
  const Layout L = layout(d);
  const Work w = work(d);
  const int N = d->n, W = d->width, H = d->hidden, mx = d->modes[0], my = d->modes[1], mz = d->modes[2];
  const bf16* pb = (const bf16*)params_bf16;
  cudaError_t e;
  dft_tables_kernel<<<16, 256, 0, s>>>(at<bf16>(ws, w.fz), at<bf16>(ws, w.gz), N, mz);
  lift_kernel<<<grid1(w.V * W, 256), 256, 0, s>>>(x, params + L.P, params + L.bP, at<bf16>(ws, w.hb[0]), w.V, W);
  if ((e = cudaGetLastError()) != cudaSuccess) return st(e);
  for (int l = 0; l < d->layers; ++l) {
    const bf16* h = at<bf16>(ws, w.hb[l]);
    // z transform: per line [W x N] (c, z) x [N x 2mz]
    Gemm g = gemm_base();
    g.M = W; g.N = 2 * mz; g.K = N; g.batch = (int)w.lines;
    g.A = h; g.a_rs = 1; g.a_cs = W; g.a_bs = (long long)N * W;
    g.B = at<bf16>(ws, w.fz); g.b_rs = 2 * mz; g.b_cs = 1; g.b_bs = 0;
    g.C = at<float>(ws, w.zgemm); g.c_rs = 2 * mz; g.c_cs = 1; g.c_bs = (long long)W * 2 * mz;
    if ((e = gemm(g, s)) != cudaSuccess) return st(e);
    float2* hz = at<float2>(ws, w.hz[l]);
    z_to_mode_major<<<grid1(w.lines * mz * W, 256), 256, 0, s>>>(at<float>(ws, w.zgemm), hz, w.lines, W, mz);
    // y then x transforms to the kept modes: [x][y][kz c] -> [x][ky][kz c] -> [kx][ky][kz c]
    float2* ca = at<float2>(ws, w.cplx_a);
    float2* hx = at<float2>(ws, w.hx[l]);
    axis_dft_kernel<<<grid1((long long)N * my * mz * W, 256), 256, 0, s>>>(hz, ca, N, N, my, mz * W, -1, 0, 1.f, 0);
    axis_dft_kernel<<<grid1((long long)mx * my * mz * W, 256), 256, 0, s>>>(ca, hx, 1, N, mx, my * mz * W, -1, 0, 1.f, 0);
    // mixing
    float2* cb = at<float2>(ws, w.cplx_b);
    mix_kernel<<<grid1((long long)mx * my * mz * W, 256), 256, 0, s>>>(hx, params + L.R[l], cb, mx * my * mz, W, 0);
    // inverse x then y (kept -> full), scaled later by the z inverse weights (1/N^3)
    axis_dft_kernel<<<grid1((long long)N * my * mz * W, 256), 256, 0, s>>>(cb, ca, 1, N, mx, my * mz * W, 1, 1, 1.f, 0);
    axis_dft_kernel<<<grid1((long long)N * N * mz * W, 256), 256, 0, s>>>(ca, cb, N, N, my, mz * W, 1, 1, 1.f, 0);
    bf16* ob = at<bf16>(ws, w.bfa);
    mode_to_gemm_bf16<<<grid1(w.lines * mz * W, 256), 256, 0, s>>>(cb, ob, w.lines, W, mz);
    if ((e = cudaGetLastError()) != cudaSuccess) return st(e);
    // spectral branch: s[(line, z)][o] = sum_(kz, r) gz[z][kz r] O[line][kz r][o]
    Gemm gi = gemm_base();
    gi.M = N; gi.N = W; gi.K = 2 * mz; gi.batch = (int)w.lines;
    gi.A = at<bf16>(ws, w.gz); gi.a_rs = 2 * mz; gi.a_cs = 1; gi.a_bs = 0;
    gi.B = ob; gi.b_rs = W; gi.b_cs = 1; gi.b_bs = 2LL * mz * W;
    gi.C = at<float>(ws, w.s); gi.c_rs = W; gi.c_cs = 1; gi.c_bs = (long long)N * W;
    if ((e = gemm(gi, s)) != cudaSuccess) return st(e);
    // t = s + h W_l + b_l;  h_{l+1} = GELU(t) (not after the last layer)
    Gemm gl = gemm_base();
    gl.M = (int)w.V; gl.N = W; gl.K = W;
    gl.A = h; gl.a_rs = W; gl.a_cs = 1;
    gl.B = pb + L.W[l]; gl.b_rs = W; gl.b_cs = 1;
    gl.C = at<float>(ws, w.t[l]); gl.c_rs = W; gl.c_cs = 1;
    gl.Cb = at<bf16>(ws, w.hb[l + 1]);
    gl.bias = params + L.b[l];
    gl.addend = at<float>(ws, w.s);
    gl.gelu = l < d->layers - 1;
    if ((e = gemm(gl, s)) != cudaSuccess) return st(e);
  }
  // projection
  Gemm g1 = gemm_base();
  g1.M = (int)w.V; g1.N = H; g1.K = W;
  g1.A = at<bf16>(ws, w.hb[d->layers]); g1.a_rs = W; g1.a_cs = 1;
  g1.B = pb + L.Q1; g1.b_rs = H; g1.b_cs = 1;
  g1.C = at<float>(ws, w.u); g1.c_rs = H; g1.c_cs = 1;
  g1.Cb = at<bf16>(ws, w.gb);
  g1.bias = params + L.bQ1;
  g1.gelu = 1;
  if ((e = gemm(g1, s)) != cudaSuccess) return st(e);
  Gemm g2 = gemm_base();
  g2.M = (int)w.V; g2.N = 8; g2.K = H;
  g2.A = at<bf16>(ws, w.gb); g2.a_rs = H; g2.a_cs = 1;
  g2.B = pb + L.Q2; g2.b_rs = 8; g2.b_cs = 1;
  g2.C = at<float>(ws, w.y); g2.c_rs = 8; g2.c_cs = 1;
  g2.bias = params + L.bQ2;
  if ((e = gemm(g2, s)) != cudaSuccess) return st(e);
  if (y) {
    e = cudaMemcpyAsync(y, at<float>(ws, w.y), w.V * 8 * 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return st(e);
  }
  return st(cudaGetLastError());
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
  const int ksplit_v = (int)std::min<long long>(64, (w.V + 4095) / 4096);
  Gemm g = gemm_base();
  g.M = H; g.N = 8; g.K = (int)w.V; g.ksplit = ksplit_v; g.accumulate = 1;
  g.A = at<bf16>(ws, w.gb); g.a_rs = 1; g.a_cs = H;
  g.B = dyb; g.b_rs = 8; g.b_cs = 1;
  g.C = grads + L.Q2; g.c_rs = 8; g.c_cs = 1;
  if ((e = gemm(g, s)) != cudaSuccess) return st(e);
  col_sum_kernel<<<152, 256, 0, s>>>(dy, grads + L.bQ2, w.V, 8);
  // dg = dy Q2^T ; du = dg * GELU'(u)
  float* dg = at<float>(ws, w.dh2);
  g = gemm_base();
  g.M = (int)w.V; g.N = H; g.K = 8;
  g.A = dyb; g.a_rs = 8; g.a_cs = 1;
  g.B = pb + L.Q2; g.b_rs = 1; g.b_cs = 8;
  g.C = dg; g.c_rs = H; g.c_cs = 1;
  if ((e = gemm(g, s)) != cudaSuccess) return st(e);
  bf16* dub = at<bf16>(ws, w.bfa);
  float* du = at<float>(ws, w.dh);
  gelu_back_kernel<<<grid1(w.V * H, 256), 256, 0, s>>>(dg, at<float>(ws, w.u), du, dub, w.V * H, 1);
  // dQ1 += h_L^T du, dbQ1 += sum du, dh_L = du Q1^T
  g = gemm_base();
  g.M = W; g.N = H; g.K = (int)w.V; g.ksplit = ksplit_v; g.accumulate = 1;
  g.A = at<bf16>(ws, w.hb[d->layers]); g.a_rs = 1; g.a_cs = W;
  g.B = dub; g.b_rs = H; g.b_cs = 1;
  g.C = grads + L.Q1; g.c_rs = H; g.c_cs = 1;
  if ((e = gemm(g, s)) != cudaSuccess) return st(e);
  col_sum_kernel<<<152, 256, 0, s>>>(du, grads + L.bQ1, w.V, H);
  float* dh = at<float>(ws, w.dh2);
  g = gemm_base();
  g.M = (int)w.V; g.N = W; g.K = H;
  g.A = dub; g.a_rs = H; g.a_cs = 1;
  g.B = pb + L.Q1; g.b_rs = 1; g.b_cs = H;
  g.C = dh; g.c_rs = W; g.c_cs = 1;
  if ((e = gemm(g, s)) != cudaSuccess) return st(e);
  for (int l = d->layers - 1; l >= 0; --l) {
    // dt = dh (* GELU'(t) if activated); dh is in ws.dh2, write dt to ws.dh / bf16 ws.bfa
    float* dt = at<float>(ws, w.dh);
    bf16* dtb = at<bf16>(ws, w.bfa);
    gelu_back_kernel<<<grid1(w.V * W, 256), 256, 0, s>>>(dh, at<float>(ws, w.t[l]), dt, dtb, w.V * W,
                                                         l < d->layers - 1);
    col_sum_kernel<<<152, 256, 0, s>>>(dt, grads + L.b[l], w.V, W);
    // dW_l += h_l^T dt
    g = gemm_base();
    g.M = W; g.N = W; g.K = (int)w.V; g.ksplit = ksplit_v; g.accumulate = 1;
    g.A = at<bf16>(ws, w.hb[l]); g.a_rs = 1; g.a_cs = W;
    g.B = dtb; g.b_rs = W; g.b_cs = 1;
    g.C = grads + L.W[l]; g.c_rs = W; g.c_cs = 1;
    if ((e = gemm(g, s)) != cudaSuccess) return st(e);
    // spectral branch adjoint: dO[line][kz r][o] = sum_z gz[z][kz r] dt[(line, z)][o]
    g = gemm_base();
    g.M = 2 * mz; g.N = W; g.K = N; g.batch = (int)w.lines;
    g.A = at<bf16>(ws, w.gz); g.a_rs = 1; g.a_cs = 2 * mz; g.a_bs = 0;
    g.B = dtb; g.b_rs = W; g.b_cs = 1; g.b_bs = (long long)N * W;
    g.C = at<float>(ws, w.zgemm); g.c_rs = W; g.c_cs = 1; g.c_bs = 2LL * mz * W;
    if ((e = gemm(g, s)) != cudaSuccess) return st(e);
    float2* ca = at<float2>(ws, w.cplx_a);
    float2* cb = at<float2>(ws, w.cplx_b);
    pairs_to_complex<<<grid1(w.lines * mz * W, 256), 256, 0, s>>>(at<float>(ws, w.zgemm), cb, w.lines, W, mz);
    // adjoints of the inverse y and x transforms (full -> kept, conjugate phase)
    axis_dft_kernel<<<grid1((long long)N * my * mz * W, 256), 256, 0, s>>>(cb, ca, N, N, my, mz * W, -1, 0, 1.f, 0);
    axis_dft_kernel<<<grid1((long long)mx * my * mz * W, 256), 256, 0, s>>>(ca, cb, 1, N, mx, my * mz * W, -1, 0, 1.f, 0);
    // mixing: dR += conj(H) dO, dH = dO conj(R)^T
    const float2* hx = at<float2>(ws, w.hx[l]);
    mix_grad_kernel<<<grid1((long long)mx * my * mz * W * W, 256), 256, 0, s>>>(hx, cb, grads + L.R[l], mx * my * mz, W);
    mix_kernel<<<grid1((long long)mx * my * mz * W, 256), 256, 0, s>>>(cb, params + L.R[l], ca, mx * my * mz, W, 1);
    // adjoints of the forward x and y transforms (kept -> full, conjugate phase)
    axis_dft_kernel<<<grid1((long long)N * my * mz * W, 256), 256, 0, s>>>(ca, cb, 1, N, mx, my * mz * W, 1, 1, 1.f, 0);
    axis_dft_kernel<<<grid1((long long)N * N * mz * W, 256), 256, 0, s>>>(cb, ca, N, N, my, mz * W, 1, 1, 1.f, 0);
    bf16* dzb = at<bf16>(ws, w.bfa);  // dt (bf16) is no longer needed after the next GEMM reads it
    // dh_l = dt W_l^T first (reads dtb), then the z-transform adjoint accumulates
    float* dhn = at<float>(ws, w.dh2);
    g = gemm_base();
    g.M = (int)w.V; g.N = W; g.K = W;
    g.A = dtb; g.a_rs = W; g.a_cs = 1;
    g.B = pb + L.W[l]; g.b_rs = 1; g.b_cs = W;
    g.C = dhn; g.c_rs = W; g.c_cs = 1;
    if ((e = gemm(g, s)) != cudaSuccess) return st(e);
    mode_to_zgrad_bf16<<<grid1(w.lines * mz * W, 256), 256, 0, s>>>(ca, dzb, w.lines, W, mz);
    // dh[(line, z)][c] += sum_(kz r) fz[z][kz r] dZ[line][c][kz r]
    g = gemm_base();
    g.M = N; g.N = W; g.K = 2 * mz; g.batch = (int)w.lines; g.accumulate = 1;
    g.A = at<bf16>(ws, w.fz); g.a_rs = 2 * mz; g.a_cs = 1; g.a_bs = 0;
    g.B = dzb; g.b_rs = 1; g.b_cs = 2 * mz; g.b_bs = (long long)W * 2 * mz;
    g.C = dhn; g.c_rs = W; g.c_cs = 1; g.c_bs = (long long)N * W;
    if ((e = gemm(g, s)) != cudaSuccess) return st(e);
    dh = dhn;
  }
  lift_grad_kernel<<<152, 256, 0, s>>>(x, dh, grads + L.P, grads + L.bP, w.V, W);
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
