// Pair-split z sweep for the longest compiled line (L = 1280 = 32 x 40).
#pragma once

#include "sweeps2.cuh"

namespace vp {

// Pair-split form for long lines on half tiles (8 lines, 2 mirror groups), 512 threads:
// step 2 gives each (line, k1) task to a lane pair, which splits the length-B DFT by one
// radix-2 stage so that each lane holds B/2 values.  Forward (decimation in frequency),
// lane h of the pair forms u_j = (z_j + (-1)^h z_{j+B/2}) w_B^(h j), j < B/2, from the
// shared-memory row and transforms it, giving X[2k + h]; after the spectrum multiply the
// inverse runs the mirror steps (decimation in time) and the pair combines its halves
// with one exchange of B/2 values.  At L = 1280 the 8-line tile holds one CTA per SM;
// half the registers a thread let it run 16 warps there instead of 8.
// Shared memory: as line2_conv_pipe_kernel with NL = 8, plus the pair twiddles w_B^(h j).
constexpr int kThreadsPair = 512;
__host__ __device__ constexpr size_t conv_pair8_smem(int A, int B, int Oz) {
  return conv_pipe_smem(A, B, Oz, 8) + (size_t)B * sizeof(float2);
}

template <int A, int B>
__global__ void __launch_bounds__(kThreadsPair)
    line2_conv_pair8_kernel(const __grid_constant__ LineSweep p, long long ntiles, int NI) {
  constexpr int NL = 8;
  constexpr int L = A * B;
  constexpr int H = B / 2;
  constexpr int BP = line2_bpitch(B);
  constexpr int LP = line2_pitch(A, B);
  constexpr int AH = conv_rows_in(A);
  constexpr int TP = conv_tw_pitch(B);
  constexpr int NW = kThreadsPair / 32;
  constexpr int NG = NL / 4;
  static_assert(H % 2 == 0, "the spectrum fold splits the half-length DFT at H / 2");
  static_assert(2 * NL * A == kThreadsPair, "one step-2 task per lane pair");
  static_assert(NL * B <= kThreadsPair, "one step-1 task per thread at most");
  extern __shared__ __align__(16) float2 S[];
  const int Oz = p.Oz;
  float2* I = S + NL * LP;
  float2* K = I + NL * NI;   // [NG][Oz]
  float2* T = K + NG * Oz;   // [A][TP]: w_L^(b k1)
  float2* W2 = T + A * TP;   // [2][H]: w_B^(h j)
  __shared__ long long line_of[2][NL];
  __shared__ int oct_of[2][NG];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  struct Rec {
    long long line;      // the line this warp stages (line warp % NL, half warp / NL of it)
    long long my_line;   // line slot threadIdx.x (< NL)
    int my_oct;          // octant id slot threadIdx.x (< NG)
    int spec_oct;        // the octant line this warp stages: g = warp % NG
  };
  // half tile lt: lines 8 (lt & 1) .. of host tile lt >> 1, octant ids 2 (lt & 1) ..
  auto read_rec = [&](long long lt) {
    Rec r;
    const long long lb = 20LL * (lt >> 1) + 8 * (lt & 1), ob = 20LL * (lt >> 1) + 16 + 2 * (lt & 1);
    r.line = p.tiles[lb + (warp % NL)];
    r.my_line = threadIdx.x < NL ? p.tiles[lb + threadIdx.x] : -1;
    r.my_oct = threadIdx.x < NG ? p.tiles[ob + threadIdx.x] : -1;
    r.spec_oct = p.tiles[ob + warp % NG];
    return r;
  };
  auto fetch_lines = [&](const Rec& r, int slot) {
    const int b = warp % NL;
    const long long l = r.line;
    const float2* src = p.data + (l < 0 ? 0 : l * p.ld);
    for (int n = (warp / NL) * 32 + lane; n < NI; n += (NW / NL) * 32)
      cp_async8(&I[b * NI + n], &src[n < p.n_in ? n : 0], l >= 0 && n < p.n_in);
    if (threadIdx.x < NL) line_of[slot][threadIdx.x] = r.my_line;
    if (threadIdx.x < NG) oct_of[slot][threadIdx.x] = r.my_oct;
  };
  auto fetch_spectrum = [&](const Rec& r) {
    const int g = warp % NG;
    const int oc = r.spec_oct;
    const float2* kl = p.khat + (oc < 0 ? 0 : (long long)oc * Oz);
    for (int i = (warp / NG) * 32 + lane; i < Oz; i += (NW / NG) * 32) cp_async8(&K[g * Oz + i], &kl[i], oc >= 0);
  };

  for (int i = threadIdx.x; i < A * TP; i += blockDim.x) {
    const int k1 = i / TP, b = i - k1 * TP;
    cp_async8(&T[i], &p.ax.tw[b < B ? b * k1 : 0], true);
  }
  // w_B^(h j) = w_L^(A h j)
  for (int i = threadIdx.x; i < B; i += blockDim.x) cp_async8(&W2[i], &p.ax.tw[A * (i / H) * (i % H)], true);
  long long t = blockIdx.x;
  if (t < ntiles) {
    const Rec r0 = read_rec(t);
    fetch_lines(r0, 0);
    fetch_spectrum(r0);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int cur = it & 1;
    const long long tn = t + gridDim.x;
    Rec nrec{};
    if (tn < ntiles) nrec = read_rec(tn);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    // forward step 1 (at most one task per thread): lanes of a quarter warp = the 8 lines
    if (threadIdx.x < NL * B) {
      const int line = threadIdx.x & (NL - 1);
      const int b = threadIdx.x >> 3;
      const float2* src = I + line * NI;
      float2 v[A];
#pragma unroll
      for (int a = 0; a < AH; ++a) v[a] = src[B * a + b];
      dft_reg_nz<A, false, AH>(v);
      float2* sp = S + line * LP + b;
      const float2* tw = T + b;
      sp[0] = v[0];
#pragma unroll
      for (int k1 = 1; k1 < A; ++k1) sp[k1 * BP] = cmul(v[k1], tw[k1 * TP]);
    }
    __syncthreads();
    if (tn < ntiles) fetch_lines(nrec, cur ^ 1);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    // step 2: lane pair (h = lane parity) per (line, k1)
    {
      const int h = threadIdx.x & 1;
      const int line = (threadIdx.x >> 1) & (NL - 1);
      const int k1 = threadIdx.x >> 4;
      const float sg = h ? -1.f : 1.f;
      float2* sp = S + line * LP + k1 * BP;
      const float2* w2 = W2 + h * H;
      float2 u[H];
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const float2 a = sp[j], c = sp[j + H];
        u[j] = cmul(make_float2(fmaf(sg, c.x, a.x), fmaf(sg, c.y, a.y)), w2[j]);
      }
      dft_reg<H, false>(u);  // u[k] = X[2k + h]
      if (oct_of[cur][line >> 2] >= 0) {
        // f = k1 + A (2k + h) folds to min(f, L - f): f below k = H/2, L - f from there on
        const float2* lo = K + (line >> 2) * Oz + k1 + A * h;
        const float2* hi = K + (line >> 2) * Oz + (L - k1 - A * h);
#pragma unroll
        for (int k = 0; k < H; ++k) u[k] = cmul(u[k], 2 * k < H ? lo[2 * A * k] : hi[-2 * A * k]);
      }
      dft_reg<H, true>(u);  // V_h[j]
      const float2* tw = T + k1 * TP + h * H;
      float2* so = sp + h * H;
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const float2 mine = cmulc(u[j], w2[j]);  // V_h[j] w_B^(-h j)
        const float ox = __shfl_xor_sync(0xffffffffu, mine.x, 1);
        const float oy = __shfl_xor_sync(0xffffffffu, mine.y, 1);
        // lane 0: x_j = V_0 + w^-j V_1; lane 1: x_{j+H} = V_0 - w^-j V_1
        const float2 x = make_float2(fmaf(sg, mine.x, ox), fmaf(sg, mine.y, oy));
        so[j] = cmulc(x, tw[j]);
      }
    }
    __syncthreads();
    if (tn < ntiles) fetch_spectrum(nrec);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    // inverse step 1 and store (at most one task per thread): lanes along b
    if (threadIdx.x < NL * B) {
      const int line = threadIdx.x / B;
      const int b = threadIdx.x - line * B;
      float2 v[A];
      const float2* sp = S + line * LP + b;
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) v[k1] = sp[k1 * BP];
      dft_reg<A, true>(v);
      const long long l = line_of[cur][line];
      if (l >= 0) {
        float2* dst = p.data + l * p.ld;
#pragma unroll
        for (int a = 0; a < AH; ++a) {
          const int n = B * a + b;
          if (n < p.n_out) dst[n] = v[a];
        }
      }
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

}  // namespace vp
