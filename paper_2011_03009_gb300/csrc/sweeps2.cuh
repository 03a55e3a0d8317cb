// Two-level register FFT sweeps (compile-time line length L = A * B).
//
// A line x[n], n = B a + b (a < A, b < B), is transformed in two register steps with one
// shared-memory transpose between them (four-step decomposition):
//   step 1  thread (line, b):  Y_b[k1] = DFT_A over a of x[B a + b], times w_L^(b k1)
//   step 2  thread (line, k1): X[k1 + A k2] = DFT_B over b of Y_b[k1]
// The output is in natural frequency order.  The inverse runs the same two steps in
// reverse with conjugate twiddles (x L, the 1/(M_x M_y M_z) scale is applied by the
// last sweep).  Global memory is read and written directly from registers:
// - column sweeps (strided axis) map the 16 lines of a tile to the 16 lanes of a
//   half-warp, so every access is one 128-byte row segment;
// - line sweeps (contiguous axis) map b (or k1) to the lanes, so a warp reads and
//   writes consecutive elements of one line.
// The transpose buffer pads each line to an odd pitch so that the 16 lanes of a
// half-warp never share a bank.
#pragma once

#include "regfft.cuh"

namespace vp {

constexpr int kLines2 = 16;    // lines per CTA
constexpr int kThreads2 = 256;

__host__ __device__ constexpr int col2_pitch(int L) { return L + 1; }
// Transpose buffer of a column tile, element (column line, k1, b) of x[B k1' ...]:
// - 16 columns: line-major, pitch L + 1 (odd): the 16 lanes of a half-warp, one per
//   column, fall on distinct banks;
// - 8 columns: [k1][b][column] with rows of 8 (B + 1) elements: a half-warp holds 8
//   columns x 2 consecutive b (first step) or 8 columns x 2 consecutive k1 (second
//   step), and both read 16 distinct bank pairs (with the line-major odd pitch the
//   second pair of a half-warp landed on the first's banks).
__host__ __device__ constexpr size_t col2_smem_elems(int A, int B, int NL) {
  return NL == 8 ? (size_t)A * 8 * (B + 1) : (size_t)NL * col2_pitch(A * B);
}
template <int A, int B, int NL>
__device__ __forceinline__ int col2_at(int line, int k1, int b) {
  if constexpr (NL == 8) return k1 * (8 * (B + 1)) + b * 8 + line;
  else return line * col2_pitch(A * B) + k1 * B + b;
}
// Loads of the column sweeps.  A CTA reads one 64-byte (8 columns) or 128-byte (16
// columns) segment of each row of its columns, and the CTAs holding the neighbouring
// columns of the same rows are launched next to it.  VP_COL_PREFETCH = 128 or 256 adds
// the L2 prefetch-size hint, so that the first of them to miss fetches the whole aligned
// block (a block never crosses a page, so the hint cannot reach unmapped memory); 0 is a
// plain read-only load.
#ifndef VP_COL_PREFETCH
#define VP_COL_PREFETCH 256
#endif
__device__ __forceinline__ float2 ldg_col(const float2* q) {
#if VP_COL_PREFETCH == 256
  float2 v;
  asm("ld.global.nc.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(q));
  return v;
#elif VP_COL_PREFETCH == 128
  float2 v;
  asm("ld.global.nc.L2::128B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(q));
  return v;
#else
  return __ldg(q);
#endif
}
// Resident CTAs per SM the column kernels are compiled for: three while three tiles fit
// in shared memory (the register cap then is 85 per thread), else one.
__host__ __device__ constexpr int col2_min_blocks(int L, int dir) {
  // forward sweeps up to L = 384 fit four CTAs (64 registers) without spilling much and
  // are latency-bound, so the fourth CTA pays; their inverse variants spill there
  return (L <= 384 && dir == kForward) ? 4 : (L <= 512 ? 3 : 1);
}
// Rows a of x[B a + b] that can be nonzero on a zero-padded line (n <= L / 2).
__host__ __device__ constexpr int conv_rows_in(int A) { return (A + 1) / 2; }
__host__ __device__ constexpr int line2_bpitch(int B) { return B + 1; }
__host__ __device__ constexpr int line2_pitch(int A, int B) { return A * (B + 1) + 1; }

// One 16-column tile (tile index `tile` of p's n_outer x ceil(C/16) tiles).
// HALF: the forward input has rows_in <= L / 2 (zero-padded), or the inverse output has
// rows_out <= L / 2 (cropped), so only rows a < AH of x[B a + b] are read or written.
template <int A, int B, int DIR, bool SRC, bool HALF, int NL = kLines2>
__device__ __forceinline__ void col2_tile(const ColSweep& p, int tile, float2* S) {
  constexpr int AH = HALF ? conv_rows_in(A) : A;
  constexpr int LSH = NL == 16 ? 4 : (NL == 8 ? 3 : 2);
  const int ncb = (p.C + NL - 1) / NL;
  const int o = tile / ncb;
  const int c0 = (tile - o * ncb) * NL;
  const float2* __restrict__ tw = p.ax.tw;
  const float2 zero = make_float2(0.f, 0.f);

  if constexpr (DIR == kForward) {
    for (int tau = threadIdx.x; tau < NL * B; tau += blockDim.x) {
      const int line = tau & (NL - 1);
      const int b = tau >> LSH;
      const int c = c0 + line;
      const bool colok = c < p.C;
      const long long base = (long long)o * p.in_os + c;
      float2 v[A];
      if constexpr (SRC) {
        // f_n = C_n sum_{m=1}^{n-1} p_m p_{n-m} (Eq. 2.6), summed over pairs m <= n - m
#pragma unroll
        for (int a = 0; a < A; ++a) v[a] = zero;
        const int n = p.harmonic;
        for (int m = 1; 2 * m <= n; ++m) {
          const float2* __restrict__ pa = p.lower[m - 1];
          const float2* __restrict__ pb = p.lower[n - m - 1];
          const float w = ((2 * m == n) ? 1.f : 2.f) * p.cn;
#pragma unroll
          for (int a = 0; a < AH; ++a) {
            const int row = B * a + b;
            if (colok && row < p.rows_in) {
              const long long off = base + (long long)row * p.in_rs;
              const float2 x = ldg_col(&pa[off]), y = ldg_col(&pb[off]);
              const float2 xy = cmul(x, y);
              v[a].x = fmaf(w, xy.x, v[a].x);
              v[a].y = fmaf(w, xy.y, v[a].y);
            }
          }
        }
      } else {
#pragma unroll
        for (int a = 0; a < AH; ++a) {
          const int row = B * a + b;
          v[a] = (colok && row < p.rows_in)
                     ? ldg_col(&p.in[base + (long long)row * p.in_rs + (long long)(row / kRowGroup) * p.in_rs_extra])
                     : zero;
        }
      }
      dft_reg_nz<A, false, AH>(v);
      S[col2_at<A, B, NL>(line, 0, b)] = v[0];
#pragma unroll
      for (int k1 = 1; k1 < A; ++k1) S[col2_at<A, B, NL>(line, k1, b)] = cmul(v[k1], __ldg(&tw[b * k1]));
    }
    __syncthreads();
    for (int tau = threadIdx.x; tau < NL * A; tau += blockDim.x) {
      const int line = tau & (NL - 1);
      const int k1 = tau >> LSH;
      float2 z[B];
#pragma unroll
      for (int b = 0; b < B; ++b) z[b] = S[col2_at<A, B, NL>(line, k1, b)];
      dft_reg<B, false>(z);
      const int c = c0 + line;
      if (c < p.C) {
        const long long base = (long long)o * p.out_os + c;
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
          const int row = k1 + A * k2;
          if (row < p.rows_out) p.out[base + (long long)row * p.out_rs] = z[k2];
        }
      }
    }
  } else {
    for (int tau = threadIdx.x; tau < NL * A; tau += blockDim.x) {
      const int line = tau & (NL - 1);
      const int k1 = tau >> LSH;
      const int c = c0 + line;
      const bool colok = c < p.C;
      const long long base = (long long)o * p.in_os + c;
      float2 z[B];
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2)
        z[k2] = colok ? ldg_col(&p.in[base + (long long)(k1 + A * k2) * p.in_rs]) : zero;
      dft_reg<B, true>(z);
      S[col2_at<A, B, NL>(line, k1, 0)] = z[0];
#pragma unroll
      for (int b = 1; b < B; ++b) S[col2_at<A, B, NL>(line, k1, b)] = cmulc(z[b], __ldg(&tw[b * k1]));
    }
    __syncthreads();
    for (int tau = threadIdx.x; tau < NL * B; tau += blockDim.x) {
      const int line = tau & (NL - 1);
      const int b = tau >> LSH;
      float2 v[A];
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) v[k1] = S[col2_at<A, B, NL>(line, k1, b)];
      dft_reg<A, true>(v);
      const int c = c0 + line;
      if (c < p.C) {
        const long long base = (long long)o * p.out_os + c;
#pragma unroll
        for (int a = 0; a < AH; ++a) {
          const int row = B * a + b;
          if (row < p.rows_out) p.out[base + (long long)row * p.out_rs] = cscale(v[a], p.scale);
        }
      }
    }
  }
}

template <int A, int B, int DIR, bool SRC, bool HALF>
__global__ void __launch_bounds__(kThreads2, col2_min_blocks(A * B, DIR)) col2_kernel(const ColSweep p) {
  extern __shared__ __align__(16) float2 S[];
  col2_tile<A, B, DIR, SRC, HALF>(p, blockIdx.x, S);
}

// Long columns (L > 512): 8 columns per CTA, so that two CTAs share an SM; a quarter warp
// covers one 64-byte row segment.
// 8 max(A, B) threads (rounded to warps), so that each step's tasks take one round: 320
// at L = 1200 (30 x 40), whose first forward step has 320 tasks; 256 elsewhere.
__host__ __device__ constexpr int col8_threads(int A, int B) { return ((8 * (A > B ? A : B) + 31) / 32) * 32; }
template <int A, int B, int DIR, bool SRC, bool HALF>
__global__ void __launch_bounds__(col8_threads(A, B), 2) col2_kernel8(const ColSweep p) {
  extern __shared__ __align__(16) float2 S[];
  col2_tile<A, B, DIR, SRC, HALF, 8>(p, blockIdx.x, S);
}

// 16 columns a CTA at the long lengths (one CTA an SM), 512 threads: the inverse sweeps
// that write rows megabytes apart, whole 128-byte segments a row.
template <int A, int B, int DIR, bool SRC, bool HALF>
__global__ void __launch_bounds__(512, 1) col2_kernel16w(const ColSweep p) {
  extern __shared__ __align__(16) float2 S[];
  col2_tile<A, B, DIR, SRC, HALF>(p, blockIdx.x, S);
}

// The same, compiled for three CTAs an SM (80 registers, a few bytes of spills).  The
// column sweeps wait on memory, and a third CTA's loads pay where rows are close in
// memory; where each row of a column is megabytes from the next (the x sweeps of the
// larger grids) the third CTA measured slower.  Used up to L = 864.
template <int A, int B, int DIR, bool SRC, bool HALF>
__global__ void __launch_bounds__(kThreads2, 3) col2_kernel8x3(const ColSweep p) {
  extern __shared__ __align__(16) float2 S[];
  col2_tile<A, B, DIR, SRC, HALF, 8>(p, blockIdx.x, S);
}

// Batched form: the parameters of up to kMaxBatch plans travel in the kernel's own
// parameter block (constant bank), with offsets[i] the first CTA (or tile) of plan i;
// CTA b finds its plan by a binary search over the constant-bank offsets.
template <typename T>
__device__ __forceinline__ int batch_owner(const BatchParams<T>& bp, int b) {
  int lo = 0, hi = bp.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bp.offsets[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__device__ __forceinline__ void copy_params(T* dst, const T* src) {
  static_assert(sizeof(T) % 4 == 0, "parameter blocks are word-sized");
  const int* s = (const int*)src;
  int* d = (int*)dst;
  for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = __ldg(&s[i]);
}

template <int A, int B, int DIR, bool SRC, bool HALF>
__global__ void __launch_bounds__(kThreads2, col2_min_blocks(A * B, DIR))
    col2_batch_kernel(const __grid_constant__ BatchParams<ColSweep> bp) {
  extern __shared__ __align__(16) float2 S[];
  const int owner = batch_owner(bp, blockIdx.x);
  col2_tile<A, B, DIR, SRC, HALF>(bp.item[owner], blockIdx.x - bp.offsets[owner], S);
}

// One tile of 16 lines (conv: tile `tile` of the tile list; forward: lines 16 tile ..).
template <int A, int B, int MODE>
__device__ __forceinline__ void line2_tile(const LineSweep& p, long long tile, float2* S) {
  constexpr int L = A * B;
  constexpr int BP = line2_bpitch(B);
  constexpr int LP = line2_pitch(A, B);
  __shared__ long long line_of[kLines2];
  __shared__ int oct_of[4];
  const float2* __restrict__ tw = p.ax.tw;
  const float2 zero = make_float2(0.f, 0.f);

  if (threadIdx.x < kLines2) {
    long long l;
    if (MODE == kConv) {
      l = p.tiles[20LL * tile + threadIdx.x];
    } else {
      l = tile * kLines2 + threadIdx.x;
      if (l >= p.nlines) l = -1;
    }
    line_of[threadIdx.x] = l;
  }
  if (MODE == kConv && threadIdx.x < 4) oct_of[threadIdx.x] = p.tiles[20LL * tile + 16 + threadIdx.x];
  __syncthreads();

  // forward step 1: task (line, b), b fastest across lanes (coalesced along the line)
  for (int tau = threadIdx.x; tau < kLines2 * B; tau += blockDim.x) {
    const int line = tau / B;
    const int b = tau - line * B;
    const long long l = line_of[line];
    const float2* src = p.data + (l < 0 ? 0 : l * p.ld);
    float2 v[A];
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const int n = B * a + b;
      v[a] = (l >= 0 && n < p.n_in) ? __ldg(&src[n]) : zero;
    }
    dft_reg<A, false>(v);
    float2* s = S + line * LP + b;
    s[0] = v[0];
#pragma unroll
    for (int k1 = 1; k1 < A; ++k1) s[k1 * BP] = cmul(v[k1], __ldg(&tw[b * k1]));
  }
  __syncthreads();

  // forward step 2 (+ spectrum multiply and inverse step 2): task (line, k1)
  for (int tau = threadIdx.x; tau < kLines2 * A; tau += blockDim.x) {
    const int line = tau / A;
    const int k1 = tau - line * A;
    float2 z[B];
    float2* s = S + line * LP + k1 * BP;
#pragma unroll
    for (int b = 0; b < B; ++b) z[b] = s[b];
    dft_reg<B, false>(z);
    if constexpr (MODE == kConv) {
      const int oc = oct_of[line >> 2];
      if (oc >= 0) {
        const float2* __restrict__ kl = p.khat + (long long)oc * p.Oz;
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
          const int f = k1 + A * k2;
          z[k2] = cmul(z[k2], __ldg(&kl[min(f, L - f)]));
        }
      }
      dft_reg<B, true>(z);
      s[0] = z[0];
#pragma unroll
      for (int b = 1; b < B; ++b) s[b] = cmulc(z[b], __ldg(&tw[b * k1]));
    } else {
      const long long l = line_of[line];
      if (l >= 0) {
        float2* dst = p.data + l * p.ld;
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
          const int f = k1 + A * k2;
          if (f < p.n_out) dst[f] = z[k2];
        }
      }
    }
  }

  if constexpr (MODE == kConv) {
    __syncthreads();
    // inverse step 1: task (line, b)
    for (int tau = threadIdx.x; tau < kLines2 * B; tau += blockDim.x) {
      const int line = tau / B;
      const int b = tau - line * B;
      float2 v[A];
      const float2* s = S + line * LP + b;
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) v[k1] = s[k1 * BP];
      dft_reg<A, true>(v);
      const long long l = line_of[line];
      if (l >= 0) {
        float2* dst = p.data + l * p.ld;
#pragma unroll
        for (int a = 0; a < A; ++a) {
          const int n = B * a + b;
          if (n < p.n_out) dst[n] = v[a];
        }
      }
    }
  }
}

template <int A, int B, int MODE>
__global__ void __launch_bounds__(kThreads2) line2_kernel(const LineSweep p) {
  extern __shared__ __align__(16) float2 S[];
  line2_tile<A, B, MODE>(p, blockIdx.x, S);
}

template <int A, int B>
__global__ void __launch_bounds__(kThreads2) line2_batch_kernel(const __grid_constant__ BatchParams<LineSweep> bp) {
  extern __shared__ __align__(16) float2 S[];
  const int owner = batch_owner(bp, blockIdx.x);
  line2_tile<A, B, kConv>(bp.item[owner], blockIdx.x - bp.offsets[owner], S);
}

// Persistent, software-pipelined form of line2_kernel<kConv>: each CTA walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  The 16 input lines of the next tile are
// copied into a staging buffer with cp.async while the current tile runs its forward
// step 2, spectrum multiply and inverse step 2; the next tile's four octant lines of
// the spectrum are copied while the current tile runs its inverse step 1.  The
// twiddle table is staged once.  The compute phases then touch only registers and
// shared memory.  Each tile's host record is read into registers before the tile ahead
// of it runs its forward step 1, so its latency is hidden there.
// Shared memory: transpose buffer (16 x line2_pitch), staging buffer (16 x ni),
// spectrum lines (4 x Oz), twiddles (A x conv_tw_pitch(B)).
// NL = 8 or 4 (long lines): a CTA takes half or a quarter of a tile of the host's list
// (2 or 1 mirror groups of 4 lines and their octant lines), so the buffers fit in shared
// memory at L >= 1024, or more CTAs share an SM.  NT threads a CTA (NT / 32 warps): the
// 4-line form runs NL x max(A, B) threads, one task of each step per thread.
// The staging pitch that holds rows a < conv_rows_in(A) of a line (odd: lanes = lines).
// Pitches (in float2 elements) of the pipelined z sweep's buffers.  With 16 or 8 lines a
// tile, the 16 lanes of a half-warp access the same element of 16 (or 8) lines, so an odd
// pitch keeps them on distinct banks.  With 4 lines a half-warp touches 4 consecutive
// elements of each of the 4 lines (or 4 twiddle rows): a pitch of 4 (mod 16) puts the
// lines 8 banks apart, conflict-free.
__host__ __device__ constexpr int pitch_mod(int v, int m, int r) { return v + (((r - v % m) % m) + m) % m; }
__host__ __device__ constexpr int conv_line_pitch(int A, int B, int NL) {
  return NL == 4 ? pitch_mod(A * (B + 1), 16, 4) : line2_pitch(A, B);
}
__host__ __device__ constexpr int conv_stage_pitch(int A, int B, int NL = kLines2) {
  return NL == 4 ? pitch_mod(B * conv_rows_in(A), 16, 4) : (B * conv_rows_in(A)) | 1;
}
// Row pitch of the z sweep's twiddle table: 8 elements past B, so that rows k1 and k1 + 1
// start 16 banks apart.
__host__ __device__ constexpr int conv_tw_pitch(int B, int NL = kLines2) { return NL == 4 ? pitch_mod(B, 16, 4) : B + 8; }
// TWG: the inter-step twiddles are read from the plan's table in global memory (through
// L1) instead of a shared-memory copy, which frees A x conv_tw_pitch elements a CTA.
__host__ __device__ constexpr size_t conv_pipe_smem(int A, int B, int Oz, int NL = kLines2, bool TWG = false,
                                                    bool BULK = false) {
  return ((size_t)NL * conv_line_pitch(A, B, NL) + (size_t)NL * conv_stage_pitch(A, B, NL) +
          (size_t)(NL / 4) * (Oz + (BULK ? 2 : 0)) +
          (TWG ? 0 : (size_t)A * conv_tw_pitch(B, NL))) *
         sizeof(float2);
}

// p is a __grid_constant__ parameter, so &p is one address valid in every thread.
// BATCH = false: the tiles of plan p.  BATCH = true: the tiles of every plan of a group,
// numbered consecutively (plan i owns [offsets[i], offsets[i + 1])), all with the same
// line length L and spectrum octant length; ni is the staging pitch for the longest
// input line.
// BULK (single plan, 4-line tiles, lines and spectrum 16-byte aligned): each line and the
// octant line are staged by one bulk asynchronous copy each (cp.async.bulk, issued by
// one thread, completion counted in bytes on an mbarrier) instead of 8-byte cp.async
// per element; the waits on those mbarriers are bounded (kWaitCycles), and a CTA whose
// wait expires records it in *p.status and returns.
template <int A, int B, bool BATCH, int NL = kLines2, int NT = kThreads2, bool TWG = false, bool BULK = false>
__global__ void __launch_bounds__(NT)
    line2_conv_pipe_kernel(const __grid_constant__ LineSweep p, const __grid_constant__ BatchParams<LineSweep> bp,
                           long long ntiles, int NI) {
  constexpr int L = A * B;
  constexpr int BP = line2_bpitch(B);
  constexpr int LP = conv_line_pitch(A, B, NL);
  constexpr int AH = conv_rows_in(A);
  constexpr int TP = conv_tw_pitch(B, NL);
  static_assert(B % 2 == 0, "the spectrum fold takes an even B");
  extern __shared__ __align__(16) float2 S[];
  const int Oz = p.Oz;  // shared by every plan of a batch group
  constexpr int NG = NL / 4;       // mirror groups per CTA tile
  constexpr int LSH = NL == 16 ? 4 : (NL == 8 ? 3 : 2);
  constexpr int NW = NT / 32;      // warps
  constexpr int SUB = 16 / NL;     // CTA tiles per tile of the host's list
  // line staging: with at least NL warps, WPL warps share a line; with fewer, a warp
  // stages LPW lines
  constexpr int WPL = NW >= NL ? NW / NL : 1;
  constexpr int LPW = NW >= NL ? 1 : NL / NW;
  constexpr int STAGERS = NW >= NL ? NL * WPL : NW;
  static_assert(!BULK || (!BATCH && NL == 4), "bulk staging: one plan, 4-line tiles");
  float2* I = S + NL * LP;
  float2* K = I + NL * NI;  // [NG][Oz]; with BULK one row of Oz + 2, element i at K[i + (oc Oz mod 2)]
  float2* T = K + NG * (Oz + (BULK ? 2 : 0));  // twiddles
  __shared__ long long line_of[2][NL];
  __shared__ __align__(8) unsigned long long bars[2];  // BULK: lines, spectrum
  const unsigned bar_lines = smem_addr(&bars[0]), bar_spec = smem_addr(&bars[1]);
  __shared__ int oct_of[2][NG];
  __shared__ const LineSweep* plan_of[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // The 20-int host record of a tile, read into registers one phase before it is used,
  // so that the load latency hides behind the previous tile's forward step 1.
  struct Rec {
    const LineSweep* q;       // plan of the tile
    long long line[LPW];      // the lines this warp stages
    long long my_line;        // line slot threadIdx.x (< NL)
    int my_oct;               // octant id slot threadIdx.x (< NG)
    int spec_oct;             // the octant line this warp stages: g = warp % NG
  };
  auto read_rec = [&](long long t) {
    Rec r;
    long long lt = t;
    r.q = &p;
    if constexpr (BATCH) {
      const int i = batch_owner(bp, (int)t);
      lt = t - bp.offsets[i];
      r.q = &bp.item[i];
    }
    const int* tiles = BATCH ? r.q->tiles : p.tiles;
    // line slots and octant ids of local tile lt in the host's 20-int tile records
    const long long lb = 20LL * (lt / SUB) + NL * (lt % SUB);
    const long long ob = 20LL * (lt / SUB) + 16 + NG * (lt % SUB);
#pragma unroll
    for (int h = 0; h < LPW; ++h) r.line[h] = tiles[lb + (NW >= NL ? warp % NL : warp + NW * h)];
    r.my_line = threadIdx.x < NL ? tiles[lb + threadIdx.x] : -1;
    r.my_oct = threadIdx.x < NG ? tiles[ob + threadIdx.x] : -1;
    r.spec_oct = tiles[ob + warp % NG];
    return r;
  };
  auto fetch_lines = [&](const Rec& r, int slot, bool skip) {
    const LineSweep& q = BATCH ? *r.q : p;
    const float2* data = q.data;
    const long long ld = q.ld;
    const int n_in = q.n_in;
    if constexpr (BULK) {
      // thread h < 4 stages line slot h: one arrival each, announcing its bytes; a
      // padding slot (-1) arrives with none and keeps stale data, whose output is
      // never stored
      if (threadIdx.x < NL && !skip) {
        const long long l = r.my_line;
        const unsigned bytes = l >= 0 ? 8u * (unsigned)n_in : 0u;
        mbar_arrive_expect(bar_lines, bytes);
        if (l >= 0) bulk_g2s(smem_addr(&I[threadIdx.x * NI]), data + l * ld, bytes, bar_lines);
      }
    } else if (warp < STAGERS) {
#pragma unroll
      for (int h = 0; h < LPW; ++h) {
        const int b = NW >= NL ? warp % NL : warp + NW * h;
        const long long l = r.line[h];
        const float2* src = data + (l < 0 ? 0 : l * ld);
        for (int n = (NW >= NL ? (warp / NL) * 32 : 0) + lane; n < NI; n += 32 * WPL)
          cp_async8(&I[b * NI + n], &src[n < n_in ? n : 0], l >= 0 && n < n_in);
      }
    }
    if (threadIdx.x < NL) line_of[slot][threadIdx.x] = r.my_line;
    if (threadIdx.x < NG) oct_of[slot][threadIdx.x] = r.my_oct;
    if (threadIdx.x == 0) plan_of[slot] = r.q;
  };
  auto fetch_spectrum = [&](const Rec& r, bool skip) {
    const float2* khat = BATCH ? r.q->khat : p.khat;
    const int g = warp % NG;
    const int oc = r.spec_oct;
    const float2* kl = khat + (oc < 0 ? 0 : (long long)oc * Oz);
    if constexpr (BULK) {
      // element i of the octant line goes to K[s0 + i], s0 = (oc Oz) mod 2, so that the
      // bulk run [s0, s0 + cnt) starts 16-byte aligned on both sides; the one element
      // left over when Oz is odd travels by cp.async
      if (threadIdx.x == 0 && !skip) {
        const int s0 = oc < 0 ? 0 : (int)(((long long)oc * Oz) & 1);
        const int cnt = (Oz - s0) & ~1;
        mbar_arrive_expect(bar_spec, oc < 0 ? 0u : 8u * (unsigned)cnt);
        if (oc >= 0) {
          bulk_g2s(smem_addr(&K[2 * s0]), kl + s0, 8u * (unsigned)cnt, bar_spec);
          if (s0 == 1) cp_async8(&K[1], kl, true);
          if (s0 + cnt < Oz) cp_async8(&K[s0 + Oz - 1], kl + Oz - 1, true);
        }
      }
    } else {
      for (int i = (warp / NG) * 32 + lane; i < Oz; i += (NW / NG) * 32)
        cp_async8(&K[g * Oz + i], &kl[i], oc >= 0);
    }
  };
  static_assert((NL == 4 || NL == 8 || NL == 16) && NT % 32 == 0 && NW % NG == 0 && (NW >= NL || NL % NW == 0),
                "tiles of 4, 8 or 16 lines; whole warps per mirror group and per staged line");

  if constexpr (BULK) {
    // the launcher takes this form only for aligned buffers; a violation is recorded
    // (bit 1) and the CTA returns before any copy is issued
    if (((smem_addr(I) | smem_addr(K)) & 15) != 0 || (((uintptr_t)p.data | (uintptr_t)p.khat) & 15) != 0 ||
        ((p.ld | p.n_in) & 1) != 0) {
      if (threadIdx.x == 0 && p.status != nullptr) atomicOr(p.status, 2);
      return;
    }
  }
  // inter-step twiddles laid out as T[k1 TP + b] = w_L^(b k1), TP = B + 8: with either
  // index fixed at compile time, every read is a register base plus a constant offset,
  // and the two k1 rows a warp reads in step 2 fall on different banks
  if constexpr (!TWG) {
    for (int i = threadIdx.x; i < A * TP; i += blockDim.x) {
      const int k1 = i / TP, b = i - k1 * TP;
      cp_async8(&T[i], &p.ax.tw[b < B ? b * k1 : 0], true);
    }
  }
  const float2* __restrict__ twg = p.ax.tw;
  if constexpr (BULK) {
    // rows a < AH of a staged line hold elements [0, B AH); the bulk copies write
    // [0, n_in), so the zeros of [n_in, B AH) are written once here
    const int nz = B * AH - p.n_in;
    if (nz > 0)
      for (int i = threadIdx.x; i < NL * nz; i += blockDim.x) I[(i / nz) * NI + p.n_in + i % nz] = make_float2(0.f, 0.f);
    if (threadIdx.x == 0) {
      mbar_init(bar_lines, NL);
      mbar_init(bar_spec, 1);
      mbar_init_fence();
    }
    __syncthreads();
  }
  long long t = blockIdx.x;
  if (t < ntiles) {
    const Rec r0 = read_rec(t);
    // test hook: the first copies are never issued, so the first wait expires
    fetch_lines(r0, 0, BULK && p.expire_waits);
    fetch_spectrum(r0, BULK && p.expire_waits);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int cur = it & 1;
    const long long tn = t + gridDim.x;
    // (the batched form reads the record where it is used: holding it over step 2
    // would cost it its second CTA per SM)
    Rec nrec{};
    if (!BATCH && tn < ntiles) nrec = read_rec(tn);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if constexpr (BULK) {
      // both mbarriers complete one phase per tile
      const bool ok = mbar_wait2(bar_lines, bar_spec, (unsigned)(it & 1), kWaitCycles);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0 && p.status != nullptr) atomicOr(p.status, 1);
        // copies still in flight land before the CTA's shared memory is given up
        mbar_wait2(bar_lines, bar_spec, (unsigned)(it & 1), kWaitCycles);
        return;
      }
    } else {
      __syncthreads();
    }
    const LineSweep& q = BATCH ? *plan_of[cur] : p;
    const int n_out = q.n_out;
    float2* const data = q.data;
    const long long ld = q.ld;
    // forward step 1 from the staging buffer; the 16 lanes of a half-warp hold the 16
    // lines (odd staging pitch), so every twiddle read is a broadcast.  The line is
    // zero from n_in <= L / 2 on: only rows a < AH are read (the staging buffer holds
    // zeros from n_in to B AH), and the DFT skips the rest.
    for (int tau = threadIdx.x; tau < NL * B; tau += blockDim.x) {
      const int line = tau & (NL - 1);
      const int b = tau >> LSH;
      const float2* src = I + line * NI;
      float2 v[A];
#pragma unroll
      for (int a = 0; a < AH; ++a) v[a] = src[B * a + b];
      dft_reg_nz<A, false, AH>(v);
      float2* s = S + line * LP + b;
      const float2* tw = T + b;
      s[0] = v[0];
#pragma unroll
      for (int k1 = 1; k1 < A; ++k1) s[k1 * BP] = cmul(v[k1], TWG ? __ldg(&twg[b * k1]) : tw[k1 * TP]);
    }
    __syncthreads();
    if (BATCH && tn < ntiles) nrec = read_rec(tn);
    if (tn < ntiles) fetch_lines(nrec, cur ^ 1, false);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    // forward step 2, spectrum multiply, inverse step 2 (lanes = lines again)
    for (int tau = threadIdx.x; tau < NL * A; tau += blockDim.x) {
      const int line = tau & (NL - 1);
      const int k1 = tau >> LSH;
      float2 z[B];
      float2* s = S + line * LP + k1 * BP;
#pragma unroll
      for (int b = 0; b < B; ++b) z[b] = s[b];
      dft_reg<B, false>(z);
      const int oc = oct_of[cur][line >> 2];
      if (oc >= 0) {
        // frequency f = k1 + A k2 folds to min(f, L - f): f itself below k2 = B / 2,
        // L - f from there on (B is even), so both reads take constant offsets
        const int kb = BULK ? (int)(((long long)oc * Oz) & 1) : (line >> 2) * Oz;
        const float2* lo = K + kb + k1;
        const float2* hi = K + kb + (L - k1);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) z[k2] = cmul(z[k2], 2 * k2 < B ? lo[A * k2] : hi[-A * k2]);
      }
      dft_reg<B, true>(z);
      const float2* tw = T + k1 * TP;
      s[0] = z[0];
#pragma unroll
      for (int b = 1; b < B; ++b) s[b] = cmulc(z[b], TWG ? __ldg(&twg[b * k1]) : tw[b]);
    }
    __syncthreads();
    if (BATCH && tn < ntiles) nrec = read_rec(tn);
    if (tn < ntiles) fetch_spectrum(nrec, false);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    // inverse step 1 and store
    for (int tau = threadIdx.x; tau < NL * B; tau += blockDim.x) {
      const int line = tau / B;
      const int b = tau - line * B;
      float2 v[A];
      const float2* s = S + line * LP + b;
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) v[k1] = s[k1 * BP];
      dft_reg<A, true>(v);  // rows a >= AH lie past n_out <= L / 2: never stored, not computed
      const long long l = line_of[cur][line];
      if (l >= 0) {
        float2* dst = data + l * ld;
#pragma unroll
        for (int a = 0; a < AH; ++a) {
          const int n = B * a + b;
          if (n < n_out) dst[n] = v[a];
        }
      }
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

}  // namespace vp
