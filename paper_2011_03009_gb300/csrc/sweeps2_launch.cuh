// Launchers of the two-level sweep kernels for the sizes of one part of kFastSizes.
// Included by vp_sweeps2_part{0,1,2}.cu with VP_PART defined.
#pragma once

#include "sweeps2.cuh"
#include "sweeps2_pair.cuh"

namespace vp {
namespace {

template <typename K>
cudaError_t grant_smem(K kernel, size_t bytes, volatile int* granted) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (bytes <= 48 * 1024 || granted[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) granted[dev] = 1;
  return e;
}

template <int A, int B, int DIR, bool SRC, bool HALF>
cudaError_t col2_launch(const ColSweep& p, cudaStream_t s) {
  static volatile int granted[64] = {0};
  if constexpr (A * B > 512) {
    // one 16-column CTA per SM at these lengths: 8-column CTAs, two per SM, instead
    static volatile int granted8[64] = {0};
    const size_t smem = col2_smem_elems(A, B, 8) * sizeof(float2);
    const long long blocks = (long long)((p.C + 7) / 8) * p.n_outer;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if constexpr (A * B <= 864) {
      // three CTAs an SM where the rows a sweep writes (forward) or reads and writes
      // (inverse) lie within 1 MB of each other (measured at L = 640-864: y sweeps 5-20 %
      // faster; x inverse sweeps of 384^3-432^3 grids slower; x forward sweeps into the
      // grouped layout, whose far-apart rows are only read, 0.33 -> 0.28 ms at L = 768
      // and 0.50 -> 0.43 ms at L = 864)
      static volatile int granted83[64] = {0};
      const long long stride =
          (DIR == kForward ? p.out_rs : (p.in_rs > p.out_rs ? p.in_rs : p.out_rs)) * (long long)sizeof(float2);
      if (stride < (1LL << 20)) {
        auto k3 = col2_kernel8x3<A, B, DIR, SRC, HALF>;
        cudaError_t e = grant_smem(k3, smem, granted83);
        if (e != cudaSuccess) return e;
        k3<<<(unsigned)blocks, kThreads2, smem, s>>>(p);
        return cudaGetLastError();
      }
    }
    if constexpr (DIR == kInverse) {
      // an inverse sweep whose output rows lie 1 MB apart or more (the x inverse into
      // the caller's x-major field from 384^3 up) writes whole 128-byte row segments
      // from 16-column CTAs: with 64-byte segments from two CTAs the writes ran at half
      // the rate (x inverse at L = 1200: 1.31 against 1.74 ms; at L = 1024 0.69 against
      // 0.99 ms; at L = 768 0.33 against 0.38 ms).  The y inverse (rows N_z apart) keeps
      // 8 columns: 16 measured slower at L = 1200 (2.63 against 2.44 ms)
      if (p.out_rs * (long long)sizeof(float2) >= (1LL << 20)) {
        const size_t smem16 = (size_t)kLines2 * col2_pitch(A * B) * sizeof(float2);
        const long long b16 = (long long)((p.C + kLines2 - 1) / kLines2) * p.n_outer;
        // 512 threads: each step's 16 A or 16 B tasks in one or two rounds (at 256
        // threads, 1.52 against 1.31 ms at L = 1200)
        static volatile int granted16w[64] = {0};
        auto k16w = col2_kernel16w<A, B, DIR, SRC, HALF>;
        cudaError_t e = grant_smem(k16w, smem16, granted16w);
        if (e != cudaSuccess) return e;
        k16w<<<(unsigned)b16, 512, smem16, s>>>(p);
        return cudaGetLastError();
      }
    }
    auto k = col2_kernel8<A, B, DIR, SRC, HALF>;
    cudaError_t e = grant_smem(k, smem, granted8);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)blocks, col8_threads(A, B), smem, s>>>(p);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)kLines2 * col2_pitch(A * B) * sizeof(float2);
  const long long ncb = (p.C + kLines2 - 1) / kLines2;
  const long long blocks = ncb * p.n_outer;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  auto k = col2_kernel<A, B, DIR, SRC, HALF>;
  cudaError_t e = grant_smem(k, smem, granted);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)blocks, kThreads2, smem, s>>>(p);
  return cudaGetLastError();
}

template <int A, int B, int MODE>
cudaError_t line2_launch(const LineSweep& p, cudaStream_t s) {
  static volatile int granted[64] = {0};
  const size_t smem = (size_t)kLines2 * line2_pitch(A, B) * sizeof(float2);
  const long long blocks = MODE == kConv ? p.nlines : (p.nlines + kLines2 - 1) / kLines2;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  auto k = line2_kernel<A, B, MODE>;
  cudaError_t e = grant_smem(k, smem, granted);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)blocks, kThreads2, smem, s>>>(p);
  return cudaGetLastError();
}

// Whether a column sweep reads (forward) or writes (inverse) only the first half of its
// columns: true for every sweep of the zero-padded convolution, false for the kernel
// spectrum, whose lattice fills the whole embedding.
inline bool col2_half(const ColSweep& p, int L, int dir) {
  return dir == kForward ? 2 * p.rows_in <= L : 2 * p.rows_out <= L;
}

template <int A, int B>
cudaError_t col2_dispatch_forward(const ColSweep& p, bool src, cudaStream_t s) {
  const bool half = col2_half(p, A * B, kForward);
  if (src) {
    // the source's grid is the embedded one: N <= M / 2 for every even M >= 2 N - 1
    if (!half) return cudaErrorInvalidValue;
    return col2_launch<A, B, kForward, true, true>(p, s);
  }
  return half ? col2_launch<A, B, kForward, false, true>(p, s) : col2_launch<A, B, kForward, false, false>(p, s);
}

template <int A, int B>
cudaError_t col2_dispatch_inverse(const ColSweep& p, cudaStream_t s) {
  return col2_half(p, A * B, kInverse) ? col2_launch<A, B, kInverse, false, true>(p, s)
                                       : col2_launch<A, B, kInverse, false, false>(p, s);
}

template <int A, int B>
cudaError_t col2_dispatch(const ColSweep& p, int dir, bool src, cudaStream_t s) {
  return dir == kForward ? col2_dispatch_forward<A, B>(p, src, s) : col2_dispatch_inverse<A, B>(p, s);
}

// Persistent pipelined convolution sweep: one CTA per resident slot, tiles strided.
// Resident CTAs per SM for a given shared-memory size, cached per (device, size).
template <typename K>
cudaError_t resident_slots(K kernel, size_t smem, volatile int* granted, int* grid_out, int threads = kThreads2) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!granted[dev]) {
    // the staging buffer depends on n_in: grant the largest pipelined size once
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    granted[dev] = 1;
  }
  static int sms[64] = {0};
  if (!sms[dev]) {
    int v = 0;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    sms[dev] = v;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  *grid_out = per_sm * sms[dev];
  return cudaSuccess;
}

// Threads of the 4-line form: one task of each step per thread.
__host__ __device__ constexpr int conv4_threads(int A, int B) { return ((4 * (A > B ? A : B) + 31) / 32) * 32; }

// The pipelined z sweep in one of its forms (VP_ZFORM_*): 16-line tiles (256 threads),
// 8-line half tiles (256 threads), 4-line quarter tiles (4 max(A, B) threads), or the
// pair-split 8-line form (512 threads, L = 1280 only).  p.zform = 0 takes the form that
// keeps the most warps resident per SM (ties below); a form asked for that is not
// compiled for L or whose shared memory does not fit leaves the choice to that rule.  *used = false: no form
// applies (the caller falls back to the unpipelined kernel).
template <int A, int B>
cudaError_t line2_conv_pipe_launch(const LineSweep& p, cudaStream_t s, bool* used) {
  static volatile int granted16[64] = {0};
  static volatile int granted8[64] = {0};
  static volatile int granted4[64] = {0};
  static volatile int grantedp[64] = {0};
  static volatile int granted4t[64] = {0};
  static volatile int granted4b[64] = {0};
  static volatile int granted4tb[64] = {0};
  constexpr int L = A * B;
  constexpr int NT4 = conv4_threads(A, B);
  // the 4-line form with the two factors swapped (the shorter one in the full middle step)
  constexpr bool kSwap = (A == 32 && B == 40) || (L >= 640 && A < B && A % 2 == 0);
  // from L = 1024 the 4-line forms read their twiddles from global memory: the shared
  // copy would cost them a resident CTA an SM (6.40 against 6.91 ms for the 600 x 600 x
  // 640 grid; at L = 1024, with bulk staging, 2.98 against 3.02 ms, where with cp.async
  // staging the extra CTA had not paid: 3.30 against 3.26 ms)
  constexpr bool kTwg = L >= 1024;
  *used = false;
  // the kernel reads and writes the first half of each line only (zero-padded input,
  // cropped output); any other line goes to line2_kernel
  if (2 * p.n_in > L || 2 * p.n_out > L) return cudaSuccess;
  const int ni = conv_stage_pitch(A, B);
  // the 4-line forms stage each line and the octant line with one bulk copy where every
  // line starts and ends on a 16-byte boundary (cudaMalloc'd buffers, even n_in and ld)
  const bool bulk = p.staging == 0 && p.n_in % 2 == 0 && p.ld % 2 == 0 && ((uintptr_t)p.data & 15) == 0 &&
                    ((uintptr_t)p.khat & 15) == 0;
  constexpr int kForms = 6;
  int grid[kForms] = {0, 0, 0, 0, 0, 0};  // resident CTAs on the GPU, per form
  int threads[kForms] = {0, kThreads2, kThreads2, NT4, kThreadsPair, conv4_threads(B, A)};
  size_t smem[kForms] = {0, conv_pipe_smem(A, B, p.Oz), conv_pipe_smem(A, B, p.Oz, 8),
                         conv_pipe_smem(A, B, p.Oz, 4, kTwg, bulk), conv_pair8_smem(A, B, p.Oz),
                         conv_pipe_smem(B, A, p.Oz, 4, kTwg, bulk)};
  cudaError_t e;
  // a form asked for that is not compiled for L, or does not fit, leaves the choice open
  bool any = p.zform == 0;
  if (!any) {
    const bool compiled = p.zform == 1 || (p.zform == 2 && L >= 640) || (p.zform == 3 && L >= 512) ||
                          (p.zform == 4 && A == 32 && B == 40) || (p.zform == 5 && kSwap);
    any = !compiled || smem[p.zform] > 200 * 1024;
  }
  auto want = [&](int f) { return any || p.zform == f; };
  if (want(1) && smem[1] <= 200 * 1024) {
    e = resident_slots(line2_conv_pipe_kernel<A, B, false>, smem[1], granted16, &grid[1]);
    if (e != cudaSuccess) return e;
  }
  if constexpr (L >= 640) {
    if (want(2) && smem[2] <= 200 * 1024) {
      e = resident_slots(line2_conv_pipe_kernel<A, B, false, 8>, smem[2], granted8, &grid[2]);
      if (e != cudaSuccess) return e;
    }
  }
  if constexpr (L >= 512) {
    if (want(3) && smem[3] <= 200 * 1024) {
      e = bulk ? resident_slots(line2_conv_pipe_kernel<A, B, false, 4, NT4, kTwg, true>, smem[3], granted4b, &grid[3], NT4)
               : resident_slots(line2_conv_pipe_kernel<A, B, false, 4, NT4, kTwg>, smem[3], granted4, &grid[3], NT4);
      if (e != cudaSuccess) return e;
    }
  }
  if constexpr (A == 32 && B == 40) {
    if (want(4) && smem[4] <= 200 * 1024) {
      e = resident_slots(line2_conv_pair8_kernel<A, B>, smem[4], grantedp, &grid[4], kThreadsPair);
      if (e != cudaSuccess) return e;
    }
  }
  if constexpr (kSwap) {
    if (want(5) && smem[5] <= 200 * 1024) {
      e = bulk ? resident_slots(line2_conv_pipe_kernel<B, A, false, 4, conv4_threads(B, A), kTwg, true>, smem[5],
                                granted4tb, &grid[5], conv4_threads(B, A))
               : resident_slots(line2_conv_pipe_kernel<B, A, false, 4, conv4_threads(B, A), kTwg>, smem[5], granted4t,
                                &grid[5], conv4_threads(B, A));
      if (e != cudaSuccess) return e;
    }
  }
  // ties: from L = 640 the shorter tile (measured faster: 2.31 against 2.49 ms at L = 864
  // on 432^3, 1.64 against 1.73 ms at L = 768); below, the longer one (at L = 512 the
  // 4-line form leaves half its threads idle in the second step: 0.65 against 0.41 ms)
  auto rank = [&](int f) { return L >= 640 ? f : kForms - f; };
  int best = 0;
  for (int f = 1; f < kForms; ++f) {
    if (grid[f] < 1) continue;
    const long long wf = (long long)grid[f] * threads[f], wb = best ? (long long)grid[best] * threads[best] : 0;
    if (best == 0 || wf > wb || (wf == wb && rank(f) > rank(best))) best = f;
  }
  // L = 1280: the swapped 40 x 32 split puts the 40-point DFTs in the pruned first and
  // last steps (half their inputs zero, half their outputs cropped) and leaves radix-2
  // 32-point DFTs for the full middle step: 7.64 against 8.34 ms for the pair-split
  // form on the 600 x 600 x 640 grid, with fewer resident warps
  if constexpr (kSwap) {
    if (grid[5] >= 1 && (p.zform == 0 || p.zform == 5 || any)) best = 5;
  }
  if (best == 0) return cudaSuccess;  // too large to pipeline (or the form asked for is not compiled)
  *used = true;
  if (p.nlines <= 0) return cudaSuccess;
  static BatchParams<LineSweep> none{};  // unused by the single-plan form
  const long long units = p.nlines * (best == 1 ? 1 : (best == 3 || best == 5 ? 4 : 2));
  const int g = (int)(grid[best] > units ? units : grid[best]);
  switch (best) {
    case 1:
      line2_conv_pipe_kernel<A, B, false><<<(unsigned)g, kThreads2, smem[1], s>>>(p, none, units, ni);
      break;
    case 2:
      if constexpr (L >= 640) line2_conv_pipe_kernel<A, B, false, 8><<<(unsigned)g, kThreads2, smem[2], s>>>(p, none, units, ni);
      break;
    case 3:
      if constexpr (L >= 512) {
        if (bulk)
          line2_conv_pipe_kernel<A, B, false, 4, NT4, kTwg, true>
              <<<(unsigned)g, NT4, smem[3], s>>>(p, none, units, conv_stage_pitch(A, B, 4));
        else
          line2_conv_pipe_kernel<A, B, false, 4, NT4, kTwg>
              <<<(unsigned)g, NT4, smem[3], s>>>(p, none, units, conv_stage_pitch(A, B, 4));
      }
      break;
    case 5:
      if constexpr (kSwap) {
        if (bulk)
          line2_conv_pipe_kernel<B, A, false, 4, conv4_threads(B, A), kTwg, true>
              <<<(unsigned)g, conv4_threads(B, A), smem[5], s>>>(p, none, units, conv_stage_pitch(B, A, 4));
        else
          line2_conv_pipe_kernel<B, A, false, 4, conv4_threads(B, A), kTwg>
              <<<(unsigned)g, conv4_threads(B, A), smem[5], s>>>(p, none, units, conv_stage_pitch(B, A, 4));
      }
      break;
    default:
      if constexpr (A == 32 && B == 40) line2_conv_pair8_kernel<A, B><<<(unsigned)g, kThreadsPair, smem[4], s>>>(p, units, ni);
      break;
  }
  return cudaGetLastError();
}

template <int A, int B>
cudaError_t line2_dispatch(const LineSweep& p, int mode, cudaStream_t s) {
  if (mode == kConv) {
    bool used = false;
    cudaError_t e = line2_conv_pipe_launch<A, B>(p, s, &used);
    if (e != cudaSuccess || used) return e;
    return line2_launch<A, B, kConv>(p, s);
  }
  return line2_launch<A, B, kForwardOnly>(p, s);
}

template <int A, int B, int DIR, bool SRC, bool HALF>
cudaError_t col2_batch_launch(const BatchParams<ColSweep>& bp, int total, cudaStream_t s) {
  static volatile int granted[64] = {0};
  const size_t smem = (size_t)kLines2 * col2_pitch(A * B) * sizeof(float2);
  if (total <= 0) return cudaSuccess;
  auto k = col2_batch_kernel<A, B, DIR, SRC, HALF>;
  cudaError_t e = grant_smem(k, smem, granted);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)total, kThreads2, smem, s>>>(bp);
  return cudaGetLastError();
}

template <int A, int B>
cudaError_t col2_batch_dispatch(const BatchParams<ColSweep>& bp, int total, int dir, bool src, cudaStream_t s) {
  bool half = true;
  for (int i = 0; i < bp.count; ++i) half = half && col2_half(bp.item[i], A * B, dir);
  if (dir == kForward && src) {
    if (!half) return cudaErrorInvalidValue;
    return col2_batch_launch<A, B, kForward, true, true>(bp, total, s);
  }
  if (dir == kForward) return half ? col2_batch_launch<A, B, kForward, false, true>(bp, total, s)
                                   : col2_batch_launch<A, B, kForward, false, false>(bp, total, s);
  return half ? col2_batch_launch<A, B, kInverse, false, true>(bp, total, s)
              : col2_batch_launch<A, B, kInverse, false, false>(bp, total, s);
}

// Batched z sweep: the pipelined persistent kernel over every tile of the group when
// its shared memory fits, else one CTA per tile.  first: any plan of the group (for the
// shared twiddle table and octant length); ni_max: longest input or output line of the
// group.
template <int A, int B>
cudaError_t line2_batch_dispatch(const LineSweep& first, int ni_max, const BatchParams<LineSweep>& bp, int total,
                                 cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const size_t psmem = conv_pipe_smem(A, B, first.Oz);
  if (psmem <= 200 * 1024 && 2 * ni_max <= A * B) {
    static volatile int pgranted[64] = {0};
    auto k = line2_conv_pipe_kernel<A, B, true>;
    int grid = 0;
    cudaError_t e = resident_slots(k, psmem, pgranted, &grid);
    if (e != cudaSuccess) return e;
    if (grid >= 1) {
      if (grid > total) grid = total;
      k<<<(unsigned)grid, kThreads2, psmem, s>>>(first, bp, total, conv_stage_pitch(A, B));
      return cudaGetLastError();
    }
  }
  static volatile int granted[64] = {0};
  const size_t smem = (size_t)kLines2 * line2_pitch(A, B) * sizeof(float2);
  auto k = line2_batch_kernel<A, B>;
  cudaError_t e = grant_smem(k, smem, granted);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)total, kThreads2, smem, s>>>(bp);
  return cudaGetLastError();
}

}  // namespace
}  // namespace vp
