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
    const size_t smem = (size_t)8 * col2_pitch(A * B) * sizeof(float2);
    const long long blocks = (long long)((p.C + 7) / 8) * p.n_outer;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    auto k = col2_kernel8<A, B, DIR, SRC, HALF>;
    cudaError_t e = grant_smem(k, smem, granted8);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)blocks, kThreads2, smem, s>>>(p);
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
cudaError_t col2_dispatch(const ColSweep& p, int dir, bool src, cudaStream_t s) {
  const bool half = col2_half(p, A * B, dir);
  if (dir == kForward && src) {
    // the source's grid is the embedded one: N <= M / 2 for every even M >= 2 N - 1
    if (!half) return cudaErrorInvalidValue;
    return col2_launch<A, B, kForward, true, true>(p, s);
  }
  if (dir == kForward) return half ? col2_launch<A, B, kForward, false, true>(p, s)
                                   : col2_launch<A, B, kForward, false, false>(p, s);
  return half ? col2_launch<A, B, kInverse, false, true>(p, s) : col2_launch<A, B, kInverse, false, false>(p, s);
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

template <int A, int B>
cudaError_t line2_conv_pipe_launch(const LineSweep& p, cudaStream_t s, bool* used) {
  static volatile int granted[64] = {0};
  static volatile int granted8[64] = {0};
  *used = false;
  // the kernel reads and writes the first half of each line only (zero-padded input,
  // cropped output); any other line goes to line2_kernel
  if (2 * p.n_in > A * B || 2 * p.n_out > A * B) return cudaSuccess;
  const int ni = conv_stage_pitch(A, B);
  if constexpr (A == 32 && B == 40) {
    // L = 1280: the pair-split half-tile form, 16 warps a CTA (at L = 1024 the halves'
    // rows share banks and it measured slower)
    static volatile int grantedp[64] = {0};
    const size_t smemp = conv_pair8_smem(A, B, p.Oz);
    int gridp = 0;
    if (smemp <= 200 * 1024) {
      cudaError_t e = resident_slots(line2_conv_pair8_kernel<A, B>, smemp, grantedp, &gridp, kThreadsPair);
      if (e != cudaSuccess) return e;
    }
    if (gridp >= 1) {
      *used = true;
      if (p.nlines <= 0) return cudaSuccess;
      const long long halves = 2LL * p.nlines;
      const int grid = (int)(gridp > halves ? halves : gridp);
      line2_conv_pair8_kernel<A, B><<<(unsigned)grid, kThreadsPair, smemp, s>>>(p, halves, ni);
      return cudaGetLastError();
    }
  }
  static BatchParams<LineSweep> none{};  // unused by the single-plan form
  // tiles of 16 lines, or (long lines) half tiles of 8 lines when those fit more CTAs per
  // SM: at L = 640-864 one 16-line CTA fills an SM's shared memory, two 8-line CTAs fit;
  // from L = 1024 only the 8-line form fits at all
  const size_t smem16 = conv_pipe_smem(A, B, p.Oz);
  int grid16 = 0, grid8 = 0;
  cudaError_t e;
  if (smem16 <= 200 * 1024) {
    e = resident_slots(line2_conv_pipe_kernel<A, B, false>, smem16, granted, &grid16);
    if (e != cudaSuccess) return e;
  }
  size_t smem8 = 0;
  if constexpr (A * B >= 640) {
    smem8 = conv_pipe_smem(A, B, p.Oz, 8);
    if (smem8 <= 200 * 1024) {
      e = resident_slots(line2_conv_pipe_kernel<A, B, false, 8>, smem8, granted8, &grid8);
      if (e != cudaSuccess) return e;
    }
  }
  if (grid16 < 1 && grid8 < 1) return cudaSuccess;  // too large to pipeline: caller falls back
  if (p.nlines <= 0) {
    *used = true;
    return cudaSuccess;
  }
  if constexpr (A * B >= 640) {
    if (grid8 > grid16) {
      const long long halves = 2LL * p.nlines;
      const int grid = (int)(grid8 > halves ? halves : grid8);
      line2_conv_pipe_kernel<A, B, false, 8><<<(unsigned)grid, kThreads2, smem8, s>>>(p, none, halves, ni);
      *used = true;
      return cudaGetLastError();
    }
  }
  const int grid = (int)(grid16 > p.nlines ? p.nlines : grid16);
  line2_conv_pipe_kernel<A, B, false><<<(unsigned)grid, kThreads2, smem16, s>>>(p, none, p.nlines, ni);
  *used = true;
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
