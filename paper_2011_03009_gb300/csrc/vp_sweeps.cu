// FFT sweeps of the circulant-embedding convolution (Section 3.1, Section 6 step 3).
//
// vp_apply runs five sweeps over the padded cube, pruned so that the zero padding
// is never read and the cropped half is never written:
//   1. x forward   (N_x N_y N_z  -> M_x N_y N_z), optionally fused with the source
//                  assembly of Eq. 2.6
//   2. y forward   (M_x N_y N_z  -> M_x M_y N_z)
//   3. z forward, multiply by the kernel spectrum, z inverse (M_x M_y N_z in place)
//   4. y inverse   (M_x M_y N_z  -> M_x N_y N_z)
//   5. x inverse, crop and scale by 1/(M_x M_y M_z)  (-> N_x N_y N_z)
#include "fft_engine.cuh"

namespace vp {

namespace {

constexpr int kColP = kTileB;  // column tiles: rows of 16 columns (row-wise accesses only)
constexpr int kSrcChunk = 8;   // elements per thread per batch of source-assembly loads

// Shared memory of one column-sweep CTA: twiddles (L) then the tile (16 L).
__host__ __device__ constexpr size_t col_smem(int L) { return (size_t)L * (1 + kColP) * sizeof(float2); }
// Shared memory of one line-sweep CTA: the tile (16 L, swizzled), the z fold table
// (L ints) and four staged octant lines of the spectrum (4 Oz).
__host__ __device__ constexpr size_t line_smem(int L, int Oz) {
  return (size_t)L * kTileB * sizeof(float2) + (size_t)((L + 1) & ~1) * sizeof(int) +
         (size_t)Oz * 4 * sizeof(float2);
}

template <int DIR, bool SRC>
__global__ void __launch_bounds__(kThreads) col_sweep_kernel(const ColSweep p) {
  extern __shared__ float2 smem[];
  const int L = p.ax.L;
  float2* tw_s = smem;
  float2* tile = smem + L;
  const int ncb = (p.C + kTileB - 1) / kTileB;
  const int o = blockIdx.x / ncb;
  const int c0 = (blockIdx.x - o * ncb) * kTileB;

  stage_twiddles(tw_s, p.ax);
  const int nload = p.rows_in * kTileB;
  if constexpr (SRC) {
    // f_n = C_n sum_{m=1}^{n-1} p_m p_{n-m} (Eq. 2.6), summed over the pairs m <= n - m:
    // each unordered pair appears twice in the sum unless m = n - m.
    const int n = p.harmonic;
    for (int e0 = threadIdx.x; e0 < nload; e0 += kSrcChunk * blockDim.x) {
      float2 acc[kSrcChunk];
      long long off[kSrcChunk];
      bool ok[kSrcChunk];
#pragma unroll
      for (int j = 0; j < kSrcChunk; ++j) {
        const int e = e0 + j * blockDim.x;
        const int c = c0 + (e & (kTileB - 1));
        ok[j] = e < nload && c < p.C;
        off[j] = ok[j] ? (long long)o * p.in_os + (long long)(e >> 4) * p.in_rs + c : 0;
        acc[j] = make_float2(0.f, 0.f);
      }
      for (int m = 1; 2 * m <= n; ++m) {
        const float2* __restrict__ pa = p.lower[m - 1];
        const float2* __restrict__ pb = p.lower[n - m - 1];
        const float w = (2 * m == n) ? 1.f : 2.f;
        float2 a[kSrcChunk], bb[kSrcChunk];
#pragma unroll
        for (int j = 0; j < kSrcChunk; ++j) {
          a[j] = ok[j] ? __ldg(&pa[VP_CHKL(off[j], p.in_elems, 201)]) : make_float2(0.f, 0.f);
          bb[j] = ok[j] ? __ldg(&pb[VP_CHKL(off[j], p.in_elems, 202)]) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < kSrcChunk; ++j) acc[j] = cadd(acc[j], cscale(cmul(a[j], bb[j]), w));
      }
#pragma unroll
      for (int j = 0; j < kSrcChunk; ++j) {
        const int e = e0 + j * blockDim.x;
        if (e < nload) tile[VP_CHK(e, L * 16, 203)] = cscale(acc[j], p.cn);
      }
    }
  } else {
    for (int e = threadIdx.x; e < nload; e += blockDim.x) {
      const int c = c0 + (e & (kTileB - 1));
      const bool ok = c < p.C;
      const long long off = ok ? (long long)o * p.in_os + (long long)(e >> 4) * p.in_rs + c : 0;
      cp_async8(&tile[VP_CHK(e, L * 16, 204)], &p.in[VP_CHKL(off, p.in_elems, 205)], ok);
    }
  }
  cp_async_wait_all();
  __syncthreads();

  if (DIR == kForward) tile_forward<kColP, false>(tile, p.ax, tw_s, p.rows_in);
  else tile_inverse<kColP, false>(tile, p.ax, tw_s);

  const int nstore = p.rows_out * kTileB;
  for (int e = threadIdx.x; e < nstore; e += blockDim.x) {
    const int c = c0 + (e & (kTileB - 1));
    if (c < p.C) {
      const long long off = (long long)o * p.out_os + (long long)(e >> 4) * p.out_rs + c;
      float2 v = tile[VP_CHK(e, L * 16, 206)];
      if (DIR == kInverse) v = cscale(v, p.scale);
      p.out[VP_CHKL(off, p.out_elems, 207)] = v;
    }
  }
}

// Lines along the contiguous axis: 16 lines per CTA, copied into the swizzled tile so
// that the engine sees the same [row][line] layout as the column sweeps.
template <int MODE>
__global__ void __launch_bounds__(kThreads) line_sweep_kernel(const LineSweep p) {
  extern __shared__ float2 smem[];
  __shared__ long long line_of[kTileB];
  __shared__ int oct_of[4];
  const int L = p.ax.L;
  float2* tile = smem;
  int* fz_s = (int*)(smem + (size_t)L * kTileB);
  float2* ks = (float2*)(fz_s + ((L + 1) & ~1));  // [Oz][4], 8-byte aligned
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;

  if (threadIdx.x < kTileB) {
    long long l;
    if (MODE == kConv) {
      l = p.tiles[20LL * blockIdx.x + threadIdx.x];
    } else {
      l = (long long)blockIdx.x * kTileB + threadIdx.x;
      if (l >= p.nlines) l = -1;
    }
    line_of[threadIdx.x] = l;
  }
  if (MODE == kConv && threadIdx.x < 4) oct_of[threadIdx.x] = p.tiles[20LL * blockIdx.x + 16 + threadIdx.x];
  __syncthreads();

  for (int b = warp; b < kTileB; b += nwarps) {
    const long long l = line_of[b];
    const float2* src = p.data + (l < 0 ? 0 : l * p.ld);
#ifdef VP_DEBUG_CHECKS
    if (l >= 0) VP_CHKL(l * p.ld + p.n_in - 1, p.data_elems, 301);
#endif
    for (int z = lane; z < p.n_in; z += 32)
      cp_async8(&tile[VP_CHK((tix<16, true>(z, b)), L * 16, 302)], &src[z], l >= 0);
  }
  if (MODE == kConv) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) cp_async4(&fz_s[i], &p.fold_z[i]);
    for (int g = warp & 3; g < 4; g += 4) {
      const int oc = oct_of[g];
      const float2* kl = p.khat + (oc < 0 ? 0 : (long long)oc * p.Oz);
      for (int oz = (warp >> 2) * 32 + lane; oz < p.Oz; oz += (nwarps >> 2) * 32)
        cp_async8(&ks[VP_CHK(oz * 4 + g, p.Oz * 4, 303)], &kl[oz], oc >= 0);
    }
  }
  cp_async_wait_all();
  __syncthreads();

  if (MODE == kForwardOnly) {
    tile_forward<16, true>(tile, p.ax, p.ax.tw, p.n_in);
  } else {
    // forward passes except the last; the last forward pass, the spectrum multiply and
    // the first inverse pass run on the same registers (the last DIF pass has unit
    // twiddles, and so has the first DIT pass).
    const int P = p.ax.npass;
    for (int q = 0; q < P - 1; ++q) {
      dif_pass_rt<16, true>(p.ax, q, tile, p.ax.tw, q == 0 ? p.n_in : L);
      __syncthreads();
    }
    const int R = p.ax.radix[P - 1];
    const int nb = (L / R) * kTileB;
    const int rows_nz = P == 1 ? p.n_in : L;
#define VP_CONV_CASE(RR)                                                               \
  case RR: {                                                                           \
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {                               \
      const int b = t & (kTileB - 1);                                                  \
      const int base = (t >> 4) * RR;                                                  \
      float2 v[RR];                                                                    \
      _Pragma("unroll") for (int r = 0; r < RR; ++r) {                                 \
        const int row = base + r;                                                      \
        v[r] = row < rows_nz ? tile[tix<16, true>(row, b)] : make_float2(0.f, 0.f);    \
      }                                                                                \
      dft<RR, false>(v);                                                               \
      _Pragma("unroll") for (int r = 0; r < RR; ++r)                                   \
        v[r] = cmul(v[r], ks[VP_CHK(fz_s[VP_CHK(base + r, L, 304)] * 4 + (b >> 2), p.Oz * 4, 305)]); \
      dft<RR, true>(v);                                                                \
      _Pragma("unroll") for (int r = 0; r < RR; ++r) tile[tix<16, true>(base + r, b)] = v[r]; \
    }                                                                                  \
  } break;
    switch (R) {
      VP_CONV_CASE(16)
      VP_CONV_CASE(8)
      VP_CONV_CASE(4)
      VP_CONV_CASE(2)
      VP_CONV_CASE(5)
      VP_CONV_CASE(3)
      default: break;
    }
#undef VP_CONV_CASE
    __syncthreads();
    for (int q = P - 2; q >= 0; --q) {
      dit_pass_rt<16, true>(p.ax, q, tile, p.ax.tw);
      __syncthreads();
    }
  }

  for (int b = warp; b < kTileB; b += nwarps) {
    const long long l = line_of[b];
    if (l < 0) continue;
    float2* dst = p.data + l * p.ld;
#ifdef VP_DEBUG_CHECKS
    VP_CHKL(l * p.ld + p.n_out - 1, p.data_elems, 306);
#endif
    for (int z = lane; z < p.n_out; z += 32) dst[z] = tile[VP_CHK((tix<16, true>(z, b)), L * 16, 307)];
  }
}

// Grant a sweep kernel the largest tile it can be launched with, once per device.
// Each instantiation (TAG) keeps its own per-device flag.
constexpr size_t kColMax = col_smem(kMaxL);
constexpr size_t kLineMax = line_smem(kMaxL, kMaxL / 2 + 1);

template <int TAG, typename K>
cudaError_t set_smem(K kernel, size_t bytes, size_t max_bytes) {
  static volatile int granted[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (bytes <= 48 * 1024 || granted[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_bytes);
  if (e == cudaSuccess) granted[dev] = 1;
  return e;
}

}  // namespace

cudaError_t launch_col_sweep(const ColSweep& p, int dir, bool source_prologue, cudaStream_t s) {
  const size_t smem = col_smem(p.ax.L);
  const long long ncb = (p.C + kTileB - 1) / kTileB;
  const long long blocks = ncb * p.n_outer;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  cudaError_t e;
  if (dir == kForward && source_prologue) {
    auto k = col_sweep_kernel<kForward, true>;
    if ((e = set_smem<0>(k, smem, kColMax)) != cudaSuccess) return e;
    k<<<(unsigned)blocks, kThreads, smem, s>>>(p);
  } else if (dir == kForward) {
    auto k = col_sweep_kernel<kForward, false>;
    if ((e = set_smem<1>(k, smem, kColMax)) != cudaSuccess) return e;
    k<<<(unsigned)blocks, kThreads, smem, s>>>(p);
  } else {
    auto k = col_sweep_kernel<kInverse, false>;
    if ((e = set_smem<2>(k, smem, kColMax)) != cudaSuccess) return e;
    k<<<(unsigned)blocks, kThreads, smem, s>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_line_sweep(const LineSweep& p, int mode, cudaStream_t s) {
  const size_t smem = line_smem(p.ax.L, mode == kConv ? p.Oz : 0);
  const long long blocks = mode == kConv ? p.nlines : (p.nlines + kTileB - 1) / kTileB;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  cudaError_t e;
  if (mode == kConv) {
    auto k = line_sweep_kernel<kConv>;
    if ((e = set_smem<3>(k, smem, kLineMax)) != cudaSuccess) return e;
    k<<<(unsigned)blocks, kThreads, smem, s>>>(p);
  } else {
    auto k = line_sweep_kernel<kForwardOnly>;
    if ((e = set_smem<4>(k, smem, kLineMax)) != cudaSuccess) return e;
    k<<<(unsigned)blocks, kThreads, smem, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace vp

namespace vp {

cudaError_t launch_col_any(const ColSweep& p, int dir, bool src, cudaStream_t s) {
  // grouped row input: forward sweeps of the two-level engine without the source prologue
  if (p.in_rs_extra != 0 && (!p.ax.fast || dir != kForward || src)) return cudaErrorInvalidValue;
  if (!p.ax.fast) return launch_col_sweep(p, dir, src, s);
  cudaError_t e = launch_col2_part0(p, dir, src, s);
  if (e == cudaErrorNotSupported) e = launch_col2_part1(p, dir, src, s);
  if (e == cudaErrorNotSupported) e = launch_col2_part2(p, dir, src, s);
  return e;
}

cudaError_t launch_line_any(const LineSweep& p, int mode, cudaStream_t s) {
  if (!p.ax.fast) return launch_line_sweep(p, mode, s);
  cudaError_t e = launch_line2_part0(p, mode, s);
  if (e == cudaErrorNotSupported) e = launch_line2_part1(p, mode, s);
  if (e == cudaErrorNotSupported) e = launch_line2_part2(p, mode, s);
  return e;
}

}  // namespace vp

#ifdef VP_DEBUG_CHECKS
extern "C" VP_API int vp_debug_checks(int* out8, int reset) {
  if (cudaMemcpyFromSymbol(out8, vp::g_vp_debug, 8 * sizeof(int)) != cudaSuccess) return VP_ERR_CUDA;
  if (reset) {
    int z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (cudaMemcpyToSymbol(vp::g_vp_debug, z, sizeof(z)) != cudaSuccess) return VP_ERR_CUDA;
  }
  return VP_OK;
}
#endif
