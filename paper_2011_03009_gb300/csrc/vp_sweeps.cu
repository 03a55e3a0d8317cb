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

constexpr int kColP = kTileB;       // column tiles: rows of 16 columns, no padding needed
constexpr int kLineP = kTileB + 1;  // line tiles are written transposed: pad to dodge conflicts
constexpr size_t kColMax = (size_t)kMaxL * kColP * sizeof(float2);
constexpr size_t kLineMax = (size_t)kMaxL * kLineP * sizeof(float2);

template <int DIR, bool SRC>
__global__ void __launch_bounds__(kThreads) col_sweep_kernel(const ColSweep p) {
  extern __shared__ float2 tile[];
  const int ncb = (p.C + kTileB - 1) / kTileB;
  const int o = blockIdx.x / ncb;
  const int c0 = (blockIdx.x - o * ncb) * kTileB;
  const int L = p.ax.L;

  // load rows [0, rows_in) of 16 columns; forward sweeps treat the rest as zero
  const int nload = p.rows_in * kTileB;
  for (int e = threadIdx.x; e < nload; e += blockDim.x) {
    const int i = e >> 4;
    const int b = e & (kTileB - 1);
    const int c = c0 + b;
    float2 v = make_float2(0.f, 0.f);
    if (c < p.C) {
      const long long off = (long long)o * p.in_os + (long long)i * p.in_rs + c;
      if constexpr (SRC) {
        // f_n = C_n sum_{m=1}^{n-1} p_m p_{n-m}  (Eq. 2.6)
        float2 f[kMaxLower];
        const int nl = p.harmonic - 1;
#pragma unroll
        for (int m = 0; m < kMaxLower; ++m)
          if (m < nl) f[m] = __ldg(&p.lower[m][off]);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 1; m <= kMaxLower; ++m) {
          if (m <= nl) {
            const float2 a = f[m - 1];
            float2 bb = a;
#pragma unroll
            for (int j = 0; j < kMaxLower; ++j)
              if (j == p.harmonic - m - 1) bb = f[j];
            acc = cadd(acc, cmul(a, bb));
          }
        }
        v = cscale(acc, p.cn);
      } else {
        v = __ldg(&p.in[off]);
      }
    }
    tile[i * kColP + b] = v;
  }
  __syncthreads();

  if (DIR == kForward) tile_forward<kColP>(tile, p.ax, p.rows_in);
  else tile_inverse<kColP>(tile, p.ax);

  const int nstore = p.rows_out * kTileB;
  for (int e = threadIdx.x; e < nstore; e += blockDim.x) {
    const int i = e >> 4;
    const int b = e & (kTileB - 1);
    const int c = c0 + b;
    if (c < p.C) {
      const long long off = (long long)o * p.out_os + (long long)i * p.out_rs + c;
      float2 v = tile[i * kColP + b];
      if (DIR == kInverse) v = cscale(v, p.scale);
      p.out[off] = v;
    }
  }
  (void)L;
}

// Lines along the contiguous axis: 16 lines per CTA, loaded coalesced and stored
// transposed into the tile so that the engine sees the same [row][line] layout.
template <int MODE>
__global__ void __launch_bounds__(kThreads) line_sweep_kernel(const LineSweep p) {
  extern __shared__ float2 tile[];
  __shared__ long long kbase[kTileB];
  const long long l0 = (long long)blockIdx.x * kTileB;
  const int L = p.ax.L;

  if (MODE == kConv && threadIdx.x < kTileB) {
    const long long l = l0 + threadIdx.x;
    long long kb = 0;
    if (l < p.nlines) {
      const int px = (int)(l / p.My);
      const int py = (int)(l - (long long)px * p.My);
      kb = ((long long)p.fold_x[px] * p.Oy + p.fold_y[py]) * p.Oz;
    }
    kbase[threadIdx.x] = kb;
  }

  const int nload = kTileB * p.n_in;
  for (int e = threadIdx.x; e < nload; e += blockDim.x) {
    const int b = e / p.n_in;
    const int z = e - b * p.n_in;
    const long long l = l0 + b;
    float2 v = make_float2(0.f, 0.f);
    if (l < p.nlines) v = p.data[l * p.ld + z];
    tile[z * kLineP + b] = v;
  }
  __syncthreads();

  if (MODE == kForwardOnly) {
    tile_forward<kLineP>(tile, p.ax, p.n_in);
  } else {
    // forward passes except the last; the last forward pass, the spectrum multiply and
    // the first inverse pass run on the same registers (the last DIF pass has unit
    // twiddles, and so has the first DIT pass).
    const int P = p.ax.npass;
    for (int q = 0; q < P - 1; ++q) {
      dif_pass_rt<kLineP>(p.ax.radix[q], tile, L, p.ax.lp[q], p.ax.tw, q == 0 ? p.n_in : L);
      __syncthreads();
    }
    const int R = p.ax.radix[P - 1];
    const int nb = (L / R) * kTileB;
    const float2* __restrict__ kh = p.khat;
    const int* __restrict__ fz = p.fold_z;
    const int rows_nz = P == 1 ? p.n_in : L;
#define VP_CONV_CASE(RR)                                                         \
  case RR: {                                                                     \
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {                         \
      const int b = t & (kTileB - 1);                                            \
      const int base = (t >> 4) * RR;                                            \
      float2 v[RR];                                                              \
      _Pragma("unroll") for (int r = 0; r < RR; ++r) {                           \
        const int row = base + r;                                                \
        v[r] = row < rows_nz ? tile[row * kLineP + b] : make_float2(0.f, 0.f);   \
      }                                                                          \
      dft<RR, false>(v);                                                         \
      const long long kb = kbase[b];                                             \
      _Pragma("unroll") for (int r = 0; r < RR; ++r)                             \
        v[r] = cmul(v[r], __ldg(&kh[kb + __ldg(&fz[base + r])]));                \
      dft<RR, true>(v);                                                          \
      _Pragma("unroll") for (int r = 0; r < RR; ++r) tile[(base + r) * kLineP + b] = v[r]; \
    }                                                                            \
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
      dit_pass_rt<kLineP>(p.ax.radix[q], tile, L, p.ax.lp[q], p.ax.tw);
      __syncthreads();
    }
  }

  const int nstore = kTileB * p.n_out;
  for (int e = threadIdx.x; e < nstore; e += blockDim.x) {
    const int b = e / p.n_out;
    const int z = e - b * p.n_out;
    const long long l = l0 + b;
    if (l < p.nlines) p.data[l * p.ld + z] = tile[z * kLineP + b];
  }
}

// Grant a sweep kernel the largest tile it can be launched with, once per device.
// Each instantiation (TAG) keeps its own per-device flag.
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
  const size_t smem = (size_t)p.ax.L * kColP * sizeof(float2);
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
  const size_t smem = (size_t)p.ax.L * kLineP * sizeof(float2);
  const long long blocks = (p.nlines + kTileB - 1) / kTileB;
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
