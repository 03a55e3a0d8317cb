// Non-FFT kernels: quadrature-kernel lattice with the self cell (Eq. 3.9), octant
// extraction of its spectrum, standalone source assembly (Eq. 2.6), trilinear
// restriction between nested grids (Section 6) and the incident field (Eq. 3.10).
#include <math.h>

#include <algorithm>
#include <cmath>

#include "fft_engine.cuh"

namespace vp {

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTwoPi = 6.283185307179586476925286766559005768;
constexpr double kInvTwoPi = 0.159154943091895335768883763372514362;

// exp(i * phase) with the phase reduced modulo 2 pi in FP64 before the FP32 sine/cosine.
__device__ __forceinline__ float2 unit_phasor(double phase) {
  const double red = fma(-kTwoPi, rint(phase * kInvTwoPi), phase);
  float s, c;
  sincosf((float)red, &s, &c);
  return make_float2(c, s);
}

struct cd { double re, im; };
__device__ __forceinline__ cd cd_mul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cd cd_div(cd a, cd b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// Integral of G_k over the ball of radius a about its centre: ((1 - i k a) e^{i k a} - 1) / k^2,
// or, for |k a| < 0.1, the power series sum_m (i k a)^m a^2 / (m! (m + 2)) of the same integral.
__device__ cd self_cell_fp64(double kr, double ki, double a) {
  const cd ka = {kr * a, ki * a};
  if (sqrt(ka.re * ka.re + ka.im * ka.im) < 0.1) {
    cd total = {0.0, 0.0}, term = {1.0, 0.0};
    const cd ika = {-ka.im, ka.re};
    for (int m = 0; m < 24; ++m) {
      total.re += term.re / (m + 2);
      total.im += term.im / (m + 2);
      term = cd_mul(term, ika);
      term.re /= (m + 1);
      term.im /= (m + 1);
    }
    return {total.re * a * a, total.im * a * a};
  }
  // e^{i k a} = e^{-Im(ka)} (cos Re(ka) + i sin Re(ka))
  double s, c;
  sincos(ka.re, &s, &c);
  const double m = exp(-ka.im);
  const cd e = {m * c, m * s};
  const cd one_m_ika = {1.0 + ka.im, -ka.re};  // 1 - i k a
  cd num = cd_mul(one_m_ika, e);
  num.re -= 1.0;
  const cd k = {kr, ki};
  return cd_div(num, cd_mul(k, k));
}

// Distance in FP64 without a full-precision square root: one Newton step on the
// single-precision reciprocal square root brings it to about 1e-14 relative.
__device__ __forceinline__ double fp64_norm(double r2) {
  double y = (double)rsqrtf((float)r2);
  y = y * fma(-0.5 * r2, y * y, 1.5);
  return r2 * y;
}

// Kernel lattice of Eq. 3.9 for the circulant embedding (Section 3.1): for every offset
// d in (-N, N)^3, h^3 e^{i k |d| h} / (4 pi |d| h) at index d mod M, the self-cell integral
// at d = 0.  The lattice is even in every axis, so one thread evaluates |d| for
// non-negative offsets and writes the value to each of its (up to 8) mirror positions;
// indices no offset maps to are zeroed beforehand.  |d| in FP64 (one Newton step on the
// FP32 reciprocal square root), phase reduced modulo 2 pi in FP64, amplitude in FP32.
__global__ void lattice_kernel(float2* out, int nx, int ny, int nz, int mx, int my, int mz, double h,
                               double kr, double ki) {
  const long long total = (long long)nx * ny * nz;
  const double h3_4pi = h * h * h / (4.0 * kPi);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int dz = (int)(idx % nz);
    const long long r1 = idx / nz;
    const int dy = (int)(r1 % ny);
    const int dx = (int)(r1 / ny);
    float2 v;
    if (dx == 0 && dy == 0 && dz == 0) {
      const double a = 0.62035049089940001666800681204778 * h;  // (3 / (4 pi))^(1/3) h
      const cd s = self_cell_fp64(kr, ki, a);
      v = make_float2((float)s.re, (float)s.im);
    } else {
      const double d2 = (double)((long long)dx * dx + (long long)dy * dy + (long long)dz * dz);
      const double r = fp64_norm(d2) * h;
      const float amp = (float)(h3_4pi / r) * expf(-(float)(ki * r));
      const float2 ph = unit_phasor(kr * r);
      v = make_float2(amp * ph.x, amp * ph.y);
    }
    const int xs[2] = {dx, dx > 0 ? mx - dx : -1};
    const int ys[2] = {dy, dy > 0 ? my - dy : -1};
    const int zs[2] = {dz, dz > 0 ? mz - dz : -1};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      if (xs[a] < 0) continue;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        if (ys[b] < 0) continue;
        float2* row = out + ((long long)xs[a] * my + ys[b]) * mz;
        row[zs[0]] = v;
        if (zs[1] >= 0) row[zs[1]] = v;
      }
    }
  }
}

__global__ void octant_kernel(const float2* __restrict__ scr, float2* __restrict__ oct, int my, int mz,
                              int ox, int oy, int oz, const int* __restrict__ pos_x,
                              const int* __restrict__ pos_y, const int* __restrict__ pos_z) {
  const long long total = (long long)ox * oy * oz;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int iz = (int)(idx % oz);
    const long long r1 = idx / oz;
    const int iy = (int)(r1 % oy);
    const int ix = (int)(r1 / oy);
    oct[idx] = scr[((long long)pos_x[ix] * my + pos_y[iy]) * mz + pos_z[iz]];
  }
}

struct LowerPtrs { const float2* p[kMaxLower]; };

__global__ void source_kernel(LowerPtrs lo, int harmonic, float cn, float2* __restrict__ out,
                              long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int m = 1; m < harmonic; ++m) acc = cadd(acc, cmul(__ldg(&lo.p[m - 1][i]), __ldg(&lo.p[harmonic - m - 1][i])));
    out[i] = cscale(acc, cn);
  }
}

// Target position along one axis in source-voxel units, t = a + i b, held in 64-bit
// fixed point with kFixBits fractional bits: T = A + i B exactly, with A and B the
// host-rounded a 2^kFixBits and b 2^kFixBits (error below 2^-kFixBits per unit of i).
constexpr int kFixBits = 40;

struct AxisFix { long long A, B; int n; };

// Interpolation stencil of one target along one axis: cnt source indices i0 .. i0+cnt-1
// with weights w[0..cnt-1].
//   ORD 1 (linear, Section 6): i0 = floor(t) clamped to [0, n-2], f = t - i0,
//         w = (1 - f, f).
//   ORD 2 (quadratic Lagrange through the three nearest centres): c = floor(t + 1/2)
//         clamped to [1, n-2], u = t - c, i0 = c - 1,
//         w = (u (u - 1) / 2, 1 - u^2, u (u + 1) / 2); a two-voxel axis falls back to
//         ORD 1.
// A one-voxel axis has cnt = 1, w = (1).  Returns whether t lies inside [0, n-1]
// (with 1e-9 voxel of slack).
// A fixed-point offset (kFixBits fractional bits) as a float: clamped to +-4 voxels
// (offsets of in-range targets are within [-1.5, 1.5]), dropped to 24 fractional bits and
// converted from 32 bits (a 64-bit integer conversion is a slow multi-cycle operation).
__device__ __forceinline__ float frac_to_float(long long d) {
  const long long lim = 4LL << kFixBits;
  d = d < -lim ? -lim : (d > lim ? lim : d);
  return (float)(int)(d >> (kFixBits - 24)) * (1.0f / 16777216.0f);
}

template <int ORD>
__device__ __forceinline__ bool stencil(const AxisFix& m, int i, int& i0, float (&w)[3], int& cnt) {
  const long long T = m.A + (long long)i * m.B;
  const long long tol = 1100;  // 1e-9 voxel in fixed point
  const bool inside = T >= -tol && T <= ((long long)(m.n - 1) << kFixBits) + tol;
  w[0] = 1.f;
  w[1] = w[2] = 0.f;
  if (m.n == 1) {
    i0 = 0;
    cnt = 1;
    return inside;
  }
  if (ORD == 2 && m.n >= 3) {
    long long c = (T + (1LL << (kFixBits - 1))) >> kFixBits;  // floor(t + 1/2)
    if (c < 1) c = 1;
    if (c > m.n - 2) c = m.n - 2;
    const float u = frac_to_float(T - (c << kFixBits));
    i0 = (int)c - 1;
    cnt = 3;
    w[0] = 0.5f * u * (u - 1.f);
    w[1] = (1.f - u) * (1.f + u);
    w[2] = 0.5f * u * (u + 1.f);
    return inside;
  }
  long long fl = T >> kFixBits;  // floor (arithmetic shift)
  if (fl < 0) fl = 0;
  if (fl > m.n - 2) fl = m.n - 2;
  i0 = (int)fl;
  cnt = 2;
  const float f = fminf(fmaxf(frac_to_float(T - (fl << kFixBits)), 0.f), 1.f);
  w[0] = 1.f - f;
  w[1] = f;
  return inside;
}

// The tensor-product stencil sum of one target, read from global memory.
__device__ __forceinline__ float2 gather_stencil(const float2* __restrict__ src, int sny, int snz, int x0, int y0,
                                                 int z0, const float (&wx)[3], const float (&wy)[3],
                                                 const float (&wz)[3], int cx, int cy, int cz) {
  const long long sy = snz, sx = (long long)sny * snz;
  float2 acc = make_float2(0.f, 0.f);
  for (int a = 0; a < cx; ++a) {
    float2 py = make_float2(0.f, 0.f);
    for (int b = 0; b < cy; ++b) {
      const float2* row = src + (x0 + a) * sx + (y0 + b) * sy + z0;
      float2 pz = make_float2(0.f, 0.f);
      for (int c = 0; c < cz; ++c) {
        const float2 v = __ldg(row + c);
        pz.x = fmaf(wz[c], v.x, pz.x);
        pz.y = fmaf(wz[c], v.y, pz.y);
      }
      py.x = fmaf(wy[b], pz.x, py.x);
      py.y = fmaf(wy[b], pz.y, py.y);
    }
    acc.x = fmaf(wx[a], py.x, acc.x);
    acc.y = fmaf(wx[a], py.y, acc.y);
  }
  return acc;
}

// Direct form: one thread per target, gathers from global memory (any spacing ratio).
template <int ORD>
__global__ void __launch_bounds__(128) restrict_kernel(const float2* __restrict__ src, int snx, int sny, int snz,
                                                       float2* __restrict__ dst, int dnx, int dny, int dnz,
                                                       AxisFix mx, AxisFix my, AxisFix mz, int zero_outside) {
  const int iz = blockIdx.x * blockDim.x + threadIdx.x;
  const int iy = blockIdx.y;
  const int ix = blockIdx.z;
  if (iz >= dnz) return;
  const long long idx = ((long long)ix * dny + iy) * dnz + iz;
  int x0, y0, z0, cx, cy, cz;
  float wx[3], wy[3], wz[3];
  bool in = stencil<ORD>(mx, ix, x0, wx, cx);
  in &= stencil<ORD>(my, iy, y0, wy, cy);
  in &= stencil<ORD>(mz, iz, z0, wz, cz);
  if (!in && zero_outside) {
    dst[idx] = make_float2(0.f, 0.f);
    return;
  }
  dst[idx] = gather_stencil(src, sny, snz, x0, y0, z0, wx, wy, wz, cx, cy, cz);
}

// Shared-memory tiled form: one CTA computes a 1 x 16 x 64 block of targets (four rows
// per thread) from the source sub-block they touch (ORD + 1 x planes, at most kRsY x kRsZ
// source voxels), staged once with coalesced loads.  Every stencil of the block (its x
// stencil, the 16 y and the 64 z stencils) is computed once, in parallel, into shared
// memory, so a target costs only its tile reads and multiply-adds.  Used when the target
// spacing is at most about the source spacing on y and z (nested grids of higher
// harmonics are finer), so the sub-block always fits.  (A persistent variant that
// prefetched the next tile with cp.async measured slower: fewer resident warps and more
// barriers per tile.)
constexpr int kRtY = 16, kRtZ = 64, kRsY = 20, kRsZ = 80, kRowsPerThread = kRtY / 4;

struct RStencil {
  int i0, cnt, in;
  float w[3];
};

// Stencils of one 1 x 16 x 64 target block into shared memory: threads 0..63 the z
// stencils, 64..79 the y stencils, 80 the x stencil (targets past the grid's end reuse
// the last target's stencil so that the source ranges stay valid).
template <int ORD>
__device__ __forceinline__ void block_stencils(const AxisFix& mx, const AxisFix& my, const AxisFix& mz, int ix,
                                               int iy0, int iz0, int dny, int dnz, RStencil* sx_, RStencil* sy_,
                                               RStencil* sz_) {
  const int t = threadIdx.x;
  RStencil r;
  if (t < kRtZ) {
    r.in = stencil<ORD>(mz, min(iz0 + t, dnz - 1), r.i0, r.w, r.cnt);
    sz_[t] = r;
  } else if (t < kRtZ + kRtY) {
    r.in = stencil<ORD>(my, min(iy0 + t - kRtZ, dny - 1), r.i0, r.w, r.cnt);
    sy_[t - kRtZ] = r;
  } else if (t == kRtZ + kRtY) {
    r.in = stencil<ORD>(mx, ix, r.i0, r.w, r.cnt);
    sx_[0] = r;
  }
}

// The source sub-block a target block touches (its x planes, at most FY x FZ source
// voxels each; the host sizes FY, FZ from the spacing ratio), one warp per source row,
// lanes along z, copied with cp.async: every copy is in flight at once, the caller
// commits and waits.  Tile layout: [x plane][y row][z], plane = FY * FZ, pitch = FZ.
template <int ORD>
__device__ __forceinline__ void stage_block_async(const float2* __restrict__ src, int sny, int snz,
                                                  const RStencil* sx_, const RStencil* sy_, const RStencil* sz_,
                                                  float2* tile, int plane, int pitch) {
  const int x0 = sx_[0].i0, cx = sx_[0].cnt;
  const int ys = sy_[0].i0, zs = sz_[0].i0;
  const int ny_r = min(sy_[kRtY - 1].i0 + sy_[kRtY - 1].cnt - 1, sny - 1) - ys + 1;
  const int nz_r = min(sz_[kRtZ - 1].i0 + sz_[kRtZ - 1].cnt - 1, snz - 1) - zs + 1;
  const long long sy = snz, sxs = (long long)sny * snz;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = warp; r < cx * ny_r; r += (int)(blockDim.x >> 5)) {
    const int xi = r >= 2 * ny_r ? 2 : (r >= ny_r ? 1 : 0);
    const int yy = r - xi * ny_r;
    const float2* row = src + (x0 + xi) * sxs + (ys + yy) * sy + zs;
    float2* trow = tile + xi * plane + yy * pitch;
    for (int zz = lane; zz < nz_r; zz += 32) cp_async8(&trow[zz], &row[zz], true);
  }
}

// One target from the staged sub-block; y0, z0 are its stencils' first rows within it.
template <int ORD>
__device__ __forceinline__ float2 interp_block(const float2* tile, int plane, int pitch, const RStencil& xst,
                                               const RStencil& yst, const RStencil& zst, int y0, int z0) {
  const float wx0 = xst.w[0], wx1 = xst.w[1], wx2 = xst.w[2];
  const float2* t0 = tile + y0 * pitch + z0;
  if (ORD == 1 && xst.cnt == 2 && yst.cnt == 2 && zst.cnt == 2) {
    // interior of a linear restriction: the 2 x 2 x 2 stencil, straight-line
    const float2* t1 = t0 + plane;
    const float wz0 = zst.w[0], wz1 = zst.w[1], wy0 = yst.w[0], wy1 = yst.w[1];
    const float2 a00 = t0[0], a01 = t0[1], a10 = t0[pitch], a11 = t0[pitch + 1];
    const float2 b00 = t1[0], b01 = t1[1], b10 = t1[pitch], b11 = t1[pitch + 1];
    float2 p0, p1;
    p0.x = wy0 * fmaf(wz1, a01.x, wz0 * a00.x) + wy1 * fmaf(wz1, a11.x, wz0 * a10.x);
    p0.y = wy0 * fmaf(wz1, a01.y, wz0 * a00.y) + wy1 * fmaf(wz1, a11.y, wz0 * a10.y);
    p1.x = wy0 * fmaf(wz1, b01.x, wz0 * b00.x) + wy1 * fmaf(wz1, b11.x, wz0 * b10.x);
    p1.y = wy0 * fmaf(wz1, b01.y, wz0 * b00.y) + wy1 * fmaf(wz1, b11.y, wz0 * b10.y);
    return make_float2(fmaf(wx1, p1.x, wx0 * p0.x), fmaf(wx1, p1.y, wx0 * p0.y));
  }
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int a = 0; a <= ORD; ++a) {
    if (a >= xst.cnt) break;
    float2 py = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b <= ORD; ++b) {
      if (b >= yst.cnt) break;
      float2 pz = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c <= ORD; ++c) {
        if (c >= zst.cnt) break;
        const float2 v = t0[a * plane + b * pitch + c];
        pz.x = fmaf(zst.w[c], v.x, pz.x);
        pz.y = fmaf(zst.w[c], v.y, pz.y);
      }
      py.x = fmaf(yst.w[b], pz.x, py.x);
      py.y = fmaf(yst.w[b], pz.y, py.y);
    }
    const float wxa = a == 0 ? wx0 : (a == 1 ? wx1 : wx2);
    acc.x = fmaf(wxa, py.x, acc.x);
    acc.y = fmaf(wxa, py.y, acc.y);
  }
  return acc;
}

template <int ORD>
__global__ void __launch_bounds__(256) restrict_tiled_kernel(const float2* __restrict__ src, int snx, int sny,
                                                             int snz, float2* __restrict__ dst, int dnx, int dny,
                                                             int dnz, AxisFix mx, AxisFix my, AxisFix mz,
                                                             int zero_outside) {
  __shared__ float2 tile[ORD + 1][kRsY][kRsZ];
  __shared__ RStencil sx_[1], sy_[kRtY], sz_[kRtZ];
  const int ix = blockIdx.z, iy0 = blockIdx.y * kRtY, iz0 = blockIdx.x * kRtZ;
  (void)snx;
  (void)dnx;
  block_stencils<ORD>(mx, my, mz, ix, iy0, iz0, dny, dnz, sx_, sy_, sz_);
  __syncthreads();
  stage_block_async<ORD>(src, sny, snz, sx_, sy_, sz_, &tile[0][0][0], kRsY * kRsZ, kRsZ);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  const int lz = threadIdx.x & (kRtZ - 1);
  const int iz = iz0 + lz;
  if (iz >= dnz) return;
  const RStencil xst = sx_[0], zst = sz_[lz];
  const int z0 = zst.i0 - sz_[0].i0;
#pragma unroll
  for (int k = 0; k < kRowsPerThread; ++k) {
    const int ly = (threadIdx.x / kRtZ) * kRowsPerThread + k;
    const int iy = iy0 + ly;
    if (iy >= dny) break;
    const RStencil yst = sy_[ly];
    const long long idx = ((long long)ix * dny + iy) * dnz + iz;
    if (!(xst.in && zst.in && yst.in) && zero_outside) {
      dst[idx] = make_float2(0.f, 0.f);
      continue;
    }
    dst[idx] = interp_block<ORD>(&tile[0][0][0], kRsY * kRsZ, kRsZ, xst, yst, zst, yst.i0 - sy_[0].i0, z0);
  }
}

// ---- source on a nested grid: restriction fused with the Eq. 2.6 products -------------
// Lower harmonic p_m (m = 1..NS) lives on its own grid q.s[m-1]; its value at a target
// voxel is the restriction above (the same stencils and FP32 operations), and the target
// gets f_n = C_n sum_{m=1}^{n-1} p_m p_{n-m}, n = NS + 1, summed over the pairs
// m <= n - m with weight 2 off the diagonal (as the source prologue of the first sweep).
// The restricted fields are never stored.
template <int NS>
struct NestedSrcs {
  const float2* f[NS];
  int sny[NS], snz[NS];
  AxisFix m[NS][3];
};

template <int NS>
__device__ __forceinline__ float2 pair_products(const float2 (&r)[NS], float cn) {
  constexpr int n = NS + 1;
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 1; 2 * m <= n; ++m) {
    const float w = ((2 * m == n) ? 1.f : 2.f) * cn;
    const float2 xy = cmul(r[m - 1], r[n - m - 1]);
    acc.x = fmaf(w, xy.x, acc.x);
    acc.y = fmaf(w, xy.y, acc.y);
  }
  return acc;
}

// Tiled form (every source's sub-block fits the staging tile).  The stencils of every
// source are computed first; the sources' sub-blocks are then staged with cp.async into
// two tiles in turn, the next one in flight while the current one is interpolated.  Each
// thread keeps its four targets' restricted values of every source in registers.  The
// tiles are sized to the largest footprint of the sources (FY x FZ per x plane), so that
// as many CTAs as possible share an SM.
// Dynamic shared memory: two tiles, then NS x (1 + kRtY + kRtZ) stencils (x, y, z).
constexpr int kStencilsPerSrc = 1 + kRtY + kRtZ;

template <int ORD>
size_t nested_tiled_smem(int ns, int fy, int fz) {
  return 2 * sizeof(float2) * (size_t)(ORD + 1) * fy * fz + sizeof(RStencil) * (size_t)ns * kStencilsPerSrc;
}

template <int ORD, int NS>
__global__ void __launch_bounds__(256) source_nested_tiled_kernel(const __grid_constant__ NestedSrcs<NS> q, float cn,
                                                                  float2* __restrict__ dst, int dny, int dnz, int fy,
                                                                  int fz) {
  extern __shared__ float4 smem_raw[];
  float2* tiles = reinterpret_cast<float2*>(smem_raw);
  const int plane = fy * fz, tile_size = (ORD + 1) * plane;
  RStencil* st = reinterpret_cast<RStencil*>(tiles + 2 * tile_size);  // source m: x, y[16], z[64]
  const int ix = blockIdx.z, iy0 = blockIdx.y * kRtY, iz0 = blockIdx.x * kRtZ;
  const int lz = threadIdx.x & (kRtZ - 1);
  // stencils of every source (targets past the grid's end reuse the last target's)
  for (int i = threadIdx.x; i < NS * kStencilsPerSrc; i += blockDim.x) {
    const int m = i / kStencilsPerSrc, t = i - m * kStencilsPerSrc;
    RStencil r;
    if (t == 0) r.in = stencil<ORD>(q.m[m][0], ix, r.i0, r.w, r.cnt);
    else if (t <= kRtY) r.in = stencil<ORD>(q.m[m][1], min(iy0 + t - 1, dny - 1), r.i0, r.w, r.cnt);
    else r.in = stencil<ORD>(q.m[m][2], min(iz0 + t - 1 - kRtY, dnz - 1), r.i0, r.w, r.cnt);
    st[i] = r;
  }
  __syncthreads();
  auto stage = [&](int m) {
    const RStencil* s0 = st + m * kStencilsPerSrc;
    stage_block_async<ORD>(q.f[m], q.sny[m], q.snz[m], s0, s0 + 1, s0 + 1 + kRtY, tiles + (m & 1) * tile_size,
                           plane, fz);
  };
  stage(0);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  if (NS > 1) stage(1);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  float2 r[kRowsPerThread][NS];
#pragma unroll
  for (int m = 0; m < NS; ++m) {
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // source m's group is complete
    __syncthreads();
    const RStencil* s0 = st + m * kStencilsPerSrc;
    const RStencil xst = s0[0], zst = s0[1 + kRtY + lz];
    const int z0 = zst.i0 - s0[1 + kRtY].i0;
    const float2* tile = tiles + (m & 1) * tile_size;
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
      const RStencil yst = s0[1 + (threadIdx.x / kRtZ) * kRowsPerThread + k];
      r[k][m] = interp_block<ORD>(tile, plane, fz, xst, yst, zst, yst.i0 - s0[1].i0, z0);
    }
    if (m + 2 < NS) {
      __syncthreads();  // every thread is done with this tile
      stage(m + 2);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  const int iz = iz0 + lz;
  if (iz >= dnz) return;
#pragma unroll
  for (int k = 0; k < kRowsPerThread; ++k) {
    const int iy = iy0 + (threadIdx.x / kRtZ) * kRowsPerThread + k;
    if (iy >= dny) break;
    dst[((long long)ix * dny + iy) * dnz + iz] = pair_products<NS>(r[k], cn);
  }
}

// Linear form of the tiled kernel for sources with at least two voxels on every axis,
// where every stencil is the 2 x 2 x 2 one (cnt = 2, w = (1 - f, f)): no per-target
// stencil-size tests, and each interpolation is seven lerps a + f (b - a) on paired FP32
// (f32x2) operations, the real and imaginary parts in one instruction each.  The
// per-target stencil data is packed once per CTA: {row offset in the tile, (f, f)} for
// the 16 y rows and the 64 z columns of each source, and (f, f) for x.
struct LinStencil {
  int off;
  int pad;
  float2 f;  // (f, f): the fraction on both lanes of a paired operation
};

__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float2 f) {
  return __ffma2_rn(f, __fadd2_rn(b, make_float2(-a.x, -a.y)), a);
}

template <int NS>
__global__ void __launch_bounds__(256) source_nested_lin_kernel(const __grid_constant__ NestedSrcs<NS> q, float cn,
                                                                float2* __restrict__ dst, int dny, int dnz, int fy,
                                                                int fz) {
  extern __shared__ float4 smem_raw[];
  float2* tiles = reinterpret_cast<float2*>(smem_raw);
  const int plane = fy * fz, tile_size = 2 * plane;
  RStencil* st = reinterpret_cast<RStencil*>(tiles + 2 * tile_size);  // source m: x, y[16], z[64]
  LinStencil* ls = reinterpret_cast<LinStencil*>(st + NS * kStencilsPerSrc);  // source m: x, y[16], z[64]
  const int ix = blockIdx.z, iy0 = blockIdx.y * kRtY, iz0 = blockIdx.x * kRtZ;
  const int lz = threadIdx.x & (kRtZ - 1);
  for (int i = threadIdx.x; i < NS * kStencilsPerSrc; i += blockDim.x) {
    const int m = i / kStencilsPerSrc, t = i - m * kStencilsPerSrc;
    RStencil r;
    if (t == 0) r.in = stencil<1>(q.m[m][0], ix, r.i0, r.w, r.cnt);
    else if (t <= kRtY) r.in = stencil<1>(q.m[m][1], min(iy0 + t - 1, dny - 1), r.i0, r.w, r.cnt);
    else r.in = stencil<1>(q.m[m][2], min(iz0 + t - 1 - kRtY, dnz - 1), r.i0, r.w, r.cnt);
    st[i] = r;
  }
  __syncthreads();
  // packed form: offsets from the staged block's first row and column
  for (int i = threadIdx.x; i < NS * kStencilsPerSrc; i += blockDim.x) {
    const int m = i / kStencilsPerSrc, t = i - m * kStencilsPerSrc;
    const RStencil* s0 = st + m * kStencilsPerSrc;
    LinStencil l;
    l.pad = 0;
    l.f = make_float2(st[i].w[1], st[i].w[1]);
    if (t == 0) l.off = 0;
    else if (t <= kRtY) l.off = (st[i].i0 - s0[1].i0) * fz;
    else l.off = st[i].i0 - s0[1 + kRtY].i0;
    ls[i] = l;
  }
  auto stage = [&](int m) {
    const RStencil* s0 = st + m * kStencilsPerSrc;
    stage_block_async<1>(q.f[m], q.sny[m], q.snz[m], s0, s0 + 1, s0 + 1 + kRtY, tiles + (m & 1) * tile_size, plane,
                         fz);
  };
  stage(0);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  if (NS > 1) stage(1);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  float2 r[kRowsPerThread][NS];
  const int row0 = (threadIdx.x / kRtZ) * kRowsPerThread;
#pragma unroll
  for (int m = 0; m < NS; ++m) {
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // source m's group is complete
    __syncthreads();
    const LinStencil* l0 = ls + m * kStencilsPerSrc;
    const float2 fx = l0[0].f;
    const LinStencil zl = l0[1 + kRtY + lz];
    const float2* tile = tiles + (m & 1) * tile_size + zl.off;
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
      const LinStencil yl = l0[1 + row0 + k];
      const float2* t0 = tile + yl.off;
      const float2* t1 = t0 + plane;
      const float2 a0 = lerp2(t0[0], t0[1], zl.f), a1 = lerp2(t0[fz], t0[fz + 1], zl.f);
      const float2 b0 = lerp2(t1[0], t1[1], zl.f), b1 = lerp2(t1[fz], t1[fz + 1], zl.f);
      r[k][m] = lerp2(lerp2(a0, a1, yl.f), lerp2(b0, b1, yl.f), fx);
    }
    if (m + 2 < NS) {
      __syncthreads();  // every thread is done with this tile
      stage(m + 2);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  const int iz = iz0 + lz;
  if (iz >= dnz) return;
#pragma unroll
  for (int k = 0; k < kRowsPerThread; ++k) {
    const int iy = iy0 + row0 + k;
    if (iy >= dny) break;
    dst[((long long)ix * dny + iy) * dnz + iz] = pair_products<NS>(r[k], cn);
  }
}

// Direct form (any spacing ratio): one thread per target, gathers from global memory.
template <int ORD, int NS>
__global__ void __launch_bounds__(128) source_nested_kernel(const __grid_constant__ NestedSrcs<NS> q, float cn,
                                                            float2* __restrict__ dst, int dny, int dnz) {
  const int iz = blockIdx.x * blockDim.x + threadIdx.x;
  const int iy = blockIdx.y;
  const int ix = blockIdx.z;
  if (iz >= dnz) return;
  float2 r[NS];
#pragma unroll
  for (int m = 0; m < NS; ++m) {
    int x0, y0, z0, cx, cy, cz;
    float wx[3], wy[3], wz[3];
    stencil<ORD>(q.m[m][0], ix, x0, wx, cx);
    stencil<ORD>(q.m[m][1], iy, y0, wy, cy);
    stencil<ORD>(q.m[m][2], iz, z0, wz, cz);
    r[m] = gather_stencil(q.f[m], q.sny[m], q.snz[m], x0, y0, z0, wx, wy, wz, cx, cy, cz);
  }
  dst[((long long)ix * dny + iy) * dnz + iz] = pair_products<NS>(r, cn);
}

// Localisation measure of Section 5: Q(x) = log10(|f(x)| / max |f|).  The smallest box
// holding every voxel with Q >= Q0 is found in two passes: max |f|^2, then the index
// bounds of the voxels with |f|^2 >= 10^(2 Q0) max |f|^2.  Squares are formed in FP64
// from the FP32 parts (exact products, one rounding in the sum), so the decision is
// reproducible on the host.  Non-negative doubles order like their bit patterns, which
// lets atomicMax work on the 64-bit integer view.
__device__ __forceinline__ double abs2_fp64(float2 v) {
  const double re = v.x, im = v.y;
  return re * re + im * im;
}

__global__ void __launch_bounds__(256) max_abs2_kernel(const float2* __restrict__ f, long long count,
                                                       unsigned long long* __restrict__ out_bits) {
  __shared__ double part[8];
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, abs2_fp64(__ldg(&f[i])));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, part[w]);
    atomicMax(out_bits, (unsigned long long)__double_as_longlong(m));
  }
}

// box[0..2] = min index per axis, box[3..5] = max index (initialised to n and -1)
__global__ void __launch_bounds__(256) q0_box_kernel(const float2* __restrict__ f, int nx, int ny, int nz,
                                                     const unsigned long long* __restrict__ max_bits,
                                                     double factor, int* __restrict__ box) {
  __shared__ int sb[6];
  if (threadIdx.x < 6) sb[threadIdx.x] = threadIdx.x < 3 ? 0x7fffffff : -1;
  __syncthreads();
  const double thr = __longlong_as_double((long long)*max_bits) * factor;
  const long long count = (long long)nx * ny * nz;
  int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {-1, -1, -1};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    if (abs2_fp64(__ldg(&f[i])) >= thr) {
      const int iz = (int)(i % nz);
      const long long r = i / nz;
      const int iy = (int)(r % ny), ix = (int)(r / ny);
      lo[0] = min(lo[0], ix); hi[0] = max(hi[0], ix);
      lo[1] = min(lo[1], iy); hi[1] = max(hi[1], iy);
      lo[2] = min(lo[2], iz); hi[2] = max(hi[2], iz);
    }
  }
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
    for (int a = 0; a < 3; ++a) {
      atomicMin(&sb[a], lo[a]);
      atomicMax(&sb[3 + a], hi[a]);
    }
  }
  __syncthreads();
  if (threadIdx.x < 3) atomicMin(&box[threadIdx.x], sb[threadIdx.x]);
  else if (threadIdx.x < 6) atomicMax(&box[threadIdx.x], sb[threadIdx.x]);
}

__global__ void q0_init_kernel(unsigned long long* max_bits, int* box) {
  if (threadIdx.x == 0) *max_bits = 0ULL;
  if (threadIdx.x < 3) box[threadIdx.x] = 0x7fffffff;
  else if (threadIdx.x < 6) box[threadIdx.x] = -1;
}

constexpr int kIncBlock = 256;
constexpr int kIncTx = 4, kIncTy = 8, kIncTz = 8;  // voxel tile of one CTA (kIncBlock voxels)


// Incident field of Eq. 3.10 on a voxel grid, one CTA per 4 x 8 x 8 voxel tile.
// For each bowl point p and the tile centre c, the FP64 work is done once per CTA:
// d = c - p, r_c = |d|, the phase k r_c reduced modulo 2 pi, and e^{-k'' r_c} / (4 pi).
// For a voxel x = c + delta of the tile, r - r_c = u / (r_c (1 + sqrt(1 + u / r_c^2)))
// with u = 2 d.delta + |delta|^2 (the cancellation-free root of r^2 = r_c^2 + u),
// which is small (|r - r_c| <= |delta| <= 5.1 h), so it, the phase increment k' (r - r_c)
// and the attenuation factor e^{-k''(r - r_c)} = 1 - k''(r - r_c) + O(1e-9) are
// accurate in FP32 to about 1e-7 of a radian.  Points closer to the tile than four
// tile radii take the direct FP64 evaluation instead.
__global__ void __launch_bounds__(kIncBlock) incident_kernel(const double* __restrict__ pts, int npts,
                                                             int nx, int ny, int nz, double ox,
                                                             double oy, double oz, double h, double kr,
                                                             double ki, double sre, double sim,
                                                             float2* __restrict__ out) {
  __shared__ float sd[3][kIncBlock];   // d = c - p (FP32)
  __shared__ float sinv[kIncBlock];    // 1 / r_c^2, NaN: evaluate directly in FP64
  __shared__ float src_[kIncBlock];    // r_c
  __shared__ float sphi[kIncBlock];    // k' r_c mod 2 pi
  __shared__ float samp[kIncBlock];    // e^{-k'' r_c} / (4 pi)
  __shared__ double sp[3][kIncBlock];  // the points themselves (direct path)
  const int tiles_z = (nz + kIncTz - 1) / kIncTz, tiles_y = (ny + kIncTy - 1) / kIncTy;
  const long long tile = blockIdx.x;
  const int tz = (int)(tile % tiles_z);
  const long long r1 = tile / tiles_z;
  const int ty = (int)(r1 % tiles_y);
  const int tx = (int)(r1 / tiles_y);
  const int lz = threadIdx.x % kIncTz, ly = (threadIdx.x / kIncTz) % kIncTy, lx = threadIdx.x / (kIncTz * kIncTy);
  const int ix = tx * kIncTx + lx, iy = ty * kIncTy + ly, iz = tz * kIncTz + lz;
  const bool active = ix < nx && iy < ny && iz < nz;
  // tile centre (in voxel units from the tile's first voxel: 1.5, 3.5, 3.5)
  const double cx = fma(tx * kIncTx + 0.5 * (kIncTx - 1), h, ox);
  const double cy = fma(ty * kIncTy + 0.5 * (kIncTy - 1), h, oy);
  const double cz = fma(tz * kIncTz + 0.5 * (kIncTz - 1), h, oz);
  const float hf = (float)h;
  const float dlx = (lx - 0.5f * (kIncTx - 1)) * hf, dly = (ly - 0.5f * (kIncTy - 1)) * hf,
              dlz = (lz - 0.5f * (kIncTz - 1)) * hf;
  const float dl2 = dlx * dlx + dly * dly + dlz * dlz;
  const double tile_r = 0.5 * h * sqrt((double)((kIncTx - 1) * (kIncTx - 1) + (kIncTy - 1) * (kIncTy - 1) +
                                                (kIncTz - 1) * (kIncTz - 1)));
  const double near2 = 16.0 * tile_r * tile_r;
  const float krf = (float)kr, kif = (float)ki;
  const float inv4pi = (float)(1.0 / (4.0 * kPi));
  double are = 0.0, aim = 0.0;
  for (int c0 = 0; c0 < npts; c0 += kIncBlock) {
    const int j = c0 + threadIdx.x;
    if (j < npts) {
      const double px = pts[3 * (long long)j + 0], py = pts[3 * (long long)j + 1], pz = pts[3 * (long long)j + 2];
      sp[0][threadIdx.x] = px;
      sp[1][threadIdx.x] = py;
      sp[2][threadIdx.x] = pz;
      const double dx = cx - px, dy = cy - py, dz = cz - pz;
      const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
      const double rc = sqrt(r2);
      sd[0][threadIdx.x] = (float)dx;
      sd[1][threadIdx.x] = (float)dy;
      sd[2][threadIdx.x] = (float)dz;
      sinv[threadIdx.x] = r2 > near2 ? (float)(1.0 / r2) : __int_as_float(0x7fffffff);
      src_[threadIdx.x] = (float)rc;
      const double ph = kr * rc;
      sphi[threadIdx.x] = (float)fma(-kTwoPi, rint(ph * kInvTwoPi), ph);
      samp[threadIdx.x] = (float)(exp(-ki * rc) / (4.0 * kPi));
    }
    __syncthreads();
    const int cnt = min(kIncBlock, npts - c0);
    float fre = 0.f, fim = 0.f;
    for (int q = 0; q < cnt; ++q) {
      const float u = 2.f * fmaf(sd[0][q], dlx, fmaf(sd[1][q], dly, sd[2][q] * dlz)) + dl2;
      const float t = u * sinv[q];
      if (t > -0.5f) {
        const float rc = src_[q];
        const float dr = u / (rc * (1.f + sqrtf(1.f + t)));
        float sn, cs;
        sincosf(fmaf(krf, dr, sphi[q]), &sn, &cs);
        const float amp = samp[q] * (1.f - kif * dr) / (rc + dr);
        fre = fmaf(amp, cs, fre);
        fim = fmaf(amp, sn, fim);
      } else {  // near the tile (or NaN flag): direct FP64 distance and phase
        const double x = fma((double)ix, h, ox), y = fma((double)iy, h, oy), z = fma((double)iz, h, oz);
        const double dx = x - sp[0][q], dy = y - sp[1][q], dz = z - sp[2][q];
        const double r = fp64_norm(fma(dx, dx, fma(dy, dy, dz * dz)));
        const float2 ph = unit_phasor(kr * r);
        const float amp = expf(-(float)(ki * r)) * inv4pi / (float)r;
        fre = fmaf(amp, ph.x, fre);
        fim = fmaf(amp, ph.y, fim);
      }
    }
    are += fre;
    aim += fim;
    __syncthreads();
  }
  if (active) {
    const long long idx = ((long long)ix * ny + iy) * nz + iz;
    out[idx] = make_float2((float)(sre * are - sim * aim), (float)(sre * aim + sim * are));
  }
}

int grid_for(long long total, int threads) {
  long long b = (total + threads - 1) / threads;
  const long long cap = 152LL * 64;  // grid-stride beyond 64 CTAs per SM
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_kernel_lattice(float2* out, const int n[3], const int m[3], double h, double kr,
                                  double ki, cudaStream_t s) {
  const long long cube = (long long)m[0] * m[1] * m[2];
  cudaError_t e = cudaMemsetAsync(out, 0, (size_t)cube * sizeof(float2), s);
  if (e != cudaSuccess) return e;
  const long long total = (long long)n[0] * n[1] * n[2];
  lattice_kernel<<<grid_for(total, 256), 256, 0, s>>>(out, n[0], n[1], n[2], m[0], m[1], m[2], h, kr, ki);
  return cudaGetLastError();
}

cudaError_t launch_octant_extract(const float2* scr, float2* oct, const int m[3], const int o[3],
                                  const int* pos_x, const int* pos_y, const int* pos_z, cudaStream_t s) {
  const long long total = (long long)o[0] * o[1] * o[2];
  octant_kernel<<<grid_for(total, 256), 256, 0, s>>>(scr, oct, m[1], m[2], o[0], o[1], o[2], pos_x, pos_y,
                                                      pos_z);
  return cudaGetLastError();
}

cudaError_t launch_source_assemble(const float2* const* lower, int harmonic, float cn, float2* out,
                                   long long count, cudaStream_t s) {
  LowerPtrs lo;
  for (int i = 0; i < kMaxLower; ++i) lo.p[i] = i < harmonic - 1 ? lower[i] : nullptr;
  source_kernel<<<grid_for(count, 256), 256, 0, s>>>(lo, harmonic, cn, out, count);
  return cudaGetLastError();
}

// t = a + i b in source-voxel units, as fixed point (the host rounding of a and b).
AxisFix axis_fix(double a, double b, int n) {
  AxisFix m;
  m.A = llround(a * (double)(1LL << kFixBits));
  m.B = llround(b * (double)(1LL << kFixBits));
  m.n = n;
  return m;
}

// Tiled form when the source footprint of a 16 x 64 (y, z) target block fits the staging
// tile: (16 - 1) b_y + order + 2 <= kRsY and (64 - 1) b_z + order + 2 <= kRsZ source
// voxels (b = target spacing / source spacing), with a margin for rounding.
bool block_fits(const double b[3], int order) {
  const double extra = order + 2.0;
  return b[1] * (kRtY - 1) + extra <= kRsY && b[2] * (kRtZ - 1) + extra <= kRsZ;
}

// Source rows one 16 x 64 target block spans along y (z): at most ceil(15 b) (ceil(63 b))
// stencil starts apart, plus the stencil width and one for rounding.
int block_footprint(double b, int targets, int order) { return (int)std::ceil((targets - 1) * b) + order + 2; }

template <int ORD, int NS>
cudaError_t source_nested_launch(const NestedSrcDesc* d, float cn, float2* dst, const int nd[3], bool tiled,
                                 cudaStream_t s) {
  NestedSrcs<NS> q{};
  for (int m = 0; m < NS; ++m) {
    q.f[m] = d[m].f;
    q.sny[m] = d[m].n[1];
    q.snz[m] = d[m].n[2];
    for (int i = 0; i < 3; ++i) q.m[m][i] = axis_fix(d[m].a[i], d[m].b[i], d[m].n[i]);
  }
  if (tiled) {
    const dim3 grid((unsigned)((nd[2] + kRtZ - 1) / kRtZ), (unsigned)((nd[1] + kRtY - 1) / kRtY), (unsigned)nd[0]);
    int fy = 1, fz = 1;
    for (int m = 0; m < NS; ++m) {
      fy = std::max(fy, std::min(kRsY, block_footprint(d[m].b[1], kRtY, ORD)));
      fz = std::max(fz, std::min(kRsZ, block_footprint(d[m].b[2], kRtZ, ORD)));
    }
    size_t smem = nested_tiled_smem<ORD>(NS, fy, fz);
    // every source has two voxels or more on each axis: the linear kernel without
    // stencil-size tests
    bool lin = ORD == 1;
    for (int m = 0; m < NS; ++m) lin = lin && d[m].n[0] >= 2 && d[m].n[1] >= 2 && d[m].n[2] >= 2;
    if (lin) {
      smem += sizeof(LinStencil) * (size_t)NS * kStencilsPerSrc;
      static volatile int granted_lin[64] = {0};
      int dev = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e != cudaSuccess) return e;
      if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
      if (!granted_lin[dev]) {
        e = cudaFuncSetAttribute(source_nested_lin_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(nested_tiled_smem<1>(NS, kRsY, kRsZ) +
                                       sizeof(LinStencil) * (size_t)NS * kStencilsPerSrc));
        if (e != cudaSuccess) return e;
        granted_lin[dev] = 1;
      }
      source_nested_lin_kernel<NS><<<grid, 256, smem, s>>>(q, cn, dst, nd[1], nd[2], fy, fz);
      return cudaGetLastError();
    }
    // the largest size, once per device; a repeated grant is harmless
    static volatile int granted[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!granted[dev]) {
      e = cudaFuncSetAttribute(source_nested_tiled_kernel<ORD, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)nested_tiled_smem<ORD>(NS, kRsY, kRsZ));
      if (e != cudaSuccess) return e;
      granted[dev] = 1;
    }
    source_nested_tiled_kernel<ORD, NS><<<grid, 256, smem, s>>>(q, cn, dst, nd[1], nd[2], fy, fz);
  } else {
    const dim3 grid((unsigned)((nd[2] + 127) / 128), (unsigned)nd[1], (unsigned)nd[0]);
    source_nested_kernel<ORD, NS><<<grid, 128, 0, s>>>(q, cn, dst, nd[1], nd[2]);
  }
  return cudaGetLastError();
}

template <int ORD>
cudaError_t source_nested_order(const NestedSrcDesc* d, int ns, float cn, float2* dst, const int nd[3], bool tiled,
                                cudaStream_t s) {
  static_assert(kMaxLower == 8, "one instantiation per source count");
  switch (ns) {
    case 1: return source_nested_launch<ORD, 1>(d, cn, dst, nd, tiled, s);
    case 2: return source_nested_launch<ORD, 2>(d, cn, dst, nd, tiled, s);
    case 3: return source_nested_launch<ORD, 3>(d, cn, dst, nd, tiled, s);
    case 4: return source_nested_launch<ORD, 4>(d, cn, dst, nd, tiled, s);
    case 5: return source_nested_launch<ORD, 5>(d, cn, dst, nd, tiled, s);
    case 6: return source_nested_launch<ORD, 6>(d, cn, dst, nd, tiled, s);
    case 7: return source_nested_launch<ORD, 7>(d, cn, dst, nd, tiled, s);
    case 8: return source_nested_launch<ORD, 8>(d, cn, dst, nd, tiled, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_source_nested(const NestedSrcDesc* d, int ns, int order, float cn, float2* dst, const int nd[3],
                                 cudaStream_t s) {
  if (nd[1] > 65535 || nd[0] > 65535) return cudaErrorInvalidConfiguration;
  bool tiled = true;
  for (int m = 0; m < ns; ++m) tiled = tiled && block_fits(d[m].b, order);
  return order == 2 ? source_nested_order<2>(d, ns, cn, dst, nd, tiled, s)
                    : source_nested_order<1>(d, ns, cn, dst, nd, tiled, s);
}

cudaError_t launch_restrict(const float2* src, const int ns[3], float2* dst, const int nd[3],
                            const double a[3], const double b[3], int order, int zero_outside, cudaStream_t s) {
  if (nd[1] > 65535 || nd[0] > 65535) return cudaErrorInvalidConfiguration;
  AxisFix m[3];
  for (int i = 0; i < 3; ++i) m[i] = axis_fix(a[i], b[i], ns[i]);
  if (block_fits(b, order)) {
    const dim3 grid((unsigned)((nd[2] + kRtZ - 1) / kRtZ), (unsigned)((nd[1] + kRtY - 1) / kRtY), (unsigned)nd[0]);
    if (order == 2)
      restrict_tiled_kernel<2><<<grid, 256, 0, s>>>(src, ns[0], ns[1], ns[2], dst, nd[0], nd[1], nd[2], m[0], m[1],
                                                    m[2], zero_outside);
    else
      restrict_tiled_kernel<1><<<grid, 256, 0, s>>>(src, ns[0], ns[1], ns[2], dst, nd[0], nd[1], nd[2], m[0], m[1],
                                                    m[2], zero_outside);
    return cudaGetLastError();
  }
  const dim3 grid((unsigned)((nd[2] + 127) / 128), (unsigned)nd[1], (unsigned)nd[0]);
  if (order == 2)
    restrict_kernel<2><<<grid, 128, 0, s>>>(src, ns[0], ns[1], ns[2], dst, nd[0], nd[1], nd[2], m[0], m[1], m[2],
                                             zero_outside);
  else
    restrict_kernel<1><<<grid, 128, 0, s>>>(src, ns[0], ns[1], ns[2], dst, nd[0], nd[1], nd[2], m[0], m[1], m[2],
                                             zero_outside);
  return cudaGetLastError();
}

cudaError_t launch_incident(const double* pts, int npts, const int n[3], const double origin[3], double h,
                            double kr, double ki, double scale_re, double scale_im, float2* out,
                            cudaStream_t s) {
  const long long blocks = (long long)((n[0] + kIncTx - 1) / kIncTx) * ((n[1] + kIncTy - 1) / kIncTy) *
                           ((n[2] + kIncTz - 1) / kIncTz);
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  incident_kernel<<<(unsigned)blocks, kIncBlock, 0, s>>>(pts, npts, n[0], n[1], n[2], origin[0], origin[1],
                                                         origin[2], h, kr, ki, scale_re, scale_im, out);
  return cudaGetLastError();
}

cudaError_t launch_q0_box(const float2* f, const int n[3], double factor, void* scratch, cudaStream_t s) {
  unsigned long long* max_bits = static_cast<unsigned long long*>(scratch);
  int* box = reinterpret_cast<int*>(max_bits + 1);
  const long long count = (long long)n[0] * n[1] * n[2];
  q0_init_kernel<<<1, 32, 0, s>>>(max_bits, box);
  max_abs2_kernel<<<grid_for(count, 256), 256, 0, s>>>(f, count, max_bits);
  q0_box_kernel<<<grid_for(count, 256), 256, 0, s>>>(f, n[0], n[1], n[2], max_bits, factor, box);
  return cudaGetLastError();
}

}  // namespace vp
