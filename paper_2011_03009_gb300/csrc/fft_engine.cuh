// Shared-memory mixed-radix FFT engine for the volume-potential sweeps.
//
// A CTA holds a tile of kTileB = 16 independent lines of length L in shared memory,
// element (row i, line b) at tile[i * P + b].  Lane b of every half-warp owns line b,
// so each half-warp touches 16 consecutive complex values (128 B) per access: no
// bank conflicts for any radix or stride.
//
// Forward transforms are in-place decimation-in-frequency (DIF): natural-order input,
// output in mixed-radix digit-reversed order.  Inverse transforms are the matching
// decimation-in-time (DIT) passes run in reverse order with conjugate twiddles: they
// take the digit-reversed order and return natural order, scaled by L.  The
// convolution never needs the natural frequency order, so no permutation pass exists;
// the spectrum multiply looks frequencies up through per-axis position tables.
//
// DIF pass p with radix R over sub-transforms of length Lp (stride s = Lp / R):
//   for every block start b0 (multiple of Lp) and k in [0, s):
//     v[r] = x[b0 + k + r s];  y = DFT_R(v);  x[b0 + k + q s] = y[q] * w_Lp^(q k)
// with w_Lp = exp(-2 pi i / Lp) = tw[L / Lp].  The DIT pass is the conjugate transpose
// of the same step.
#pragma once

#include "vp_internal.cuh"

namespace vp {

// Debug builds (-DVP_DEBUG_CHECKS) check every shared- and global-memory index of the
// sweep kernels: an index outside [0, n) is recorded (first one wins) and replaced by
// 0, so the access stays in bounds.  Release builds compile the checks away.
#ifdef VP_DEBUG_CHECKS
static __device__ int g_vp_debug[8];  // per translation unit; read by vp_debug_checks
__device__ __forceinline__ long long vp_chk(long long i, long long n, int code, int x0 = 0, int x1 = 0,
                                            int x2 = 0, int x3 = 0) {
  if (i < 0 || i >= n) {
    if (atomicCAS(&g_vp_debug[0], 0, code) == 0) {
      g_vp_debug[1] = (int)i;
      g_vp_debug[2] = (int)n;
      g_vp_debug[3] = (int)blockIdx.x;
      g_vp_debug[4] = x0;
      g_vp_debug[5] = x1;
      g_vp_debug[6] = x2;
      g_vp_debug[7] = x3;
    }
    return 0;
  }
  return i;
}
#define VP_CHK(i, n, code) ((int)vp_chk((i), (n), (code)))
#define VP_CHKL(i, n, code) (vp_chk((i), (n), (code)))
#define VP_CHKX(i, n, code, a, b, c, d) ((int)vp_chk((i), (n), (code), (a), (b), (c), (d)))
#else
#define VP_CHK(i, n, code) (i)
#define VP_CHKL(i, n, code) (i)
#define VP_CHKX(i, n, code, a, b, c, d) (i)
#endif

// Complex add and subtract as one paired FP32 add (f32x2) each: per component the same
// round-to-nearest add as the scalar form, in half the instruction issues.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
// t + (-i) d and t - (-i) d (forward), t + i d and t - i d (inverse): the swapped
// operand suits scalar adds, so these two stay scalar.
template <bool INV>
__device__ __forceinline__ float2 add_mi(float2 t, float2 d) {
  return INV ? make_float2(t.x - d.y, t.y + d.x) : make_float2(t.x + d.y, t.y - d.x);
}
template <bool INV>
__device__ __forceinline__ float2 sub_mi(float2 t, float2 d) {
  return INV ? make_float2(t.x + d.y, t.y - d.x) : make_float2(t.x - d.y, t.y + d.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// multiply by the constant (cr, ci) or its conjugate
template <bool INV>
__device__ __forceinline__ float2 mul_const(float2 a, float cr, float ci) {
  const float c = INV ? -ci : ci;
  return make_float2(fmaf(a.x, cr, -a.y * c), fmaf(a.x, c, a.y * cr));
}

// ---- small DFTs: y[q] = sum_r v[r] exp(-+2 pi i r q / R), natural order in and out ----

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  float2 t0 = cadd(v0, v2), t1 = csub(v0, v2);
  float2 t2 = cadd(v1, v3), d = csub(v1, v3);
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = add_mi<INV>(t1, d);
  v3 = sub_mi<INV>(t1, d);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
  const float c = -0.5f, s = 0.86602540378443865f;  // cos(2pi/3), sin(2pi/3)
  float2 t = cadd(v[1], v[2]);
  float2 d = csub(v[1], v[2]);
  float2 m = make_float2(fmaf(c, t.x, v[0].x), fmaf(c, t.y, v[0].y));
  v[0] = cadd(v[0], t);
  float2 sd = cscale(d, s);
  v[1] = add_mi<INV>(m, sd);
  v[2] = sub_mi<INV>(m, sd);
}

template <bool INV>
__device__ __forceinline__ void dft5(float2* v) {
  const float c1 = 0.30901699437494742f;   // cos(2pi/5)
  const float c2 = -0.80901699437494742f;  // cos(4pi/5)
  const float s1 = 0.95105651629515357f;   // sin(2pi/5)
  const float s2 = 0.58778525229247313f;   // sin(4pi/5)
  float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
  float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
  float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
  float2 b1 = make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
  float2 b2 = make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
  v[0] = cadd(v[0], cadd(t1, t2));
  v[1] = add_mi<INV>(a1, b1);
  v[4] = sub_mi<INV>(a1, b1);
  v[2] = add_mi<INV>(a2, b2);
  v[3] = sub_mi<INV>(a2, b2);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  const float c = 0.70710678118654752f;
  // radix-2 decimation in time over two 4-point DFTs
  dft4<INV>(v[0], v[2], v[4], v[6]);
  dft4<INV>(v[1], v[3], v[5], v[7]);
  float2 o1 = mul_const<INV>(v[3], c, -c);
  float2 o2 = v[5];  // times -i (forward) or i (inverse), taken by add_mi / sub_mi
  float2 o3 = mul_const<INV>(v[7], -c, -c);
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = add_mi<INV>(e2, o2);
  v[6] = sub_mi<INV>(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  const float c1 = 0.92387953251128674f;  // cos(pi/8)
  const float s1 = 0.38268343236508977f;  // sin(pi/8)
  const float c = 0.70710678118654752f;
  // 4 x 4: first DFT4 over r1 for each r2 (elements r2 + 4 r1)
#pragma unroll
  for (int r2 = 0; r2 < 4; ++r2) dft4<INV>(v[r2], v[r2 + 4], v[r2 + 8], v[r2 + 12]);
  // now v[r2 + 4 q1] = Z_{r2}[q1]; twiddle by w16^(r2 q1)
  v[5] = mul_const<INV>(v[5], c1, -s1);    // r2=1,q1=1: w^1
  v[9] = mul_const<INV>(v[9], c, -c);      // r2=1,q1=2: w^2
  v[13] = mul_const<INV>(v[13], s1, -c1);  // r2=1,q1=3: w^3
  v[6] = mul_const<INV>(v[6], c, -c);      // r2=2,q1=1: w^2
  v[10] = mul_mi<INV>(v[10]);              // r2=2,q1=2: w^4
  v[14] = mul_const<INV>(v[14], -c, -c);   // r2=2,q1=3: w^6
  v[7] = mul_const<INV>(v[7], s1, -c1);    // r2=3,q1=1: w^3
  v[11] = mul_const<INV>(v[11], -c, -c);   // r2=3,q1=2: w^6
  v[15] = mul_const<INV>(v[15], -c1, s1);  // r2=3,q1=3: w^9
  // second DFT4 over r2 for each q1: y[q1 + 4 q2]
  float2 t[16];
#pragma unroll
  for (int q1 = 0; q1 < 4; ++q1) {
    float2 a = v[4 * q1 + 0], b = v[4 * q1 + 1], d = v[4 * q1 + 2], e = v[4 * q1 + 3];
    dft4<INV>(a, b, d, e);
    t[q1 + 0] = a;
    t[q1 + 4] = b;
    t[q1 + 8] = d;
    t[q1 + 12] = e;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = t[i];
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 5) dft5<INV>(v);
  else if constexpr (R == 8) dft8<INV>(v);
  else if constexpr (R == 16) dft16<INV>(v);
}

// ---- asynchronous global -> shared copies (cp.async, all in flight at once) ---------

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 8 : 0;  // 0: zero-fill, nothing read
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ---- bulk asynchronous copies (one instruction per contiguous run) and mbarriers ----
// A bulk copy moves `bytes` (a multiple of 16) from a 16-byte aligned global address to
// a 16-byte aligned shared address and reports its bytes to the mbarrier at `bar`
// (complete_tx).  A phase of the mbarrier completes when its expected arrivals have
// arrived and every byte announced by arrive.expect_tx has landed.

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(arrivals) : "memory");
}
// makes the initialised mbarriers visible to the bulk-copy unit
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// one arrival that also announces `bytes` still to land in the current phase
__device__ __forceinline__ void mbar_arrive_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for the phase of parity `parity` on two mbarriers: false once about
// `limit` SM clock cycles have passed without both completing.
__device__ __forceinline__ bool mbar_wait2(unsigned bar0, unsigned bar1, unsigned parity, long long limit) {
  const long long t0 = clock64();
  bool d0 = false, d1 = false;
  while (true) {
    if (!d0) d0 = mbar_test(bar0, parity);
    if (!d1) d1 = mbar_test(bar1, parity);
    if (d0 && d1) return true;
    if (clock64() - t0 > limit) return false;
  }
}
// about one second at the GB300's 2.07 GHz SM clock
constexpr long long kWaitCycles = 1LL << 31;

// u / s for 0 <= u < 2^16 and 1 < s < 2^16 with magic = floor(2^32 / s) + 1: the
// high word of u * magic is u/s + u e / 2^32 with 0 < e <= 1, exact below 2^16.
// magic = 0 encodes s = 1.
__device__ __forceinline__ int fast_div(int u, unsigned magic) {
  return magic == 0u ? u : (int)__umulhi((unsigned)u, magic);
}

// ---- passes over a shared-memory tile -----------------------------------------------
// tw points to the twiddle table (shared or global memory).  Element (row, line b) of
// the tile sits at row * P + b, or with SW at row * 16 + (b ^ (row & 15)) (P = 16): the
// XOR swizzle keeps both row-wise accesses (16 lines of one row) and column-wise
// accesses (16 consecutive rows of one line) free of bank conflicts.
template <int P, bool SW>
__device__ __forceinline__ int tix(int row, int b) {
  return SW ? row * 16 + (b ^ (row & 15)) : row * P + b;
}

// Forward DIF pass.  Rows >= rows_nz are treated as zero without being read.
template <int R, int P, bool SW>
__device__ __forceinline__ void dif_pass(float2* tile, int L, int Lp, unsigned magic,
                                         const float2* tw, int rows_nz) {
  const int s = Lp / R;
  const int tws = L / Lp;
  const int nb = (L / R) * kTileB;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    const int b = t & (kTileB - 1);
    const int u = t >> 4;
    const int blk = fast_div(u, magic);
    const int k = u - blk * s;
    const int base = blk * Lp + k;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = base + r * s;
      v[r] = row < rows_nz ? tile[VP_CHKX((tix<P, SW>(row, b)), L * 16, 101, u, Lp, (int)magic, blk)]
                           : make_float2(0.f, 0.f);
    }
    dft<R, false>(v);
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = cmul(v[q], tw[VP_CHK(q * k * tws, L, 102)]);
#pragma unroll
    for (int q = 0; q < R; ++q) tile[VP_CHK((tix<P, SW>(base + q * s, b)), L * 16, 103)] = v[q];
  }
}

// Inverse DIT pass (conjugate transpose of dif_pass).
template <int R, int P, bool SW>
__device__ __forceinline__ void dit_pass(float2* tile, int L, int Lp, unsigned magic,
                                         const float2* tw) {
  const int s = Lp / R;
  const int tws = L / Lp;
  const int nb = (L / R) * kTileB;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    const int b = t & (kTileB - 1);
    const int u = t >> 4;
    const int blk = fast_div(u, magic);
    const int k = u - blk * s;
    const int base = blk * Lp + k;
    float2 v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = tile[VP_CHK((tix<P, SW>(base + q * s, b)), L * 16, 104)];
#pragma unroll
    for (int q = 1; q < R; ++q) v[q] = cmulc(v[q], tw[VP_CHK(q * k * tws, L, 105)]);
    dft<R, true>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) tile[VP_CHK((tix<P, SW>(base + r * s, b)), L * 16, 106)] = v[r];
  }
}

template <int P, bool SW>
__device__ __forceinline__ void dif_pass_rt(const AxisDesc& ax, int p, float2* tile, const float2* tw,
                                            int rows_nz) {
  const int L = ax.L, Lp = ax.lp[p];
  const unsigned mg = ax.magic[p];
  switch (ax.radix[p]) {
    case 16: dif_pass<16, P, SW>(tile, L, Lp, mg, tw, rows_nz); break;
    case 8: dif_pass<8, P, SW>(tile, L, Lp, mg, tw, rows_nz); break;
    case 4: dif_pass<4, P, SW>(tile, L, Lp, mg, tw, rows_nz); break;
    case 2: dif_pass<2, P, SW>(tile, L, Lp, mg, tw, rows_nz); break;
    case 5: dif_pass<5, P, SW>(tile, L, Lp, mg, tw, rows_nz); break;
    case 3: dif_pass<3, P, SW>(tile, L, Lp, mg, tw, rows_nz); break;
    default: break;
  }
}

template <int P, bool SW>
__device__ __forceinline__ void dit_pass_rt(const AxisDesc& ax, int p, float2* tile, const float2* tw) {
  const int L = ax.L, Lp = ax.lp[p];
  const unsigned mg = ax.magic[p];
  switch (ax.radix[p]) {
    case 16: dit_pass<16, P, SW>(tile, L, Lp, mg, tw); break;
    case 8: dit_pass<8, P, SW>(tile, L, Lp, mg, tw); break;
    case 4: dit_pass<4, P, SW>(tile, L, Lp, mg, tw); break;
    case 2: dit_pass<2, P, SW>(tile, L, Lp, mg, tw); break;
    case 5: dit_pass<5, P, SW>(tile, L, Lp, mg, tw); break;
    case 3: dit_pass<3, P, SW>(tile, L, Lp, mg, tw); break;
    default: break;
  }
}

// Full forward transform of the tile (DIF, digit-reversed output).
template <int P, bool SW>
__device__ __forceinline__ void tile_forward(float2* tile, const AxisDesc& ax, const float2* tw, int rows_nz) {
  for (int p = 0; p < ax.npass; ++p) {
    dif_pass_rt<P, SW>(ax, p, tile, tw, p == 0 ? rows_nz : ax.L);
    __syncthreads();
  }
}

// Full inverse transform of the tile (DIT, digit-reversed input, natural output, x L).
template <int P, bool SW>
__device__ __forceinline__ void tile_inverse(float2* tile, const AxisDesc& ax, const float2* tw) {
  for (int p = ax.npass - 1; p >= 0; --p) {
    dit_pass_rt<P, SW>(ax, p, tile, tw);
    __syncthreads();
  }
}

// Stage the axis twiddle table into shared memory (cp.async; caller waits).
__device__ __forceinline__ void stage_twiddles(float2* tw_s, const AxisDesc& ax) {
  for (int i = threadIdx.x; i < ax.L; i += blockDim.x) cp_async8(&tw_s[VP_CHK(i, ax.L, 107)], &ax.tw[i], true);
}

}  // namespace vp
