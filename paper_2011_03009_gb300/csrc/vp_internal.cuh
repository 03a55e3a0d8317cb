// Internal declarations shared by the translation units of libvp.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vp.h"

namespace vp {

constexpr int kMaxPass = 8;      // radix passes per axis
constexpr int kMaxLower = 8;     // lower harmonics fed to one source assembly
constexpr int kTileB = 16;       // lines per CTA tile in every FFT sweep
constexpr int kThreads = 256;    // threads per CTA of the FFT sweeps
constexpr int kMaxL = 1536;      // longest FFT line the shared-memory tile holds

// Line lengths with a compile-time two-level register engine (L = A * B, see
// sweeps2.cuh), split into three groups compiled as separate translation units.
struct FastSize {
  int L, A, B, part;
};
constexpr FastSize kFastSizes[] = {
    {32, 4, 8, 0},     {64, 8, 8, 0},     {128, 8, 16, 0},   {192, 12, 16, 0},  {256, 16, 16, 0},
    {320, 16, 20, 1},  {384, 16, 24, 1},  {512, 16, 32, 1},  {640, 20, 32, 1},  {768, 24, 32, 2},
    {864, 27, 32, 2},  {1024, 32, 32, 2}, {1200, 30, 40, 2}, {1280, 32, 40, 2},
};
constexpr int kNumFastSizes = sizeof(kFastSizes) / sizeof(kFastSizes[0]);

// One FFT axis: its length, radix schedule and twiddle table.
struct AxisDesc {
  int L;
  int fast;  // 1: two-level register engine (natural order), 0: shared-memory radix passes
  int npass;
  int radix[kMaxPass];
  int lp[kMaxPass];        // sub-transform length entering pass p (L, L/R0, L/(R0 R1), ...)
  unsigned magic[kMaxPass];  // floor(2^32 / s_p) + 1 for s_p = lp[p] / radix[p] > 1; 0 when s_p = 1
  const float2* tw;        // L entries, exp(-2 pi i t / L), built in FP64 on the host
};

// Column sweep: FFT along a strided axis, batched over 16 contiguous columns.
// Element (outer o, row i, column c) lives at base + o*os + i*rs + c; an input read in
// groups of kRowGroup rows (the y forward sweep over the grouped layout of the x sweep's
// output) adds (i / kRowGroup) * in_rs_extra.
struct ColSweep {
  const float2* in;
  float2* out;
  long long in_os, in_rs, out_os, out_rs;
  long long in_rs_extra;  // 0 for a plain strided input
  int C;          // columns (contiguous extent)
  int n_outer;
  int rows_in;    // rows read (rows beyond are zero padding)
  int rows_out;   // rows written
  long long in_elems, out_elems;  // buffer sizes (elements), for debug-build bounds checks
  float scale;
  AxisDesc ax;
  // source-assembly prologue (first forward sweep fused with Eq. 2.6)
  int harmonic;   // n; the prologue forms sum_{m=1}^{n-1} p_m p_{n-m}
  float cn;       // C_n
  const float2* lower[kMaxLower];
};

// Line sweep: FFT along the contiguous axis, 16 lines per CTA.
// Convolution mode: tile t holds the lines listed in tiles[20 t .. 20 t + 15] (line
// index or -1) and multiplies lines 4g..4g+3 by octant line tiles[20 t + 16 + g] of the
// kernel spectrum; each group of four lines are the mirror images (f_x, M_x - f_x) x
// (f_y, M_y - f_y) of one octant line.  Forward-only mode: tile t holds lines 16t..16t+15.
struct LineSweep {
  float2* data;
  long long nlines;     // forward-only mode: number of lines; convolution mode: number of tiles
  long long ld;   // distance between consecutive lines (elements)
  int n_in;       // elements read per line (rest is zero padding up to L)
  int n_out;      // elements written per line
  long long data_elems;  // buffer size (elements), for debug-build bounds checks
  AxisDesc ax;
  // spectrum multiply (convolution mode)
  const float2* khat;   // octant (Ox, Oy, Oz)
  int Oz;
  const int* tiles;     // 20 ints per tile
  const int* fold_z;    // z position -> folded frequency
  int zform;            // pipelined z-sweep form (VP_ZFORM_*; 0 = chosen by occupancy)
  int staging;          // 0: bulk copies where the 4-line forms allow them, 1: cp.async only
  int expire_waits;     // test hook: the bulk-staged z sweep issues no first copies
  int* status;          // device word; bit 0 set when a bounded wait expired
};

enum SweepDir { kForward = 0, kInverse = 1 };
// Rows per group of the grouped layout: a power of two that divides every second factor
// B of the two-level engine, so that (B a + b) / kRowGroup = (B / kRowGroup) a + b / kRowGroup
// and the group term of an unrolled column read is a constant stride.
constexpr int kRowGroup = 4;
enum LineMode { kConv = 0, kForwardOnly = 1 };

// Launchers (vp_sweeps.cu).  Return a cudaError_t.
cudaError_t launch_col_sweep(const ColSweep& p, int dir, bool source_prologue, cudaStream_t s);
cudaError_t launch_line_sweep(const LineSweep& p, int mode, cudaStream_t s);
// Two-level engine (vp_sweeps2_part*.cu); cudaErrorNotSupported if L is not in the part.
cudaError_t launch_col2_part0(const ColSweep& p, int dir, bool src, cudaStream_t s);
cudaError_t launch_col2_part1(const ColSweep& p, int dir, bool src, cudaStream_t s);
cudaError_t launch_col2_part2(const ColSweep& p, int dir, bool src, cudaStream_t s);
cudaError_t launch_line2_part0(const LineSweep& p, int mode, cudaStream_t s);
cudaError_t launch_line2_part1(const LineSweep& p, int mode, cudaStream_t s);
cudaError_t launch_line2_part2(const LineSweep& p, int mode, cudaStream_t s);
// Batched two-level sweeps: the parameters of up to kMaxBatch plans (and the first
// CTA of each, offsets[i]) in the kernel parameter block.
constexpr int kMaxBatch = 64;
template <typename T>
struct BatchParams {
  int count;
  int offsets[kMaxBatch + 1];
  T item[kMaxBatch];
};
cudaError_t launch_col2_batch_part0(int L, const BatchParams<ColSweep>& bp, int total, int dir, bool src,
                                    cudaStream_t s);
cudaError_t launch_col2_batch_part1(int L, const BatchParams<ColSweep>& bp, int total, int dir, bool src,
                                    cudaStream_t s);
cudaError_t launch_col2_batch_part2(int L, const BatchParams<ColSweep>& bp, int total, int dir, bool src,
                                    cudaStream_t s);
cudaError_t launch_line2_batch_part0(int L, const LineSweep& first, int ni_max, const BatchParams<LineSweep>& bp,
                                     int total, cudaStream_t s);
cudaError_t launch_line2_batch_part1(int L, const LineSweep& first, int ni_max, const BatchParams<LineSweep>& bp,
                                     int total, cudaStream_t s);
cudaError_t launch_line2_batch_part2(int L, const LineSweep& first, int ni_max, const BatchParams<LineSweep>& bp,
                                     int total, cudaStream_t s);
// Dispatch on p.ax.fast: two-level engine or shared-memory radix passes.
cudaError_t launch_col_any(const ColSweep& p, int dir, bool src, cudaStream_t s);
cudaError_t launch_line_any(const LineSweep& p, int mode, cudaStream_t s);

// Other kernels (vp_kernels.cu).
cudaError_t launch_kernel_lattice(float2* out, const int n[3], const int m[3], double h,
                                  double kr, double ki, cudaStream_t s);
cudaError_t launch_octant_extract(const float2* scr, float2* oct, const int m[3], const int o[3],
                                  const int* pos_x, const int* pos_y, const int* pos_z,
                                  cudaStream_t s);
cudaError_t launch_source_assemble(const float2* const* lower, int harmonic, float cn, float2* out,
                                   long long count, cudaStream_t s);
// One lower harmonic of a nested source: field f on a grid of n voxels, and the target
// axis maps t = a + i b in its voxel units (as vp_restrict_to_nested_box forms them).
struct NestedSrcDesc {
  const float2* f;
  int n[3];
  double a[3], b[3];
};
// f_n of harmonic ns + 1 on the nd grid from the ns lower harmonics, each restricted
// (order 1 linear, 2 quadratic) inside the kernel.
cudaError_t launch_source_nested(const NestedSrcDesc* d, int ns, int order, float cn, float2* dst, const int nd[3],
                                 cudaStream_t s);
cudaError_t launch_restrict(const float2* src, const int ns[3], float2* dst, const int nd[3],
                            const double a[3], const double b[3], int order, int zero_outside,
                            cudaStream_t s);
// field vector operations and the Eq. 2.5 source (vp_vec.cu)
cudaError_t launch_axpby(long long n, float2 a, const float2* x, float2 b, const float2* y, float2* out,
                         cudaStream_t s);
cudaError_t launch_mul(long long n, const float2* x, const float2* y, float2* out, cudaStream_t s);
cudaError_t launch_dot(long long n, const float2* x, const float2* y, int conj_x, double* acc, cudaStream_t s);
cudaError_t launch_source_full(const float2* const* fields, int n, int nh, float cn, float2* out, long long count,
                               cudaStream_t s);
// scratch: 8-byte max |f|^2 followed by int box[6]
cudaError_t launch_q0_box(const float2* f, const int n[3], double factor, void* scratch, cudaStream_t s);
cudaError_t launch_incident(const double* pts, int npts, const int n[3], const double origin[3],
                            double h, double kr, double ki, double scale_re, double scale_im,
                            float2* out, cudaStream_t s);

}  // namespace vp
