// Two-level sweep kernels for line lengths 32, 64, 128, 192, 256 (part 0 of kFastSizes).
#include "sweeps2_launch.cuh"

namespace vp {

cudaError_t launch_col2_part0(const ColSweep& p, int dir, bool src, cudaStream_t s) {
  switch (p.ax.L) {
    case 32: return col2_dispatch<4, 8>(p, dir, src, s);
    case 64: return col2_dispatch<8, 8>(p, dir, src, s);
    case 128: return col2_dispatch<8, 16>(p, dir, src, s);
    case 192: return col2_dispatch<12, 16>(p, dir, src, s);
    case 256: return col2_dispatch<16, 16>(p, dir, src, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_line2_part0(const LineSweep& p, int mode, cudaStream_t s) {
  switch (p.ax.L) {
    case 32: return line2_dispatch<4, 8>(p, mode, s);
    case 64: return line2_dispatch<8, 8>(p, mode, s);
    case 128: return line2_dispatch<8, 16>(p, mode, s);
    case 192: return line2_dispatch<12, 16>(p, mode, s);
    case 256: return line2_dispatch<16, 16>(p, mode, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_col2_batch_part0(int L, const BatchParams<ColSweep>& bp, int total, int dir, bool src,
                                     cudaStream_t s) {
  switch (L) {
    case 32: return col2_batch_dispatch<4, 8>(bp, total, dir, src, s);
    case 64: return col2_batch_dispatch<8, 8>(bp, total, dir, src, s);
    case 128: return col2_batch_dispatch<8, 16>(bp, total, dir, src, s);
    case 192: return col2_batch_dispatch<12, 16>(bp, total, dir, src, s);
    case 256: return col2_batch_dispatch<16, 16>(bp, total, dir, src, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_line2_batch_part0(int L, const LineSweep& first, int ni_max,
                                      const BatchParams<LineSweep>& bp, int total, cudaStream_t s) {
  switch (L) {
    case 32: return line2_batch_dispatch<4, 8>(first, ni_max, bp, total, s);
    case 64: return line2_batch_dispatch<8, 8>(first, ni_max, bp, total, s);
    case 128: return line2_batch_dispatch<8, 16>(first, ni_max, bp, total, s);
    case 192: return line2_batch_dispatch<12, 16>(first, ni_max, bp, total, s);
    case 256: return line2_batch_dispatch<16, 16>(first, ni_max, bp, total, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace vp
