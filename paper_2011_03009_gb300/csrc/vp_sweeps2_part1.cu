// Two-level sweep kernels for line lengths 320, 384, 512, 640 (part 1 of kFastSizes).
#include "sweeps2_launch.cuh"

namespace vp {

cudaError_t launch_col2_part1(const ColSweep& p, int dir, bool src, cudaStream_t s) {
  switch (p.ax.L) {
    case 320: return col2_dispatch<16, 20>(p, dir, src, s);
    case 384: return col2_dispatch<16, 24>(p, dir, src, s);
    case 512: return col2_dispatch<16, 32>(p, dir, src, s);
    case 640: return col2_dispatch<20, 32>(p, dir, src, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_line2_part1(const LineSweep& p, int mode, cudaStream_t s) {
  switch (p.ax.L) {
    case 320: return line2_dispatch<16, 20>(p, mode, s);
    case 384: return line2_dispatch<16, 24>(p, mode, s);
    case 512: return line2_dispatch<16, 32>(p, mode, s);
    case 640: return line2_dispatch<20, 32>(p, mode, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_col2_batch_part1(int L, const BatchParams<ColSweep>& bp, int total, int dir, bool src,
                                     cudaStream_t s) {
  switch (L) {
    case 320: return col2_batch_dispatch<16, 20>(bp, total, dir, src, s);
    case 384: return col2_batch_dispatch<16, 24>(bp, total, dir, src, s);
    case 512: return col2_batch_dispatch<16, 32>(bp, total, dir, src, s);
    case 640: return col2_batch_dispatch<20, 32>(bp, total, dir, src, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_line2_batch_part1(int L, const LineSweep& first, int ni_max,
                                      const BatchParams<LineSweep>& bp, int total, cudaStream_t s) {
  switch (L) {
    case 320: return line2_batch_dispatch<16, 20>(first, ni_max, bp, total, s);
    case 384: return line2_batch_dispatch<16, 24>(first, ni_max, bp, total, s);
    case 512: return line2_batch_dispatch<16, 32>(first, ni_max, bp, total, s);
    case 640: return line2_batch_dispatch<20, 32>(first, ni_max, bp, total, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace vp
