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

}  // namespace vp
