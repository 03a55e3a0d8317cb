// Two-level sweep kernels for line lengths 768, 864, 1024, 1200, 1280 (part 2 of kFastSizes).
#include "sweeps2_launch.cuh"

namespace vp {

cudaError_t launch_col2_part2(const ColSweep& p, int dir, bool src, cudaStream_t s) {
  switch (p.ax.L) {
    case 768: return col2_dispatch<24, 32>(p, dir, src, s);
    case 864: return col2_dispatch<27, 32>(p, dir, src, s);
    case 1024: return col2_dispatch<32, 32>(p, dir, src, s);
    case 1200: return col2_dispatch<30, 40>(p, dir, src, s);
    case 1280: return col2_dispatch<32, 40>(p, dir, src, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_line2_part2(const LineSweep& p, int mode, cudaStream_t s) {
  switch (p.ax.L) {
    case 768: return line2_dispatch<24, 32>(p, mode, s);
    case 864: return line2_dispatch<27, 32>(p, mode, s);
    case 1024: return line2_dispatch<32, 32>(p, mode, s);
    case 1200: return line2_dispatch<30, 40>(p, mode, s);
    case 1280: return line2_dispatch<32, 40>(p, mode, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_col2_batch_part2(int L, const BatchParams<ColSweep>& bp, int total, int dir, bool src,
                                     cudaStream_t s) {
  switch (L) {
    case 768: return col2_batch_dispatch<24, 32>(bp, total, dir, src, s);
    case 864: return col2_batch_dispatch<27, 32>(bp, total, dir, src, s);
    case 1024: return col2_batch_dispatch<32, 32>(bp, total, dir, src, s);
    case 1200: return col2_batch_dispatch<30, 40>(bp, total, dir, src, s);
    case 1280: return col2_batch_dispatch<32, 40>(bp, total, dir, src, s);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_line2_batch_part2(int L, const LineSweep& first, int ni_max,
                                      const BatchParams<LineSweep>& bp, int total, cudaStream_t s) {
  switch (L) {
    case 768: return line2_batch_dispatch<24, 32>(first, ni_max, bp, total, s);
    case 864: return line2_batch_dispatch<27, 32>(first, ni_max, bp, total, s);
    case 1024: return line2_batch_dispatch<32, 32>(first, ni_max, bp, total, s);
    case 1200: return line2_batch_dispatch<30, 40>(first, ni_max, bp, total, s);
    case 1280: return line2_batch_dispatch<32, 40>(first, ni_max, bp, total, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace vp
