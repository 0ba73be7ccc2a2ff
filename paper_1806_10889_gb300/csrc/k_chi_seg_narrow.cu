// K_chi, persistent segmented form: the 16-bit-count instantiations for cells
// of more than 256 voxels (Notch-Delta model; both shared-memory layouts).  The kernel
// template is in chi_seg.cuh; the launcher in k_chi_seg.cu runs the cells
// these give up on (a count above 65535) through the 32-bit instantiations.
#include "chi_seg.cuh"

namespace tsg {

ChiSegKernel chi_seg_kernel_narrow(int H, bool pre, bool qb) {
  // V > 256 makes B > H for 8 and 16 lanes; 32 lanes cover V <= 1024 with B <= H.
  // The recompute layout: 32 lanes, or 16 lanes with up to four sub-blocks per block.
  if (!pre) {
    if (H == 32) return qb ? nullptr : k_chi_seg<32, false, false, 0, true>;
    if (H == 16) return qb ? k_chi_seg<16, false, true, 0, true> : nullptr;
    return nullptr;
  }
  if (H == 8) return qb ? k_chi_seg<8, true, true, 0, true> : nullptr;
  if (H == 16) return qb ? k_chi_seg<16, true, true, 0, true> : nullptr;
  return qb ? nullptr : k_chi_seg<32, true, false, 0, true>;
}

}  // namespace tsg
