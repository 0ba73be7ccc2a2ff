// K_chi, persistent segmented form: the instantiations that take tissues of
// either single-cell model (Notch-Delta or promoter) in one launch.  The
// kernel template is in chi_seg.cuh.
#include "chi_seg.cuh"

namespace tsg {

ChiSegKernel chi_seg_kernel_gen(int H, bool pre, bool qb) {
  if (H == 8) {
    if (!pre) return k_chi_seg<8, false, false, 1, false>;
    return qb ? k_chi_seg<8, true, true, 1, false> : k_chi_seg<8, true, false, 1, false>;
  }
  if (H == 16) {
    if (!pre) return k_chi_seg<16, false, false, 1, false>;
    return qb ? k_chi_seg<16, true, true, 1, false> : k_chi_seg<16, true, false, 1, false>;
  }
  if (!pre) return k_chi_seg<32, false, false, 1, false>;
  return qb ? k_chi_seg<32, true, true, 1, false> : k_chi_seg<32, true, false, 1, false>;
}

}  // namespace tsg
