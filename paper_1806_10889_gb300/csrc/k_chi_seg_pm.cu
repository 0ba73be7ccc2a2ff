// K_chi, persistent segmented form: the instantiations for launches whose
// tissues all run the promoter model (the per-cell model test folded away).
// The kernel template is in chi_seg.cuh.
#include "chi_seg.cuh"

namespace tsg {

ChiSegKernel chi_seg_kernel_pm(int H, bool pre, bool qb) {
  if (H == 8) {
    if (!pre) return k_chi_seg<8, false, false, 2, false>;
    return qb ? k_chi_seg<8, true, true, 2, false> : k_chi_seg<8, true, false, 2, false>;
  }
  if (H == 16) {
    if (!pre) return k_chi_seg<16, false, false, 2, false>;
    return qb ? k_chi_seg<16, true, true, 2, false> : k_chi_seg<16, true, false, 2, false>;
  }
  if (!pre) return k_chi_seg<32, false, false, 2, false>;
  return qb ? k_chi_seg<32, true, true, 2, false> : k_chi_seg<32, true, false, 2, false>;
}

}  // namespace tsg
