// mc_paths_lv.cu -- instantiations of the forward and reverse path kernels
// for the LvModel model, one per (precision, segment length K).
#include "mc_internal.h"
#include "mc_paths.cuh"

namespace mcaad {

template <typename Real>
static bool pick(int K, KernelPair *out) {
    switch (K) {
    case 25:
        out->fwd = (const void *)path_forward_kernel<LvModel<Real>, 25>;
        out->rev = (const void *)path_reverse_kernel<LvModel<Real>, 25>;
        return true;
    case 5:
        out->fwd = (const void *)path_forward_kernel<LvModel<Real>, 5>;
        out->rev = (const void *)path_reverse_kernel<LvModel<Real>, 5>;
        return true;
    case 1:
        out->fwd = (const void *)path_forward_kernel<LvModel<Real>, 1>;
        out->rev = (const void *)path_reverse_kernel<LvModel<Real>, 1>;
        return true;
    default:
        return false;
    }
}

bool lv_kernels(int precision, int K, KernelPair *out) {
    return precision == 0 ? pick<double>(K, out) : pick<float>(K, out);
}

}  // namespace mcaad
