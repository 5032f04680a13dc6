// mc_paths_lv.cu -- instantiations of the forward and reverse path kernels
// (checkpoint/recompute, stored-normals and full-storage variants)
// for the LvModel model, one per (precision, segment length K, paths per thread).
#include "mc_internal.h"
#include "mc_paths.cuh"

namespace mcaad {

template <typename Real>
static bool pick(int K, int ppt, KernelPair *out) {
    if (K == 25 && ppt == 1) {
        set_kernels<LvModel<Real>, 25, 1>(out);
        return true;
    }
    if (K == 5 && ppt == 1) {
        set_kernels<LvModel<Real>, 5, 1>(out);
        return true;
    }
    if (K == 1 && ppt == 1) {
        set_kernels<LvModel<Real>, 1, 1>(out);
        return true;
    }
    if (K == 5 && ppt == 2) {
        set_kernels<LvModel<Real>, 5, 2>(out);
        return true;
    }
    if (K == 5 && ppt == 4) {
        set_kernels<LvModel<Real>, 5, 4>(out);
        return true;
    }
    return false;
}

bool lv_kernels(int precision, int K, int ppt, KernelPair *out) {
    return precision == 0 ? pick<double>(K, ppt, out) : pick<float>(K, ppt, out);
}

}  // namespace mcaad
