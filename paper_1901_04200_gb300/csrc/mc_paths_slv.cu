// mc_paths_slv.cu -- instantiations of the forward and reverse path kernels
// (checkpoint/recompute, stored-normals and full-storage variants)
// for the SlvModel model, one per (precision, segment length K, paths per thread).
#include "mc_internal.h"
#include "mc_paths.cuh"

namespace mcaad {

template <typename Real>
static bool pick(int K, int ppt, KernelPair *out) {
    if (K == 8 && ppt == 1) {
        set_kernels<SlvModel<Real>, 8, 1>(out);
        return true;
    }
    if (K == 4 && ppt == 1) {
        set_kernels<SlvModel<Real>, 4, 1>(out);
        return true;
    }
    if (K == 2 && ppt == 1) {
        set_kernels<SlvModel<Real>, 2, 1>(out);
        return true;
    }
    if (K == 1 && ppt == 1) {
        set_kernels<SlvModel<Real>, 1, 1>(out);
        return true;
    }
    return false;
}

bool slv_kernels(int precision, int K, int ppt, KernelPair *out) {
    return precision == 0 ? pick<double>(K, ppt, out) : pick<float>(K, ppt, out);
}

}  // namespace mcaad
