// mc_paths_gbm.cu -- instantiations of the forward and reverse path kernels
// for the GbmModel model, one per (precision, segment length K).
#include "mc_internal.h"
#include "mc_paths.cuh"

namespace mcaad {

template <typename Real>
static bool pick(int K, KernelPair *out) {
    switch (K) {
    case 16:
        out->fwd = (const void *)path_forward_kernel<GbmModel<Real>, 16>;
        out->rev = (const void *)path_reverse_kernel<GbmModel<Real>, 16>;
        return true;
    case 8:
        out->fwd = (const void *)path_forward_kernel<GbmModel<Real>, 8>;
        out->rev = (const void *)path_reverse_kernel<GbmModel<Real>, 8>;
        return true;
    case 4:
        out->fwd = (const void *)path_forward_kernel<GbmModel<Real>, 4>;
        out->rev = (const void *)path_reverse_kernel<GbmModel<Real>, 4>;
        return true;
    case 2:
        out->fwd = (const void *)path_forward_kernel<GbmModel<Real>, 2>;
        out->rev = (const void *)path_reverse_kernel<GbmModel<Real>, 2>;
        return true;
    case 1:
        out->fwd = (const void *)path_forward_kernel<GbmModel<Real>, 1>;
        out->rev = (const void *)path_reverse_kernel<GbmModel<Real>, 1>;
        return true;
    default:
        return false;
    }
}

bool gbm_kernels(int precision, int K, KernelPair *out) {
    return precision == 0 ? pick<double>(K, out) : pick<float>(K, out);
}

}  // namespace mcaad
