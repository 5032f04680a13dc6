// mc_paths_lv.cuh -- the local-vol kernel table: which (segment length K, paths per thread)
// are instantiated, for one precision per translation unit (mc_paths_lv.cu: FP32,
// mc_paths_lv_fp64.cu: FP64, compiled in parallel).
#pragma once
#include "mc_internal.h"
#include "mc_paths.cuh"

namespace mcaad {

template <typename Real>
bool lv_pick(int K, int ppt, KernelPair *out) {
    if (K == 25 && ppt == 1) {
        set_kernels<LvModel<Real>, 25, 1>(out);
        return true;
    }
    if constexpr (sizeof(Real) == 4) {  // the 25-step recompute with two paths per thread: FP32 only
        if (K == 25 && ppt == 2) {
            set_kernels<LvModel<Real>, 25, 2>(out);
            return true;
        }
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

}  // namespace mcaad
