// mc_paths_lv.cu -- instantiations of the forward and reverse path kernels
// (checkpoint/recompute, stored-normals, full-storage and stored-states variants)
// for the LvModel model in FP32, and the local-vol kernel lookup.
#include "mc_paths_lv.cuh"

namespace mcaad {

bool lv_kernels(int precision, int K, int ppt, KernelPair *out) {
    return precision == 0 ? lv_kernels_fp64(K, ppt, out) : lv_pick<float>(K, ppt, out);
}

}  // namespace mcaad
