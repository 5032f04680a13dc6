// mc_paths_lv_fp64.cu -- the local-vol path kernels in FP64 (a translation unit of its own, so
// that the two precisions compile in parallel).
#include "mc_paths_lv.cuh"

namespace mcaad {

bool lv_kernels_fp64(int K, int ppt, KernelPair *out) { return lv_pick<double>(K, ppt, out); }

}  // namespace mcaad
