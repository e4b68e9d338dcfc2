// kf_staged_p2r_f64.cu -- instantiations of the staged step kernel for
// p2r with the double-arithmetic variants (FP64 update, all-FP64).
#include "kf_step_staged.cuh"

namespace kf {
namespace staged {

int launch_staged_p2r_f64(int precision, const StepArgs &a, cudaStream_t s, int grid, int dev,
                          int ctas) {
  if (precision == KF_FP64_UPDATE) return launch_v<kP2r, kFP64Update>(a, s, grid, dev, ctas);
  return launch_v<kP2r, kFP64>(a, s, grid, dev, ctas);
}

}  // namespace staged
}  // namespace kf
