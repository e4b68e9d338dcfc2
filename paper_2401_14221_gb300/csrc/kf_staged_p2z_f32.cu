// kf_staged_p2z_f32.cu -- instantiations of the staged step kernel for
// p2z with the float-arithmetic variants (FP32, Joseph, adaptive,
// double-float update).
#include "kf_step_staged.cuh"

namespace kf {
namespace staged {

int launch_staged_p2z_f32(int precision, const StepArgs &a, cudaStream_t s, int grid, int dev,
                          int ctas) {
  switch (precision) {
    case KF_FP32: return launch_v<kP2z, kFP32>(a, s, grid, dev, ctas);
    case KF_JOSEPH: return launch_v<kP2z, kJoseph>(a, s, grid, dev, ctas);
    case KF_DF_UPDATE: return launch_v<kP2z, kDFUpdate>(a, s, grid, dev, ctas);
    default: return launch_v<kP2z, kAdaptive>(a, s, grid, dev, ctas);
  }
}

}  // namespace staged
}  // namespace kf
