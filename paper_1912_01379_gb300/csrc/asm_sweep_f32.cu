// FP32 chain state (the mixed-precision path): instantiations of the sweep kernel.
#include "asm_sweep.cuh"

namespace asmgb {

cudaError_t launch_sweeps_f32(const SweepParams<float> &p, int kv, int warps_per_cta, cudaStream_t s)
{
    switch (kv) {
    case 1: return launch_sweep_kernel<float, 1>(p, warps_per_cta, s);
    case 2: return launch_sweep_kernel<float, 2>(p, warps_per_cta, s);
    case 4: return launch_sweep_kernel<float, 4>(p, warps_per_cta, s);
    case 8: return launch_sweep_kernel<float, 8>(p, warps_per_cta, s);
    case 16: return launch_sweep_kernel<float, 16>(p, warps_per_cta, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace asmgb
