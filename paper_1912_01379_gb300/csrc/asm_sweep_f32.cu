// FP32 chain state (the mixed-precision path): instantiations of the sweep kernel.
#include "asm_sweep.cuh"

namespace asmgb {

cudaError_t launch_sweeps_f32(const SweepParams<float> &p, int kv, cudaStream_t s)
{
    switch (kv) {
    case 1: return launch_sweep_kernel<float, 1>(p, s);
    case 2: return launch_sweep_kernel<float, 2>(p, s);
    case 4: return launch_sweep_kernel<float, 4>(p, s);
    case 8: return launch_sweep_kernel<float, 8>(p, s);
    case 16: return launch_sweep_kernel<float, 16>(p, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace asmgb
