// FP64 chain state (the plain FP64 path): instantiations of the sweep kernel.
#include "asm_sweep.cuh"

namespace asmgb {

cudaError_t launch_sweeps_f64(const SweepParams<double> &p, int kv, int warps_per_cta, cudaStream_t s)
{
    switch (kv) {
    case 1: return launch_sweep_kernel<double, 1>(p, warps_per_cta, s);
    case 2: return launch_sweep_kernel<double, 2>(p, warps_per_cta, s);
    case 4: return launch_sweep_kernel<double, 4>(p, warps_per_cta, s);
    case 8: return launch_sweep_kernel<double, 8>(p, warps_per_cta, s);
    case 16: return launch_sweep_kernel<double, 16>(p, warps_per_cta, s);
    case 32: return launch_sweep_kernel<double, 32>(p, warps_per_cta, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace asmgb
