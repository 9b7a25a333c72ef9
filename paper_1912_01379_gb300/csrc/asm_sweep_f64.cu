// FP64 chain state (the plain FP64 path): instantiations of the sweep kernel.
#include "asm_sweep.cuh"

namespace asmgb {

cudaError_t launch_sweeps_f64(const SweepParams<double> &p, int kv, cudaStream_t s)
{
    switch (kv) {
    case 1: return launch_sweep_kernel<double, 1>(p, s);
    case 2: return launch_sweep_kernel<double, 2>(p, s);
    case 4: return launch_sweep_kernel<double, 4>(p, s);
    case 8: return launch_sweep_kernel<double, 8>(p, s);
    case 16: return launch_sweep_kernel<double, 16>(p, s);
    case 32: return launch_sweep_kernel<double, 32>(p, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace asmgb
