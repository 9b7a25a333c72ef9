// FP64 chain state: instantiations of the sweep kernel.
#include "asm_sweep.cuh"

namespace asmgb {

using DispatchF64 = SweepDispatch<double, 1, 2, 4, 8, 16, 32>;

cudaError_t launch_sweeps_f64(const SweepParams<double> &p0, const SweepParams<double> *probs, const WorkItem *items,
                              RunCtrl *ctrl, const LaunchShape &shape, int kv, bool batch, int ctas, cudaStream_t s)
{
    return DispatchF64::launch(p0, probs, items, ctrl, shape, kv, batch, ctas, s);
}

int sweep_ctas_per_sm_f64(const LaunchShape &shape, int kv, bool batch)
{
    return DispatchF64::per_sm(shape, kv, batch);
}

}  // namespace asmgb
