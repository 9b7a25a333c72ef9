// FP64 chain state: instantiations of the sweep kernel budgeted for 2 CTAs per SM (at most 128 registers per thread).
#include "asm_sweep.cuh"

namespace asmgb {

using Dispatch = SweepDispatch<double, 2, false, 1, 2, 4, 8, 16, 32>;

cudaError_t launch_sweeps_f64_m2(const SweepParams<double> &p0, const SweepParams<double> *probs,
                                  const WorkItem *items, RunCtrl *ctrl, const LaunchShape &shape, int kv,
                                  bool batch, int ctas, cudaStream_t s)
{
    return Dispatch::launch(p0, probs, items, ctrl, shape, kv, batch, ctas, s);
}

int sweep_ctas_per_sm_f64_m2(const LaunchShape &shape, int kv, bool batch)
{
    return Dispatch::per_sm(shape, kv, batch);
}

}  // namespace asmgb
