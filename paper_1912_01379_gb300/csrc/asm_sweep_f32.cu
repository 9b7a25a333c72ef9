// FP32 chain state (the mixed-precision path): instantiations of the sweep kernel.
#include "asm_sweep.cuh"

namespace asmgb {

using DispatchF32 = SweepDispatch<float, 1, 2, 4, 8, 16>;

cudaError_t launch_sweeps_f32(const SweepParams<float> &p0, const SweepParams<float> *probs, const WorkItem *items,
                              RunCtrl *ctrl, const LaunchShape &shape, int kv, bool batch, int ctas, cudaStream_t s)
{
    return DispatchF32::launch(p0, probs, items, ctrl, shape, kv, batch, ctas, s);
}

int sweep_ctas_per_sm_f32(const LaunchShape &shape, int kv, bool batch)
{
    return DispatchF32::per_sm(shape, kv, batch);
}

}  // namespace asmgb
