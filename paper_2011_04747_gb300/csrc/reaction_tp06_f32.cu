// Step A, ten Tusscher-Panfilov 2006, float state.
#include "reaction_impl.cuh"

namespace daeti {

template <>
void launch_tp06<float, false>(const DevState& s, const ModelArgs& m, double dt, StepRef step, bool lists, int par,
                          int src, bool fused, const DiffOp& op, const ReactTuning& tune, cudaStream_t st) {
    const ReactArgs<float> a = react_args<float, false>(s, m, dt, step, lists, par, src, fused, tune);
    const int block = react_block(tune);
    const int grid = (int)((s.n + block - 1) / block);
    if (grid == 0) return;
    if (tune.min_blocks >= 10) launch_react_dims<float, M_TP06, false, 10>(a, s, op, fused, grid, block, tune, st);
    else if (tune.min_blocks <= 6) launch_react_dims<float, M_TP06, false, 6>(a, s, op, fused, grid, block, tune, st);
    else launch_react_dims<float, M_TP06, false, 8>(a, s, op, fused, grid, block, tune, st);
}

}  // namespace daeti
