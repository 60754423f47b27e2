// Step A, ten Tusscher-Panfilov 2006, double state.
#include "reaction_impl.cuh"

namespace daeti {

template <>
void launch_tp06<double, false>(const DevState& s, const ModelArgs& m, double dt, StepRef step, bool lists, int par,
                          int src, bool fused, const DiffOp& op, const ReactTuning& tune, cudaStream_t st) {
    const ReactArgs<double> a = react_args<double, false>(s, m, dt, step, lists, par, src, fused, tune);
    const int block = react_block(tune);
    const int grid = (int)((s.n + block - 1) / block);
    if (grid == 0) return;
    launch_react_dims<double, M_TP06, false, 1>(a, s, op, fused, grid, block, tune, st);
}

}  // namespace daeti
