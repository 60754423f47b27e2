// Step A, Mitchell-Schaeffer, all precisions.
#include "reaction_impl.cuh"

namespace daeti {

#define DAETI_MS_LAUNCH(R, K)                                                                                  \
    template <>                                                                                                \
    void launch_ms<R, K>(const DevState& s, const ModelArgs& m, double dt, StepRef step, bool lists, int par,  \
                         int src, bool fused, const DiffOp& op, const ReactTuning& tune, cudaStream_t st) {    \
        const ReactArgs<R> a = react_args<R, K>(s, m, dt, step, lists, par, src, fused, tune);                \
        const int block = react_block(tune);                                                                   \
        const int grid = (int)((s.n + block - 1) / block);                                                     \
        if (grid == 0) return;                                                                                 \
        launch_react_dims<R, M_MS, K, 1>(a, s, op, fused, grid, block, tune, st);                                       \
    }

DAETI_MS_LAUNCH(float, true)
DAETI_MS_LAUNCH(float, false)
DAETI_MS_LAUNCH(double, false)

void launch_reaction(const DevState& s, const ModelArgs& m, double dt, StepRef step, bool lists, int par, int src,
                     bool fused, const DiffOp& op, const ReactTuning& tune, cudaStream_t st) {
    if (m.model == M_MS) {
        if (s.prec == P_F64) launch_ms<double, false>(s, m, dt, step, lists, par, src, fused, op, tune, st);
        else if (s.kahan) launch_ms<float, true>(s, m, dt, step, lists, par, src, fused, op, tune, st);
        else launch_ms<float, false>(s, m, dt, step, lists, par, src, fused, op, tune, st);
    } else {
        if (s.prec == P_F64) launch_tp06<double, false>(s, m, dt, step, lists, par, src, fused, op, tune, st);
        else if (s.kahan) launch_tp06<float, true>(s, m, dt, step, lists, par, src, fused, op, tune, st);
        else launch_tp06<float, false>(s, m, dt, step, lists, par, src, fused, op, tune, st);
    }
}

}  // namespace daeti
