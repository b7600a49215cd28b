// One explicit instance of the nonlinear (iterated linearisation) solver; the
// build compiles this file once per model and precision.
#include "solve_impl.cuh"
namespace mapk {
#if INST_CT
template const Ops* coord_turn_ops<INST_S>();
#else
template const Ops* cubic_ops<INST_N, INST_M, INST_S>();
#endif
}  // namespace mapk
